// OHM occupancy-map oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, sequential CPU implementation of the ray-integration path of
// "OHM: GPU Based Occupancy Map Generation" (arxiv 2206.06079).  Only the test
// suite, the smoke check and the CPU-baseline leg of the benchmark may load it.
// It shares no code, header or constant with the CUDA library: it has its own
// parameter struct, its own quantiser, its own line walk and its own storage.
//
// What it computes, and where each step comes from:
//   * Map storage: space is cut into regions of 32^3 voxels kept in an ordered
//     map keyed by region coordinates (Sec. III-A, "Memory Layout"; 3.2 m
//     regions at 0.1 m voxels, Sec. III-B).
//   * Quantisation: world points become fixed-point coordinates with F
//     fractional bits per voxel, q = rint((x - origin) * 2^F / voxel_size),
//     evaluated in IEEE double without contraction.  Rays longer than the
//     maximum range are truncated to that range and become miss-only (Sec. IV-A
//     truncates rays at 20 m; reading: a truncated ray carries no sample).
//   * Line walk: the 3D voxel traversal of Amanatides & Woo cited in Sec. III-B.
//     Each iteration steps exactly one axis: the one whose next voxel boundary
//     is reached first along the ray.  Ties (paper silent) step z before y
//     before x.  Times are compared exactly as integer cross products.
//   * Occupancy: log-odds additive update l <- l + delta (Eq. 2, 3) with the
//     clamp of Sec. II-B, applied one observation at a time.  Within one
//     integrate call all misses are applied first and all samples second (the
//     two-phase order of Sec. III-C).  An unknown voxel starts at l = 0.
//   * Hit / miss counts H_i, M_i per voxel (Sec. II-D, NDT-TM permeability).
//   * NDT-OM: per-voxel count, sum and outer-product sum of the sample positions
//     (Sec. II-D, III-C), from which mean and covariance are the sample
//     statistics of the points that fell in the voxel.
//   * Decay rate (Sec. II-E): per voxel the summed distance sum_j d_i(j) that
//     the rays travel through it, the denominator of lambda_i = H_i / sum d_i;
//     with the counts layer H_i is the numerator.  A ray from a to b with
//     length L (after truncation) is parametrised by t in [0, 1]; it enters a
//     voxel at the crossing time of the boundary it last stepped (t = dist /
//     |delta| of that axis, Amanatides & Woo's tMax) and leaves at the next
//     crossing, or at t = 1 in the voxel of b; d = (t_out - t_in) L.
//     Reading (the paper gives no precision): distances are integers in units
//     of 2^-20 m.  L = rint(|b - a| * voxel_size / 2^F * 2^20) in double; a
//     crossing's t is floor(2^32 dist / |delta|) / 2^32 and its position along
//     the ray P(t) = rint(t L); d = P(t_out) - P(t_in).  P is monotone, so
//     no d is negative, the d of one ray add up to exactly L, and the sums
//     do not depend on the order of the rays.
//   * Voxel mean (Sec. III-C): per voxel a sample count n and the mean sample
//     position inside the voxel, 10 bits per axis packed in 32 bits (the
//     paper's footnote).  A sample's position is quantised down to 1/1024 of
//     the voxel.  Reading (the paper updates the mean per sample by CAS, whose
//     rounding depends on thread order): per call, with c samples of summed
//     positions S in the voxel, m <- round-half-up((m n + S) / (n + c)),
//     n <- n + c (saturating at 2^32 - 1), the running mean taken one call at
//     a time like the TSDF average below.
//   * TSDF: projective signed distance s = d - (c - o).u along the ray,
//     truncated to [-tau, tau], for the voxels the walk visits between ranges
//     max(0, d - tau) and d + tau; per call the voxel keeps the running
//     weighted average D <- (W D + sum s) / (W + count) (Sec. II-F; the paper
//     gives no formula, this is the Curless-Levoy average it cites).
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -fPIC -shared (oracle/build.py).

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kRegionDim = 32;                       // voxels per region edge
constexpr int kRegionVoxels = kRegionDim * kRegionDim * kRegionDim;

constexpr int kLayerOccupancy = 1;
constexpr int kLayerNdt = 2;
constexpr int kLayerTsdf = 4;
constexpr int kLayerCounts = 8;
constexpr int kLayerDecay = 16;
constexpr int kLayerMean = 32;

constexpr double kPathUnitsPerMetre = 1048576.0;  // 2^20

constexpr uint8_t kFlagNoReturn = 1;

}  // namespace

extern "C" {

// Parameters of an oracle map.  All lengths are metres.
struct OracleParams {
  double voxel_size;     // voxel edge length
  double map_origin[3];  // world position of voxel (0,0,0)'s lower corner
  int32_t frac_bits;     // F: fixed-point fraction bits per voxel
  int32_t layers;        // bit mask of kLayer*
  float hit;             // log-odds increment for a sample (Eq. 3)
  float miss;            // log-odds increment for a pass-through (Eq. 3)
  float l_min;           // lower clamp (Sec. II-B)
  float l_max;           // upper clamp (Sec. II-B)
  float ndt_clear_below; // NDT samples are cleared when a miss takes l below this (Sec. II-D)
  double max_range;      // truncation length (Sec. IV-A)
  double min_range;      // TSDF: samples at or below this range are ignored
  double tsdf_trunc;     // TSDF truncation distance tau
  double tsdf_wmax;      // TSDF weight cap
};

}  // extern "C"

namespace {

// floor(a / b) for b > 0, written out so negative numerators round down.
int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b) != 0 && (a < 0)) q -= 1;
  return q;
}

struct Voxel {
  int64_t v[3];
};

struct RegionKey {
  int64_t r[3];
  bool operator<(const RegionKey& o) const {
    return std::tie(r[0], r[1], r[2]) < std::tie(o.r[0], o.r[1], o.r[2]);
  }
};

struct Region {
  std::vector<float> occupancy;     // log-odds, NaN = unknown
  std::vector<uint32_t> hits;       // H_i
  std::vector<uint32_t> misses;     // M_i
  std::vector<__int128> ndt;        // 10 per voxel: n, Sx, Sy, Sz, Sxx, Sxy, Sxz, Syy, Syz, Szz
  std::vector<double> tsdf_d;       // running signed distance
  std::vector<double> tsdf_w;       // running weight
  std::vector<uint64_t> path;       // decay rate: sum_j d_i(j) in 2^-20 m
  std::vector<uint32_t> mean_n;     // voxel mean: sample count
  std::vector<uint32_t> mean_m;     // voxel mean: 3 per voxel, position in 1/1024 voxel
};

struct Map {
  OracleParams p;
  double scale;  // 2^F / voxel_size
  int64_t unit;  // 2^F
  std::map<RegionKey, Region> regions;
};

RegionKey region_of(const Voxel& v) {
  RegionKey k;
  for (int a = 0; a < 3; ++a) k.r[a] = floor_div(v.v[a], kRegionDim);
  return k;
}

// Linear index of a voxel inside its region: x fastest, then y, then z.
int local_index(const Voxel& v) {
  int l[3];
  for (int a = 0; a < 3; ++a) l[a] = (int)(v.v[a] - floor_div(v.v[a], kRegionDim) * kRegionDim);
  return l[0] + kRegionDim * (l[1] + kRegionDim * l[2]);
}

Region& region_for(Map& m, const Voxel& v) {
  RegionKey k = region_of(v);
  auto it = m.regions.find(k);
  if (it != m.regions.end()) return it->second;
  Region r;
  const int L = m.p.layers;
  if (L & kLayerOccupancy) r.occupancy.assign(kRegionVoxels, std::nanf(""));
  if (L & kLayerCounts) {
    r.hits.assign(kRegionVoxels, 0u);
    r.misses.assign(kRegionVoxels, 0u);
  }
  if (L & kLayerTsdf) {
    r.tsdf_d.assign(kRegionVoxels, 0.0);
    r.tsdf_w.assign(kRegionVoxels, 0.0);
  }
  if (L & kLayerDecay) r.path.assign(kRegionVoxels, 0ull);
  if (L & kLayerMean) {
    r.mean_n.assign(kRegionVoxels, 0u);
    r.mean_m.assign((size_t)kRegionVoxels * 3, 0u);
  }
  return m.regions.emplace(k, std::move(r)).first->second;
}

// Fixed-point coordinate of one axis: rint((x - origin) * 2^F / voxel_size) in
// double precision, one rounding per operation.
int64_t quantise_axis(float x, double origin, double scale) {
  double d = (double)x - origin;
  double s = d * scale;
  return (int64_t)std::llrint(s);
}

Voxel voxel_of(const int64_t q[3], int64_t unit) {
  Voxel v;
  for (int a = 0; a < 3; ++a) v.v[a] = floor_div(q[a], unit);
  return v;
}

// Amanatides & Woo voxel walk from fixed-point point a to fixed-point point b.
// Returns every voxel visited, first the voxel of a and last the voxel of b.
// At each iteration, among the axes that still have boundaries to cross before
// reaching b's voxel, the axis whose next boundary lies at the smallest ray
// parameter t steps.  For axis k the next boundary is dist[k] fixed-point units
// away along that axis and the ray advances |delta_k| units per unit t, so
// t_k = dist[k] / |delta_k|; t_j < t_k is decided exactly by
// dist[j] * |delta_k| < dist[k] * |delta_j|.  Equal t: z, then y, then x.
std::vector<Voxel> walk(const int64_t a[3], const int64_t b[3], int64_t unit) {
  Voxel v = voxel_of(a, unit);
  const Voxel end = voxel_of(b, unit);
  int64_t remaining[3], step[3], adelta[3], dist[3];
  for (int k = 0; k < 3; ++k) {
    int64_t delta = b[k] - a[k];
    adelta[k] = delta < 0 ? -delta : delta;
    step[k] = delta < 0 ? -1 : 1;
    remaining[k] = end.v[k] - v.v[k];
    if (remaining[k] < 0) remaining[k] = -remaining[k];
    // Distance from a to the first boundary crossed along axis k.  Moving up,
    // that is the upper face of the voxel; moving down, the lower face (a point
    // lying exactly on the lower face leaves the voxel immediately, at t = 0).
    if (step[k] > 0)
      dist[k] = (v.v[k] + 1) * unit - a[k];
    else
      dist[k] = a[k] - v.v[k] * unit;
  }
  std::vector<Voxel> out;
  out.push_back(v);
  while (remaining[0] + remaining[1] + remaining[2] > 0) {
    int best = -1;
    for (int k = 2; k >= 0; --k) {  // z first so that ties keep the higher axis
      if (remaining[k] == 0) continue;
      if (best < 0) {
        best = k;
        continue;
      }
      __int128 tk = (__int128)dist[k] * adelta[best];
      __int128 tb = (__int128)dist[best] * adelta[k];
      if (tk < tb) best = k;
    }
    v.v[best] += step[best];
    dist[best] += unit;
    remaining[best] -= 1;
    out.push_back(v);
  }
  return out;
}

// One voxel of a walk with the ray parameters at which the ray enters and
// leaves it (Sec. II-E needs the distance travelled inside each voxel), as
// fractions of 2^32: t = 2^32 means the end point b.
struct TimedVoxel {
  Voxel v;
  uint64_t t_in, t_out;
};

// The same walk as walk(), also reporting each voxel's entry and exit times.
// The crossing of axis k happens at t = dist[k] / |delta_k|, kept as
// floor(2^32 dist[k] / |delta_k|).
std::vector<TimedVoxel> walk_timed(const int64_t a[3], const int64_t b[3], int64_t unit) {
  Voxel v = voxel_of(a, unit);
  const Voxel end = voxel_of(b, unit);
  int64_t remaining[3], step[3], adelta[3], dist[3];
  for (int k = 0; k < 3; ++k) {
    int64_t delta = b[k] - a[k];
    adelta[k] = delta < 0 ? -delta : delta;
    step[k] = delta < 0 ? -1 : 1;
    remaining[k] = end.v[k] - v.v[k];
    if (remaining[k] < 0) remaining[k] = -remaining[k];
    if (step[k] > 0)
      dist[k] = (v.v[k] + 1) * unit - a[k];
    else
      dist[k] = a[k] - v.v[k] * unit;
  }
  std::vector<TimedVoxel> out;
  uint64_t t = 0;
  while (remaining[0] + remaining[1] + remaining[2] > 0) {
    int best = -1;
    for (int k = 2; k >= 0; --k) {
      if (remaining[k] == 0) continue;
      if (best < 0) {
        best = k;
        continue;
      }
      __int128 tk = (__int128)dist[k] * adelta[best];
      __int128 tb = (__int128)dist[best] * adelta[k];
      if (tk < tb) best = k;
    }
    const uint64_t t_cross = (uint64_t)(((__int128)dist[best] << 32) / adelta[best]);
    out.push_back(TimedVoxel{v, t, t_cross});
    t = t_cross;
    v.v[best] += step[best];
    dist[best] += unit;
    remaining[best] -= 1;
  }
  out.push_back(TimedVoxel{v, t, (uint64_t)1 << 32});
  return out;
}

struct PreparedRay {
  int64_t qo[3];
  int64_t qe[3];
  bool has_sample;  // the endpoint is a return (a sample) inside the maximum range
  double length;    // |qe - qo| in fixed-point units, before truncation
};

// Quantise one ray and truncate it to the maximum range (Sec. IV-A).
// Returns false for a ray that is skipped: a non-finite coordinate, or a point
// outside the addressable extent (|voxel index| < 2^24 per axis after
// truncation; before it, |fixed-point value| < 2^52 so rounding is exact).
bool prepare_ray(const Map& m, const float* o, const float* e, uint8_t flag, PreparedRay* r) {
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(o[a]) || !std::isfinite(e[a])) return false;
  const double fp_limit = std::ldexp(1.0, 52);
  for (int a = 0; a < 3; ++a) {
    double so = ((double)o[a] - m.p.map_origin[a]) * m.scale;
    double se = ((double)e[a] - m.p.map_origin[a]) * m.scale;
    if (!(std::fabs(so) < fp_limit) || !(std::fabs(se) < fp_limit)) return false;
    r->qo[a] = quantise_axis(o[a], m.p.map_origin[a], m.scale);
    r->qe[a] = quantise_axis(e[a], m.p.map_origin[a], m.scale);
  }
  r->has_sample = (flag & kFlagNoReturn) == 0;
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = (double)(r->qe[a] - r->qo[a]);
  double len2 = d[0] * d[0];
  len2 = len2 + d[1] * d[1];
  len2 = len2 + d[2] * d[2];
  double len = std::sqrt(len2);
  r->length = len;
  double rmax = m.p.max_range * m.scale;
  if (len > rmax) {
    double ratio = rmax / len;
    for (int a = 0; a < 3; ++a) r->qe[a] = r->qo[a] + (int64_t)std::llrint(d[a] * ratio);
    r->has_sample = false;
  }
  const int64_t vlimit = (int64_t)1 << 24;
  for (int a = 0; a < 3; ++a) {
    int64_t vo = floor_div(r->qo[a], m.unit), ve = floor_div(r->qe[a], m.unit);
    if (vo <= -vlimit || vo >= vlimit || ve <= -vlimit || ve >= vlimit) return false;
  }
  return true;
}

void apply_miss(Map& m, const Voxel& v) {
  Region& r = region_for(m, v);
  int i = local_index(v);
  if (m.p.layers & kLayerOccupancy) {
    float l = r.occupancy[i];
    float l0 = std::isnan(l) ? 0.0f : l;
    float u = l0 + m.p.miss;
    float ln = std::fmin(std::fmax(u, m.p.l_min), m.p.l_max);
    r.occupancy[i] = ln;
    // Sample clearing (Sec. II-D): falling below the threshold (from at or
    // above it, or from unknown) drops the voxel's NDT samples.
    const bool was_above = std::isnan(l) || !(l < m.p.ndt_clear_below);
    if (was_above && ln < m.p.ndt_clear_below && !r.ndt.empty())
      for (int k = 0; k < 10; ++k) r.ndt[(size_t)i * 10 + k] = 0;
  }
  if (m.p.layers & kLayerCounts) r.misses[i] += 1u;
}

// Length of the walk from qo to qe in 2^-20 m (the L of Sec. II-E).
uint64_t walk_length(const Map& m, const int64_t qo[3], const int64_t qe[3]) {
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = (double)(qe[a] - qo[a]);
  double len2 = d[0] * d[0];
  len2 = len2 + d[1] * d[1];
  len2 = len2 + d[2] * d[2];
  const double metres = std::sqrt(len2) * (m.p.voxel_size / (double)m.unit);
  return (uint64_t)std::llrint(metres * kPathUnitsPerMetre);
}

// Position along the ray, in 2^-20 m, at parameter t (a fraction of 2^32).
uint64_t ray_position(uint64_t t, uint64_t length) {
  return (uint64_t)(((unsigned __int128)t * length + ((unsigned __int128)1 << 31)) >> 32);
}

// Decay rate (Sec. II-E): add the distance a ray travels inside the voxel.
void apply_path(Map& m, const TimedVoxel& tv, uint64_t length) {
  Region& r = region_for(m, tv.v);
  r.path[local_index(tv.v)] += ray_position(tv.t_out, length) - ray_position(tv.t_in, length);
}

void apply_hit(Map& m, const Voxel& v, const int64_t qe[3]) {
  Region& r = region_for(m, v);
  int i = local_index(v);
  if (m.p.layers & kLayerOccupancy) {
    float l = r.occupancy[i];
    float l0 = std::isnan(l) ? 0.0f : l;
    float u = l0 + m.p.hit;
    r.occupancy[i] = std::fmin(std::fmax(u, m.p.l_min), m.p.l_max);
  }
  if (m.p.layers & kLayerCounts) r.hits[i] += 1u;
  if (m.p.layers & kLayerNdt) {
    if (r.ndt.empty()) r.ndt.assign((size_t)kRegionVoxels * 10, (__int128)0);  // first sample in this region
    // Sample position relative to the voxel's lower corner, in fixed-point units.
    __int128 p[3];
    for (int a = 0; a < 3; ++a) p[a] = (__int128)(qe[a] - v.v[a] * m.unit);
    __int128* s = &r.ndt[(size_t)i * 10];
    s[0] += 1;
    s[1] += p[0];
    s[2] += p[1];
    s[3] += p[2];
    s[4] += p[0] * p[0];
    s[5] += p[0] * p[1];
    s[6] += p[0] * p[2];
    s[7] += p[1] * p[1];
    s[8] += p[1] * p[2];
    s[9] += p[2] * p[2];
  }
}

struct VoxelHash {
  size_t operator()(const std::tuple<int64_t, int64_t, int64_t>& t) const {
    uint64_t h = (uint64_t)std::get<0>(t) * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)std::get<1>(t) * 0xC2B2AE3D27D4EB4Full + (h << 6) + (h >> 2);
    h ^= (uint64_t)std::get<2>(t) * 0x165667B19E3779F9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

// TSDF contribution of one ray (Sec. II-F).  All geometry in metres, double.
int64_t tsdf_ray(Map& m, const PreparedRay& r,
                 std::unordered_map<std::tuple<int64_t, int64_t, int64_t>, std::pair<double, int64_t>, VoxelHash>& acc) {
  const double tau_q = m.p.tsdf_trunc * m.scale;
  const double len = r.length;
  double d[3];
  for (int a = 0; a < 3; ++a) d[a] = (double)(r.qe[a] - r.qo[a]);
  // Band end points along the ray at ranges max(0, len - tau) and len + tau,
  // quantised with the same rule as a truncated endpoint.
  double t0 = len - tau_q;
  if (t0 < 0.0) t0 = 0.0;
  double t1 = len + tau_q;
  double f0 = t0 / len, f1 = t1 / len;
  int64_t a0[3], a1[3];
  for (int a = 0; a < 3; ++a) {
    a0[a] = r.qo[a] + (int64_t)std::llrint(d[a] * f0);
    a1[a] = r.qo[a] + (int64_t)std::llrint(d[a] * f1);
  }
  // Range d and direction u in metres from the quantised sensor origin.
  const double inv_scale = m.p.voxel_size / (double)m.unit;
  const double dist_m = len * inv_scale;
  double u[3];
  for (int a = 0; a < 3; ++a) u[a] = d[a] / len;
  std::vector<Voxel> vox = walk(a0, a1, m.unit);
  for (const Voxel& v : vox) {
    double proj = 0.0;
    for (int a = 0; a < 3; ++a) {
      double centre = ((double)v.v[a] + 0.5) * m.p.voxel_size;  // relative to the map origin
      double origin = (double)r.qo[a] * inv_scale;
      proj += (centre - origin) * u[a];
    }
    double s = dist_m - proj;
    if (s > m.p.tsdf_trunc) s = m.p.tsdf_trunc;
    if (s < -m.p.tsdf_trunc) s = -m.p.tsdf_trunc;
    auto& e = acc[std::make_tuple(v.v[0], v.v[1], v.v[2])];
    e.first += s;
    e.second += 1;
  }
  return (int64_t)vox.size();
}

}  // namespace

extern "C" {

void* oracle_create(const OracleParams* p) {
  Map* m = new Map();
  m->p = *p;
  m->unit = (int64_t)1 << p->frac_bits;
  m->scale = std::ldexp(1.0, p->frac_bits) / p->voxel_size;
  return m;
}

void oracle_destroy(void* h) { delete static_cast<Map*>(h); }

// Integrate one ray set (one scan).  origins holds n_origins points (1 = a
// shared sensor origin, else one per ray); endpoints holds n points; flags may
// be null.  Returns the number of voxel visits made by the occupancy walk plus
// the TSDF band walks, or -1 on bad arguments.
int64_t oracle_integrate(void* h, const float* origins, int64_t n_origins, const float* endpoints,
                         const uint8_t* flags, int64_t n) {
  Map& m = *static_cast<Map*>(h);
  if (n < 0 || (n > 0 && (!origins || !endpoints)) || (n_origins != 1 && n_origins != n)) return -1;
  std::vector<PreparedRay> rays;
  rays.reserve((size_t)n);
  for (int64_t i = 0; i < n; ++i) {
    const float* o = origins + 3 * (n_origins == 1 ? 0 : i);
    PreparedRay r;
    if (prepare_ray(m, o, endpoints + 3 * i, flags ? flags[i] : 0, &r)) rays.push_back(r);
  }
  int64_t visits = 0;
  const int occ_like = kLayerOccupancy | kLayerCounts | kLayerNdt | kLayerDecay | kLayerMean;
  if (m.p.layers & occ_like) {
    // Phase 1: every pass-through (miss) of every ray.
    for (const PreparedRay& r : rays) {
      std::vector<Voxel> vox = walk(r.qo, r.qe, m.unit);
      visits += (int64_t)vox.size();
      size_t count = vox.size();
      if (r.has_sample) count -= 1;  // the sample voxel gets the hit instead
      for (size_t j = 0; j < count; ++j) apply_miss(m, vox[j]);
      if (m.p.layers & kLayerDecay) {
        const uint64_t length = walk_length(m, r.qo, r.qe);
        for (const TimedVoxel& tv : walk_timed(r.qo, r.qe, m.unit)) apply_path(m, tv, length);
      }
    }
    // Phase 2: every sample (hit).
    std::map<std::tuple<int64_t, int64_t, int64_t>, std::array<uint64_t, 4>> mean_acc;  // c, Sx, Sy, Sz
    for (const PreparedRay& r : rays) {
      if (!r.has_sample) continue;
      const Voxel v = voxel_of(r.qe, m.unit);
      apply_hit(m, v, r.qe);
      if (m.p.layers & kLayerMean) {
        auto& acc = mean_acc[std::make_tuple(v.v[0], v.v[1], v.v[2])];
        acc[0] += 1;
        for (int a = 0; a < 3; ++a) acc[1 + a] += (uint64_t)(((r.qe[a] - v.v[a] * m.unit) * 1024) / m.unit);
      }
    }
    for (const auto& kv : mean_acc) {
      Voxel v;
      v.v[0] = std::get<0>(kv.first);
      v.v[1] = std::get<1>(kv.first);
      v.v[2] = std::get<2>(kv.first);
      Region& reg = region_for(m, v);
      const int i = local_index(v);
      const uint64_t n = reg.mean_n[i], c = kv.second[0], total = n + c;
      for (int a = 0; a < 3; ++a) {
        const uint64_t num = (uint64_t)reg.mean_m[(size_t)i * 3 + a] * n + kv.second[1 + a];
        reg.mean_m[(size_t)i * 3 + a] = (uint32_t)((2 * num + total) / (2 * total));  // round half up
      }
      reg.mean_n[i] = (uint32_t)(total < 0xffffffffull ? total : 0xffffffffull);
    }
  }
  if (m.p.layers & kLayerTsdf) {
    std::unordered_map<std::tuple<int64_t, int64_t, int64_t>, std::pair<double, int64_t>, VoxelHash> acc;
    const double rmin = m.p.min_range * m.scale;
    const double rmax = m.p.max_range * m.scale;
    for (const PreparedRay& r : rays) {
      if (!r.has_sample) continue;                          // no surface observed
      if (!(r.length > rmin) || r.length > rmax) continue;  // outside the valid range
      visits += tsdf_ray(m, r, acc);
    }
    for (const auto& kv : acc) {
      Voxel v;
      v.v[0] = std::get<0>(kv.first);
      v.v[1] = std::get<1>(kv.first);
      v.v[2] = std::get<2>(kv.first);
      Region& reg = region_for(m, v);
      int i = local_index(v);
      double W = reg.tsdf_w[i], D = reg.tsdf_d[i];
      double c = (double)kv.second.second;
      reg.tsdf_d[i] = (W * D + kv.second.first) / (W + c);
      double w2 = W + c;
      reg.tsdf_w[i] = w2 < m.p.tsdf_wmax ? w2 : m.p.tsdf_wmax;
    }
  }
  return visits;
}

int64_t oracle_region_count(void* h) { return (int64_t)static_cast<Map*>(h)->regions.size(); }

// Dump regions [first, first + count) of the (rx, ry, rz) lexicographic order.
// Any output pointer may be null.  Per region: keys 3 x int64; occupancy 32768
// float; hits, misses 32768 uint32; ndt 32768 x 10 int64 (n, Sx, Sy, Sz, Sxx,
// Sxy, Sxz, Syy, Syz, Szz; zeros for a region without samples); tsdf 32768 x 2
// double (D, W); path 32768 uint64 (decay rate: summed distance, 2^-20 m);
// mean 32768 x 4 uint32 (voxel mean: count, mx, my, mz in 1/1024 voxel).
// Voxel order inside a region: x fastest.  Returns 0, or 1 if an NDT sum does
// not fit in int64.
int oracle_export(void* h, int64_t first, int64_t count, int64_t* keys, float* occupancy, uint32_t* hits,
                  uint32_t* misses, int64_t* ndt, double* tsdf, uint64_t* path, uint32_t* mean) {
  Map& m = *static_cast<Map*>(h);
  int rc = 0;
  int64_t pos = 0;
  size_t idx = 0;
  for (const auto& kv : m.regions) {
    if (pos++ < first) continue;
    if ((int64_t)idx >= count) break;
    const Region& r = kv.second;
    if (keys)
      for (int a = 0; a < 3; ++a) keys[idx * 3 + a] = kv.first.r[a];
    if (occupancy && !r.occupancy.empty())
      std::memcpy(occupancy + idx * kRegionVoxels, r.occupancy.data(), sizeof(float) * kRegionVoxels);
    if (hits && !r.hits.empty()) std::memcpy(hits + idx * kRegionVoxels, r.hits.data(), sizeof(uint32_t) * kRegionVoxels);
    if (misses && !r.misses.empty())
      std::memcpy(misses + idx * kRegionVoxels, r.misses.data(), sizeof(uint32_t) * kRegionVoxels);
    if (ndt) {
      int64_t* dst = ndt + idx * (size_t)kRegionVoxels * 10;
      if (r.ndt.empty()) {
        std::memset(dst, 0, sizeof(int64_t) * (size_t)kRegionVoxels * 10);
      } else {
        for (size_t j = 0; j < (size_t)kRegionVoxels * 10; ++j) {
          __int128 s = r.ndt[j];
          if (s > (__int128)INT64_MAX || s < (__int128)INT64_MIN) rc = 1;
          dst[j] = (int64_t)s;
        }
      }
    }
    if (tsdf && !r.tsdf_d.empty()) {
      for (int j = 0; j < kRegionVoxels; ++j) {
        tsdf[(idx * kRegionVoxels + j) * 2 + 0] = r.tsdf_d[j];
        tsdf[(idx * kRegionVoxels + j) * 2 + 1] = r.tsdf_w[j];
      }
    }
    if (path && !r.path.empty()) std::memcpy(path + idx * kRegionVoxels, r.path.data(), sizeof(uint64_t) * kRegionVoxels);
    if (mean && !r.mean_n.empty()) {
      for (int j = 0; j < kRegionVoxels; ++j) {
        uint32_t* o = mean + (idx * kRegionVoxels + j) * 4;
        o[0] = r.mean_n[j];
        for (int a = 0; a < 3; ++a) o[1 + a] = r.mean_m[(size_t)j * 3 + a];
      }
    }
    ++idx;
  }
  return rc;
}

// Every voxel holding at least one sample, in (region order, x-fastest voxel
// order): voxel coordinates (cap x 3 int64) and its 10 moments (cap x 10
// int64).  Writes at most cap entries; returns how many exist.
int64_t oracle_ndt_sparse(void* h, int64_t cap, int64_t* voxels, int64_t* moments) {
  Map& m = *static_cast<Map*>(h);
  int64_t c = 0;
  for (const auto& kv : m.regions) {
    const Region& r = kv.second;
    if (r.ndt.empty()) continue;
    for (int li = 0; li < kRegionVoxels; ++li) {
      const __int128* s = &r.ndt[(size_t)li * 10];
      if (s[0] == 0) continue;
      if (c < cap) {
        const int l[3] = {li % kRegionDim, (li / kRegionDim) % kRegionDim, li / (kRegionDim * kRegionDim)};
        for (int a = 0; a < 3; ++a) voxels[3 * c + a] = kv.first.r[a] * kRegionDim + l[a];
        for (int k = 0; k < 10; ++k) moments[10 * c + k] = (int64_t)s[k];
      }
      ++c;
    }
  }
  return c;
}

// Number of regions holding NDT samples.
int64_t oracle_ndt_region_count(void* h) {
  int64_t c = 0;
  for (const auto& kv : static_cast<Map*>(h)->regions) c += kv.second.ndt.empty() ? 0 : 1;
  return c;
}

// Look up n world points.  occupancy: log-odds (NaN if unknown); known: 1 if
// the voxel has been observed by the occupancy layer; ndt: n x 10 doubles
// (count, mean xyz in metres, covariance xx xy xz yy yz zz in m^2; zeros if no
// sample); tsdf: n x 2 (D, W).  Any output may be null.
void oracle_query(void* h, const float* pts, int64_t n, float* occupancy, uint8_t* known, double* ndt,
                  double* tsdf, uint64_t* path, double* mean) {
  Map& m = *static_cast<Map*>(h);
  const double cell = m.p.voxel_size / (double)m.unit;  // metres per fixed-point unit
  for (int64_t i = 0; i < n; ++i) {
    int64_t q[3];
    for (int a = 0; a < 3; ++a) q[a] = quantise_axis(pts[3 * i + a], m.p.map_origin[a], m.scale);
    Voxel v = voxel_of(q, m.unit);
    auto it = m.regions.find(region_of(v));
    const Region* r = it == m.regions.end() ? nullptr : &it->second;
    int li = local_index(v);
    if (occupancy) occupancy[i] = (r && !r->occupancy.empty()) ? r->occupancy[li] : std::nanf("");
    if (known) known[i] = (r && !r->occupancy.empty() && !std::isnan(r->occupancy[li])) ? 1 : 0;
    if (ndt) {
      double* o = ndt + 10 * i;
      for (int k = 0; k < 10; ++k) o[k] = 0.0;
      if (r && !r->ndt.empty() && r->ndt[(size_t)li * 10] > 0) {
        const __int128* s = &r->ndt[(size_t)li * 10];
        double cnt = (double)s[0];
        o[0] = cnt;
        for (int a = 0; a < 3; ++a) {
          double corner = (double)(v.v[a] * m.unit);
          o[1 + a] = m.p.map_origin[a] + (corner + (double)s[1 + a] / cnt) * cell;
        }
        // Population covariance: (n * Sab - Sa * Sb) / n^2, numerator exact.
        const int pairs[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
        for (int k = 0; k < 6; ++k) {
          __int128 num = s[0] * s[4 + k] - s[1 + pairs[k][0]] * s[1 + pairs[k][1]];
          o[4 + k] = (double)num / (cnt * cnt) * cell * cell;
        }
      }
    }
    if (tsdf) {
      tsdf[2 * i] = (r && !r->tsdf_d.empty()) ? r->tsdf_d[li] : 0.0;
      tsdf[2 * i + 1] = (r && !r->tsdf_w.empty()) ? r->tsdf_w[li] : 0.0;
    }
    if (path) path[i] = (r && !r->path.empty()) ? r->path[li] : 0ull;
    if (mean) {
      // voxel-mean position: lower corner + (m + 1/2) / 1024 of the voxel; NaN without samples
      const uint32_t cnt = (r && !r->mean_n.empty()) ? r->mean_n[li] : 0u;
      for (int a = 0; a < 3; ++a)
        mean[4 * i + a] = cnt ? m.p.map_origin[a] +
                                    ((double)v.v[a] + ((double)r->mean_m[(size_t)li * 3 + a] + 0.5) / 1024.0) * m.p.voxel_size
                              : std::nan("");
      mean[4 * i + 3] = (double)cnt;
    }
  }
}

// ---------------------------------------------------------------------------
// TSDF adjoint (the voxel sets held fixed).
//
// For one frame of rays with nominal float endpoints (which fix, through the
// same quantised band walk as oracle_integrate, the voxels each ray updates),
// evaluate in double precision at continuous geometry (o_eval, e_eval)
//   L = sum_q g_q D_new(v_q),
//   D_new(v) = (W D + sum_{j: v in band_j} s_j(v)) / (W + c(v))   (c(v) > 0)
//            = D                                                  (c(v) = 0)
//   s_j(v) = clamp(d_j - (centre(v) - o).u_j, -tau, tau),  d_j = |e_j - o|,
// with W, D the map's current state (the state before this frame; the map is
// not modified).  Also the analytic gradient: for an unclamped s,
//   ds/de = u + r_perp / d,  ds/do = -r_perp / d,  r = e - centre,
//   r_perp = r - (r.u) u,  dD_new/ds = 1 / (W + c).
// qvox: m voxel indices (x, y, z) with weights g.  grad_e: n x 3, grad_o: 3
// (either may be null).  Returns 0, or -1 on bad arguments.
}  // extern "C"

namespace {

// The voxels each ray of a frame updates (the quantised band walk of
// oracle_integrate), from the nominal float rays.
std::vector<std::vector<Voxel>> frozen_bands(Map& m, const float* o_nom, const float* e_nom, const uint8_t* flags,
                                             int64_t n) {
  std::vector<std::vector<Voxel>> bands((size_t)n);
  const double rmin = m.p.min_range * m.scale, rmax = m.p.max_range * m.scale;
  for (int64_t j = 0; j < n; ++j) {
    PreparedRay r;
    if (!prepare_ray(m, o_nom, e_nom + 3 * j, flags ? flags[j] : 0, &r)) continue;
    if (!r.has_sample || !(r.length > rmin) || r.length > rmax) continue;
    const double tau_q = m.p.tsdf_trunc * m.scale;
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = (double)(r.qe[a] - r.qo[a]);
    double t0 = r.length - tau_q;
    if (t0 < 0.0) t0 = 0.0;
    const double f0 = t0 / r.length, f1 = (r.length + tau_q) / r.length;
    int64_t a0[3], a1[3];
    for (int a = 0; a < 3; ++a) {
      a0[a] = r.qo[a] + (int64_t)std::llrint(d[a] * f0);
      a1[a] = r.qo[a] + (int64_t)std::llrint(d[a] * f1);
    }
    bands[(size_t)j] = walk(a0, a1, m.unit);
  }
  return bands;
}

}  // namespace

extern "C" {

int oracle_tsdf_frame_eval(void* h, const float* o_nom, const float* e_nom, const uint8_t* flags, int64_t n,
                           const double* o_eval, const double* e_eval, const int64_t* qvox, const double* g,
                           int64_t m_q, double* loss, double* grad_e, double* grad_o) {
  Map& m = *static_cast<Map*>(h);
  if (!(m.p.layers & kLayerTsdf)) return -1;
  typedef std::tuple<int64_t, int64_t, int64_t> Key;
  // gradient weight per voxel
  std::map<Key, double> G;
  for (int64_t q = 0; q < m_q; ++q) G[std::make_tuple(qvox[3 * q], qvox[3 * q + 1], qvox[3 * q + 2])] += g[q];
  // frozen band voxel lists from the nominal rays, and counts c(v)
  const std::vector<std::vector<Voxel>> bands = frozen_bands(m, o_nom, e_nom, flags, n);
  std::map<Key, int64_t> count;
  for (int64_t j = 0; j < n; ++j)
    for (const Voxel& v : bands[(size_t)j]) count[std::make_tuple(v.v[0], v.v[1], v.v[2])] += 1;
  // loss: unchanged voxels contribute g D, changed ones g D_new
  double L = 0.0;
  std::map<Key, double> sum_s;
  const double tau = m.p.tsdf_trunc;
  if (grad_o)
    for (int a = 0; a < 3; ++a) grad_o[a] = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    double ge[3] = {0.0, 0.0, 0.0};
    if (!bands[(size_t)j].empty()) {
      const double* e = e_eval + 3 * j;
      double u[3], dist = 0.0;
      for (int a = 0; a < 3; ++a) {
        u[a] = e[a] - o_eval[a];
        dist += u[a] * u[a];
      }
      dist = std::sqrt(dist);
      for (int a = 0; a < 3; ++a) u[a] /= dist;
      for (const Voxel& v : bands[(size_t)j]) {
        double r[3], ru = 0.0;
        for (int a = 0; a < 3; ++a) {
          const double centre = m.p.map_origin[a] + ((double)v.v[a] + 0.5) * m.p.voxel_size;
          r[a] = e[a] - centre;
          ru += r[a] * u[a];
        }
        // s = d - (centre - o).u = (e - centre).u
        double s = ru;
        const bool clamped = s >= tau || s <= -tau;
        if (s > tau) s = tau;
        if (s < -tau) s = -tau;
        const Key k = std::make_tuple(v.v[0], v.v[1], v.v[2]);
        sum_s[k] += s;
        auto gi = G.find(k);
        if (gi == G.end() || clamped) continue;
        auto rit = m.regions.find(region_of(v));  // lookup only: the map is not modified
        const double W = (rit != m.regions.end() && !rit->second.tsdf_w.empty()) ? rit->second.tsdf_w[local_index(v)] : 0.0;
        const double w = gi->second / (W + (double)count[k]);
        for (int a = 0; a < 3; ++a) {
          const double rp = r[a] - ru * u[a];
          ge[a] += w * (u[a] + rp / dist);
          if (grad_o) grad_o[a] += -w * rp / dist;
        }
      }
    }
    if (grad_e)
      for (int a = 0; a < 3; ++a) grad_e[3 * j + a] = ge[a];
  }
  for (const auto& kv : G) {
    Voxel v;
    v.v[0] = std::get<0>(kv.first);
    v.v[1] = std::get<1>(kv.first);
    v.v[2] = std::get<2>(kv.first);
    auto it = m.regions.find(region_of(v));
    double W = 0.0, D = 0.0;
    if (it != m.regions.end() && !it->second.tsdf_w.empty()) {
      W = it->second.tsdf_w[local_index(v)];
      D = it->second.tsdf_d[local_index(v)];
    }
    auto c = count.find(kv.first);
    if (c == count.end())
      L += kv.second * D;
    else
      L += kv.second * (W * D + sum_s[kv.first]) / (W + (double)c->second);
  }
  *loss = L;
  return 0;
}

// NDT-OM adjoint (Sec. II-D / III-C sample statistics; the voxel assignment
// of every sample held fixed).
//
// The nominal float rays fix, through the quantisation and truncation of
// oracle_integrate, which rays carry a sample and the voxel v_j of each.  At
// continuous sample positions e_eval (world metres, double) the NDT state of
// a voxel v after the frame is, relative to its lower corner c(v),
//   n = n0 + #{j: v_j = v},  S = S0 + sum_j (e_j - c),  Q = Q0 + sum_j (e_j - c)(e_j - c)^T,
//   mean = c + S / n,  C = Q / n - (S / n)(S / n)^T      (population covariance)
// with n0, S0, Q0 the map's moments before the frame (the map's integer sums
// scaled to metres; the map is not modified).  For query voxels v_q with
// weights gm_q (3) and gc_q (6, packed xx xy xz yy yz zz)
//   L = sum_q [ gm_q . mean(v_q) + gc_q . packed C(v_q) ]     (n(v_q) > 0; else 0)
// and, with d_j = e_j - c - S / n and G the upper-triangular matrix of the
// summed gc of v_j's queries,
//   dL/de_j = (1/n) [ gm + (G + G^T) d_j ].
// grad_e: n x 3 (zeros for rays without a sample).  Returns 0, or -1 on bad
// arguments or a map without the NDT layer.
int oracle_ndt_frame_eval(void* h, const float* o_nom, int64_t n_origins, const float* e_nom, const uint8_t* flags,
                          int64_t n, const double* e_eval, const int64_t* qvox, const double* gm, const double* gc,
                          int64_t m_q, double* loss, double* grad_e) {
  Map& m = *static_cast<Map*>(h);
  if (!(m.p.layers & kLayerNdt) || (n_origins != 1 && n_origins != n)) return -1;
  typedef std::tuple<int64_t, int64_t, int64_t> Key;
  const double cell = m.p.voxel_size / (double)m.unit;  // metres per fixed-point unit
  // the frame's samples and their voxels
  std::vector<int> has(n, 0);
  std::vector<Voxel> vox((size_t)n);
  for (int64_t j = 0; j < n; ++j) {
    PreparedRay r;
    const float* o = o_nom + (n_origins == 1 ? 0 : 3 * j);
    if (!prepare_ray(m, o, e_nom + 3 * j, flags ? flags[j] : 0, &r) || !r.has_sample) continue;
    for (int a = 0; a < 3; ++a) vox[(size_t)j].v[a] = floor_div(r.qe[a], m.unit);
    has[(size_t)j] = 1;
  }
  // per voxel: n, S (3), Q (3 x 3) in metres relative to the corner
  struct Stat {
    double n = 0.0, S[3] = {0.0, 0.0, 0.0}, Q[3][3] = {{0.0}};
  };
  std::map<Key, Stat> stat;
  auto corner = [&](const Voxel& v, int a) { return m.p.map_origin[a] + (double)v.v[a] * m.p.voxel_size; };
  auto stat_of = [&](const Voxel& v) -> Stat& {
    const Key k = std::make_tuple(v.v[0], v.v[1], v.v[2]);
    auto it = stat.find(k);
    if (it != stat.end()) return it->second;
    Stat s;
    auto rit = m.regions.find(region_of(v));
    if (rit != m.regions.end() && !rit->second.ndt.empty()) {
      const __int128* q = &rit->second.ndt[(size_t)local_index(v) * 10];
      s.n = (double)q[0];
      for (int a = 0; a < 3; ++a) s.S[a] = (double)q[1 + a] * cell;
      const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
      for (int k6 = 0; k6 < 6; ++k6) {
        s.Q[pa[k6]][pb[k6]] = (double)q[4 + k6] * cell * cell;
        s.Q[pb[k6]][pa[k6]] = s.Q[pa[k6]][pb[k6]];
      }
    }
    return stat.emplace(k, s).first->second;
  };
  for (int64_t j = 0; j < n; ++j) {
    if (!has[(size_t)j]) continue;
    Stat& s = stat_of(vox[(size_t)j]);
    double p[3];
    for (int a = 0; a < 3; ++a) p[a] = e_eval[3 * j + a] - corner(vox[(size_t)j], a);
    s.n += 1.0;
    for (int a = 0; a < 3; ++a) {
      s.S[a] += p[a];
      for (int b = 0; b < 3; ++b) s.Q[a][b] += p[a] * p[b];
    }
  }
  // upstream weights per voxel, summed over its queries
  std::map<Key, std::array<double, 9>> G;
  for (int64_t q = 0; q < m_q; ++q) {
    auto& g = G[std::make_tuple(qvox[3 * q], qvox[3 * q + 1], qvox[3 * q + 2])];
    for (int a = 0; a < 3; ++a) g[a] += gm[3 * q + a];
    for (int k6 = 0; k6 < 6; ++k6) g[3 + k6] += gc[6 * q + k6];
  }
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
  double L = 0.0;
  for (const auto& kv : G) {
    Voxel v;
    v.v[0] = std::get<0>(kv.first);
    v.v[1] = std::get<1>(kv.first);
    v.v[2] = std::get<2>(kv.first);
    const Stat& s = stat_of(v);
    if (!(s.n > 0.0)) continue;
    double mu[3];
    for (int a = 0; a < 3; ++a) mu[a] = s.S[a] / s.n;
    for (int a = 0; a < 3; ++a) L += kv.second[a] * (corner(v, a) + mu[a]);
    for (int k6 = 0; k6 < 6; ++k6)
      L += kv.second[3 + k6] * (s.Q[pa[k6]][pb[k6]] / s.n - mu[pa[k6]] * mu[pb[k6]]);
  }
  *loss = L;
  if (grad_e) {
    for (int64_t j = 0; j < n; ++j) {
      double* ge = grad_e + 3 * j;
      ge[0] = ge[1] = ge[2] = 0.0;
      if (!has[(size_t)j]) continue;
      const Voxel& v = vox[(size_t)j];
      auto gi = G.find(std::make_tuple(v.v[0], v.v[1], v.v[2]));
      if (gi == G.end()) continue;
      const Stat& s = stat_of(v);
      double d[3];
      for (int a = 0; a < 3; ++a) d[a] = e_eval[3 * j + a] - corner(v, a) - s.S[a] / s.n;
      double Gm[3][3] = {{0.0}};
      for (int k6 = 0; k6 < 6; ++k6) Gm[pa[k6]][pb[k6]] = gi->second[3 + k6];
      for (int k = 0; k < 3; ++k) {
        double t = gi->second[k];
        for (int b = 0; b < 3; ++b) t += (Gm[k][b] + Gm[b][k]) * d[b];
        ge[k] = t / s.n;
      }
    }
  }
  return 0;
}

// For each ray of a frame (band voxels frozen as in oracle_tsdf_frame_eval),
// the distance of the clamp from the nearest unclamped value among its band
// voxels: min over the band of | |s_j(v)| - tau | with s_j(v) = (e - centre).u
// at the continuous geometry (o_eval, e_eval), double; +inf for a ray that
// updates no voxel.  Where it is tiny, evaluations of s that differ by
// rounding or quantisation can disagree on whether s is clamped, and with it
// on that voxel's gradient.  Returns 0, or -1 on bad arguments.
int oracle_tsdf_band_margin(void* h, const float* o_nom, const float* e_nom, const uint8_t* flags, int64_t n,
                            const double* o_eval, const double* e_eval, double* margin) {
  Map& m = *static_cast<Map*>(h);
  if (!(m.p.layers & kLayerTsdf)) return -1;
  const std::vector<std::vector<Voxel>> bands = frozen_bands(m, o_nom, e_nom, flags, n);
  const double tau = m.p.tsdf_trunc;
  for (int64_t j = 0; j < n; ++j) {
    double best = INFINITY;
    if (!bands[(size_t)j].empty()) {
      const double* e = e_eval + 3 * j;
      double u[3], dist = 0.0;
      for (int a = 0; a < 3; ++a) {
        u[a] = e[a] - o_eval[a];
        dist += u[a] * u[a];
      }
      dist = std::sqrt(dist);
      for (int a = 0; a < 3; ++a) u[a] /= dist;
      for (const Voxel& v : bands[(size_t)j]) {
        double s = 0.0;
        for (int a = 0; a < 3; ++a) s += (e[a] - (m.p.map_origin[a] + ((double)v.v[a] + 0.5) * m.p.voxel_size)) * u[a];
        const double gap = std::fabs(std::fabs(s) - tau);
        if (gap < best) best = gap;
      }
    }
    margin[j] = best;
  }
  return 0;
}

// The walk alone, for tests: writes up to cap visited voxels (x, y, z) and
// returns how many the walk visits.
int64_t oracle_walk(const int64_t* a, const int64_t* b, int32_t frac_bits, int64_t* out, int64_t cap) {
  std::vector<Voxel> vox = walk(a, b, (int64_t)1 << frac_bits);
  for (int64_t i = 0; i < (int64_t)vox.size() && i < cap; ++i)
    for (int k = 0; k < 3; ++k) out[3 * i + k] = vox[(size_t)i].v[k];
  return (int64_t)vox.size();
}

// The timed walk alone, for tests: voxels (cap x 3) and their (t_in, t_out)
// (cap x 2, fractions of 2^32).  Returns the number of voxels.
int64_t oracle_walk_timed(const int64_t* a, const int64_t* b, int32_t frac_bits, int64_t* out, uint64_t* times,
                          int64_t cap) {
  std::vector<TimedVoxel> vox = walk_timed(a, b, (int64_t)1 << frac_bits);
  for (int64_t i = 0; i < (int64_t)vox.size() && i < cap; ++i) {
    for (int k = 0; k < 3; ++k) out[3 * i + k] = vox[(size_t)i].v.v[k];
    times[2 * i] = vox[(size_t)i].t_in;
    times[2 * i + 1] = vox[(size_t)i].t_out;
  }
  return (int64_t)vox.size();
}

// Quantisation and truncation alone, for tests.  Writes qo, qe (n x 3 int64)
// and has_sample (n uint8); valid[i] = 0 for a skipped (non-finite) ray.
void oracle_prepare(void* h, const float* origins, int64_t n_origins, const float* endpoints, const uint8_t* flags,
                    int64_t n, int64_t* qo, int64_t* qe, uint8_t* has_sample, uint8_t* valid) {
  Map& m = *static_cast<Map*>(h);
  for (int64_t i = 0; i < n; ++i) {
    PreparedRay r;
    bool ok = prepare_ray(m, origins + 3 * (n_origins == 1 ? 0 : i), endpoints + 3 * i, flags ? flags[i] : 0, &r);
    valid[i] = ok ? 1 : 0;
    has_sample[i] = ok && r.has_sample ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
      qo[3 * i + a] = ok ? r.qo[a] : 0;
      qe[3 * i + a] = ok ? r.qe[a] : 0;
    }
  }
}

}  // extern "C"
