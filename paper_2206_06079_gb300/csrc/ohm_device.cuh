// Device-side data structures of the GB300 ray-integration library: the map
// (region hash table, region pool, layers), the per-call scratch, and the
// exact fixed-point voxel walk shared by every kernel.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

// Loop unrolling hint for code compiled for both host and device.
#ifdef __CUDA_ARCH__
#define OHM_UNROLL _Pragma("unroll")
#else
#define OHM_UNROLL
#endif

namespace ohm {

constexpr int kRegionShift = 5;                  // 32 voxels per region edge (Sec. III-B: 3.2 m at 0.1 m)
constexpr int kRegionVoxels = 1 << (3 * kRegionShift);
constexpr long long kEmptyKey = -1;              // never a packed key (packed keys are < 2^63)
constexpr long long kTombKey = -2;               // a key removed by a rolled-back call

constexpr uint32_t kLayerOcc = 1, kLayerNdt = 2, kLayerTsdf = 4, kLayerCounts = 8, kLayerDecay = 16, kLayerMean = 32;
constexpr uint8_t kFlagNoReturn = 1;

// Status bits latched in device memory (0 = fine).
constexpr int kStatusCapacity = 1;   // region or NDT pool full
constexpr int kStatusProbe = 2;      // hash probe bound exceeded
constexpr int kStatusScratch = 4;    // per-call scratch too small (a library bug)
constexpr int kStatusMissing = 8;    // a region expected in the table was not found (a library bug)
constexpr int kStatusCasLimit = 16;  // a CAS loop gave up (a library bug)
constexpr int kStatusRestore = 32;   // the call touched evicted regions: restore them, then repeat it

// Hash-entry slot values below zero.
constexpr long long kSlotPending = -1;    // inserted by this kernel, slot not yet written (or none left)
constexpr long long kSlotEvicted = -3;    // region evicted to host memory
constexpr long long kSlotRestoring = -4;  // evicted, and a restore was requested by the current call

constexpr int32_t kRayValid = 1, kRaySample = 2, kRayAxisShift = 4, kRaySignShift = 8;

// Ray record written by the occupancy prepare kernel: the walk from a to b
// (fixed point) reduced to per-axis 32-bit constants, so that every segment of
// the ray starts from them without redoing the 64-bit set-up.
//   v0  voxel of a;  A = |b - a|  (< 2^30, see Walker);  d0 = distance from a
//   to the first boundary crossed (0 .. 2^F);  n = steps along the axis;
//   sign bit k (flags bit kRaySignShift + k) set when b_k < a_k.
struct __align__(16) RayRec {
  int32_t v0[3];
  int32_t A[3];
  int32_t d0[3];
  int32_t n[3];
  unsigned long long inv;  // reciprocal64 of A[dominant axis] (0 if that is 0)
  int32_t flags;           // kRayValid | kRaySample | dominant axis << kRayAxisShift | signs
  int32_t nseg;            // number of segments
};

// Decay-rate record of a ray (written only for maps with the decay layer):
// reciprocal64 of A per axis and the walk length L in 2^-20 m.
struct __align__(16) DecayRec {
  unsigned long long inv[3];
  unsigned long long length;
};

// Length of the walk from a to b in units of 2^-20 m (the decay layer's L):
// rint(sqrt(|b - a|^2) * voxel_size / 2^F * 2^20), double, one rounding per
// operation.
__host__ __device__ __forceinline__ unsigned long long walk_length_units(const long long a[3], const long long b[3],
                                                                         double voxel_size, int F) {
  double d[3];
OHM_UNROLL
  for (int k = 0; k < 3; ++k) d[k] = (double)(b[k] - a[k]);
  const double per_unit = voxel_size / (double)(1LL << F);
#ifdef __CUDA_ARCH__
  double l2 = __dmul_rn(d[0], d[0]);
  l2 = __dadd_rn(l2, __dmul_rn(d[1], d[1]));
  l2 = __dadd_rn(l2, __dmul_rn(d[2], d[2]));
  return (unsigned long long)__double2ll_rn(__dmul_rn(__dmul_rn(__dsqrt_rn(l2), per_unit), 1048576.0));
#else
  double l2 = d[0] * d[0];
  l2 = l2 + d[1] * d[1];
  l2 = l2 + d[2] * d[2];
  return (unsigned long long)std::llrint((std::sqrt(l2) * per_unit) * 1048576.0);
#endif
}

// A ray kept as its two fixed-point end points (the allocation-free entry
// point's record).
struct __align__(16) EndpointRec {
  long long a[3];
  long long b[3];
  unsigned long long inv;
  int32_t flags;
  int32_t nseg;
};

// Ray record written by the TSDF prepare kernel: the walk covers the band
// [max(0, d - tau), d + tau] of the ray from the sensor to the sample e.
struct __align__(16) TsdfRec {
  long long a[3];   // band start, fixed point
  long long b[3];   // band end, fixed point
  long long e[3];   // sample, fixed point
  float u[3];       // unit direction sensor -> sample
  int32_t flags;    // kRayValid when the ray updates the TSDF
};

// Per-call counters in device memory.
// A float-float value hi + lo with |lo| <= ulp(hi) / 2 (the arithmetic is
// with the TSDF band below).
struct FF {
  float hi, lo;
};

// The TSDF band's constants as float-float (tsdf_band_ff).
struct BandConsts {
  FF tau, rmin, rmax;  // fixed-point units
};

struct CallCounters {
  unsigned long long segments;
  unsigned long long visits;
  unsigned long long touched;
  int32_t region_start;   // pool counters when the call began (rollback point)
  int32_t ndt_start;
  unsigned long long rays;
  unsigned long long total_visits;  // every call since the map was made
  int32_t seq;                      // sequence number of the current call (LRU stamps, birth marks)
  int32_t free_used_start;          // free-list positions when the call began (rollback point)
  int32_t ndt_free_used_start;
  int32_t mean_touched;             // entries of mean_list written by the current call
  unsigned long long restores;      // evicted region keys this call asked to restore
  long long origin_q[3];            // the call's shared sensor origin, quantised (one origin only)
  int32_t origin_ok;                // 1 if origin_q is valid
  int32_t pad2;
  unsigned long long atomics;       // log-odds CAS operations the miss walk issued (single-map calls)
  unsigned long long ndt_pending;   // entries of DeviceMap::ndt_pending written by the current call
};

// Everything a kernel needs, passed by value.
struct DeviceMap {
  // region hash table: key -> pool slot (Sec. III-A); entry = (key, slot)
  longlong2* htab;
  uint32_t hmask;
  int32_t max_probe;
  // region pool
  int32_t* region_count;
  int32_t max_regions;
  int32_t* region_coords;        // [max_regions][3]
  float* occ;                    // [max_regions][32768], Morton order inside a region
  unsigned long long* counts;    // [max_regions][32768], hits << 32 | misses
  unsigned long long* decay;     // [max_regions][32768], summed path length, 2^-20 m
  unsigned long long* vmean;     // [max_regions][32768], count << 32 | z10 << 20 | y10 << 10 | x10
  unsigned long long* vmean_acc; // [max_regions][32768][2], per-call sums: Sx | Sy << 32, Sz | c << 32
  int32_t* mean_list;            // [max_rays], voxels given samples by the current call
  int32_t* ndt_slot;             // [max_regions], -1 = no NDT layer yet
  int32_t* ndt_count;
  int32_t max_ndt;
  int32_t* ndt_pending;          // [max_rays] sample rays whose region prepare could not give an NDT block
  long long* ndt;                // [max_ndt][10][32768]
  float2* tsdf;                  // [max_regions][32768] (D, W)
  uint32_t* tsdf_cnt;            // [max_regions][32768] per-call scratch, zero between calls
  long long* tsdf_sum;           // [max_regions][32768] per-call scratch, 2^-32 m units
  float* grad;                   // [max_regions][32768] adjoint weights, allocated by the first backward call
  float* ndt_grad;               // [max_ndt][32768][9] NDT adjoint weights, allocated by the first NDT backward call
  int32_t* status;
  CallCounters* calls;
  // region cache (Sec. III-A: regions move between device and host memory)
  int32_t* stamp;                // [max_regions] seq of the last call that touched the region
  int32_t* born;                 // [max_regions] seq of the call that inserted the region
  int32_t* ndt_born;             // [max_regions] seq of the call that gave the region its NDT block
  int32_t* free_slots;           // [max_regions] region slots released by eviction
  int32_t* ndt_free;             // [max_ndt] NDT blocks released by eviction
  int32_t* free_info;            // [0] free slots, [1] used, [2] free NDT blocks, [3] used
  long long* restore_keys;       // [max_restore] evicted keys touched by the current call
  int32_t max_restore;
  // per-call scratch
  RayRec* rays;
  DecayRec* decay_rays;  // [max_rays], decay layer only
  TsdfRec* trays;
  int2* segs;                    // (ray, segment index)
  long long max_segs;
  int32_t* touched;              // TSDF voxels touched by this call (slot * 32768 + morton)
  long long max_touched;
  // parameters
  double origin[3];
  double scale;                  // 2^F / voxel_size
  double rmax_q, rmin_q, tau_q;  // ranges in fixed-point units
  BandConsts band;               // tau_q, rmin_q, rmax_q as float-float
  // a ray with |b - a|^2 <= rmax_in2 (fixed-point units^2) is certainly
  // within max_range
  unsigned long long rmax_in2;
  double voxel_size;
  int32_t frac_bits;
  uint32_t layers;
  int32_t seg_steps;
  float hit, miss, l_min, l_max;
  float ndt_clear;               // clear NDT samples when a miss crosses below this (-inf: never)
  float tau_m, wmax;
};

// Arguments of one integrate call.
struct CallArgs {
  const float* origins;
  const float* endpoints;
  const uint8_t* flags;
  long long n;
  long long n_origins;
};

// ---------------------------------------------------------------------------
// Region keys and the hash table.
// ---------------------------------------------------------------------------
__host__ __device__ inline long long pack_region(int rx, int ry, int rz) {
  const unsigned long long m = (1ULL << 21) - 1;
  return (long long)((((unsigned long long)rx & m) << 42) | (((unsigned long long)ry & m) << 21) |
                     ((unsigned long long)rz & m));
}

// 64-bit finaliser of MurmurHash3 (Appleby), a published bit mixer.
__device__ __forceinline__ uint32_t hash_key(long long k) {
  unsigned long long x = (unsigned long long)k;
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return (uint32_t)x;
}

// Pool slot of a region, or -1.  Read-only use of the table: one 16-byte
// load per probe brings the key and its slot together.
__device__ __forceinline__ int32_t find_region(const DeviceMap& m, long long key) {
  uint32_t h = hash_key(key) & m.hmask;
  for (int i = 0; i < m.max_probe; ++i) {
    const longlong2 e = m.htab[h];
    if (e.x == key) return (int32_t)e.y;
    if (e.x == kEmptyKey) return -1;
    h = (h + 1) & m.hmask;
  }
  return -1;
}

// A pool slot for a new region: a slot released by eviction if any is left,
// else the next never-used one; -1 when the pool is full.
__device__ __forceinline__ int32_t alloc_region_slot(const DeviceMap& m) {
  const int32_t i = atomicAdd(&m.free_info[1], 1);
  if (i < m.free_info[0]) return m.free_slots[i];
  const int32_t s = atomicAdd(m.region_count, 1);
  return s < m.max_regions ? s : -1;
}

// An NDT block for a region, the same way.
__device__ __forceinline__ int32_t alloc_ndt_block(const DeviceMap& m) {
  const int32_t i = atomicAdd(&m.free_info[3], 1);
  if (i < m.free_info[2]) return m.ndt_free[i];
  const int32_t s = atomicAdd(m.ndt_count, 1);
  return s < m.max_ndt ? s : -1;
}

// Insert a region if absent, and mark it used by the current call.  The
// inserting thread takes a pool slot; other threads only learn that the key
// exists (slots are read after this kernel).  Returns the region's slot where
// this thread knows it (it inserted the key, or found it with its slot), else
// -1 (another thread is inserting it right now, it is evicted, or the call
// failed).  A key whose region was evicted
// to host memory is queued for restoring and the call is stopped (it will be
// repeated once the region is back).  The first probe may read a stale cached
// entry: a key once written never changes within a call, and a stale "empty"
// only sends us to the CAS below.
__device__ inline int32_t insert_region(const DeviceMap& m, int rx, int ry, int rz) {
  const long long key = pack_region(rx, ry, rz);
  const int32_t seq = m.calls->seq;
  uint32_t h = hash_key(key) & m.hmask;
  for (int i = 0; i < m.max_probe; ++i) {
    const longlong2 e = m.htab[h];
    long long k = e.x;
    if (k == kEmptyKey) {
      const long long prev = (long long)atomicCAS((unsigned long long*)&m.htab[h].x, (unsigned long long)kEmptyKey,
                                                  (unsigned long long)key);
      if (prev == kEmptyKey) {
        const int32_t s = alloc_region_slot(m);
        if (s >= 0) {
          m.htab[h].y = s;
          m.region_coords[3 * s + 0] = rx;
          m.region_coords[3 * s + 1] = ry;
          m.region_coords[3 * s + 2] = rz;
          m.born[s] = seq;
          m.stamp[s] = seq;
        } else {
          atomicOr(m.status, kStatusCapacity);
        }
        return s;
      }
      if (prev != key) {
        h = (h + 1) & m.hmask;
        continue;
      }
      return -1;  // another thread inserted it just now; it stamps the slot
    }
    if (k == key) {
      const long long slot = e.y;
      if (slot >= 0) {
        m.stamp[slot] = seq;
        return (int32_t)slot;
      } else if (slot == kSlotEvicted || slot == kSlotRestoring) {
        if (atomicCAS((unsigned long long*)&m.htab[h].y, (unsigned long long)kSlotEvicted,
                      (unsigned long long)kSlotRestoring) == (unsigned long long)kSlotEvicted) {
          const unsigned long long r = atomicAdd(&m.calls->restores, 1ULL);
          if (r < (unsigned long long)m.max_restore) m.restore_keys[r] = key;
        }
        atomicOr(m.status, kStatusRestore);
      }
      return -1;
    }
    h = (h + 1) & m.hmask;
  }
  atomicOr(m.status, kStatusProbe);
  return -1;
}

// ---------------------------------------------------------------------------
// Fixed-point quantisation: q = rint((x - origin) * scale), double, one
// rounding per operation (no contraction).  Returns false when |value| would
// not be exactly representable (>= 2^52).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool quantise(float x, double origin, double scale, long long* q) {
  double d = __dsub_rn((double)x, origin);
  double s = __dmul_rn(d, scale);
  // |s| < 2^52 (also rejects NaN), tested on the bit pattern
  if (!((__double_as_longlong(s) & 0x7fffffffffffffffLL) < 0x4330000000000000LL)) return false;
  *q = __double2ll_rn(s);
  return true;
}

// ---------------------------------------------------------------------------
// Morton order inside a region: bit 3i = x_i, 3i+1 = y_i, 3i+2 = z_i.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t spread5(uint32_t x) {
  uint32_t r = 0;
  for (int b = 0; b < 5; ++b) r |= ((x >> b) & 1u) << (3 * b);
  return r;
}
__host__ __device__ __forceinline__ uint32_t morton(uint32_t x, uint32_t y, uint32_t z) {
  return spread5(x) | (spread5(y) << 1) | (spread5(z) << 2);
}

// Morton index of a voxel inside its region.
__host__ __device__ __forceinline__ uint32_t region_morton(int32_t vx, int32_t vy, int32_t vz) {
  const int32_t mask = (1 << kRegionShift) - 1;
  return morton((uint32_t)(vx & mask), (uint32_t)(vy & mask), (uint32_t)(vz & mask));
}

// Step one axis of a Morton index by +-1, wrapping inside the 5 bits of that axis.
__host__ __device__ __forceinline__ uint32_t morton_step(uint32_t m, uint32_t mask, int sign) {
  uint32_t moved = sign > 0 ? ((m | ~mask) + 1u) : ((m & mask) - 1u);
  return (moved & mask) | (m & ~mask);
}

// ---------------------------------------------------------------------------
// Exact integer voxel walk (Amanatides & Woo, as adapted in Sec. III-B).
//
// Along axis k the ray from a to b moves A_k = |b_k - a_k| fixed-point units
// per unit of the ray parameter t; the next boundary of the current voxel is
// dist_k units away, reached at t_k = dist_k / A_k.  Every iteration steps the
// axis with the smallest t_k (ties: z, then y, then x), never an axis that has
// already reached b's voxel.  Instead of comparing quotients the walker keeps
// the three pairwise differences
//     C_xy = dist_x A_y - dist_y A_x   (t_x < t_y  <=>  C_xy < 0)
//     C_xz = dist_x A_z - dist_z A_x
//     C_yz = dist_y A_z - dist_z A_y
// which change by constants when an axis steps (dist_k grows by U = 2^F).
// Magnitudes stay below 2^61 because every ray is shorter than 2^30
// fixed-point units (checked when the map is made).
//
// An axis with no steps left ("exhausted") keeps exact differences: its next
// boundary lies at or beyond b, so t >= 1 while every remaining crossing has
// t <= 1.  It can therefore only be picked on a tie at t = 1, when every axis
// with steps left also sits at t = 1; the highest such axis steps then, which
// is what the tie order prescribes among them.
//
// Segments (Sec. III-B "breaking long rays into several segments"): the walk
// of one ray is split by the number K of steps taken along its dominant axis
// M.  walk_init(K) reconstructs the exact state right after the K-th M step
// without walking: for every other axis it counts, by integer division, the
// boundary crossings that come before that step in walk order.  So every
// segment visits exactly the voxels the unsplit walk visits, in order.
// ---------------------------------------------------------------------------
struct Walker {
  long long cxy, cxz, cyz;
  long long ua, ub, uc;   // U*A_x, U*A_y, U*A_z
  int32_t vx, vy, vz;     // current voxel
  int32_t nx, ny, nz;     // steps left per axis
  int32_t sx, sy, sz;     // step sign per axis (+1 / -1)
  int32_t total;          // steps left in the whole ray
};

__host__ __device__ __forceinline__ long long sel3(int k, long long a, long long b, long long c) {
  return k == 0 ? a : (k == 1 ? b : c);
}

// Returns the index of the dominant axis (the lowest of equal ones) and the
// number of steps it takes.
__host__ __device__ __forceinline__ int dominant_axis(const long long a[3], const long long b[3], int F, int32_t* nmaj) {
  long long d0 = (b[0] >> F) - (a[0] >> F), d1 = (b[1] >> F) - (a[1] >> F), d2 = (b[2] >> F) - (a[2] >> F);
  d0 = d0 < 0 ? -d0 : d0;
  d1 = d1 < 0 ? -d1 : d1;
  d2 = d2 < 0 ? -d2 : d2;
  int M = 0;
  long long best = d0;
  if (d1 > best) {
    best = d1;
    M = 1;
  }
  if (d2 > best) {
    best = d2;
    M = 2;
  }
  *nmaj = (int32_t)best;
  return M;
}

// High 64 bits of the 128-bit product x * y.
__host__ __device__ __forceinline__ unsigned long long umulhi64(unsigned long long x, unsigned long long y) {
#ifdef __CUDA_ARCH__
  return __umul64hi(x, y);
#else
  return (unsigned long long)(((unsigned __int128)x * y) >> 64);
#endif
}

// Reciprocal of a divisor d >= 1 for div_by_inv: floor((2^64 - 1) / d).
__host__ __device__ __forceinline__ unsigned long long reciprocal64(unsigned long long d) {
  return d ? ~0ULL / d : 0ULL;
}

// floor(x / d) for 0 <= x < 2^63 and d >= 1, given inv = reciprocal64(d).
// inv <= 2^64 / d gives q = floor(x inv / 2^64) <= x / d, and
// inv >= 2^64 / d - 1 gives x inv / 2^64 >= x / d - x / 2^64 > x / d - 1, so
// q is floor(x / d) or one less; one remainder test makes it exact.
__host__ __device__ __forceinline__ unsigned long long div_by_inv(unsigned long long x, unsigned long long d,
                                                                unsigned long long inv) {
  unsigned long long q = umulhi64(x, inv);
  if (x - q * d >= d) q += 1;
  return q;
}

// Crossings of a non-dominant axis (distance d0k to its first boundary,
// speed Ak) that come before the K-th step of the dominant axis M (distance
// d0M, speed AM), in walk order: crossing i precedes it when
// (d0k + i U) / Ak < (d0M + (K-1) U) / AM, or the two are equal and the axis
// is above M (ties step z, then y, then x).  Capped at the axis' total ntot.
// Division by U AM is done as floor(floor(x / U) / AM); inv_am is
// reciprocal64(AM), or 0 to divide directly.
__host__ __device__ __forceinline__ long long crossings_before(long long d0k, long long Ak, long long d0M, long long AM,
                                                              int F, long long K, bool above_major, int32_t ntot,
                                                              unsigned long long inv_am) {
  const long long U = 1LL << F;
  const long long R = (d0M + (K - 1) * U) * Ak - d0k * AM;
  long long c;
  if (!above_major ? R <= 0 : R < 0) {
    c = 0;
  } else {
    const unsigned long long x = ((unsigned long long)(above_major ? R : R - 1)) >> F;
    const unsigned long long q = inv_am ? div_by_inv(x, (unsigned long long)AM, inv_am) : x / (unsigned long long)AM;
    c = (long long)q + 1;
  }
  return c < ntot ? c : (long long)ntot;
}

// State of the walk from a to b right after K steps along the dominant axis M
// (K = 0: the start).  inv_am: reciprocal64(|b_M - a_M|), or 0.
__host__ __device__ inline void walker_init(Walker& w, const long long a[3], const long long b[3], int F, int M, long long K,
                                            unsigned long long inv_am = 0) {
  const long long U = 1LL << F;
  long long A[3], d0[3], cnt[3];
  int32_t ntot[3], sgn[3], v0[3];
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    long long delta = b[k] - a[k];
    A[k] = delta < 0 ? -delta : delta;
    sgn[k] = delta < 0 ? -1 : 1;
    long long va = a[k] >> F;  // arithmetic shift: floor
    long long vb = b[k] >> F;
    long long nt = vb - va;
    ntot[k] = (int32_t)(nt < 0 ? -nt : nt);
    d0[k] = delta < 0 ? (a[k] - va * U) : ((va + 1) * U - a[k]);
    v0[k] = (int32_t)va;
  }
  const long long d0M = sel3(M, d0[0], d0[1], d0[2]);
  const long long AM = sel3(M, A[0], A[1], A[2]);
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    if (K == 0)
      cnt[k] = 0;
    else if (k == M)
      cnt[k] = K;
    else
      cnt[k] = crossings_before(d0[k], A[k], d0M, AM, F, K, k > M, ntot[k], inv_am);
  }
  long long dist[3];
OHM_UNROLL
  for (int k = 0; k < 3; ++k) dist[k] = d0[k] + cnt[k] * U;
  w.vx = v0[0] + (int32_t)(sgn[0] * cnt[0]);
  w.vy = v0[1] + (int32_t)(sgn[1] * cnt[1]);
  w.vz = v0[2] + (int32_t)(sgn[2] * cnt[2]);
  w.nx = ntot[0] - (int32_t)cnt[0];
  w.ny = ntot[1] - (int32_t)cnt[1];
  w.nz = ntot[2] - (int32_t)cnt[2];
  w.sx = sgn[0];
  w.sy = sgn[1];
  w.sz = sgn[2];
  w.ua = U * A[0];
  w.ub = U * A[1];
  w.uc = U * A[2];
  w.cxy = dist[0] * A[1] - dist[1] * A[0];
  w.cxz = dist[0] * A[2] - dist[2] * A[0];
  w.cyz = dist[1] * A[2] - dist[2] * A[1];
  w.total = w.nx + w.ny + w.nz;
}

// Per-ray walk constants of the walk from a to b (see RayRec); keeps the
// other fields of r.
__host__ __device__ inline void ray_constants(const long long a[3], const long long b[3], int F, RayRec* r) {
  const long long U = 1LL << F;
  int32_t signs = 0;
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    const long long delta = b[k] - a[k];
    const long long va = a[k] >> F, vb = b[k] >> F;
    const long long nt = vb - va;
    r->v0[k] = (int32_t)va;
    r->A[k] = (int32_t)(delta < 0 ? -delta : delta);
    r->d0[k] = (int32_t)(delta < 0 ? (a[k] - va * U) : ((va + 1) * U - a[k]));
    r->n[k] = (int32_t)(nt < 0 ? -nt : nt);
    if (delta < 0) signs |= 1 << k;
  }
  r->flags = (r->flags & ~(7 << kRaySignShift)) | (signs << kRaySignShift);
}

// The end point b of a ray, from its constants.
__host__ __device__ inline void ray_end(const RayRec& r, int F, long long b[3]) {
  const long long U = 1LL << F;
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    const bool neg = (r.flags >> (kRaySignShift + k)) & 1;
    const long long a = neg ? (long long)r.v0[k] * U + r.d0[k] : ((long long)r.v0[k] + 1) * U - r.d0[k];
    b[k] = neg ? a - r.A[k] : a + r.A[k];
  }
}

// walker_init from the per-ray constants (same state, cheaper set-up).
__host__ __device__ inline void walker_init_rec(Walker& w, const RayRec& r, int F, int M, long long K) {
  const long long U = 1LL << F;
  const long long d0M = M == 0 ? r.d0[0] : (M == 1 ? r.d0[1] : r.d0[2]);
  const long long AM = M == 0 ? r.A[0] : (M == 1 ? r.A[1] : r.A[2]);
  long long cnt[3];
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    if (K == 0)
      cnt[k] = 0;
    else if (k == M)
      cnt[k] = K;
    else
      cnt[k] = crossings_before(r.d0[k], r.A[k], d0M, AM, F, K, k > M, r.n[k], r.inv);
  }
  const int32_t sx = ((r.flags >> kRaySignShift) & 1) ? -1 : 1;
  const int32_t sy = ((r.flags >> (kRaySignShift + 1)) & 1) ? -1 : 1;
  const int32_t sz = ((r.flags >> (kRaySignShift + 2)) & 1) ? -1 : 1;
  const long long dx = r.d0[0] + cnt[0] * U, dy = r.d0[1] + cnt[1] * U, dz = r.d0[2] + cnt[2] * U;
  w.vx = r.v0[0] + sx * (int32_t)cnt[0];
  w.vy = r.v0[1] + sy * (int32_t)cnt[1];
  w.vz = r.v0[2] + sz * (int32_t)cnt[2];
  w.nx = r.n[0] - (int32_t)cnt[0];
  w.ny = r.n[1] - (int32_t)cnt[1];
  w.nz = r.n[2] - (int32_t)cnt[2];
  w.sx = sx;
  w.sy = sy;
  w.sz = sz;
  w.ua = U * r.A[0];
  w.ub = U * r.A[1];
  w.uc = U * r.A[2];
  w.cxy = dx * r.A[1] - dy * r.A[0];
  w.cxz = dx * r.A[2] - dz * r.A[0];
  w.cyz = dy * r.A[2] - dz * r.A[1];
  w.total = w.nx + w.ny + w.nz;
}

// Axis of the next step (requires w.total > 0).
__host__ __device__ __forceinline__ int walker_choose(const Walker& w) {
  int axis = (w.cxy < 0 && w.cxz < 0) ? 0 : ((w.cxy >= 0 && w.cyz < 0) ? 1 : 2);
  const int32_t left = axis == 0 ? w.nx : (axis == 1 ? w.ny : w.nz);
  if (left == 0) axis = w.nz > 0 ? 2 : (w.ny > 0 ? 1 : 0);  // a tie at t = 1 (see above)
  return axis;
}

// Take one step along `axis`; returns the new coordinate along that axis and
// its step sign through *coord / *sign.  Written with selects so that lanes
// stepping different axes do not diverge.
__host__ __device__ __forceinline__ void walker_step(Walker& w, int axis, int32_t* coord, int32_t* sign) {
  const bool bx = axis == 0, by = axis == 1, bz = axis == 2;
  w.cxy += bx ? w.ub : (by ? -w.ua : 0LL);
  w.cxz += bx ? w.uc : (bz ? -w.ua : 0LL);
  w.cyz += by ? w.uc : (bz ? -w.ub : 0LL);
  w.vx += bx ? w.sx : 0;
  w.vy += by ? w.sy : 0;
  w.vz += bz ? w.sz : 0;
  w.nx -= bx ? 1 : 0;
  w.ny -= by ? 1 : 0;
  w.nz -= bz ? 1 : 0;
  w.total -= 1;
  *coord = bx ? w.vx : (by ? w.vy : w.vz);
  *sign = bx ? w.sx : (by ? w.sy : w.sz);
}

__host__ __device__ __forceinline__ uint32_t morton_mask(int axis) {
  return axis == 0 ? 0x1249u : (axis == 1 ? 0x2492u : 0x4924u);
}

// ---------------------------------------------------------------------------
// Filtered exact walk: the integrate kernels' voxel walk.  It visits exactly
// the voxels of Walker, in the same order, with cheaper steps.
//
// Along every axis k it keeps c_k, the boundary crossings taken so far, and
// an FP32 estimate of the exact crossing parameter of the next boundary,
//     t_k = (d0_k + c_k U) / A_k,
//     t^_k = fma(c_k, dU_k, t0_k),  r_k = rcp(float(A_k)),  dU_k = U r_k,  t0_k = d0_k r_k.
// float(A_k), the reciprocal, d0_k r_k and the fma each round once (U is a
// power of two and d0_k <= 2^20, c_k < 2^24 are exact in float), so
// t^_k = t_k (1 + e) with |e| <= (1 + u)^3 / (1 - u) - 1 < 4.01 u, u = 2^-24.
// A step is decided on the estimates when exactly one axis a has
// t^_a <= thr = fl(g min_k t^_k), g = 1 + 2^-20 = 1 + 16 u.  Then for every
// other axis j, t^_j > thr >= g (1 - u) t^_a, so
//     t_j >= t^_j / (1 + 4.01 u) > t^_a g (1 - u) / (1 + 4.01 u) >= t^_a / (1 - 4.01 u) >= t_a
// (g (1 - u)(1 - 4.01 u) >= 1 + 4.01 u holds since 16 - 1 - 4.01 > 4.01):
// a is the strict minimum of the exact parameters, which is the axis the
// exact rule steps.  It is never an axis without steps left (those have
// t >= 1, and an axis with steps left has t <= 1).  When the estimates do not
// single out one axis (a near-tie), the exact 64-bit comparison of Walker
// decides, from c_k (exact_pick).  An axis with A_k = 0 never steps:
// dU_k = 0, t0_k = +inf, so t^_k = +inf.
//
// Morton indices are stepped in a sign-normalised form: the bits of an axis
// walked in the negative direction are stored inverted, so that every step is
// +1 on its axis and leaving the region is the wrap from 31 to 0 in both
// directions.  The voxel's real Morton index is mo ^ neg.
// ---------------------------------------------------------------------------
struct FWalker {
  float tx, ty, tz;  // t^ per axis
  float cx, cy, cz;  // crossings taken per axis (exact integers)
  float ux, uy, uz;  // dU
  float ox, oy, oz;  // t0
};

__host__ __device__ __forceinline__ float rcp_rn(float x) {
#ifdef __CUDA_ARCH__
  return __frcp_rn(x);
#else
  return 1.0f / x;
#endif
}
__host__ __device__ __forceinline__ float fmul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// FP32 constants of one axis.
__host__ __device__ __forceinline__ void fwalker_axis(int32_t A, int32_t d0, int F, float c, float* u, float* o, float* t) {
  if (A == 0) {
    *u = 0.0f;
    *o = INFINITY;
  } else {
    const float r = rcp_rn((float)A);
    *u = fmul_rn(r, (float)(1 << F));  // exact: a power of two
    *o = fmul_rn((float)d0, r);
  }
  *t = fma_rn(c, *u, *o);
}

// Filtered state after c[k] crossings along each axis.
__host__ __device__ __forceinline__ void fwalker_init(FWalker& f, const RayRec& r, int F, const long long c[3]) {
  f.cx = (float)c[0];
  f.cy = (float)c[1];
  f.cz = (float)c[2];
  fwalker_axis(r.A[0], r.d0[0], F, f.cx, &f.ux, &f.ox, &f.tx);
  fwalker_axis(r.A[1], r.d0[1], F, f.cy, &f.uy, &f.oy, &f.ty);
  fwalker_axis(r.A[2], r.d0[2], F, f.cz, &f.uz, &f.oz, &f.tz);
}

// The axis the estimates single out, or -1 (near-tie: decide exactly).
__host__ __device__ __forceinline__ int fwalker_pick(const FWalker& f) {
  const float tm = fminf(f.tx, fminf(f.ty, f.tz));
  const float thr = fmul_rn(tm, 1.00000095367431640625f);  // 1 + 2^-20
  const bool nx = f.tx <= thr, ny = f.ty <= thr, nz = f.tz <= thr;
  if ((int)nx + (int)ny + (int)nz != 1) return -1;
  return nx ? 0 : (ny ? 1 : 2);
}

// The exact rule of Walker (walker_init / walker_choose) from the crossing
// counts: the axis with the smallest t_k (ties: z, then y, then x), and on a
// tie at t = 1 never an axis without steps left.
__host__ __device__ inline int exact_pick(const RayRec& r, int F, int32_t c0, int32_t c1, int32_t c2) {
  const long long U = 1LL << F;
  const long long dx = r.d0[0] + (long long)c0 * U, dy = r.d0[1] + (long long)c1 * U, dz = r.d0[2] + (long long)c2 * U;
  const long long cxy = dx * r.A[1] - dy * r.A[0];
  const long long cxz = dx * r.A[2] - dz * r.A[0];
  const long long cyz = dy * r.A[2] - dz * r.A[1];
  int axis = (cxy < 0 && cxz < 0) ? 0 : ((cxy >= 0 && cyz < 0) ? 1 : 2);
  const int32_t left = axis == 0 ? r.n[0] - c0 : (axis == 1 ? r.n[1] - c1 : r.n[2] - c2);
  if (left == 0) axis = r.n[2] - c2 > 0 ? 2 : (r.n[1] - c1 > 0 ? 1 : 0);
  return axis;
}

// One crossing along `axis`.
__host__ __device__ __forceinline__ void fwalker_advance(FWalker& f, int axis) {
  if (axis == 0) {
    f.cx += 1.0f;
    f.tx = fma_rn(f.cx, f.ux, f.ox);
  } else if (axis == 1) {
    f.cy += 1.0f;
    f.ty = fma_rn(f.cy, f.uy, f.oy);
  } else {
    f.cz += 1.0f;
    f.tz = fma_rn(f.cz, f.uz, f.oz);
  }
}

// Morton bits of the axes a ray walks in the negative direction.
__host__ __device__ __forceinline__ uint32_t morton_neg(int32_t flags) {
  uint32_t m = 0;
  if ((flags >> kRaySignShift) & 1) m |= 0x1249u;
  if ((flags >> (kRaySignShift + 1)) & 1) m |= 0x2492u;
  if ((flags >> (kRaySignShift + 2)) & 1) m |= 0x4924u;
  return m;
}

// +1 along the axis of `mask` in a sign-normalised Morton index; true when
// the step left the region (the axis wrapped from 31 to 0).
__host__ __device__ __forceinline__ bool morton_advance(uint32_t& mo, uint32_t mask) {
  const bool wrap = (mo & mask) == mask;
  mo = (((mo | ~mask) + 1u) & mask) | (mo & ~mask);
  return wrap;
}


// Number of segments of a walk whose dominant axis takes nmaj steps, cut
// every S dominant-axis steps (the allocation-free entry point's split).
__host__ __device__ __forceinline__ int32_t segment_count(int32_t nmaj, int32_t S) { return nmaj / S + 1; }

// Ray segments of the integrate kernels (Sec. III-B "breaking long rays into
// several segments").  A walk whose dominant axis takes nmaj steps has
// nmaj + 1 dominant-axis "slots": slot 0 is the start voxel, slot k the voxel
// entered by the k-th dominant-axis step; every other voxel belongs to the
// slot of the dominant-axis step before it.  The slots are dealt out to nseg
// segments as evenly as integers allow, q = (nmaj + 1) / nseg each and one
// more to the first (nmaj + 1) % nseg, so all segments of a ray are about
// equally long.  nseg = ceil((nsteps + 1) / target) for a walk of nsteps voxel
// steps, so a segment holds about `target` voxels whatever the ray's
// direction; nseg is raised where needed to keep q <= 65535.
struct SegSplit {
  int32_t nseg;
  int32_t q;  // slots per segment (the first r segments take q + 1)
};

__host__ __device__ __forceinline__ SegSplit ray_segment_split(int32_t nmaj, long long nsteps, int32_t target) {
  const long long slots = (long long)nmaj + 1;
  long long nseg = (nsteps + target) / target;  // ceil((nsteps + 1) / target)
  if (nseg > slots) nseg = slots;
  const long long min_seg = (slots + 65534) / 65535;
  if (nseg < min_seg) nseg = min_seg;
  SegSplit s;
  s.nseg = (int32_t)nseg;
  s.q = (int32_t)(slots / nseg);
  return s;
}

// Dominant-axis steps before segment j starts (K0) and before the segment
// after it starts (K1), for a ray with nmaj dominant-axis steps split into
// nseg segments of q or q + 1 slots.  The segment visits the voxels from the
// one entered by the K0-th dominant-axis step (the start voxel when K0 = 0) up
// to, not including, the one entered by the K1-th; the last segment runs to
// the end of the ray.
__host__ __device__ __forceinline__ void segment_bounds(int32_t nmaj, int32_t nseg, int32_t q, int32_t j, long long* K0,
                                                        long long* K1) {
  const long long r = (long long)nmaj + 1 - (long long)nseg * q;
  *K0 = (long long)j * q + (j < r ? j : r);
  *K1 = *K0 + q + (j < r ? 1 : 0);
}
constexpr int kRaySegShift = 16;  // RayRec flags bits 16..31: q, the ray's dominant-axis slots per segment

// Where segment j of a ray starts and ends, for the filtered walk.
struct SegStart {
  long long c[3];    // crossings taken along each axis before the segment's first voxel
  int32_t v[3];      // the segment's first voxel
  int32_t ve[3];     // the segment's last voxel
  long long visits;  // voxels the segment visits
};

__host__ __device__ inline void segment_start(const RayRec& r, int F, int32_t j, SegStart* s) {
  const int M = (r.flags >> kRayAxisShift) & 3;
  const int32_t q = (int32_t)((uint32_t)r.flags >> kRaySegShift);
  const int32_t nmaj = M == 0 ? r.n[0] : (M == 1 ? r.n[1] : r.n[2]);
  const long long d0M = M == 0 ? r.d0[0] : (M == 1 ? r.d0[1] : r.d0[2]);
  const long long AM = M == 0 ? r.A[0] : (M == 1 ? r.A[1] : r.A[2]);
  long long K0, K1;
  segment_bounds(nmaj, r.nseg, q, j, &K0, &K1);
  const bool last = j == r.nseg - 1;
  long long c1[3];
  long long steps = 0;
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    s->c[k] = K0 == 0 ? 0 : (k == M ? K0 : crossings_before(r.d0[k], r.A[k], d0M, AM, F, K0, k > M, r.n[k], r.inv));
    if (last)
      c1[k] = r.n[k];
    else
      c1[k] = k == M ? K1 - 1 : crossings_before(r.d0[k], r.A[k], d0M, AM, F, K1, k > M, r.n[k], r.inv);
    steps += c1[k] - s->c[k];
    const int32_t sg = ((r.flags >> (kRaySignShift + k)) & 1) ? -1 : 1;
    s->v[k] = r.v0[k] + sg * (int32_t)s->c[k];
    s->ve[k] = r.v0[k] + sg * (int32_t)c1[k];
  }
  s->visits = steps + 1;
}

// ---------------------------------------------------------------------------
// Warp-aggregated reservation: every lane of a full warp calls this together
// with its own count (possibly 0); returns this lane's first index.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long* counter, unsigned int count) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  unsigned int incl = count;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned int t = __shfl_up_sync(full, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned int total = __shfl_sync(full, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total != 0) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(full, base, 31);
  return base + incl - count;
}

// Warp sum of a 32-bit value, added by one lane to two 64-bit counters; full warp.
// ---------------------------------------------------------------------------
// TSDF band of a ray (Sec. II-F) from the double length len of its fixed-point
// difference d (ray_length) and the band half-width tau (fixed-point units):
// with t0 = max(fl(len - tau), 0) and t1 = fl(len + tau),
//     a_k = qo_k + rint(fl(d_k fl(t0 / len))),   b_k likewise with t1,
//     u_k = float(fl(d_k / len)),
// every operation in IEEE double as written.  The device's double divisions
// are slow, so the five quotients go through one reciprocal
// rho = fl(1 / len), and the result is taken when it provably equals the
// one above.  With u = 2^-53 and |e_i| <= u:
//   f' = fl(t rho) = (t / len)(1 + e1)(1 + e2), P' = fl(d_k f') = X (1 + e1)(1 + e2)(1 + e3)
//   with X = d_k t / len, against P = fl(d_k fl(t / len)) = X (1 + e4)(1 + e5):
//   |P' - P| < 5.01 u |X| < 6 ulp(P').  So rint(P) = rint(P') unless a
//   half-integer lies within 6 ulp of P'; P' is taken when none lies within
//   16 ulp (near_half_integer).
//   q' = fl(d_k rho) = (d_k / len)(1 + e1)(1 + e6), q = fl(d_k / len):
//   |q' - q| < 4 ulp(q'), so float(q) = float(q') unless a float rounding
//   boundary (a midpoint between adjacent floats: the 29 bits below float
//   precision equal 2^28) lies within 4 ulp; q' is taken when it lies more
//   than 16 ulp away (near_float_midpoint).
// Otherwise every quotient is formed as written.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ unsigned long long dbits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  std::memcpy(&b, &x, sizeof(b));
  return b;
#endif
}
__host__ __device__ __forceinline__ double dmul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ double ddiv_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __ddiv_rn(a, b);
#else
  return a / b;
#endif
}
__host__ __device__ __forceinline__ double drcp_rn(double a) {
#ifdef __CUDA_ARCH__
  return __drcp_rn(a);
#else
  return 1.0 / a;
#endif
}
__host__ __device__ __forceinline__ long long d2ll_rn(double a) {
#ifdef __CUDA_ARCH__
  return __double2ll_rn(a);
#else
  return std::llrint(a);  // round to nearest even (the default rounding mode)
#endif
}

// A half-integer k + 1/2 within 16 ulp of |x| (|x| < 2^52)?
__host__ __device__ __forceinline__ bool near_half_integer(double x) {
  const unsigned long long b = dbits(x) & 0x7fffffffffffffffULL;
  const int e = (int)(b >> 52) - 1023;  // |x| in [2^e, 2^(e+1))
  const unsigned long long m = b & ((1ULL << 52) - 1);
  if (e >= 52) return false;  // an integer
  if (e >= 0) {
    const int w = 52 - e;  // fraction bits, in units of ulp(x)
    const unsigned long long f = m & ((1ULL << w) - 1), h = 1ULL << (w - 1);
    return (f > h ? f - h : h - f) <= 16;
  }
  if (e == -1) return m <= 16;                   // just above 1/2
  if (e == -2) return m >= (1ULL << 52) - 32;    // just below 1/2
  return false;
}

// A float rounding boundary within 16 ulp of the (normal) double q?
__host__ __device__ __forceinline__ bool near_float_midpoint(double q) {
  const unsigned long long low = dbits(q) & ((1ULL << 29) - 1), mid = 1ULL << 28;
  return (low > mid ? low - mid : mid - low) <= 16;
}

__host__ __device__ inline void tsdf_band(const long long qo[3], const double d[3], double len, double tau,
                                          long long a[3], long long b[3], float u[3]) {
  double t0 = len - tau;
  if (t0 < 0.0) t0 = 0.0;
  const double t1 = len + tau;
  const double rho = drcp_rn(len);
  const double f0 = dmul_rn(t0, rho), f1 = dmul_rn(t1, rho);
  bool exact = false;
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    const double p0 = dmul_rn(d[k], f0), p1 = dmul_rn(d[k], f1), q = dmul_rn(d[k], rho);
    exact = exact || near_half_integer(p0) || near_half_integer(p1) || near_float_midpoint(q);
    a[k] = qo[k] + d2ll_rn(p0);
    b[k] = qo[k] + d2ll_rn(p1);
    u[k] = (float)q;
  }
  if (!exact) return;
  const double g0 = ddiv_rn(t0, len), g1 = ddiv_rn(t1, len);
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    a[k] = qo[k] + d2ll_rn(dmul_rn(d[k], g0));
    b[k] = qo[k] + d2ll_rn(dmul_rn(d[k], g1));
    u[k] = (float)ddiv_rn(d[k], len);
  }
}

// ---------------------------------------------------------------------------
// Float-float (double-word) arithmetic: a value is an unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi) / 2.  The error-free transformations
// are Knuth's TwoSum, Dekker's FastTwoSum and the product's exact error from
// one fused multiply-add (Dekker 1971; Ogita, Rump, Oishi 2005); the
// compound operations follow the double-word algorithms whose relative error
// bounds Joldes, Muller and Popescu (2017) prove: addition <= 3 u^2,
// product <= 5 u^2, product by a float <= 2 u^2 (u = 2^-24).  Every step
// rounds once, written with explicit-rounding intrinsics so that no
// contraction changes it.
// ---------------------------------------------------------------------------

__host__ __device__ __forceinline__ float fadd_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float fsub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float fdiv_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
__host__ __device__ __forceinline__ float fsqrt_rn(float a) {
#ifdef __CUDA_ARCH__
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}

// s + e = a + b exactly.
__host__ __device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = fadd_rn(a, b);
  const float bb = fsub_rn(s, a);
  const float e = fadd_rn(fsub_rn(a, fsub_rn(s, bb)), fsub_rn(b, bb));
  return {s, e};
}
// s + e = a + b exactly, for |a| >= |b| (or a = 0).
__host__ __device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = fadd_rn(a, b);
  return {s, fsub_rn(b, fsub_rn(s, a))};
}
// p + e = a b exactly.
__host__ __device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = fmul_rn(a, b);
  return {p, fma_rn(a, b, -p)};
}
__host__ __device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = two_sum(x.hi, y.hi), t = two_sum(x.lo, y.lo);
  const FF v = fast_two_sum(s.hi, fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, fadd_rn(v.lo, t.lo));
}
__host__ __device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__host__ __device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const FF c = two_prod(x.hi, y.hi);
  const float t = fma_rn(x.lo, y.hi, fma_rn(x.hi, y.lo, fmul_rn(x.lo, y.lo)));
  return fast_two_sum(c.hi, fadd_rn(c.lo, t));
}
__host__ __device__ __forceinline__ FF ff_mul_f(FF x, float y) {
  const FF c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, fma_rn(x.lo, y, c.lo));
}
// sqrt(x) for x > 0: the float root r and one Newton correction
// (x - r^2) / (2 r), with x - r^2 formed from the exact square of r.
// Relative error below 4 u^2 for x exact (the truncated Newton term is
// under u^2 / 2, the residual's two roundings and the quotient's add 3 u^2).
__host__ __device__ __forceinline__ FF ff_sqrt(FF x) {
  const float r = fsqrt_rn(x.hi);
  const FF p = two_prod(r, r);
  const float res = fadd_rn(fsub_rn(fsub_rn(x.hi, p.hi), p.lo), x.lo);  // x.hi - p.hi exact (Sterbenz)
  return fast_two_sum(r, fdiv_rn(res, fadd_rn(r, r)));
}
// 1 / x for x > 0: the float reciprocal r and one Newton correction r (1 - x r).
// Relative error below 6 u^2 (the truncated Newton term under u^2, the
// residual's roundings and x.lo r about 4 u^2, the correction's product u^2).
__host__ __device__ __forceinline__ FF ff_rcp(FF x) {
  const float r = fdiv_rn(1.0f, x.hi);
  const FF p = two_prod(x.hi, r);
  const float e = fsub_rn(fsub_rn(fsub_rn(1.0f, p.hi), p.lo), fmul_rn(x.lo, r));  // 1 - p.hi exact (Sterbenz)
  return fast_two_sum(r, fmul_rn(r, e));
}
// A double as float-float (hi = float(v), lo = float(v - hi)): within
// 2^-48 |v| of v; an infinite or huge v keeps lo = 0.
__host__ __device__ __forceinline__ FF ff_of_double(double v) {
  const float hi = (float)v;
  if (!(hi - hi == 0.0f)) return {hi, 0.0f};
  return {hi, (float)(v - (double)hi)};
}

// rint(x) of a float-float x with |x| < 2^25, as an integer, when every value
// within e of x rounds to it (no half-integer in [x - e, x + e]); else false.
__host__ __device__ __forceinline__ bool ff_rint(FF x, float e, long long* out) {
  const float n = rintf(x.hi);                         // an integer within 1/2 of x.hi
  const float f = fadd_rn(fsub_rn(x.hi, n), x.lo);     // x - n, one rounding (|f| <= 1.5)
  const float m = e + 1e-6f;                           // covers the rounding of f
  long long k = (long long)n;
  if (fabsf(f) < 0.5f - m) {
  } else if (f > 0.5f + m && f < 1.5f - m) {
    k += 1;
  } else if (f < -0.5f - m && f > -1.5f + m) {
    k -= 1;
  } else {
    return false;
  }
  *out = k;
  return true;
}

// float(q) of a float-float q when every value within e of q rounds to the
// same float (no midpoint between adjacent floats in [q - e, q + e]); else false.
__host__ __device__ __forceinline__ bool ff_to_float(FF q, float e, float* out) {
  if (q.hi == 0.0f) {
    if (q.lo != 0.0f || e > 0.0f) return false;
    *out = 0.0f;
    return true;
  }
  // the nearest midpoints lie half a gap to either neighbour of |hi|; the
  // gaps are exact float differences of adjacent floats
  const float a = fabsf(q.hi);
  uint32_t ab;
  std::memcpy(&ab, &a, sizeof(ab));
  const uint32_t up_bits = ab + 1u, down_bits = ab - 1u;
  float up, down;
  std::memcpy(&up, &up_bits, sizeof(up));
  std::memcpy(&down, &down_bits, sizeof(down));
  const float half_gap = 0.5f * fminf(up - a, a - down);
  if (!(fabsf(q.lo) + e < half_gap)) return false;
  *out = q.hi;
  return true;
}
// ---------------------------------------------------------------------------
// The TSDF band of tsdf_band (with its range test len > rmin, len <= rmax on
// the double length of ray_length) settled in float-float arithmetic, for
// rays with |d_k| < 2^24 (every d_k exact as a float).  The double
// evaluation's roundings stay below u^2 / 16 of each quantity (u = 2^-24);
// the float-float one's, from the bounds above (relative errors add, to
// first order): S = sum d_k^2 to 6.1 u^2 (all terms positive), len =
// sqrt(S) to 7.1 u^2, 1 / len to 13.1 u^2, t = len -+ tau (tau within u^2
// of the double) to 3 u^2 |t| + 8.1 u^2 (len + tau), g = t rho to that over
// len plus 18.1 u^2 g, and the products by d_k to 2 u^2.  With
// (len + tau) / len = g1, the end points d_k g differ from the double's by
// less than 32 u^2 |d_k| (1 + g0 + g1), d_k / len by less than 16 u^2
// |d_k / len|, len by less than 7.2 u^2 len, t0 by less than 12 u^2
// (len + tau).  Each rounding decision (range test, t0 > 0, rint, float) is
// taken only when the float-float value is farther than 2^-40 = 256 u^2 of
// that scale from where the decision changes; otherwise the function returns
// false and the caller evaluates in double.  The GB300's FP64 pipe runs a
// warp instruction in 64 cycles of a scheduler, the FP32 pipe in one or two.
// ---------------------------------------------------------------------------

// len_out (optional): the ray length's high part.
__host__ __device__ inline bool tsdf_band_ff(const long long qo[3], const long long qe[3], const BandConsts& c,
                                             bool* in_range, long long a[3], long long b[3], float u[3],
                                             float* len_out = nullptr) {
  constexpr float kMargin = 9.094947e-13f;  // 2^-40
  float d[3];
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    const long long dk = qe[k] - qo[k];
    if (dk <= -(1LL << 24) || dk >= (1LL << 24)) return false;
    d[k] = (float)dk;
  }
  const FF S = ff_add(ff_add(two_prod(d[0], d[0]), two_prod(d[1], d[1])), two_prod(d[2], d[2]));
  if (!(S.hi > 0.0f)) return false;
  const FF len = ff_sqrt(S);
  if (len_out) *len_out = len.hi;
  // range test
  const float tol_len = kMargin * len.hi;
  const FF over_min = ff_add(len, ff_neg(c.rmin)), over_max = ff_add(len, ff_neg(c.rmax));
  if (!(fabsf(over_min.hi) > tol_len + kMargin * fabsf(c.rmin.hi))) return false;
  if (!(fabsf(over_max.hi) > tol_len + kMargin * fabsf(c.rmax.hi))) return false;
  *in_range = over_min.hi > 0.0f && over_max.hi < 0.0f;
  if (!*in_range) return true;
  // band ends as fractions of the ray: t0 = max(len - tau, 0), t1 = len + tau
  const float tol_t = kMargin * (len.hi + c.tau.hi);
  const FF t0 = ff_add(len, ff_neg(c.tau));
  if (!(fabsf(t0.hi) > tol_t)) return false;
  const bool t0_pos = t0.hi > 0.0f;
  const FF t1 = ff_add(len, c.tau);
  const FF rho = ff_rcp(len);
  const FF g0 = t0_pos ? ff_mul(t0, rho) : FF{0.0f, 0.0f};
  const FF g1 = ff_mul(t1, rho);
  const float gsum = 1.0f + g0.hi + g1.hi;
OHM_UNROLL
  for (int k = 0; k < 3; ++k) {
    const float tol_p = kMargin * fabsf(d[k]) * gsum;
    long long pa, pb;
    if (!ff_rint(ff_mul_f(g0, d[k]), tol_p, &pa)) return false;
    if (!ff_rint(ff_mul_f(g1, d[k]), tol_p, &pb)) return false;
    const FF q = ff_mul_f(rho, d[k]);
    if (!ff_to_float(q, kMargin * fabsf(q.hi), &u[k])) return false;
    a[k] = qo[k] + pa;
    b[k] = qo[k] + pb;
  }
  return true;
}

__device__ __forceinline__ void warp_add(unsigned long long* counter, unsigned long long* counter2, unsigned int value) {
  unsigned int total = __reduce_add_sync(0xffffffffu, value);
  if ((threadIdx.x & 31) == 0 && total != 0) {
    atomicAdd(counter, (unsigned long long)total);
    atomicAdd(counter2, (unsigned long long)total);
  }
}

}  // namespace ohm
