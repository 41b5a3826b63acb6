// Per-item device functions of the ray-integration kernels (Sec. III-B,
// III-C of arxiv 2206.06079, re-designed for sm_103a).  The single-map
// kernels (ohm_integrate.cu) and the multi-map batch kernels (ohm_batch.cu)
// are thin loops around these.
#pragma once

#include <climits>

#include "ohm_host.h"

namespace ohm {

constexpr int kBlock = 256;
// regions whose first hash probes one thread of the prepare walk loads together
#ifndef OHM_REGION_BATCH
#define OHM_REGION_BATCH 4
#endif
constexpr int kRegionBatch = OHM_REGION_BATCH;

__device__ __forceinline__ bool latched(const DeviceMap& m) { return *(volatile int32_t*)m.status != 0; }

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation may be scheduled while the kernel before
// it in the stream is still draining.  chain_enter() first waits until that
// kernel has completed and its writes are visible (griddepcontrol.wait; a
// no-op for an ordinary launch), then allows the next kernel of the stream to
// be scheduled.  Called first thing by every kernel of an integrate chain
// (single map or batched), so each body still runs strictly after its
// predecessor; only the launch latency and the block scheduling overlap.
__device__ __forceinline__ void chain_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host side: launch one kernel of a chain with programmatic stream
// serialisation: its blocks may be scheduled while the previous kernel of the
// stream drains, and wait in chain_enter() until that kernel has completed.
// Where the attribute is refused the kernel is launched the ordinary way.
template <typename... K, typename... A>
inline void launch_chained(void (*kernel)(K...), unsigned grid, cudaStream_t stream, A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, kernel, args...) != cudaSuccess) {
    (void)cudaGetLastError();
    cfg.numAttrs = 0;
    (void)cudaLaunchKernelEx(&cfg, kernel, args...);
  }
}

// Log-odds of a stored occupancy word for an update: an unknown voxel (NaN)
// starts from the prior 0, and a value stored below l_min stands for l_min
// (the miss walk may leave it there, see walk_segment_fast).
__device__ __forceinline__ float logodds_value(float s, float l_min) { return s != s ? 0.0f : fmaxf(s, l_min); }

// Log-odds a stored occupancy word reports: NaN stays unknown, a value stored
// below l_min reads as l_min.
__device__ __forceinline__ float logodds_read(float s, float l_min) { return s < l_min ? l_min : s; }

// Quantise a ray, returns false when it is skipped (non-finite coordinate or
// a point beyond the fixed-point range).
__device__ __forceinline__ bool quantise_ray(const DeviceMap& m, const float o[3], const float e[3], long long qo[3],
                                             long long qe[3]) {
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ok = ok && isfinite(o[k]) && isfinite(e[k]);
    ok = ok && quantise(o[k], m.origin[k], m.scale, &qo[k]);
    ok = ok && quantise(e[k], m.origin[k], m.scale, &qe[k]);
  }
  return ok;
}

// |qe - qo| in fixed-point units, double, fixed evaluation order.
__device__ __forceinline__ double ray_length(const long long qo[3], const long long qe[3], double d[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) d[k] = (double)(qe[k] - qo[k]);
  double l2 = __dmul_rn(d[0], d[0]);
  l2 = __dadd_rn(l2, __dmul_rn(d[1], d[1]));
  l2 = __dadd_rn(l2, __dmul_rn(d[2], d[2]));
  return __dsqrt_rn(l2);
}

__device__ __forceinline__ bool in_extent(const long long q[3], int F) {
  const long long lim = 1LL << 24;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    long long v = q[k] >> F;
    ok = ok && v > -lim && v < lim;
  }
  return ok;
}

__device__ __forceinline__ void load_ray(const CallArgs& a, long long i, float o[3], float e[3], uint8_t* flag) {
  const long long oi = a.n_origins == 1 ? 0 : i;
  o[0] = a.origins[3 * oi + 0];
  o[1] = a.origins[3 * oi + 1];
  o[2] = a.origins[3 * oi + 2];
  e[0] = a.endpoints[3 * i + 0];
  e[1] = a.endpoints[3 * i + 1];
  e[2] = a.endpoints[3 * i + 2];
  *flag = a.flags ? a.flags[i] : 0;
}

// Walk the regions (32^3 voxel blocks) a ray passes through, inserting each
// into the hash table.  The same exact walk at region resolution visits
// exactly the regions of the voxels the voxel walk visits: region boundaries
// are voxel boundaries, crossed at the same t in the same tie order.
//
// The lookups of successive regions do not depend on one another, and a
// 131,072-ray scan runs as one wave, so the kernel lasts as long as its
// longest chain of dependent loads (a ray to the range limit crosses dozens
// of regions).  So the walk goes kRegionBatch regions ahead and loads their
// first probe entries together.  A first entry holding the key with a slot
// is the common case (the region exists): it is stamped as insert_region
// would.  Every other case goes through insert_region.  A ray visits a
// region once, so a batch holds distinct keys.
//
// Returns the slot of the last region (the one holding the end point) where
// this thread learnt it, else -1 (see insert_region).
__device__ __forceinline__ int32_t insert_ray_regions(const DeviceMap& m, const long long a[3], const long long b[3]) {
  Walker w;
  walker_init(w, a, b, m.frac_bits + kRegionShift, 0, 0);
  const int32_t seq = m.calls->seq;
  int32_t last = -1;
  bool more = true;
  while (more) {
    long long key[kRegionBatch];
    uint32_t h[kRegionBatch];
    unsigned n = 0;
#pragma unroll
    for (int j = 0; j < kRegionBatch; ++j) {
      key[j] = kEmptyKey;
      h[j] = 0;
      if (more) {
        key[j] = pack_region(w.vx, w.vy, w.vz);
        h[j] = hash_key(key[j]) & m.hmask;
        n = j + 1;
        if (w.total > 0) {
          int32_t c, s;
          walker_step(w, walker_choose(w), &c, &s);
        } else {
          more = false;
        }
      }
    }
    longlong2 e[kRegionBatch];
#pragma unroll
    for (int j = 0; j < kRegionBatch; ++j)
      if (j < (int)n) e[j] = m.htab[h[j]];
#pragma unroll
    for (int j = 0; j < kRegionBatch; ++j) {
      if (j < (int)n) {
        if (e[j].x == key[j] && e[j].y >= 0) {
          m.stamp[e[j].y] = seq;
          last = (int32_t)e[j].y;
        } else {
          const unsigned long long k = (unsigned long long)key[j];
          const int32_t mask = (1 << 21) - 1;
          // sign-extend the 21-bit fields of the packed key
          const int rx = (int32_t)((uint32_t)((k >> 42) & mask) << 11) >> 11;
          const int ry = (int32_t)((uint32_t)((k >> 21) & mask) << 11) >> 11;
          const int rz = (int32_t)((uint32_t)(k & mask) << 11) >> 11;
          last = insert_region(m, rx, ry, rz);
        }
      }
    }
  }
  return last;
}

// Give region `slot` an NDT block if it has none: one thread wins the claim
// (-1 -> -2) and takes a block from the pool.
__device__ __forceinline__ void ndt_claim(const DeviceMap& m, int32_t slot) {
  if (*(volatile int32_t*)&m.ndt_slot[slot] != -1) return;
  if (atomicCAS(&m.ndt_slot[slot], -1, -2) == -1) {
    const int32_t id = alloc_ndt_block(m);
    if (id >= 0) {
      m.ndt_born[slot] = m.calls->seq;
      m.ndt_slot[slot] = id;
    } else {
      atomicOr(m.status, kStatusCapacity);
    }
  }
}

__device__ __forceinline__ long long voxel_offset(int32_t slot, uint32_t mo) {
  return (long long)slot * kRegionVoxels + mo;
}

__device__ __forceinline__ int32_t region_slot_of(const DeviceMap& m, int32_t vx, int32_t vy, int32_t vz) {
  return find_region(m, pack_region(vx >> kRegionShift, vy >> kRegionShift, vz >> kRegionShift));
}

__device__ __forceinline__ uint32_t local_morton(int32_t vx, int32_t vy, int32_t vz) { return region_morton(vx, vy, vz); }

// Sample clearing (Sec. II-D): a miss that took voxel `off` from at or above
// the threshold (or from unknown) to below it clears the voxel's NDT samples.
// Misses only lower a voxel within the miss phase, so exactly one successful
// CAS per voxel and call can make this crossing.
__device__ __forceinline__ void after_miss(const DeviceMap& m, long long off, unsigned int old_bits, unsigned int new_bits) {
  const float lo = __uint_as_float(old_bits), ln = __uint_as_float(new_bits);
  if (!(ln < m.ndt_clear) || (lo < m.ndt_clear)) return;  // NaN (unknown) compares false: counts as above
  if (!(m.layers & kLayerNdt)) return;
  const int32_t ns = m.ndt_slot[off >> (3 * kRegionShift)];
  if (ns < 0) return;
  long long* base = m.ndt + (long long)ns * 10 * kRegionVoxels + (off & (kRegionVoxels - 1));
#pragma unroll
  for (int k = 0; k < 10; ++k) base[(long long)k * kRegionVoxels] = 0;
}

// Retry a clamped log-odds CAS whose first attempt found `cur` instead of
// the value it expected (see logodds_update_n).
static __device__ __noinline__ void logodds_retry(const DeviceMap& m, unsigned int* u, unsigned int cur, float delta) {
  for (int it = 0; it < 256; ++it) {
    const float l0 = logodds_value(__uint_as_float(cur), m.l_min);
    const unsigned int nb = __float_as_uint(fminf(fmaxf(__fadd_rn(l0, delta), m.l_min), m.l_max));
    if (nb == cur) return;
    const unsigned int prev = atomicCAS(u, cur, nb);
    if (prev == cur) {
      if (delta < 0.f) after_miss(m, u - reinterpret_cast<unsigned int*>(m.occ), cur, nb);
      return;
    }
    cur = prev;
  }
  atomicOr(m.status, kStatusCasLimit);
}

// Clamped compare-and-swap miss of one voxel whose word was read as `old`
// (with NDT sample clearing: clears its samples if the miss crosses the
// threshold).
__device__ __forceinline__ void miss_cas(const DeviceMap& m, unsigned int* u, unsigned int old, unsigned int& ops) {
  const float l0 = logodds_value(__uint_as_float(old), m.l_min);
  const unsigned int nb = __float_as_uint(fminf(fmaxf(__fadd_rn(l0, m.miss), m.l_min), m.l_max));
  if (nb == old) return;
  ++ops;
  const unsigned int prev = atomicCAS(u, old, nb);
  if (prev != old)
    logodds_retry(m, u, prev, m.miss);
  else
    after_miss(m, u - reinterpret_cast<unsigned int*>(m.occ), old, nb);
}

// Launch shapes (measured on GB300, tunnel scans of 131,072 rays):
//  OHM_WALK_BATCH          voxels in flight per thread in the miss walk
//  OHM_WALK_MIN_BLOCKS     blocks of 256 threads per SM the walk is compiled for
//                          (5: 48 registers; 4 and 6 were slower)
//  OHM_WALK_OVERSUBSCRIBE  the walk's grid-stride launch covers this many
//                          times the resident blocks
//  OHM_PREPARE_MIN_BLOCKS  blocks per SM of the prepare kernels (4: a
//                          131,072-ray scan fits one wave on 152 SMs)
#ifndef OHM_WALK_BATCH
#define OHM_WALK_BATCH 4
#endif
#ifndef OHM_WALK_MIN_BLOCKS
#define OHM_WALK_MIN_BLOCKS 5
#endif
constexpr int kWalkBatch = OHM_WALK_BATCH;
#ifndef OHM_WALK_OVERSUBSCRIBE
#define OHM_WALK_OVERSUBSCRIBE 8
#endif
#ifndef OHM_PREPARE_MIN_BLOCKS
#define OHM_PREPARE_MIN_BLOCKS 4
#endif

// Snapshot of the pool counters at the start of a call (the rollback point).
__device__ __forceinline__ void begin_call(const DeviceMap& m, const CallArgs& a) {
  const long long n = a.n;
  m.calls->region_start = *m.region_count;
  m.calls->ndt_start = *m.ndt_count;
  m.calls->free_used_start = m.free_info[1];
  m.calls->ndt_free_used_start = m.free_info[3];
  m.calls->seq += 1;
  m.calls->segments = 0;
  m.calls->visits = 0;
  m.calls->touched = 0;
  m.calls->mean_touched = 0;
  m.calls->restores = 0;
  m.calls->atomics = 0;
  m.calls->ndt_pending = 0;
  m.calls->rays = (unsigned long long)n;
  // a shared sensor origin is quantised once for the whole call
  bool ok = false;
  if (a.n_origins == 1 && n > 0) {
    ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float o = a.origins[k];
      long long q = 0;
      ok = ok && isfinite(o) && quantise(o, m.origin[k], m.scale, &q);
      m.calls->origin_q[k] = q;
    }
  }
  m.calls->origin_ok = ok ? 1 : 0;
}

// quantise_ray for the rays of the current call: a shared origin comes
// quantised from begin_call.
__device__ __forceinline__ bool quantise_call_ray(const DeviceMap& m, const CallArgs& a, const float o[3],
                                                  const float e[3], long long qo[3], long long qe[3]) {
  if (a.n_origins != 1) return quantise_ray(m, o, e, qo, qe);
  bool ok = m.calls->origin_ok != 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    qo[k] = m.calls->origin_q[k];
    ok = ok && isfinite(e[k]) && quantise(e[k], m.origin[k], m.scale, &qe[k]);
  }
  return ok;
}

// Segment table entries (ray i, segment j) of the rays of a full warp, in
// (j, lane) order: the first segments of the warp's 32 rays, then their second
// segments, and so on.  Neighbouring rays' j-th segments lie close together in
// space, so the walk's warps (which take consecutive entries) touch compact
// patches of the map; the stores of each j are coalesced.  Every lane calls
// this together with its ray's segment count (0 for none).
__device__ __forceinline__ void write_segments(const DeviceMap& m, long long i, unsigned int nseg) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned int total = __reduce_add_sync(full, nseg);
  unsigned long long base = 0;
  if (lane == 0 && total) base = atomicAdd(&m.calls->segments, (unsigned long long)total);
  base = __shfl_sync(full, base, 0);
  if (total == 0) return;
  if (base + total > (unsigned long long)m.max_segs) {
    if (lane == 0) atomicOr(m.status, kStatusScratch);
    return;
  }
  const unsigned int rounds = __reduce_max_sync(full, nseg);
  const unsigned int below = (1u << lane) - 1u;
  unsigned long long pos = base;
  for (unsigned int j = 0; j < rounds; ++j) {
    const unsigned int has = __ballot_sync(full, nseg > j);
    if (nseg > j) m.segs[pos + __popc(has & below)] = make_int2((int)i, (int)j);
    pos += __popc(has);
  }
}

// Per ray: fixed-point quantisation, max-range truncation, region walk with
// hash insertion, segment table.  Every lane of the warp must call this
// together with the same map (the segment reservation is warp-aggregated);
// lanes without a ray pass active = false.
__device__ __forceinline__ void prepare_occ_ray(const DeviceMap& m, const CallArgs& args, long long i, bool active) {
  active = active && !latched(m);
  const int F = m.frac_bits;
  unsigned int nseg = 0, nvisit = 0;
  bool ndt_listed = false;
  RayRec r;
  r.flags = 0;
  r.nseg = 0;
  r.inv = 0;
  if (active) {
    float o[3], e[3];
    uint8_t flag;
    load_ray(args, i, o, e, &flag);
    long long qo[3], qe[3];
    bool ok = quantise_call_ray(m, args, o, e, qo, qe);
    bool sample = (flag & kFlagNoReturn) == 0;
    if (ok) {
      // Truncation test len > rmax_q with len the double length: settled by
      // the exact integer |b - a|^2 unless it lies in a band around rmax_q^2
      // (or an axis difference is too large for it), where the double
      // evaluation decides.
      bool in_range = false;
      const long long dx = qe[0] - qo[0], dy = qe[1] - qo[1], dz = qe[2] - qo[2];
      const long long lim = 1LL << 30;
      if (dx > -lim && dx < lim && dy > -lim && dy < lim && dz > -lim && dz < lim) {
        const unsigned long long l2 = (unsigned long long)(dx * dx) + (unsigned long long)(dy * dy) +
                                      (unsigned long long)(dz * dz);
        in_range = l2 <= m.rmax_in2;
      }
      if (!in_range) {
        double d[3];
        const double len = ray_length(qo, qe, d);
        if (len > m.rmax_q) {
          const double ratio = __ddiv_rn(m.rmax_q, len);
#pragma unroll
          for (int k = 0; k < 3; ++k) qe[k] = qo[k] + __double2ll_rn(__dmul_rn(d[k], ratio));
          sample = false;
        }
      }
      ok = in_extent(qo, F) && in_extent(qe, F);
    }
    if (ok) {
      int32_t nmaj;
      const int M = dominant_axis(qo, qe, F, &nmaj);
      long long l1 = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        long long dv = (qe[k] >> F) - (qo[k] >> F);
        l1 += dv < 0 ? -dv : dv;
      }
      const SegSplit sp = ray_segment_split(nmaj, l1, m.seg_steps);
      nseg = (unsigned int)sp.nseg;
      const long long am = sel3(M, qe[0] - qo[0], qe[1] - qo[1], qe[2] - qo[2]);
      r.inv = reciprocal64((unsigned long long)(am < 0 ? -am : am));
      r.flags = kRayValid | (sample ? kRaySample : 0) | (M << kRayAxisShift) | (int32_t)((uint32_t)sp.q << kRaySegShift);
      ray_constants(qo, qe, F, &r);
      r.nseg = (int32_t)nseg;
      if (m.layers & kLayerDecay) {
        DecayRec dr;
#pragma unroll
        for (int k = 0; k < 3; ++k) dr.inv[k] = reciprocal64((unsigned long long)r.A[k]);
        dr.length = walk_length_units(qo, qe, m.voxel_size, F);
        m.decay_rays[i] = dr;
      }
      nvisit = (unsigned int)(1 + l1);
      const int32_t last = insert_ray_regions(m, qo, qe);
      // NDT-OM: the sample's region (the ray's last) gets its NDT block here
      // when this thread learnt the region's slot; otherwise the ray is
      // listed for the NDT pass after this kernel
      if (sample && (m.layers & kLayerNdt)) {
        if (last >= 0)
          ndt_claim(m, last);
        else
          ndt_listed = true;
      }
    }
    m.rays[i] = r;
  }
  if (m.layers & kLayerNdt) {
    const unsigned full = 0xffffffffu;
    const unsigned listed = __ballot_sync(full, ndt_listed);
    if (listed) {
      const int lane = threadIdx.x & 31;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(&m.calls->ndt_pending, (unsigned long long)__popc(listed));
      base = __shfl_sync(full, base, 0);
      if (ndt_listed) m.ndt_pending[base + __popc(listed & ((1u << lane) - 1u))] = (int32_t)i;
    }
  }
  write_segments(m, i, nseg);
  warp_add(&m.calls->visits, &m.calls->total_visits, nvisit);
}

// Per sample: give the sample's region an NDT layer.
__device__ __forceinline__ void ndt_alloc_ray(const DeviceMap& m, long long i) {
  const RayRec r = m.rays[i];
  if (!(r.flags & kRaySample)) return;
  const int32_t vx = r.v0[0] + (((r.flags >> kRaySignShift) & 1) ? -r.n[0] : r.n[0]);
  const int32_t vy = r.v0[1] + (((r.flags >> (kRaySignShift + 1)) & 1) ? -r.n[1] : r.n[1]);
  const int32_t vz = r.v0[2] + (((r.flags >> (kRaySignShift + 2)) & 1) ? -r.n[2] : r.n[2]);
  const int32_t slot = region_slot_of(m, vx, vy, vz);
  if (slot < 0) {
    atomicOr(m.status, kStatusMissing);
    return;
  }
  ndt_claim(m, slot);
}

// Miss phase (Sec. III-C phase one) for one segment: every voxel a ray passes
// through, except the voxel holding its sample, takes one miss.  Segment j of
// a ray covers the voxels entered after j*S and before (j+1)*S steps of the
// ray's dominant axis (the last segment runs to the end).
//
// The walk itself is cheap integer arithmetic; the cost is the read-modify-
// write of each voxel in global memory.  So the thread walks kWalkBatch voxels
// ahead, then issues all their loads at once, then all their CASes at once,
// keeping that many memory operations in flight instead of one.
// Decay layer: distance along the ray, in 2^-20 m, at which the walk crosses
// a boundary of an axis that has taken `done` steps.  The crossing happens at
// t = dist / A with dist = d0 + done U; t is taken as floor(2^32 dist / A) /
// 2^32 (exact, by the reciprocal inv = reciprocal64(A); 2^32 dist < 2^62) and
// the distance as rint(t L).  Monotone in t, so per-voxel differences are
// never negative, and they add up to L over the ray.
__device__ __forceinline__ unsigned long long decay_position(long long dist, int32_t A, unsigned long long inv,
                                                             unsigned long long length) {
  const unsigned long long tq = div_by_inv((unsigned long long)dist << 32, (unsigned long long)A, inv);
  const unsigned long long lo = tq * length, hi = __umul64hi(tq, length);
  const unsigned long long lo2 = lo + (1ULL << 31);
  return ((hi + (lo2 < lo ? 1ULL : 0ULL)) << 32) | (lo2 >> 32);
}

template <bool kOcc, bool kCounts, bool kDecay>
__device__ __forceinline__ void walk_segment(const DeviceMap& m, long long si, unsigned int& cas) {
  const int F = m.frac_bits;
  const int2 sg = m.segs[si];
  const RayRec r = m.rays[sg.x];
  const int M = (r.flags >> kRayAxisShift) & 3;
  const bool last = sg.y == r.nseg - 1;
  const bool sample = (r.flags & kRaySample) != 0;
  long long K0, K1;
  segment_bounds(M == 0 ? r.n[0] : (M == 1 ? r.n[1] : r.n[2]), r.nseg, (int32_t)((uint32_t)r.flags >> kRaySegShift),
                 sg.y, &K0, &K1);
  Walker w;
  walker_init_rec(w, r, F, M, K0);
  int32_t mrem = last ? INT_MAX : (int32_t)(K1 - K0 - 1);
  int32_t slot = region_slot_of(m, w.vx, w.vy, w.vz);
  if (slot < 0) {
    atomicOr(m.status, kStatusMissing);
    return;
  }
  uint32_t mo = local_morton(w.vx, w.vy, w.vz);
  // decay layer: position (2^-20 m along the ray) where the walk entered the current voxel
  DecayRec dr;
  unsigned long long pos_in = 0;
  if (kDecay) {
    dr = m.decay_rays[sg.x];
    if (K0 > 0) {
      const int32_t d0M = M == 0 ? r.d0[0] : (M == 1 ? r.d0[1] : r.d0[2]);
      const int32_t AM = M == 0 ? r.A[0] : (M == 1 ? r.A[1] : r.A[2]);
      pos_in = decay_position((long long)d0M + ((K0 - 1) << F), AM, r.inv, dr.length);
    }
  }
  bool done = false;
  while (!done) {
    uint32_t off[kWalkBatch];  // voxel offsets (< 2^31: at most 2^16 regions of 2^15 voxels)
    uint32_t todo = 0;         // bit j: off[j] takes a miss
#pragma unroll
    for (int j = 0; j < kWalkBatch; ++j) {
      off[j] = 0;
      if (done) continue;
      // the current voxel takes a miss unless it holds this ray's sample
      off[j] = (uint32_t)voxel_offset(slot, mo);
      if (!(sample && w.total == 0)) {
        todo |= 1u << j;
        if (kCounts) atomicAdd(m.counts + off[j], 1ULL);
      }
      if (w.total == 0) {
        if (kDecay && dr.length != pos_in) atomicAdd(m.decay + off[j], dr.length - pos_in);
        done = true;
        continue;
      }
      const int axis = walker_choose(w);
      if (kDecay) {
        const int32_t d0a = axis == 0 ? r.d0[0] : (axis == 1 ? r.d0[1] : r.d0[2]);
        const int32_t Aa = axis == 0 ? r.A[0] : (axis == 1 ? r.A[1] : r.A[2]);
        const int32_t taken = axis == 0 ? r.n[0] - w.nx : (axis == 1 ? r.n[1] - w.ny : r.n[2] - w.nz);
        const unsigned long long inv = axis == 0 ? dr.inv[0] : (axis == 1 ? dr.inv[1] : dr.inv[2]);
        const unsigned long long pos_out = decay_position((long long)d0a + ((long long)taken << F), Aa, inv, dr.length);
        const unsigned long long d = pos_out - pos_in;
        if (d) atomicAdd(m.decay + off[j], d);
        pos_in = pos_out;
      }
      if (axis == M) {
        if (mrem == 0) {
          done = true;
          continue;
        }
        --mrem;
      }
      int32_t c, s;
      walker_step(w, axis, &c, &s);
      mo = morton_step(mo, morton_mask(axis), s);
      if ((c & ((1 << kRegionShift) - 1)) == (s > 0 ? 0 : (1 << kRegionShift) - 1)) {
        slot = region_slot_of(m, w.vx, w.vy, w.vz);
        if (slot < 0) {
          atomicOr(m.status, kStatusMissing);
          done = true;
        }
      }
    }
    if (kOcc) {
      unsigned int* base = reinterpret_cast<unsigned int*>(m.occ);
      unsigned int old[kWalkBatch];
#pragma unroll
      for (int j = 0; j < kWalkBatch; ++j) old[j] = (todo >> j) & 1u ? base[off[j]] : 0u;
#pragma unroll
      for (int j = 0; j < kWalkBatch; ++j)
        if ((todo >> j) & 1u) miss_cas(m, base + off[j], old[j], cas);
    }
  }
}

// Pool slots of two regions (or -1), their first probes issued together.
__device__ __forceinline__ void find_region2(const DeviceMap& m, long long k1, long long k2, int32_t* s1, int32_t* s2) {
  const longlong2 e1 = m.htab[hash_key(k1) & m.hmask];
  const longlong2 e2 = m.htab[hash_key(k2) & m.hmask];
  *s1 = e1.x == k1 ? (int32_t)e1.y : (e1.x == kEmptyKey ? -1 : find_region(m, k1));
  *s2 = e2.x == k2 ? (int32_t)e2.y : (e2.x == kEmptyKey ? -1 : find_region(m, k2));
}

// Out of line: the rare paths of the filtered walk (a near-tie decided
// exactly from the ray record, a third region inside one segment), so that
// neither the record nor the hash loop takes registers in the walk.
static __device__ __noinline__ int exact_pick_rec(const RayRec* rp, int F, int32_t c0, int32_t c1, int32_t c2) {
  return exact_pick(*rp, F, c0, c1, c2);
}
static __device__ __noinline__ int32_t find_region_rare(const DeviceMap& m, long long key) { return find_region(m, key); }

// Voxels per batch of the filtered walk: pipelined (two batches in flight,
// the single-map walk kernel) and plain (one batch stepped, loaded and
// applied at a time, the multi-map batch kernel, whose run-time choice of
// layers leaves fewer registers for the pipeline).
#ifndef OHM_FAST_BATCH
#define OHM_FAST_BATCH 4
#endif
#ifndef OHM_FAST_BATCH_PLAIN
#define OHM_FAST_BATCH_PLAIN 8
#endif
#ifndef OHM_FAST_MIN_BLOCKS
#define OHM_FAST_MIN_BLOCKS 4
#endif
constexpr int kFastBatch = OHM_FAST_BATCH;
constexpr int kFastBatchPlain = OHM_FAST_BATCH_PLAIN;
template <bool kPipe>
constexpr int kFastBatchOf = kPipe ? kFastBatch : kFastBatchPlain;


// Miss phase (Sec. III-C phase one) of one segment with the filtered walk
// (FWalker): every voxel the ray passes through, except the voxel holding its
// sample, takes one miss.  The segment's first and last regions are looked up
// together before the walk; a region boundary inside the segment costs a
// comparison with the last region's key and only a hash lookup when the
// segment passes through a third region.
//
// Occupancy update.  With kCas false (the miss increment is negative and the
// map does not clear NDT samples) a miss is a fire-and-forget float atomic add
// of the increment, and the lower clamp is applied where log-odds are read:
// a voxel's log-odds is max(stored, l_min).  Within a call every miss of a
// voxel adds the same delta < 0, so whatever the order the adds produce the
// floats l, fl(l + delta), fl(fl(l + delta) + delta), ...  While they stay at or
// above l_min these are the values of the clamped one-at-a-time updates
// l <- min(max(l + delta, l_min), l_max) (Eq. 2 with the clamp of Sec. II-B);
// once one drops below l_min the clamped sequence stays at l_min (fl(l_min +
// delta) <= l_min), which is what max(stored, l_min) reads, however far below
// the later adds take the stored value.  So the result is bit for bit that of
// the sequential updates.  A voxel already at or below l_min takes no add (a
// miss leaves it at l_min), and an unknown voxel (NaN) is first set to
// fl(0 + delta) by compare-and-swap; a thread that loses that race adds its
// miss to the value it found.  No value comes near the float subnormal range
// (create rejects increments and bounds below 2^-100 in magnitude), where the
// atomic add would flush to zero.  With kCas (NDT sample clearing, which must
// see the update that crosses its threshold, or a miss increment >= 0) every
// miss is a clamped compare-and-swap.
//
// kPipe: walk the next batch of voxels and issue its loads while the loads of
// the batch before are in flight, then apply that batch (a software pipeline
// of two batches); otherwise walk, load and apply one batch at a time.  The
// pipeline wins where many voxels are still unknown (their compare-and-swaps
// wait for a result) and costs a little on well-observed maps.
template <bool kOcc, bool kCounts, bool kCas, bool kPipe = true>
__device__ __forceinline__ void walk_segment_fast(const DeviceMap& m, int2 sg, unsigned int& ops,
                                                  const RayRec* prefetch = nullptr) {
  const int F = m.frac_bits;
  const RayRec* rp = m.rays + sg.x;
  FWalker f;
  uint32_t mo, neg;
  int32_t rcx, rcy, rcz, sgn, left, slot, slotE;
  long long keyE;
  {
    const RayRec r = *rp;
    SegStart s;
    segment_start(r, F, sg.y, &s);
    const bool last = sg.y == r.nseg - 1;
    left = (int32_t)s.visits - ((last && (r.flags & kRaySample)) ? 1 : 0);
    fwalker_init(f, r, F, s.c);
    neg = morton_neg(r.flags);
    sgn = (r.flags >> kRaySignShift) & 7;
    mo = local_morton(s.v[0], s.v[1], s.v[2]) ^ neg;
    rcx = s.v[0] >> kRegionShift;
    rcy = s.v[1] >> kRegionShift;
    rcz = s.v[2] >> kRegionShift;
    keyE = pack_region(s.ve[0] >> kRegionShift, s.ve[1] >> kRegionShift, s.ve[2] >> kRegionShift);
    find_region2(m, pack_region(rcx, rcy, rcz), keyE, &slot, &slotE);
  }
  // the record of the thread's next segment, into L2 while this one walks
  if (prefetch) asm volatile("prefetch.global.L2 [%0];" ::"l"(prefetch));
  if (left <= 0) return;
  if (slot < 0 || slotE < 0) {
    atomicOr(m.status, kStatusMissing);
    return;
  }
  uint32_t base = (uint32_t)slot << (3 * kRegionShift);
  unsigned int* occ = reinterpret_cast<unsigned int*>(m.occ);
  const unsigned int miss0 = __float_as_uint(__fadd_rn(0.0f, m.miss));  // an unknown voxel's first miss
  auto fill = [&](uint32_t (&off)[kFastBatchOf<kPipe>]) -> uint32_t {
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < kFastBatchOf<kPipe>; ++j) {
      off[j] = base | (mo ^ neg);  // voxel offset (< 2^31: at most 2^16 regions of 2^15 voxels)
      if (left > 0) {
        valid |= 1u << j;
        --left;
        if (left > 0) {
          int axis = fwalker_pick(f);
          if (axis < 0) axis = exact_pick_rec(rp, F, (int32_t)f.cx, (int32_t)f.cy, (int32_t)f.cz);
          fwalker_advance(f, axis);
          if (morton_advance(mo, morton_mask(axis))) {
            const int32_t d = ((sgn >> axis) & 1) ? -1 : 1;
            if (axis == 0)
              rcx += d;
            else if (axis == 1)
              rcy += d;
            else
              rcz += d;
            const long long key = pack_region(rcx, rcy, rcz);
            const int32_t ns = key == keyE ? slotE : find_region_rare(m, key);
            if (ns < 0) {
              atomicOr(m.status, kStatusMissing);
              left = 0;
            } else {
              base = (uint32_t)ns << (3 * kRegionShift);
            }
          }
        }
      }
    }
    return valid;
  };
  auto issue = [&](const uint32_t (&off)[kFastBatchOf<kPipe>], uint32_t valid, unsigned int (&old)[kFastBatchOf<kPipe>]) {
    if (kCounts) {
#pragma unroll
      for (int j = 0; j < kFastBatchOf<kPipe>; ++j)
        if ((valid >> j) & 1u) atomicAdd(m.counts + off[j], 1ULL);
    }
    if (kOcc) {
#pragma unroll
      for (int j = 0; j < kFastBatchOf<kPipe>; ++j) old[j] = ((valid >> j) & 1u) ? occ[off[j]] : 0u;
    }
  };
  auto apply = [&](const uint32_t (&off)[kFastBatchOf<kPipe>], uint32_t valid, unsigned int (&old)[kFastBatchOf<kPipe>]) {
    if (!kOcc) return;
    if (kCas) {
#pragma unroll
      for (int j = 0; j < kFastBatchOf<kPipe>; ++j)
        if ((valid >> j) & 1u) miss_cas(m, occ + off[j], old[j], ops);
      return;
    }
    if constexpr (!kPipe) {
      // Plain loop: an unknown voxel (NaN) is first set to the prior 0 by a
      // compare-and-swap whose result is not needed (one that loses finds a
      // value another thread set), then takes its miss as one more add of
      // delta, like a known voxel above l_min.  All of a call's misses of
      // the voxel are then adds of delta to 0, in any order: the values 0,
      // fl(0 + delta), ... of the clamped sequence that starts from the
      // prior (the clamp on read as above).  Same-address atomics of one
      // thread stay in order, so a thread's add never lands before its own
      // compare-and-swap.  Nothing here waits for a result, which the plain
      // loop (no second batch in flight) cannot hide; the pipelined loop
      // hides that wait and does better with one atomic per unknown voxel.
#pragma unroll
      for (int j = 0; j < kFastBatchOf<kPipe>; ++j) {
        if (!((valid >> j) & 1u)) continue;
        const float l = __uint_as_float(old[j]);
        if (l != l) {
          atomicCAS(occ + off[j], old[j], 0u);
          ++ops;
        }
        if (!(l <= m.l_min)) {
          atomicAdd(reinterpret_cast<float*>(occ + off[j]), m.miss);
          ++ops;
        }
      }
      return;
    }
    // adds go out at once; the compare-and-swaps that set unknown voxels
    // are all issued before any of their results is looked at.  A CAS
    // that won returns the NaN it replaced; one that lost returns the
    // (known) value another thread wrote, to which this ray's miss is then
    // added -- so the word read back replaces the one loaded.
    uint32_t init = 0;
#pragma unroll
    for (int j = 0; j < kFastBatchOf<kPipe>; ++j) {
      if (!((valid >> j) & 1u)) continue;
      const float l = __uint_as_float(old[j]);
      if (l > m.l_min) {
        atomicAdd(reinterpret_cast<float*>(occ + off[j]), m.miss);
        ++ops;
      } else if (l != l) {
        old[j] = atomicCAS(occ + off[j], old[j], miss0);
        init |= 1u << j;
        ++ops;
      }
    }
#pragma unroll
    for (int j = 0; j < kFastBatchOf<kPipe>; ++j) {
      if (((init >> j) & 1u) && __uint_as_float(old[j]) > m.l_min) {
        atomicAdd(reinterpret_cast<float*>(occ + off[j]), m.miss);
        ++ops;
      }
    }
  };
  if constexpr (kPipe) {
    uint32_t offA[kFastBatchOf<kPipe>], offB[kFastBatchOf<kPipe>];
    unsigned int oldA[kFastBatchOf<kPipe>], oldB[kFastBatchOf<kPipe>];
    uint32_t vA = fill(offA), vB;
    issue(offA, vA, oldA);
    while (vA) {
      vB = fill(offB);
      issue(offB, vB, oldB);
      apply(offA, vA, oldA);
      if (!vB) break;
      vA = fill(offA);
      issue(offA, vA, oldA);
      apply(offB, vB, oldB);
    }
  } else {
    while (left > 0) {
      uint32_t off[kFastBatchOf<kPipe>];
      unsigned int old[kFastBatchOf<kPipe>];
      const uint32_t v = fill(off);
      issue(off, v, old);
      apply(off, v, old);
    }
  }
}

// Whether a map's misses need the compare-and-swap form of walk_segment_fast.
__device__ __host__ __forceinline__ bool walk_needs_cas(uint32_t layers, float miss, float ndt_clear) {
  return !(miss < 0.0f) || ((layers & kLayerNdt) && ndt_clear > -INFINITY);
}

// Which miss walk a map takes: kWalkDecay (walk_segment, decay layer), else
// the filtered walk's template arguments as bits (4: occupancy, 2: counts,
// 1: every miss a compare-and-swap), or kWalkNone (no layer the walk updates).
constexpr int kWalkNone = -1;
constexpr int kWalkDecay = 8;
__device__ __host__ __forceinline__ int walk_variant(uint32_t layers, float miss, float ndt_clear) {
  const bool occ = (layers & kLayerOcc) != 0, cnt = (layers & kLayerCounts) != 0;
  if (layers & kLayerDecay) return kWalkDecay;
  if (!occ && !cnt) return kWalkNone;
  return (occ ? 4 : 0) | (cnt ? 2 : 0) | ((occ && walk_needs_cas(layers, miss, ndt_clear)) ? 1 : 0);
}

// Position of a sample inside its voxel (fixed-point offset 0 .. 2^F - 1) in
// 1/1024 of the voxel, rounded down: the voxel-mean layer's 10-bit field.
__device__ __forceinline__ unsigned long long sub_voxel10(long long offset, int F) {
  return F >= 10 ? (unsigned long long)(offset >> (F - 10)) : (unsigned long long)(offset << (10 - F));
}

// Clamped log-odds update of a voxel by n hits of the same delta (Eq. 2 with
// the clamp of Sec. II-B): n steps l <- min(max(l + delta, l_min), l_max)
// from the stored value (0 for an unknown voxel), written with one
// compare-and-swap.  Within a kernel all updates of a voxel use the same
// delta and the step map composes, so the result depends neither on their
// order nor on how they are grouped.  The loop is bounded: every failed CAS
// means another thread advanced the value toward its clamp.
__device__ __forceinline__ void logodds_update_n(const DeviceMap& m, float* p, float delta, unsigned int n) {
  unsigned int* u = reinterpret_cast<unsigned int*>(p);
  unsigned int old = *u;
  for (int it = 0; it < 256; ++it) {
    float v = logodds_value(__uint_as_float(old), m.l_min);
    for (unsigned int t = 0; t < n; ++t) {
      const float nv = fminf(fmaxf(__fadd_rn(v, delta), m.l_min), m.l_max);
      if (nv == v) break;  // at a clamp: later steps change nothing
      v = nv;
    }
    const unsigned int nb = __float_as_uint(v);
    if (nb == old) return;
    const unsigned int prev = atomicCAS(u, old, nb);
    if (prev == old) return;
    old = prev;
  }
  atomicOr(m.status, kStatusCasLimit);
}

// Sample phase (Sec. III-C phase two) for one ray: the voxel holding its
// sample takes a hit; with the NDT layer it also accumulates the sample's
// exact integer moments (count, sum, outer-product sum of the position inside
// the voxel), from which mean and covariance are formed when queried.
//
// Every lane of the warp calls this together (active = false for a lane
// without a ray of this map).  Neighbouring rays often end in the same voxel,
// and concurrent compare-and-swaps on one word retry, so the lanes holding the
// same voxel (__match_any_sync) form a group whose lowest lane applies all of
// the group's occupancy hits, n clamped steps in one compare-and-swap, and
// adds the group's hit count.  The voxel-mean fields and NDT moments are
// fire-and-forget integer adds per lane (summing them across the group first
// was measured slower).
template <bool kOcc, bool kCounts, bool kNdt>
__device__ __forceinline__ void hit_ray(const DeviceMap& m, long long i, bool active) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  bool ok = false;
  long long b[3] = {0, 0, 0};
  int32_t vx = 0, vy = 0, vz = 0, slot = 0;
  uint32_t mo = 0;
  if (active) {
    const RayRec r = m.rays[i];
    if (r.flags & kRaySample) {
      ray_end(r, F, b);
      vx = (int32_t)(b[0] >> F);
      vy = (int32_t)(b[1] >> F);
      vz = (int32_t)(b[2] >> F);
      slot = region_slot_of(m, vx, vy, vz);
      if (slot < 0) {
        atomicOr(m.status, kStatusMissing);
      } else {
        ok = true;
        mo = local_morton(vx, vy, vz);
      }
    }
  }
  // the NDT block is looked up before the occupancy update, so that the two
  // loads are in flight together
  int32_t ns = -1;
  if (kNdt && ok) ns = m.ndt_slot[slot];
  const long long off = ok ? voxel_offset(slot, mo) : 0;
  const unsigned grp = __match_any_sync(full, ok ? (uint32_t)off : 0xffffffffu);  // offsets are < 2^31
  const bool lead = ok && lane == __ffs(grp) - 1;
  const unsigned int n = __popc(grp);
  if (kOcc && lead) logodds_update_n(m, m.occ + off, m.hit, n);
  if (kCounts && lead) atomicAdd(m.counts + off, (unsigned long long)n << 32);
  if (!ok) return;
  if (m.layers & kLayerMean) {
    // 10-bit position inside the voxel per axis; per-call sums (x | y << 32, z | count << 32)
    const unsigned long long p0 =
        sub_voxel10(b[0] - (long long)vx * U, F) | (sub_voxel10(b[1] - (long long)vy * U, F) << 32);
    const unsigned long long p1 = sub_voxel10(b[2] - (long long)vz * U, F) | (1ULL << 32);
    atomicAdd(m.vmean_acc + 2 * off, p0);
    const unsigned long long prev = atomicAdd(m.vmean_acc + 2 * off + 1, p1);
    if ((prev >> 32) == 0) m.mean_list[atomicAdd(&m.calls->mean_touched, 1)] = (int32_t)off;
  }
  if (kNdt) {
    if (ns < 0) {
      atomicOr(m.status, kStatusMissing);
      return;
    }
    const long long px = b[0] - (long long)vx * U;
    const long long py = b[1] - (long long)vy * U;
    const long long pz = b[2] - (long long)vz * U;
    unsigned long long* base = reinterpret_cast<unsigned long long*>(m.ndt) + (long long)ns * 10 * kRegionVoxels + mo;
    const long long vals[10] = {1, px, py, pz, px * px, px * py, px * pz, py * py, py * pz, pz * pz};
#pragma unroll
    for (int k = 0; k < 10; ++k) atomicAdd(base + (long long)k * kRegionVoxels, (unsigned long long)vals[k]);
  }
}

// TSDF band of one ray (Sec. II-F): from range max(0, d - tau) to d + tau,
// quantised like a truncated endpoint.  Full warp, like prepare_occ_ray.
__device__ __forceinline__ void prepare_tsdf_ray(const DeviceMap& m, const CallArgs& args, long long i, bool active) {
  active = active && !latched(m);
  const int F = m.frac_bits;
  unsigned int nvisit = 0;
  TsdfRec r;
  r.flags = 0;
  if (active) {
    float o[3], e[3];
    uint8_t flag;
    load_ray(args, i, o, e, &flag);
    long long qo[3], qe[3];
    bool ok = quantise_call_ray(m, args, o, e, qo, qe) && (flag & kFlagNoReturn) == 0;
    if (ok) {
      // the range test and the band in float-float; in double where that
      // cannot settle them (tsdf_band_ff)
      bool in_range = false;
      if (!tsdf_band_ff(qo, qe, m.band, &in_range, r.a, r.b, r.u)) {
        double d[3];
        const double len = ray_length(qo, qe, d);
        in_range = len > m.rmin_q && len <= m.rmax_q;
        if (in_range && in_extent(qo, F) && in_extent(qe, F)) tsdf_band(qo, d, len, m.tau_q, r.a, r.b, r.u);
      }
      ok = in_range && in_extent(qo, F) && in_extent(qe, F);
    }
    if (ok) {
#pragma unroll
      for (int k = 0; k < 3; ++k) r.e[k] = qe[k];
      r.flags = kRayValid;
      long long l1 = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        long long dv = (r.b[k] >> F) - (r.a[k] >> F);
        l1 += dv < 0 ? -dv : dv;
      }
      nvisit = (unsigned int)(1 + l1);
      insert_ray_regions(m, r.a, r.b);
    }
    m.trays[i] = r;
  }
  warp_add(&m.calls->visits, &m.calls->total_visits, nvisit);
}

// TSDF band walk of one ray: per visited voxel c, s = (e - c).u (equal to
// d - (c - o).u), truncated to [-tau, tau], summed in 2^-32 m fixed point
// with a count.  The first visitor of a voxel in this call records it for the
// apply pass.
//
// Every lane of the warp calls this together (active = false for a lane
// without a ray of this map); blocks have kBlock threads.  Neighbouring
// pixels' rays cross the same band voxels (a 5 cm voxel at 1-2 m is crossed by
// hundreds of them per frame), so the updates are aggregated per warp: each
// thread walks kTsdfBatch voxels ahead; for each of them the lanes holding the
// same voxel (__match_any_sync) form a group whose lowest lane adds the
// group's count and sum of s with one atomic each (the s values pass through
// shared memory).  The sums are of integers, so the result does not depend on
// the grouping.  The first visitors the counts reveal are appended to the
// touched list with one atomic per warp and batch.
#ifndef OHM_TSDF_BATCH
#define OHM_TSDF_BATCH 4
#endif
constexpr int kTsdfBatch = OHM_TSDF_BATCH;
__device__ __forceinline__ void tsdf_walk_ray(const DeviceMap& m, long long i, bool active) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  const long long half = U >> 1;
  const float to_m = (float)(m.voxel_size / (double)(1LL << F));
  bool walking = false;
  Walker w;
  int32_t slot = -1;
  uint32_t mo = 0;
  long long e[3] = {0, 0, 0};
  float u[3] = {0.f, 0.f, 0.f};
  if (active) {
    const TsdfRec r = m.trays[i];
    if (r.flags & kRayValid) {
      walker_init(w, r.a, r.b, F, 0, 0);
      slot = region_slot_of(m, w.vx, w.vy, w.vz);
      if (slot < 0) {
        atomicOr(m.status, kStatusMissing);
      } else {
        walking = true;
        mo = local_morton(w.vx, w.vy, w.vz);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          e[k] = r.e[k];
          u[k] = r.u[k];
        }
      }
    }
  }
  unsigned int* cnt = m.tsdf_cnt;
  unsigned long long* sum = reinterpret_cast<unsigned long long*>(m.tsdf_sum);
  __shared__ long long sbuf[kBlock];
  while (__any_sync(full, walking)) {
    uint32_t off[kTsdfBatch];  // voxel offsets (< 2^31: at most 2^16 regions of 2^15 voxels)
    long long sq[kTsdfBatch];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < kTsdfBatch; ++j) {
      off[j] = 0;
      sq[j] = 0;
      if (walking) {
        const float ex = (float)(e[0] - ((long long)w.vx * U + half));
        const float ey = (float)(e[1] - ((long long)w.vy * U + half));
        const float ez = (float)(e[2] - ((long long)w.vz * U + half));
        float sv = (ex * u[0] + ey * u[1] + ez * u[2]) * to_m;
        sv = fminf(fmaxf(sv, -m.tau_m), m.tau_m);
        sq[j] = __float2ll_rn(sv * 4294967296.0f);
        off[j] = (uint32_t)voxel_offset(slot, mo);
        valid |= 1u << j;
        if (w.total == 0) {
          walking = false;
        } else {
          const int axis = walker_choose(w);
          int32_t c, sg;
          walker_step(w, axis, &c, &sg);
          mo = morton_step(mo, morton_mask(axis), sg);
          if ((c & ((1 << kRegionShift) - 1)) == (sg > 0 ? 0 : (1 << kRegionShift) - 1)) {
            slot = region_slot_of(m, w.vx, w.vy, w.vz);
            if (slot < 0) {
              atomicOr(m.status, kStatusMissing);
              walking = false;
            }
          }
        }
      }
    }
    unsigned int prev[kTsdfBatch];
#pragma unroll
    for (int j = 0; j < kTsdfBatch; ++j) {
      const bool vj = (valid >> j) & 1u;
      const unsigned grp = __match_any_sync(full, vj ? off[j] : 0xffffffffu);  // offsets are < 2^31
      sbuf[threadIdx.x] = sq[j];
      __syncwarp();
      prev[j] = 1u;
      if (vj && lane == __ffs(grp) - 1) {
        long long tot = 0;
        for (unsigned g = grp; g; g &= g - 1) tot += sbuf[(threadIdx.x & ~31u) + __ffs(g) - 1];
        prev[j] = atomicAdd(cnt + off[j], (unsigned int)__popc(grp));
        atomicAdd(sum + off[j], (unsigned long long)tot);
      }
      __syncwarp();
    }
    // first visitors of a voxel in this call: one table range per warp
    uint32_t first = 0;
#pragma unroll
    for (int j = 0; j < kTsdfBatch; ++j)
      if (prev[j] == 0) first |= 1u << j;
    const unsigned int nf = __popc(first);
    unsigned int incl = nf;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned int t = __shfl_up_sync(full, incl, d);
      if (lane >= d) incl += t;
    }
    const unsigned int total = __shfl_sync(full, incl, 31);
    if (total == 0) continue;
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(&m.calls->touched, (unsigned long long)total);
    base = __shfl_sync(full, base, 31);
    unsigned long long pos = base + (incl - nf);
#pragma unroll
    for (int j = 0; j < kTsdfBatch; ++j) {
      if ((first >> j) & 1u) {
        if (pos < (unsigned long long)m.max_touched)
          m.touched[pos] = (int32_t)off[j];
        else
          atomicOr(m.status, kStatusScratch);
        ++pos;
      }
    }
  }
}

// Weighted average of one touched voxel: D <- (W D + sum s) / (W + c),
// W <- min(W + c, W_max); the per-call sums are cleared for the next call.
__device__ __forceinline__ void tsdf_apply_one(const DeviceMap& m, long long t) {
  const int32_t off = m.touched[t];
  const unsigned int c = m.tsdf_cnt[off];
  const long long sum = m.tsdf_sum[off];
  m.tsdf_cnt[off] = 0;
  m.tsdf_sum[off] = 0;
  // in float (D and W are stored as floats; W and W + c are integers below
  // 2^24, exact): the rounding of D is far below the layer's 1e-5 m
  // tolerance, and the device's double division is slow
  const float2 dw = m.tsdf[off];
  const float S = (float)sum * 2.3283064365386962890625e-10f;  // 2^-32
  const float Wn = dw.y + (float)c;
  const float Dn = (dw.y * dw.x + S) / Wn;
  m.tsdf[off] = make_float2(Dn, fminf(Wn, m.wmax));
}

// Voxel-mean update of one voxel given samples by the call: per axis
// m <- floor((m n + S + floor((n + c) / 2)) / (n + c)), n <- min(n + c, 2^32 - 1);
// the per-call sums are cleared.  apply = false (a failed call) only clears.
__device__ __forceinline__ void mean_apply_one(const DeviceMap& m, long long t, bool apply) {
  const int32_t off = m.mean_list[t];
  const unsigned long long a0 = m.vmean_acc[2LL * off], a1 = m.vmean_acc[2LL * off + 1];
  m.vmean_acc[2LL * off] = 0;
  m.vmean_acc[2LL * off + 1] = 0;
  if (!apply) return;
  const unsigned long long S[3] = {a0 & 0xffffffffULL, a0 >> 32, a1 & 0xffffffffULL};
  const unsigned long long c = a1 >> 32;
  const unsigned long long w = m.vmean[off];
  const unsigned long long n0 = w >> 32, nt = n0 + c;
  unsigned long long packed = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const unsigned long long mk = (w >> (10 * k)) & 1023ULL;
    packed |= ((mk * n0 + S[k] + nt / 2) / nt) << (10 * k);
  }
  m.vmean[off] = ((nt < 0xffffffffULL ? nt : 0xffffffffULL) << 32) | packed;
}

__device__ __forceinline__ long long mean_touched_count(const DeviceMap& m) { return (long long)m.calls->mean_touched; }

__device__ __forceinline__ long long touched_count(const DeviceMap& m) {
  unsigned long long nt = m.calls->touched;
  return (long long)(nt > (unsigned long long)m.max_touched ? (unsigned long long)m.max_touched : nt);
}

// Undo the allocations of a failed call (threads t0, t0 + stride, ...): keys
// inserted by it become tombstones, keys it asked to restore go back to
// "evicted", its NDT blocks are released, and the pool counters and free-list
// positions are restored.  Stamps stay: regions the call touched count as
// recently used.
__device__ __forceinline__ void rollback_call(const DeviceMap& m, long long t0, long long stride) {
  const int32_t seq = m.calls->seq;
  for (long long h = t0; h <= (long long)m.hmask; h += stride) {
    const longlong2 e = m.htab[h];
    if (e.x == kEmptyKey || e.x == kTombKey) continue;
    if (e.y == kSlotRestoring)
      m.htab[h].y = kSlotEvicted;
    else if (e.y == kSlotPending || (e.y >= 0 && m.born[e.y] == seq))
      m.htab[h] = make_longlong2(kTombKey, -1);
  }
  for (long long s = t0; s < m.max_regions; s += stride) {
    const int32_t v = m.ndt_slot[s];
    if (v == -2 || (v >= 0 && (m.ndt_born[s] == seq || m.born[s] == seq))) m.ndt_slot[s] = -1;
  }
  if (t0 == 0) {
    *m.region_count = m.calls->region_start;
    *m.ndt_count = m.calls->ndt_start;
    m.free_info[1] = m.calls->free_used_start;
    m.free_info[3] = m.calls->ndt_free_used_start;
  }
}

}  // namespace ohm
