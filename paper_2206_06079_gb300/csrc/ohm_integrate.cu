// Ray integration kernels (Sec. III-B, III-C of arxiv 2206.06079, re-designed
// for sm_103a).
//
// One integrate call is one "ray set".  Kernels, in stream order:
//   k_begin          snapshot the pool counters (the rollback point)
//   k_prepare_occ    per ray: fixed-point quantisation, max-range truncation,
//                    region walk with hash insertion (the paper does this on
//                    the CPU, Sec. III-B; here it is a device pass), and the
//                    segment table (Sec. III-B ray segments)
//   k_ndt_alloc      per sample: give its region an NDT layer
//   k_prepare_tsdf   per ray: TSDF band end points and their regions
//   k_walk_miss      per segment: exact voxel walk, miss update per voxel
//   k_hits           per sample: hit update, hit count, NDT moments
//   k_tsdf_walk      per ray: band walk, fixed-point s sums and counts
//   k_tsdf_apply     per touched voxel: weighted average, scratch cleared
//   k_end            if any kernel latched a failure: undo the allocations
// Every kernel after k_begin returns at once when the status word is set, so
// a failed call changes no voxel.
#include <climits>

#include "ohm_host.h"

namespace ohm {

namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ bool latched(const DeviceMap& m) { return *(volatile int32_t*)m.status != 0; }

// Clamped log-odds update of one voxel (Eq. 2 with the clamp of Sec. II-B):
// l <- min(max(l0 + delta, l_min), l_max), l0 = 0 for an unknown (NaN) voxel.
// Concurrent updates of one voxel are serialised by compare-and-swap; within
// a kernel all updates of a voxel use the same delta, so the result does not
// depend on their order.  The loop is bounded: every failed CAS means another
// thread advanced the value one step toward its clamp.
__device__ __forceinline__ void logodds_update(const DeviceMap& m, float* p, float delta) {
  unsigned int* u = reinterpret_cast<unsigned int*>(p);
  unsigned int old = *u;
  for (int it = 0; it < 256; ++it) {
    const float l = __uint_as_float(old);
    const float l0 = (l != l) ? 0.0f : l;
    const float nv = fminf(fmaxf(__fadd_rn(l0, delta), m.l_min), m.l_max);
    const unsigned int nb = __float_as_uint(nv);
    if (nb == old) return;
    const unsigned int prev = atomicCAS(u, old, nb);
    if (prev == old) return;
    old = prev;
  }
  atomicOr(m.status, kStatusCasLimit);
}

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
__device__ __forceinline__ void insert_ray_regions(const DeviceMap& m, const long long a[3], const long long b[3]) {
  Walker w;
  walker_init(w, a, b, m.frac_bits + kRegionShift, 0, 0);
  insert_region(m, w.vx, w.vy, w.vz);
  while (w.total > 0) {
    int32_t c, s;
    walker_step(w, walker_choose(w), &c, &s);
    insert_region(m, w.vx, w.vy, w.vz);
  }
}

__device__ __forceinline__ long long voxel_offset(int32_t slot, uint32_t mo) {
  return (long long)slot * kRegionVoxels + mo;
}

__device__ __forceinline__ int32_t region_slot_of(const DeviceMap& m, int32_t vx, int32_t vy, int32_t vz) {
  return find_region(m, pack_region(vx >> kRegionShift, vy >> kRegionShift, vz >> kRegionShift));
}

// The same lookup kept out of line: the walk kernels call it from every slot
// of an unrolled batch, and one shared copy keeps the instruction cache warm.
__device__ __noinline__ int32_t region_slot_call(const DeviceMap& m, int32_t vx, int32_t vy, int32_t vz) {
  return region_slot_of(m, vx, vy, vz);
}

__device__ __forceinline__ uint32_t local_morton(int32_t vx, int32_t vy, int32_t vz) {
  const int32_t mask = (1 << kRegionShift) - 1;
  return morton((uint32_t)(vx & mask), (uint32_t)(vy & mask), (uint32_t)(vz & mask));
}

}  // namespace

__global__ void k_begin(DeviceMap m, long long n) {
  m.calls->region_start = *m.region_count;
  m.calls->ndt_start = *m.ndt_count;
  m.calls->segments = 0;
  m.calls->visits = 0;
  m.calls->touched = 0;
  m.calls->rays = (unsigned long long)n;
}

__global__ void __launch_bounds__(kBlock) k_prepare_occ(DeviceMap m, CallArgs args) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < args.n && !latched(m);
  const int F = m.frac_bits;
  unsigned int nseg = 0, nvisit = 0;
  RayRec r;
  r.flags = 0;
  r.nseg = 0;
  r.inv = 0;
  if (active) {
    float o[3], e[3];
    uint8_t flag;
    load_ray(args, i, o, e, &flag);
    long long qo[3], qe[3];
    bool ok = quantise_ray(m, o, e, qo, qe);
    bool sample = (flag & kFlagNoReturn) == 0;
    if (ok) {
      double d[3];
      const double len = ray_length(qo, qe, d);
      if (len > m.rmax_q) {
        const double ratio = __ddiv_rn(m.rmax_q, len);
#pragma unroll
        for (int k = 0; k < 3; ++k) qe[k] = qo[k] + __double2ll_rn(__dmul_rn(d[k], ratio));
        sample = false;
      }
      ok = in_extent(qo, F) && in_extent(qe, F);
    }
    if (ok) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        r.a[k] = qo[k];
        r.b[k] = qe[k];
      }
      int32_t nmaj;
      const int M = dominant_axis(qo, qe, F, &nmaj);
      nseg = (unsigned int)segment_count(nmaj, m.seg_steps);
      const long long am = sel3(M, qe[0] - qo[0], qe[1] - qo[1], qe[2] - qo[2]);
      r.inv = reciprocal64((unsigned long long)(am < 0 ? -am : am));
      r.flags = kRayValid | (sample ? kRaySample : 0) | (M << kRayAxisShift);
      r.nseg = (int32_t)nseg;
      long long l1 = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        long long dv = (qe[k] >> F) - (qo[k] >> F);
        l1 += dv < 0 ? -dv : dv;
      }
      nvisit = (unsigned int)(1 + l1);
      insert_ray_regions(m, qo, qe);
    }
  }
  if (i < args.n) m.rays[i] = r;
  const unsigned long long base = warp_reserve(&m.calls->segments, nseg);
  if (nseg > 0) {
    if (base + nseg > (unsigned long long)m.max_segs) {
      atomicOr(m.status, kStatusScratch);
    } else {
      for (unsigned int j = 0; j < nseg; ++j) m.segs[base + j] = make_int2((int)i, (int)j);
    }
  }
  warp_add(&m.calls->visits, &m.calls->total_visits, nvisit);
}

__global__ void __launch_bounds__(kBlock) k_ndt_alloc(DeviceMap m, long long n) {
  if (latched(m)) return;
  const int F = m.frac_bits;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const RayRec r = m.rays[i];
    if (!(r.flags & kRaySample)) continue;
    const int32_t slot = region_slot_of(m, (int32_t)(r.b[0] >> F), (int32_t)(r.b[1] >> F), (int32_t)(r.b[2] >> F));
    if (slot < 0) {
      atomicOr(m.status, kStatusMissing);
      continue;
    }
    if (*(volatile int32_t*)&m.ndt_slot[slot] != -1) continue;
    if (atomicCAS(&m.ndt_slot[slot], -1, -2) == -1) {
      const int32_t id = atomicAdd(m.ndt_count, 1);
      if (id < m.max_ndt)
        m.ndt_slot[slot] = id;
      else
        atomicOr(m.status, kStatusCapacity);
    }
  }
}

// Retry a clamped log-odds CAS whose first attempt found `cur` instead of
// the value it expected (see logodds_update).
__device__ __noinline__ void logodds_retry(const DeviceMap& m, unsigned int* u, unsigned int cur, float delta) {
  for (int it = 0; it < 256; ++it) {
    const float l = __uint_as_float(cur);
    const float l0 = (l != l) ? 0.0f : l;
    const unsigned int nb = __float_as_uint(fminf(fmaxf(__fadd_rn(l0, delta), m.l_min), m.l_max));
    if (nb == cur) return;
    const unsigned int prev = atomicCAS(u, cur, nb);
    if (prev == cur) return;
    cur = prev;
  }
  atomicOr(m.status, kStatusCasLimit);
}

// Miss phase (Sec. III-C phase one): every voxel a ray passes through, except
// the voxel holding its sample, takes one miss.  One thread per segment;
// segment j of a ray covers the voxels entered after j*S and before
// (j+1)*S steps of the ray's dominant axis (the last segment runs to the end).
//
// The walk itself is cheap integer arithmetic; the cost is the read-modify-
// write of each voxel in global memory.  So a thread walks kWalkBatch voxels
// ahead, then issues all their loads at once, then all their CASes at once,
// keeping that many memory operations in flight instead of one.
#ifndef OHM_WALK_BATCH
#define OHM_WALK_BATCH 4
#endif
#ifndef OHM_WALK_MIN_BLOCKS
#define OHM_WALK_MIN_BLOCKS 4
#endif
constexpr int kWalkBatch = OHM_WALK_BATCH;

template <bool kOcc, bool kCounts>
__global__ void __launch_bounds__(kBlock, OHM_WALK_MIN_BLOCKS) k_walk_miss(DeviceMap m) {
  if (latched(m)) return;
  const long long nseg = (long long)m.calls->segments;
  const int F = m.frac_bits;
  const int32_t S = m.seg_steps;
  const float miss = m.miss;
  for (long long si = (long long)blockIdx.x * blockDim.x + threadIdx.x; si < nseg;
       si += (long long)gridDim.x * blockDim.x) {
    const int2 sg = m.segs[si];
    const RayRec r = m.rays[sg.x];
    const int M = (r.flags >> kRayAxisShift) & 3;
    const bool last = sg.y == r.nseg - 1;
    const bool sample = (r.flags & kRaySample) != 0;
    Walker w;
    walker_init(w, r.a, r.b, F, M, (long long)sg.y * S, r.inv);
    int32_t mrem = last ? INT_MAX : S - 1;
    int32_t slot = region_slot_of(m, w.vx, w.vy, w.vz);
    if (slot < 0) {
      atomicOr(m.status, kStatusMissing);
      continue;
    }
    uint32_t mo = local_morton(w.vx, w.vy, w.vz);
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
          done = true;
          continue;
        }
        const int axis = walker_choose(w);
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
          slot = region_slot_call(m, w.vx, w.vy, w.vz);
          if (slot < 0) {
            atomicOr(m.status, kStatusMissing);
            done = true;
          }
        }
      }
      if (kOcc) {
        unsigned int* base = reinterpret_cast<unsigned int*>(m.occ);
        unsigned int old[kWalkBatch], prev[kWalkBatch];
#pragma unroll
        for (int j = 0; j < kWalkBatch; ++j) old[j] = (todo >> j) & 1u ? base[off[j]] : 0u;
#pragma unroll
        for (int j = 0; j < kWalkBatch; ++j) {
          prev[j] = old[j];
          if (!((todo >> j) & 1u)) continue;
          const float l = __uint_as_float(old[j]);
          const float l0 = (l != l) ? 0.0f : l;
          const unsigned int nb = __float_as_uint(fminf(fmaxf(__fadd_rn(l0, miss), m.l_min), m.l_max));
          if (nb == old[j]) continue;
          prev[j] = atomicCAS(base + off[j], old[j], nb);
        }
#pragma unroll
        for (int j = 0; j < kWalkBatch; ++j)
          if (prev[j] != old[j]) logodds_retry(m, base + off[j], prev[j], miss);
      }
    }
  }
}

// Sample phase (Sec. III-C phase two): the voxel holding each sample takes a
// hit; with the NDT layer it also accumulates the sample's exact integer
// moments (count, sum, outer-product sum of the position inside the voxel),
// from which mean and covariance are formed when queried.
template <bool kOcc, bool kCounts, bool kNdt>
__global__ void __launch_bounds__(kBlock) k_hits(DeviceMap m, long long n) {
  if (latched(m)) return;
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const RayRec r = m.rays[i];
    if (!(r.flags & kRaySample)) continue;
    const int32_t vx = (int32_t)(r.b[0] >> F), vy = (int32_t)(r.b[1] >> F), vz = (int32_t)(r.b[2] >> F);
    const int32_t slot = region_slot_of(m, vx, vy, vz);
    if (slot < 0) {
      atomicOr(m.status, kStatusMissing);
      continue;
    }
    const uint32_t mo = local_morton(vx, vy, vz);
    const long long off = voxel_offset(slot, mo);
    if (kOcc) logodds_update(m, m.occ + off, m.hit);
    if (kCounts) atomicAdd(m.counts + off, 1ULL << 32);
    if (kNdt) {
      const int32_t ns = m.ndt_slot[slot];
      if (ns < 0) {
        atomicOr(m.status, kStatusMissing);
        continue;
      }
      const long long px = r.b[0] - (long long)vx * U;
      const long long py = r.b[1] - (long long)vy * U;
      const long long pz = r.b[2] - (long long)vz * U;
      unsigned long long* base = reinterpret_cast<unsigned long long*>(m.ndt) + (long long)ns * 10 * kRegionVoxels + mo;
      const long long vals[10] = {1, px, py, pz, px * px, px * py, px * pz, py * py, py * pz, pz * pz};
#pragma unroll
      for (int k = 0; k < 10; ++k) atomicAdd(base + (long long)k * kRegionVoxels, (unsigned long long)vals[k]);
    }
  }
}

// TSDF band of each ray (Sec. II-F): from range max(0, d - tau) to d + tau,
// quantised like a truncated endpoint.
__global__ void __launch_bounds__(kBlock) k_prepare_tsdf(DeviceMap m, CallArgs args) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = i < args.n && !latched(m);
  const int F = m.frac_bits;
  unsigned int nvisit = 0;
  TsdfRec r;
  r.flags = 0;
  if (active) {
    float o[3], e[3];
    uint8_t flag;
    load_ray(args, i, o, e, &flag);
    long long qo[3], qe[3];
    bool ok = quantise_ray(m, o, e, qo, qe) && (flag & kFlagNoReturn) == 0;
    double d[3], len = 0.0;
    if (ok) {
      len = ray_length(qo, qe, d);
      ok = len > m.rmin_q && len <= m.rmax_q && in_extent(qo, F) && in_extent(qe, F);
    }
    if (ok) {
      double t0 = __dsub_rn(len, m.tau_q);
      if (t0 < 0.0) t0 = 0.0;
      const double t1 = __dadd_rn(len, m.tau_q);
      const double f0 = __ddiv_rn(t0, len), f1 = __ddiv_rn(t1, len);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        r.a[k] = qo[k] + __double2ll_rn(__dmul_rn(d[k], f0));
        r.b[k] = qo[k] + __double2ll_rn(__dmul_rn(d[k], f1));
        r.e[k] = qe[k];
        r.u[k] = (float)__ddiv_rn(d[k], len);
      }
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
  }
  if (i < args.n) m.trays[i] = r;
  warp_add(&m.calls->visits, &m.calls->total_visits, nvisit);
}

// Band walk: per visited voxel c, s = (e - c).u (equal to d - (c - o).u),
// truncated to [-tau, tau], summed in 2^-32 m fixed point with a count.  The
// first visitor of a voxel in this call records it for the apply pass.
__global__ void __launch_bounds__(kBlock) k_tsdf_walk(DeviceMap m, long long n) {
  if (latched(m)) return;
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  const long long half = U >> 1;
  const float to_m = (float)(m.voxel_size / (double)(1LL << F));
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const TsdfRec r = m.trays[i];
    if (!(r.flags & kRayValid)) continue;
    Walker w;
    walker_init(w, r.a, r.b, F, 0, 0);
    int32_t slot = region_slot_of(m, w.vx, w.vy, w.vz);
    if (slot < 0) {
      atomicOr(m.status, kStatusMissing);
      continue;
    }
    uint32_t mo = local_morton(w.vx, w.vy, w.vz);
    for (;;) {
      const float ex = (float)(r.e[0] - ((long long)w.vx * U + half));
      const float ey = (float)(r.e[1] - ((long long)w.vy * U + half));
      const float ez = (float)(r.e[2] - ((long long)w.vz * U + half));
      float s = (ex * r.u[0] + ey * r.u[1] + ez * r.u[2]) * to_m;
      s = fminf(fmaxf(s, -m.tau_m), m.tau_m);
      const long long sq = __float2ll_rn(s * 4294967296.0f);
      const long long off = voxel_offset(slot, mo);
      const unsigned int prev = atomicAdd(m.tsdf_cnt + off, 1u);
      atomicAdd(reinterpret_cast<unsigned long long*>(m.tsdf_sum) + off, (unsigned long long)sq);
      if (prev == 0) {
        const unsigned long long t = atomicAdd(&m.calls->touched, 1ULL);
        if (t < (unsigned long long)m.max_touched)
          m.touched[t] = (int32_t)off;
        else
          atomicOr(m.status, kStatusScratch);
      }
      if (w.total == 0) break;
      const int axis = walker_choose(w);
      int32_t c, sg;
      walker_step(w, axis, &c, &sg);
      mo = morton_step(mo, morton_mask(axis), sg);
      if ((c & ((1 << kRegionShift) - 1)) == (sg > 0 ? 0 : (1 << kRegionShift) - 1)) {
        slot = region_slot_of(m, w.vx, w.vy, w.vz);
        if (slot < 0) {
          atomicOr(m.status, kStatusMissing);
          break;
        }
      }
    }
  }
}

// Weighted average per touched voxel: D <- (W D + sum s) / (W + c),
// W <- min(W + c, W_max); the per-call sums are cleared for the next call.
__global__ void __launch_bounds__(kBlock) k_tsdf_apply(DeviceMap m) {
  if (latched(m)) return;
  unsigned long long nt = m.calls->touched;
  if (nt > (unsigned long long)m.max_touched) nt = (unsigned long long)m.max_touched;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)nt;
       t += (long long)gridDim.x * blockDim.x) {
    const int32_t off = m.touched[t];
    const unsigned int c = m.tsdf_cnt[off];
    const long long sum = m.tsdf_sum[off];
    m.tsdf_cnt[off] = 0;
    m.tsdf_sum[off] = 0;
    const float2 dw = m.tsdf[off];
    const double W = (double)dw.y, D = (double)dw.x;
    const double S = (double)sum * (1.0 / 4294967296.0);
    const double Wn = W + (double)c;
    const double Dn = (W * D + S) / Wn;
    m.tsdf[off] = make_float2((float)Dn, (float)(Wn < (double)m.wmax ? Wn : (double)m.wmax));
  }
}

// Undo the allocations of a failed call: keys inserted by it become
// tombstones, its NDT slots are released, the pool counters are restored.
__global__ void k_end(DeviceMap m) {
  if (!latched(m)) return;
  const int32_t rs = m.calls->region_start, ns = m.calls->ndt_start;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long h = t0; h <= (long long)m.hmask; h += stride) {
    const longlong2 e = m.htab[h];
    if (e.x == kEmptyKey || e.x == kTombKey) continue;
    if (e.y < 0 || e.y >= rs) m.htab[h] = make_longlong2(kTombKey, -1);
  }
  for (long long s = t0; s < m.max_regions; s += stride) {
    const int32_t v = m.ndt_slot[s];
    if (s >= rs || v == -2 || v >= ns) m.ndt_slot[s] = -1;
  }
  if (t0 == 0) {
    *m.region_count = rs;
    *m.ndt_count = ns;
  }
}

// ---------------------------------------------------------------------------
// Query and export.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_query(DeviceMap m, const float* pts, long long n, float* occupancy,
                                                   uint8_t* known, float* ndt, float* tsdf, uint32_t* counts) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int F = m.frac_bits;
  long long q[3];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) ok = ok && isfinite(pts[3 * i + k]) && quantise(pts[3 * i + k], m.origin[k], m.scale, &q[k]);
  ok = ok && in_extent(q, F);
  int32_t slot = -1;
  uint32_t mo = 0;
  int32_t v[3] = {0, 0, 0};
  if (ok) {
    v[0] = (int32_t)(q[0] >> F);
    v[1] = (int32_t)(q[1] >> F);
    v[2] = (int32_t)(q[2] >> F);
    slot = region_slot_of(m, v[0], v[1], v[2]);
    mo = local_morton(v[0], v[1], v[2]);
  }
  const long long off = voxel_offset(slot, mo);
  if (occupancy || known) {
    float l = __int_as_float(0x7fc00000);
    if (slot >= 0 && (m.layers & kLayerOcc)) l = m.occ[off];
    if (occupancy) occupancy[i] = l;
    if (known) known[i] = (l == l) ? 1 : 0;
  }
  if (counts) {
    unsigned long long c = 0;
    if (slot >= 0 && (m.layers & kLayerCounts)) c = m.counts[off];
    counts[2 * i + 0] = (uint32_t)(c >> 32);
    counts[2 * i + 1] = (uint32_t)(c & 0xffffffffu);
  }
  if (tsdf) {
    float2 dw = make_float2(0.f, 0.f);
    if (slot >= 0 && (m.layers & kLayerTsdf)) dw = m.tsdf[off];
    tsdf[2 * i + 0] = dw.x;
    tsdf[2 * i + 1] = dw.y;
  }
  if (ndt) {
    float out[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) out[k] = 0.f;
    const int32_t ns = (slot >= 0 && (m.layers & kLayerNdt)) ? m.ndt_slot[slot] : -1;
    if (ns >= 0) {
      const long long* base = m.ndt + (long long)ns * 10 * kRegionVoxels + mo;
      long long s[10];
#pragma unroll
      for (int k = 0; k < 10; ++k) s[k] = base[(long long)k * kRegionVoxels];
      if (s[0] > 0) {
        const double cnt = (double)s[0];
        const double cell = m.voxel_size / (double)(1LL << F);
        out[0] = (float)cnt;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double corner = (double)((long long)v[k] * (1LL << F));
          out[1 + k] = (float)(m.origin[k] + (corner + (double)s[1 + k] / cnt) * cell);
        }
        const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          const __int128 num = (__int128)s[0] * s[4 + k] - (__int128)s[1 + pa[k]] * s[1 + pb[k]];
          out[4 + k] = (float)((double)num / (cnt * cnt) * cell * cell);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) ndt[10 * i + k] = out[k];
  }
}

__global__ void __launch_bounds__(kBlock) k_export(DeviceMap m, long long first, long long count, int32_t* keys,
                                                    float* occupancy, uint32_t* counts, long long* ndt, float* tsdf) {
  const long long total = count * kRegionVoxels;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / kRegionVoxels;
    const int32_t lin = (int32_t)(t % kRegionVoxels);
    const int32_t slot = (int32_t)(first + r);
    const uint32_t mo = morton(lin & 31, (lin >> 5) & 31, lin >> 10);
    const long long off = voxel_offset(slot, mo);
    if (keys && lin < 3) keys[3 * r + lin] = m.region_coords[3 * slot + lin];
    if (occupancy) occupancy[t] = (m.layers & kLayerOcc) ? m.occ[off] : __int_as_float(0x7fc00000);
    if (counts) {
      const unsigned long long c = (m.layers & kLayerCounts) ? m.counts[off] : 0ULL;
      counts[2 * t + 0] = (uint32_t)(c >> 32);
      counts[2 * t + 1] = (uint32_t)(c & 0xffffffffu);
    }
    if (tsdf) {
      const float2 dw = (m.layers & kLayerTsdf) ? m.tsdf[off] : make_float2(0.f, 0.f);
      tsdf[2 * t + 0] = dw.x;
      tsdf[2 * t + 1] = dw.y;
    }
    if (ndt) {
      const int32_t ns = (m.layers & kLayerNdt) ? m.ndt_slot[slot] : -1;
#pragma unroll
      for (int k = 0; k < 10; ++k)
        ndt[10 * t + k] = ns >= 0 ? m.ndt[(long long)ns * 10 * kRegionVoxels + (long long)k * kRegionVoxels + mo] : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
int walk_blocks_per_sm() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk_miss<true, true>, kBlock, 0);
  return b > 0 ? b : 1;
}

static long long blocks_for(long long n) { return (n + kBlock - 1) / kBlock; }

// Launch one kernel as stage `stage`, with event timing when it is profiled.
#define OHM_LAUNCH(stage, ...)                  \
  do {                                          \
    cudaEvent_t ev_ = nullptr;                  \
    stage_begin(map, (stage), stream, &ev_);    \
    __VA_ARGS__;                                \
    stage_end(map, (stage), stream, ev_);       \
    map->launches += 1;                         \
  } while (0)

cudaError_t launch_integrate(ohm_map* map, const CallArgs& args, cudaStream_t stream) {
  DeviceMap& m = map->d;
  const bool occ = (m.layers & kLayerOcc) != 0, cnt = (m.layers & kLayerCounts) != 0, ndt = (m.layers & kLayerNdt) != 0;
  const bool tsdf = (m.layers & kLayerTsdf) != 0;
  const long long n = args.n;
  const int grid = map->walk_blocks;
  const long long per_ray_blocks = blocks_for(n) > 0 ? blocks_for(n) : 1;
  const int ray_grid = (int)(per_ray_blocks < grid ? per_ray_blocks : grid);
  const unsigned prb = (unsigned)per_ray_blocks;
  OHM_LAUNCH(OHM_STAGE_BEGIN, k_begin<<<1, 1, 0, stream>>>(m, n));
  if (occ || cnt || ndt) {
    OHM_LAUNCH(OHM_STAGE_PREPARE, k_prepare_occ<<<prb, kBlock, 0, stream>>>(m, args));
    if (ndt) OHM_LAUNCH(OHM_STAGE_NDT_ALLOC, k_ndt_alloc<<<ray_grid, kBlock, 0, stream>>>(m, n));
  }
  if (tsdf) OHM_LAUNCH(OHM_STAGE_PREPARE_TSDF, k_prepare_tsdf<<<prb, kBlock, 0, stream>>>(m, args));
  if (occ || cnt) {
    if (occ && cnt)
      OHM_LAUNCH(OHM_STAGE_WALK, k_walk_miss<true, true><<<grid, kBlock, 0, stream>>>(m));
    else if (occ)
      OHM_LAUNCH(OHM_STAGE_WALK, k_walk_miss<true, false><<<grid, kBlock, 0, stream>>>(m));
    else
      OHM_LAUNCH(OHM_STAGE_WALK, k_walk_miss<false, true><<<grid, kBlock, 0, stream>>>(m));
  }
  if (occ || cnt || ndt) {
    const int sel = (occ ? 4 : 0) | (cnt ? 2 : 0) | (ndt ? 1 : 0);
    switch (sel) {
      case 7: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<true, true, true><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 6: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<true, true, false><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 5: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<true, false, true><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 4: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<true, false, false><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 3: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<false, true, true><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 2: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<false, true, false><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      case 1: OHM_LAUNCH(OHM_STAGE_HITS, k_hits<false, false, true><<<ray_grid, kBlock, 0, stream>>>(m, n)); break;
      default: break;
    }
  }
  if (tsdf) {
    OHM_LAUNCH(OHM_STAGE_TSDF_WALK, k_tsdf_walk<<<ray_grid, kBlock, 0, stream>>>(m, n));
    OHM_LAUNCH(OHM_STAGE_TSDF_APPLY, k_tsdf_apply<<<grid, kBlock, 0, stream>>>(m));
  }
  OHM_LAUNCH(OHM_STAGE_END, k_end<<<grid, kBlock, 0, stream>>>(m));
  return cudaGetLastError();
}

cudaError_t launch_query(ohm_map* map, const float* points, long long n, float* occupancy, uint8_t* known, float* ndt,
                         float* tsdf, uint32_t* counts, cudaStream_t stream) {
  if (n > 0)
    k_query<<<(unsigned)blocks_for(n), kBlock, 0, stream>>>(map->d, points, n, occupancy, known, ndt, tsdf, counts);
  return cudaGetLastError();
}

cudaError_t launch_export(ohm_map* map, long long first, long long count, int32_t* keys, float* occupancy,
                          uint32_t* counts, long long* ndt, float* tsdf, cudaStream_t stream) {
  if (count > 0) {
    long long b = blocks_for(count * kRegionVoxels);
    if (b > 65535LL * 16) b = 65535LL * 16;
    k_export<<<(unsigned)b, kBlock, 0, stream>>>(map->d, first, count, keys, occupancy, counts, ndt, tsdf);
  }
  return cudaGetLastError();
}

}  // namespace ohm
