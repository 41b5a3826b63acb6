// Ray integration kernels (Sec. III-B, III-C of arxiv 2206.06079, re-designed
// for sm_103a).
//
// One integrate call is one "ray set".  Kernels, in stream order:
//   k_begin          snapshot the pool counters (the rollback point)
//   k_prepare_occ    per ray: fixed-point quantisation, max-range truncation,
//                    region walk with hash insertion (the paper does this on
//                    the CPU, Sec. III-B; here it is a device pass), the
//                    segment table (Sec. III-B ray segments), and the NDT
//                    block of the sample's region
//   k_ndt_alloc      sample rays prepare left: give their regions an NDT layer
//   k_prepare_tsdf   per ray: TSDF band end points and their regions
//   k_walk_fast      per segment: exact voxel walk, miss update per voxel
//                    (k_walk_miss for maps with the decay layer)
//   k_hits           per sample: hit update, hit count, NDT moments
//   k_tsdf_walk      per ray: band walk, fixed-point s sums and counts
//   k_tsdf_apply     per touched voxel: weighted average, scratch cleared
//   k_end            if any kernel latched a failure: undo the allocations
// Every kernel after k_begin returns at once when the status word is set, so
// a failed call changes no voxel.
#include "ohm_kernels.cuh"

namespace ohm {

#define OHM_GRID_STRIDE(i, n) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// Chained like the kernels after it: its launch overlaps the tail of the
// previous call's last kernel, and its body waits for that kernel.
__global__ void k_begin(DeviceMap m, CallArgs args) {
  chain_enter();
  if (blockIdx.x == 0 && threadIdx.x == 0) begin_call(m, args);
}

__global__ void __launch_bounds__(kBlock, OHM_PREPARE_MIN_BLOCKS) k_prepare_occ(DeviceMap m, CallArgs args) {
  chain_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  prepare_occ_ray(m, args, i, i < args.n);
}

// Blocks of the NDT pass: it has only the rays prepare could not settle (a
// few per scan), read from the device-side count.
constexpr int kNdtPendingGrid = 64;

// The sample rays whose region slot prepare did not learn (another thread
// was inserting the region at the time): their regions get NDT blocks here.
__global__ void __launch_bounds__(kBlock) k_ndt_alloc(DeviceMap m) {
  chain_enter();
  if (latched(m)) return;
  const long long n = (long long)m.calls->ndt_pending;
  OHM_GRID_STRIDE(k, n) ndt_alloc_ray(m, m.ndt_pending[k]);
}

template <bool kOcc, bool kCounts, bool kDecay>
__global__ void __launch_bounds__(kBlock, OHM_WALK_MIN_BLOCKS) k_walk_miss(DeviceMap m) {
  chain_enter();
  if (latched(m)) return;
  const long long nseg = (long long)m.calls->segments;
  unsigned int cas = 0;
  OHM_GRID_STRIDE(si, nseg) walk_segment<kOcc, kCounts, kDecay>(m, si, cas);
  // every thread gets here: one atomic per warp for the call's CAS count
  cas = __reduce_add_sync(0xffffffffu, cas);
  if ((threadIdx.x & 31) == 0 && cas) atomicAdd(&m.calls->atomics, (unsigned long long)cas);
}

// The miss walk of maps without the decay layer (filtered walk, see
// walk_segment_fast).
// OHM_SINGLE_PIPE: the single-map walk runs the pipelined loop (the plain
// loop of the multi-map batch, with its unchecked CAS initialisation, was
// slower on tunnel scans at 4 and 5 blocks per SM).
#ifndef OHM_SINGLE_PIPE
#define OHM_SINGLE_PIPE true
#endif
template <bool kOcc, bool kCounts, bool kCas>
__global__ void __launch_bounds__(kBlock, OHM_FAST_MIN_BLOCKS) k_walk_fast(DeviceMap m) {
  chain_enter();
  if (latched(m)) return;
  const long long nseg = (long long)m.calls->segments;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned int ops = 0;
  long long si = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int2 sg = si < nseg ? m.segs[si] : make_int2(0, 0);
  for (; si < nseg; si += stride) {
    // the next segment's table entry is loaded while this one walks
    const int2 next = si + stride < nseg ? m.segs[si + stride] : make_int2(-1, 0);
    walk_segment_fast<kOcc, kCounts, kCas, OHM_SINGLE_PIPE>(m, sg, ops, next.x >= 0 ? m.rays + next.x : nullptr);
    sg = next;
  }
  // every thread gets here: one atomic per warp for the call's atomic count
  ops = __reduce_add_sync(0xffffffffu, ops);
  if ((threadIdx.x & 31) == 0 && ops) atomicAdd(&m.calls->atomics, (unsigned long long)ops);
}

template <bool kOcc, bool kCounts, bool kNdt>
__global__ void __launch_bounds__(kBlock) k_hits(DeviceMap m, long long n) {
  chain_enter();
  if (latched(m)) return;
  // whole warps iterate together (the update is warp-collective)
  const long long np = (n + 31) & ~31LL;
  OHM_GRID_STRIDE(i, np) hit_ray<kOcc, kCounts, kNdt>(m, i, i < n);
}

// Runs for failed calls too: it then only clears the per-call sums.
__global__ void __launch_bounds__(kBlock) k_mean_apply(DeviceMap m) {
  chain_enter();
  const bool apply = !latched(m);
  const long long nt = mean_touched_count(m);
  OHM_GRID_STRIDE(t, nt) mean_apply_one(m, t, apply);
}

// Compiled for 4 blocks per SM (64 registers; 78 unbounded, which fits 3).
__global__ void __launch_bounds__(kBlock, 4) k_prepare_tsdf(DeviceMap m, CallArgs args) {
  chain_enter();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  prepare_tsdf_ray(m, args, i, i < args.n);
}

__global__ void __launch_bounds__(kBlock) k_tsdf_walk(DeviceMap m, long long n) {
  chain_enter();
  if (latched(m)) return;
  // whole warps iterate together (the walk is warp-collective)
  const long long np = (n + 31) & ~31LL;
  OHM_GRID_STRIDE(i, np) tsdf_walk_ray(m, i, i < n);
}

__global__ void __launch_bounds__(kBlock) k_tsdf_apply(DeviceMap m) {
  chain_enter();
  if (latched(m)) return;
  const long long nt = touched_count(m);
  OHM_GRID_STRIDE(t, nt) tsdf_apply_one(m, t);
}

__global__ void k_end(DeviceMap m) {
  chain_enter();
  if (!latched(m)) return;
  rollback_call(m, (long long)blockIdx.x * blockDim.x + threadIdx.x, (long long)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Query and export.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_query(DeviceMap m, const float* pts, long long n, float* occupancy,
                                                   uint8_t* known, float* ndt, float* tsdf, uint32_t* counts,
                                                   unsigned long long* path_sum, float* mean) {
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
    if (slot >= 0 && (m.layers & kLayerOcc)) l = logodds_read(m.occ[off], m.l_min);
    if (occupancy) occupancy[i] = l;
    if (known) known[i] = (l == l) ? 1 : 0;
  }
  if (path_sum) path_sum[i] = (slot >= 0 && (m.layers & kLayerDecay)) ? m.decay[off] : 0ULL;
  if (mean) {
    const unsigned long long w = (slot >= 0 && (m.layers & kLayerMean)) ? m.vmean[off] : 0ULL;
    const unsigned long long cnt = w >> 32;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double frac = ((double)((w >> (10 * k)) & 1023ULL) + 0.5) / 1024.0;
      mean[4 * i + k] = cnt ? (float)(m.origin[k] + ((double)v[k] + frac) * m.voxel_size) : __int_as_float(0x7fc00000);
    }
    mean[4 * i + 3] = (float)cnt;
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
                                                    float* occupancy, uint32_t* counts, long long* ndt, float* tsdf,
                                                    unsigned long long* path_sum, unsigned long long* mean) {
  const long long total = count * kRegionVoxels;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / kRegionVoxels;
    const int32_t lin = (int32_t)(t % kRegionVoxels);
    const int32_t slot = (int32_t)(first + r);
    const uint32_t mo = morton(lin & 31, (lin >> 5) & 31, lin >> 10);
    const long long off = voxel_offset(slot, mo);
    if (keys && lin < 3) keys[3 * r + lin] = m.region_coords[3 * slot + lin];
    if (occupancy) occupancy[t] = (m.layers & kLayerOcc) ? logodds_read(m.occ[off], m.l_min) : __int_as_float(0x7fc00000);
    if (counts) {
      const unsigned long long c = (m.layers & kLayerCounts) ? m.counts[off] : 0ULL;
      counts[2 * t + 0] = (uint32_t)(c >> 32);
      counts[2 * t + 1] = (uint32_t)(c & 0xffffffffu);
    }
    if (path_sum) path_sum[t] = (m.layers & kLayerDecay) ? m.decay[off] : 0ULL;
    if (mean) mean[t] = (m.layers & kLayerMean) ? m.vmean[off] : 0ULL;
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
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_walk_fast<true, false, false>, kBlock, 0);
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
  map->profile_call += 1;  // the call's index for sampled stage timing
  const bool occ = (m.layers & kLayerOcc) != 0, cnt = (m.layers & kLayerCounts) != 0, ndt = (m.layers & kLayerNdt) != 0;
  const bool tsdf = (m.layers & kLayerTsdf) != 0;
  const bool mean = (m.layers & kLayerMean) != 0;
  const bool occ_like = occ || cnt || ndt || mean || (m.layers & kLayerDecay);
  const long long n = args.n;
  const int grid = map->walk_blocks;
  // the walk's grid-stride loop runs on OHM_WALK_OVERSUBSCRIBE times the
  // resident blocks: a block whose segments took longer holds its SM while
  // blocks that finished early are replaced by new ones (no long tail)
  const int wgrid = grid * OHM_WALK_OVERSUBSCRIBE;
  const long long per_ray_blocks = blocks_for(n) > 0 ? blocks_for(n) : 1;
  const int ray_grid = (int)(per_ray_blocks < grid ? per_ray_blocks : grid);
  const unsigned prb = (unsigned)per_ray_blocks;
  OHM_LAUNCH(OHM_STAGE_BEGIN, launch_chained(k_begin, 1, stream, m, args));
  if (occ_like) {
    OHM_LAUNCH(OHM_STAGE_PREPARE, launch_chained(k_prepare_occ, prb, stream, m, args));
    if (ndt) OHM_LAUNCH(OHM_STAGE_NDT_ALLOC, launch_chained(k_ndt_alloc, kNdtPendingGrid, stream, m));
  }
  if (tsdf) OHM_LAUNCH(OHM_STAGE_PREPARE_TSDF, launch_chained(k_prepare_tsdf, prb, stream, m, args));
  const bool dec = (m.layers & kLayerDecay) != 0;
  if (dec) {
    const int sel = (occ ? 2 : 0) | (cnt ? 1 : 0);
    switch (sel) {
      case 3: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_miss<true, true, true>, wgrid, stream, m)); break;
      case 2: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_miss<true, false, true>, wgrid, stream, m)); break;
      case 1: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_miss<false, true, true>, wgrid, stream, m)); break;
      default: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_miss<false, false, true>, wgrid, stream, m)); break;
    }
  } else if (occ || cnt) {
    const bool c = walk_needs_cas(m.layers, m.miss, m.ndt_clear);
    const int sel = (occ ? 4 : 0) | (cnt ? 2 : 0) | (c ? 1 : 0);
    switch (sel) {
      case 7: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_fast<true, true, true>, wgrid, stream, m)); break;
      case 6: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_fast<true, true, false>, wgrid, stream, m)); break;
      case 5: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_fast<true, false, true>, wgrid, stream, m)); break;
      case 4: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_fast<true, false, false>, wgrid, stream, m)); break;
      default: OHM_LAUNCH(OHM_STAGE_WALK, launch_chained(k_walk_fast<false, true, false>, wgrid, stream, m)); break;
    }
  }
  if (occ || cnt || ndt || mean) {
    const int sel = (occ ? 4 : 0) | (cnt ? 2 : 0) | (ndt ? 1 : 0);
    switch (sel) {
      case 7: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<true, true, true>, ray_grid, stream, m, n)); break;
      case 6: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<true, true, false>, ray_grid, stream, m, n)); break;
      case 5: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<true, false, true>, ray_grid, stream, m, n)); break;
      case 4: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<true, false, false>, ray_grid, stream, m, n)); break;
      case 3: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<false, true, true>, ray_grid, stream, m, n)); break;
      case 2: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<false, true, false>, ray_grid, stream, m, n)); break;
      case 1: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<false, false, true>, ray_grid, stream, m, n)); break;
      default: OHM_LAUNCH(OHM_STAGE_HITS, launch_chained(k_hits<false, false, false>, ray_grid, stream, m, n)); break;
    }
    if (mean) OHM_LAUNCH(OHM_STAGE_MEAN_APPLY, launch_chained(k_mean_apply, ray_grid, stream, m));
  }
  if (tsdf) {
    OHM_LAUNCH(OHM_STAGE_TSDF_WALK, launch_chained(k_tsdf_walk, ray_grid, stream, m, n));
    OHM_LAUNCH(OHM_STAGE_TSDF_APPLY, launch_chained(k_tsdf_apply, grid, stream, m));
  }
  // one block per SM: the body only runs (a grid-stride rollback) after a failure
  OHM_LAUNCH(OHM_STAGE_END, launch_chained(k_end, (unsigned)map->num_sms, stream, m));
  return cudaGetLastError();
}

// 64-bit finaliser of SplitMix64 (Steele, Lea, Flood 2014), a published mixer.
__device__ __forceinline__ unsigned long long splitmix64_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// Throughput probe: per round, four random words are loaded, then each is
// compare-and-swapped to its value + 1.
__global__ void __launch_bounds__(kBlock, 4) k_probe_cas(unsigned int* buf, unsigned long long mask, int rounds) {
  const unsigned long long threads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < rounds; ++r) {
    unsigned long long a[4];
    unsigned int old[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) a[j] = splitmix64_mix((unsigned long long)r * threads * 4 + t * 4 + j) & mask;
#pragma unroll
    for (int j = 0; j < 4; ++j) old[j] = buf[a[j]];
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicCAS(buf + a[j], old[j], old[j] + 1u);
  }
}

cudaError_t probe_cas_rate(int device, long long words, long long ops, double* rate) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  const unsigned long long threads = (unsigned long long)sms * 4 * kBlock;
  int rounds = (int)(ops / (long long)(threads * 4));
  if (rounds < 1) rounds = 1;
  unsigned int* buf = nullptr;
  e = cudaMalloc(reinterpret_cast<void**>(&buf), sizeof(unsigned int) * (size_t)words);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemset(buf, 0, sizeof(unsigned int) * (size_t)words);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_probe_cas<<<sms * 4, kBlock>>>(buf, (unsigned long long)words - 1, rounds);  // warm-up
    cudaEventRecord(e0);
    k_probe_cas<<<sms * 4, kBlock>>>(buf, (unsigned long long)words - 1, rounds);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
  }
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) *rate = (double)threads * 4.0 * rounds / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return e;
}

// Probe kernels for ohm_probe_rate; per round each thread touches kProbeInFlight
// random locations: a float atomic add of 1 to a word (fire and forget), a
// load then compare-and-swap of a word, or a load of a word of a random
// 32-byte sector then a store of it plus one (the sector is read from and
// written back to memory when the buffer is larger than L2).
constexpr int kProbeInFlight = 8;
template <int kKind>
__global__ void __launch_bounds__(kBlock) k_probe(unsigned int* buf, unsigned long long mask, int rounds) {
  const unsigned long long threads = (unsigned long long)gridDim.x * blockDim.x;
  const unsigned long long t = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (int r = 0; r < rounds; ++r) {
    unsigned long long a[kProbeInFlight];
#pragma unroll
    for (int j = 0; j < kProbeInFlight; ++j)
      a[j] = splitmix64_mix(((unsigned long long)r * threads + t) * kProbeInFlight + j) & mask;
    if (kKind == OHM_PROBE_L2_ADD) {
#pragma unroll
      for (int j = 0; j < kProbeInFlight; ++j) atomicAdd(reinterpret_cast<float*>(buf) + a[j], 1.0f);
    } else {
      unsigned int old[kProbeInFlight];
      if (kKind == OHM_PROBE_SECTOR_RMW) {
#pragma unroll
        for (int j = 0; j < kProbeInFlight; ++j) a[j] = (a[j] << 3) | (t & 7);  // word t % 8 of sector a
      }
#pragma unroll
      for (int j = 0; j < kProbeInFlight; ++j) old[j] = buf[a[j]];
#pragma unroll
      for (int j = 0; j < kProbeInFlight; ++j) {
        if (kKind == OHM_PROBE_L2_CAS)
          atomicCAS(buf + a[j], old[j], old[j] + 1u);
        else
          buf[a[j]] = old[j] + 1u;
      }
    }
  }
}

cudaError_t probe_rate(int device, int kind, long long units, long long ops, double* rate) {
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  const int blocks = sms * 8;
  const unsigned long long threads = (unsigned long long)blocks * kBlock;
  int rounds = (int)(ops / (long long)(threads * kProbeInFlight));
  if (rounds < 1) rounds = 1;
  const long long words = kind == OHM_PROBE_SECTOR_RMW ? units * 8 : units;
  unsigned int* buf = nullptr;
  e = cudaMalloc(reinterpret_cast<void**>(&buf), sizeof(unsigned int) * (size_t)words);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMemset(buf, 0, sizeof(unsigned int) * (size_t)words);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const unsigned long long mask = (unsigned long long)units - 1;
  auto launch = [&]() {
    if (kind == OHM_PROBE_L2_ADD)
      k_probe<OHM_PROBE_L2_ADD><<<blocks, kBlock>>>(buf, mask, rounds);
    else if (kind == OHM_PROBE_L2_CAS)
      k_probe<OHM_PROBE_L2_CAS><<<blocks, kBlock>>>(buf, mask, rounds);
    else
      k_probe<OHM_PROBE_SECTOR_RMW><<<blocks, kBlock>>>(buf, mask, rounds);
  };
  float best = 0.f;
  if (e == cudaSuccess) {
    launch();  // warm-up (and L2 fill for the L2-resident kinds)
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      cudaEventRecord(e0);
      launch();
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) *rate = (double)threads * kProbeInFlight * rounds / (best * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  return e;
}

cudaError_t launch_query(ohm_map* map, const float* points, long long n, float* occupancy, uint8_t* known, float* ndt,
                         float* tsdf, uint32_t* counts, unsigned long long* path_sum, float* mean,
                         cudaStream_t stream) {
  if (n > 0)
    k_query<<<(unsigned)blocks_for(n), kBlock, 0, stream>>>(map->d, points, n, occupancy, known, ndt, tsdf, counts,
                                                            path_sum, mean);
  return cudaGetLastError();
}

cudaError_t launch_export(ohm_map* map, long long first, long long count, int32_t* keys, float* occupancy,
                          uint32_t* counts, long long* ndt, float* tsdf, unsigned long long* path_sum,
                          unsigned long long* mean, cudaStream_t stream) {
  if (count > 0) {
    long long b = blocks_for(count * kRegionVoxels);
    if (b > 65535LL * 16) b = 65535LL * 16;
    k_export<<<(unsigned)b, kBlock, 0, stream>>>(map->d, first, count, keys, occupancy, counts, ndt, tsdf, path_sum,
                                                  mean);
  }
  return cudaGetLastError();
}

}  // namespace ohm
