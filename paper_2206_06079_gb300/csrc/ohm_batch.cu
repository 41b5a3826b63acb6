// Multi-map batched integration: one step integrates one ray set into each of
// up to 32 independent maps with one launch per kernel stage for all maps, and
// the whole step is captured once into a CUDA graph and replayed.
//
// Work of all maps shares one index space per stage.  Rays: map i owns the
// range [R_i, R_i + pad32(n_i)) so that a warp never spans two maps (the
// segment reservation of the prepare stage is warp-aggregated per map).
// Segments, samples and touched TSDF voxels: plain concatenation.  Each block
// stages the maps' descriptors in shared memory and finds the map of an index
// by a scan over at most 32 prefix sums.
//
// Per-step inputs (device pointers and ray counts per map) live in a small
// device-resident table copied before each graph launch, so the graph itself
// never changes between steps; the tile parameters (segment length, walk grid)
// are fixed into it and changed by ohm_batch_tune, which re-captures.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "ohm_kernels.cuh"

namespace ohm {

constexpr int kMaxBatchMaps = OHM_BATCH_MAX_MAPS;

struct BatchDesc {
  int32_t n_maps;
  DeviceMap maps[kMaxBatchMaps];
};

struct BatchStep {
  const float* origins[kMaxBatchMaps];
  const float* endpoints[kMaxBatchMaps];
  const uint8_t* flags[kMaxBatchMaps];
  long long n[kMaxBatchMaps];
  long long n_origins[kMaxBatchMaps];
};

namespace {

// Shared-memory copy of the maps and of one prefix table.
struct BatchShared {
  DeviceMap maps[kMaxBatchMaps];
  long long pref[kMaxBatchMaps + 1];
  int32_t n_maps;
};

enum PrefixKind { kRaysPadded, kRays, kSegments, kTouched, kMeanTouched, kNdtPending };

// Load the descriptors and build the prefix table of the requested kind
// (segments: of the maps whose walk is `variant` only, unless it is kAnyWalk).
constexpr int kAnyWalk = -2;
__device__ void batch_stage(BatchShared& sh, const BatchDesc* desc, const BatchStep* step, PrefixKind kind,
                            int variant = kAnyWalk) {
  const int nm = desc->n_maps;
  const int words = (int)(sizeof(DeviceMap) / sizeof(int)) * nm;
  const int* src = reinterpret_cast<const int*>(desc->maps);
  int* dst = reinterpret_cast<int*>(sh.maps);
  for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  if (threadIdx.x == 0) {
    sh.n_maps = nm;
    long long acc = 0;
    for (int i = 0; i < nm; ++i) {
      sh.pref[i] = acc;
      long long c = 0;
      const DeviceMap& m = desc->maps[i];
      const bool live = *(volatile int32_t*)m.status == 0;
      if (kind == kRaysPadded)
        c = (step->n[i] + 31) & ~31LL;
      else if (kind == kRays)
        c = live ? step->n[i] : 0;
      else if (kind == kSegments)
        c = live && (variant == kAnyWalk || walk_variant(m.layers, m.miss, m.ndt_clear) == variant)
                ? (long long)m.calls->segments
                : 0;
      else if (kind == kNdtPending)
        c = live && (m.layers & kLayerNdt) ? (long long)m.calls->ndt_pending : 0;
      else if (kind == kMeanTouched)
        c = (m.layers & kLayerMean) ? mean_touched_count(m) : 0;  // failed maps too: their sums are cleared
      else
        c = live ? touched_count(m) : 0;
      acc += c;
    }
    sh.pref[nm] = acc;
  }
  __syncthreads();
}

__device__ __forceinline__ int batch_find(const BatchShared& sh, long long g) {
  int i = 0;
  while (i + 1 < sh.n_maps && sh.pref[i + 1] <= g) ++i;
  return i;
}

__device__ __forceinline__ CallArgs batch_args(const BatchStep* step, int i) {
  CallArgs a;
  a.origins = step->origins[i];
  a.endpoints = step->endpoints[i];
  a.flags = step->flags[i];
  a.n = step->n[i];
  a.n_origins = step->n_origins[i];
  return a;
}

#define OHM_BATCH_STRIDE(g, total) \
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < (total); g += (long long)gridDim.x * blockDim.x)

// Chained like the stage kernels after it (its launch overlaps the tail of the
// previous step's last kernel).
__global__ void k_batch_begin(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  const int i = threadIdx.x;
  if (blockIdx.x == 0 && i < desc->n_maps) begin_call(desc->maps[i], batch_args(step, i));
}

// One instantiation per pass (occupancy-like layers, or the TSDF band), so
// that each kernel holds only its own per-ray code.
template <bool kTsdf>
__global__ void __launch_bounds__(kBlock, OHM_PREPARE_MIN_BLOCKS) k_batch_prepare(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kRaysPadded);
  const long long total = sh.pref[sh.n_maps];  // a multiple of 32: whole warps iterate together
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    const long long i = g - sh.pref[mi];
    const CallArgs a = batch_args(step, mi);
    const bool active = i < a.n;
    if constexpr (kTsdf) {
      if (m.layers & kLayerTsdf) prepare_tsdf_ray(m, a, i, active);
    } else {
      if (m.layers & (kLayerOcc | kLayerCounts | kLayerNdt | kLayerDecay | kLayerMean)) prepare_occ_ray(m, a, i, active);
    }
  }
}

// The sample rays each map's prepare listed (their region was being inserted
// by another thread): their regions get NDT blocks here.
__global__ void __launch_bounds__(kBlock) k_batch_ndt_alloc(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kNdtPending);
  const long long total = sh.pref[sh.n_maps];
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    ndt_alloc_ray(m, m.ndt_pending[g - sh.pref[mi]]);
  }
}

// Miss walk of the maps with the decay layer (walk_segment).
__global__ void __launch_bounds__(kBlock, OHM_WALK_MIN_BLOCKS) k_batch_walk(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kSegments, kWalkDecay);
  const long long total = sh.pref[sh.n_maps];
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    const long long si = g - sh.pref[mi];
    unsigned int cas = 0;  // not attributed per map in a batched step
    const bool occ = (m.layers & kLayerOcc) != 0, cnt = (m.layers & kLayerCounts) != 0;
    if (occ && cnt)
      walk_segment<true, true, true>(m, si, cas);
    else if (occ)
      walk_segment<true, false, true>(m, si, cas);
    else if (cnt)
      walk_segment<false, true, true>(m, si, cas);
    else
      walk_segment<false, false, true>(m, si, cas);
  }
}

// Filtered miss walk of the maps whose walk is kVariant (walk_variant): one
// launch per variant present in the batch, so that each kernel holds only its
// own update code (one kernel for every variant spills heavily).
#ifndef OHM_BATCH_PIPE
#define OHM_BATCH_PIPE false
#endif
template <int kVariant>
__global__ void __launch_bounds__(kBlock, OHM_FAST_MIN_BLOCKS) k_batch_walk_fast(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kSegments, kVariant);
  const long long total = sh.pref[sh.n_maps];
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    unsigned int ops = 0;  // not attributed per map in a batched step
    walk_segment_fast<(kVariant & 4) != 0, (kVariant & 2) != 0, (kVariant & 1) != 0, OHM_BATCH_PIPE>(
        m, m.segs[g - sh.pref[mi]], ops);
  }
}

__global__ void __launch_bounds__(kBlock) k_batch_hits(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kRaysPadded);
  const long long total = sh.pref[sh.n_maps];  // a multiple of 32: whole warps iterate together
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    const long long i = g - sh.pref[mi];
    const bool a = i < step->n[mi] && !latched(m);
    const int sel = ((m.layers & kLayerOcc) ? 4 : 0) | ((m.layers & kLayerCounts) ? 2 : 0) | ((m.layers & kLayerNdt) ? 1 : 0);
    switch (sel) {
      case 7: hit_ray<true, true, true>(m, i, a); break;
      case 6: hit_ray<true, true, false>(m, i, a); break;
      case 5: hit_ray<true, false, true>(m, i, a); break;
      case 4: hit_ray<true, false, false>(m, i, a); break;
      case 3: hit_ray<false, true, true>(m, i, a); break;
      case 2: hit_ray<false, true, false>(m, i, a); break;
      case 1: hit_ray<false, false, true>(m, i, a); break;
      default:
        if (m.layers & kLayerMean) hit_ray<false, false, false>(m, i, a);
        break;
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_batch_mean_apply(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kMeanTouched);
  const long long total = sh.pref[sh.n_maps];
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    mean_apply_one(m, g - sh.pref[mi], !latched(m));
  }
}

__global__ void __launch_bounds__(kBlock) k_batch_tsdf_walk(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kRaysPadded);
  const long long total = sh.pref[sh.n_maps];  // a multiple of 32: whole warps iterate together
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    const long long i = g - sh.pref[mi];
    if (m.layers & kLayerTsdf) tsdf_walk_ray(m, i, i < step->n[mi] && !latched(m));
  }
}

__global__ void __launch_bounds__(kBlock) k_batch_tsdf_apply(const BatchDesc* desc, const BatchStep* step) {
  chain_enter();
  __shared__ BatchShared sh;
  batch_stage(sh, desc, step, kTouched);
  const long long total = sh.pref[sh.n_maps];
  OHM_BATCH_STRIDE(g, total) {
    const int mi = batch_find(sh, g);
    const DeviceMap& m = sh.maps[mi];
    if (m.layers & kLayerTsdf) tsdf_apply_one(m, g - sh.pref[mi]);
  }
}

// One group of blocks per map rolls back that map if its call failed.
__global__ void k_batch_end(const BatchDesc* desc) {
  chain_enter();
  const int per_map = gridDim.x / kMaxBatchMaps;
  const int mi = blockIdx.x / per_map;
  if (mi >= desc->n_maps) return;
  const DeviceMap& m = desc->maps[mi];
  if (!latched(m)) return;
  const long long b = blockIdx.x % per_map;
  rollback_call(m, b * blockDim.x + threadIdx.x, (long long)per_map * blockDim.x);
}

}  // namespace
}  // namespace ohm

struct ohm_batch {
  int32_t n_maps;
  int device;
  ohm_map* maps[OHM_BATCH_MAX_MAPS];
  ohm::BatchDesc* d_desc;
  ohm::BatchStep* d_step;
  ohm::BatchStep h_step;       // pageable: its copy is staged before the call returns
  int walk_blocks_per_sm;
  int num_sms;
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool have_exec;
  bool any_ndt, any_tsdf, any_occ, any_mean;
  uint32_t walk_variants;      // bit v: some map's walk is variant v (walk_variant)
  long long launches;
  long long graph_launches;
  int graph_kernels;           // kernel nodes in the captured step
};

namespace {

ohm_status bfail(ohm_status code, const std::string& msg) {
  ohm::set_last_error(msg);
  return code;
}

cudaError_t write_desc(ohm_batch* b) {
  ohm::BatchDesc h;
  std::memset(&h, 0, sizeof(h));
  h.n_maps = b->n_maps;
  for (int i = 0; i < b->n_maps; ++i) h.maps[i] = b->maps[i]->d;
  cudaError_t e = cudaMemcpy(b->d_desc, &h, sizeof(h), cudaMemcpyHostToDevice);
  return e;
}

void drop_graph(ohm_batch* b) {
  if (b->have_exec) {
    cudaGraphExecDestroy(b->exec);
    cudaGraphDestroy(b->graph);
    b->have_exec = false;
  }
}

// The kernels of one step, in stream order; returns their number in *count.
cudaError_t enqueue_step(ohm_batch* b, cudaStream_t s, int* count) {
  using namespace ohm;
  const int grid = b->num_sms * b->walk_blocks_per_sm;
  const int ray_grid = b->num_sms * 4;
  launch_chained(k_batch_begin, 1, s, b->d_desc, b->d_step);
  int n = 1;
  if (b->any_occ || b->any_ndt || b->any_mean) {
    launch_chained(k_batch_prepare<false>, ray_grid, s, b->d_desc, b->d_step);
    ++n;
    if (b->any_ndt) {
      launch_chained(k_batch_ndt_alloc, (unsigned)b->num_sms, s, b->d_desc, b->d_step);
      ++n;
    }
  }
  if (b->any_tsdf) {
    launch_chained(k_batch_prepare<true>, ray_grid, s, b->d_desc, b->d_step);
    ++n;
  }
  // oversubscribed grid-stride launches, like the single-map walk
  const int wgrid = grid * OHM_WALK_OVERSUBSCRIBE;
  const uint32_t wv = b->walk_variants;
  if (wv & (1u << kWalkDecay)) launch_chained(k_batch_walk, wgrid, s, b->d_desc, b->d_step);
  if (wv & (1u << 7)) launch_chained(k_batch_walk_fast<7>, wgrid, s, b->d_desc, b->d_step);
  if (wv & (1u << 6)) launch_chained(k_batch_walk_fast<6>, wgrid, s, b->d_desc, b->d_step);
  if (wv & (1u << 5)) launch_chained(k_batch_walk_fast<5>, wgrid, s, b->d_desc, b->d_step);
  if (wv & (1u << 4)) launch_chained(k_batch_walk_fast<4>, wgrid, s, b->d_desc, b->d_step);
  if (wv & (1u << 2)) launch_chained(k_batch_walk_fast<2>, wgrid, s, b->d_desc, b->d_step);
  n += __builtin_popcount(wv);
  if (b->any_occ || b->any_ndt || b->any_mean) {
    launch_chained(k_batch_hits, ray_grid, s, b->d_desc, b->d_step);
    ++n;
  }
  if (b->any_mean) {
    launch_chained(k_batch_mean_apply, ray_grid, s, b->d_desc, b->d_step);
    ++n;
  }
  if (b->any_tsdf) {
    launch_chained(k_batch_tsdf_walk, ray_grid, s, b->d_desc, b->d_step);
    launch_chained(k_batch_tsdf_apply, ray_grid, s, b->d_desc, b->d_step);
    n += 2;
  }
  launch_chained(k_batch_end, kMaxBatchMaps * 8, s, b->d_desc);
  ++n;
  *count = n;
  return cudaGetLastError();
}

struct BatchGuard {
  int prev = -1;
  explicit BatchGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~BatchGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

ohm_status ohm_batch_create(ohm_map* const* maps, int32_t n_maps, ohm_batch** out) {
  if (!maps || !out) return bfail(OHM_ERR_INVALID, "batch_create: NULL argument");
  *out = nullptr;
  if (n_maps < 1 || n_maps > OHM_BATCH_MAX_MAPS)
    return bfail(OHM_ERR_INVALID, "batch_create: n_maps must be in [1, OHM_BATCH_MAX_MAPS]");
  for (int i = 0; i < n_maps; ++i) {
    if (!maps[i]) return bfail(OHM_ERR_INVALID, "batch_create: NULL map");
    if (maps[i]->device != maps[0]->device) return bfail(OHM_ERR_INVALID, "batch_create: maps on different devices");
    for (int j = 0; j < i; ++j)
      if (maps[j] == maps[i]) return bfail(OHM_ERR_INVALID, "batch_create: a map appears twice");
  }
  BatchGuard guard(maps[0]->device);
  ohm_batch* b = new ohm_batch();
  b->n_maps = n_maps;
  b->device = maps[0]->device;
  for (int i = 0; i < n_maps; ++i) {
    b->maps[i] = maps[i];
    const uint32_t L = maps[i]->p.layers;
    b->any_occ = b->any_occ || (L & (OHM_LAYER_OCCUPANCY | OHM_LAYER_COUNTS | OHM_LAYER_DECAY));
    b->any_ndt = b->any_ndt || (L & OHM_LAYER_NDT);
    b->any_tsdf = b->any_tsdf || (L & OHM_LAYER_TSDF);
    b->any_mean = b->any_mean || (L & OHM_LAYER_MEAN);
    const int v = ohm::walk_variant(maps[i]->d.layers, maps[i]->d.miss, maps[i]->d.ndt_clear);
    if (v != ohm::kWalkNone) b->walk_variants |= 1u << v;
  }
  b->walk_blocks_per_sm = ohm::walk_blocks_per_sm();
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&b->d_desc), sizeof(ohm::BatchDesc));
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&b->d_step), sizeof(ohm::BatchStep));
  if (e == cudaSuccess) e = cudaMemset(b->d_step, 0, sizeof(ohm::BatchStep));
  if (e == cudaSuccess) e = write_desc(b);
  if (e != cudaSuccess) {
    ohm_batch_destroy(b);
    return bfail(OHM_ERR_CUDA, std::string("batch_create: ") + cudaGetErrorString(e));
  }
  *out = b;
  return OHM_OK;
}

void ohm_batch_destroy(ohm_batch* b) {
  if (!b) return;
  BatchGuard guard(b->device);
  cudaDeviceSynchronize();
  drop_graph(b);
  if (b->d_desc) cudaFree(b->d_desc);
  if (b->d_step) cudaFree(b->d_step);
  delete b;
}

ohm_status ohm_batch_tune(ohm_batch* b, int32_t segment_steps, int32_t walk_blocks_per_sm) {
  if (!b) return bfail(OHM_ERR_INVALID, "batch_tune: batch is NULL");
  if (segment_steps < 0 || walk_blocks_per_sm < 0 || walk_blocks_per_sm > 64)
    return bfail(OHM_ERR_INVALID, "batch_tune: bad parameters");
  BatchGuard guard(b->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return bfail(OHM_ERR_CUDA, std::string("batch_tune: ") + cudaGetErrorString(e));
  if (segment_steps > 0) {
    for (int i = 0; i < b->n_maps; ++i) {
      ohm_map* m = b->maps[i];
      const long long vox_steps = (long long)std::ceil(m->p.max_range / m->p.voxel_size) + 2;
      const long long need = m->p.max_rays * (vox_steps / std::max(1, segment_steps / 3) + 1);
      if (need > m->d.max_segs) {
        int2* segs = nullptr;
        e = cudaMalloc(reinterpret_cast<void**>(&segs), sizeof(int2) * need);
        if (e != cudaSuccess) return bfail(OHM_ERR_CUDA, std::string("batch_tune: ") + cudaGetErrorString(e));
        cudaFree(m->d.segs);
        m->d.segs = segs;
        m->d.max_segs = need;
      }
      m->d.seg_steps = segment_steps;
      m->p.segment_steps = segment_steps;
    }
  }
  if (walk_blocks_per_sm > 0) b->walk_blocks_per_sm = walk_blocks_per_sm;
  e = write_desc(b);
  if (e != cudaSuccess) return bfail(OHM_ERR_CUDA, std::string("batch_tune: ") + cudaGetErrorString(e));
  drop_graph(b);
  return OHM_OK;
}

ohm_status ohm_batch_integrate(ohm_batch* b, const float* const* origins, const int64_t* n_origins,
                               const float* const* endpoints, const uint8_t* const* flags, const int64_t* n,
                               int32_t use_graph, void* stream) {
  if (!b || !origins || !n_origins || !endpoints || !n) return bfail(OHM_ERR_INVALID, "batch_integrate: NULL argument");
  for (int i = 0; i < b->n_maps; ++i) {
    if (n[i] < 0 || n[i] > b->maps[i]->p.max_rays)
      return bfail(OHM_ERR_INVALID, "batch_integrate: n[i] outside [0, max_rays of map i]");
    if (n[i] > 0 && (!origins[i] || !endpoints[i] || (n_origins[i] != 1 && n_origins[i] != n[i])))
      return bfail(OHM_ERR_INVALID, "batch_integrate: bad inputs for map " + std::to_string(i));
  }
  if (use_graph && !stream)
    return bfail(OHM_ERR_INVALID, "batch_integrate: graph mode needs a created stream (the legacy default stream cannot be captured)");
  BatchGuard guard(b->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->n_maps; ++i) {
    b->h_step.origins[i] = origins[i];
    b->h_step.endpoints[i] = endpoints[i];
    b->h_step.flags[i] = flags ? flags[i] : nullptr;
    b->h_step.n[i] = n[i];
    b->h_step.n_origins[i] = n_origins[i];
  }
  cudaError_t e = cudaMemcpyAsync(b->d_step, &b->h_step, sizeof(ohm::BatchStep), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return bfail(OHM_ERR_CUDA, std::string("batch_integrate: ") + cudaGetErrorString(e));
  if (!use_graph) {
    int count = 0;
    e = enqueue_step(b, s, &count);
    b->launches += count;
  } else {
    if (!b->have_exec) {
      // Capture the step once; later steps replay it.
      e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t el = enqueue_step(b, s, &b->graph_kernels);
        e = cudaStreamEndCapture(s, &b->graph);
        if (e == cudaSuccess) e = el;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e == cudaSuccess) b->have_exec = true;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
    if (e == cudaSuccess) {
      b->graph_launches += 1;
      b->launches += b->graph_kernels;
    }
  }
  if (e != cudaSuccess) return bfail(OHM_ERR_CUDA, std::string("batch_integrate: ") + cudaGetErrorString(e));
  for (int i = 0; i < b->n_maps; ++i) ohm::note_work(b->maps[i], s);
  return OHM_OK;
}

ohm_status ohm_batch_sync(ohm_batch* b, void* stream) {
  if (!b) return bfail(OHM_ERR_INVALID, "batch_sync: batch is NULL");
  ohm_status first = OHM_OK;
  for (int i = 0; i < b->n_maps; ++i) {
    ohm_status st = ohm_map_sync(b->maps[i], stream);
    if (st != OHM_OK && first == OHM_OK) first = st;
  }
  return first;
}

ohm_status ohm_batch_stats(ohm_batch* b, int64_t* kernel_launches, int64_t* graph_launches) {
  if (!b || !kernel_launches || !graph_launches) return bfail(OHM_ERR_INVALID, "batch_stats: NULL argument");
  *kernel_launches = b->launches;
  *graph_launches = b->graph_launches;
  return OHM_OK;
}

}  // extern "C"
