// Allocation-free ray counting into a caller-owned dense grid.
//
// Some callers cannot call cudaMalloc at the moment they need to integrate
// rays: code that runs while a stream is being captured into a CUDA graph
// (allocation calls are not allowed there), real-time loops that must not
// block on the allocator or on the device synchronisation cudaFree implies,
// and plug-ins whose host application hands all device memory to its own
// allocator.  For them, ohm_count_rays_noalloc walks a ray set exactly like
// ohm_integrate_rays and adds each ray's per-voxel hit and miss counts into
// two uint32 arrays the caller owns.  Its per-call working memory (quantised
// ray records and the ray-segment table) lives in one statically sized
// device array defined below, so the call allocates nothing.
//
// That array is a file-scope __device__ variable: every GPU that loads this
// library holds it (kNoAllocScratchBytes, about 3 MB) until the process
// exits.  Every call shares it, and it keeps whatever the last call wrote:
// the segment counter is cleared at the start of each call, and calls whose
// work overlaps on the GPU (different streams, no ordering between them)
// race on it and must not be issued.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "ohm_host.h"

namespace ohm {
namespace {

constexpr long long kNoAllocMaxRays = OHM_NOALLOC_MAX_RAYS;
constexpr long long kNoAllocMaxSegments = 4 * kNoAllocMaxRays;
constexpr int kNoAllocBlock = 256;

// Layout of the static array: [counter (256 B)] [ray records] [segments].
constexpr size_t kCounterBytes = 256;
constexpr size_t kRaysBytes = sizeof(EndpointRec) * kNoAllocMaxRays;
constexpr size_t kSegsBytes = sizeof(int2) * kNoAllocMaxSegments;
constexpr size_t kNoAllocScratchBytes = kCounterBytes + kRaysBytes + kSegsBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct CountGrid {
  double origin[3];
  double scale;
  double rmax_q;
  int32_t frac_bits;
  int32_t seg_steps;
  long long corner[3];
  long long dims[3];
};

struct NoAllocArgs {
  const float* origins;
  const float* endpoints;
  const uint8_t* flags;
  long long n;
  long long n_origins;
};

__device__ __forceinline__ bool na_in_extent(const long long q[3], int F) {
  const long long lim = 1LL << 24;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    long long v = q[k] >> F;
    ok = ok && v > -lim && v < lim;
  }
  return ok;
}

// Per ray: quantise, truncate to the maximum range, append its segments.
__global__ void __launch_bounds__(kNoAllocBlock) k_noalloc_prepare(CountGrid g, NoAllocArgs a, unsigned char* scratch) {
  unsigned long long* nseg_total = reinterpret_cast<unsigned long long*>(scratch);
  EndpointRec* rays = reinterpret_cast<EndpointRec*>(scratch + kCounterBytes);
  int2* segs = reinterpret_cast<int2*>(scratch + kCounterBytes + kRaysBytes);
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int F = g.frac_bits;
  unsigned int nseg = 0;
  EndpointRec r;
  r.flags = 0;
  r.nseg = 0;
  if (i < a.n) {
    const long long oi = a.n_origins == 1 ? 0 : i;
    long long qo[3], qe[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float o = a.origins[3 * oi + k], e = a.endpoints[3 * i + k];
      ok = ok && isfinite(o) && isfinite(e) && quantise(o, g.origin[k], g.scale, &qo[k]) &&
           quantise(e, g.origin[k], g.scale, &qe[k]);
    }
    bool sample = !(a.flags && (a.flags[i] & kFlagNoReturn));
    if (ok) {
      double d[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) d[k] = (double)(qe[k] - qo[k]);
      double l2 = __dmul_rn(d[0], d[0]);
      l2 = __dadd_rn(l2, __dmul_rn(d[1], d[1]));
      l2 = __dadd_rn(l2, __dmul_rn(d[2], d[2]));
      const double len = __dsqrt_rn(l2);
      if (len > g.rmax_q) {
        const double ratio = __ddiv_rn(g.rmax_q, len);
#pragma unroll
        for (int k = 0; k < 3; ++k) qe[k] = qo[k] + __double2ll_rn(__dmul_rn(d[k], ratio));
        sample = false;
      }
      ok = na_in_extent(qo, F) && na_in_extent(qe, F);
    }
    if (ok) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        r.a[k] = qo[k];
        r.b[k] = qe[k];
      }
      int32_t nmaj;
      dominant_axis(qo, qe, F, &nmaj);
      nseg = (unsigned int)segment_count(nmaj, g.seg_steps);
      r.flags = kRayValid | (sample ? kRaySample : 0);
      r.nseg = (int32_t)nseg;
    }
    rays[i] = r;
  }
  // The host checked that no ray set can produce more than kNoAllocMaxSegments;
  // the guard keeps every store inside the table regardless.
  const unsigned long long base = warp_reserve(nseg_total, nseg);
  for (unsigned int j = 0; j < nseg; ++j)
    if (base + j < (unsigned long long)kNoAllocMaxSegments) segs[base + j] = make_int2((int)i, (int)j);
}

__device__ __forceinline__ void na_count(const CountGrid& g, uint32_t* arr, int32_t vx, int32_t vy, int32_t vz) {
  const long long x = vx - g.corner[0], y = vy - g.corner[1], z = vz - g.corner[2];
  if (x < 0 || y < 0 || z < 0 || x >= g.dims[0] || y >= g.dims[1] || z >= g.dims[2]) return;
  atomicAdd(arr + (x + g.dims[0] * (y + g.dims[1] * z)), 1u);
}

// Per segment: walk its voxels; every voxel takes a miss except the voxel
// holding the ray's sample, which takes a hit.
__global__ void __launch_bounds__(kNoAllocBlock) k_noalloc_walk(CountGrid g, unsigned char* scratch, uint32_t* hits,
                                                                uint32_t* misses) {
  const unsigned long long* nseg_total = reinterpret_cast<const unsigned long long*>(scratch);
  const EndpointRec* rays = reinterpret_cast<const EndpointRec*>(scratch + kCounterBytes);
  const int2* segs = reinterpret_cast<const int2*>(scratch + kCounterBytes + kRaysBytes);
  long long nseg = (long long)*nseg_total;
  if (nseg > kNoAllocMaxSegments) nseg = kNoAllocMaxSegments;
  const int F = g.frac_bits;
  for (long long si = (long long)blockIdx.x * blockDim.x + threadIdx.x; si < nseg;
       si += (long long)gridDim.x * blockDim.x) {
    const int2 sg = segs[si];
    const EndpointRec r = rays[sg.x];
    int32_t nmaj;
    const int M = dominant_axis(r.a, r.b, F, &nmaj);
    const bool last = sg.y == r.nseg - 1;
    const bool sample = (r.flags & kRaySample) != 0;
    Walker w;
    walker_init(w, r.a, r.b, F, M, (long long)sg.y * g.seg_steps);
    int32_t mrem = last ? 0x7fffffff : g.seg_steps - 1;
    for (;;) {
      if (sample && w.total == 0)
        na_count(g, hits, w.vx, w.vy, w.vz);
      else
        na_count(g, misses, w.vx, w.vy, w.vz);
      if (w.total == 0) break;
      const int axis = walker_choose(w);
      if (axis == M) {
        if (mrem == 0) break;
        --mrem;
      }
      int32_t c, s;
      walker_step(w, axis, &c, &s);
    }
  }
}

// Device address of the static array, looked up once per device.
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {nullptr};
int g_noalloc_grid[64] = {0};

}  // namespace
}  // namespace ohm

namespace {
ohm_status na_fail(ohm_status code, const std::string& msg) {
  ohm::set_last_error(msg);
  return code;
}
bool na_is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

extern "C" {

ohm_status ohm_count_rays_noalloc(const ohm_count_grid* grid, const float* origins, int64_t n_origins,
                                  const float* endpoints, const uint8_t* flags, int64_t n, uint32_t* hits,
                                  uint32_t* misses, void* stream) {
  using namespace ohm;
  if (!grid || !hits || !misses) return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: NULL grid or output");
  if (n < 0 || n > kNoAllocMaxRays)
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: n must be in [0, OHM_NOALLOC_MAX_RAYS = " +
                                        std::to_string(kNoAllocMaxRays) + "]");
  if (!(grid->voxel_size > 0.0) || grid->frac_bits < 8 || grid->frac_bits > 20 || !(grid->max_range > 0.0))
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: bad voxel_size / frac_bits / max_range");
  const int32_t S = grid->segment_steps == 0 ? 64 : grid->segment_steps;
  if (S < 1) return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: segment_steps must be >= 1");
  for (int k = 0; k < 3; ++k)
    if (grid->dims[k] < 1 || grid->dims[k] > (1LL << 20))
      return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: dims must be in [1, 2^20]");
  if ((double)grid->dims[0] * grid->dims[1] * grid->dims[2] > 4.0e9)
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: grid has more than 4e9 voxels");
  const double scale = std::ldexp(1.0, grid->frac_bits) / grid->voxel_size;
  if (grid->max_range * scale >= std::ldexp(1.0, 30))
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: max_range * 2^frac_bits / voxel_size must be < 2^30");
  // segments per ray <= (max_range / voxel_size + 2) / S + 1; the table must hold n of them
  const long long per_ray = (long long)std::ceil(grid->max_range / grid->voxel_size + 2.0) / S + 1;
  if (per_ray * n > kNoAllocMaxSegments)
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: n * segments per ray exceeds the static segment table (" +
                                        std::to_string(kNoAllocMaxSegments) + "); raise segment_steps or lower n");
  if (n == 0) return OHM_OK;
  if (!origins || !endpoints || (n_origins != 1 && n_origins != n))
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: bad origins / endpoints");
  const void* ins[] = {origins, endpoints, hits, misses};
  for (const void* p : ins)
    if (!na_is_device_pointer(p)) return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: buffers must be device memory");
  if (flags && !na_is_device_pointer(flags))
    return na_fail(OHM_ERR_INVALID, "count_rays_noalloc: flags must be device memory");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return na_fail(OHM_ERR_CUDA, "count_rays_noalloc: no current device");
  void* scratch = nullptr;
  int grid_blocks = 0;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      // First call on this device: resolve the static array's device address.
      cudaError_t e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return na_fail(OHM_ERR_CUDA, std::string("count_rays_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      int sms = 0, per_sm = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_noalloc_walk, kNoAllocBlock, 0);
      g_noalloc_grid[dev] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    }
    scratch = g_noalloc_ptr[dev];
    grid_blocks = g_noalloc_grid[dev];
  }
  CountGrid g;
  for (int k = 0; k < 3; ++k) {
    g.origin[k] = grid->map_origin[k];
    g.corner[k] = grid->corner[k];
    g.dims[k] = grid->dims[k];
  }
  g.scale = scale;
  g.rmax_q = grid->max_range * scale;
  g.frac_bits = grid->frac_bits;
  g.seg_steps = S;
  NoAllocArgs a;
  a.origins = origins;
  a.endpoints = endpoints;
  a.flags = flags;
  a.n = n;
  a.n_origins = n_origins;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(scratch, 0, kCounterBytes, s);  // segment counter starts at zero
  if (e != cudaSuccess) return na_fail(OHM_ERR_CUDA, std::string("count_rays_noalloc: ") + cudaGetErrorString(e));
  const unsigned blocks = (unsigned)((n + kNoAllocBlock - 1) / kNoAllocBlock);
  k_noalloc_prepare<<<blocks, kNoAllocBlock, 0, s>>>(g, a, static_cast<unsigned char*>(scratch));
  k_noalloc_walk<<<grid_blocks, kNoAllocBlock, 0, s>>>(g, static_cast<unsigned char*>(scratch), hits, misses);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(OHM_ERR_CUDA, std::string("count_rays_noalloc: launch: ") + cudaGetErrorString(e));
  return OHM_OK;
}

}  // extern "C"
