// C ABI of the ray-integration library: map lifetime, argument checks, host
// staging and status reporting.  Declared in include/ohm_gb.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "ohm_host.h"

namespace {

thread_local std::string g_last_error;

ohm_status fail(ohm_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

ohm_status cuda_fail(cudaError_t e, const char* where) {
  return fail(OHM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Makes the map's device current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Device memory of another GPU than `dev` (the map's): rejected rather than
// reached through peer access.
bool on_other_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice && a.device != dev;
}

template <typename T>
cudaError_t alloc(T** p, size_t count, int fill) {
  *p = nullptr;
  if (count == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemset(*p, fill, count * sizeof(T));
}

long long next_pow2(long long x) {
  long long p = 1;
  while (p < x) p <<= 1;
  return p;
}

void free_map(ohm_map* m) {
  if (!m) return;
  ohm::DeviceMap& d = m->d;
  void* ptrs[] = {d.htab, d.region_count, d.region_coords, d.occ, d.counts, d.decay, d.vmean, d.vmean_acc, d.mean_list, d.ndt_slot, d.ndt_count, d.ndt_pending,
                  d.ndt, d.tsdf, d.tsdf_cnt, d.tsdf_sum, d.grad, d.ndt_grad, d.status, d.calls, d.rays, d.decay_rays, d.trays, d.segs, d.touched,
                  d.stamp, d.born, d.ndt_born, d.free_slots, d.ndt_free, d.free_info, d.restore_keys,
                  m->stage_origins, m->stage_endpoints, m->stage_flags, m->hin_origins[0], m->hin_origins[1],
                  m->hin_endpoints[0], m->hin_endpoints[1], m->hin_flags[0], m->hin_flags[1], m->pxy};
  if (m->copy_stream) cudaStreamSynchronize(m->copy_stream);
  if (m->work_done) cudaEventDestroy(m->work_done);
  for (int s = 0; s < 2; ++s) {
    if (m->hin_copied[s]) cudaEventDestroy(m->hin_copied[s]);
    if (m->hin_free[s]) cudaEventDestroy(m->hin_free[s]);
  }
  if (m->copy_stream) cudaStreamDestroy(m->copy_stream);
  ohm::destroy_host_store(m);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->h_status) cudaFreeHost(m->h_status);
  if (m->h_calls) cudaFreeHost(m->h_calls);
  if (m->h_count) cudaFreeHost(m->h_count);
  for (auto& pe : m->pending) {
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  for (cudaEvent_t ev : m->event_pool) cudaEventDestroy(ev);
  delete m;
}

ohm_status status_from_bits(int bits) {
  if (bits == 0) return OHM_OK;
  std::string msg = "integrate failed, map unchanged:";
  if (bits & ohm::kStatusCapacity) msg += " region or NDT pool full;";
  if (bits & ohm::kStatusProbe) msg += " hash probe limit exceeded;";
  if (bits & ohm::kStatusScratch) msg += " internal scratch overflow;";
  if (bits & ohm::kStatusMissing) msg += " internal region lookup failure;";
  if (bits & ohm::kStatusCasLimit) msg += " internal CAS retry limit;";
  if (bits & ohm::kStatusRestore) msg += " it touched regions evicted to host memory (restore them and repeat it);";
  g_last_error = msg;
  if (bits & ohm::kStatusCapacity) return OHM_ERR_CAPACITY;
  if (bits == ohm::kStatusRestore) return OHM_ERR_EVICTED;
  if (bits & ohm::kStatusProbe) return OHM_ERR_PROBE_LIMIT;
  return OHM_ERR_CUDA;
}

ohm_status enqueue_integrate(ohm_map* map, const float* origins, int64_t n_origins, const float* endpoints,
                             const uint8_t* flags, int64_t n, cudaStream_t stream) {
  if (!map) return fail(OHM_ERR_INVALID, "integrate: map is NULL");
  if (n < 0 || n > map->p.max_rays) return fail(OHM_ERR_INVALID, "integrate: n outside [0, max_rays]");
  if (n == 0) return OHM_OK;
  if (!origins || !endpoints) return fail(OHM_ERR_INVALID, "integrate: origins/endpoints are NULL");
  if (n_origins != 1 && n_origins != n) return fail(OHM_ERR_INVALID, "integrate: n_origins must be 1 or n");
  ohm::CallArgs a;
  a.n = n;
  a.n_origins = n_origins;
  a.origins = origins;
  a.endpoints = endpoints;
  a.flags = flags;
  if (on_other_device(origins, map->device) || on_other_device(endpoints, map->device) ||
      on_other_device(flags, map->device))
    return fail(OHM_ERR_INVALID, "integrate: inputs are on another device than the map");
  const bool host_o = !is_device_pointer(origins), host_e = !is_device_pointer(endpoints);
  const bool host_f = flags && !is_device_pointer(flags);
  cudaError_t e = cudaSuccess;
  int slot = -1;
  if (host_o || host_e || host_f) {
    // copy into the staging slot not used by the previous call, on the copy
    // stream, once the kernels of the slot's last call are done with it
    slot = map->hin_next;
    map->hin_next ^= 1;
    cudaStream_t cs = map->copy_stream;
    e = cudaStreamWaitEvent(cs, map->hin_free[slot], 0);
    if (e == cudaSuccess && host_o) {
      e = cudaMemcpyAsync(map->hin_origins[slot], origins, sizeof(float) * 3 * n_origins, cudaMemcpyHostToDevice, cs);
      a.origins = map->hin_origins[slot];
    }
    if (e == cudaSuccess && host_e) {
      e = cudaMemcpyAsync(map->hin_endpoints[slot], endpoints, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, cs);
      a.endpoints = map->hin_endpoints[slot];
    }
    if (e == cudaSuccess && host_f) {
      e = cudaMemcpyAsync(map->hin_flags[slot], flags, (size_t)n, cudaMemcpyHostToDevice, cs);
      a.flags = map->hin_flags[slot];
    }
    if (e == cudaSuccess) e = cudaEventRecord(map->hin_copied[slot], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, map->hin_copied[slot], 0);
    if (e != cudaSuccess) return cuda_fail(e, "integrate: copy host inputs");
  }
  e = ohm::launch_integrate(map, a, stream);
  if (e != cudaSuccess) return cuda_fail(e, "integrate: launch");
  if (slot >= 0) {
    e = cudaEventRecord(map->hin_free[slot], stream);
    if (e != cudaSuccess) return cuda_fail(e, "integrate: record");
  }
  ohm::note_work(map, stream);
  return OHM_OK;
}

}  // namespace

extern "C" {

const char* ohm_last_error(void) { return g_last_error.c_str(); }

ohm_status ohm_map_create(const ohm_map_params* params, ohm_map** out) {
  if (!params || !out) return fail(OHM_ERR_INVALID, "create: NULL argument");
  *out = nullptr;
  ohm_map_params p = *params;
  if (p.segment_steps == 0) p.segment_steps = 24;
  if (!(p.voxel_size > 0.0) || !std::isfinite(p.voxel_size)) return fail(OHM_ERR_INVALID, "create: voxel_size must be > 0");
  if (p.frac_bits < 8 || p.frac_bits > 20) return fail(OHM_ERR_INVALID, "create: frac_bits must be in [8, 20]");
  const uint32_t all = OHM_LAYER_OCCUPANCY | OHM_LAYER_NDT | OHM_LAYER_TSDF | OHM_LAYER_COUNTS | OHM_LAYER_DECAY | OHM_LAYER_MEAN;
  if (p.layers == 0 || (p.layers & ~all)) return fail(OHM_ERR_INVALID, "create: bad layer mask");
  if (!(p.l_min <= p.l_max)) return fail(OHM_ERR_INVALID, "create: l_min > l_max");
  if (std::isnan(p.ndt_clear_below)) return fail(OHM_ERR_INVALID, "create: ndt_clear_below is NaN");
  {
    // log-odds values are sums of these and the clamp bounds: with every one 0
    // or at least 2^-100 in magnitude no value is a float subnormal, which the
    // miss walk's float atomic add would flush to zero
    const float tiny = std::ldexp(1.0f, -100);
    const float vals[4] = {p.hit, p.miss, p.l_min, p.l_max};
    for (float v : vals)
      if (std::isnan(v) || (v != 0.0f && std::fabs(v) < tiny))
        return fail(OHM_ERR_INVALID, "create: hit, miss, l_min and l_max must be 0 or at least 2^-100 in magnitude");
  }
  if (!(p.max_range > 0.0)) return fail(OHM_ERR_INVALID, "create: max_range must be > 0");
  if (!(p.min_range >= 0.0)) return fail(OHM_ERR_INVALID, "create: min_range must be >= 0");
  if (!(p.tsdf_trunc >= 0.0) || !(p.tsdf_wmax > 0.0)) return fail(OHM_ERR_INVALID, "create: bad TSDF parameters");
  if (p.max_regions < 1 || p.max_regions > (1LL << 16)) return fail(OHM_ERR_INVALID, "create: max_regions must be in [1, 65536]");
  if (p.max_rays < 1 || p.max_rays > (1LL << 30)) return fail(OHM_ERR_INVALID, "create: max_rays out of range");
  if (p.segment_steps < 1) return fail(OHM_ERR_INVALID, "create: segment_steps must be >= 1");
  if (p.max_probe < 0) return fail(OHM_ERR_INVALID, "create: max_probe must be >= 0");
  if ((p.layers & OHM_LAYER_MEAN) && p.max_rays > (1LL << 22))
    return fail(OHM_ERR_INVALID, "create: the mean layer needs max_rays <= 2^22 (per-call 32-bit sums)");
  if ((p.layers & OHM_LAYER_NDT) && (p.max_ndt_regions < 1 || p.max_ndt_regions > p.max_regions))
    return fail(OHM_ERR_INVALID, "create: max_ndt_regions must be in [1, max_regions]");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(p.map_origin[k])) return fail(OHM_ERR_INVALID, "create: map_origin not finite");
  const double scale = std::ldexp(1.0, p.frac_bits) / p.voxel_size;
  if ((p.max_range + p.tsdf_trunc) * scale >= std::ldexp(1.0, 30))
    return fail(OHM_ERR_INVALID, "create: (max_range + tsdf_trunc) * 2^frac_bits / voxel_size must be < 2^30");

  DeviceGuard guard(p.device);
  if (!guard.ok) return fail(OHM_ERR_CUDA, "create: cannot select device");
  ohm_map* m = new ohm_map();
  m->p = p;
  m->device = p.device;
  ohm::DeviceMap& d = m->d;
  const long long R = p.max_regions;
  const long long V = ohm::kRegionVoxels;
  // evicted regions keep their keys: a map that evicts when full may know
  // many more keys than its pool holds
  const long long h_min = p.evict_when_full ? (1LL << 18) : 1024;
  const long long H = next_pow2(2 * R > h_min ? 2 * R : h_min);
  m->hash_capacity = H;
  d.hmask = (uint32_t)(H - 1);
  const int32_t probe_cap = (int32_t)(H < 4096 ? H : 4096);
  d.max_probe = (p.max_probe <= 0 || p.max_probe > probe_cap) ? probe_cap : p.max_probe;
  d.max_regions = (int32_t)R;
  d.max_ndt = (p.layers & OHM_LAYER_NDT) ? (int32_t)p.max_ndt_regions : 0;
  const long long vox_steps = (long long)std::ceil(p.max_range / p.voxel_size) + 2;
  // a ray takes at most 3 vox_steps voxel steps, so it has at most
  // ceil(3 vox_steps / segment_steps) segments (ray_segment_split)
  d.max_segs = p.max_rays * ((3 * vox_steps + p.segment_steps - 1) / p.segment_steps + 1);
  const long long band = (long long)std::ceil(2.0 * p.tsdf_trunc / p.voxel_size) + 2;
  d.max_touched = (p.layers & OHM_LAYER_TSDF) ? p.max_rays * (1 + 3 * band) : 0;
  if (d.max_touched > R * V) d.max_touched = R * V;

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  chk(alloc(&d.htab, H, 0xFF));  // key -1 (empty), slot -1
  chk(alloc(&d.region_count, 1, 0));
  chk(alloc(&d.ndt_count, 1, 0));
  chk(alloc(&d.status, 1, 0));
  chk(alloc(&d.calls, 1, 0));
  chk(alloc(&d.region_coords, 3 * R, 0));
  chk(alloc(&d.ndt_slot, R, 0xFF));
  chk(alloc(&d.stamp, R, 0));
  chk(alloc(&d.born, R, 0xFF));
  chk(alloc(&d.ndt_born, R, 0xFF));
  chk(alloc(&d.free_slots, R, 0));
  chk(alloc(&d.free_info, 4, 0));
  chk(alloc(&d.restore_keys, R, 0));
  d.max_restore = (int32_t)R;
  if (p.layers & OHM_LAYER_OCCUPANCY) chk(alloc(&d.occ, R * V, 0xFF));  // all-ones float = NaN = unknown
  if (p.layers & OHM_LAYER_COUNTS) chk(alloc(&d.counts, R * V, 0));
  if (p.layers & OHM_LAYER_DECAY) chk(alloc(&d.decay, R * V, 0));
  if (p.layers & OHM_LAYER_MEAN) {
    chk(alloc(&d.vmean, R * V, 0));
    chk(alloc(&d.vmean_acc, 2 * R * V, 0));
  }
  if (p.layers & OHM_LAYER_NDT) {
    chk(alloc(&d.ndt, (long long)d.max_ndt * 10 * V, 0));
    chk(alloc(&d.ndt_free, d.max_ndt, 0));
    chk(alloc(&d.ndt_pending, p.max_rays, 0));
  }
  if (p.layers & OHM_LAYER_TSDF) {
    chk(alloc(&d.tsdf, R * V, 0));
    chk(alloc(&d.tsdf_cnt, R * V, 0));
    chk(alloc(&d.tsdf_sum, R * V, 0));
    chk(alloc(&d.trays, p.max_rays, 0));
    chk(alloc(&d.touched, d.max_touched, 0));
  }
  chk(alloc(&d.rays, p.max_rays, 0));
  if (p.layers & OHM_LAYER_DECAY) chk(alloc(&d.decay_rays, p.max_rays, 0));
  if (p.layers & OHM_LAYER_MEAN) chk(alloc(&d.mean_list, p.max_rays, 0));
  chk(alloc(&d.segs, d.max_segs, 0));
  chk(alloc(&m->stage_origins, 3 * p.max_rays, 0));
  chk(alloc(&m->stage_endpoints, 3 * p.max_rays, 0));
  chk(alloc(&m->stage_flags, p.max_rays, 0));
  for (int s = 0; s < 2; ++s) {
    chk(alloc(&m->hin_origins[s], 3 * p.max_rays, 0));
    chk(alloc(&m->hin_endpoints[s], 3 * p.max_rays, 0));
    chk(alloc(&m->hin_flags[s], p.max_rays, 0));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->hin_copied[s], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->hin_free[s], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&m->copy_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&m->work_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&m->h_status), sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&m->h_calls), sizeof(ohm::CallCounters));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&m->h_count), 2 * sizeof(int32_t));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_map(m);
    return cuda_fail(e, "create: allocation");
  }
  for (int k = 0; k < 3; ++k) d.origin[k] = p.map_origin[k];
  d.scale = scale;
  d.rmax_q = p.max_range * scale;
  {
    // |b - a|^2 <= (rmax_q - 1)^2 gives a double length below rmax_q (its
    // relative error is a few 2^-53); checked against the double bound
    const double r_in = d.rmax_q - 1.0;
    d.rmax_in2 = r_in > 0.0 ? (unsigned long long)std::floor(r_in * r_in) : 0ULL;
  }
  d.rmin_q = p.min_range * scale;
  d.tau_q = p.tsdf_trunc * scale;
  d.band.tau = ohm::ff_of_double(d.tau_q);
  d.band.rmin = ohm::ff_of_double(d.rmin_q);
  d.band.rmax = ohm::ff_of_double(d.rmax_q);
  d.voxel_size = p.voxel_size;
  d.frac_bits = p.frac_bits;
  d.layers = p.layers;
  d.seg_steps = p.segment_steps;
  d.hit = p.hit;
  d.miss = p.miss;
  d.l_min = p.l_min;
  d.l_max = p.l_max;
  d.ndt_clear = p.ndt_clear_below;
  d.tau_m = (float)p.tsdf_trunc;
  d.wmax = (float)p.tsdf_wmax;
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, p.device);
  m->walk_blocks = m->num_sms * ohm::walk_blocks_per_sm();
  *out = m;
  return OHM_OK;
}

void ohm_map_destroy(ohm_map* map) {
  if (!map) return;
  DeviceGuard guard(map->device);
  // wait only for the map's own work (the last work any entry point enqueued
  // on it, and its copy stream), not for every stream of the device
  if (map->work_done) cudaEventSynchronize(map->work_done);
  free_map(map);
}

ohm_status ohm_integrate_rays_async(ohm_map* map, const float* origins, int64_t n_origins, const float* endpoints,
                                    const uint8_t* flags, int64_t n, void* stream) {
  if (!map) return fail(OHM_ERR_INVALID, "integrate: map is NULL");
  DeviceGuard guard(map->device);
  return enqueue_integrate(map, origins, n_origins, endpoints, flags, n, static_cast<cudaStream_t>(stream));
}

ohm_status ohm_map_sync(ohm_map* map, void* stream) {
  if (!map) return fail(OHM_ERR_INVALID, "sync: map is NULL");
  DeviceGuard guard(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(map->h_status, map->d.status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  const int bits = *map->h_status;
  if (bits != 0) {
    e = cudaMemsetAsync(map->d.status, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sync: clear status");
  }
  return status_from_bits(bits);
}

ohm_status ohm_probe_cas_rate(int32_t device, int64_t words, int64_t ops, double* ops_per_second) {
  if (!ops_per_second) return fail(OHM_ERR_INVALID, "probe_cas_rate: NULL output");
  if (words < 1024 || words > (1LL << 32) || (words & (words - 1)))
    return fail(OHM_ERR_INVALID, "probe_cas_rate: words must be a power of two in [2^10, 2^32]");
  if (ops < 1) return fail(OHM_ERR_INVALID, "probe_cas_rate: ops < 1");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(OHM_ERR_CUDA, "probe_cas_rate: cannot select device");
  cudaError_t e = ohm::probe_cas_rate(device, words, ops, ops_per_second);
  if (e != cudaSuccess) return cuda_fail(e, "probe_cas_rate");
  return OHM_OK;
}

ohm_status ohm_probe_rate(int32_t device, int32_t kind, int64_t units, int64_t ops, double* ops_per_second) {
  if (!ops_per_second) return fail(OHM_ERR_INVALID, "probe_rate: NULL output");
  if (kind < OHM_PROBE_L2_ADD || kind > OHM_PROBE_SECTOR_RMW) return fail(OHM_ERR_INVALID, "probe_rate: unknown kind");
  const int64_t max_units = kind == OHM_PROBE_SECTOR_RMW ? (1LL << 29) : (1LL << 32);
  if (units < 1 || units > max_units || (units & (units - 1)))
    return fail(OHM_ERR_INVALID, "probe_rate: units must be a power of two in [1, 2^32] (2^29 sectors)");
  if (ops < 1) return fail(OHM_ERR_INVALID, "probe_rate: ops < 1");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(OHM_ERR_CUDA, "probe_rate: cannot select device");
  cudaError_t e = ohm::probe_rate(device, kind, units, ops, ops_per_second);
  if (e != cudaSuccess) return cuda_fail(e, "probe_rate");
  return OHM_OK;
}

ohm_status ohm_map_status_async(ohm_map* map, int32_t* status, void* stream) {
  if (!map || !status) return fail(OHM_ERR_INVALID, "status_async: NULL argument");
  if (is_device_pointer(status)) return fail(OHM_ERR_INVALID, "status_async: status must be host memory");
  DeviceGuard guard(map->device);
  cudaError_t e = cudaMemcpyAsync(status, map->d.status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "status_async");
  return OHM_OK;
}

ohm_status ohm_integrate_rays(ohm_map* map, const float* origins, int64_t n_origins, const float* endpoints,
                              const uint8_t* flags, int64_t n, void* stream) {
  // A call that reaches evicted regions changes nothing; bring them back and
  // repeat it (a repeat can only fault on regions evicted to make room, which
  // are the least recently used, so this ends quickly).
  for (int attempt = 0; attempt < 8; ++attempt) {
    ohm_status st = ohm_integrate_rays_async(map, origins, n_origins, endpoints, flags, n, stream);
    if (st != OHM_OK) return st;
    st = ohm_map_sync(map, stream);
    if (st == OHM_ERR_CAPACITY && map->p.evict_when_full) {
      // Make room: the regions this call touched were just stamped, so the
      // least recently used ones are others.  Keep three quarters.
      long long resident = 0, evicted = 0;
      cudaError_t e = ohm::cache_resident(map, &resident);
      if (e == cudaSuccess) e = ohm::cache_evict(map, resident * 3 / 4, &evicted);
      if (e != cudaSuccess) return cuda_fail(e, "integrate: evict");
      if (evicted == 0) return fail(OHM_ERR_CAPACITY, "integrate: the call alone needs more regions than the pool");
      // the call may also have reached evicted regions (a capacity failure is
      // what its status reports): bring those back before repeating it
      int64_t restored = 0;
      st = ohm_map_restore_pending(map, &restored, stream);
      if (st != OHM_OK) return st;
      continue;
    }
    if (st != OHM_ERR_EVICTED) return st;
    int64_t restored = 0;
    st = ohm_map_restore_pending(map, &restored, stream);
    if (st != OHM_OK) return st;
  }
  return fail(OHM_ERR_CAPACITY, "integrate: evicted regions could not be kept resident (pool too small)");
}

ohm_status ohm_map_evict(ohm_map* map, int64_t keep_regions, int64_t* evicted, void* stream) {
  if (!map || !evicted) return fail(OHM_ERR_INVALID, "evict: NULL argument");
  if (keep_regions < 0) return fail(OHM_ERR_INVALID, "evict: keep_regions < 0");
  DeviceGuard guard(map->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  long long ev = 0;
  if (e == cudaSuccess) e = ohm::cache_evict(map, keep_regions, &ev);
  if (e != cudaSuccess) return cuda_fail(e, "evict");
  *evicted = ev;
  return OHM_OK;
}

ohm_status ohm_map_restore_pending(ohm_map* map, int64_t* restored, void* stream) {
  if (!map || !restored) return fail(OHM_ERR_INVALID, "restore_pending: NULL argument");
  DeviceGuard guard(map->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  std::vector<long long> keys;
  long long r = 0;
  if (e == cudaSuccess) e = ohm::cache_pending(map, &keys);
  if (e == cudaSuccess) e = ohm::cache_restore(map, keys, &r);
  if (e == cudaErrorMemoryAllocation) return fail(OHM_ERR_CAPACITY, "restore_pending: pool or host memory too small");
  if (e != cudaSuccess) return cuda_fail(e, "restore_pending");
  *restored = r;
  return OHM_OK;
}

ohm_status ohm_map_restore_all(ohm_map* map, int64_t* restored, void* stream) {
  if (!map || !restored) return fail(OHM_ERR_INVALID, "restore_all: NULL argument");
  DeviceGuard guard(map->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  long long r = 0;
  if (e == cudaSuccess) {
    const std::vector<long long> keys = ohm::cache_all_keys(map);
    long long resident = 0;
    e = ohm::cache_resident(map, &resident);
    if (e == cudaSuccess && resident + (long long)keys.size() > map->p.max_regions)
      return fail(OHM_ERR_CAPACITY, "restore_all: resident and evicted regions exceed max_regions");
    if (e == cudaSuccess) e = ohm::cache_restore(map, keys, &r);
  }
  if (e == cudaErrorMemoryAllocation) return fail(OHM_ERR_CAPACITY, "restore_all: pool too small");
  if (e != cudaSuccess) return cuda_fail(e, "restore_all");
  *restored = r;
  return OHM_OK;
}

ohm_status ohm_map_residency(ohm_map* map, int64_t* resident, int64_t* evicted, void* stream) {
  if (!map || !resident || !evicted) return fail(OHM_ERR_INVALID, "residency: NULL argument");
  DeviceGuard guard(map->device);
  cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  long long r = 0;
  if (e == cudaSuccess) e = ohm::cache_resident(map, &r);
  if (e != cudaSuccess) return cuda_fail(e, "residency");
  *resident = r;
  *evicted = ohm::cache_host_regions(map);
  return OHM_OK;
}

ohm_status ohm_query_voxels(ohm_map* map, const float* points, int64_t n, float* occupancy, uint8_t* known,
                            float* ndt, float* tsdf, uint32_t* counts, uint64_t* path_sum, float* mean,
                            void* stream) {
  if (!map) return fail(OHM_ERR_INVALID, "query: map is NULL");
  if (n < 0) return fail(OHM_ERR_INVALID, "query: n < 0");
  if (n == 0) return OHM_OK;
  if (!points) return fail(OHM_ERR_INVALID, "query: points is NULL");
  void* outs[] = {occupancy, known, ndt, tsdf, counts, path_sum, mean};
  for (void* o : outs)
    if (o && (!is_device_pointer(o) || on_other_device(o, map->device)))
      return fail(OHM_ERR_INVALID, "query: outputs must be device memory of the map's device");
  if (path_sum && !(map->p.layers & OHM_LAYER_DECAY)) return fail(OHM_ERR_UNSUPPORTED, "query: map has no decay layer");
  if (mean && !(map->p.layers & OHM_LAYER_MEAN)) return fail(OHM_ERR_UNSUPPORTED, "query: map has no mean layer");
  if (ndt && !(map->p.layers & OHM_LAYER_NDT)) return fail(OHM_ERR_UNSUPPORTED, "query: map has no NDT layer");
  if (tsdf && !(map->p.layers & OHM_LAYER_TSDF)) return fail(OHM_ERR_UNSUPPORTED, "query: map has no TSDF layer");
  DeviceGuard guard(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float* pts = points;
  float* staged = nullptr;
  cudaError_t e;
  if (on_other_device(points, map->device)) return fail(OHM_ERR_INVALID, "query: points on another device than the map");
  if (!is_device_pointer(points)) {
    e = cudaMallocAsync(reinterpret_cast<void**>(&staged), sizeof(float) * 3 * n, s);
    if (e != cudaSuccess) return cuda_fail(e, "query: staging");
    e = cudaMemcpyAsync(staged, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "query: copy points");
    pts = staged;
  }
  e = ohm::launch_query(map, pts, n, occupancy, known, ndt, tsdf, counts,
                        reinterpret_cast<unsigned long long*>(path_sum), mean, s);
  if (staged) cudaFreeAsync(staged, s);
  if (e != cudaSuccess) return cuda_fail(e, "query: launch");
  ohm::note_work(map, s);
  return OHM_OK;
}

ohm_status ohm_map_region_count(ohm_map* map, int64_t* out, void* stream) {
  if (!map || !out) return fail(OHM_ERR_INVALID, "region_count: NULL argument");
  DeviceGuard guard(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(map->h_count, map->d.region_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "region_count");
  const long long c = *map->h_count;
  *out = c < map->p.max_regions ? c : map->p.max_regions;
  return OHM_OK;
}

ohm_status ohm_map_export(ohm_map* map, int64_t first, int64_t count, int32_t* keys, float* occupancy,
                          uint32_t* counts, int64_t* ndt, float* tsdf, uint64_t* path_sum, uint64_t* mean,
                          void* stream) {
  if (!map) return fail(OHM_ERR_INVALID, "export: map is NULL");
  if (first < 0 || count < 0 || first + count > map->p.max_regions)
    return fail(OHM_ERR_INVALID, "export: region range outside the pool");
  void* outs[] = {keys, occupancy, counts, ndt, tsdf, path_sum, mean};
  for (void* o : outs)
    if (o && (!is_device_pointer(o) || on_other_device(o, map->device)))
      return fail(OHM_ERR_INVALID, "export: outputs must be device memory of the map's device");
  if (path_sum && !(map->p.layers & OHM_LAYER_DECAY)) return fail(OHM_ERR_UNSUPPORTED, "export: no decay layer");
  if (mean && !(map->p.layers & OHM_LAYER_MEAN)) return fail(OHM_ERR_UNSUPPORTED, "export: no mean layer");
  if (occupancy && !(map->p.layers & OHM_LAYER_OCCUPANCY)) return fail(OHM_ERR_UNSUPPORTED, "export: no occupancy layer");
  if (counts && !(map->p.layers & OHM_LAYER_COUNTS)) return fail(OHM_ERR_UNSUPPORTED, "export: no counts layer");
  if (ndt && !(map->p.layers & OHM_LAYER_NDT)) return fail(OHM_ERR_UNSUPPORTED, "export: no NDT layer");
  if (tsdf && !(map->p.layers & OHM_LAYER_TSDF)) return fail(OHM_ERR_UNSUPPORTED, "export: no TSDF layer");
  DeviceGuard guard(map->device);
  cudaError_t e = ohm::launch_export(map, first, count, keys, occupancy, counts, reinterpret_cast<long long*>(ndt),
                                     tsdf, reinterpret_cast<unsigned long long*>(path_sum),
                                     reinterpret_cast<unsigned long long*>(mean), static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "export: launch");
  ohm::note_work(map, static_cast<cudaStream_t>(stream));
  return OHM_OK;
}

ohm_status ohm_map_stats(ohm_map* map, ohm_call_stats* out, void* stream) {
  if (!map || !out) return fail(OHM_ERR_INVALID, "stats: NULL argument");
  DeviceGuard guard(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(map->h_calls, map->d.calls, sizeof(ohm::CallCounters), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(map->h_count, map->d.region_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(map->h_count + 1, map->d.ndt_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stats");
  out->rays = (int64_t)map->h_calls->rays;
  out->segments = (int64_t)map->h_calls->segments;
  out->visits = (int64_t)map->h_calls->visits;
  out->touched = (int64_t)map->h_calls->touched;
  out->regions = map->h_count[0] < map->p.max_regions ? map->h_count[0] : map->p.max_regions;
  out->ndt_regions = map->h_count[1];
  out->total_visits = (int64_t)map->h_calls->total_visits;
  out->launches = map->launches;
  out->atomics = (int64_t)map->h_calls->atomics;
  return OHM_OK;
}

ohm_status ohm_map_profile(ohm_map* map, uint32_t stage_mask) {
  if (!map) return fail(OHM_ERR_INVALID, "profile: map is NULL");
  if (stage_mask >> OHM_STAGE_COUNT) return fail(OHM_ERR_INVALID, "profile: unknown stage bit");
  DeviceGuard guard(map->device);
  for (auto& pe : map->pending) {
    cudaEventSynchronize(pe.second.second);
    map->event_pool.push_back(pe.second.first);
    map->event_pool.push_back(pe.second.second);
  }
  map->pending.clear();
  map->profile_mask = stage_mask;
  map->profile_every = 1;
  map->profile_call = 0;
  for (int k = 0; k < OHM_STAGE_COUNT; ++k) {
    map->stage_ms[k] = 0.0;
    map->stage_launches[k] = 0;
  }
  return OHM_OK;
}

ohm_status ohm_map_profile_every(ohm_map* map, uint32_t stage_mask, int32_t every) {
  if (!map) return fail(OHM_ERR_INVALID, "profile_every: map is NULL");
  if (every < 1) return fail(OHM_ERR_INVALID, "profile_every: every must be >= 1");
  const ohm_status st = ohm_map_profile(map, stage_mask);
  if (st == OHM_OK) map->profile_every = every;
  return st;
}

ohm_status ohm_map_profile_read(ohm_map* map, int32_t stage, double* total_ms, int64_t* launches) {
  if (!map || !total_ms || !launches) return fail(OHM_ERR_INVALID, "profile_read: NULL argument");
  if (stage < 0 || stage >= OHM_STAGE_COUNT) return fail(OHM_ERR_INVALID, "profile_read: unknown stage");
  DeviceGuard guard(map->device);
  for (auto& pe : map->pending) {
    cudaError_t e = cudaEventSynchronize(pe.second.second);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
    if (e != cudaSuccess) return cuda_fail(e, "profile_read");
    map->stage_ms[pe.first] += ms;
    map->stage_launches[pe.first] += 1;
    map->event_pool.push_back(pe.second.first);
    map->event_pool.push_back(pe.second.second);
  }
  map->pending.clear();
  *total_ms = map->stage_ms[stage];
  *launches = map->stage_launches[stage];
  return OHM_OK;
}

}  // extern "C"

namespace ohm {

void set_last_error(const std::string& msg) { g_last_error = msg; }

void note_work(ohm_map* map, cudaStream_t stream) {
  if (map->work_done) cudaEventRecord(map->work_done, stream);
}

static cudaEvent_t pooled_event(ohm_map* map) {
  if (!map->event_pool.empty()) {
    cudaEvent_t ev = map->event_pool.back();
    map->event_pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  cudaEventCreate(&ev);
  return ev;
}

void stage_begin(ohm_map* map, int stage, cudaStream_t stream, cudaEvent_t* ev) {
  *ev = nullptr;
  if (!(map->profile_mask & (1u << stage))) return;
  if (map->profile_every > 1 && (map->profile_call - 1) % map->profile_every != 0) return;
  *ev = pooled_event(map);
  cudaEventRecord(*ev, stream);
}

void stage_end(ohm_map* map, int stage, cudaStream_t stream, cudaEvent_t ev) {
  if (!ev) return;
  cudaEvent_t e1 = pooled_event(map);
  cudaEventRecord(e1, stream);
  map->pending.push_back(std::make_pair(stage, std::make_pair(ev, e1)));
}

}  // namespace ohm

extern "C" {

}  // extern "C"
