// Host-side definition of the map handle and the launch functions shared by
// the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/ohm_gb.h"
#include "ohm_device.cuh"

namespace ohm {
struct HostStore;
}

struct ohm_map {
  ohm_map_params p;
  ohm::DeviceMap d;
  int device;
  int num_sms;
  int walk_blocks;          // persistent grid for the walk kernels
  long long hash_capacity;
  // device staging for inputs generated on the device (depth frames)
  float* stage_origins;
  float* stage_endpoints;
  uint8_t* stage_flags;
  // host inputs: two staging slots filled on copy_stream, so that the copy of
  // one call overlaps the kernels of the previous one
  float* hin_origins[2];
  float* hin_endpoints[2];
  uint8_t* hin_flags[2];
  cudaStream_t copy_stream;
  cudaEvent_t hin_copied[2];  // slot filled
  cudaEvent_t hin_free[2];    // kernels of the slot's last call done
  int hin_next;
  // pinned host mirrors for status / counters
  int32_t* h_status;
  ohm::CallCounters* h_calls;
  int32_t* h_count;
  long long launches;       // kernels launched by this map
  // per-stage event timing
  uint32_t profile_mask;
  int32_t profile_every;    // record only every profile_every-th call (0 or 1: every call)
  long long profile_call;   // integrate calls since the mask was set
  std::vector<cudaEvent_t> event_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  double stage_ms[OHM_STAGE_COUNT];
  long long stage_launches[OHM_STAGE_COUNT];
  ohm::HostStore* store;    // evicted regions in pinned host memory
  // depth frames: (u - cx) / fx per column and (v - cy) / fy per row, for the
  // last image size and intrinsics (pxy_key: width, height, fx, fy, cx, cy)
  double* pxy;
  long long pxy_cap;
  double pxy_key[6];
  cudaEvent_t work_done;    // recorded behind the last work any entry point enqueued on the map
};

namespace ohm {

// Enqueue every kernel of one integrate call on `stream`.
cudaError_t launch_integrate(ohm_map* map, const CallArgs& args, cudaStream_t stream);
cudaError_t probe_cas_rate(int device, long long words, long long ops, double* rate);
cudaError_t probe_rate(int device, int kind, long long units, long long ops, double* rate);
cudaError_t launch_query(ohm_map* map, const float* points, long long n, float* occupancy, uint8_t* known, float* ndt,
                         float* tsdf, uint32_t* counts, unsigned long long* path_sum, float* mean,
                         cudaStream_t stream);
cudaError_t launch_export(ohm_map* map, long long first, long long count, int32_t* keys, float* occupancy,
                          uint32_t* counts, long long* ndt, float* tsdf, unsigned long long* path_sum,
                          unsigned long long* mean, cudaStream_t stream);
int walk_blocks_per_sm();

// Region cache (ohm_cache.cu).
cudaError_t cache_evict(ohm_map* m, long long target, long long* evicted);
cudaError_t cache_restore(ohm_map* m, const std::vector<long long>& keys, long long* restored);
cudaError_t cache_pending(ohm_map* m, std::vector<long long>* keys);
cudaError_t cache_resident(ohm_map* m, long long* resident);
long long cache_host_regions(ohm_map* m);
std::vector<long long> cache_all_keys(ohm_map* m);
void destroy_host_store(ohm_map* m);

// Set the message ohm_last_error() returns on this thread.
void set_last_error(const std::string& msg);

// Record, on `stream`, that the map has work enqueued up to here (waited for
// by ohm_map_destroy).
void note_work(ohm_map* map, cudaStream_t stream);

// Stage timing helpers (no-ops unless the stage is being profiled).
void stage_begin(ohm_map* map, int stage, cudaStream_t stream, cudaEvent_t* ev);
void stage_end(ohm_map* map, int stage, cudaStream_t stream, cudaEvent_t ev);

}  // namespace ohm
