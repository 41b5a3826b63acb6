// Region cache: moving regions between device memory and pinned host memory.
//
// The paper keeps regions in a GPU cache backed by host memory (Sec. III-A).
// Here every region in the device pool carries the sequence number of the
// last integrate call that touched it; ohm_map_evict copies the least
// recently touched regions to pinned host memory, resets their pool slots and
// puts the slots (and their NDT blocks) on free lists.  An evicted region
// keeps its key in the hash table, marked evicted.  An integrate call that
// reaches such a key records it, stops and rolls back (nothing changes); the
// library then copies the region back into a free slot and the call is
// repeated (ohm_integrate_rays does this by itself; after the asynchronous
// entry points ohm_map_sync reports OHM_ERR_EVICTED and the caller restores
// with ohm_map_restore_pending and repeats the call).
#include <algorithm>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "ohm_host.h"

namespace ohm {

// Fixed-size pinned blocks carved from chunks allocated with cudaMallocHost.
class PinnedSlab {
 public:
  explicit PinnedSlab(size_t block) : block_(block) {}
  ~PinnedSlab() {
    for (void* c : chunks_) cudaFreeHost(c);
  }
  void* get() {
    if (free_.empty()) {
      const int per = 16;
      void* c = nullptr;
      if (cudaMallocHost(&c, block_ * per) != cudaSuccess) return nullptr;
      chunks_.push_back(c);
      for (int i = 0; i < per; ++i) free_.push_back(static_cast<char*>(c) + block_ * i);
    }
    void* p = free_.back();
    free_.pop_back();
    return p;
  }
  void put(void* p) {
    if (p) free_.push_back(p);
  }

 private:
  size_t block_;
  std::vector<void*> chunks_;
  std::vector<void*> free_;
};

struct HostRegion {
  int32_t coords[3];
  void* occ = nullptr;
  void* counts = nullptr;
  void* decay = nullptr;
  void* vmean = nullptr;
  void* ndt = nullptr;
  void* tsdf = nullptr;
};

struct HostStore {
  PinnedSlab occ{sizeof(float) * kRegionVoxels};
  PinnedSlab counts{sizeof(unsigned long long) * kRegionVoxels};
  PinnedSlab decay{sizeof(unsigned long long) * kRegionVoxels};
  PinnedSlab vmean{sizeof(unsigned long long) * kRegionVoxels};
  PinnedSlab ndt{sizeof(long long) * 10 * kRegionVoxels};
  PinnedSlab tsdf{sizeof(float2) * kRegionVoxels};
  std::unordered_map<long long, HostRegion> regions;
};

HostStore* host_store(ohm_map* m) {
  if (!m->store) m->store = new HostStore();
  return m->store;
}

void destroy_host_store(ohm_map* m) {
  delete m->store;
  m->store = nullptr;
}

namespace {

constexpr int kCacheBlock = 256;

// Mark the hash entries of `keys` with `value` (kSlotEvicted, or the slot of a
// restored region, in which case its bookkeeping is filled in too).
__global__ void k_set_entries(DeviceMap m, const long long* keys, const int32_t* slots, const int32_t* ndt_blocks,
                              const int32_t* coords, int n, int evict) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long key = keys[i];
  uint32_t h = hash_key(key) & m.hmask;
  for (int p = 0; p < m.max_probe; ++p) {
    const longlong2 e = m.htab[h];
    if (e.x == key) {
      if (evict) {
        m.htab[h].y = kSlotEvicted;
      } else {
        const int32_t s = slots[i];
        m.htab[h].y = s;
        m.region_coords[3 * s + 0] = coords[3 * i + 0];
        m.region_coords[3 * s + 1] = coords[3 * i + 1];
        m.region_coords[3 * s + 2] = coords[3 * i + 2];
        const int32_t seq = m.calls->seq;
        m.stamp[s] = seq;
        m.born[s] = seq - 1;  // not born in the call that will repeat: a rollback must keep it
        m.ndt_slot[s] = ndt_blocks[i];
        m.ndt_born[s] = seq - 1;
      }
      return;
    }
    if (e.x == kEmptyKey) return;
    h = (h + 1) & m.hmask;
  }
}

// Reset released pool slots to "never observed" and clear released NDT blocks.
__global__ void k_reset_slots(DeviceMap m, const int32_t* slots, int n, const int32_t* ndt_blocks, int n_ndt) {
  const long long per = kRegionVoxels;
  const long long total = (long long)(n + n_ndt) * per;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const long long r = t / per, v = t % per;
    if (r < n) {
      const long long off = (long long)slots[r] * per + v;
      if (m.occ) reinterpret_cast<unsigned int*>(m.occ)[off] = 0xFFFFFFFFu;
      if (m.counts) m.counts[off] = 0ULL;
      if (m.decay) m.decay[off] = 0ULL;
      if (m.vmean) m.vmean[off] = 0ULL;
      if (m.tsdf) m.tsdf[off] = make_float2(0.f, 0.f);
      if (v == 0) m.ndt_slot[slots[r]] = -1;
    } else {
      long long* base = m.ndt + (long long)ndt_blocks[r - n] * 10 * per + v;
#pragma unroll
      for (int k = 0; k < 10; ++k) base[(long long)k * per] = 0;
    }
  }
}

template <typename T>
cudaError_t d2h(std::vector<T>& out, const T* src, size_t n) {
  out.resize(n);
  if (!n) return cudaSuccess;
  return cudaMemcpy(out.data(), src, sizeof(T) * n, cudaMemcpyDeviceToHost);
}

template <typename T>
cudaError_t h2d(T* dst, const std::vector<T>& src) {
  if (src.empty()) return cudaSuccess;
  return cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice);
}

// Device memory for small per-operation arrays (keys, slots, coords).
template <typename T>
struct DevVec {
  T* p = nullptr;
  ~DevVec() {
    if (p) cudaFree(p);
  }
  cudaError_t load(const std::vector<T>& v) {
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), sizeof(T) * v.size());
    if (e == cudaSuccess) e = cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
  }
};

struct PoolView {
  int32_t region_count, ndt_count;
  int32_t info[4];
  std::vector<int32_t> free_slots;  // released and not yet reused
  std::vector<int32_t> free_ndt;
};

cudaError_t read_pool(ohm_map* m, PoolView* v) {
  DeviceMap& d = m->d;
  cudaError_t e = cudaMemcpy(&v->region_count, d.region_count, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&v->ndt_count, d.ndt_count, sizeof(int32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(v->info, d.free_info, sizeof(v->info), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  v->region_count = std::min<int32_t>(v->region_count, d.max_regions);
  v->ndt_count = std::min<int32_t>(v->ndt_count, d.max_ndt);
  std::vector<int32_t> fs, fn;
  e = d2h(fs, d.free_slots, (size_t)std::max(0, v->info[0]));
  if (e == cudaSuccess && d.max_ndt > 0) e = d2h(fn, d.ndt_free, (size_t)std::max(0, v->info[2]));
  if (e != cudaSuccess) return e;
  v->free_slots.assign(fs.begin() + std::min<int32_t>(v->info[1], v->info[0]), fs.end());
  v->free_ndt.clear();
  if (!fn.empty()) v->free_ndt.assign(fn.begin() + std::min<int32_t>(v->info[3], v->info[2]), fn.end());
  return cudaSuccess;
}

cudaError_t write_pool(ohm_map* m, const PoolView& v) {
  DeviceMap& d = m->d;
  int32_t info[4] = {(int32_t)v.free_slots.size(), 0, (int32_t)v.free_ndt.size(), 0};
  cudaError_t e = h2d(d.free_slots, v.free_slots);
  if (e == cudaSuccess && d.max_ndt > 0) e = h2d(d.ndt_free, v.free_ndt);
  if (e == cudaSuccess) e = cudaMemcpy(d.free_info, info, sizeof(info), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d.region_count, &v.region_count, sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d.ndt_count, &v.ndt_count, sizeof(int32_t), cudaMemcpyHostToDevice);
  return e;
}

// Slots in use: [0, region_count) minus the released ones.
std::vector<int32_t> live_slots(const PoolView& v) {
  std::vector<char> freed((size_t)v.region_count, 0);
  for (int32_t s : v.free_slots)
    if (s >= 0 && s < v.region_count) freed[(size_t)s] = 1;
  std::vector<int32_t> live;
  for (int32_t s = 0; s < v.region_count; ++s)
    if (!freed[(size_t)s]) live.push_back(s);
  return live;
}

}  // namespace

// Evict the least recently touched regions until at most `target` remain.
cudaError_t cache_evict(ohm_map* m, long long target, long long* evicted) {
  *evicted = 0;
  DeviceMap& d = m->d;
  PoolView v;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = read_pool(m, &v);
  if (e != cudaSuccess) return e;
  std::vector<int32_t> live = live_slots(v);
  if ((long long)live.size() <= target) return cudaSuccess;
  std::vector<int32_t> stamps, coords, ndt_slots;
  e = d2h(stamps, d.stamp, (size_t)v.region_count);
  if (e == cudaSuccess) e = d2h(coords, d.region_coords, (size_t)v.region_count * 3);
  if (e == cudaSuccess) e = d2h(ndt_slots, d.ndt_slot, (size_t)v.region_count);
  if (e != cudaSuccess) return e;
  const size_t n = live.size() - (size_t)std::max(0LL, target);
  std::stable_sort(live.begin(), live.end(), [&](int32_t a, int32_t b) { return stamps[a] < stamps[b]; });
  std::vector<int32_t> victims(live.begin(), live.begin() + n);
  HostStore* hs = host_store(m);
  std::vector<long long> keys;
  std::vector<int32_t> freed_ndt;
  for (int32_t s : victims) {
    HostRegion r;
    for (int k = 0; k < 3; ++k) r.coords[k] = coords[3 * (size_t)s + k];
    const long long off = (long long)s * kRegionVoxels;
    if (d.occ) {
      r.occ = hs->occ.get();
      if (!r.occ) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.occ, d.occ + off, sizeof(float) * kRegionVoxels, cudaMemcpyDeviceToHost, 0);
    }
    if (e == cudaSuccess && d.counts) {
      r.counts = hs->counts.get();
      if (!r.counts) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.counts, d.counts + off, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyDeviceToHost, 0);
    }
    if (e == cudaSuccess && d.decay) {
      r.decay = hs->decay.get();
      if (!r.decay) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.decay, d.decay + off, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyDeviceToHost, 0);
    }
    if (e == cudaSuccess && d.vmean) {
      r.vmean = hs->vmean.get();
      if (!r.vmean) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.vmean, d.vmean + off, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyDeviceToHost, 0);
    }
    if (e == cudaSuccess && d.tsdf) {
      r.tsdf = hs->tsdf.get();
      if (!r.tsdf) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.tsdf, d.tsdf + off, sizeof(float2) * kRegionVoxels, cudaMemcpyDeviceToHost, 0);
    }
    const int32_t nb = ndt_slots[(size_t)s];
    if (e == cudaSuccess && d.ndt && nb >= 0) {
      r.ndt = hs->ndt.get();
      if (!r.ndt) return cudaErrorMemoryAllocation;
      e = cudaMemcpyAsync(r.ndt, d.ndt + (long long)nb * 10 * kRegionVoxels, sizeof(long long) * 10 * kRegionVoxels,
                          cudaMemcpyDeviceToHost, 0);
      freed_ndt.push_back(nb);
    }
    if (e != cudaSuccess) return e;
    const long long key = pack_region(r.coords[0], r.coords[1], r.coords[2]);
    keys.push_back(key);
    hs->regions[key] = r;
  }
  e = cudaDeviceSynchronize();
  DevVec<long long> dk;
  DevVec<int32_t> dv, dn;
  if (e == cudaSuccess) e = dk.load(keys);
  if (e == cudaSuccess) e = dv.load(victims);
  if (e == cudaSuccess) e = dn.load(freed_ndt);
  if (e != cudaSuccess) return e;
  const int nk = (int)keys.size();
  k_set_entries<<<(nk + kCacheBlock - 1) / kCacheBlock, kCacheBlock>>>(d, dk.p, nullptr, nullptr, nullptr, nk, 1);
  k_reset_slots<<<1024, kCacheBlock>>>(d, dv.p, nk, dn.p, (int)freed_ndt.size());
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  v.free_slots.insert(v.free_slots.end(), victims.begin(), victims.end());
  v.free_ndt.insert(v.free_ndt.end(), freed_ndt.begin(), freed_ndt.end());
  e = write_pool(m, v);
  if (e == cudaSuccess) *evicted = (long long)victims.size();
  return e;
}

// Copy the given evicted regions back into free slots.
cudaError_t cache_restore(ohm_map* m, const std::vector<long long>& want, long long* restored) {
  *restored = 0;
  DeviceMap& d = m->d;
  HostStore* hs = host_store(m);
  std::vector<long long> keys;
  for (long long k : want)
    if (hs->regions.count(k) && std::find(keys.begin(), keys.end(), k) == keys.end()) keys.push_back(k);
  if (keys.empty()) return cudaSuccess;
  PoolView v;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = read_pool(m, &v);
  if (e != cudaSuccess) return e;
  long long avail = (long long)v.free_slots.size() + (d.max_regions - v.region_count);
  if (avail < (long long)keys.size()) {
    // make room: evict the least recently used resident regions
    const long long live = (long long)live_slots(v).size();
    long long ev = 0;
    e = cache_evict(m, live - ((long long)keys.size() - avail), &ev);
    if (e == cudaSuccess) e = read_pool(m, &v);
    if (e != cudaSuccess) return e;
    avail = (long long)v.free_slots.size() + (d.max_regions - v.region_count);
    if (avail < (long long)keys.size()) return cudaErrorMemoryAllocation;
  }
  std::vector<int32_t> slots, nblocks, coords;
  for (long long k : keys) {
    const HostRegion& r = hs->regions[k];
    int32_t s;
    if (!v.free_slots.empty()) {
      s = v.free_slots.back();
      v.free_slots.pop_back();
    } else {
      s = v.region_count++;
    }
    int32_t nb = -1;
    if (r.ndt) {
      if (!v.free_ndt.empty()) {
        nb = v.free_ndt.back();
        v.free_ndt.pop_back();
      } else if (v.ndt_count < d.max_ndt) {
        nb = v.ndt_count++;
      } else {
        return cudaErrorMemoryAllocation;
      }
    }
    slots.push_back(s);
    nblocks.push_back(nb);
    for (int a = 0; a < 3; ++a) coords.push_back(r.coords[a]);
    const long long off = (long long)s * kRegionVoxels;
    if (r.occ) e = cudaMemcpyAsync(d.occ + off, r.occ, sizeof(float) * kRegionVoxels, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess && r.counts)
      e = cudaMemcpyAsync(d.counts + off, r.counts, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess && r.tsdf)
      e = cudaMemcpyAsync(d.tsdf + off, r.tsdf, sizeof(float2) * kRegionVoxels, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess && r.decay)
      e = cudaMemcpyAsync(d.decay + off, r.decay, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess && r.vmean)
      e = cudaMemcpyAsync(d.vmean + off, r.vmean, sizeof(unsigned long long) * kRegionVoxels, cudaMemcpyHostToDevice, 0);
    if (e == cudaSuccess && r.ndt)
      e = cudaMemcpyAsync(d.ndt + (long long)nb * 10 * kRegionVoxels, r.ndt, sizeof(long long) * 10 * kRegionVoxels,
                          cudaMemcpyHostToDevice, 0);
    if (e != cudaSuccess) return e;
  }
  e = cudaDeviceSynchronize();
  DevVec<long long> dk;
  DevVec<int32_t> ds, dn, dc;
  if (e == cudaSuccess) e = dk.load(keys);
  if (e == cudaSuccess) e = ds.load(slots);
  if (e == cudaSuccess) e = dn.load(nblocks);
  if (e == cudaSuccess) e = dc.load(coords);
  if (e != cudaSuccess) return e;
  const int nk = (int)keys.size();
  k_set_entries<<<(nk + kCacheBlock - 1) / kCacheBlock, kCacheBlock>>>(d, dk.p, ds.p, dn.p, dc.p, nk, 0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  e = write_pool(m, v);
  if (e != cudaSuccess) return e;
  for (long long k : keys) {
    HostRegion& r = hs->regions[k];
    hs->occ.put(r.occ);
    hs->counts.put(r.counts);
    hs->decay.put(r.decay);
    hs->vmean.put(r.vmean);
    hs->ndt.put(r.ndt);
    hs->tsdf.put(r.tsdf);
    hs->regions.erase(k);
  }
  *restored = (long long)keys.size();
  return cudaSuccess;
}

// Keys the last (rolled back) call asked to restore.
cudaError_t cache_pending(ohm_map* m, std::vector<long long>* keys) {
  CallCounters c;
  cudaError_t e = cudaMemcpy(&c, m->d.calls, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  const long long n = std::min<long long>((long long)c.restores, m->d.max_restore);
  return d2h(*keys, m->d.restore_keys, (size_t)n);
}

long long cache_host_regions(ohm_map* m) { return m->store ? (long long)m->store->regions.size() : 0; }

std::vector<long long> cache_all_keys(ohm_map* m) {
  std::vector<long long> k;
  if (m->store)
    for (const auto& kv : m->store->regions) k.push_back(kv.first);
  return k;
}

cudaError_t cache_resident(ohm_map* m, long long* resident) {
  PoolView v;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = read_pool(m, &v);
  if (e == cudaSuccess) *resident = (long long)live_slots(v).size();
  return e;
}

}  // namespace ohm
