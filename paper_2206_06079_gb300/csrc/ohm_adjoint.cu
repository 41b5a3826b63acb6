// Depth-image integration and the TSDF adjoint.
//
// ohm_integrate_depth back-projects a z-depth image into rays on the device
// and integrates them (every layer of the map, Sec. II-F for TSDF).
//
// ohm_tsdf_backward gives the gradient of L = sum_q g_q D(v_q), D the TSDF
// distance right after the frame was integrated, with respect to the frame's
// per-pixel depths and its pose (a left twist xi = (rho, phi) moving every
// world point p to p + rho + phi x p), with the voxel sets of the band walks
// and the per-voxel counts held fixed.  It recomputes each pixel's band walk
// instead of storing traces.  For an unclamped s = (e - c).u:
//   ds/de = u + r_perp / d,  ds/do = -r_perp / d,  r = e - c,
//   r_perp = r - (r.u) u,  dD/ds = 1 / W   (W = the weight after the frame),
// so per ray, with w_v = G(v) / W(v) summed over its unclamped band voxels,
//   dL/de = (sum w) u + (sum w r_perp) / d,  dL/do = -(sum w r_perp) / d,
//   dL/dz = dL/de . R p~,  p~ = ((u - cx) / fx, (v - cy) / fy, 1),
//   dL/drho += dL/de + dL/do,  dL/dphi += e x dL/de + o x dL/do.
//
// ohm_integrate_posed moves sensor-frame rays to the world by a pose and
// integrates them; ohm_ndt_backward gives the gradient of
// L = sum_q gm_q . mean(v_q) + gc_q . packed C(v_q), mean and C the NDT-OM
// sample statistics (Sec. II-D, III-C) right after that frame, with respect to
// the frame's sensor-frame endpoints and its pose twist, the voxel of every
// sample held fixed.  With n, S the voxel's count and sum of sample positions
// p (relative to its corner) and d = p_j - S / n,
//   dL/dp_j = (1 / n) [ gm + (G + G^T) d ],  G = upper-triangular(gc),
// then dL/de_sensor = R^T dL/dp_j and the twist as for the TSDF.
#include <cstring>
#include <string>
#include <vector>

#include "ohm_kernels.cuh"

namespace ohm {
namespace {

struct DepthFrame {
  const float* depth;
  int32_t width, height;
  double fx, fy, cx, cy;
  double R[9];
  double t[3];
  double z_min, z_max;
  const double* pxy;  // (u - cx) / fx for u < width, then (v - cy) / fy for v < height
};

// Back-projection of one pixel, one rounding per double operation:
// x = ((u - cx) / fx) z, y = ((v - cy) / fy) z, e_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k,
// rounded to float.  A depth outside (z_min, z_max] gives a NO_RETURN ray at z_max.
// The quotients depend on the column or the row only: they come from the
// frame's table, formed on the host by the same double operations.
__device__ __forceinline__ bool depth_ray(const DepthFrame& f, long long pix, float e[3], double pt[3]) {
  const int u = (int)(pix % f.width), v = (int)(pix / f.width);
  const double z = (double)f.depth[pix];
  const bool valid = z > f.z_min && z <= f.z_max;
  const double zz = valid ? z : f.z_max;
  const double px = f.pxy[u];
  const double py = f.pxy[f.width + v];
  const double x = __dmul_rn(px, zz), y = __dmul_rn(py, zz);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double a = __dmul_rn(f.R[3 * k], x);
    a = __dadd_rn(a, __dmul_rn(f.R[3 * k + 1], y));
    a = __dadd_rn(a, __dmul_rn(f.R[3 * k + 2], zz));
    a = __dadd_rn(a, f.t[k]);
    e[k] = __double2float_rn(a);
  }
  pt[0] = px;
  pt[1] = py;
  pt[2] = 1.0;
  return valid;
}

__global__ void __launch_bounds__(kBlock) k_depth_rays(DepthFrame f, float* origins, float* endpoints, uint8_t* flags) {
  const long long n = (long long)f.width * f.height;
  if (blockIdx.x == 0 && threadIdx.x < 3) origins[threadIdx.x] = __double2float_rn(f.t[threadIdx.x]);
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    float e[3];
    double pt[3];
    const bool valid = depth_ray(f, p, e, pt);
    endpoints[3 * p + 0] = e[0];
    endpoints[3 * p + 1] = e[1];
    endpoints[3 * p + 2] = e[2];
    flags[p] = valid ? 0 : kFlagNoReturn;
  }
}

__device__ __forceinline__ long long point_offset(const DeviceMap& m, const float* p) {
  long long q[3];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) ok = ok && isfinite(p[k]) && quantise(p[k], m.origin[k], m.scale, &q[k]);
  ok = ok && in_extent(q, m.frac_bits);
  if (!ok) return -1;
  const int F = m.frac_bits;
  const int32_t vx = (int32_t)(q[0] >> F), vy = (int32_t)(q[1] >> F), vz = (int32_t)(q[2] >> F);
  const int32_t slot = region_slot_of(m, vx, vy, vz);
  return slot < 0 ? -1 : voxel_offset(slot, local_morton(vx, vy, vz));
}

// G(v) += g_q for each query point (clear = 0), or G(v) = 0 (clear = 1).
__global__ void __launch_bounds__(kBlock) k_grad_scatter(DeviceMap m, const float* pts, const float* g, long long n,
                                                         int clear) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const long long off = point_offset(m, pts + 3 * q);
    if (off < 0) continue;
    if (clear)
      m.grad[off] = 0.f;
    else
      atomicAdd(m.grad + off, g[q]);
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(kBlock) k_tsdf_backward(DeviceMap m, DepthFrame f, float* grad_depth,
                                                          double* grad_twist) {
  __shared__ double red[kBlock / 32][6];
  const long long n = (long long)f.width * f.height;
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  const long long half = U >> 1;
  const float to_m = (float)(m.voxel_size / (double)U);
  double acc[6] = {0, 0, 0, 0, 0, 0};
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long n_round = (n + stride - 1) / stride * stride;  // whole blocks iterate together
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_round; p += stride) {
    float gz = 0.f;
    if (p < n) {
      float e[3], o[3];
      double pt[3];
      bool ok = depth_ray(f, p, e, pt);
#pragma unroll
      for (int k = 0; k < 3; ++k) o[k] = __double2float_rn(f.t[k]);
      long long qo[3], qe[3];
      ok = ok && quantise_ray(m, o, e, qo, qe);
      // the band of the forward pass, recomputed the same way
      long long a[3], b[3];
      float u[3], lenf = 0.f;
      if (ok) {
        bool in_range = false;
        if (!tsdf_band_ff(qo, qe, m.band, &in_range, a, b, u, &lenf)) {
          double d[3];
          const double len = ray_length(qo, qe, d);
          in_range = len > m.rmin_q && len <= m.rmax_q;
          if (in_range && in_extent(qo, F) && in_extent(qe, F)) tsdf_band(qo, d, len, m.tau_q, a, b, u);
          lenf = (float)len;
        }
        ok = in_range && in_extent(qo, F) && in_extent(qe, F);
      }
      if (ok) {
        const float dm = lenf * to_m;  // ray length in metres (chain rule only)
        Walker w;
        walker_init(w, a, b, F, 0, 0);
        int32_t slot = region_slot_of(m, w.vx, w.vy, w.vz);
        uint32_t mo = local_morton(w.vx, w.vy, w.vz);
        float A = 0.f, B[3] = {0.f, 0.f, 0.f};
        while (slot >= 0) {
          const long long off = voxel_offset(slot, mo);
          const float G = m.grad[off];
          if (G != 0.f) {
            const float ex = (float)(qe[0] - ((long long)w.vx * U + half));
            const float ey = (float)(qe[1] - ((long long)w.vy * U + half));
            const float ez = (float)(qe[2] - ((long long)w.vz * U + half));
            const float s = (ex * u[0] + ey * u[1] + ez * u[2]) * to_m;  // as in the forward pass
            if (s > -m.tau_m && s < m.tau_m) {
              const float wv = G / m.tsdf[off].y;
              const float r[3] = {ex * to_m, ey * to_m, ez * to_m};
              A += wv;
#pragma unroll
              for (int k = 0; k < 3; ++k) B[k] += wv * (r[k] - s * u[k]);
            }
          }
          if (w.total == 0) break;
          const int axis = walker_choose(w);
          int32_t c, sg;
          walker_step(w, axis, &c, &sg);
          mo = morton_step(mo, morton_mask(axis), sg);
          if ((c & ((1 << kRegionShift) - 1)) == (sg > 0 ? 0 : (1 << kRegionShift) - 1))
            slot = region_slot_of(m, w.vx, w.vy, w.vz);
        }
        // The chain rule from here on is plain float arithmetic (its inputs
        // are floats; the gradients are checked to 1e-3 relative), summed
        // over pixels in double.  The band above is recomputed exactly as
        // the forward pass forms it (the same float-float settlement, else
        // the same double evaluation), since it decides the voxel set.
        const float rdm = 1.0f / dm;
        float ge[3], go[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          go[k] = -B[k] * rdm;
          ge[k] = A * u[k] - go[k];
        }
        const float ptf[3] = {(float)pt[0], (float)pt[1], (float)pt[2]};
        float dz = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k)
          dz += ge[k] * ((float)f.R[3 * k] * ptf[0] + (float)f.R[3 * k + 1] * ptf[1] + (float)f.R[3 * k + 2] * ptf[2]);
        gz = dz;
        const float O[3] = {(float)f.t[0], (float)f.t[1], (float)f.t[2]};
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[k] += (double)(ge[k] + go[k]);
        acc[3] += (double)(e[1] * ge[2] - e[2] * ge[1] + O[1] * go[2] - O[2] * go[1]);
        acc[4] += (double)(e[2] * ge[0] - e[0] * ge[2] + O[2] * go[0] - O[0] * go[2]);
        acc[5] += (double)(e[0] * ge[1] - e[1] * ge[0] + O[0] * go[1] - O[1] * go[0]);
      }
      grad_depth[p] = gz;
    }
  }
  // block reduction of the twist gradient, one double atomic per component
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) v += red[i][threadIdx.x];
    atomicAdd(grad_twist + threadIdx.x, v);
  }
}

// A camera-to-world pose [R | t], row major.
struct Pose34 {
  double m[12];
};

// p_k = ((R_k0 x + R_k1 y) + R_k2 z) + t_k in double, one rounding per
// operation, rounded to float (the depth back-projection's order).
__device__ __forceinline__ void pose_point(const Pose34& P, const float* in, float* out) {
  const double x = in[0], y = in[1], z = in[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double a = __dmul_rn(P.m[4 * k], x);
    a = __dadd_rn(a, __dmul_rn(P.m[4 * k + 1], y));
    a = __dadd_rn(a, __dmul_rn(P.m[4 * k + 2], z));
    out[k] = __double2float_rn(__dadd_rn(a, P.m[4 * k + 3]));
  }
}

__global__ void __launch_bounds__(kBlock) k_pose_rays(Pose34 P, CallArgs in, float* origins, float* endpoints,
                                                      uint8_t* flags) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < in.n; i += (long long)gridDim.x * blockDim.x) {
    pose_point(P, in.endpoints + 3 * i, endpoints + 3 * i);
    if (i < in.n_origins) pose_point(P, in.origins + 3 * i, origins + 3 * i);
    flags[i] = in.flags ? in.flags[i] : 0;
  }
}

// Upstream weights of the NDT statistics per voxel: 9 floats (mean x y z,
// covariance xx xy xz yy yz zz) per voxel of every NDT block.
__device__ __forceinline__ float* ndt_grad_of(const DeviceMap& m, const float* p) {
  long long q[3];
  bool ok = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) ok = ok && isfinite(p[k]) && quantise(p[k], m.origin[k], m.scale, &q[k]);
  ok = ok && in_extent(q, m.frac_bits);
  if (!ok) return nullptr;
  const int F = m.frac_bits;
  const int32_t vx = (int32_t)(q[0] >> F), vy = (int32_t)(q[1] >> F), vz = (int32_t)(q[2] >> F);
  const int32_t slot = region_slot_of(m, vx, vy, vz);
  const int32_t ns = slot < 0 ? -1 : m.ndt_slot[slot];
  if (ns < 0) return nullptr;  // no samples in the region: nothing to differentiate
  return m.ndt_grad + ((long long)ns * kRegionVoxels + local_morton(vx, vy, vz)) * 9;
}

__global__ void __launch_bounds__(kBlock) k_ndt_grad_scatter(DeviceMap m, const float* pts, const float* gmean,
                                                             const float* gcov, long long n, int clear) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    float* g = ndt_grad_of(m, pts + 3 * q);
    if (!g) continue;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (clear)
        g[k] = 0.f;
      else
        atomicAdd(g + k, k < 3 ? gmean[3 * q + k] : gcov[6 * q + k - 3]);
    }
  }
}

// Per ray of the frame (world rays in `a`, as integrated): the sample's voxel
// by the quantisation and truncation of the forward pass, then dL/dp from the
// voxel's moments and weights.
__global__ void __launch_bounds__(kBlock) k_ndt_backward(DeviceMap m, CallArgs a, Pose34 P, float* grad_e,
                                                         double* grad_twist) {
  __shared__ double red[kBlock / 32][6];
  const int F = m.frac_bits;
  const long long U = 1LL << F;
  const double cell = m.voxel_size / (double)U;
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const long long n = a.n;
  const long long nb = ((n + kBlock - 1) / kBlock) * kBlock;  // every thread of a block reaches the reduction
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nb; i += (long long)gridDim.x * blockDim.x) {
    if (i >= n) continue;
    double gp[3] = {0.0, 0.0, 0.0};
    float o[3], e[3];
    uint8_t flag;
    load_ray(a, i, o, e, &flag);
    long long qo[3], qe[3];
    bool ok = (flag & kFlagNoReturn) == 0 && quantise_ray(m, o, e, qo, qe);
    if (ok) {
      double d[3];
      ok = ray_length(qo, qe, d) <= m.rmax_q && in_extent(qo, F) && in_extent(qe, F);
    }
    if (ok) {
      const int32_t v[3] = {(int32_t)(qe[0] >> F), (int32_t)(qe[1] >> F), (int32_t)(qe[2] >> F)};
      const int32_t slot = region_slot_of(m, v[0], v[1], v[2]);
      const int32_t ns = slot < 0 ? -1 : m.ndt_slot[slot];
      if (ns < 0) {
        atomicOr(m.status, kStatusMissing);
      } else {
        const uint32_t mo = local_morton(v[0], v[1], v[2]);
        const float* g = m.ndt_grad + ((long long)ns * kRegionVoxels + mo) * 9;
        float w[9];
        bool any = false;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
          w[k] = g[k];
          any = any || w[k] != 0.f;
        }
        const long long* mom = m.ndt + (long long)ns * 10 * kRegionVoxels + mo;
        const double cnt = (double)mom[0];
        if (any && cnt > 0.0) {
          double dv[3];
#pragma unroll
          for (int k = 0; k < 3; ++k)
            dv[k] = (double)(qe[k] - (long long)v[k] * U) * cell - (double)mom[(long long)(1 + k) * kRegionVoxels] * cell / cnt;
          // (G + G^T) d with G upper triangular from the packed xx xy xz yy yz zz
          const double Gs[3][3] = {{2.0 * w[3], w[4], w[5]}, {w[4], 2.0 * w[6], w[7]}, {w[5], w[7], 2.0 * w[8]}};
#pragma unroll
          for (int k = 0; k < 3; ++k) gp[k] = ((double)w[k] + Gs[k][0] * dv[0] + Gs[k][1] * dv[1] + Gs[k][2] * dv[2]) / cnt;
        }
      }
    }
    // sensor frame: dL/de = R^T dL/dp
#pragma unroll
    for (int c = 0; c < 3; ++c)
      grad_e[3 * i + c] = (float)(P.m[c] * gp[0] + P.m[4 + c] * gp[1] + P.m[8 + c] * gp[2]);
    const double E[3] = {e[0], e[1], e[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) acc[k] += gp[k];
    acc[3] += E[1] * gp[2] - E[2] * gp[1];
    acc[4] += E[2] * gp[0] - E[0] * gp[2];
    acc[5] += E[0] * gp[1] - E[1] * gp[0];
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double v = 0.0;
    for (int i = 0; i < kBlock / 32; ++i) v += red[i][threadIdx.x];
    atomicAdd(grad_twist + threadIdx.x, v);
  }
}

bool frame_from(const float* depth, int32_t width, int32_t height, const double* K, const double* pose, double z_min,
                double z_max, DepthFrame* f) {
  if (!depth || width < 1 || height < 1 || !K || !pose || !(z_max > z_min)) return false;
  f->depth = depth;
  f->width = width;
  f->height = height;
  f->fx = K[0];
  f->fy = K[1];
  f->cx = K[2];
  f->cy = K[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) f->R[3 * r + c] = pose[4 * r + c];
    f->t[r] = pose[4 * r + 3];
  }
  f->z_min = z_min;
  f->z_max = z_max;
  f->pxy = nullptr;
  return f->fx != 0.0 && f->fy != 0.0;
}

// The frame's per-column and per-row quotients, kept on the device for the
// last image size and intrinsics (rebuilt when they change).
cudaError_t frame_tables(ohm_map* map, DepthFrame* f, cudaStream_t s) {
  const double key[6] = {(double)f->width, (double)f->height, f->fx, f->fy, f->cx, f->cy};
  const long long n = (long long)f->width + f->height;
  if (map->pxy && std::memcmp(key, map->pxy_key, sizeof(key)) == 0) {
    f->pxy = map->pxy;
    return cudaSuccess;
  }
  // earlier work of the map may still read the old table
  cudaError_t e = map->work_done ? cudaStreamWaitEvent(s, map->work_done, 0) : cudaSuccess;
  if (e == cudaSuccess && n > map->pxy_cap) {
    if (map->pxy) {
      e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaFree(map->pxy);
      map->pxy = nullptr;
      map->pxy_cap = 0;
    }
    const long long cap = n > 4096 ? n : 4096;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&map->pxy), sizeof(double) * cap);
    if (e != cudaSuccess) return e;
    map->pxy_cap = cap;
  }
  if (e != cudaSuccess) return e;
  std::vector<double> t((size_t)n);
  for (int u = 0; u < f->width; ++u) t[u] = ((double)u - f->cx) / f->fx;
  for (int v = 0; v < f->height; ++v) t[f->width + v] = ((double)v - f->cy) / f->fy;
  e = cudaMemcpyAsync(map->pxy, t.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  std::memcpy(map->pxy_key, key, sizeof(key));
  f->pxy = map->pxy;
  return cudaSuccess;
}

ohm_status afail(ohm_status code, const std::string& msg) {
  set_last_error(msg);
  return code;
}

bool is_device(const void* p) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace ohm

extern "C" {

ohm_status ohm_integrate_depth(ohm_map* map, const float* depth, int32_t width, int32_t height,
                               const double* intrinsics, const double* pose, double z_min, double z_max,
                               void* stream) {
  using namespace ohm;
  if (!map) return afail(OHM_ERR_INVALID, "integrate_depth: map is NULL");
  DepthFrame f;
  if (!frame_from(depth, width, height, intrinsics, pose, z_min, z_max, &f))
    return afail(OHM_ERR_INVALID, "integrate_depth: bad image, intrinsics, pose or depth range");
  const long long n = (long long)width * height;
  if (n > map->p.max_rays) return afail(OHM_ERR_INVALID, "integrate_depth: width * height exceeds max_rays");
  if (!is_device(depth)) return afail(OHM_ERR_INVALID, "integrate_depth: depth must be device memory");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != map->device) cudaSetDevice(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = (int)((n + kBlock - 1) / kBlock < 4096 ? (n + kBlock - 1) / kBlock : 4096);
  cudaError_t et = frame_tables(map, &f, s);
  if (et != cudaSuccess) {
    if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
    return afail(OHM_ERR_CUDA, std::string("integrate_depth: ") + cudaGetErrorString(et));
  }
  k_depth_rays<<<blocks, kBlock, 0, s>>>(f, map->stage_origins, map->stage_endpoints, map->stage_flags);
  map->launches += 1;
  CallArgs a;
  a.origins = map->stage_origins;
  a.endpoints = map->stage_endpoints;
  a.flags = map->stage_flags;
  a.n = n;
  a.n_origins = 1;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_integrate(map, a, s);
  if (e == cudaSuccess) note_work(map, s);
  if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return afail(OHM_ERR_CUDA, std::string("integrate_depth: ") + cudaGetErrorString(e));
  return OHM_OK;
}

ohm_status ohm_tsdf_backward(ohm_map* map, const float* depth, int32_t width, int32_t height,
                             const double* intrinsics, const double* pose, double z_min, double z_max,
                             const float* query_points, const float* grad_query, int64_t n_query, float* grad_depth,
                             double* grad_twist, void* stream) {
  using namespace ohm;
  if (!map) return afail(OHM_ERR_INVALID, "tsdf_backward: map is NULL");
  if (!(map->p.layers & OHM_LAYER_TSDF)) return afail(OHM_ERR_UNSUPPORTED, "tsdf_backward: map has no TSDF layer");
  DepthFrame f;
  if (!frame_from(depth, width, height, intrinsics, pose, z_min, z_max, &f))
    return afail(OHM_ERR_INVALID, "tsdf_backward: bad image, intrinsics, pose or depth range");
  if (n_query < 0 || (n_query > 0 && (!query_points || !grad_query)) || !grad_depth || !grad_twist)
    return afail(OHM_ERR_INVALID, "tsdf_backward: NULL buffer");
  const void* bufs[] = {depth, grad_depth, grad_twist};
  for (const void* b : bufs)
    if (!is_device(b)) return afail(OHM_ERR_INVALID, "tsdf_backward: buffers must be device memory");
  if (n_query > 0 && (!is_device(query_points) || !is_device(grad_query)))
    return afail(OHM_ERR_INVALID, "tsdf_backward: buffers must be device memory");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != map->device) cudaSetDevice(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!map->d.grad) {
    // per-voxel gradient weights, allocated on the first backward call
    e = cudaMalloc(reinterpret_cast<void**>(&map->d.grad), sizeof(float) * (size_t)map->p.max_regions * kRegionVoxels);
    if (e == cudaSuccess) e = cudaMemset(map->d.grad, 0, sizeof(float) * (size_t)map->p.max_regions * kRegionVoxels);
  }
  const long long n = (long long)width * height;
  const int qb = (int)(n_query > 0 ? ((n_query + kBlock - 1) / kBlock < 4096 ? (n_query + kBlock - 1) / kBlock : 4096) : 0);
  const int pb = (int)((n + kBlock - 1) / kBlock < 4096 ? (n + kBlock - 1) / kBlock : 4096);
  if (e == cudaSuccess) e = frame_tables(map, &f, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(grad_twist, 0, 6 * sizeof(double), s);
  if (e == cudaSuccess && qb) {
    k_grad_scatter<<<qb, kBlock, 0, s>>>(map->d, query_points, grad_query, n_query, 0);
    map->launches += 1;
  }
  if (e == cudaSuccess) {
    k_tsdf_backward<<<pb, kBlock, 0, s>>>(map->d, f, grad_depth, grad_twist);
    map->launches += 1;
  }
  if (e == cudaSuccess && qb) {
    k_grad_scatter<<<qb, kBlock, 0, s>>>(map->d, query_points, grad_query, n_query, 1);
    map->launches += 1;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) note_work(map, s);
  if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return afail(OHM_ERR_CUDA, std::string("tsdf_backward: ") + cudaGetErrorString(e));
  return OHM_OK;
}

static ohm_status posed_args(ohm_map* map, const double* pose, const float* origins, int64_t n_origins,
                             const float* endpoints, const uint8_t* flags, int64_t n, const char* who,
                             ohm::Pose34* P) {
  using namespace ohm;
  if (!map || !pose) return afail(OHM_ERR_INVALID, std::string(who) + ": NULL map or pose");
  if (n < 0 || n > map->p.max_rays) return afail(OHM_ERR_INVALID, std::string(who) + ": n outside [0, max_rays]");
  if (n > 0 && (!origins || !endpoints || (n_origins != 1 && n_origins != n)))
    return afail(OHM_ERR_INVALID, std::string(who) + ": bad origins / endpoints");
  if (n > 0 && (!is_device(origins) || !is_device(endpoints) || (flags && !is_device(flags))))
    return afail(OHM_ERR_INVALID, std::string(who) + ": rays must be device memory");
  for (int k = 0; k < 12; ++k) {
    if (!std::isfinite(pose[k])) return afail(OHM_ERR_INVALID, std::string(who) + ": pose not finite");
    P->m[k] = pose[k];
  }
  return OHM_OK;
}

// Transform into the map's staging buffers; returns the call arguments.
static cudaError_t stage_posed(ohm_map* map, const ohm::Pose34& P, const float* origins, int64_t n_origins,
                               const float* endpoints, const uint8_t* flags, int64_t n, cudaStream_t s,
                               ohm::CallArgs* a) {
  using namespace ohm;
  CallArgs in;
  in.origins = origins;
  in.endpoints = endpoints;
  in.flags = flags;
  in.n = n;
  in.n_origins = n_origins;
  const int blocks = (int)((n + kBlock - 1) / kBlock < 4096 ? (n + kBlock - 1) / kBlock : 4096);
  k_pose_rays<<<blocks > 0 ? blocks : 1, kBlock, 0, s>>>(P, in, map->stage_origins, map->stage_endpoints,
                                                         map->stage_flags);
  map->launches += 1;
  a->origins = map->stage_origins;
  a->endpoints = map->stage_endpoints;
  a->flags = map->stage_flags;
  a->n = n;
  a->n_origins = n_origins;
  return cudaGetLastError();
}

ohm_status ohm_integrate_posed(ohm_map* map, const double* pose, const float* origins, int64_t n_origins,
                               const float* endpoints, const uint8_t* flags, int64_t n, void* stream) {
  using namespace ohm;
  Pose34 P;
  const ohm_status st = posed_args(map, pose, origins, n_origins, endpoints, flags, n, "integrate_posed", &P);
  if (st != OHM_OK || n == 0) return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != map->device) cudaSetDevice(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CallArgs a;
  cudaError_t e = stage_posed(map, P, origins, n_origins, endpoints, flags, n, s, &a);
  if (e == cudaSuccess) e = launch_integrate(map, a, s);
  if (e == cudaSuccess) note_work(map, s);
  if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return afail(OHM_ERR_CUDA, std::string("integrate_posed: ") + cudaGetErrorString(e));
  return OHM_OK;
}

ohm_status ohm_ndt_backward(ohm_map* map, const double* pose, const float* origins, int64_t n_origins,
                            const float* endpoints, const uint8_t* flags, int64_t n, const float* query_points,
                            const float* grad_mean, const float* grad_cov, int64_t n_query, float* grad_endpoints,
                            double* grad_twist, void* stream) {
  using namespace ohm;
  Pose34 P;
  ohm_status st = posed_args(map, pose, origins, n_origins, endpoints, flags, n, "ndt_backward", &P);
  if (st != OHM_OK) return st;
  if (!(map->p.layers & OHM_LAYER_NDT)) return afail(OHM_ERR_UNSUPPORTED, "ndt_backward: map has no NDT layer");
  if (map->p.ndt_clear_below > -INFINITY)
    return afail(OHM_ERR_UNSUPPORTED, "ndt_backward: sample clearing changes the statistics discontinuously; "
                                      "the adjoint needs ndt_clear_below = -inf");
  if (n_query < 0 || (n_query > 0 && (!query_points || !grad_mean || !grad_cov)) || (n > 0 && !grad_endpoints) ||
      !grad_twist)
    return afail(OHM_ERR_INVALID, "ndt_backward: NULL buffer");
  if ((n > 0 && !is_device(grad_endpoints)) || !is_device(grad_twist) ||
      (n_query > 0 && (!is_device(query_points) || !is_device(grad_mean) || !is_device(grad_cov))))
    return afail(OHM_ERR_INVALID, "ndt_backward: buffers must be device memory");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != map->device) cudaSetDevice(map->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (!map->d.ndt_grad) {
    // upstream weights per NDT voxel, allocated on the first backward call
    const size_t bytes = sizeof(float) * 9 * (size_t)map->d.max_ndt * kRegionVoxels;
    e = cudaMalloc(reinterpret_cast<void**>(&map->d.ndt_grad), bytes);
    if (e == cudaSuccess) e = cudaMemset(map->d.ndt_grad, 0, bytes);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(grad_twist, 0, 6 * sizeof(double), s);
  const int qb = (int)(n_query > 0 ? ((n_query + kBlock - 1) / kBlock < 4096 ? (n_query + kBlock - 1) / kBlock : 4096) : 0);
  if (e == cudaSuccess && qb) {
    k_ndt_grad_scatter<<<qb, kBlock, 0, s>>>(map->d, query_points, grad_mean, grad_cov, n_query, 0);
    map->launches += 1;
  }
  if (e == cudaSuccess && n > 0) {
    CallArgs a;
    e = stage_posed(map, P, origins, n_origins, endpoints, flags, n, s, &a);
    const int pb = (int)((n + kBlock - 1) / kBlock < 4096 ? (n + kBlock - 1) / kBlock : 4096);
    if (e == cudaSuccess) {
      k_ndt_backward<<<pb, kBlock, 0, s>>>(map->d, a, P, grad_endpoints, grad_twist);
      map->launches += 1;
    }
  }
  if (e == cudaSuccess && qb) {
    k_ndt_grad_scatter<<<qb, kBlock, 0, s>>>(map->d, query_points, grad_mean, grad_cov, n_query, 1);
    map->launches += 1;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) note_work(map, s);
  if (prev >= 0 && prev != map->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return afail(OHM_ERR_CUDA, std::string("ndt_backward: ") + cudaGetErrorString(e));
  return OHM_OK;
}

ohm_status ohm_twist_pose(const double* xi, const double* pose0, double* pose) {
  if (!xi || !pose0 || !pose) return ohm::afail(OHM_ERR_INVALID, "twist_pose: NULL argument");
  // T = exp(xi) as a rigid motion (Rodrigues' formula for the rotation R and
  // V rho for the translation, V the left Jacobian of SO(3)); pose = T pose0.
  const double rho[3] = {xi[0], xi[1], xi[2]}, phi[3] = {xi[3], xi[4], xi[5]};
  const double th = std::sqrt(phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2]);
  const double Kx[3][3] = {{0.0, -phi[2], phi[1]}, {phi[2], 0.0, -phi[0]}, {-phi[1], phi[0], 0.0}};
  double K2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) K2[i][j] = Kx[i][0] * Kx[0][j] + Kx[i][1] * Kx[1][j] + Kx[i][2] * Kx[2][j];
  // small angles: the series to first order, as an exact rotation is not needed there
  const double a = th < 1e-12 ? 1.0 : std::sin(th) / th;
  const double b = th < 1e-12 ? 0.0 : (1.0 - std::cos(th)) / (th * th);
  const double bv = th < 1e-12 ? 0.5 : b;
  const double cv = th < 1e-12 ? 0.0 : (th - std::sin(th)) / (th * th * th);
  double R[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double I = i == j ? 1.0 : 0.0;
      R[i][j] = I + a * Kx[i][j] + b * K2[i][j];
      V[i][j] = I + bv * Kx[i][j] + cv * K2[i][j];
    }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      pose[4 * i + j] = R[i][0] * pose0[0 + j] + R[i][1] * pose0[4 + j] + R[i][2] * pose0[8 + j];
    pose[4 * i + 3] = R[i][0] * pose0[3] + R[i][1] * pose0[7] + R[i][2] * pose0[11] +
                      (V[i][0] * rho[0] + V[i][1] * rho[1] + V[i][2] * rho[2]);
  }
  return OHM_OK;
}

}  // extern "C"
