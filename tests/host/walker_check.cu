// Host-side check of the device walker: compiles the library's walker
// (ohm_device.cuh, host+device functions) for the CPU and prints, for every
// ray, the voxels visited by all of its segments in segment order.  The
// Python test compares this with the oracle's walk.  No GPU is needed.
//
// stdin:  F S n, then n lines "ax ay az bx by bz" (fixed point)
// stdout: per ray "count" then count lines "x y z"
#include <climits>
#include <cstdio>

#include "../../paper_2206_06079_gb300/csrc/ohm_device.cuh"

int main(int argc, char** argv) {
  int F, S;
  long long n;
  const bool use_inv = argc > 1;  // jump into segments with the reciprocal division
  if (scanf("%d %d %lld", &F, &S, &n) != 3) return 1;
  static int vox[1 << 20][3];
  for (long long r = 0; r < n; ++r) {
    long long a[3], b[3];
    if (scanf("%lld %lld %lld %lld %lld %lld", &a[0], &a[1], &a[2], &b[0], &b[1], &b[2]) != 6) return 1;
    int32_t nmaj;
    const int M = ohm::dominant_axis(a, b, F, &nmaj);
    long long nsteps = 0;
    for (int k = 0; k < 3; ++k) {
      const long long dv = (b[k] >> F) - (a[k] >> F);
      nsteps += dv < 0 ? -dv : dv;
    }
    // the kernels' per-ray segment length (S is the target voxel steps per segment)
    const int Sr = use_inv ? ohm::ray_segment_steps(nmaj, nsteps, S) : S;
    const int nseg = ohm::segment_count(nmaj, Sr);
    long long c = 0;
    for (int j = 0; j < nseg; ++j) {
      ohm::Walker w;
      const long long am = b[M] - a[M];
      const unsigned long long inv = use_inv ? ohm::reciprocal64((unsigned long long)(am < 0 ? -am : am)) : 0ULL;
      if (use_inv) {
        // the kernels' path: per-ray constants, then the segment's state
        ohm::RayRec rec;
        rec.flags = 0;
        rec.inv = inv;
        ohm::ray_constants(a, b, F, &rec);
        long long bb[3];
        ohm::ray_end(rec, F, bb);
        if (bb[0] != b[0] || bb[1] != b[1] || bb[2] != b[2]) return 3;
        ohm::walker_init_rec(w, rec, F, M, (long long)j * Sr);
      } else {
        ohm::walker_init(w, a, b, F, M, (long long)j * Sr, inv);
      }
      const bool last = j == nseg - 1;
      int mrem = last ? INT_MAX : Sr - 1;
      uint32_t mo = ohm::morton((uint32_t)(w.vx & 31), (uint32_t)(w.vy & 31), (uint32_t)(w.vz & 31));
      for (;;) {
        // the incrementally stepped Morton index must equal the recomputed one
        if (mo != ohm::morton((uint32_t)(w.vx & 31), (uint32_t)(w.vy & 31), (uint32_t)(w.vz & 31))) return 2;
        if (c < (1 << 20)) {
          vox[c][0] = w.vx;
          vox[c][1] = w.vy;
          vox[c][2] = w.vz;
        }
        ++c;
        if (w.total == 0) break;
        const int axis = ohm::walker_choose(w);
        if (axis == M) {
          if (mrem == 0) break;
          --mrem;
        }
        int32_t cc, sg;
        ohm::walker_step(w, axis, &cc, &sg);
        mo = ohm::morton_step(mo, ohm::morton_mask(axis), sg);
      }
    }
    printf("%lld\n", c);
    for (long long i = 0; i < c && i < (1 << 20); ++i) printf("%d %d %d\n", vox[i][0], vox[i][1], vox[i][2]);
  }
  return 0;
}
