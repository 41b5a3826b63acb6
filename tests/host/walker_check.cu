// Host-side check of the device walkers: compiles the library's walkers
// (ohm_device.cuh, host+device functions) for the CPU and prints, for every
// ray, the voxels visited by all of its segments in segment order.  The
// Python test compares this with the oracle's walk.  No GPU is needed.
//
// argv[1] = mode:
//   plain  Walker from the end points, segments of S dominant-axis steps
//          (the allocation-free entry point's walk)
//   rec    Walker from the per-ray record, the integrate kernels' balanced
//          segments for a target of S voxels (the decay-layer walk)
//   fast   the filtered walk (FWalker) of the integrate kernels, from the
//          per-ray record, with the kernels' sign-normalised Morton stepping
//          and region tracking
// stdin:  F S n, then n lines "ax ay az bx by bz" (fixed point)
// stdout: per ray "count" then count lines "x y z"
// stderr: "exact <n>" -- near-ties the fast walk decided exactly
// exit codes: 2 Morton mismatch, 3 bad record, 4 region tracking mismatch,
//             5 segment end or visit count mismatch
#include <climits>
#include <cstdio>
#include <cstring>

#include "../../paper_2206_06079_gb300/csrc/ohm_device.cuh"

static int vox[1 << 20][3];

int main(int argc, char** argv) {
  int F, S;
  long long n;
  const char* mode = argc > 1 ? argv[1] : "plain";
  const bool plain = std::strcmp(mode, "plain") == 0, fast = std::strcmp(mode, "fast") == 0;
  if (scanf("%d %d %lld", &F, &S, &n) != 3) return 1;
  long long exact_steps = 0;
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
    const long long am = b[M] - a[M];
    ohm::RayRec rec;
    rec.flags = 0;
    rec.inv = ohm::reciprocal64((unsigned long long)(am < 0 ? -am : am));
    ohm::ray_constants(a, b, F, &rec);
    int nseg;
    if (plain) {
      nseg = ohm::segment_count(nmaj, S);
    } else {
      const ohm::SegSplit sp = ohm::ray_segment_split(nmaj, nsteps, S);
      nseg = sp.nseg;
      rec.flags |= (M << ohm::kRayAxisShift) | (int32_t)((uint32_t)sp.q << ohm::kRaySegShift);
      rec.nseg = nseg;
      long long bb[3];
      ohm::ray_end(rec, F, bb);
      if (bb[0] != b[0] || bb[1] != b[1] || bb[2] != b[2]) return 3;
    }
    long long c = 0;
    for (int j = 0; j < nseg; ++j) {
      const bool last = j == nseg - 1;
      if (fast) {
        ohm::SegStart s;
        ohm::segment_start(rec, F, j, &s);
        ohm::FWalker f;
        ohm::fwalker_init(f, rec, F, s.c);
        const uint32_t neg = ohm::morton_neg(rec.flags);
        const int32_t sgn = (rec.flags >> ohm::kRaySignShift) & 7;
        uint32_t mo = ohm::region_morton(s.v[0], s.v[1], s.v[2]) ^ neg;
        int32_t v[3] = {s.v[0], s.v[1], s.v[2]};
        int32_t rc[3] = {s.v[0] >> 5, s.v[1] >> 5, s.v[2] >> 5};
        for (long long left = s.visits; left > 0; --left) {
          if ((mo ^ neg) != ohm::region_morton(v[0], v[1], v[2])) return 2;
          if (rc[0] != (v[0] >> 5) || rc[1] != (v[1] >> 5) || rc[2] != (v[2] >> 5)) return 4;
          if (c < (1 << 20)) {
            vox[c][0] = v[0];
            vox[c][1] = v[1];
            vox[c][2] = v[2];
          }
          ++c;
          if (left == 1) {
            if (v[0] != s.ve[0] || v[1] != s.ve[1] || v[2] != s.ve[2]) return 5;
            break;
          }
          int axis = ohm::fwalker_pick(f);
          if (axis < 0) {
            axis = ohm::exact_pick(rec, F, (int32_t)f.cx, (int32_t)f.cy, (int32_t)f.cz);
            ++exact_steps;
          }
          ohm::fwalker_advance(f, axis);
          const int32_t d = ((sgn >> axis) & 1) ? -1 : 1;
          v[axis] += d;
          if (ohm::morton_advance(mo, ohm::morton_mask(axis))) rc[axis] += d;
        }
        continue;
      }
      ohm::Walker w;
      int mrem;
      if (plain) {
        ohm::walker_init(w, a, b, F, M, (long long)j * S, 0ULL);
        mrem = last ? INT_MAX : S - 1;
      } else {
        long long K0, K1;
        ohm::segment_bounds(nmaj, rec.nseg, (int32_t)((uint32_t)rec.flags >> ohm::kRaySegShift), j, &K0, &K1);
        ohm::walker_init_rec(w, rec, F, M, K0);
        mrem = last ? INT_MAX : (int)(K1 - K0 - 1);
      }
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
  fprintf(stderr, "exact %lld\n", exact_steps);
  return 0;
}
