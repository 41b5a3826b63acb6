// Host-side check of tsdf_band_ff (ohm_device.cuh, compiled for the CPU): on
// every case it settles, its range test, band end points and unit direction
// must equal those of the double evaluation (ray_length's length, the range
// test on it, tsdf_band); on the rest it must say so (return false).  Cases:
// random rays of voxel to range scale, rays built so that an end point lands
// on a half-integer, rays whose length sits at the range limits or at tau,
// and random band constants.  No GPU is needed.
//
// stdout: "cases <n> settled <k> random <n> settled <k>" (all cases, then the
// random rays alone); exit code 1 on a mismatch (the case is
// printed to stderr), 2 when a float-float primitive check fails.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "../../paper_2206_06079_gb300/csrc/ohm_device.cuh"

static uint64_t state = 0x2545f4914f6cdd1dULL;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static long long uniform(long long lo, long long hi) { return lo + (long long)(next_u64() % (uint64_t)(hi - lo + 1)); }
static double unit() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }

// ray_length of the kernels, on the host: every operation in IEEE double.
static double length_of(const long long qo[3], const long long qe[3], double d[3]) {
  for (int k = 0; k < 3; ++k) d[k] = (double)(qe[k] - qo[k]);
  double l2 = d[0] * d[0];
  l2 = l2 + d[1] * d[1];
  l2 = l2 + d[2] * d[2];
  return std::sqrt(l2);
}

static long long n_cases = 0, n_settled = 0;

static int check(const long long qo[3], const long long qe[3], double tau, double rmin, double rmax) {
  double d[3];
  const double len = length_of(qo, qe, d);
  if (!(len > 0.0)) return 0;
  ++n_cases;
  const bool in_range = len > rmin && len <= rmax;
  long long a0[3] = {0, 0, 0}, b0[3] = {0, 0, 0};
  float u0[3] = {0.f, 0.f, 0.f};
  if (in_range) ohm::tsdf_band(qo, d, len, tau, a0, b0, u0);
  ohm::BandConsts c;
  c.tau = ohm::ff_of_double(tau);
  c.rmin = ohm::ff_of_double(rmin);
  c.rmax = ohm::ff_of_double(rmax);
  bool r1 = false;
  long long a1[3], b1[3];
  float u1[3];
  if (!ohm::tsdf_band_ff(qo, qe, c, &r1, a1, b1, u1)) return 0;
  ++n_settled;
  bool bad = r1 != in_range;
  if (!bad && in_range) {
    for (int k = 0; k < 3; ++k)
      bad = bad || a0[k] != a1[k] || b0[k] != b1[k] || std::memcmp(&u0[k], &u1[k], sizeof(float)) != 0;
  }
  if (bad) {
    std::fprintf(stderr, "mismatch: d = %lld %lld %lld tau = %.17g rmin = %.17g rmax = %.17g len = %.17g\n",
                 qe[0] - qo[0], qe[1] - qo[1], qe[2] - qo[2], tau, rmin, rmax, len);
    return 1;
  }
  return 0;
}

// The float-float primitives against double arithmetic (exact for these).
static int primitives() {
  for (int i = 0; i < 200000; ++i) {
    const float a = (float)((unit() - 0.5) * std::ldexp(1.0, (int)uniform(-20, 30)));
    const float b = (float)((unit() - 0.5) * std::ldexp(1.0, (int)uniform(-20, 30)));
    const ohm::FF s = ohm::two_sum(a, b), p = ohm::two_prod(a, b);
    if ((double)s.hi + (double)s.lo != (double)a + (double)b) return 2;
    if ((double)p.hi + (double)p.lo != (double)a * (double)b) return 2;
    // square roots and reciprocals to within 8 u^2
    const double x = std::ldexp(1.0 + unit(), (int)uniform(0, 48));
    const ohm::FF xf = ohm::ff_of_double(x);
    const ohm::FF r = ohm::ff_sqrt(xf), q = ohm::ff_rcp(xf);
    const double u2 = std::ldexp(1.0, -48);
    if (std::fabs(((double)r.hi + (double)r.lo) - std::sqrt(x)) > 8 * u2 * std::sqrt(x)) return 2;
    if (std::fabs(((double)q.hi + (double)q.lo) - 1.0 / x) > 8 * u2 / x) return 2;
  }
  // rint and float decisions at and next to their boundaries
  long long k = 0;
  float f = 0.f;
  if (ohm::ff_rint({2.5f, 0.0f}, 0.0f, &k) || ohm::ff_rint({2.0f, 0.5f}, 0.0f, &k)) return 2;
  if (!ohm::ff_rint({2.0f, 0.25f}, 1e-6f, &k) || k != 2) return 2;
  if (!ohm::ff_rint({3.0f, -0.25f}, 1e-6f, &k) || k != 3) return 2;
  if (!ohm::ff_rint({16777216.0f, 1.0f}, 1e-6f, &k) || k != 16777217) return 2;
  if (!ohm::ff_rint({-7.0f, -0.75f}, 1e-6f, &k) || k != -8) return 2;
  const float one = 1.0f, below = std::nextafter(1.0f, 0.0f);
  if (ohm::ff_to_float({one, (one - below) / 2}, 0.0f, &f)) return 2;           // the midpoint below 1
  if (!ohm::ff_to_float({one, (one - below) / 4}, 0.0f, &f) || f != one) return 2;
  if (ohm::ff_to_float({one, (one - below) / 4}, (one - below) / 2, &f)) return 2;
  return 0;
}

int main() {
  if (int rc = primitives()) return rc;
  long long qo[3], qe[3];
  // random rays in 2^-16 fixed point, voxel to range scale
  for (int i = 0; i < 600000; ++i) {
    const int bits = (int)uniform(3, 24);
    for (int k = 0; k < 3; ++k) {
      qo[k] = uniform(-(1LL << 30), 1LL << 30);
      qe[k] = qo[k] + uniform(-(1LL << bits) + 1, (1LL << bits) - 1);
    }
    if (i % 7 == 0) {
      const int k0 = (int)uniform(0, 2);
      qe[k0] = qo[k0];
    }
    const double tau = (double)uniform(0, 1LL << (int)uniform(8, 24)) + (i % 3 == 0 ? 0.25 : 0.0);
    const double rmin = (i % 5 == 0) ? 0.0 : (double)uniform(0, 1LL << 20) * 0.37;
    const double rmax = (double)uniform(1LL << 18, 1LL << 25) * 1.13;
    if (check(qo, qe, tau, rmin, rmax)) return 1;
  }
  const long long random_cases = n_cases, random_settled = n_settled;
  // tau chosen so that d_0 t0 / len lands on a half-integer, to rounding
  for (int i = 0; i < 200000; ++i) {
    for (int k = 0; k < 3; ++k) {
      qo[k] = uniform(-1000, 1000);
      qe[k] = qo[k] + uniform(-(1LL << 23), 1LL << 23);
    }
    if (qe[0] == qo[0]) qe[0] += 12345;
    double d[3];
    const double len = length_of(qo, qe, d);
    const double j = (double)uniform(0, (long long)std::fabs(d[0]) - 1) + 0.5;
    const double tau = len - j * len / std::fabs(d[0]);  // d_0 (len - tau) / len = +-j
    if (tau >= 0.0 && check(qo, qe, tau, 0.0, 1e12)) return 1;
    // and t1: d_0 (len + tau) / len = +-(j + |d_0|)
    if (check(qo, qe, (j + std::fabs(d[0])) * len / std::fabs(d[0]) - len, 0.0, 1e12)) return 1;
  }
  // lengths at the range limits and at tau: rmin, rmax, tau = len and its neighbours
  for (int i = 0; i < 100000; ++i) {
    for (int k = 0; k < 3; ++k) {
      qo[k] = uniform(-100000, 100000);
      qe[k] = qo[k] + uniform(-(1LL << 22), 1LL << 22);
    }
    double d[3];
    const double len = length_of(qo, qe, d);
    if (!(len > 0.0)) continue;
    const double around[3] = {std::nextafter(len, 0.0), len, std::nextafter(len, 1e300)};
    for (double v : around) {
      if (check(qo, qe, 262144.0, v, 1e12)) return 1;
      if (check(qo, qe, 262144.0, 0.0, v)) return 1;
      if (check(qo, qe, v, 0.0, 1e12)) return 1;
    }
  }
  // exact cases: axis-aligned rays with tau = len / 2 (half-integers for odd lengths)
  for (int e = 2; e < 24; ++e) {
    for (int i = 0; i < 200; ++i) {
      const long long dx = 2 * uniform(0, (1LL << (e - 1)) - 1) + 1;
      qo[0] = qo[1] = qo[2] = 0;
      qe[0] = dx;
      qe[1] = qe[2] = 0;
      if (check(qo, qe, (double)dx / 2, 0.0, 1e12)) return 1;
      qe[0] = 1LL << e;
      if (check(qo, qe, (double)(1LL << e) / 2, 0.0, 1e12)) return 1;
    }
  }
  std::printf("cases %lld settled %lld random %lld settled %lld\n", n_cases, n_settled, random_cases, random_settled);
  return 0;
}
