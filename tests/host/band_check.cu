// Host-side check of tsdf_band (ohm_device.cuh, compiled for the CPU): the
// band end points and unit direction it forms through one reciprocal must
// equal those of the direct double evaluation on every case, including cases
// built to land on half-integers and float rounding midpoints, where it must
// fall back to the divisions.  No GPU is needed.
//
// stdout: "cases <n> fallback <k>"; exit code 1 on a mismatch (the case is
// printed to stderr), 2 when a predicate check fails.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "../../paper_2206_06079_gb300/csrc/ohm_device.cuh"

static uint64_t state = 0x9e3779b97f4a7c15ULL;
static uint64_t next_u64() {  // splitmix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
static long long uniform(long long lo, long long hi) { return lo + (long long)(next_u64() % (uint64_t)(hi - lo + 1)); }

static double length_of(const double d[3]) {
  double l2 = d[0] * d[0];
  l2 = l2 + d[1] * d[1];
  l2 = l2 + d[2] * d[2];
  return std::sqrt(l2);
}

// The direct evaluation the kernels used before (every quotient a division).
static void direct(const long long qo[3], const double d[3], double len, double tau, long long a[3], long long b[3],
                   float u[3]) {
  double t0 = len - tau;
  if (t0 < 0.0) t0 = 0.0;
  const double t1 = len + tau;
  const double f0 = t0 / len, f1 = t1 / len;
  for (int k = 0; k < 3; ++k) {
    a[k] = qo[k] + std::llrint(d[k] * f0);
    b[k] = qo[k] + std::llrint(d[k] * f1);
    u[k] = (float)(d[k] / len);
  }
}

static long long n_cases = 0, n_fallback = 0;

static int check(const long long qo[3], const long long di[3], double tau) {
  const double d[3] = {(double)di[0], (double)di[1], (double)di[2]};
  const double len = length_of(d);
  if (!(len > 0.0)) return 0;
  long long a0[3], b0[3], a1[3], b1[3];
  float u0[3], u1[3];
  direct(qo, d, len, tau, a0, b0, u0);
  ohm::tsdf_band(qo, d, len, tau, a1, b1, u1);
  ++n_cases;
  // did the fast path need the fallback?
  {
    double t0 = len - tau;
    if (t0 < 0.0) t0 = 0.0;
    const double rho = 1.0 / len, f0 = t0 * rho, f1 = (len + tau) * rho;
    bool fb = false;
    for (int k = 0; k < 3; ++k)
      fb = fb || ohm::near_half_integer(d[k] * f0) || ohm::near_half_integer(d[k] * f1) ||
           ohm::near_float_midpoint(d[k] * rho);
    if (fb) ++n_fallback;
  }
  for (int k = 0; k < 3; ++k) {
    if (a0[k] != a1[k] || b0[k] != b1[k] || std::memcmp(&u0[k], &u1[k], sizeof(float)) != 0) {
      std::fprintf(stderr, "mismatch: d = %lld %lld %lld tau = %.17g axis %d\n", di[0], di[1], di[2], tau, k);
      return 1;
    }
  }
  return 0;
}

static int predicates() {
  // near_half_integer on values a few ulp from k + 1/2, and far from it
  const double halves[] = {0.5, 1.5, 2.5, 1000.5, 12345678.5, 1073741823.5};
  for (double h : halves) {
    if (!ohm::near_half_integer(h) || !ohm::near_half_integer(-h)) return 2;
    double x = h;
    for (int i = 0; i < 8; ++i) x = std::nextafter(x, 1e300);
    if (!ohm::near_half_integer(x)) return 2;
    x = h;
    for (int i = 0; i < 8; ++i) x = std::nextafter(x, -1e300);
    if (!ohm::near_half_integer(x)) return 2;
    x = h;
    for (int i = 0; i < 40; ++i) x = std::nextafter(x, 1e300);
    if (ohm::near_half_integer(x)) return 2;
  }
  if (ohm::near_half_integer(0.0) || ohm::near_half_integer(1.0) || ohm::near_half_integer(0.25) ||
      ohm::near_half_integer(7.0))
    return 2;
  // near_float_midpoint: the midpoint of two adjacent floats, a few ulp off
  const float fs[] = {0.6f, 0.125f, 0.9999999f, 0.3f, 1e-6f};
  for (float f : fs) {
    const double lo = (double)f, hi = (double)std::nextafter(f, 2.0f), mid = 0.5 * (lo + hi);
    if (!ohm::near_float_midpoint(mid)) return 2;
    double x = mid;
    for (int i = 0; i < 8; ++i) x = std::nextafter(x, 2.0);
    if (!ohm::near_float_midpoint(x)) return 2;
    x = mid;
    for (int i = 0; i < 40; ++i) x = std::nextafter(x, 2.0);
    if (ohm::near_float_midpoint(x)) return 2;
    if (ohm::near_float_midpoint(lo)) return 2;
  }
  return 0;
}

int main() {
  if (int rc = predicates()) return rc;
  long long qo[3], d[3];
  // random rays: voxel-scale to range-scale lengths in 2^-16 fixed point
  for (int i = 0; i < 400000; ++i) {
    const int bits = (int)uniform(4, 29);
    for (int k = 0; k < 3; ++k) {
      qo[k] = uniform(-(1LL << 24), 1LL << 24);
      d[k] = uniform(-(1LL << bits), 1LL << bits);
    }
    if (i % 7 == 0) d[(int)uniform(0, 2)] = 0;
    const double tau = (double)uniform(0, 1LL << (int)uniform(8, 24)) + (i % 3 == 0 ? 0.25 : 0.0);
    if (check(qo, d, tau)) return 1;
  }
  // tau chosen so that d_0 t0 / len lands on a half-integer, to rounding
  for (int i = 0; i < 200000; ++i) {
    for (int k = 0; k < 3; ++k) {
      qo[k] = uniform(-1000, 1000);
      d[k] = uniform(-(1LL << 26), 1LL << 26);
    }
    if (d[0] == 0) d[0] = 12345;
    const double dd[3] = {(double)d[0], (double)d[1], (double)d[2]};
    const double len = length_of(dd);
    const double j = (double)uniform(0, (long long)std::fabs(dd[0]) - 1) + 0.5;
    const double tau = len - j * len / std::fabs(dd[0]);  // d_0 (len - tau) / len = +-j
    if (tau >= 0.0 && check(qo, d, tau)) return 1;
  }
  // tau = len / 2 exactly (len a power of two): d_k / 2 exact, half-integers for odd d_k
  for (int e = 2; e < 28; ++e) {
    const long long L = 1LL << e;
    for (int i = 0; i < 200; ++i) {
      const long long dx = 2 * uniform(0, L / 2 - 1) + 1;  // odd
      const long long D[3] = {L, 0, 0};
      const long long Dodd[3] = {dx, 0, 0};
      qo[0] = qo[1] = qo[2] = 0;
      if (check(qo, D, (double)L / 2)) return 1;
      if (check(qo, Dodd, (double)dx / 2)) return 1;
    }
  }
  std::printf("cases %lld fallback %lld\n", n_cases, n_fallback);
  return 0;
}
