// CPU check of the exact arithmetic that starts a secondary ray
// (csrc/bounce_arith.cuh, the code bounce_kernel runs): the snapped origin
// parameter, the mirror direction and the per-ray side constant, against
// 128-bit integer division, on random and adversarial cases (rays nearly
// parallel to the hit edge, hits at the edge's ends, edges of one or two
// units, directions with tiny components, axis-aligned directions).
// Usage: bounce_arith_check <cases> <seed>; prints the counts; exit 1 on a mismatch.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <random>
#include <string>

#include "bounce_arith.cuh"

typedef __int128 i128;
using namespace cct::bounce;

static i128 floordiv128(i128 n, i128 d) {
  i128 q = n / d;
  if (n % d != 0 && n < 0) q -= 1;
  return q;
}

// "round <count> <seed>": prints n m round_div_sqrt(n, m) for random and
// adversarial pairs (perfect squares, halves, extreme magnitudes), one per line.
static int round_mode(long long count, unsigned long long seed) {
  std::mt19937_64 g(seed);
  auto rnd = [&](long long lo, long long hi) { return lo + (long long)(g() % (unsigned long long)(hi - lo + 1)); };
  for (long long k = 0; k < count; ++k) {
    long long m, n;
    switch (k % 4) {
      case 0:  // a frame computation's range: |n| < 2^43, m = |u|^2 < 2^41
        m = rnd(1, 1ll << 41);
        n = rnd(-(1ll << 43), 1ll << 43);
        break;
      case 1: {  // perfect squares with exact halves
        const long long r = rnd(1, 1 << 20);
        m = r * r;
        n = (2 * rnd(-(1ll << 21), 1ll << 21) + 1) * r / 2;
        if ((r & 1) == 0) n = (2 * rnd(-(1ll << 21), 1ll << 21) + 1) * (r / 2);
        break;
      }
      case 2:  // small values
        m = rnd(1, 50);
        n = rnd(-200, 200);
        break;
      default: {  // near a half: n ~ (q + 1/2) sqrt(m)
        m = rnd(2, 1ll << 41);
        const double q = (double)rnd(-(1 << 22), 1 << 22) + 0.5;
        n = llround(q * sqrt((double)m));
      }
    }
    printf("%lld %lld %lld\n", n, m, round_div_sqrt(n, m));
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc > 1 && std::string(argv[1]) == "round")
    return round_mode(argc > 2 ? atoll(argv[2]) : 100000, argc > 3 ? strtoull(argv[3], nullptr, 10) : 1);
  const long long cases = argc > 1 ? atoll(argv[1]) : 1000000;
  std::mt19937_64 g(argc > 2 ? strtoull(argv[2], nullptr, 10) : 1);
  const long long D = 1 << 20;
  auto rnd = [&](long long lo, long long hi) { return lo + (long long)(g() % (unsigned long long)(hi - lo + 1)); };
  long long n = 0, bad = 0, grazing = 0;
  for (long long trial = 0; trial < cases; ++trial) {
    const int mode = (int)(trial % 6);
    long long ax = rnd(0, D), ay = rnd(0, D), bx, by;
    if (mode == 1) {  // an edge of one to three units
      bx = std::min(D, ax + rnd(1, 3));
      by = std::min(D, ay + rnd(0, 2));
    } else {
      bx = rnd(0, D);
      by = rnd(0, D);
    }
    if (bx == ax && by == ay) continue;
    double th = (double)(g() % 1000000) / 1000000.0 * 6.283185307179586;
    if (mode == 3)  // nearly parallel to the edge
      th = atan2((double)(by - ay), (double)(bx - ax)) + ((g() & 1) ? 1 : -1) * ldexp(1.0, -(int)rnd(10, 40));
    long long kx = llround(cos(th) * 4194304.0), ky = llround(sin(th) * 4194304.0);
    if (mode == 4) {  // tiny components
      kx = rnd(-3, 3);
      ky = rnd(-3, 3);
    }
    if (mode == 5) {  // (nearly) axis-aligned
      kx = (g() & 1) ? 4194304 : -4194304;
      ky = rnd(-2, 2);
    }
    if (kx == 0 && ky == 0) continue;
    long long ex = bx - ax, ey = by - ay;
    if (kx * ey - ky * ex < 0) {  // orient the edge: a right of the ray, b left
      std::swap(ax, bx);
      std::swap(ay, by);
      ex = -ex;
      ey = -ey;
    }
    if (kx * ey - ky * ex == 0) continue;
    // the ray's origin: the hit point a + m (b - a) (m dyadic, at the ends in mode 2) moved back along k
    const long long m40 = mode == 2 ? ((g() & 1) ? rnd(0, 3) : (1ll << 40) - rnd(0, 3)) : rnd(0, 1ll << 40);
    const double tt = (double)rnd(1, 1 << 21) / ((g() & 1) ? 1.0 : 4096.0);
    const double Px = ax + ldexp((double)m40, -40) * ex - tt * kx / 4194304.0;
    const double Py = ay + ldexp((double)m40, -40) * ey - tt * ky / 4194304.0;
    if (Px < 0 || Py < 0 || Px > D || Py > D) continue;
    const long long X = llround(ldexp(Px, 32)), Y = llround(ldexp(Py, 32));
    const i128 Q = (i128)1 << 32;
    const i128 Sa = (i128)kx * ((i128)ay * Q - Y) - (i128)ky * ((i128)ax * Q - X);
    const i128 Sb = (i128)kx * ((i128)by * Q - Y) - (i128)ky * ((i128)bx * Q - X);
    if (!(Sa < 0 && Sb >= 0)) continue;  // not the exit edge of this ray
    ++n;
    // snapped parameter
    const long long i = snap_param((int)kx, (int)ky, X - (ax << 32), Y - (ay << 32), ex, ey);
    const i128 N = (i128)kx * ((i128)Y - (i128)ay * Q) - (i128)ky * ((i128)X - (i128)ax * Q);
    const i128 Dd = (i128)kx * ey - (i128)ky * ex;
    i128 ie = floordiv128(2 * N + Dd, 2 * Dd);
    ie = ie < 1 ? 1 : (ie > Q - 1 ? Q - 1 : ie);
    if ((i128)i != ie) {
      if (bad < 10) printf("snap mismatch (mode %d)\n", mode);
      ++bad;
    }
    // mirror direction
    int k2x, k2y;
    const bool back = mirror_dir((int)kx, (int)ky, ex, ey, k2x, k2y);
    const i128 ku = (i128)kx * ex + (i128)ky * ey, uu = (i128)ex * ex + (i128)ey * ey;
    i128 rx = floordiv128(2 * (2 * ku * ex - uu * kx) + uu, 2 * uu);
    i128 ry = floordiv128(2 * (2 * ku * ey - uu * ky) + uu, 2 * uu);
    const i128 L = (i128)1 << 22;
    rx = rx > L ? L : (rx < -L ? -L : rx);
    ry = ry > L ? L : (ry < -L ? -L : ry);
    const i128 c0 = (i128)ex * ky - (i128)ey * kx, c1 = (i128)ex * ry - (i128)ey * rx;
    const bool back_e = (c0 > 0 && c1 < 0) || (c0 < 0 && c1 > 0);
    if ((i128)k2x != rx || (i128)k2y != ry || back != back_e) {
      if (bad < 10) printf("mirror mismatch (mode %d)\n", mode);
      ++bad;
    }
    grazing += !back_e;
    // side constant
    const i128 C = (i128)kx * Y - (i128)ky * X;
    if ((i128)ceil_cross_q((int)kx, (int)ky, X, Y) != -floordiv128(-C, Q)) {
      if (bad < 10) printf("side constant mismatch (mode %d)\n", mode);
      ++bad;
    }
  }
  printf("cases %lld mismatches %lld grazing %lld\n", n, bad, grazing);
  return bad != 0;
}
