// Exact integer arithmetic of a secondary ray's start (the snapped origin
// parameter, the mirror direction or the caller's direction in the hit edge's
// frame), shared by bounce_kernel and its CPU check.  Host builds use the IEEE operations the device intrinsics compute
// (round to nearest; floor for the float -> int64 conversion).
#pragma once

#include <math.h>
#include <stdint.h>

namespace cct {
namespace bounce {

#ifdef __CUDA_ARCH__
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float ll2f(long long v) { return __ll2float_rn(v); }
__device__ __forceinline__ long long f2ll_rd(float x) { return __float2ll_rd(x); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float sqrt_rn(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
#define CCT_BX __device__ __forceinline__
#else
inline float rcp_rn(float x) {
  volatile float r = 1.0f / x;
  return r;
}
inline float ll2f(long long v) { return (float)v; }
inline long long f2ll_rd(float x) { return (long long)floorf(x); }
inline float mul_rn(float a, float b) {
  volatile float r = a * b;
  return r;
}
inline float fma_rn(float a, float b, float c) { return fmaf(a, b, c); }
inline float sqrt_rn(float x) { return sqrtf(x); }
inline float div_rn(float a, float b) {
  volatile float r = a / b;
  return r;
}
#define CCT_BX inline
#endif

constexpr long long kQ = 1ll << 32;  // origins are held in units of 2^-32
constexpr long long kKLim = 1ll << 22;

// floor(m / d) for d > 0 when the quotient is known to lie in [lo, hi]
// (|lo|, |hi| < 2^40), m is given modulo 2^64 (mm) and approximately (mf, an
// fp32 value whose error divided by d is below 2^40).  The first estimate is
// clamped to [lo, hi], so its remainder m - q d is below 2^63 in magnitude and
// equals its value modulo 2^64; each further estimate of the remaining
// quotient is within 2^-21 relative plus 1, so after two of them the quotient
// is within 2 and exact int64 steps finish.
CCT_BX long long floordiv_mod(unsigned long long mm, float mf, long long d, long long lo, long long hi) {
  const float rd = rcp_rn(ll2f(d));
  long long q = f2ll_rd(mul_rn(mf, rd));
  q = q < lo ? lo : (q > hi ? hi : q);
  long long r = (long long)(mm - (unsigned long long)q * (unsigned long long)d);
  for (int k = 0; k < 2; ++k) {
    q += f2ll_rd(mul_rn(ll2f(r), rd));
    r = (long long)(mm - (unsigned long long)q * (unsigned long long)d);
  }
  while (r < 0) {
    --q;
    r += d;
  }
  while (r >= d) {
    ++q;
    r -= d;
  }
  return q;
}

// ceil((kx Y - ky X) / 2^32) from the 32-bit halves of X and Y (no 128-bit
// product): with X = Xh 2^32 + Xl, the value is (kx Yh - ky Xh) + ceil(B / 2^32),
// B = kx Yl - ky Xl (|B| < 2^55).  X, Y in [0, 2^52].
CCT_BX long long ceil_cross_q(int kx, int ky, long long X, long long Y) {
  const long long Xh = X >> 32, Yh = Y >> 32;
  const long long Xl = X & 0xffffffffll, Yl = Y & 0xffffffffll;
  const long long B = (long long)kx * Yl - (long long)ky * Xl;
  return ((long long)kx * Yh - (long long)ky * Xh) - ((-B) >> 32);
}

// The snapped parameter of the next origin on the hit edge (a -> b), a right
// of the ray (P, k) and b left of it or on its line: i = round(2^32 mu)
// (halves up) clamped to [1, 2^32 - 1], mu = (k x (P - a)) / (k x (b - a)).
// (Rx, Ry) = P - a in units of 2^-32 (|.| <= 2^52), (ex, ey) = b - a.
// 2^32 mu = N / Dd with N = kx Ry - ky Rx (|N| < 2^75) and Dd = k x e > 0.
CCT_BX long long snap_param(int kx, int ky, long long Rx, long long Ry, long long ex, long long ey) {
  const long long Dd = (long long)kx * ey - (long long)ky * ex;
  const unsigned long long Nm = (unsigned long long)(long long)kx * (unsigned long long)Ry -
                                (unsigned long long)(long long)ky * (unsigned long long)Rx;
  const float Nf = fma_rn((float)kx, ll2f(Ry), -mul_rn((float)ky, ll2f(Rx)));
  long long i = floordiv_mod(2ull * Nm + (unsigned long long)Dd, fma_rn(2.0f, Nf, ll2f(Dd)), 2 * Dd, 0, kQ);
  return i < 1 ? 1 : (i > kQ - 1 ? kQ - 1 : i);
}

// The mirror direction of k about u = (ex, ey): k' = 2 (k.u) u / |u|^2 - k
// rounded componentwise (halves up: floor((2 n + uu) / (2 uu)),
// n = 2 (k.u) u - uu k, |k'| <= 2^22.5), clamped to [-2^22, 2^22].  Returns
// whether k' points strictly back to the side k came from (u x k' and u x k
// of opposite signs).
CCT_BX bool mirror_dir(int kx, int ky, long long ex, long long ey, int& k2x_out, int& k2y_out) {
  const long long ku = (long long)kx * ex + (long long)ky * ey, uu = ex * ex + ey * ey;
  const float kuf = ll2f(ku), uuf = ll2f(uu);
  const unsigned long long ku2 = 2ull * (unsigned long long)ku, uum = (unsigned long long)uu;
  const unsigned long long mxm = 2ull * (ku2 * (unsigned long long)ex - uum * (unsigned long long)(long long)kx) + uum;
  const unsigned long long mym = 2ull * (ku2 * (unsigned long long)ey - uum * (unsigned long long)(long long)ky) + uum;
  const float mxf = fma_rn(2.0f, fma_rn(2.0f * kuf, (float)ex, -mul_rn(uuf, (float)kx)), uuf);
  const float myf = fma_rn(2.0f, fma_rn(2.0f * kuf, (float)ey, -mul_rn(uuf, (float)ky)), uuf);
  long long k2x = floordiv_mod(mxm, mxf, 2 * uu, -2 * kKLim, 2 * kKLim);
  long long k2y = floordiv_mod(mym, myf, 2 * uu, -2 * kKLim, 2 * kKLim);
  k2x = k2x > kKLim ? kKLim : (k2x < -kKLim ? -kKLim : k2x);
  k2y = k2y > kKLim ? kKLim : (k2y < -kKLim ? -kKLim : k2y);
  k2x_out = (int)k2x;
  k2y_out = (int)k2y;
  const long long c0 = ex * ky - ey * kx, c1 = ex * k2y - ey * k2x;
  return (c0 > 0 && c1 < 0) || (c0 < 0 && c1 > 0);
}

// Whether a < b sqrt(m), exactly (m >= 0, |a| < 2^62, |b| sqrt(m) < 2^62).
CCT_BX bool lt_sqrt(long long a, long long b, long long m) {
  const __int128 a2 = (__int128)a * a, b2m = (__int128)b * b * m;
  if (b >= 0) return a < 0 || a2 < b2m;
  return a < 0 && a2 > b2m;
}

// round(n / sqrt(m)) with halves up (m >= 1, |n / sqrt(m)| < 2^40): the q with
// (2q - 1) sqrt(m) <= 2n < (2q + 1) sqrt(m), from an fp32 estimate and exact steps.
CCT_BX long long round_div_sqrt(long long n, long long m) {
  long long q = f2ll_rd(div_rn(ll2f(n), sqrt_rn(ll2f(m))) + 0.5f);
  while (!lt_sqrt(2 * n, 2 * q + 1, m)) ++q;
  while (lt_sqrt(2 * n, 2 * q - 1, m)) --q;
  return q;
}

// The caller's direction (kc, ks) = 2^22 (c, s) in the frame of the hit edge
// u = (ex, ey) (a right of the parent ray k, b left): k' = round(2^22 (c u + s n) / |u|),
// n = (-u_y, u_x) (the normal on the parent's side), clamped to [-2^22, 2^22].
// Returns whether k' points strictly back to the parent's side (as mirror_dir).
CCT_BX bool frame_dir(int kc, int ks, int kx, int ky, long long ex, long long ey, int& k2x_out, int& k2y_out) {
  const long long m = ex * ex + ey * ey;
  long long k2x = round_div_sqrt((long long)kc * ex - (long long)ks * ey, m);
  long long k2y = round_div_sqrt((long long)kc * ey + (long long)ks * ex, m);
  k2x = k2x > kKLim ? kKLim : (k2x < -kKLim ? -kKLim : k2x);
  k2y = k2y > kKLim ? kKLim : (k2y < -kKLim ? -kKLim : k2y);
  k2x_out = (int)k2x;
  k2y_out = (int)k2y;
  const long long c0 = ex * ky - ey * kx, c1 = ex * k2y - ey * k2x;
  return (c0 > 0 && c1 < 0) || (c0 < 0 && c1 > 0);
}

#undef CCT_BX

}  // namespace bounce
}  // namespace cct
