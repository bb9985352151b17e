// FP32 real part of the Faddeeva function, Re w(x + iy) = sqrt(pi) * K(x, y), for the
// Voigt profile V(dnu) = Re w((dnu + i gamma_L)/gamma_G) / (gamma_G sqrt(pi))
// (pyROX paper, "Compute line profiles": Voigt profile as the real part of the
// Faddeeva function, Gandhi et al. 2020 Eq. 12; the paper evaluates it with
// scipy.special.wofz in double precision).
//
// Region split on s = x^2 + y^2 (x >= 0; Re w is even in x), each method written
// from its published definition and checked against wofz (max relative error of
// Re w about 1.1e-5 over x in [0, 1e5], y in [0, 1e4]):
//   s >= 22^2          2-level Laplace continued fraction (Humlicek 1982, region I form)
//   10^2 <= s < 22^2   3-level continued fraction, in closed real form
//   6^2  <= s < 10^2   5-level continued fraction (+ Gaussian term for y < 1e-6)
//   s < 6^2, y >= 0.1  Weideman (1994) rational approximation, N = 20
//   s < 6^2, y <  0.1  Re w = e^{y^2-x^2} cos(2xy) - (2/sqrt(pi)) Im F(x + iy), with
//                      Dawson's F from its complex Taylor series around the nearest
//                      node x_c (step 1/8, nodes to 7.25). This form keeps relative accuracy
//                      in the Gaussian tail near the real axis, where Re w is tiny next to
//                      Im w.
// The two core forms (rox_re_w_core) hold 1.1e-5 out to |z| = 7.1 for y < 0.5 and 2e-6 for
// 0.5 <= y <= 1.01; the Voigt kernel uses them directly in the |z| < 6.5 zones of lines with the
// Pade far form (boundary 6.5^2 for y < 1.006).
// The continued fraction truncations miss the exponentially small e^{-z^2} part of w,
// which can matter just outside |z| = 6 when y is essentially zero; it is added there.
//
// The Voigt kernel's far zone (rox_re_w_far) uses one rational form in u = x^2 per line,
// whose coefficients depend on y only: for y < 11.5 a [1/2] Pade approximant in 1/u of the
// large-|x| expansion of Re w at fixed y, valid for s >= 6.5^2 (y < 0.75),
// 6.5^2 + 3.5 / |4 y^2 - 3| (0.75 <= y < 0.95, around its coefficients' pole at y = 0.866) or
// max(6.5^2, 42 y) (0.95 <= y < 11.5); where that boundary would pass 22^2 (within 0.0012 of
// the pole, and y >= 11.5) the 2-level fraction, valid for s >= 22^2.
#pragma once
#include <math.h>

#ifdef __CUDACC__
#define ROX_FN __device__ __forceinline__
#define ROX_TABLE static __constant__ const
#else
#define ROX_FN static inline
#define ROX_TABLE static const
#endif

#include "rox_faddeeva_tables.h"

#define ROX_INV_SQRT_PI 0.564189583547756287f
#define ROX_TWO_INV_SQRT_PI 1.128379167095512574f

// region boundaries on s = x^2 + y^2
#define ROX_S_FAR 484.0f     // 22^2
#define ROX_S_CF3 100.0f     // 10^2
#define ROX_S_CF5 36.0f      // 6^2
#define ROX_Y_WEIDEMAN 0.1f
#define ROX_S_PADE 42.25f    // 6.5^2: the smallest far-zone boundary of the per-line Pade form
#define ROX_Y_PADE 0.75f     // the Pade form: boundary s = 6.5^2 for y below this,
#define ROX_Y_POLE_HI 0.95f  // 6.5^2 + 3.5 / |4 y^2 - 3| up to here (its coefficients' pole is at y = 0.866),
#define ROX_Y_PADE_MAX 11.5f // max(6.5^2, 42 y) up to here
#define ROX_PADE_R2_PER_Y 42.0f
#define ROX_PADE_R2_POLE 3.5f

ROX_FN float rox_rcp(float v) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
#else
  return 1.0f / v;
#endif
}

ROX_FN float rox_rsqrt(float v) {
#ifdef __CUDA_ARCH__
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
#else
  return 1.0f / sqrtf(v);
#endif
}

ROX_FN float rox_exp2(float v) {
#ifdef __CUDA_ARCH__
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
#else
  return exp2f(v);
#endif
}

// e^{y^2 - x^2} cos(2xy): the part of w(z) = e^{-z^2} + (2i/sqrt(pi)) F(z) that the
// asymptotic (continued fraction) forms do not contain. Used only where y < 0.1 and
// |x| < 7.1, or y < 1e-6 and |x| < 10, so |2xy| < 1.42: cos by its Taylor polynomial to
// u^10 (truncation below 2e-7, on a term that is below e^-36 of the peak wherever |u| > 1.2),
// the exponential as 2^(log2(e) (y^2 - x^2)) (relative error about 3e-6 at |x| = 7 from the
// rounded argument; results below 2^-126 flush to 0).
ROX_FN float rox_gauss_part(float x, float y) {
  const float u = 2.0f * x * y;
  const float u2 = u * u;
  float c = fmaf(u2, -2.755731922398589e-07f, 2.48015873015873e-05f);
  c = fmaf(u2, c, -1.388888888888889e-03f);
  c = fmaf(u2, c, 4.166666666666667e-02f);
  c = fmaf(u2, c, -0.5f);
  c = fmaf(u2, c, 1.0f);
  return rox_exp2(1.4426950408889634f * ((y - x) * (y + x))) * c;
}

// 2-level continued fraction: w ~ (i/sqrt(pi)) z / (z^2 - 1/2).
// Re = y (s + 1/2) / (sqrt(pi) ((s - 1/2)^2 + 2 y^2)).
ROX_FN float rox_re_w_cf2(float x, float y) {
  float v = y * y;
  float s = fmaf(x, x, v);
  float t = s - 0.5f;
  float d = fmaf(t, t, 2.0f * v);
  return ROX_INV_SQRT_PI * y * (s + 0.5f) * rox_rcp(d);
}

// Far-zone form with per-line coefficients, in t = u + alpha (u = x^2):
//   Re w ~ (y / sqrt(pi)) (t + kappa) / (t^2 + beta),   valid for s = u + y^2 >= r2.
// For the Pade ranges of y the coefficients make (u + b)/(u^2 + c u + d) (alpha = c/2, kappa = b - c/2,
// beta = d - c^2/4) agree with the first four terms of the expansion of Re w(x + iy)
// sqrt(pi)/y in powers of 1/u at fixed v = y^2, obtained from the asymptotic series
// w ~ (i/sqrt(pi)) sum_n (2n-1)!!/2^n z^-(2n+1):
//   1/u + (3/2 - v)/u^2 + (v^2 - 5v + 15/4)/u^3 + (-v^3 + 21v^2/2 - 105v/4 + 105/8)/u^4.
// Max relative error against wofz 3.4e-6 beyond those boundaries, for y >= 1e-9 (each boundary
// rule covers the smallest radius that holds that bound, found by a scan of y against wofz: it
// grows near the pole, where the coefficients diverge, and with y, because the expansion's
// coefficients grow like powers of v). The form lacks the Gaussian part e^{-x^2} (below 4.5e-19 of the line peak
// there), which is why the relative bound needs y >= 1e-9; for smaller y the absolute error stays
// below 4.5e-19 of the peak. Real roots of the denominator (y <= 1.5 only, at
// t = sqrt(-beta)) lie below t at the zone boundary for every y (the same scan): the form is
// never used there.
// Next to the pole (v = 3/4: |4v - 3| < 0.0079) and beyond y = 11.5 the boundary would pass 22:
// there the 2-level continued fraction, alpha = v - 1/2, beta = 2v, kappa = 1, s >= 22^2.
struct rox_far {
  float alpha, beta, kappa, r2;
};
ROX_FN rox_far rox_far_coefs(float y) {
  rox_far f;
  const float v = y * y;
  const float g = fmaf(4.0f, v, -3.0f);            // the coefficients' pole: g = 0
  float r2 = ROX_S_FAR;
  if (y < ROX_Y_PADE) r2 = ROX_S_PADE;
  else if (y < ROX_Y_POLE_HI) r2 = ROX_S_PADE + ROX_PADE_R2_POLE * rox_rcp(fabsf(g));   // inf at the pole
  else if (y < ROX_Y_PADE_MAX) r2 = fmaxf(ROX_S_PADE, ROX_PADE_R2_PER_Y * y);
  if (r2 < ROX_S_FAR) {   // |g| >= 0.0079 here
    const float q = rox_rcp(g);
    f.alpha = 0.5f * fmaf(v, fmaf(8.0f, v, -30.0f), 15.0f) * q;
    f.beta = 0.5f * fmaf(v, fmaf(v, fmaf(64.0f, v, -216.0f), 180.0f), -45.0f) * q * q;
    f.kappa = 3.0f * fmaf(-2.0f, v, 1.0f) * q;
    f.r2 = r2;
  } else {
    f.alpha = v - 0.5f;
    f.beta = 2.0f * v;
    f.kappa = 1.0f;
    f.r2 = ROX_S_FAR;
  }
  return f;
}

// Re w by the far-zone form (only for s >= rox_far_coefs(y).r2)
ROX_FN float rox_re_w_far(float x, float y) {
  const rox_far f = rox_far_coefs(y);
  const float t = fmaf(x, x, f.alpha);
  return ROX_INV_SQRT_PI * y * (t + f.kappa) * rox_rcp(fmaf(t, t, f.beta));
}

// complex multiply-add helpers on (re, im) pairs
struct rox_c { float r, i; };
ROX_FN rox_c rox_cmul(rox_c a, rox_c b) {
  rox_c o;
  o.r = fmaf(a.r, b.r, -a.i * b.i);
  o.i = fmaf(a.r, b.i, a.i * b.r);
  return o;
}

// One complex Horner step with a real coefficient, acc * m + c, in four FP32 operations (the
// coefficient enters the real part's FMA chain instead of a separate add).
ROX_FN rox_c rox_horner_step(rox_c acc, rox_c m, float c) {
  rox_c o;
  o.r = fmaf(acc.r, m.r, fmaf(-acc.i, m.i, c));
  o.i = fmaf(acc.r, m.i, acc.i * m.r);
  return o;
}

// Horner in zeta = z^2 with real coefficients c[0..n-1] (highest first)
template <int N>
ROX_FN rox_c rox_horner_zeta(const float* c, rox_c zeta) {
  rox_c acc;
  acc.r = c[0];
  acc.i = 0.0f;
#pragma unroll
  for (int k = 1; k < N; k++) acc = rox_horner_step(acc, zeta, c[k]);
  return acc;
}

// n-level continued fraction truncation w ~ (i/sqrt(pi)) A(z)/B(z), with
// A = z^{a_odd} a(z^2), B = z^{1-a_odd} b(z^2). Re w = -Im(A conj(B)) / (sqrt(pi) |B|^2).
template <int NA, int NB, int AODD>
ROX_FN float rox_re_w_cf(const float* ca, const float* cb, float x, float y) {
  rox_c zeta;
  zeta.r = (x - y) * (x + y);
  zeta.i = 2.0f * x * y;
  rox_c a = rox_horner_zeta<NA>(ca, zeta);
  rox_c b = rox_horner_zeta<NB>(cb, zeta);
  rox_c z;
  z.r = x;
  z.i = y;
  if (AODD) a = rox_cmul(a, z); else b = rox_cmul(b, z);
  float num = fmaf(a.r, b.i, -a.i * b.r);          // -Im(A conj B) = A_r B_i - A_i B_r
  float den = fmaf(b.r, b.r, b.i * b.i);
  return ROX_INV_SQRT_PI * num * rox_rcp(den);
}

// 3-level: w ~ (i/sqrt(pi)) (z^2 - 1) / (z^3 - 3z/2). With u = x^2, v = y^2, s = u + v:
// Re w = y (s^2 - 3s/2 + 4v + 3/2) / (sqrt(pi) [u (u - 3v - 3/2)^2 + v (3u - v - 3/2)^2]).
ROX_FN float rox_re_w_cf3(float x, float y) {
  const float u = x * x, v = y * y;
  const float s = u + v;
  const float num = fmaf(s, s - 1.5f, fmaf(4.0f, v, 1.5f));
  const float a = u - fmaf(3.0f, v, 1.5f);
  const float b = fmaf(3.0f, u, -(v + 1.5f));
  const float den = fmaf(u * a, a, (v * b) * b);
  return ROX_INV_SQRT_PI * y * num * rox_rcp(den);
}

ROX_FN float rox_re_w_cf5(float x, float y) {
  return rox_re_w_cf<3, 3, ROX_CF5_A_ODD>(rox_cf5_a, rox_cf5_b, x, y);
}

// Weideman (1994): w(z) ~ [2 p(Z) + (L - iz)/sqrt(pi)] / (L - iz)^2, Z = (L + iz)/(L - iz).
ROX_FN float rox_re_w_weideman(float x, float y) {
  const float L = ROX_WEI_L;
  float lpy = L + y;
  float q2 = rox_rcp(fmaf(lpy, lpy, x * x));        // 1/|L - iz|^2
  rox_c q;                                           // 1/(L - iz) = (L + y + ix)/|L - iz|^2
  q.r = lpy * q2;
  q.i = x * q2;
  rox_c Z;                                           // ((L^2 - s) + 2iLx)/|L - iz|^2
  Z.r = (fmaf(L, L, -fmaf(x, x, y * y))) * q2;
  Z.i = 2.0f * L * x * q2;
  rox_c p;
  p.r = rox_wei_a[0];
  p.i = 0.0f;
#pragma unroll
  for (int k = 1; k < ROX_WEI_N; k++) p = rox_horner_step(p, Z, rox_wei_a[k]);
  rox_c t = rox_cmul(p, q);                          // p/(L - iz)
  t.r = fmaf(2.0f, t.r, ROX_INV_SQRT_PI);
  t.i = 2.0f * t.i;
  return fmaf(t.r, q.r, -t.i * q.i);                 // Re[(2p/(L-iz) + 1/sqrt(pi)) / (L-iz)]
}

// Near the real axis: Re w = e^{y^2-x^2} cos 2xy - (2/sqrt(pi)) Im F(x+iy), F Dawson's
// integral from its Taylor series at the nearest node, evaluated at the complex offset
// (x - x_c) + iy by complex Horner (imaginary parts stay O(y), so the O(y) result keeps
// its relative accuracy). `tab` is rox_daw_taylor, possibly copied to shared memory.
ROX_FN float rox_re_w_dawson(const float* tab, float x, float y) {
  int node = (int)rintf(x * ROX_DAW_INV_STEP);
  node = node > ROX_DAW_NODES - 1 ? ROX_DAW_NODES - 1 : (node < 0 ? 0 : node);
  const float* d = tab + node * ROX_DAW_STRIDE;
  float t = fmaf(-(float)node, ROX_DAW_STEP, x);
  float ar = d[ROX_DAW_DEG], ai = 0.0f;
#pragma unroll
  for (int n = ROX_DAW_DEG - 1; n >= 0; n--) {
    float nr = fmaf(ar, t, fmaf(-ai, y, d[n]));
    float ni = fmaf(ar, y, ai * t);
    ar = nr;
    ai = ni;
  }
  return fmaf(-ROX_TWO_INV_SQRT_PI, ai, rox_gauss_part(x, y));
}

// 5-level fraction with the Gaussian part kept for (essentially) zero y
ROX_FN float rox_re_w_cf5g(float x, float y) {
  float r = rox_re_w_cf5(x, y);
  return y < 1e-6f ? r + rox_gauss_part(x, y) : r;
}

// |z| < 6: Weideman away from the real axis, the Dawson form near it (y is per line)
ROX_FN float rox_re_w_core(const float* daw, float x, float y) {
  return y >= ROX_Y_WEIDEMAN ? rox_re_w_weideman(x, y) : rox_re_w_dawson(daw, x, y);
}

// Re w(x + iy) for x any sign, y >= 0, all regions. `daw` points at rox_daw_taylor.
ROX_FN float rox_re_w(const float* daw, float x, float y) {
  x = fabsf(x);
  float s = fmaf(x, x, y * y);
  if (s >= ROX_S_FAR) return rox_re_w_cf2(x, y);
  if (s >= ROX_S_CF3) return rox_re_w_cf3(x, y);
  if (s >= ROX_S_CF5) return rox_re_w_cf5g(x, y);
  return rox_re_w_core(daw, x, y);
}
