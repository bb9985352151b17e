// a4 / a5: Voigt evaluation and accumulation onto the wavenumber grid, for every (P,T).
// pyROX paper, "Compute line profiles" (Voigt = Re of the Faddeeva function, Gandhi et al.
// 2020 Eq. 12) and "Combine and save" (profiles summed into a cross-section per
// temperature-pressure point).
//
// Persistent kernel; the unit of work is one warp and one span of ROX_SPAN consecutive grid
// points at one (P,T) point, taken from an atomic counter by the warp itself, so warps never
// wait for one another. Each lane owns ROX_K points of the span, strided by 32, in registers.
// The lines that reach the span form a contiguous range of the nu0-sorted list (precomputed
// per span); they pass through the warp in batches of 32: each lane stages one line's
// geometry and strength with cp.async one batch ahead, turns it into per-line constants in
// the warp's shared-memory slots, and then all lanes walk the batch's lines in order. The
// span is written once at the end, so the summation order is fixed.
//
// Work per (line, point) pair, in physical units X = nu_j - nu0, Y = gamma_L: outside a
// per-line slow zone the far-zone form of rox_faddeeva.cuh (rox_re_w_far: per-line
// coefficients alpha, beta, kappa of y = gamma_L/gamma_G), scaled by gamma_G, gives
// S V = (S Y / pi)(t + K) / (t^2 + B) with t = X^2 + A, A = alpha gamma_G^2,
// B = beta gamma_G^4, K = kappa gamma_G^2, i.e. 4 FMAs and one reciprocal; two lines share
// one reciprocal (n1/d1 + n2/d2 = (n1 d2 + n2 d1)/(d1 d2)), so a pair costs 12 FP32
// operations and one MUFU per point, three of them as paired (f32x2) instructions. The slow
// zone is x^2 + y^2 < r^2(y) for the lines with the per-line Pade form (y < 11.5 except next to
// its coefficients' pole at y = 0.866; r^2 from 6.5^2 to below 22^2, rox_far_coefs) and < 22^2
// for the others (2-level continued fraction), at least the precision margin.
// Lines are evaluated in two passes per batch. Pass 1 applies the far formula to every line at
// every point of its window, in pairs; a line whose slow zone meets the span has t clamped to
// the zone boundary, t = max(t, t_z), so inside the zone it adds the far form's (finite) value
// at the boundary. Pass 2 visits exactly those points (t < t_z, decided on the same rounded t)
// and adds the full FP32 Faddeeva forms (rox_faddeeva.cuh) minus that boundary value, one form
// per 32-point sub-span where possible, accumulated in warp-private shared memory.
#include <cuda_fp16.h>
#include "rox_internal.cuh"
#include "rox_faddeeva.cuh"

namespace {

#define ROX_NDAW (ROX_DAW_NODES * ROX_DAW_STRIDE)
#define ROX_INV_PI 0.318309886183790672f

// Per-line constants of one (P,T) point for the batch in hand. Each line has a slot; slots are
// ordered by class -- lines whose window covers the whole span and whose slow zone misses it
// ("clean") first, then the other covering lines, then the lines cut by a window edge -- and
// slots 2k, 2k+1 form pair k. The pair tables hold both lines' far-form constants side by side,
// so one 16-byte load brings a field of both; the line table holds what window edges and pass 2
// need per slot. S is scaled by 2^-e (e the exponent of the largest strength at this
// temperature).
struct PairTab {
  float4 ab[16];   // {A0, A1, B0, B1}: far form t = X^2 + A, d = t^2 + B
  float4 pq[16];   // {P0, P1, Q0, Q1}: S V = (P t + Q) / d, P = S Y / pi, Q = P K
  float4 ef[16];   // uniform grid {E0, E1, F0, F1}: X at the lane's first point = (lane + E) dnu + F,
                   // E = (span start) - k0 (exact), F = -f dnu; nodes {ch0, ch1, cl0, cl1}: X = (D.hi - ch) + (D.lo - cl)
  float2 tz[16];   // {t_z0, t_z1}: the far form holds for t >= t_z; pass 1 evaluates it at max(t, t_z)
};
struct LineTab {
  int2 W[32];      // window [jlo, jhi] (grid indices)
  int2 Z[32];      // slow zone [zlo, zhi] (grid indices; nodes: the window)
  float iG[32];    // 1/gamma_G; negative if the slow zone is |z| < 6.5 not widened by the margin
  float y[32];     // gamma_L / gamma_G
  float pc[32];    // S / (gamma_G sqrt(pi))
  float cf[32];    // the far form at t = t_z, which pass 1 adds at every point of the slow zone
};
// one line's field out of a pair table row: half h (0, 1) of {lo, hi} pairs
__device__ __forceinline__ float row_lo(const float4& v, int h) { return h ? v.y : v.x; }
__device__ __forceinline__ float row_hi(const float4& v, int h) { return h ? v.w : v.z; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ float load_width(const void* p, int f16, long long i) {
  return f16 ? __half2float(reinterpret_cast<const __half*>(p)[i])
             : reinterpret_cast<const float*>(p)[i];
}

// the two per-line width inputs of line i: {gamma_ref, n_T} of the single power law, or, for
// broadened lists (BRD), {the broadeners' sum at the job's temperature, the natural width}
template <bool BRD>
__device__ __forceinline__ void load_widths(const RoxJobDev& J, const RoxListDev& L, int f16, long long i, float& a,
                                            float& b) {
  if constexpr (BRD) {
    a = L.gLT[(long long)J.t_row * L.gLT_stride + i];
    b = L.gN ? L.gN[i] : 0.0f;
  } else {
    a = load_width(L.gamma_ref, f16, i);
    b = load_width(L.n_t, f16, i);
  }
}

// Two FP32 values in one 64-bit register pair, for the paired FP32 instructions of sm_100 and
// later (fma.rn.f32x2 / add.rn.f32x2: two IEEE operations, each rounded as the scalar one). A
// paired instruction takes one issue slot for two operations, which leaves issue slots to the
// reciprocal, the clamps and the loads while the FMA pipes stay busy.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// Far-form constants of pair k, packed for the paired instructions.
struct PairC {
  f32x2 A, B, P, Q;
  float2 T;
  float e0, e1, f0, f1;
};
template <bool CLAMP>
__device__ __forceinline__ PairC pair_consts(const PairTab& P, int k) {
  PairC c;
  const float4 ab = P.ab[k], pq = P.pq[k], ef = P.ef[k];
  c.A = f2_pack(ab.x, ab.y);
  c.B = f2_pack(ab.z, ab.w);
  c.P = f2_pack(pq.x, pq.y);
  c.Q = f2_pack(pq.z, pq.w);
  c.T = CLAMP ? P.tz[k] : make_float2(0.0f, 0.0f);
  c.e0 = ef.x;
  c.e1 = ef.y;
  c.f0 = ef.z;
  c.f1 = ef.w;
  return c;
}

// acc + S0 V0 + S1 V1 for the pair's offsets x0, x1 at one point, the two fractions over one
// reciprocal, n0/d0 + n1/d1 = (n0 d1 + n1 d0)/(d0 d1). CLAMP: t = max(X^2 + A, t_z) per line
// (inside its slow zone a line contributes the far form's value at the zone boundary, which
// pass 2 takes out again). MASK: u0, u1 tell whether the point is in each line's window.
// Paired: X^2 + A, t^2 + B, P t + Q; scalar: 4 FP32 operations and 1 MUFU (+ 2 clamps).
template <bool CLAMP, bool MASK>
__device__ __forceinline__ float pair_add(float x0, float x1, const PairC& c, bool u0, bool u1, float acc) {
  const f32x2 x = f2_pack(x0, x1);
  f32x2 t = f2_fma(x, x, c.A);
  if (CLAMP) {
    float t0, t1;
    f2_unpack(t, t0, t1);
    t = f2_pack(fmaxf(t0, c.T.x), fmaxf(t1, c.T.y));
  }
  float d0, d1, n0, n1;
  f2_unpack(f2_fma(t, t, c.B), d0, d1);
  f2_unpack(f2_fma(t, c.P, c.Q), n0, n1);
  if (MASK) {
    n0 = u0 ? n0 : 0.0f;
    n1 = u1 ? n1 : 0.0f;
  }
  return fmaf(fmaf(n1, d0, n0 * d1), rox_rcp(d0 * d1), acc);
}

// The pair's offsets at this lane's first point (uniform grid): X = (lane + E) dnu + F, with
// lane + E = (span start + lane) - k0 exact, so X is the exact index decomposition rounded once.
template <bool NU>
__device__ __forceinline__ void pair_x0(const PairC& c, float lanef, float dnu_f, float& X0, float& X1) {
  if constexpr (NU) {
    X0 = X1 = 0.0f;
  } else {
    f2_unpack(f2_fma(f2_add(f2_pack(lanef, lanef), f2_pack(c.e0, c.e1)), f2_pack(dnu_f, dnu_f), f2_pack(c.f0, c.f1)),
              X0, X1);
  }
}

// X = nu - nu0 at this lane's point of sub-span m. Uniform grid: X0 + 32 m dnu (one rounding more).
// User-provided nodes: the node's double-float offset from the span's first node, D[32 m] =
// {hi, lo}, minus the line's {ch, cl}; the hi parts cancel exactly near the line, so X keeps
// its relative accuracy.
template <bool NU>
__device__ __forceinline__ float pos(int m, float X0, float ch, float cl, const float2* D, float dnu_f) {
  if constexpr (NU) {
    const float2 d = D[32 * m];
    return (d.x - ch) + (d.y - cl);
  } else {
    return fmaf((float)(32 * m), dnu_f, X0);
  }
}

// Pass 1 for covering pair k: every point of the span (CLAMP unless both lines are clean).
template <bool NU, bool CLAMP>
__device__ __forceinline__ void cover_pair(const PairTab& P, int k, float lanef, float dnu_f, const float2* D,
                                           float (&acc)[ROX_K]) {
  const PairC c = pair_consts<CLAMP>(P, k);
  float X0, X1;
  pair_x0<NU>(c, lanef, dnu_f, X0, X1);
#pragma unroll
  for (int m = 0; m < ROX_K; m++)
    acc[m] = pair_add<CLAMP, false>(pos<NU>(m, X0, c.e0, c.f0, D, dnu_f), pos<NU>(m, X1, c.e1, c.f1, D, dnu_f), c,
                                    true, true, acc[m]);
}

// Pass 1 for pair k of which at least one line is cut by a window edge: the sub-spans outside
// both windows are skipped (warp-uniform test); the sub-spans inside both windows take every
// point; elsewhere each point takes line i iff it lies in the line's window, m in
// [ceil((jlo-Aw-lane)/32), floor((jhi-Aw-lane)/32)] (the exact integer window). Lines arrive
// sorted by nu0, so paired edge lines have their edges in the same or a neighbouring sub-span.
template <bool NU>
__device__ __forceinline__ void edge_pair(const PairTab& P, const LineTab& L, int k, int Aw, int lane, float lanef,
                                          float dnu_f, const float2* D, float (&acc)[ROX_K]) {
  const PairC c = pair_consts<true>(P, k);
  const int2 w0 = L.W[2 * k], w1 = L.W[2 * k + 1];
  const int lo0 = w0.x - Aw, hi0 = w0.y - Aw, lo1 = w1.x - Aw, hi1 = w1.y - Aw;
  const int mf = max(0, min(lo0, lo1) >> 5), ml = min(ROX_K - 1, max(hi0, hi1) >> 5);
  const int mlo0 = (lo0 - lane + 31) >> 5, mhi0 = (hi0 - lane) >> 5;   // this lane's window, in m
  const int mlo1 = (lo1 - lane + 31) >> 5, mhi1 = (hi1 - lane) >> 5;
  const int cf = max((lo0 + 31) >> 5, (lo1 + 31) >> 5), cl = min((hi0 - 31) >> 5, (hi1 - 31) >> 5);
  float X0, X1;
  pair_x0<NU>(c, lanef, dnu_f, X0, X1);
#pragma unroll
  for (int m = 0; m < ROX_K; m++) {
    if (m < mf || m > ml) continue;
    const float x0 = pos<NU>(m, X0, c.e0, c.f0, D, dnu_f), x1 = pos<NU>(m, X1, c.e1, c.f1, D, dnu_f);
    if (m >= cf && m <= cl) {
      acc[m] = pair_add<true, false>(x0, x1, c, true, true, acc[m]);
    } else {
      acc[m] = pair_add<true, true>(x0, x1, c, m >= mlo0 && m <= mhi0, m >= mlo1 && m <= mhi1, acc[m]);
    }
  }
}

// Pass 1 for the line in slot s alone (the last of an odd count), window-masked per sub-span
// and point.
template <bool NU>
__device__ __forceinline__ void edge_line(const PairTab& P, const LineTab& L, int s, int Aw, int lane, float lanef,
                                          float dnu_f, const float2* D, float (&acc)[ROX_K]) {
  const int k = s >> 1, h = s & 1;
  const float4 ab = P.ab[k], pq = P.pq[k], ef = P.ef[k];
  const float A = row_lo(ab, h), B = row_hi(ab, h), Pc = row_lo(pq, h), Qc = row_hi(pq, h);
  const float e = row_lo(ef, h), f = row_hi(ef, h);
  const float tz = h ? P.tz[k].y : P.tz[k].x;
  const int2 w = L.W[s];
  const float X0 = NU ? 0.0f : fmaf(lanef + e, dnu_f, f);
#pragma unroll
  for (int m = 0; m < ROX_K; m++) {
    const int am = Aw + 32 * m, bm = am + 31;
    if (bm < w.x || am > w.y) continue;
    const int j = am + lane;
    const float x = pos<NU>(m, X0, e, f, D, dnu_f);
    const float t = fmaxf(fmaf(x, x, A), tz);
    const float v = fmaf(t, Pc, Qc) * rox_rcp(fmaf(t, t, B));
    acc[m] += (j >= w.x && j <= w.y) ? v : 0.0f;
  }
}

// Pass 2 for the line in slot s, whose slow zone meets the span: at exactly the points where
// pass 1 clamped t (t < t_z on the same rounded t, inside the window), the full FP32 Faddeeva
// forms replace the far form's boundary value that pass 1 added there: + S V - cf.
// A zone of |z| < 6.5 takes the core forms at every point (rox_re_w_core holds 1.1e-5 out to
// |z| = 7.1); on a uniform grid the lanes then take consecutive points of the zone rather than
// aligned 32-point sub-spans (fewer, fuller warp steps). Otherwise, per 32-point sub-span, one
// form for all points where possible: the 3-level fraction if even the sub-span's point nearest
// the centre has |z| >= 10, the 5-level one if |z| >= 6 there (both only get more accurate
// further out), else rox_re_w per point. Accumulated into the warp's shared-memory row zacc
// (one add per line and point; within a warp step the lanes touch distinct points).
template <bool NU>
__device__ __forceinline__ void zone_line(const PairTab& P, const LineTab& L, int s, int Aw, int lane, float lanef,
                                          float dnu_f, float inv_dnu, const float* daw, const float2* D, float* zacc) {
  const int k = s >> 1, h = s & 1;
  const float4 ab = P.ab[k], ef = P.ef[k];
  const float A = row_lo(ab, h), e = row_lo(ef, h), f = row_hi(ef, h);
  const float tz = h ? P.tz[k].y : P.tz[k].x;
  const int2 w = L.W[s], z = L.Z[s];
  const int lo = max(max(z.x, w.x), Aw), hi = min(min(z.y, w.y), Aw + ROX_SPAN - 1);
  if (lo > hi) return;
  const float iGs = L.iG[s], y = L.y[s], pcore = L.pc[s], cf = L.cf[s];
  const float invG = fabsf(iGs);
  if (!NU && iGs < 0.0f) {
    // lanes on consecutive points of [lo, hi]; t rounded exactly as pass 1 rounds it
    for (int q = lo - Aw + lane; q <= hi - Aw; q += 32) {
      const float X0q = fmaf((float)(q & 31) + e, dnu_f, f);
      const float Xm = fmaf((float)(q & ~31), dnu_f, X0q);
      if (!(fmaf(Xm, Xm, A) < tz)) continue;
      const float X = fmaf((float)q + e, dnu_f, f);
      zacc[q] += fmaf(pcore, rox_re_w_core(daw, fabsf(X) * invG, y), -cf);
    }
    return;
  }
  const float X0 = NU ? 0.0f : fmaf(lanef + e, dnu_f, f);
  if (iGs < 0.0f) {
    for (int m = (lo - Aw) >> 5; m <= ((hi - Aw) >> 5); m++) {
      const int j = Aw + 32 * m + lane;
      const float Xm = pos<NU>(m, X0, e, f, D, dnu_f);
      if (!(fmaf(Xm, Xm, A) < tz) || j < w.x || j > w.y) continue;
      // the uniform grid recomputes X from the index in one rounding; node offsets are exact already
      const float X = NU ? Xm : fmaf((float)(32 * m + lane) + e, dnu_f, f);
      zacc[32 * m + lane] += fmaf(pcore, rox_re_w_core(daw, fabsf(X) * invG, y), -cf);
    }
    return;
  }
  const float centre = (float)Aw - e - f * inv_dnu;     // k0 + f, within 0.25 grid steps (uniform grid)
  const float y2 = y * y;
  for (int m = (lo - Aw) >> 5; m <= ((hi - Aw) >> 5); m++) {
    const int am = Aw + 32 * m, bm = am + 31;
    const int j = am + lane;
    const float Xm = pos<NU>(m, X0, e, f, D, dnu_f);
    float xm;   // |X| of the sub-span's point nearest the line centre, in units of gamma_G
    if constexpr (NU) {
      const float Xa = __shfl_sync(0xffffffffu, Xm, 0), Xb = __shfl_sync(0xffffffffu, Xm, 31);
      xm = (Xa <= 0.0f && Xb >= 0.0f ? 0.0f : fminf(fabsf(Xa), fabsf(Xb))) * invG;
    } else {
      const float dc = (centre >= (float)am && centre <= (float)bm)
                           ? 0.0f : fminf(fabsf((float)am - centre), fabsf((float)bm - centre));
      xm = fmaxf(dc - 1.0f, 0.0f) * dnu_f * invG;
    }
    if (!(fmaf(Xm, Xm, A) < tz) || j < w.x || j > w.y) continue;
    const float sm = fmaf(xm, xm, y2);
    const float X = NU ? Xm : fmaf((float)(32 * m + lane) + e, dnu_f, f);
    const float x = fabsf(X) * invG;
    float r;
    if (sm >= ROX_S_CF3) r = rox_re_w_cf3(x, y);
    else if (sm >= ROX_S_CF5) r = rox_re_w_cf5g(x, y);
    else r = rox_re_w(daw, x, y);
    zacc[32 * m + lane] += fmaf(pcore, r, -cf);
  }
}

// Per-line constants of one (P,T) point that do not depend on the span: the far-form
// constants, the slow zone's half-width hz (at least the precision margin) and threshold t_z,
// and what pass 2 needs. nu0f: the line centre in FP32; Sp: S 2^-e; gref, nt: the width inputs
// (see load_widths). The Voigt kernel computes them per line and span, or (ROX_VX_PRE) reads
// them from k_line_params, which computes them once per line with this same function.
struct LineK {
  float A, B, P, Q, tz, iGs, y, pc, cf, hz;
};
template <bool BRD>
__device__ __forceinline__ LineK line_consts(float nu0f, float Sp, float gref, float nt, const RoxJobDev& J,
                                             float margin_cm, bool want_cf) {
  LineK k;
  const float gG = nu0f * J.gG_fac;
  const float gL = BRD ? fmaf(gref, J.p_fac, nt) : gref * rox_exp2(nt * J.l2_ratio) * J.p_fac;
  const float gG2 = gG * gG, gL2 = gL * gL;
  const float pY = Sp * gL * ROX_INV_PI;
  const float invG = rox_rcp(gG);
  k.y = gL * invG;
  const rox_far fc = rox_far_coefs(k.y);      // far-zone form of this line (rox_faddeeva.cuh)
  // slow zone: |X| < sqrt(r2 gamma_G^2 - gamma_L^2), at least the precision margin
  const float hz2 = fmaxf(0.0f, fc.r2 * gG2 - gL2);
  float hz = hz2 * rox_rsqrt(hz2);            // 0 for hz2 = 0 (rsqrt(0) = inf, product taken as 0 below)
  hz = hz2 > 0.0f ? hz : 0.0f;
  // zone |z| < 6.5 not widened by the margin: the core forms cover all of it
  const bool core_only = fc.r2 == ROX_S_PADE && hz >= margin_cm;
  k.hz = fmaxf(hz, margin_cm);
  k.A = fc.alpha * gG2;
  k.B = fc.beta * (gG2 * gG2);
  k.P = pY;
  k.Q = pY * (fc.kappa * gG2);
  k.tz = fmaf(k.hz, k.hz, k.A);
  k.iGs = core_only ? -invG : invG;
  k.pc = Sp * invG * ROX_INV_SQRT_PI;
  k.cf = want_cf ? fmaf(k.tz, k.P, k.Q) * rox_rcp(fmaf(k.tz, k.tz, k.B)) : 0.0f;
  return k;
}

// Grid indices of a line's slow zone on a uniform grid, |j - (k0 + f)| < hz / dnu, widened by 1e-4
// relative and one point on each side (covers every point with t < t_z despite the roundings).
// g: the line's geometry record {k0, f dnu, jlo, jhi}.
__device__ __forceinline__ void zone_bounds(const float4& g, float hz, float inv_dnu, int& zlo, int& zhi) {
  const int k0 = (int)g.x;
  const float hzg = fminf(hz * inv_dnu * 1.0001f, 8.0e6f);
  const float fr = g.y * inv_dnu;
  zlo = k0 + __float2int_rd(fr - hzg) - 1;
  zhi = k0 + __float2int_ru(fr + hzg) + 1;
}

// the uniform grid's precision margin of the slow zones (cm^-1; see ROX_FAST_MARGIN)
__device__ __forceinline__ float fast_margin(float dnu_f) { return ROX_FAST_MARGIN * 32.0f * (ROX_K - 1) * dnu_f; }

// k_line_params: the per-line constants of one job ((P,T) point) for lines [J.l0, J.l1) of a
// uniform-grid list, once per line, for the ROX_VX_PRE Voigt launch (which otherwise recomputes
// them in every span a line reaches). One thread per line, coalesced loads and 48-byte stores.
__global__ void k_line_params(const RoxListDev L, const RoxJobDev J, float4* rec) {
  const float margin_cm = fast_margin(L.dnu_f);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = J.l0 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < J.l1; i += stride) {
    const float4 g = L.geo[i];
    const float Sp = J.S32[i - J.l0];
    const float gref = load_width(L.gamma_ref, L.width_f16, i), nt = load_width(L.n_t, L.width_f16, i);
    const float nu0f = L.nu_min_f + fmaf(g.x, L.dnu_f, g.y);
    const LineK k = line_consts<false>(nu0f, Sp, gref, nt, J, margin_cm, true);
    int zlo, zhi;
    zone_bounds(g, k.hz, L.inv_dnu_f, zlo, zhi);
    rec[3 * i] = make_float4(k.A, k.B, k.P, k.Q);
    rec[3 * i + 1] = make_float4(k.tz, k.iGs, k.y, k.pc);
    rec[3 * i + 2] = make_float4(k.cf, __int_as_float(zlo), __int_as_float(zhi), 0.0f);
  }
}

// NU: the lists are on user-provided nodes (node offsets in dynamic shared memory, one
// ROX_SPAN row of float2 per warp). X: ROX_VX_INDEX (each list is a subset of the sorted lines,
// given by RoxListDev::idx, e.g. the kept lines of a main-contributor selection; span ranges
// then count positions in that index) and ROX_VX_BROAD (widths from the broadening pass). Each
// extra is compiled only into the instantiations that use it: in this kernel even a few added
// instructions per line batch cost several percent of the plain launch.
template <bool NU, int X, int W>
__global__ void __launch_bounds__(W * 32, 24 / W) k_voigt(const __grid_constant__ RoxVoigtArgs A) {
  constexpr bool IDX = (X & ROX_VX_INDEX) != 0;
  constexpr bool BRD = (X & ROX_VX_BROAD) != 0;
  constexpr bool PRE = (X & ROX_VX_PRE) != 0;
  extern __shared__ __align__(16) float2 s_nodes[];   // NU: node offsets; PRE: the staged per-line constants
  __shared__ float4 s_geo[W][2][32];
  __shared__ float s_S[W][2][32];
  __shared__ PairTab s_pairs[W];
  __shared__ LineTab s_lines[W];
  __shared__ float s_zacc[W][ROX_SPAN];
  __shared__ float s_tot[W][ROX_SPAN];    // the span's sum over its parts
  __shared__ float s_daw[ROX_NDAW];
  __shared__ int s_status;

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < ROX_NDAW; i += W * 32) s_daw[i] = (&rox_daw_taylor[0][0])[i];
  if (tid == 0) s_status = *(volatile int32_t*)&A.hdr->status;
  __syncthreads();
  if (s_status != ROX_OK) return;   // e.g. unsorted input: leave sigma untouched

  float4(*geo_st)[32] = s_geo[w];
  float(*S_st)[32] = s_S[w];
  PairTab& PT = s_pairs[w];
  LineTab& LT = s_lines[w];
  const float lanef = (float)lane;
  float* zacc = s_zacc[w];
  float* stot = s_tot[w];
  float2* Drow = NU ? s_nodes + w * ROX_SPAN : nullptr;   // this span's node offsets
  // PRE: per warp two buffers of 32 lines x 3 float4 of per-line constants
  float4(*rec_st)[32][3] = PRE ? reinterpret_cast<float4(*)[32][3]>(s_nodes) + 2 * w : nullptr;
  const float2* D = NU ? Drow + lane : nullptr;
  unsigned long long evals = 0;   // (line, point) pairs inside the cutoff and the job's window

  for (;;) {
    int q = 0, k = 0;
    if (lane == 0) {
      q = atomicAdd(&A.hdr->work_counter, 1);
      const int it = q < A.n_whole ? q : A.n_whole + (q - A.n_whole) / ROX_PARTS;
      int lo_k = 0, hi_k = A.n_jobs - 1;           // first job with item_end > it
      while (lo_k < hi_k) {
        const int mid = (lo_k + hi_k) >> 1;
        if (A.item_end[mid] > it) hi_k = mid; else lo_k = mid + 1;
      }
      k = lo_k;
    }
    q = __shfl_sync(0xffffffffu, q, 0);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (q >= A.n_queue) break;
    // queue entry -> item and part (-1: the whole span, all parts in order)
    const int item = q < A.n_whole ? q : A.n_whole + (q - A.n_whole) / ROX_PARTS;
    const int part = q < A.n_whole ? -1 : (q - A.n_whole) % ROX_PARTS;
    const RoxJobDev& J = A.job[k];
    const RoxListDev& Lst = A.list[J.list];
    const int local = item - (k > 0 ? A.item_end[k - 1] : 0);
    const int span = J.span_first + J.n_spans - 1 - local;       // wide-line (high nu) spans first
    const int f16 = Lst.width_f16;
    // compensation weight of the part sums: 1 (ROX_KAHAN) keeps the Kahan correction term, 0
    // zeroes it, which leaves the plain sum (one branch-free form for both)
    const float kw = (J.flags & ROX_KAHAN) ? 1.0f : 0.0f;
    const float dnu_f = Lst.dnu_f;
    // offsets on a uniform grid round once more (X0 + 32 m dnu), hence the precision margin
    const float margin_cm = NU ? 0.0f : fast_margin(dnu_f);
    const int Aw = span * ROX_SPAN;
    const int Bw = Aw + ROX_SPAN - 1;
    if (*Lst.status != ROX_OK) continue;           // list not prepared from sorted lines
    float bh = 0.f, bl = 0.f, Ws = 0.f;             // span's first node; offset of its last node
    if constexpr (NU) {
#pragma unroll
      for (int m = 0; m < ROX_K; m++) Drow[32 * m + lane] = Lst.node_d[(long long)Aw + 32 * m + lane];
      const float2 b = Lst.span_base[span];
      bh = b.x;
      bl = b.y;
      __syncwarp();
      Ws = Drow[ROX_SPAN - 1].x;
    }
    const long long lo = max(Lst.span_lo[span], J.l0), hi = min(Lst.span_hi[span], J.l1);
    const long long wlo = J.first > Aw ? J.first : Aw;             // evaluated points of this span
    const long long whi = (J.first + J.n - 1) < Bw ? (J.first + J.n - 1) : Bw;
    const double smax = __longlong_as_double((long long)*J.smax_bits);
    const int e = smax > 0.0 ? ilogb(smax) : 0;     // S32 holds S * 2^-e (FP32)
    const float* S_row = J.S32 - J.l0;              // indexed by line number

    const long long nbat = hi > lo ? (hi - lo + 31) >> 5 : 0;
    const int p_first = part < 0 ? 0 : part, p_last = part < 0 ? ROX_PARTS - 1 : part;
    for (int p = p_first; p <= p_last; p++) {
      const long long plo = lo + 32 * ((nbat * p) / ROX_PARTS);
      const long long phi = min(hi, lo + 32 * ((nbat * (p + 1)) / ROX_PARTS));
      float acc[ROX_K], tot[ROX_K], cmp[ROX_K];
#pragma unroll
      for (int m = 0; m < ROX_K; m++) { acc[m] = 0.f; tot[m] = 0.f; cmp[m] = 0.f; zacc[32 * m + lane] = 0.f; }

      // stage batch 0; widths go through registers one batch ahead (with an index, the
      // positions' line numbers two batches ahead)
      float gref = 0.f, nt = 0.f;
      long long li_n = 0;   // IDX: line number of this lane's position in the next batch
      if (plo + lane < phi) {
        const long long li = IDX ? (long long)Lst.idx[plo + lane] : plo + lane;
        cp_async16(&geo_st[0][lane], &Lst.geo[li]);
        if constexpr (PRE) {
#pragma unroll
          for (int c = 0; c < 3; c++) cp_async16(&rec_st[0][lane][c], &Lst.rec[3 * li + c]);
        } else {
          cp_async4(&S_st[0][lane], &S_row[li]);
          load_widths<BRD>(J, Lst, f16, li, gref, nt);
        }
      }
      if (IDX && plo + 32 + lane < phi) li_n = Lst.idx[plo + 32 + lane];
      cp_async_commit();
      int nb = 0;
      for (long long b0 = plo; b0 < phi; b0 += 32, nb++) {
        const int cnt = (int)min((long long)32, phi - b0);
        const int buf = nb & 1;
        float gref_n = 0.f, nt_n = 0.f;
        if (b0 + 32 + lane < phi) {
          const long long li = IDX ? li_n : b0 + 32 + lane;
          cp_async16(&geo_st[buf ^ 1][lane], &Lst.geo[li]);
          if constexpr (PRE) {
#pragma unroll
            for (int c = 0; c < 3; c++) cp_async16(&rec_st[buf ^ 1][lane][c], &Lst.rec[3 * li + c]);
          } else {
            cp_async4(&S_st[buf ^ 1][lane], &S_row[li]);
            load_widths<BRD>(J, Lst, f16, li, gref_n, nt_n);
          }
        }
        if (IDX && b0 + 64 + lane < phi) li_n = Lst.idx[b0 + 64 + lane];
        cp_async_commit();
        cp_async_wait1();   // this lane's copies of the current batch have landed

        // ---- per-line constants (lane <-> line b0 + lane), written to the line's slot
        const bool live = lane < cnt;
        bool covers = false, zoned = false;
        float ax = 0.f, ay = 0.f, vA = 1.f, vB = 0.f, vP = 0.f, vQ = 0.f, tz = 0.f, iGs = 1.f, yv = 0.f, pcv = 0.f;
        float cfv = 0.f;
        int jlo = 1, jhi = 0, zlo = 0, zhi = -1;
        if (live) {
          const float4 g = geo_st[buf][lane];
          jlo = __float_as_int(g.z);
          jhi = __float_as_int(g.w);
          const int ov = min(jhi, (int)whi) - max(jlo, (int)wlo) + 1;
          if (ov > 0) evals += (unsigned)ov;
          covers = Aw >= jlo && Bw <= jhi;
          LineK kc;
          if constexpr (PRE) {
            // uniform grid, constants from k_line_params
            const float4 r0 = rec_st[buf][lane][0], r1 = rec_st[buf][lane][1], r2 = rec_st[buf][lane][2];
            kc.A = r0.x;
            kc.B = r0.y;
            kc.P = r0.z;
            kc.Q = r0.w;
            kc.tz = r1.x;
            kc.iGs = r1.y;
            kc.y = r1.z;
            kc.pc = r1.w;
            kc.cf = r2.x;
            zlo = __float_as_int(r2.y);
            zhi = __float_as_int(r2.z);
            ax = (float)Aw - g.x;     // exact: both are integers below 2^24
            ay = -g.y;
            zoned = !(Bw < zlo || Aw > zhi);
          } else {
            const float Sp = S_st[buf][lane];
            float nu0f;   // line centre; its offset state {E, F} (uniform grid) or {c hi, c lo} (nodes)
            if constexpr (NU) {
              // c = nu0 - (span's first node) as a double-float pair (the hi parts cancel exactly)
              nu0f = g.x;
              const float ch = g.x - bh, cl = g.y - bl;
              ax = ch + cl;
              ay = cl - (ax - ch);
            } else {
              nu0f = Lst.nu_min_f + fmaf(g.x, dnu_f, g.y);
              ax = (float)Aw - g.x;     // exact: both are integers below 2^24
              ay = -g.y;
            }
            kc = line_consts<BRD>(nu0f, Sp, gref, nt, J, margin_cm, false);
            if constexpr (NU) {
              // the span's offsets run from -c to Ws - c; pass 2 then scans the window itself
              const float hzp = kc.hz * 1.001f + 1e-6f * (fabsf(ax) + Ws);
              zoned = -ax < hzp && Ws - ax > -hzp;
              zlo = jlo;
              zhi = jhi;
            } else {
              zone_bounds(g, kc.hz, Lst.inv_dnu_f, zlo, zhi);
              zoned = !(Bw < zlo || Aw > zhi);
            }
            if (zoned) kc.cf = fmaf(kc.tz, kc.P, kc.Q) * rox_rcp(fmaf(kc.tz, kc.tz, kc.B));
          }
          vA = kc.A;
          vB = kc.B;
          vP = kc.P;
          vQ = kc.Q;
          tz = kc.tz;
          iGs = kc.iGs;
          yv = kc.y;
          pcv = kc.pc;
          cfv = kc.cf;
        }
        const unsigned clean = __ballot_sync(0xffffffffu, live && covers && !zoned);
        const unsigned czone = __ballot_sync(0xffffffffu, live && covers && zoned);
        const unsigned edge = __ballot_sync(0xffffffffu, live && !covers);
        const int nclean = __popc(clean), ncov = nclean + __popc(czone);
        const unsigned below = (1u << lane) - 1u;
        const int slot = !covers ? ncov + __popc(edge & below)
                                 : (zoned ? nclean + __popc(czone & below) : __popc(clean & below));
        const unsigned zslots = __reduce_or_sync(0xffffffffu, (live && zoned) ? (1u << slot) : 0u);
        if (live) {
          const int k = slot >> 1, h = slot & 1;
          float* ab = reinterpret_cast<float*>(&PT.ab[k]);
          float* pq = reinterpret_cast<float*>(&PT.pq[k]);
          float* ef = reinterpret_cast<float*>(&PT.ef[k]);
          ab[h] = vA;
          ab[2 + h] = vB;
          pq[h] = vP;
          pq[2 + h] = vQ;
          ef[h] = ax;
          ef[2 + h] = ay;
          reinterpret_cast<float*>(&PT.tz[k])[h] = tz;
          LT.W[slot] = make_int2(jlo, jhi);
          LT.Z[slot] = make_int2(zlo, zhi);
          LT.iG[slot] = iGs;
          LT.y[slot] = yv;
          LT.pc[slot] = pcv;
          LT.cf[slot] = cfv;
        }
        gref = gref_n;
        nt = nt_n;
        __syncwarp();

        // ---- pass 1: far formula at every point of every line's window. Clean pairs as they
        // are; pairs with a zoned line with t clamped to the zone boundary; then the rest (an odd
        // covering line, the window-edge lines) in pairs with window masks. Fixed orders: the sum
        // is reproducible.
        const int kc = nclean >> 1, kz = ncov >> 1;
        for (int k = 0; k < kc; k++) cover_pair<NU, false>(PT, k, lanef, dnu_f, D, acc);
        for (int k = kc; k < kz; k++) cover_pair<NU, true>(PT, k, lanef, dnu_f, D, acc);
        for (int s2 = 2 * kz; s2 < cnt; s2 += 2) {
          if (s2 + 1 < cnt) edge_pair<NU>(PT, LT, s2 >> 1, Aw, lane, lanef, dnu_f, D, acc);
          else edge_line<NU>(PT, LT, s2, Aw, lane, lanef, dnu_f, D, acc);
        }
        // ---- pass 2: at the points each zoned line had clamped, the full Faddeeva forms
        for (unsigned z = zslots; z; z &= z - 1)
          zone_line<NU>(PT, LT, __ffs(z) - 1, Aw, lane, lanef, dnu_f, Lst.inv_dnu_f, s_daw, D, zacc);
        __syncwarp();
        // the partial sums into the part's total every 4 batches: compensated (Kahan) with
        // ROX_KAHAN, else plainly (kw = 0: the correction term stays 0)
        if ((nb & 3) == 3 || b0 + 32 >= phi) {
#pragma unroll
          for (int m = 0; m < ROX_K; m++) {
            const float yk = acc[m] - cmp[m];
            const float tk = tot[m] + yk;
            cmp[m] = ((tk - tot[m]) - yk) * kw;
            tot[m] = tk;
            acc[m] = 0.f;
          }
        }
      }
      cp_async_wait0();
      // fold in the pass-2 (near-centre) sums
#pragma unroll
      for (int m = 0; m < ROX_K; m++) {
        const float yk = zacc[32 * m + lane] - cmp[m];
        const float tk = tot[m] + yk;
        cmp[m] = ((tk - tot[m]) - yk) * kw;
        tot[m] = tk;
      }
      if (part >= 0) {           // a split item: this part's sum goes to the tail scratch
        float* dst = A.tail_part + ((size_t)(item - A.n_whole) * ROX_PARTS + p) * ROX_SPAN;
#pragma unroll
        for (int m = 0; m < ROX_K; m++) __stcg(&dst[32 * m + lane], tot[m]);
      } else {
#pragma unroll
        for (int m = 0; m < ROX_K; m++) stot[32 * m + lane] = p == 0 ? tot[m] : stot[32 * m + lane] + tot[m];
      }
      __syncwarp();
    }   // parts

    if (part >= 0) {
      // the last part to finish adds the parts in order (the same sum as a whole item)
      __threadfence();
      __syncwarp();
      int done = 0;
      if (lane == 0) done = atomicAdd(&A.tail_cnt[item - A.n_whole], 1);
      done = __shfl_sync(0xffffffffu, done, 0);
      if (done != ROX_PARTS - 1) continue;
      __threadfence();
      const float* src = A.tail_part + (size_t)(item - A.n_whole) * ROX_PARTS * ROX_SPAN;
#pragma unroll
      for (int m = 0; m < ROX_K; m++) {
        float v = __ldcg(&src[32 * m + lane]);
#pragma unroll
        for (int pp = 1; pp < ROX_PARTS; pp++) v = v + __ldcg(&src[pp * ROX_SPAN + 32 * m + lane]);
        stot[32 * m + lane] = v;
      }
    }
    // ---- write the span once (its part inside the job's window); a value beyond the FP32
    // range is written as it is and flagged (rox_ws_status: ROX_EOVERFLOW)
    float* out = J.sigma - J.first;
    bool bad = false;
#pragma unroll
    for (int m = 0; m < ROX_K; m++) {
      const long long j = (long long)Aw + 32 * m + lane;
      if (j >= wlo && j <= whi) {
        const float v = ldexpf(stot[32 * m + lane], e);
        const float o = (J.flags & ROX_ACCUMULATE) ? out[j] + v : v;
        bad |= !isfinite(o);
        out[j] = o;
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&A.hdr->overflow, 1);
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&A.hdr->evals_total, evals);
}

// Probe of the attainable rate of pass 1's inner loop: cover_pair for clean pairs (the code
// k_voigt runs for most pairs), alone, with W warps per CTA as k_voigt's launch, on synthetic
// far-wing constants held in each warp's pair table (offsets of 3-8 cm^-1, so no clamp or mask
// applies). Each warp walks its 16 pairs `reps` times; no line set-up, staging, edges or slow
// zones. Not part of the cross-section method.
template <int W>
__global__ void __launch_bounds__(W * 32, 24 / W) k_pair_loop_probe(float* out, int reps, float dnu_f) {
  __shared__ PairTab s_pairs[W];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  PairTab& PT = s_pairs[w];
  if (lane < 16) {
    const float i0 = (float)(2 * lane), i1 = (float)(2 * lane + 1);
    PT.ab[lane] = make_float4(1.0e-4f * (1.0f + i0), 1.0e-4f * (1.0f + i1), 1.0e-8f * (1.0f + i0), 1.0e-8f * (1.0f + i1));
    PT.pq[lane] = make_float4(1.0e-3f, 1.1e-3f, 2.0e-7f, 2.1e-7f);
    PT.ef[lane] = make_float4(-300.0f - 17.0f * i0, -300.0f - 17.0f * i1, -0.0037f * (i0 + 1.0f), -0.0037f * (i1 + 1.0f));
    PT.tz[lane] = make_float2(0.0f, 0.0f);
  }
  __syncwarp();
  float acc[ROX_K];
#pragma unroll
  for (int m = 0; m < ROX_K; m++) acc[m] = 0.0f;
  const float lanef = (float)lane;
  for (int r = 0; r < reps; r++) {
#pragma unroll 1
    for (int k = 0; k < 16; k++) cover_pair<false, false>(PT, k, lanef, dnu_f, nullptr, acc);
  }
  float t = 0.0f;
#pragma unroll
  for (int m = 0; m < ROX_K; m++) t += acc[m];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

__global__ void k_faddeeva(const float* x, const float* y, float* out, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = rox_re_w(&rox_daw_taylor[0][0], x[i], y[i]);
}

}  // namespace

namespace {
// dynamic shared memory of an instantiation with W warps per CTA: the node rows (NU) or the
// staged per-line constants (ROX_VX_PRE)
template <bool NU, int X, int W>
constexpr size_t voigt_dyn_smem() {
  return NU ? (size_t)W * ROX_SPAN * sizeof(float2)
            : ((X & ROX_VX_PRE) ? (size_t)W * 2 * 32 * 3 * sizeof(float4) : (size_t)0);
}
}  // namespace

// per-line constants of job J (one (P,T) point) for its lines [J.l0, J.l1): rec[3 i .. 3 i + 2]
cudaError_t rox_launch_line_params(const RoxListDev& L, const RoxJobDev& J, float4* rec, cudaStream_t s) {
  const long long n = J.l1 - J.l0;
  if (n <= 0) return cudaSuccess;
  long long b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_line_params<<<(int)b, 256, 0, s>>>(L, J, rec);
  return cudaGetLastError();
}

namespace {

template <bool NU, int X, int W>
cudaError_t launch_k(const RoxVoigtArgs& A, int n_blocks, cudaStream_t s) {
  constexpr size_t dyn = voigt_dyn_smem<NU, X, W>();
  if (dyn) {   // static shared memory plus these exceed 48 KB: opt in (idempotent, per device)
    cudaError_t e = cudaFuncSetAttribute(k_voigt<NU, X, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  k_voigt<NU, X, W><<<n_blocks, W * 32, dyn, s>>>(A);
  return cudaGetLastError();
}

template <bool NU, int X, int W>
cudaError_t blocks_k(int* nb) {
  constexpr size_t dyn = voigt_dyn_smem<NU, X, W>();
  if (dyn) {
    cudaError_t e = cudaFuncSetAttribute(k_voigt<NU, X, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_voigt<NU, X, W>, W * 32, dyn);
}

template <int W>
cudaError_t launch_w(const RoxVoigtArgs& A, int n_blocks, bool nodes, int extras, cudaStream_t s) {
  if (nodes) {
    if (extras) return cudaErrorNotSupported;   // no caller combines nodes with a selection or broadening
    return launch_k<true, 0, W>(A, n_blocks, s);
  }
  switch (extras) {
    case 0: return launch_k<false, 0, W>(A, n_blocks, s);
    case ROX_VX_INDEX: return launch_k<false, ROX_VX_INDEX, W>(A, n_blocks, s);
    case ROX_VX_BROAD: return launch_k<false, ROX_VX_BROAD, W>(A, n_blocks, s);
    case ROX_VX_PRE: return launch_k<false, ROX_VX_PRE, W>(A, n_blocks, s);
    default: return cudaErrorNotSupported;   // no entry point combines these extras
  }
}

template <int W>
cudaError_t blocks_w(int* nb, bool nodes, bool pre) {
  if (pre) return blocks_k<false, ROX_VX_PRE, W>(nb);
  if (nodes) return blocks_k<true, 0, W>(nb);
  return blocks_k<false, 0, W>(nb);
}

}  // namespace

// warps: warps per CTA of the launch (4 or 8; the launch configuration of rox_launch_config)
cudaError_t rox_launch_voigt(const RoxVoigtArgs& A, int n_blocks, bool nodes, int extras, int warps, cudaStream_t s) {
  if (warps == 4) return launch_w<4>(A, n_blocks, nodes, extras, s);
  if (warps == 8) return launch_w<8>(A, n_blocks, nodes, extras, s);
  return cudaErrorInvalidValue;
}

cudaError_t rox_voigt_blocks_per_sm(int* nb, bool nodes, bool pre, int warps) {
  if (warps == 4) return blocks_w<4>(nb, nodes, pre);
  if (warps == 8) return blocks_w<8>(nb, nodes, pre);
  return cudaErrorInvalidValue;
}

// pair-loop probe: n_blocks CTAs of `warps` warps (4 or 8); out holds n_blocks * warps * 32 floats
cudaError_t rox_launch_pair_loop_probe(int n_blocks, int warps, int reps, float* out, cudaStream_t s) {
  if (warps == 4) k_pair_loop_probe<4><<<n_blocks, 4 * 32, 0, s>>>(out, reps, 0.01f);
  else if (warps == 8) k_pair_loop_probe<8><<<n_blocks, 8 * 32, 0, s>>>(out, reps, 0.01f);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t rox_launch_faddeeva(const float* x, const float* y, float* out, long long n, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_faddeeva<<<(int)b, 256, 0, s>>>(x, y, out, n);
  return cudaGetLastError();
}
