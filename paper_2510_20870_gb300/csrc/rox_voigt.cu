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
// operations and one MUFU per point. The slow zone is x^2 + y^2 < 6.5^2 for y < 0.5 (per-line
// Pade form) and < 22^2 otherwise (2-level continued fraction), at least the precision margin.
// Lines are evaluated in two passes per batch. Pass 1 applies the far formula to every line
// whose window covers the span, in pairs, with the numerator set to zero inside the line's
// slow zone (t < t_z, one precomputed threshold); lines cut by a window edge take the same
// masked formula in pairs too, with per-point window masks. Pass 2 evaluates exactly the
// complementary points (t < t_z, decided on the same rounded t) with the full FP32 Faddeeva
// forms (rox_faddeeva.cuh), one form per 32-point sub-span where possible, accumulated in
// warp-private shared memory.
#include <cuda_fp16.h>
#include "rox_internal.cuh"
#include "rox_faddeeva.cuh"

namespace {

#define ROX_NDAW (ROX_DAW_NODES * ROX_DAW_STRIDE)
#define ROX_INV_PI 0.318309886183790672f

// Per-line constants of one (P,T) point, one record per staged line:
//   a = {k0 (exact float), f*dnu, A, B}            (far form t = X^2 + A, d = t^2 + B)
//   b = {S Y / pi, (S Y / pi) K, class bits (1: window covers the span, 2: slow zone meets
//        the span), t_z (far formula iff t >= t_z)}
//   c = {jlo, jhi, zlo, zhi} (int bits; window and slow zone, inclusive grid indices)
//   d = {1/gamma_G, y = gamma_L/gamma_G, S/(gamma_G sqrt(pi)), 1 if the slow zone is |z| < 6.5
//        (per-line Pade far form, not widened by the precision margin), else 0}
// S is scaled by 2^-e (e the exponent of the largest strength at this temperature).
struct __align__(16) Rec {
  float4 a, b, c, d;
};

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

// one point of one line outside the slow zone: S V = n / d
__device__ __forceinline__ float far_term(float X, const float4& a, const float4& b) {
  float t = fmaf(X, X, a.z);
  float d = fmaf(t, t, a.w);
  float n = fmaf(t, b.x, b.y);
  return n * rox_rcp(d);
}

// far formula with the slow-zone mask of pass 1: zero where t < t_z (there the denominator,
// which may vanish inside the zone, is replaced by 1)
__device__ __forceinline__ float masked_far(float X, const float4& a, const float4& b) {
  const float t = fmaf(X, X, a.z);
  const bool f = t >= b.w;
  const float d = f ? fmaf(t, t, a.w) : 1.0f;
  const float n = f ? fmaf(t, b.x, b.y) : 0.0f;
  return n * rox_rcp(d);
}

// X = nu - nu0 at this lane's point of sub-span m. Uniform grid: X0 + 32 m dnu, X0 the offset
// at the lane's first point (from the exact index decomposition). User-provided nodes: the
// node's double-float offset from the span's first node, D[32 m] = {hi, lo}, minus the line's,
// a = {c hi, c lo}; the hi parts cancel exactly near the line, so X keeps its relative accuracy.
template <bool NU>
__device__ __forceinline__ float pos(int m, float X0, const float4& a, const float2* D, float dnu_f) {
  if constexpr (NU) {
    const float2 d = D[32 * m];
    return (d.x - a.x) + (d.y - a.y);
  } else {
    return fmaf((float)(32 * m), dnu_f, X0);
  }
}

// Pass 1 for a line whose window edge falls inside the span: per 32-point sub-span, skipped if
// outside the window, the masked far formula otherwise, masked per point where cut.
template <bool NU>
__device__ __forceinline__ void edge_line(const float4& a, const float4& b, const float4& c, int Aw, int lane,
                                          float Jf, float dnu_f, const float2* D, float (&acc)[ROX_K]) {
  const float X0 = fmaf(Jf - a.x, dnu_f, -a.y);
  const int jlo = __float_as_int(c.x), jhi = __float_as_int(c.y);
#pragma unroll
  for (int m = 0; m < ROX_K; m++) {
    const int am = Aw + 32 * m, bm = am + 31;
    if (bm < jlo || am > jhi) continue;
    const int j = am + lane;
    const float v = masked_far(pos<NU>(m, X0, a, D, dnu_f), a, b);
    acc[m] += (j >= jlo && j <= jhi) ? v : 0.0f;
  }
}

// Pass 1 for two lines cut by window edges, sharing one reciprocal as the covering lines do.
// The sub-spans outside both windows are skipped (warp-uniform test); elsewhere each point
// takes line i iff it lies in the window, m in [ceil((jlo-Aw-lane)/32), floor((jhi-Aw-lane)/32)]
// (the exact integer window), and outside the slow zone. Lines arrive sorted by nu0, so
// paired edge lines have their edges in the same or a neighbouring sub-span.
template <bool NU>
__device__ __forceinline__ void edge_pair(const Rec& r0, const Rec& r1, int Aw, int lane, float Jf, float dnu_f,
                                          const float2* D, float (&acc)[ROX_K]) {
  const float4 a0 = r0.a, b0 = r0.b, a1 = r1.a, b1 = r1.b;
  const int lo0 = __float_as_int(r0.c.x) - Aw, hi0 = __float_as_int(r0.c.y) - Aw;
  const int lo1 = __float_as_int(r1.c.x) - Aw, hi1 = __float_as_int(r1.c.y) - Aw;
  const int mf = max(0, min(lo0, lo1) >> 5), ml = min(ROX_K - 1, max(hi0, hi1) >> 5);
  const int mlo0 = (lo0 - lane + 31) >> 5, mhi0 = (hi0 - lane) >> 5;   // this lane's window, in m
  const int mlo1 = (lo1 - lane + 31) >> 5, mhi1 = (hi1 - lane) >> 5;
  // sub-spans inside both windows, when neither line's slow zone meets the span: no masks
  const bool nozone = !((__float_as_uint(b0.z) | __float_as_uint(b1.z)) & 2u);
  const int cf = nozone ? max((lo0 + 31) >> 5, (lo1 + 31) >> 5) : ROX_K;
  const int cl = min((hi0 - 31) >> 5, (hi1 - 31) >> 5);
  const float X0 = fmaf(Jf - a0.x, dnu_f, -a0.y), X1 = fmaf(Jf - a1.x, dnu_f, -a1.y);
#pragma unroll
  for (int m = 0; m < ROX_K; m++) {
    if (m < mf || m > ml) continue;
    const float x0 = pos<NU>(m, X0, a0, D, dnu_f), x1 = pos<NU>(m, X1, a1, D, dnu_f);
    const float t0 = fmaf(x0, x0, a0.z), t1 = fmaf(x1, x1, a1.z);
    if (m >= cf && m <= cl) {
      const float d0 = fmaf(t0, t0, a0.w), d1 = fmaf(t1, t1, a1.w);
      const float n0 = fmaf(t0, b0.x, b0.y), n1 = fmaf(t1, b1.x, b1.y);
      acc[m] = fmaf(fmaf(n1, d0, n0 * d1), rox_rcp(d0 * d1), acc[m]);
      continue;
    }
    const bool f0 = t0 >= b0.w && m >= mlo0 && m <= mhi0;
    const bool f1 = t1 >= b1.w && m >= mlo1 && m <= mhi1;
    const float d0 = f0 ? fmaf(t0, t0, a0.w) : 1.0f, d1 = f1 ? fmaf(t1, t1, a1.w) : 1.0f;
    const float n0 = f0 ? fmaf(t0, b0.x, b0.y) : 0.0f, n1 = f1 ? fmaf(t1, b1.x, b1.y) : 0.0f;
    acc[m] = fmaf(fmaf(n1, d0, n0 * d1), rox_rcp(d0 * d1), acc[m]);
  }
}

// Pass 2 for a line whose slow zone meets the span: exactly the points pass 1 masked out
// (t < t_z on the same rounded t, inside the window), with the full FP32 Faddeeva forms.
// A zone of |z| < 6.5 takes the core forms at every point (rox_re_w_core holds 9e-6 out to
// |z| = 7.1); on a uniform grid the lanes then take consecutive points of the zone rather than
// aligned 32-point sub-spans (fewer, fuller warp steps). Otherwise, per 32-point sub-span, one
// form for all points where possible: the 3-level fraction if even the sub-span's point nearest
// the centre has |z| >= 10, the 5-level one if |z| >= 6 there (both only get more accurate
// further out), else rox_re_w per point. Accumulated into the warp's shared-memory row zacc
// (one add per line and point; within a warp step the lanes touch distinct points).
template <bool NU>
__device__ __forceinline__ void zone_line(const Rec& rq, int Aw, int lane, float Jf, float dnu_f, const float* daw,
                                          const float2* D, float* zacc) {
  const float X0 = fmaf(Jf - rq.a.x, dnu_f, -rq.a.y);
  const int jlo = __float_as_int(rq.c.x), jhi = __float_as_int(rq.c.y);
  const int zlo = __float_as_int(rq.c.z), zhi = __float_as_int(rq.c.w);
  const int lo = max(max(zlo, jlo), Aw), hi = min(min(zhi, jhi), Aw + ROX_SPAN - 1);
  if (lo > hi) return;
  const float invG = rq.d.x, y = rq.d.y, pcore = rq.d.z;
  if (!NU && rq.d.w != 0.0f) {
    // lanes on consecutive points of [lo, hi]; t rounded exactly as pass 1 rounds it
    for (int k = lane; k <= hi - lo; k += 32) {
      const int q = lo - Aw + k;
      const float X0q = fmaf((float)(Aw + (q & 31)) - rq.a.x, dnu_f, -rq.a.y);
      const float Xm = fmaf((float)(q & ~31), dnu_f, X0q);
      const float t = fmaf(Xm, Xm, rq.a.z);
      if (!(t < rq.b.w)) continue;
      const float X = fmaf((float)(Aw + q) - rq.a.x, dnu_f, -rq.a.y);
      zacc[q] += pcore * rox_re_w_core(daw, fabsf(X) * invG, y);
    }
    return;
  }
  if (rq.d.w != 0.0f) {
    for (int m = (lo - Aw) >> 5; m <= ((hi - Aw) >> 5); m++) {
      const int j = Aw + 32 * m + lane;
      const float Xm = pos<NU>(m, X0, rq.a, D, dnu_f);
      const float t = fmaf(Xm, Xm, rq.a.z);
      if (!(t < rq.b.w) || j < jlo || j > jhi) continue;
      // the uniform grid recomputes X from the index in one rounding; node offsets are exact already
      const float X = NU ? Xm : fmaf((float)j - rq.a.x, dnu_f, -rq.a.y);
      zacc[32 * m + lane] += pcore * rox_re_w_core(daw, fabsf(X) * invG, y);
    }
    return;
  }
  const float centre = rq.a.x + rq.a.y / dnu_f;     // k0 + f, within 0.25 grid steps (uniform grid)
  const float y2 = y * y;
  for (int m = (lo - Aw) >> 5; m <= ((hi - Aw) >> 5); m++) {
    const int am = Aw + 32 * m, bm = am + 31;
    const int j = am + lane;
    const float Xm = pos<NU>(m, X0, rq.a, D, dnu_f);
    const float t = fmaf(Xm, Xm, rq.a.z);
    float xm;   // |X| of the sub-span's point nearest the line centre, in units of gamma_G
    if constexpr (NU) {
      const float Xa = __shfl_sync(0xffffffffu, Xm, 0), Xb = __shfl_sync(0xffffffffu, Xm, 31);
      xm = (Xa <= 0.0f && Xb >= 0.0f ? 0.0f : fminf(fabsf(Xa), fabsf(Xb))) * invG;
    } else {
      const float dc = (centre >= (float)am && centre <= (float)bm)
                           ? 0.0f : fminf(fabsf((float)am - centre), fabsf((float)bm - centre));
      xm = fmaxf(dc - 1.0f, 0.0f) * dnu_f * invG;
    }
    if (!(t < rq.b.w) || j < jlo || j > jhi) continue;
    const float sm = fmaf(xm, xm, y2);
    const float X = NU ? Xm : fmaf((float)j - rq.a.x, dnu_f, -rq.a.y);
    const float x = fabsf(X) * invG;
    float r;
    if (sm >= ROX_S_CF3) r = rox_re_w_cf3(x, y);
    else if (sm >= ROX_S_CF5) r = rox_re_w_cf5g(x, y);
    else r = rox_re_w(daw, x, y);
    zacc[32 * m + lane] += pcore * r;
  }
}

// NU: the lists are on user-provided nodes (node offsets in dynamic shared memory, one
// ROX_SPAN row of float2 per warp). X: ROX_VX_INDEX (each list is a subset of the sorted lines,
// given by RoxListDev::idx, e.g. the kept lines of a main-contributor selection; span ranges
// then count positions in that index) and ROX_VX_BROAD (widths from the broadening pass). Each
// extra is compiled only into the instantiations that use it: in this kernel even a few added
// instructions per line batch cost several percent of the plain launch.
template <bool NU, int X>
__global__ void __launch_bounds__(ROX_THREADS, 3) k_voigt(const __grid_constant__ RoxVoigtArgs A) {
  constexpr bool IDX = (X & ROX_VX_INDEX) != 0;
  constexpr bool BRD = (X & ROX_VX_BROAD) != 0;
  extern __shared__ float2 s_nodes[];
  __shared__ float4 s_geo[ROX_WARPS][2][32];
  __shared__ float s_S[ROX_WARPS][2][32];
  __shared__ Rec s_rec[ROX_WARPS][32];
  __shared__ float s_zacc[ROX_WARPS][ROX_SPAN];
  __shared__ float s_tot[ROX_WARPS][ROX_SPAN];    // the span's sum over its parts
  __shared__ float s_daw[ROX_NDAW];
  __shared__ int s_status;

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  for (int i = tid; i < ROX_NDAW; i += ROX_THREADS) s_daw[i] = (&rox_daw_taylor[0][0])[i];
  if (tid == 0) s_status = *(volatile int32_t*)&A.hdr->status;
  __syncthreads();
  if (s_status != ROX_OK) return;   // e.g. unsorted input: leave sigma untouched

  float4(*geo_st)[32] = s_geo[w];
  float(*S_st)[32] = s_S[w];
  Rec* rec = s_rec[w];
  float* zacc = s_zacc[w];
  float* stot = s_tot[w];
  float2* Drow = NU ? s_nodes + w * ROX_SPAN : nullptr;   // this span's node offsets
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
    const float dnu_f = Lst.dnu_f;
    // offsets on a uniform grid round once more (X0 + 32 m dnu), hence the precision margin
    const float margin_cm = NU ? 0.0f : ROX_FAST_MARGIN * 32.0f * (ROX_K - 1) * dnu_f;
    const int Aw = span * ROX_SPAN;
    const int Bw = Aw + ROX_SPAN - 1;
    const float Jf = (float)(Aw + lane);
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
        cp_async4(&S_st[0][lane], &S_row[li]);
        load_widths<BRD>(J, Lst, f16, li, gref, nt);
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
          cp_async4(&S_st[buf ^ 1][lane], &S_row[li]);
          load_widths<BRD>(J, Lst, f16, li, gref_n, nt_n);
        }
        if (IDX && b0 + 64 + lane < phi) li_n = Lst.idx[b0 + 64 + lane];
        cp_async_commit();
        cp_async_wait1();   // this lane's copies of the current batch have landed

        // ---- per-line constants (lane <-> line b0 + lane)
        Rec r;
        if (lane < cnt) {
          const float4 g = geo_st[buf][lane];
          const float Sp = S_st[buf][lane];
          const int jlo = __float_as_int(g.z), jhi = __float_as_int(g.w);
          float nu0f, ax, ay;   // line centre; its offset state {k0, f dnu} or {c hi, c lo}
          if constexpr (NU) {
            // c = nu0 - (span's first node) as a double-float pair (the hi parts cancel exactly)
            nu0f = g.x;
            const float ch = g.x - bh, cl = g.y - bl;
            ax = ch + cl;
            ay = cl - (ax - ch);
          } else {
            nu0f = Lst.nu_min_f + fmaf(g.x, dnu_f, g.y);
            ax = g.x;
            ay = g.y;
          }
          const float gG = nu0f * J.gG_fac;
          const float gL = BRD ? fmaf(gref, J.p_fac, nt) : gref * exp2f(nt * J.l2_ratio) * J.p_fac;
          const long long ov = min((long long)jhi, whi) - max((long long)jlo, wlo) + 1;
          if (ov > 0) evals += (unsigned long long)ov;
          const float gG2 = gG * gG, gL2 = gL * gL;
          const float pY = Sp * gL * ROX_INV_PI;
          const float invG = 1.0f / gG;
          const float yv = gL * invG;
          const rox_far fc = rox_far_coefs(yv);      // far-zone form of this line (rox_faddeeva.cuh)
          // slow zone: |X| < sqrt(r2 gamma_G^2 - gamma_L^2), at least the precision margin
          float hz = sqrtf(fmaxf(0.0f, fc.r2 * gG2 - gL2));
          // zone |z| < 6.5 not widened by the margin: the core forms cover all of it
          const bool core_only = fc.r2 == ROX_S_PADE && hz >= margin_cm;
          hz = fmaxf(hz, margin_cm);
          int zlo, zhi;
          bool zoned;
          if constexpr (NU) {
            // the span's offsets run from -c to Ws - c; pass 2 then scans the window itself
            const float hzp = hz * 1.001f + 1e-6f * (fabsf(ax) + Ws);
            zoned = -ax < hzp && Ws - ax > -hzp;
            zlo = jlo;
            zhi = jhi;
          } else {
            const int k0 = (int)g.x;
            const float hzg = fminf(hz / dnu_f * 1.0001f, 8.0e6f);
            const float f = g.y / dnu_f;
            zlo = k0 + (int)floorf(f - hzg) - 1;
            zhi = k0 + (int)ceilf(f + hzg) + 1;
            zoned = !(Bw < zlo || Aw > zhi);
          }
          const bool covers = Aw >= jlo && Bw <= jhi;
          const float vg = fc.alpha * gG2;
          r.a = make_float4(ax, ay, vg, fc.beta * (gG2 * gG2));
          r.b = make_float4(pY, pY * (fc.kappa * gG2), __uint_as_float((covers ? 1u : 0u) | (zoned ? 2u : 0u)),
                            fmaf(hz, hz, vg));
          r.c = make_float4(g.z, g.w, __int_as_float(zlo), __int_as_float(zhi));
          r.d = make_float4(invG, yv, Sp * invG * ROX_INV_SQRT_PI, core_only ? 1.0f : 0.0f);
        } else {   // padding record: contributes nothing
          r.a = make_float4(0.f, 0.f, 1.f, 0.f);
          r.b = make_float4(0.f, 0.f, __uint_as_float(0u), 0.f);
          r.c = make_float4(__int_as_float(1), __int_as_float(0), __int_as_float(0), __int_as_float(0));
          r.d = make_float4(1.f, 0.f, 0.f, 0.f);
        }
        rec[lane] = r;
        gref = gref_n;
        nt = nt_n;
        __syncwarp();

        // ---- pass 1: far formula. Clean lines (window covers the span, no slow zone in it) in
        // unmasked pairs; covering lines with a slow zone in masked pairs; window-edge lines in
        // pairs with window masks. The orders are fixed, so the sum is reproducible.
        const unsigned cls = __float_as_uint(r.b.z);
        const bool live = lane < cnt;
        unsigned cmask = __ballot_sync(0xffffffffu, live && cls == 1u);
        unsigned zmask = __ballot_sync(0xffffffffu, live && cls == 3u);
        const unsigned emask = __ballot_sync(0xffffffffu, live && !(cls & 1u));
        const unsigned pmask = __ballot_sync(0xffffffffu, live && (cls & 2u));
        while (cmask) {
          const int i0 = __ffs(cmask) - 1;
          cmask &= cmask - 1;
          const float4 a0 = rec[i0].a, b0v = rec[i0].b;
          const float X0 = fmaf(Jf - a0.x, dnu_f, -a0.y);
          if (cmask) {
            const int i1 = __ffs(cmask) - 1;
            cmask &= cmask - 1;
            const float4 a1 = rec[i1].a, b1v = rec[i1].b;
            const float X1 = fmaf(Jf - a1.x, dnu_f, -a1.y);
#pragma unroll
            for (int m = 0; m < ROX_K; m++) {
              const float x0 = pos<NU>(m, X0, a0, D, dnu_f);
              const float x1 = pos<NU>(m, X1, a1, D, dnu_f);
              const float t0 = fmaf(x0, x0, a0.z), t1 = fmaf(x1, x1, a1.z);
              const float d0 = fmaf(t0, t0, a0.w), d1 = fmaf(t1, t1, a1.w);
              const float n0 = fmaf(t0, b0v.x, b0v.y), n1 = fmaf(t1, b1v.x, b1v.y);
              const float dd = d0 * d1;
              const float nn = fmaf(n1, d0, n0 * d1);
              acc[m] = fmaf(nn, rox_rcp(dd), acc[m]);
            }
          } else {
#pragma unroll
            for (int m = 0; m < ROX_K; m++) acc[m] += far_term(pos<NU>(m, X0, a0, D, dnu_f), a0, b0v);
          }
        }
        while (zmask) {
          const int i0 = __ffs(zmask) - 1;
          zmask &= zmask - 1;
          const float4 a0 = rec[i0].a, b0v = rec[i0].b;
          const float X0 = fmaf(Jf - a0.x, dnu_f, -a0.y);
          if (zmask) {
            const int i1 = __ffs(zmask) - 1;
            zmask &= zmask - 1;
            const float4 a1 = rec[i1].a, b1v = rec[i1].b;
            const float X1 = fmaf(Jf - a1.x, dnu_f, -a1.y);
#pragma unroll
            for (int m = 0; m < ROX_K; m++) {
              const float x0 = pos<NU>(m, X0, a0, D, dnu_f);
              const float x1 = pos<NU>(m, X1, a1, D, dnu_f);
              const float t0 = fmaf(x0, x0, a0.z), t1 = fmaf(x1, x1, a1.z);
              const bool f0 = t0 >= b0v.w, f1 = t1 >= b1v.w;   // outside the slow zone
              const float d0 = f0 ? fmaf(t0, t0, a0.w) : 1.0f, d1 = f1 ? fmaf(t1, t1, a1.w) : 1.0f;
              const float n0 = f0 ? fmaf(t0, b0v.x, b0v.y) : 0.0f;
              const float n1 = f1 ? fmaf(t1, b1v.x, b1v.y) : 0.0f;
              const float dd = d0 * d1;
              const float nn = fmaf(n1, d0, n0 * d1);
              acc[m] = fmaf(nn, rox_rcp(dd), acc[m]);
            }
          } else {
#pragma unroll
            for (int m = 0; m < ROX_K; m++) acc[m] += masked_far(pos<NU>(m, X0, a0, D, dnu_f), a0, b0v);
          }
        }
        for (unsigned em = emask; em;) {
          const int i0 = __ffs(em) - 1;
          em &= em - 1;
          if (!em) {
            edge_line<NU>(rec[i0].a, rec[i0].b, rec[i0].c, Aw, lane, Jf, dnu_f, D, acc);
            break;
          }
          const int i1 = __ffs(em) - 1;
          em &= em - 1;
          edge_pair<NU>(rec[i0], rec[i1], Aw, lane, Jf, dnu_f, D, acc);
        }
        // ---- pass 2: the points each zoned line left out of pass 1, full Faddeeva forms
        for (unsigned pm = pmask; pm; pm &= pm - 1) {
          const Rec rq = rec[__ffs(pm) - 1];
          zone_line<NU>(rq, Aw, lane, Jf, dnu_f, s_daw, D, zacc);
        }
        __syncwarp();
        // compensated (Kahan) accumulation of the partial sums, every 4 batches
        if ((nb & 3) == 3 || b0 + 32 >= phi) {
#pragma unroll
          for (int m = 0; m < ROX_K; m++) {
            const float yk = acc[m] - cmp[m];
            const float tk = tot[m] + yk;
            cmp[m] = (tk - tot[m]) - yk;
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
        cmp[m] = (tk - tot[m]) - yk;
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
    // ---- write the span once (its part inside the job's window)
    float* out = J.sigma - J.first;
#pragma unroll
    for (int m = 0; m < ROX_K; m++) {
      const long long j = (long long)Aw + 32 * m + lane;
      if (j >= wlo && j <= whi) {
        const float v = ldexpf(stot[32 * m + lane], e);
        out[j] = (J.flags & ROX_ACCUMULATE) ? out[j] + v : v;
      }
    }
    __syncwarp();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, o);
  if (lane == 0 && evals) atomicAdd(&A.hdr->evals_total, evals);
}

__global__ void k_faddeeva(const float* x, const float* y, float* out, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = rox_re_w(&rox_daw_taylor[0][0], x[i], y[i]);
}

}  // namespace

#define ROX_NODES_SMEM (ROX_WARPS * ROX_SPAN * sizeof(float2))

cudaError_t rox_launch_voigt(const RoxVoigtArgs& A, int n_blocks, bool nodes, int extras, cudaStream_t s) {
  if (nodes) {
    if (extras) return cudaErrorNotSupported;   // no caller combines nodes with a selection or broadening
    // static shared memory plus the node rows exceed 48 KB: opt in (idempotent, per device)
    cudaError_t e = cudaFuncSetAttribute(k_voigt<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ROX_NODES_SMEM);
    if (e != cudaSuccess) return e;
    k_voigt<true, 0><<<n_blocks, ROX_THREADS, ROX_NODES_SMEM, s>>>(A);
  } else if (extras == 0) {
    k_voigt<false, 0><<<n_blocks, ROX_THREADS, 0, s>>>(A);
  } else if (extras == ROX_VX_INDEX) {
    k_voigt<false, ROX_VX_INDEX><<<n_blocks, ROX_THREADS, 0, s>>>(A);
  } else if (extras == ROX_VX_BROAD) {
    k_voigt<false, ROX_VX_BROAD><<<n_blocks, ROX_THREADS, 0, s>>>(A);
  } else {
    return cudaErrorNotSupported;   // no entry point combines an indexed list with broadening
  }
  return cudaGetLastError();
}

cudaError_t rox_voigt_blocks_per_sm(int* nb, bool nodes) {
  if (nodes) {
    cudaError_t e = cudaFuncSetAttribute(k_voigt<true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)ROX_NODES_SMEM);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_voigt<true, 0>, ROX_THREADS, ROX_NODES_SMEM);
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_voigt<false, 0>, ROX_THREADS, 0);
}

cudaError_t rox_launch_faddeeva(const float* x, const float* y, float* out, long long n, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_faddeeva<<<(int)b, 256, 0, s>>>(x, y, out, n);
  return cudaGetLastError();
}
