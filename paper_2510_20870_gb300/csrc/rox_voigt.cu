// a4 / a5: Voigt evaluation and accumulation onto the wavenumber grid, for every (P,T).
// pyROX paper, "Compute line profiles" (Voigt = Re of the Faddeeva function, Gandhi et al.
// 2020 Eq. 12) and "Combine and save" (profiles summed into a cross-section per
// temperature-pressure point).
//
// Persistent kernel over (point, tile) work items taken from an atomic counter. A CTA owns
// one tile of ROX_TILE consecutive grid points in registers (each thread ROX_K points strided
// by 32, so a warp covers 32*ROX_K consecutive points) and streams the lines that reach the
// tile (a contiguous range of the nu0-sorted list) through shared memory in chunks of
// ROX_CHUNK lines, staged with cp.async one chunk ahead. Each chunk is first turned into
// per-line constants (one thread per line), then every warp walks the chunk's lines in
// order. The tile is written once at the end, so the summation order is fixed.
//
// Work per (line, point) pair, in physical units X = nu_j - nu0, Y = gamma_L,
// G = gamma_G^2 / 2: outside a per-line slow zone (x^2 + y^2 >= 22^2) the 2-level continued
// fraction gives S V = (S Y / pi)(t + 2G) / (t^2 + 4 G Y^2) with t = X^2 + Y^2 - G, i.e.
// 4 FMAs and one reciprocal; two lines share one reciprocal (n1/d1 + n2/d2 =
// (n1 d2 + n2 d1)/(d1 d2)), so a pair costs 12 FP32 operations and one MUFU per point.
// Points in the slow zone or at a window edge go to the full FP32 Faddeeva evaluation
// (rox_faddeeva.cuh), chosen per 32-point sub-span so that the branch is warp-uniform.
#include <cuda_fp16.h>
#include "rox_internal.cuh"
#include "rox_faddeeva.cuh"

namespace {

#define ROX_NDAW (ROX_DAW_NODES * (ROX_DAW_DEG + 1))
#define ROX_INV_PI 0.318309886183790672f

// Per-line constants of one (P,T) point, one record per staged line:
//   a = {k0 (exact float), f*dnu, Y^2 - G, 4 G Y^2}
//   b = {S Y / pi, (S Y / pi) * 2G, warp masks (bits 0-7: line meets warp, 8-15: fast), 0}
//   c = {jlo, jhi, zlo, zhi} (int bits; window and slow zone, inclusive grid indices)
//   d = {1/gamma_G, y = gamma_L/gamma_G, S/(gamma_G sqrt(pi)), 0}
// S is scaled by 2^-e (e the exponent of the largest strength at this temperature).
struct __align__(16) Rec {
  float4 a, b, c, d;
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ float load_width(const void* p, int f16, long long i) {
  return f16 ? __half2float(reinterpret_cast<const __half*>(p)[i])
             : reinterpret_cast<const float*>(p)[i];
}

// one point of one line outside the slow zone: S V = n / d
__device__ __forceinline__ float far_term(float X, const float4& a, const float4& b) {
  float t = fmaf(X, X, a.z);
  float d = fmaf(t, t, a.w);
  float n = fmaf(t, b.x, b.y);
  return n * rox_rcp(d);
}

// a point handled individually: window test, slow-zone test, then the far formula or the
// full Faddeeva evaluation (per-thread branches; used only where a sub-span is mixed)
__device__ __noinline__ float general_point(int j, Rec r, float dnu_f, const float* daw) {
  int jlo = __float_as_int(r.c.x), jhi = __float_as_int(r.c.y);
  if (j < jlo || j > jhi) return 0.0f;
  float X = fmaf((float)j - r.a.x, dnu_f, -r.a.y);
  int zlo = __float_as_int(r.c.z), zhi = __float_as_int(r.c.w);
  if (j < zlo || j > zhi) return far_term(X, r.a, r.b);
  return r.d.z * rox_re_w(daw, X * r.d.x, r.d.y);
}

__global__ void __launch_bounds__(ROX_THREADS, 2) k_voigt(const __grid_constant__ RoxVoigtArgs A) {
  __shared__ float4 s_geo[2][ROX_CHUNK];
  __shared__ double s_S[2][ROX_CHUNK];
  __shared__ Rec s_rec[ROX_CHUNK];
  __shared__ float s_daw[ROX_NDAW];
  __shared__ int s_item;

  const int tid = threadIdx.x;
  const int lane = tid & 31, w = tid >> 5;
  const unsigned bit_in = 1u << w, bit_fast = 1u << (8 + w);
  for (int i = tid; i < ROX_NDAW; i += ROX_THREADS) s_daw[i] = (&rox_daw_taylor[0][0])[i];
  if (tid == 0) s_item = *(volatile int32_t*)&A.hdr->status;
  __syncthreads();
  if (s_item != ROX_OK) return;   // e.g. unsorted input: leave sigma untouched
  if (blockIdx.x == 0 && tid == 0) A.hdr->evals_total = A.hdr->evals_lines * (unsigned long long)A.n_pt;

  const int f16 = A.width_f16;
  const float dnu_f = A.dnu_f;
  const float margin_cm = ROX_FAST_MARGIN * 32.0f * (ROX_K - 1) * dnu_f;
  const long long n_items = (long long)A.n_pt * A.n_tiles;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(&A.hdr->work_counter, 1);
    __syncthreads();
    const long long item = s_item;
    if (item >= n_items) break;
    const int pt = (int)(item / A.n_tiles);
    const int tile = A.n_tiles - 1 - (int)(item % A.n_tiles);   // wide-line (high nu) tiles first
    const RoxPt P = A.pt[pt];
    const int base = tile * ROX_TILE;
    const int Aw = base + w * 32 * ROX_K;
    const float Jf = (float)(Aw + lane);
    const long long lo = A.tile_lo[tile], hi = A.tile_hi[tile];
    const double smax = __longlong_as_double((long long)A.hdr->smax_bits[P.t_idx]);
    const int e = smax > 0.0 ? ilogb(smax) : 0;
    const double sscale = ldexp(1.0, -e);
    const double* S_row = A.S_T + (long long)P.t_idx * A.n_lines;

    float acc[ROX_K], tot[ROX_K], cmp[ROX_K];
#pragma unroll
    for (int m = 0; m < ROX_K; m++) { acc[m] = 0.f; tot[m] = 0.f; cmp[m] = 0.f; }

    const long long nch = (hi - lo + ROX_CHUNK - 1) / ROX_CHUNK;
    if (nch > 0 && lo + tid < hi) {
      cp_async16(&s_geo[0][tid], &A.geo[lo + tid]);
      cp_async8(&s_S[0][tid], &S_row[lo + tid]);
    }
    cp_async_commit();
    for (long long ch = 0; ch < nch; ch++) {
      const long long c0 = lo + ch * ROX_CHUNK;
      const int cnt = (int)min((long long)ROX_CHUNK, hi - c0);
      const int buf = (int)(ch & 1);
      if (ch + 1 < nch && c0 + ROX_CHUNK + tid < hi) {
        cp_async16(&s_geo[buf ^ 1][tid], &A.geo[c0 + ROX_CHUNK + tid]);
        cp_async8(&s_S[buf ^ 1][tid], &S_row[c0 + ROX_CHUNK + tid]);
      }
      cp_async_commit();
      cp_async_wait1();   // this thread's copies of chunk ch have landed

      // ---- per-line constants (thread tid <-> line c0 + tid)
      Rec r;
      unsigned masks = 0;
      if (tid < cnt) {
        const long long i = c0 + tid;
        const float4 g = s_geo[buf][tid];
        const float Sp = (float)(s_S[buf][tid] * sscale);
        const float gref = load_width(A.gamma_ref, f16, i);
        const float nt = load_width(A.n_t, f16, i);
        const int jlo = __float_as_int(g.z), jhi = __float_as_int(g.w);
        const int k0 = (int)g.x;
        const float nu0f = A.nu_min_f + fmaf(g.x, dnu_f, g.y);
        const float gG = nu0f * P.gG_fac;
        const float gL = gref * exp2f(nt * P.l2_ratio) * P.p_fac;
        const float gG2 = gG * gG, gL2 = gL * gL;
        const float pY = Sp * gL * ROX_INV_PI;
        const float invG = 1.0f / gG;
        r.a = make_float4(g.x, g.y, fmaf(-0.5f, gG2, gL2), 2.0f * gG2 * gL2);
        r.d = make_float4(invG, gL * invG, Sp * invG * ROX_INV_SQRT_PI, 0.f);
        // slow zone: |X| < sqrt(22^2 gamma_G^2 - gamma_L^2), at least the precision margin
        float hz = sqrtf(fmaxf(0.0f, (float)ROX_FAR_Z2 * gG2 - gL2));
        hz = fmaxf(hz, margin_cm);
        float hzg = fminf(hz / dnu_f * 1.0001f, 8.0e6f);
        const float f = g.y / dnu_f;
        const int zlo = k0 + (int)floorf(f - hzg) - 1;
        const int zhi = k0 + (int)ceilf(f + hzg) + 1;
        r.c = make_float4(g.z, g.w, __int_as_float(zlo), __int_as_float(zhi));
#pragma unroll
        for (int v = 0; v < ROX_WARPS; v++) {
          const int av = base + v * 32 * ROX_K, bv = av + 32 * ROX_K - 1;
          const bool meets = jhi >= av && jlo <= bv;
          const bool fast = meets && av >= jlo && bv <= jhi && (bv < zlo || av > zhi);
          masks |= (meets ? 1u << v : 0u) | (fast ? 1u << (8 + v) : 0u);
        }
        r.b = make_float4(pY, pY * gG2, __uint_as_float(masks), 0.f);
      } else {
        r.a = make_float4(0.f, 0.f, 1.f, 0.f);
        r.b = make_float4(0.f, 0.f, __uint_as_float(0u), 0.f);
        r.c = make_float4(__int_as_float(1), __int_as_float(0), __int_as_float(0), __int_as_float(0));
        r.d = make_float4(1.f, 0.f, 0.f, 0.f);
      }
      s_rec[tid] = r;
      __syncthreads();

      // ---- evaluation: lines in pairs, warp-uniform fast/slow decisions
      for (int i = 0; i < cnt; i += 2) {
        const float4 a0 = s_rec[i].a, b0 = s_rec[i].b;
        const float4 a1 = s_rec[i + 1].a, b1 = s_rec[i + 1].b;
        const unsigned m0 = __float_as_uint(b0.z), m1 = __float_as_uint(b1.z);
        if (m0 & m1 & bit_fast) {
          const float X0 = fmaf(Jf - a0.x, dnu_f, -a0.y);
          const float X1 = fmaf(Jf - a1.x, dnu_f, -a1.y);
#pragma unroll
          for (int m = 0; m < ROX_K; m++) {
            const float x0 = fmaf((float)(32 * m), dnu_f, X0);
            const float x1 = fmaf((float)(32 * m), dnu_f, X1);
            const float t0 = fmaf(x0, x0, a0.z), t1 = fmaf(x1, x1, a1.z);
            const float d0 = fmaf(t0, t0, a0.w), d1 = fmaf(t1, t1, a1.w);
            const float n0 = fmaf(t0, b0.x, b0.y), n1 = fmaf(t1, b1.x, b1.y);
            const float dd = d0 * d1;
            const float nn = fmaf(n1, d0, n0 * d1);
            acc[m] = fmaf(nn, rox_rcp(dd), acc[m]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 2; q++) {
            const unsigned mq = q ? m1 : m0;
            if (!(mq & bit_in)) continue;
            const Rec r = s_rec[i + q];
            const float X0 = fmaf(Jf - r.a.x, dnu_f, -r.a.y);
            if (mq & bit_fast) {
#pragma unroll
              for (int m = 0; m < ROX_K; m++)
                acc[m] += far_term(fmaf((float)(32 * m), dnu_f, X0), r.a, r.b);
            } else {
              const int jlo = __float_as_int(r.c.x), jhi = __float_as_int(r.c.y);
              const int zlo = __float_as_int(r.c.z), zhi = __float_as_int(r.c.w);
#pragma unroll
              for (int m = 0; m < ROX_K; m++) {
                const int am = Aw + 32 * m, bm = am + 31;
                if (bm < jlo || am > jhi) continue;
                if (am >= jlo && bm <= jhi && (bm < zlo || am > zhi))
                  acc[m] += far_term(fmaf((float)(32 * m), dnu_f, X0), r.a, r.b);
                else
                  acc[m] += general_point(am + lane, r, dnu_f, s_daw);
              }
            }
          }
        }
      }
      // compensated (Kahan) accumulation of the chunk partial sums
#pragma unroll
      for (int m = 0; m < ROX_K; m++) {
        const float yk = acc[m] - cmp[m];
        const float tk = tot[m] + yk;
        cmp[m] = (tk - tot[m]) - yk;
        tot[m] = tk;
        acc[m] = 0.f;
      }
      __syncthreads();
    }
    // ---- write the tile once
    float* out = A.sigma + (long long)pt * A.n_grid;
#pragma unroll
    for (int m = 0; m < ROX_K; m++) {
      const long long j = (long long)Aw + 32 * m + lane;
      if (j < A.n_grid) {
        const float v = ldexpf(tot[m], e);
        out[j] = (A.flags & ROX_ACCUMULATE) ? out[j] + v : v;
      }
    }
  }
}

__global__ void k_faddeeva(const float* x, const float* y, float* out, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = rox_re_w(&rox_daw_taylor[0][0], x[i], y[i]);
}

}  // namespace

cudaError_t rox_launch_voigt(const RoxVoigtArgs& A, int n_blocks, cudaStream_t s) {
  k_voigt<<<n_blocks, ROX_THREADS, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t rox_voigt_blocks_per_sm(int* nb) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, k_voigt, ROX_THREADS, 0);
}

cudaError_t rox_launch_faddeeva(const float* x, const float* y, float* out, long long n, cudaStream_t s) {
  long long b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  k_faddeeva<<<(int)b, 256, 0, s>>>(x, y, out, n);
  return cudaGetLastError();
}
