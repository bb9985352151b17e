// a1 / a2: per-line strength S(T) and widths gamma_G, gamma_L.
// pyROX paper, "Functionality of pyROX" -- "Compute line-strengths and -widths": the
// strength and broadening widths of every transition at the user's pressure and
// temperature. Each thread reads one line's SoA entries (coalesced) and writes its outputs.
// The strength exists in two forms: the full FP64 one (line_strength), and for the
// cross-section launches a reduced one (line_strength_fast) that keeps only the Boltzmann
// exponent and its reduction in FP64. This GPU's FP64 rate, not the bytes, bounds these
// kernels.
#include <cuda_fp16.h>
#include "rox_internal.cuh"

namespace {

__device__ __forceinline__ float load_width(const void* p, int f16, long long i) {
  return f16 ? __half2float(reinterpret_cast<const __half*>(p)[i])
             : reinterpret_cast<const float*>(p)[i];
}

struct StrengthConsts {
  int convention;
  double inv_T;        // 1/T
  double q_ratio;      // HITRAN: Q_ref/Q_T ; ExoMol: 1/Q_T
  double c2_dT;        // HITRAN: c2 (1/T - 1/T_ref) ; ExoMol: c2/T
};

// S(T) in FP64 for one line (HITRAN S_ref form or ExoMol Einstein-A form).
__device__ __forceinline__ double line_strength(const StrengthConsts& k, double nu0, double s_or_a,
                                                double g_up, double e_lower) {
  double stim_T = -expm1(-ROX_C2 * nu0 * k.inv_T);           // 1 - exp(-c2 nu0 / T)
  double boltz = exp(-e_lower * k.c2_dT);
  if (k.convention == ROX_HITRAN) {
    double stim_ref = -expm1(-ROX_C2 * nu0 / ROX_T_REF);
    return s_or_a * k.q_ratio * boltz * (stim_T / stim_ref);
  }
  return g_up * s_or_a / (8.0 * ROX_PI * ROX_C_CM * nu0 * nu0) * boltz * stim_T * k.q_ratio;
}

// The same S(T) with few FP64 operations, for the cross-section launches (this GPU runs
// FP64 at about two operations per clock per SM, and FP64 exp, expm1 and a division cost
// ~70 of them per line). Only the Boltzmann exponent needs FP64 range and accuracy: it is
// formed in FP64 and split as a = k ln 2 + r (Cody and Waite's reduction with ln 2 in two
// parts; the high part has 33 significant bits, so k * hi is exact for |k| < 2^20),
// |r| <= ln(2)/2. exp(r), the stimulated-emission factor and the prefactor are FP32, and the
// FP32 product (pre-scaled by 2^64 against underflow) is put back in range by the exact
// powers 2^-64 and 2^k in FP64. Relative error a few 1e-7 (FP32 roundings), far below the
// cross-section tolerance; exponents beyond +-700 and FP32 products beyond 2^+-100 (or zero,
// or NaN) take the FP64 form.
#define ROX_LN2_HI 0.6931471804855391       // ln 2 rounded to 33 significant bits
#define ROX_LN2_LO 7.440617110012397e-11    // ln 2 - ROX_LN2_HI
#define ROX_LOG2E 1.4426950408889634        // 1 / ln 2
__device__ __forceinline__ double line_strength_fast(const StrengthConsts& k, double nu0, float s_or_a, float g_up,
                                                     float e_lower) {
  const double a = -(double)e_lower * k.c2_dT;
  if (!(fabs(a) < 700.0)) return line_strength(k, nu0, (double)s_or_a, (double)g_up, (double)e_lower);
  const double kd = rint(a * ROX_LOG2E);
  const double r = fma(-kd, ROX_LN2_LO, fma(-kd, ROX_LN2_HI, a));
  const float m = expf((float)r);
  const float nu = (float)nu0;
  const float stim = -expm1f(-(float)(ROX_C2 * k.inv_T) * nu);
  float p;
  if (k.convention == ROX_HITRAN) {
    const float stim_ref = -expm1f(-(float)(ROX_C2 / ROX_T_REF) * nu);
    p = (s_or_a * 0x1p64f) * (float)k.q_ratio * (stim / stim_ref);
  } else {
    p = (g_up * s_or_a) * ((float)(0x1p64 / (8.0 * ROX_PI * ROX_C_CM)) / (nu * nu)) * stim * (float)k.q_ratio;
  }
  const float pm = p * m;
  if (!(fabsf(pm) >= 0x1p-100f && fabsf(pm) <= 0x1p100f))   // outside FP32's comfortable range (or 0, NaN)
    return line_strength(k, nu0, (double)s_or_a, (double)g_up, (double)e_lower);
  const double two_k = __longlong_as_double((long long)((int)kd + 1023) << 52);   // 2^k, |k| <= 1010
  return (double)pm * 0x1p-64 * two_k;
}

__global__ void k_strengths(rox_lines L, StrengthConsts k, float* S_out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
    double g = (L.convention == ROX_EXOMOL) ? (double)L.g_up[i] : 1.0;
    S_out[i] = (float)line_strength(k, L.nu0[i], (double)L.s_or_a[i], g, (double)L.e_lower[i]);
  }
}

// the reduced form alone, in double (rox_line_strengths_reduced: what the cross-section launches use)
__global__ void k_strengths_reduced(rox_lines L, StrengthConsts k, double* S_out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
    const float g = (L.convention == ROX_EXOMOL) ? L.g_up[i] : 1.0f;
    S_out[i] = line_strength_fast(k, L.nu0[i], L.s_or_a[i], g, L.e_lower[i]);
  }
}

__global__ void k_widths(rox_lines L, double gG_fac, float l2_ratio, float p_fac,
                         float* gG_out, float* gL_out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  int f16 = L.width_dtype == ROX_WIDTH_F16;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
    gG_out[i] = (float)(L.nu0[i] * gG_fac);
    float gref = load_width(L.gamma_ref, f16, i);
    float nt = load_width(L.n_t, f16, i);
    gL_out[i] = gref * exp2f(nt * l2_ratio) * p_fac;
  }
}

// S(T) for up to ROX_MAX_PT distinct temperatures in one launch, one sweep over the lines
// per temperature (FAST: the reduced form; either way FP64 issue, not the bytes, sets its
// cost); the per-temperature maximum (needed to
// scale S into FP32 range inside the Voigt kernel) is reduced per warp and combined with
// an atomic max on the (non-negative) double bit pattern, which is order-independent.
struct TempSet {
  int n;
  StrengthConsts k[ROX_MAX_PT];
};

template <bool FAST>
__global__ void k_strengths_multi(rox_lines L, TempSet ts,
                                  double* S_T, unsigned long long* smax_bits) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int t = 0; t < ts.n; t++) {
    double mx = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
      const float g = (L.convention == ROX_EXOMOL) ? L.g_up[i] : 1.0f;
      const double s = FAST ? line_strength_fast(ts.k[t], L.nu0[i], L.s_or_a[i], g, L.e_lower[i])
                            : line_strength(ts.k[t], L.nu0[i], (double)L.s_or_a[i], (double)g, (double)L.e_lower[i]);
      S_T[(long long)t * L.n + i] = s;
      mx = fmax(mx, s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0)
      atomicMax(&smax_bits[t], (unsigned long long)__double_as_longlong(mx));
  }
}

// S * 2^-e per temperature, e the exponent of the largest strength at that temperature,
// so the Voigt kernel works in FP32 well inside its range whatever the line strengths are.
// S * 2^-e in FP32 (e the exponent of the temperature's largest S). With a selection
// (bin != NULL): lines outside the bins, or below rel times their bin's largest S at that
// temperature (the product rounded once in double precision), get -0.0, which the Voigt kernel
// tells apart from a kept strength that rounds to +0.0 in FP32.
__global__ void k_scale_strengths(const double* __restrict__ S_T, long long n, int n_temps,
                                  const unsigned long long* __restrict__ smax_bits, float* S32,
                                  const int32_t* __restrict__ bin, const unsigned long long* __restrict__ binmax_bits,
                                  long long n_bins, double rel) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int t = 0; t < n_temps; t++) {
    double smax = __longlong_as_double((long long)smax_bits[t]);
    double sc = ldexp(1.0, smax > 0.0 ? -ilogb(smax) : 0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      const double S = S_T[(long long)t * n + i];
      bool keep = true;
      if (bin) {
        const int b = bin[i];
        keep = b >= 0 &&
               S >= __dmul_rn(rel, __longlong_as_double((long long)binmax_bits[(long long)t * n_bins + b]));
      }
      S32[(long long)t * n + i] = keep ? (float)(S * sc) : -0.0f;   // -0: dropped (+0: kept, below FP32)
    }
  }
}

// ---- a2 broadening descriptions: sum_b vmr_b gamma_b (296/T)^n_b of line i, l2 = log2(296/T)
__device__ __forceinline__ float broad_col(const void* p, int f16, long long i) {
  return f16 ? __half2float(reinterpret_cast<const __half*>(p)[i]) : reinterpret_cast<const float*>(p)[i];
}
__device__ __forceinline__ float broad_sum(const RoxBroadDev& B, long long i, float l2) {
  long long j = 0;
  if (B.j_lower) {
    j = B.j_lower[i];
    j = j < 0 ? 0 : (j >= B.tab_len ? B.tab_len - 1 : j);
  }
  float g = 0.0f;
  for (int b = 0; b < B.n_b; b++) {
    float gb, nb;
    if (B.tab_gamma[b]) {
      gb = B.tab_gamma[b][j];
      nb = B.tab_n[b][j];
    } else {
      gb = broad_col(B.gamma[b], B.f16, i);
      nb = broad_col(B.n[b], B.f16, i);
    }
    g = fmaf(B.vmr[b] * gb, exp2f(nb * l2), g);
  }
  return g;
}
#define ROX_INV_4PI_C 2.6544187294380724e-12f   // 1 / (4 pi c), c in cm/s

struct BroadTemps {
  int32_t n;
  float l2[ROX_MAX_PT];
};

// per distinct temperature the broadeners' sum of every line (G[t][i]); natural widths once
__global__ void k_broad_T(RoxBroadDev B, const float* __restrict__ a_coef, long long n, BroadTemps ts, float* G,
                          float* gN) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int t = 0; t < ts.n; t++) G[(long long)t * n + i] = broad_sum(B, i, ts.l2[t]);
    if (gN) gN[i] = a_coef[i] * ROX_INV_4PI_C;
  }
}

__global__ void k_lorentz_out(RoxBroadDev B, const float* __restrict__ a_coef, long long n, float l2, float p_fac,
                              float* out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = fmaf(broad_sum(B, i, l2), p_fac, B.natural ? a_coef[i] * ROX_INV_4PI_C : 0.0f);
}

// Main-contributor selection, bin of every line: floor((nu0 - origin) / width) with the
// subtraction and the division each rounded once in double precision; -1 outside [0, n_bins).
__global__ void k_line_bins(const double* __restrict__ nu0, long long n, double origin, double width,
                            long long n_bins, int32_t* bin) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double b = floor(__ddiv_rn(__dsub_rn(nu0[i], origin), width));
    bin[i] = (b >= 0.0 && b < (double)n_bins) ? (int32_t)b : -1;
  }
}

// Largest S per temperature and bin (as double bits; S >= 0, so the bit patterns order like
// the values). The list is sorted by nu0, so each bin is a run of lines: every thread folds
// a run of ROX_BIN_RUN consecutive lines and issues one atomic max per bin it meets.
#define ROX_BIN_RUN 16
__global__ void k_bin_max(const int32_t* __restrict__ bin, const double* __restrict__ S_T, long long n, int n_temps,
                          long long n_bins, unsigned long long* binmax_bits) {
  const long long runs = (n + ROX_BIN_RUN - 1) / ROX_BIN_RUN;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int t = 0; t < n_temps; t++) {
    const double* S = S_T + (long long)t * n;
    unsigned long long* bm = binmax_bits + (long long)t * n_bins;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < runs; r += stride) {
      const long long i0 = r * ROX_BIN_RUN, i1 = min(n, i0 + ROX_BIN_RUN);
      int cur = -1;
      double mx = 0.0;
      for (long long i = i0; i < i1; i++) {
        const int b = bin[i];
        if (b != cur) {
          if (cur >= 0) atomicMax(&bm[cur], (unsigned long long)__double_as_longlong(mx));
          cur = b;
          mx = S[i];
        } else {
          mx = fmax(mx, S[i]);
        }
      }
      if (cur >= 0) atomicMax(&bm[cur], (unsigned long long)__double_as_longlong(mx));
    }
  }
}

// Selection on reduced-form strengths (relative error below 5e-7, see line_strength_fast):
// every decision is taken as on the full FP64 strengths. A line whose reduced value is within
// ROX_SEL_EPS of its bin's reduced maximum may hold the exact maximum: its FP64 strength
// replaces the reduced one in S_T and the exact bin maxima are taken over those lines
// (k_bin_max_fix). A line within ROX_SEL_EPS of its threshold rel * (exact maximum) is decided
// on its FP64 strength; any other line lies on the same side of the threshold whichever form
// is used (k_select_scale).
#define ROX_SEL_EPS 1e-5
__global__ void k_bin_max_fix(const rox_lines L, const __grid_constant__ TempSet ts, const int32_t* __restrict__ bin,
                              double* S_T, long long n_bins, const unsigned long long* __restrict__ binmax_fast,
                              unsigned long long* binmax_exact) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int t = 0; t < ts.n; t++) {
    double* S = S_T + (long long)t * L.n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
      const int b = bin[i];
      if (b < 0) continue;
      const double mf = __longlong_as_double((long long)binmax_fast[(long long)t * n_bins + b]);
      if (!(S[i] >= mf * (1.0 - ROX_SEL_EPS))) continue;
      const double g = (L.convention == ROX_EXOMOL) ? (double)L.g_up[i] : 1.0;
      const double sx = line_strength(ts.k[t], L.nu0[i], (double)L.s_or_a[i], g, (double)L.e_lower[i]);
      S[i] = sx;
      atomicMax(&binmax_exact[(long long)t * n_bins + b], (unsigned long long)__double_as_longlong(sx));
    }
  }
}

__global__ void k_select_scale(const rox_lines L, const __grid_constant__ TempSet ts, const double* __restrict__ S_T,
                               const unsigned long long* __restrict__ smax_bits, const int32_t* __restrict__ bin,
                               const unsigned long long* __restrict__ binmax_exact, long long n_bins, double rel,
                               float* S32) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int t = 0; t < ts.n; t++) {
    const double smax = __longlong_as_double((long long)smax_bits[t]);
    const double sc = ldexp(1.0, smax > 0.0 ? -ilogb(smax) : 0);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += stride) {
      double S = S_T[(long long)t * L.n + i];
      const int b = bin[i];
      bool keep = false;
      if (b >= 0) {
        const double thr =
            __dmul_rn(rel, __longlong_as_double((long long)binmax_exact[(long long)t * n_bins + b]));
        if (fabs(S - thr) <= ROX_SEL_EPS * thr) {   // near the threshold: the FP64 form decides
          const double g = (L.convention == ROX_EXOMOL) ? (double)L.g_up[i] : 1.0;
          S = line_strength(ts.k[t], L.nu0[i], (double)L.s_or_a[i], g, (double)L.e_lower[i]);
        }
        keep = S >= thr;
      }
      S32[(long long)t * L.n + i] = keep ? (float)(S * sc) : -0.0f;   // -0: dropped (+0: kept, below FP32)
    }
  }
}

// keep flags of the first temperature: the same test as k_scale_strengths
__global__ void k_keep_flags(const double* __restrict__ S_T, const int32_t* __restrict__ bin,
                             const unsigned long long* __restrict__ binmax_bits, long long n, double rel,
                             uint8_t* keep) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int b = bin[i];
    keep[i] = b >= 0 && S_T[i] >= __dmul_rn(rel, __longlong_as_double((long long)binmax_bits[b]));
  }
}

// Per-job strengths (rox_xsec_jobs): each job's line range at its own temperature, the
// per-job maximum, then the job's FP32 scaled copy (second kernel, after the maximum is known).
__global__ void k_strengths_jobs(const __grid_constant__ RoxStrengthJobs J) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int q = 0; q < J.n_jobs; q++) {
    const RoxStrengthJob& jb = J.job[q];
    const RoxStrengthList& L = J.list[jb.list];
    StrengthConsts k;
    k.convention = L.convention;
    k.inv_T = jb.inv_T;
    k.q_ratio = jb.q_ratio;
    k.c2_dT = jb.c2_dT;
    double mx = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < jb.count; t += stride) {
      const long long i = jb.l0 + t;
      const float g = (L.convention == ROX_EXOMOL) ? L.g_up[i] : 1.0f;
      const double sv = line_strength_fast(k, L.nu0[i], L.s_or_a[i], g, L.e_lower[i]);
      jb.S64[t] = sv;
      mx = fmax(mx, sv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) atomicMax(jb.smax_bits, (unsigned long long)__double_as_longlong(mx));
  }
}

__global__ void k_scale_jobs(const __grid_constant__ RoxStrengthJobs J) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (int q = 0; q < J.n_jobs; q++) {
    const RoxStrengthJob& jb = J.job[q];
    const double smax = __longlong_as_double((long long)*jb.smax_bits);
    const double sc = ldexp(1.0, smax > 0.0 ? -ilogb(smax) : 0);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < jb.count; t += stride)
      jb.S32[t] = (float)(jb.S64[t] * sc);
  }
}

StrengthConsts make_consts(int convention, double T, double Q_T, double Q_ref) {
  StrengthConsts k;
  k.convention = convention;
  k.inv_T = 1.0 / T;
  if (convention == ROX_HITRAN) {
    k.q_ratio = Q_ref / Q_T;
    k.c2_dT = ROX_C2 * (1.0 / T - 1.0 / ROX_T_REF);
  } else {
    k.q_ratio = 1.0 / Q_T;
    k.c2_dT = ROX_C2 / T;
  }
  return k;
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace

cudaError_t rox_launch_strengths(const rox_lines* L, double T, double Q_T, double Q_ref,
                                 float* S_out, cudaStream_t s) {
  k_strengths<<<grid_for(L->n), 256, 0, s>>>(*L, make_consts(L->convention, T, Q_T, Q_ref), S_out);
  return cudaGetLastError();
}

cudaError_t rox_launch_strengths_reduced(const rox_lines* L, double T, double Q_T, double Q_ref, double* S_out,
                                         cudaStream_t s) {
  k_strengths_reduced<<<grid_for(L->n), 256, 0, s>>>(*L, make_consts(L->convention, T, Q_T, Q_ref), S_out);
  return cudaGetLastError();
}

cudaError_t rox_launch_widths(const rox_lines* L, double mass_amu, double P_bar, double T,
                              float* gG, float* gL, cudaStream_t s) {
  double gG_fac = sqrt(2.0 * ROX_KB * T / (mass_amu * ROX_AMU)) / ROX_C_M;
  float l2 = (float)log2(ROX_T_REF / T);
  float pf = (float)(P_bar / ROX_P_REF);
  k_widths<<<grid_for(L->n), 256, 0, s>>>(*L, gG_fac, l2, pf, gG, gL);
  return cudaGetLastError();
}

cudaError_t rox_launch_strengths_multi(const rox_lines* L, int n_temps, const double* temps,
                                       const double* q_of_temp, double Q_ref, double* S_T,
                                       unsigned long long* smax_bits, bool exact, cudaStream_t s) {
  TempSet ts;
  ts.n = n_temps;
  for (int t = 0; t < n_temps; t++) ts.k[t] = make_consts(L->convention, temps[t], q_of_temp[t], Q_ref);
  if (exact)
    k_strengths_multi<false><<<grid_for(L->n), 256, 0, s>>>(*L, ts, S_T, smax_bits);
  else
    k_strengths_multi<true><<<grid_for(L->n), 256, 0, s>>>(*L, ts, S_T, smax_bits);
  return cudaGetLastError();
}

void rox_fill_strength_consts(int convention, double T, double Q_T, double Q_ref, RoxStrengthJob* jb) {
  StrengthConsts k = make_consts(convention, T, Q_T, Q_ref);
  jb->inv_T = k.inv_T;
  jb->q_ratio = k.q_ratio;
  jb->c2_dT = k.c2_dT;
}

cudaError_t rox_launch_strengths_jobs(const RoxStrengthJobs& J, long long max_count, cudaStream_t s) {
  k_strengths_jobs<<<grid_for(max_count), 256, 0, s>>>(J);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_scale_jobs<<<grid_for(max_count), 256, 0, s>>>(J);
  return cudaGetLastError();
}

cudaError_t rox_launch_scale_strengths(const double* S_T, long long n, int n_temps,
                                       const unsigned long long* smax_bits, float* S32, cudaStream_t s) {
  k_scale_strengths<<<grid_for(n), 256, 0, s>>>(S_T, n, n_temps, smax_bits, S32, nullptr, nullptr, 0, 0.0);
  return cudaGetLastError();
}

cudaError_t rox_launch_select(const double* nu0, const double* S_T, long long n, int n_temps,
                              const unsigned long long* smax_bits, double origin, double width, long long n_bins,
                              double rel, int32_t* bin, unsigned long long* binmax_bits, float* S32, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(binmax_bits, 0, (size_t)n_temps * (size_t)n_bins * 8, s);
  if (e != cudaSuccess) return e;
  k_line_bins<<<grid_for(n), 256, 0, s>>>(nu0, n, origin, width, n_bins, bin);
  k_bin_max<<<grid_for((n + ROX_BIN_RUN - 1) / ROX_BIN_RUN), 256, 0, s>>>(bin, S_T, n, n_temps, n_bins, binmax_bits);
  k_scale_strengths<<<grid_for(n), 256, 0, s>>>(S_T, n, n_temps, smax_bits, S32, bin, binmax_bits, n_bins, rel);
  return cudaGetLastError();
}

// Selection for the cross-section launches, on strengths from k_strengths_multi<true> (the
// reduced form): bins, reduced maxima, exact maxima over the candidate lines, then the
// decisions and the scaled FP32 strengths (-0.0 for dropped lines).
cudaError_t rox_launch_select_reduced(const rox_lines* L, int n_temps, const double* temps, const double* q_of_temp,
                                      double Q_ref, double* S_T, const unsigned long long* smax_bits, double origin,
                                      double width, long long n_bins, double rel, int32_t* bin,
                                      unsigned long long* binmax_fast, unsigned long long* binmax_exact, float* S32,
                                      cudaStream_t s) {
  const long long n = L->n;
  cudaError_t e = cudaMemsetAsync(binmax_fast, 0, (size_t)n_temps * (size_t)n_bins * 8, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(binmax_exact, 0, (size_t)n_temps * (size_t)n_bins * 8, s)) != cudaSuccess) return e;
  TempSet ts;
  ts.n = n_temps;
  for (int t = 0; t < n_temps; t++) ts.k[t] = make_consts(L->convention, temps[t], q_of_temp[t], Q_ref);
  k_line_bins<<<grid_for(n), 256, 0, s>>>(L->nu0, n, origin, width, n_bins, bin);
  k_bin_max<<<grid_for((n + ROX_BIN_RUN - 1) / ROX_BIN_RUN), 256, 0, s>>>(bin, S_T, n, n_temps, n_bins, binmax_fast);
  k_bin_max_fix<<<grid_for(n), 256, 0, s>>>(*L, ts, bin, S_T, n_bins, binmax_fast, binmax_exact);
  k_select_scale<<<grid_for(n), 256, 0, s>>>(*L, ts, S_T, smax_bits, bin, binmax_exact, n_bins, rel, S32);
  return cudaGetLastError();
}

cudaError_t rox_launch_broad_T(const RoxBroadDev& B, const float* a_coef, long long n, int n_temps,
                               const double* temps, float* G, float* gN, cudaStream_t s) {
  BroadTemps ts;
  ts.n = n_temps;
  for (int t = 0; t < n_temps; t++) ts.l2[t] = (float)log2(ROX_T_REF / temps[t]);
  k_broad_T<<<grid_for(n), 256, 0, s>>>(B, a_coef, n, ts, G, gN);
  return cudaGetLastError();
}

cudaError_t rox_launch_lorentz_out(const RoxBroadDev& B, const float* a_coef, long long n, double P_bar, double T,
                                   float* out, cudaStream_t s) {
  k_lorentz_out<<<grid_for(n), 256, 0, s>>>(B, a_coef, n, (float)log2(ROX_T_REF / T), (float)(P_bar / ROX_P_REF),
                                            out);
  return cudaGetLastError();
}

cudaError_t rox_launch_keep_flags(const double* S_T, const int32_t* bin, const unsigned long long* binmax_bits,
                                  long long n, double rel, uint8_t* keep, cudaStream_t s) {
  k_keep_flags<<<grid_for(n), 256, 0, s>>>(S_T, bin, binmax_bits, n, rel, keep);
  return cudaGetLastError();
}
