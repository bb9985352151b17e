// Device-side twin of rox_synth's numpy line-list generator (input generation only; no step
// of the cross-section method). Philox4x32-10 (Salmon et al., SC'11) per (index, stream),
// the same 53-bit uniform and the same transforms, each operation rounded separately so the
// uniform, integer and width columns match the numpy generator bit for bit; the
// log-uniform and exponential columns go through exp/log and may differ by an FP32 ulp.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct synth_params {
  uint32_t seed;
  int32_t exomol;
  double nu_lo, nu_span;       // nu0 = nu_lo + nu_span * u
  double log_s_lo, log_s_span; // S = exp(log_s_lo + log_s_span * u)
  double el_mean;              // E'' = -el_mean * log(u)
  double gref_lo, gref_span;
  double nt_lo, nt_span;
  int32_t gup_max;
  int32_t width_f16;
};

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
  for (int r = 0; r < 10; r++) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

__device__ __forceinline__ double uniform01(uint32_t seed, uint32_t stream, uint64_t idx) {
  uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), stream, 0u};
  philox(c, seed, 0x524F5821u);
  const double a = (double)(c[0] >> 5), b = (double)(c[1] >> 6);
  return __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, 67108864.0), b), 0.5), 9007199254740992.0);
}

__global__ void k_lines(synth_params p, long long start, long long count, double* nu0, float* s_or_a, float* g_up,
                        float* e_lower, void* gref, void* nt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    const uint64_t i = (uint64_t)(start + t);
    nu0[t] = __dadd_rn(p.nu_lo, __dmul_rn(p.nu_span, uniform01(p.seed, 1, i)));
    s_or_a[t] = (float)exp(__dadd_rn(p.log_s_lo, __dmul_rn(p.log_s_span, uniform01(p.seed, 2, i))));
    if (p.exomol) g_up[t] = (float)(1.0 + floor(__dmul_rn(uniform01(p.seed, 3, i), (double)p.gup_max)));
    e_lower[t] = (float)(-p.el_mean * log(uniform01(p.seed, 4, i)));
    const double g = __dadd_rn(p.gref_lo, __dmul_rn(p.gref_span, uniform01(p.seed, 5, i)));
    const double n = __dadd_rn(p.nt_lo, __dmul_rn(p.nt_span, uniform01(p.seed, 6, i)));
    if (p.width_f16) {
      ((__half*)gref)[t] = __double2half(g);
      ((__half*)nt)[t] = __double2half(n);
    } else {
      ((float*)gref)[t] = (float)g;
      ((float*)nt)[t] = (float)n;
    }
  }
}

extern "C" int rox_synth_lines(const synth_params* p, long long start, long long count, double* nu0, float* s_or_a,
                               float* g_up, float* e_lower, void* gref, void* nt, void* stream) {
  if (!p || count < 0 || start < 0 || !nu0 || !s_or_a || !e_lower || !gref || !nt || (p->exomol && !g_up)) return 1;
  if (count == 0) return 0;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  k_lines<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(*p, start, count, nu0, s_or_a, g_up, e_lower, gref, nt);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}
