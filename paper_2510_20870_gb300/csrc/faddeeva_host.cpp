// Host (CPU) build of the FP32 Faddeeva code used by the CUDA kernels, so its accuracy
// can be measured against scipy.special.wofz without a GPU.
#include <stdint.h>
#include "rox_faddeeva.cuh"

extern "C" void rox_host_re_w(const float* x, const float* y, float* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = rox_re_w(&rox_daw_taylor[0][0], x[i], y[i]);
}

extern "C" void rox_host_re_w_far(const float* x, const float* y, float* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = rox_re_w_far(x[i], y[i]);
}

extern "C" float rox_host_far_r2(float y) { return rox_far_coefs(y).r2; }

extern "C" void rox_host_re_w_core(const float* x, const float* y, float* out, int64_t n) {
  for (int64_t i = 0; i < n; i++) out[i] = rox_re_w_core(&rox_daw_taylor[0][0], x[i], y[i]);
}
