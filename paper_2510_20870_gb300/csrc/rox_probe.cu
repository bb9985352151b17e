// FP32 rate probe for the Voigt kernel's roofline: the FP32 fused multiply-add rate this GPU
// sustains, measured rather than taken from SMs x 128 lanes x clock. Every thread runs 16
// independent FMA chains (enough to cover the pipeline latency), so the launch is bound by the
// FMA pipes alone. Not part of the cross-section method (the paper has no counterpart).
#include "rox_internal.cuh"

int rox_set_error(int code, const char* msg);   // rox_api.cu
cudaError_t rox_launch_pair_loop_probe(int n_blocks, int warps, int reps, float* out, cudaStream_t s);   // rox_voigt.cu

namespace {

#define ROX_PROBE_CHAINS 16
#define ROX_PROBE_UNROLL 8
#define ROX_PROBE_THREADS 256

__global__ void __launch_bounds__(ROX_PROBE_THREADS) k_fp32_probe(float* out, int reps, float a, float b) {
  float v[ROX_PROBE_CHAINS];
#pragma unroll
  for (int i = 0; i < ROX_PROBE_CHAINS; i++) v[i] = a * (float)(threadIdx.x + i);
#pragma unroll 1
  for (int r = 0; r < reps; r++) {
#pragma unroll
    for (int k = 0; k < ROX_PROBE_UNROLL; k++)
#pragma unroll
      for (int i = 0; i < ROX_PROBE_CHAINS; i++) v[i] = fmaf(v[i], a, b);   // converges to b/(1-a): no overflow
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < ROX_PROBE_CHAINS; i++) s += v[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" size_t rox_fp32_probe_out_size(int n_blocks) {
  return n_blocks > 0 ? (size_t)n_blocks * ROX_PROBE_THREADS * sizeof(float) : 0;
}

extern "C" int rox_fp32_probe(int n_blocks, int reps, float* out, size_t out_bytes, double* fma_out, void* stream) {
  if (n_blocks < 1 || reps < 1 || !out || !fma_out) return rox_set_error(ROX_EINVAL, "rox_fp32_probe: bad arguments");
  if (out_bytes < rox_fp32_probe_out_size(n_blocks)) return rox_set_error(ROX_ENOMEM, "rox_fp32_probe: out too small");
  k_fp32_probe<<<n_blocks, ROX_PROBE_THREADS, 0, (cudaStream_t)stream>>>(out, reps, 0.999f, 0.5f);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  *fma_out = (double)n_blocks * ROX_PROBE_THREADS * (double)reps * ROX_PROBE_UNROLL * ROX_PROBE_CHAINS;
  return ROX_OK;
}

extern "C" int rox_pair_loop_probe(int n_blocks, int reps, float* out, size_t out_bytes, double* evals_out,
                                   void* stream) {
  if (n_blocks < 1 || reps < 1 || !out || !evals_out) return rox_set_error(ROX_EINVAL, "rox_pair_loop_probe: bad arguments");
  if (out_bytes < rox_fp32_probe_out_size(n_blocks)) return rox_set_error(ROX_ENOMEM, "rox_pair_loop_probe: out too small");
  cudaError_t e = rox_launch_pair_loop_probe(n_blocks, ROX_PROBE_THREADS / 32, reps, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  // per thread: reps rounds x 16 pairs x 2 lines x ROX_K points
  *evals_out = (double)n_blocks * ROX_PROBE_THREADS * (double)reps * 16.0 * 2.0 * ROX_K;
  return ROX_OK;
}
