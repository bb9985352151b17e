// a3: sort by nu0, per-line grid windows and centre decomposition, per-tile line ranges.
// pyROX paper, "Combine and save": the line profiles are summed into a cross-section on
// the user's grid for each temperature-pressure point. With the lines sorted by nu0 and
// a hard wing cutoff, the lines that reach a wavenumber tile form one contiguous range,
// found here without atomics from the sorted order.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>
#include <thrust/iterator/counting_iterator.h>
#include <cuda_fp16.h>
#include "rox_internal.cuh"

namespace {

// d_j = (nu_min + j*dnu) - nu0 with each operation rounded separately (no contraction),
// exactly the double-precision expression of the cutoff test.
__device__ __forceinline__ double node_offset(double nu_min, double dnu, long long j, double nu0) {
  return __dsub_rn(__dadd_rn(nu_min, __dmul_rn((double)j, dnu)), nu0);
}

// `guard` bounds, in index units, the rounding of the candidates (nu0 - nu_min)/dnu -/+ cutoff/dnu
// and of the cutoff test for every line within reach of the grid: a candidate farther than
// that from an integer is the exact answer, and the exact test only runs for the others
// (about one line in 1e6). Lines beyond reach end up clamped to an empty or edge window
// either way.
__global__ void k_windows(const double* __restrict__ nu0s, long long n_lines, double nu_min,
                          double dnu, double inv_dnu, double c_idx, double guard, long long n_grid, double cutoff,
                          int32_t* jlo_out, int32_t* jhi_out, int32_t* k0_out, float* f_out, float4* geo_out,
                          unsigned long long* evals_out, int32_t* unsorted_out, int32_t unsorted_value) {
  long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long ev = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_lines; i += stride) {
    double nu0 = nu0s[i];
    if (i > 0 && nu0s[i - 1] > nu0 && unsorted_out) *unsorted_out = unsorted_value;
    // first j with d_j >= -cutoff, last j with d_j <= cutoff (d_j non-decreasing in j): a
    // candidate from the line centre in index units u = (nu0 - nu_min)/dnu -+ cutoff/dnu
    // (within `guard` of the exact real), then the exact test moves it. The conversions round
    // up / down straight to integers and saturate; a NaN centre gets an empty window.
    double u = (nu0 - nu_min) * inv_dnu;
    const double r_lo = u - c_idx;
    const double r_hi = u + c_idx;
    long long jlo = __double2ll_ru(r_lo), jhi = __double2ll_rd(r_hi);
    jlo = jlo < -4 ? -4 : (jlo > n_grid + 4 ? n_grid + 4 : jlo);
    jhi = jhi < -4 ? -4 : (jhi > n_grid + 4 ? n_grid + 4 : jhi);
    if (isnan(u)) { jlo = -4; jhi = -4; u = 0.0; }
    if (!(fabs(r_lo - rint(r_lo)) > guard)) {
      for (int it = 0; it < 4 && node_offset(nu_min, dnu, jlo - 1, nu0) >= -cutoff; it++) jlo--;
      for (int it = 0; it < 4 && node_offset(nu_min, dnu, jlo, nu0) < -cutoff; it++) jlo++;
    }
    if (!(fabs(r_hi - rint(r_hi)) > guard)) {
      for (int it = 0; it < 4 && node_offset(nu_min, dnu, jhi + 1, nu0) <= cutoff; it++) jhi++;
      for (int it = 0; it < 4 && node_offset(nu_min, dnu, jhi, nu0) > cutoff; it++) jhi--;
    }
    long long jl = jlo < 0 ? 0 : (jlo > n_grid ? n_grid : jlo);
    long long jh = jhi < -1 ? -1 : (jhi > n_grid - 1 ? n_grid - 1 : jhi);
    if (jh >= jl) ev += (unsigned long long)(jh - jl + 1);
    // centre decomposition (nu0 - nu_min)/dnu = k0 + f (k0 integer, f in [0, 1))
    double k0 = floor(u);
    double f = u - k0;
    if (f >= 1.0) { k0 += 1.0; f -= 1.0; }
    if (jh < jl) { k0 = 0.0; f = 0.0; }       // touches no grid point: never evaluated
    if (jlo_out) jlo_out[i] = (int32_t)jl;
    if (jhi_out) jhi_out[i] = (int32_t)jh;
    if (k0_out) k0_out[i] = (int32_t)k0;
    if (f_out) f_out[i] = (float)f;
    if (geo_out)
      geo_out[i] = make_float4((float)k0, (float)(f * dnu), __int_as_float((int)jl), __int_as_float((int)jh));
  }
  if (evals_out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd(evals_out, ev);
  }
}

// Windows on user-provided nodes (nu_k given, strictly increasing): the first node with
// nu_k - nu0 >= -cutoff and the last with nu_k - nu0 <= cutoff, the differences rounded once
// in double precision as the cutoff test is written; both are binary searches, the
// difference being non-decreasing in k. The line centre is carried as a double-float pair
// {hi, lo} (float hi = nu0 rounded, lo = the remainder) in the geometry record.
__global__ void k_node_windows(const double* __restrict__ nu0s, long long n_lines, const double* __restrict__ nodes,
                               long long n, double cutoff, int32_t* jlo_out, int32_t* jhi_out, float4* geo_out,
                               unsigned long long* evals_out, int32_t* unsorted_out, int32_t unsorted_value) {
  long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long ev = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_lines; i += stride) {
    const double nu0 = nu0s[i];
    if (i > 0 && nu0s[i - 1] > nu0 && unsorted_out) *unsorted_out = unsorted_value;
    long long a = 0, b = n;
    while (a < b) {
      const long long mid = (a + b) >> 1;
      if (__dsub_rn(nodes[mid], nu0) >= -cutoff) b = mid; else a = mid + 1;
    }
    const long long jl = a;
    b = n;
    while (a < b) {
      const long long mid = (a + b) >> 1;
      if (__dsub_rn(nodes[mid], nu0) > cutoff) b = mid; else a = mid + 1;
    }
    const long long jh = a - 1;
    if (jh >= jl) ev += (unsigned long long)(jh - jl + 1);
    if (jlo_out) jlo_out[i] = (int32_t)jl;
    if (jhi_out) jhi_out[i] = (int32_t)jh;
    if (geo_out) {
      const float hi = (float)nu0;
      geo_out[i] = make_float4(hi, (float)(nu0 - (double)hi), __int_as_float((int)jl), __int_as_float((int)jh));
    }
  }
  if (evals_out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd(evals_out, ev);
  }
}

// Per node, its offset from the first node of its ROX_SPAN-node span as a double-float pair
// {hi, lo}; per span, that first node as a pair. The node array is padded to whole spans with
// nodes continuing the last spacing (computed, never written out). Nodes that are not finite
// or not strictly increasing set *status = bad_value.
__global__ void k_node_offsets(const double* __restrict__ nodes, long long n, long long n_pad, float2* d_out,
                               float2* base_out, int32_t* status, int32_t bad_value) {
  long long stride = (long long)gridDim.x * blockDim.x;
  const double last = nodes[n - 1];
  double step = n > 1 ? last - nodes[n - 2] : 1.0;
  if (!(step > 0.0)) step = 1.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += stride) {
    const long long s = j / ROX_SPAN;
    const double base = nodes[s * ROX_SPAN];
    const double v = j < n ? nodes[j] : last + (double)(j - n + 1) * step;
    const double d = v - base;
    const float dh = (float)d;
    d_out[j] = make_float2(dh, (float)(d - (double)dh));
    if (j == s * ROX_SPAN) {
      const float bh = (float)base;
      base_out[s] = make_float2(bh, (float)(base - (double)bh));
    }
    if (j < n && (!isfinite(v) || (j > 0 && !(v > nodes[j - 1])))) *status = bad_value;
  }
}

// Tile t meets line i iff jhi_i >= t*W and jlo_i <= (t+1)*W - 1. Both bounds are
// non-decreasing along the sorted list, so lo[t] = first i with jhi_i >= t*W and
// hi[t] = first i with jlo_i >= (t+1)*W. Each line writes the boundaries between its
// predecessor's tile count and its own (the sorted-order form of a histogram prefix sum).
__device__ __forceinline__ long long tiles_reached_hi(int32_t jhi, int32_t W, long long n_tiles) {
  if (jhi < 0) return 0;
  long long c = (long long)jhi / W + 1;
  return c < n_tiles ? c : n_tiles;
}
__device__ __forceinline__ long long tiles_passed_lo(int32_t jlo, int32_t W, long long n_tiles) {
  long long c = (long long)jlo / W;
  return c < n_tiles ? c : n_tiles;
}

__global__ void k_tile_ranges(const int32_t* __restrict__ jlo, const int32_t* __restrict__ jhi,
                              long long n_lines, long long n_tiles, int32_t W,
                              long long* lo_out, long long* hi_out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n_lines; i += stride) {
    long long ch_prev = i > 0 ? tiles_reached_hi(jhi[i - 1], W, n_tiles) : 0;
    long long cl_prev = i > 0 ? tiles_passed_lo(jlo[i - 1], W, n_tiles) : 0;
    long long ch = i < n_lines ? tiles_reached_hi(jhi[i], W, n_tiles) : n_tiles;
    long long cl = i < n_lines ? tiles_passed_lo(jlo[i], W, n_tiles) : n_tiles;
    for (long long t = ch_prev; t < ch; t++) lo_out[t] = i;
    for (long long t = cl_prev; t < cl; t++) hi_out[t] = i;
  }
}

// same, reading the window bounds out of the packed geometry records
// k_tile_ranges_geo for a list given as indices into the sorted list (the kept lines of a
// selection, still in nu0 order): line i of the list is geo[idx[i]], and the list length is
// read on the device (*count, at most n_max).
__global__ void k_tile_ranges_idx(const float4* __restrict__ geo, const int32_t* __restrict__ idx,
                                  const long long* __restrict__ count, long long n_max, long long n_tiles, int32_t W,
                                  long long* lo_out, long long* hi_out) {
  const long long n_lines = *count;
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n_lines && i <= n_max; i += stride) {
    long long ch_prev = 0, cl_prev = 0, ch = n_tiles, cl = n_tiles;
    if (i > 0) {
      float4 g = geo[idx[i - 1]];
      ch_prev = tiles_reached_hi(__float_as_int(g.w), W, n_tiles);
      cl_prev = tiles_passed_lo(__float_as_int(g.z), W, n_tiles);
    }
    if (i < n_lines) {
      float4 g = geo[idx[i]];
      ch = tiles_reached_hi(__float_as_int(g.w), W, n_tiles);
      cl = tiles_passed_lo(__float_as_int(g.z), W, n_tiles);
    }
    for (long long t = ch_prev; t < ch; t++) lo_out[t] = i;
    for (long long t = cl_prev; t < cl; t++) hi_out[t] = i;
  }
}

// keep flag of every line and temperature: a selection marks dropped strengths with -0.0
__global__ void k_kept_flags(const float* __restrict__ S32, long long total, uint8_t* flags) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride)
    flags[i] = __float_as_uint(S32[i]) != 0x80000000u;
}

__global__ void k_tile_ranges_geo(const float4* __restrict__ geo, long long n_lines, long long n_tiles,
                                  int32_t W, long long* lo_out, long long* hi_out) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n_lines; i += stride) {
    long long ch_prev = 0, cl_prev = 0, ch = n_tiles, cl = n_tiles;
    if (i > 0) {
      float4 g = geo[i - 1];
      ch_prev = tiles_reached_hi(__float_as_int(g.w), W, n_tiles);
      cl_prev = tiles_passed_lo(__float_as_int(g.z), W, n_tiles);
    }
    if (i < n_lines) {
      float4 g = geo[i];
      ch = tiles_reached_hi(__float_as_int(g.w), W, n_tiles);
      cl = tiles_passed_lo(__float_as_int(g.z), W, n_tiles);
    }
    for (long long t = ch_prev; t < ch; t++) lo_out[t] = i;
    for (long long t = cl_prev; t < cl; t++) hi_out[t] = i;
  }
}

__global__ void k_iota(int32_t* v, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) v[i] = (int32_t)i;
}

template <typename T>
__global__ void k_gather(const T* __restrict__ src, const int32_t* __restrict__ perm, T* dst, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[perm[i]];
}

__global__ void k_perm64(const int32_t* __restrict__ perm, long long* out, long long n) {
  long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = perm[i];
}

int grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

size_t cub_temp_bytes(long long n) {
  size_t tb = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tb, (const unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                  (const int32_t*)nullptr, (int32_t*)nullptr, (int64_t)n, 0, 63);
  return tb;
}

}  // namespace

cudaError_t rox_launch_windows(const double* nu0, long long n_lines, const rox_grid* g, double cutoff,
                               int32_t* jlo, int32_t* jhi, int32_t* k0, float* f, float4* geo,
                               unsigned long long* evals, int32_t* unsorted, int32_t unsorted_value,
                               cudaStream_t s) {
  // rounding bound of the candidates and of the cutoff test, in index units: every quantity
  // involved is at most |nu| + 2 cutoff in cm^-1 (or n + 8 in index units) for a line within
  // reach; 16 double-precision ulps of each is a generous margin
  const double inv_dnu = 1.0 / g->dnu;
  const double nu_abs = fmax(fabs(g->nu_min), fabs(g->nu_min + (double)(g->n - 1) * g->dnu));
  const double guard = 16.0 * 2.3e-16 * ((nu_abs + 2.0 * cutoff) * inv_dnu + (double)g->n + 8.0);
  k_windows<<<grid_for(n_lines), 256, 0, s>>>(nu0, n_lines, g->nu_min, g->dnu, inv_dnu, cutoff * inv_dnu, guard, g->n,
                                               cutoff, jlo, jhi,
                                               k0,
                                               f, geo, evals, unsorted, unsorted_value);
  return cudaGetLastError();
}

cudaError_t rox_launch_node_windows(const double* nu0, long long n_lines, const double* nodes, long long n,
                                    double cutoff, int32_t* jlo, int32_t* jhi, float4* geo,
                                    unsigned long long* evals, int32_t* unsorted, int32_t unsorted_value,
                                    cudaStream_t s) {
  k_node_windows<<<grid_for(n_lines), 256, 0, s>>>(nu0, n_lines, nodes, n, cutoff, jlo, jhi, geo, evals, unsorted,
                                                   unsorted_value);
  return cudaGetLastError();
}

cudaError_t rox_launch_node_offsets(const double* nodes, long long n, long long n_pad, float2* d, float2* base,
                                    int32_t* status, int32_t bad_value, cudaStream_t s) {
  k_node_offsets<<<grid_for(n_pad), 256, 0, s>>>(nodes, n, n_pad, d, base, status, bad_value);
  return cudaGetLastError();
}

cudaError_t rox_launch_tile_ranges(const int32_t* jlo, const int32_t* jhi, long long n_lines, long long n_tiles,
                                   int32_t W, long long* lo, long long* hi, cudaStream_t s) {
  k_tile_ranges<<<grid_for(n_lines + 1), 256, 0, s>>>(jlo, jhi, n_lines, n_tiles, W, lo, hi);
  return cudaGetLastError();
}

cudaError_t rox_launch_tile_ranges_geo(const float4* geo, long long n_lines, long long n_tiles, int32_t W,
                                       long long* lo, long long* hi, cudaStream_t s) {
  k_tile_ranges_geo<<<grid_for(n_lines + 1), 256, 0, s>>>(geo, n_lines, n_tiles, W, lo, hi);
  return cudaGetLastError();
}

// indices of the flagged lines, in order (CUB DeviceSelect::Flagged over 0..n-1), and their count
size_t rox_compact_temp_bytes(long long n) {
  size_t tb = 0;
  cub::DeviceSelect::Flagged(nullptr, tb, thrust::counting_iterator<int32_t>(0), (const uint8_t*)nullptr,
                             (int32_t*)nullptr, (long long*)nullptr, (int64_t)(n > 0 ? n : 1));
  return tb;
}

cudaError_t rox_launch_compact(const float* S32_all, long long n, int n_temps, uint8_t* flags, int32_t* idx,
                               long long* counts, void* temp, size_t temp_bytes, cudaStream_t s) {
  const long long total = (long long)n_temps * n;
  k_kept_flags<<<grid_for(total), 256, 0, s>>>(S32_all, total, flags);
  cudaError_t e = cudaGetLastError();
  for (int t = 0; t < n_temps && e == cudaSuccess; t++) {
    size_t tb = temp_bytes;
    e = cub::DeviceSelect::Flagged(temp, tb, thrust::counting_iterator<int32_t>(0), flags + (size_t)t * n,
                                   idx + (size_t)t * n, counts + t, (int64_t)n, s);
  }
  return e;
}

cudaError_t rox_launch_tile_ranges_idx(const float4* geo, const int32_t* idx, const long long* count, long long n_max,
                                       long long n_tiles, int32_t W, long long* lo, long long* hi, cudaStream_t s) {
  k_tile_ranges_idx<<<grid_for(n_max + 1), 256, 0, s>>>(geo, idx, count, n_max, n_tiles, W, lo, hi);
  return cudaGetLastError();
}

size_t rox_sort_ws_bytes(long long n) {
  return rox_align256(cub_temp_bytes(n)) + rox_align256((size_t)n * 8) + 2 * rox_align256((size_t)n * 4) + 256;
}

cudaError_t rox_launch_sort(const rox_lines* in, const rox_lines_buf* out, int64_t* perm_out, void* ws,
                            cudaStream_t s) {
  long long n = in->n;
  char* p = (char*)ws;
  size_t tb = cub_temp_bytes(n);
  void* temp = p; p += rox_align256(tb);
  unsigned long long* keys_out = (unsigned long long*)p; p += rox_align256((size_t)n * 8);
  int32_t* idx_in = (int32_t*)p; p += rox_align256((size_t)n * 4);
  int32_t* idx_out = (int32_t*)p;
  k_iota<<<grid_for(n), 256, 0, s>>>(idx_in, n);
  // positive doubles order like their bit patterns; bit 63 (sign) is zero for nu0 > 0
  cudaError_t e = cub::DeviceRadixSort::SortPairs(temp, tb, (const unsigned long long*)in->nu0, keys_out,
                                                  idx_in, idx_out, (int64_t)n, 0, 63, s);
  if (e != cudaSuccess) return e;
  int gb = grid_for(n);
  k_gather<double><<<gb, 256, 0, s>>>(in->nu0, idx_out, out->nu0, n);
  k_gather<float><<<gb, 256, 0, s>>>(in->s_or_a, idx_out, out->s_or_a, n);
  if (in->convention == ROX_EXOMOL) k_gather<float><<<gb, 256, 0, s>>>(in->g_up, idx_out, out->g_up, n);
  k_gather<float><<<gb, 256, 0, s>>>(in->e_lower, idx_out, out->e_lower, n);
  if (in->width_dtype == ROX_WIDTH_F16) {
    k_gather<__half><<<gb, 256, 0, s>>>((const __half*)in->gamma_ref, idx_out, (__half*)out->gamma_ref, n);
    k_gather<__half><<<gb, 256, 0, s>>>((const __half*)in->n_t, idx_out, (__half*)out->n_t, n);
  } else {
    k_gather<float><<<gb, 256, 0, s>>>((const float*)in->gamma_ref, idx_out, (float*)out->gamma_ref, n);
    k_gather<float><<<gb, 256, 0, s>>>((const float*)in->n_t, idx_out, (float*)out->n_t, n);
  }
  if (perm_out) k_perm64<<<gb, 256, 0, s>>>(idx_out, (long long*)perm_out, n);
  return cudaGetLastError();
}
