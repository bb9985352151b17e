// CIA restructuring: collision-induced-absorption coefficient blocks (one temperature each,
// own wavenumber samples) onto the user's grid, one row per output temperature.
// pyROX paper, "Functionality of pyROX", "Combine and save": for CIA calculations the
// coefficients read from the input files are restructured into a wavelength- and
// temperature-dependent grid.
//
// A warp takes a tile of 32 x ROX_CIA_RUN consecutive points of one row, lane l the points
// p0 + l + 32 s (coalesced stores). For each block of the row's temperature, in input order,
// a lane finds the bracketing interval of its first point by binary search and then walks it
// forward (the points increase), interpolating with the interval's reciprocal width formed
// once per interval; the first block covering a point writes it, points no block covers get 0.
// The work is float64 arithmetic (this GPU's FP64 rate bounds it), within a few ulps of the
// division form k_i + (k_{i+1} - k_i) ((nu - nu_i) / (nu_{i+1} - nu_i)); samples are exact.
#include <cstdio>
#include <vector>
#include "rox_internal.cuh"

int rox_set_error(int code, const char* msg);   // rox_api.cu

namespace {

struct CiaArgs {
  int32_t n_blocks;
  int32_t n_rows;
  long long off[ROX_CIA_MAX_BLOCKS + 1];   // block b: samples off[b] .. off[b+1]-1
  int32_t row[ROX_CIA_MAX_BLOCKS];         // output row of block b, -1 if its temperature is not asked for
};

#define ROX_CIA_RUN 32

__device__ __forceinline__ double cia_point(const double* __restrict__ nodes, double nu_min, double dnu,
                                            long long j) {
  return nodes ? nodes[j] : __dadd_rn(nu_min, __dmul_rn((double)j, dnu));
}

__global__ void k_cia(const __grid_constant__ CiaArgs A, const double* __restrict__ nu, const double* __restrict__ k,
                      const double* __restrict__ nodes, double nu_min, double dnu, long long n, double* out) {
  const int lane = threadIdx.x & 31;
  const long long tile_pts = 32LL * ROX_CIA_RUN;
  const long long tiles_per_row = (n + tile_pts - 1) / tile_pts;
  const long long n_tiles = (long long)A.n_rows * tiles_per_row;
  const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long tile = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); tile < n_tiles;
       tile += warps) {
    const int t = (int)(tile / tiles_per_row);
    const long long p0 = (tile - (long long)t * tiles_per_row) * tile_pts + lane;
    double* row = out + (long long)t * n;
    unsigned done = 0;   // bit s: point p0 + 32 s written
    for (int b = 0; b < A.n_blocks; b++) {
      if (A.row[b] != t) continue;
      const long long o = A.off[b], m = A.off[b + 1] - A.off[b];
      const double* x = nu + o;
      const double* y = k + o;
      const double x_first = x[0], x_last = x[m - 1];
      long long i = -1;               // bracketing interval [x[i], x[i+1]] of the last point seen
      double xi = 0.0, yi = 0.0, dy = 0.0, r = 0.0, xi1 = 0.0;
      for (int s = 0; s < ROX_CIA_RUN; s++) {
        const long long j = p0 + 32LL * s;
        if (j >= n) break;
        if ((done >> s) & 1u) continue;
        const double v = cia_point(nodes, nu_min, dnu, j);
        if (!(v >= x_first && v <= x_last)) continue;
        double val;
        if (m == 1 || v == x_last) {
          val = y[m - 1];
        } else {
          if (i < 0 || v < xi) {       // first point inside this block (or nodes out of order): search
            long long lo = 0, hi = m;
            while (lo < hi) {
              const long long mid = (lo + hi) >> 1;
              if (x[mid] > v) hi = mid; else lo = mid + 1;
            }
            i = lo - 1;
            xi = x[i]; xi1 = x[i + 1]; yi = y[i];
            dy = y[i + 1] - yi;
            r = 1.0 / (xi1 - xi);
          }
          while (v >= xi1 && i < m - 2) {   // walk forward to the interval holding v
            i++;
            xi = xi1; yi = y[i];
            xi1 = x[i + 1];
            dy = y[i + 1] - yi;
            r = 1.0 / (xi1 - xi);
          }
          val = v == xi ? yi : fma(dy, (v - xi) * r, yi);
        }
        row[j] = val;
        done |= 1u << s;
      }
    }
    for (int s = 0; s < ROX_CIA_RUN; s++) {
      const long long j = p0 + 32LL * s;
      if (j >= n) break;
      if (!((done >> s) & 1u)) row[j] = 0.0;
    }
  }
}

int cia_launch(const rox_cia* cia, const double* nodes, double nu_min, double dnu, long long n, int n_T,
               const double* T_out, double* out, cudaStream_t s) {
  char msg[160];
  if (!cia || !cia->T_block || !cia->offset || !cia->nu || !cia->k) return rox_set_error(ROX_EINVAL, "cia arrays missing");
  if (cia->n_blocks < 1 || cia->n_blocks > ROX_CIA_MAX_BLOCKS) {
    snprintf(msg, sizeof msg, "cia->n_blocks = %d outside [1, %d]", cia->n_blocks, ROX_CIA_MAX_BLOCKS);
    return rox_set_error(ROX_EINVAL, msg);
  }
  if (n_T < 1 || n_T > ROX_CIA_MAX_TEMPS || !T_out || !out) return rox_set_error(ROX_EINVAL, "n_T, T_out or out invalid");
  static thread_local CiaArgs A;
  A.n_blocks = cia->n_blocks;
  A.n_rows = n_T;
  A.off[0] = cia->offset[0];
  if (A.off[0] != 0) return rox_set_error(ROX_EINVAL, "cia->offset[0] must be 0");
  for (int b = 0; b < cia->n_blocks; b++) {
    A.off[b + 1] = cia->offset[b + 1];
    if (A.off[b + 1] <= A.off[b]) return rox_set_error(ROX_EINVAL, "every CIA block needs at least one sample");
    A.row[b] = -1;
    for (int t = 0; t < n_T; t++)
      if (T_out[t] == cia->T_block[b]) { A.row[b] = t; break; }
  }
  if (n <= 0) return ROX_OK;
  const long long tiles = (long long)n_T * ((n + 32LL * ROX_CIA_RUN - 1) / (32LL * ROX_CIA_RUN));
  long long blocks = (tiles + 7) / 8;   // 8 warps per block, one tile per warp at a time
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_cia<<<(int)blocks, 256, 0, s>>>(A, cia->nu, cia->k, nodes, nu_min, dnu, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  return ROX_OK;
}

}  // namespace

extern "C" int rox_cia_regrid(const rox_cia* cia, const rox_grid* grid, int n_T, const double* T_out, double* out,
                              void* stream) {
  if (!grid || !(grid->dnu > 0.0) || grid->n <= 0) return rox_set_error(ROX_EINVAL, "grid invalid");
  return cia_launch(cia, nullptr, grid->nu_min, grid->dnu, grid->n, n_T, T_out, out, (cudaStream_t)stream);
}

extern "C" int rox_cia_regrid_nodes(const rox_cia* cia, const rox_nodes* nodes, int n_T, const double* T_out,
                                    double* out, void* stream) {
  if (!nodes || !nodes->nu || nodes->n <= 0) return rox_set_error(ROX_EINVAL, "nodes invalid");
  return cia_launch(cia, nodes->nu, 0.0, 0.0, nodes->n, n_T, T_out, out, (cudaStream_t)stream);
}
