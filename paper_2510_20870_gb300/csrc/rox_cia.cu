// CIA restructuring: collision-induced-absorption coefficient blocks (one temperature each,
// own wavenumber samples) onto the user's grid, one row per output temperature.
// pyROX paper, "Functionality of pyROX", "Combine and save": for CIA calculations the
// coefficients read from the input files are restructured into a wavelength- and
// temperature-dependent grid.
//
// Everything is float64, and this GPU's float64 rate is low (about two operations per clock
// per SM), so both kernels are built around doing few float64 operations per point; what
// bounds the grid kernel then is the latency of its table reads, hence short tiles and many
// warps.
//
// Uniform grid, two launches. k_cia_intervals (one thread per sample) decides which points
// each interval holds exactly as the definition has it, on the rounded points
// nu_j = nu_min + j dnu: interval [x_i, x_{i+1}) holds j in [c_i, c_{i+1}), c_i the first j
// with nu_j >= x_i (a bracketed search around (x_i - nu_min) / dnu); the last sample holds
// [c_{m-1}, e), e the first j with nu_j > x_last. It stores c_i, the interpolant at c_i,
// k_i + (k_{i+1} - k_i) ((nu_{c_i} - x_i) / h_i), and its step per grid point,
// (k_{i+1} - k_i) dnu / h_i (0 on the last sample). In k_cia_grid a warp takes 32 x
// ROX_CIA_GRUN consecutive points of a row, lane l the points p0 + l + 32 s, so every store
// is coalesced; the interval of the tile's first point comes from a warp-parallel integer
// search over c_i (32 probes a round), each lane walks on from there, evaluates the interpolant at its first point of an
// interval (k(c_i) + (j - c_i) step) and then adds 32 steps per point: one float64 addition
// per point, within ROX_CIA_GRUN roundings of the direct form and exact at samples.
//
// Nodes (k_cia): a warp takes a tile of 32 x ROX_CIA_RUN nodes, lane l the nodes
// p0 + l + 32 s (coalesced stores); a lane finds the bracketing interval of its first node by
// binary search and walks forward while the nodes increase (searching again if one goes
// back), with the interval's reciprocal width formed once per interval.
//
// In both, the first block in input order that covers a point writes it; 0 where none does.
#include <algorithm>
#include <cmath>
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
  int32_t row_start[ROX_CIA_MAX_TEMPS + 1];   // the blocks of row t: row_block[row_start[t] .. row_start[t+1]-1]
  int16_t row_block[ROX_CIA_MAX_BLOCKS];      // block indices grouped by row, input order within a row
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
    for (int q = A.row_start[t]; q < A.row_start[t + 1]; q++) {
      const int b = A.row_block[q];
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
            i = min(max(lo - 1, 0LL), m - 2);   // lo in [1, m-1] for increasing samples
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


#define ROX_CIA_GRUN 16                      // points per lane in a tile (tile: 32 x GRUN consecutive points)
#define ROX_CIA_GWARPS 4                     // warps per block

struct CiaGrid {
  double nu_min, dnu, inv_dnu;
  long long n;
};

__device__ __forceinline__ double grid_nu(const CiaGrid& g, long long j) {
  return __dadd_rn(g.nu_min, __dmul_rn((double)j, g.dnu));
}

// First j in [0, n] with nu_j >= x (strict: nu_j > x); nu_n counts as +infinity. The rounded
// points never decrease in j, so a bisection over a bracket is exact; the bracket is
// (x - nu_min) / dnu +- 4, widened to [0, n] on the side where it fails.
__device__ long long grid_first(const CiaGrid& g, double x, bool strict) {
  const double t = (x - g.nu_min) * g.inv_dnu;
  long long c;
  if (!(t > 0.0)) c = 0;
  else if (t >= (double)g.n) c = g.n;
  else c = (long long)ceil(t);
  long long lo = c - 4 < 0 ? 0 : c - 4;
  long long hi = c + 4 > g.n ? g.n : c + 4;
  auto hit = [&](long long j) { const double v = grid_nu(g, j); return strict ? v > x : v >= x; };
  if (lo > 0 && hit(lo - 1)) lo = 0;
  if (hi < g.n && !hit(hi)) hi = g.n;
  while (lo < hi) {
    const long long mid = lo + ((hi - lo) >> 1);
    if (hit(mid)) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Workspace of the uniform-grid path: per sample c_i (int64), the value at c_i, the step and 32
// steps (float64), per block e; unused for blocks whose temperature is not asked for.
struct CiaTables {
  long long* c;
  double* v0;
  double* dv;
  double* dv32;   // 32 dv, a lane's step (exact: a power-of-two multiple)
  long long* e;
};

__device__ __forceinline__ int block_of(const CiaArgs& A, long long q) {   // the block holding sample q
  int lo = 0, hi = A.n_blocks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (A.off[mid] <= q) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_cia_intervals(const __grid_constant__ CiaArgs A, const double* __restrict__ nu,
                                const double* __restrict__ k, const CiaGrid g, CiaTables T) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.off[A.n_blocks]) return;
  const int b = block_of(A, q);
  if (A.row[b] < 0) return;
  const long long last = A.off[b + 1] - 1;
  const double xi = nu[q];
  const long long c = grid_first(g, xi, false);
  T.c[q] = c;
  if (q == last) {
    T.v0[q] = k[q];
    T.dv[q] = 0.0;
    T.dv32[q] = 0.0;
    T.e[b] = grid_first(g, xi, true);
  } else {
    const double yi = k[q], dy = k[q + 1] - yi;
    const double r = 1.0 / (nu[q + 1] - xi);
    T.v0[q] = fma(dy, (grid_nu(g, c) - xi) * r, yi);
    const double dv = dy * (g.dnu * r);
    T.dv[q] = dv;
    T.dv32[q] = 32.0 * dv;
  }
}

__global__ void __launch_bounds__(32 * ROX_CIA_GWARPS, 12)   // 40 registers: 12 CTAs per SM
k_cia_grid(const __grid_constant__ CiaArgs A, const CiaGrid g, const CiaTables T, double* out) {
  const int lane = threadIdx.x & 31;
  const long long tile_pts = 32LL * ROX_CIA_GRUN;
  const long long tiles_per_row = (g.n + tile_pts - 1) / tile_pts;
  const long long n_tiles = (long long)A.n_rows * tiles_per_row;
  const long long warps = (long long)gridDim.x * ROX_CIA_GWARPS;
  for (long long tile = (long long)blockIdx.x * ROX_CIA_GWARPS + (threadIdx.x >> 5); tile < n_tiles; tile += warps) {
    const int t = (int)(tile / tiles_per_row);
    const long long p0 = (tile - (long long)t * tiles_per_row) * tile_pts;
    const long long p_end = min(p0 + tile_pts, g.n);
    double* row = out + (long long)t * g.n;
    unsigned done = 0;   // bit s: point p0 + lane + 32 s written
    for (int q = A.row_start[t]; q < A.row_start[t + 1]; q++) {
      const int b = A.row_block[q];
      const long long o = A.off[b], m = A.off[b + 1] - A.off[b];
      const long long* c = T.c + o;
      const long long e = T.e[b];
      const long long a = max(c[0], p0), z = min(e, p_end);   // the block's points in this tile: [a, z)
      if (a >= z) continue;
      long long i;
      {   // the last interval starting at or before a (c_0 <= a): 32 probes a round, one per
          // lane, narrow the range 32-fold (three dependent loads up to 32768 samples)
        long long lo = 0, len = m;
        while (len > 1) {
          const long long step = (len + 31) >> 5;
          const long long off = (long long)lane * step;
          const bool le = off < len && c[lo + off] <= a;
          // probes 0 .. k-1 are <= a; k >= 1 for increasing samples, and the clamp keeps every
          // index inside the block for any data
          const int k = max(1, __popc(__ballot_sync(0xffffffffu, le)));
          const long long nlo = lo + (long long)(k - 1) * step;
          len = min(step, lo + len - nlo);
          lo = nlo;
        }
        i = lo;
      }
      const long long d_lo = a - p0 - lane, d_hi = z - p0 - lane;
      const int s_lo = d_lo > 0 ? (int)((d_lo + 31) >> 5) : 0;   // first s with p0 + lane + 32 s >= a
      const int s_hi = d_hi > 0 ? (int)((d_hi + 31) >> 5) : 0;   // ... >= z
      long long j = p0 + lane + 32LL * s_lo;
      long long nxt = -1;   // forces the set-up at the lane's first point
      double val = 0.0, step = 0.0;
      for (int s = s_lo; s < s_hi; s++, j += 32) {
        if (j >= nxt) {   // first point of the lane in this block, or a later interval
          nxt = i + 1 < m ? c[i + 1] : e;
          while (j >= nxt && i < m - 1) {
            i++;
            nxt = i + 1 < m ? c[i + 1] : e;
          }
          val = fma((double)(j - c[i]), T.dv[o + i], T.v0[o + i]);
          step = T.dv32[o + i];   // no float64 multiply per set-up: the pipe this kernel is bound by
        }
        if (!((done >> s) & 1u)) row[j] = val;
        val += step;
      }
      if (s_hi > s_lo) done |= (s_hi - s_lo >= 32 ? ~0u : ((1u << (s_hi - s_lo)) - 1u)) << s_lo;
    }
    for (int s = 0; s < ROX_CIA_GRUN; s++) {
      const long long j = p0 + lane + 32LL * s;
      if (j < p_end && !((done >> s) & 1u)) row[j] = 0.0;
    }
  }
}

int cia_launch(const rox_cia* cia, const double* nodes, double nu_min, double dnu, long long n, int n_T,
               const double* T_out, double* out, void* ws, size_t ws_bytes, cudaStream_t s) {
  char msg[160];
  if (!cia || !cia->T_block || !cia->offset || !cia->nu || !cia->k) return rox_set_error(ROX_EINVAL, "cia arrays missing");
  if (cia->n_blocks < 1 || cia->n_blocks > ROX_CIA_MAX_BLOCKS) {
    snprintf(msg, sizeof msg, "cia->n_blocks = %d outside [1, %d]", cia->n_blocks, ROX_CIA_MAX_BLOCKS);
    return rox_set_error(ROX_EINVAL, msg);
  }
  if (n_T < 1 || n_T > ROX_CIA_MAX_TEMPS || !T_out || !out) return rox_set_error(ROX_EINVAL, "n_T, T_out or out invalid");
  {   // output temperatures: finite and distinct (each block feeds at most one row)
    std::vector<double> Ts(T_out, T_out + n_T);
    for (double v : Ts)
      if (!std::isfinite(v)) return rox_set_error(ROX_EINVAL, "T_out holds a non-finite temperature");
    std::sort(Ts.begin(), Ts.end());
    for (int t = 1; t < n_T; t++)
      if (Ts[t] == Ts[t - 1]) return rox_set_error(ROX_EINVAL, "T_out holds a temperature twice");
  }
  static thread_local CiaArgs A;
  A.n_blocks = cia->n_blocks;
  A.n_rows = n_T;
  A.off[0] = cia->offset[0];
  if (A.off[0] != 0) return rox_set_error(ROX_EINVAL, "cia->offset[0] must be 0");
  for (int t = 0; t <= n_T; t++) A.row_start[t] = 0;
  for (int b = 0; b < cia->n_blocks; b++) {
    A.off[b + 1] = cia->offset[b + 1];
    if (A.off[b + 1] <= A.off[b]) return rox_set_error(ROX_EINVAL, "every CIA block needs at least one sample");
    A.row[b] = -1;
    for (int t = 0; t < n_T; t++)
      if (T_out[t] == cia->T_block[b]) { A.row[b] = t; break; }
    if (A.row[b] >= 0) A.row_start[A.row[b] + 1]++;
  }
  for (int t = 0; t < n_T; t++) A.row_start[t + 1] += A.row_start[t];
  {
    int fill[ROX_CIA_MAX_TEMPS];
    for (int t = 0; t < n_T; t++) fill[t] = A.row_start[t];
    for (int b = 0; b < cia->n_blocks; b++)
      if (A.row[b] >= 0) A.row_block[fill[A.row[b]]++] = (int16_t)b;
  }
  if (n <= 0) return ROX_OK;
  if (!nodes) {
    CiaGrid g{nu_min, dnu, 1.0 / dnu, n};
    const long long n_samples = A.off[A.n_blocks];
    if (!ws || ((uintptr_t)ws & 7) || ws_bytes < rox_cia_workspace_size(A.n_blocks, n_samples))
      return rox_set_error(ROX_EINVAL, "CIA workspace missing, misaligned or smaller than rox_cia_workspace_size");
    CiaTables tb;
    tb.c = (long long*)ws;
    tb.v0 = (double*)(tb.c + n_samples);
    tb.dv = tb.v0 + n_samples;
    tb.dv32 = tb.dv + n_samples;
    tb.e = (long long*)(tb.dv32 + n_samples);
    k_cia_intervals<<<(unsigned)((n_samples + 255) / 256), 256, 0, s>>>(A, cia->nu, cia->k, g, tb);
    const long long tiles = (long long)n_T * ((n + 32LL * ROX_CIA_GRUN - 1) / (32LL * ROX_CIA_GRUN));
    long long blocks = (tiles + ROX_CIA_GWARPS - 1) / ROX_CIA_GWARPS;
    if (blocks > 152 * 12 * 8) blocks = 152 * 12 * 8;
    k_cia_grid<<<(int)blocks, 32 * ROX_CIA_GWARPS, 0, s>>>(A, g, tb, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
    return ROX_OK;
  }
  const long long tiles = (long long)n_T * ((n + 32LL * ROX_CIA_RUN - 1) / (32LL * ROX_CIA_RUN));
  long long blocks = (tiles + 7) / 8;   // 8 warps per block, one tile per warp at a time
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_cia<<<(int)blocks, 256, 0, s>>>(A, cia->nu, cia->k, nodes, nu_min, dnu, n, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rox_set_error(ROX_ECUDA, cudaGetErrorString(e));
  return ROX_OK;
}

}  // namespace

extern "C" size_t rox_cia_workspace_size(int32_t n_blocks, int64_t n_samples) {
  if (n_blocks < 0 || n_samples < 0) return 0;
  return sizeof(double) * (4 * (size_t)n_samples + (size_t)n_blocks);
}

extern "C" int rox_cia_regrid(const rox_cia* cia, const rox_grid* grid, int n_T, const double* T_out, double* out,
                              void* ws, size_t ws_bytes, void* stream) {
  if (!grid || !(grid->dnu > 0.0) || grid->n <= 0) return rox_set_error(ROX_EINVAL, "grid invalid");
  return cia_launch(cia, nullptr, grid->nu_min, grid->dnu, grid->n, n_T, T_out, out, ws, ws_bytes,
                    (cudaStream_t)stream);
}

extern "C" int rox_cia_regrid_nodes(const rox_cia* cia, const rox_nodes* nodes, int n_T, const double* T_out,
                                    double* out, void* stream) {
  if (!nodes || !nodes->nu || nodes->n <= 0) return rox_set_error(ROX_EINVAL, "nodes invalid");
  return cia_launch(cia, nodes->nu, 0.0, 0.0, nodes->n, n_T, T_out, out, nullptr, 0, (cudaStream_t)stream);
}
