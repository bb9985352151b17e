// C ABI of librox (include/rox.h): argument checks, workspace layout, launch order.
// Everything after the checks is enqueued on the caller's stream; nothing here
// allocates device memory or synchronises, except rox_ws_status.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include "rox_internal.cuh"

// kernels (rox_params.cu, rox_geometry.cu, rox_voigt.cu)
cudaError_t rox_launch_strengths(const rox_lines* L, double T, double Q_T, double Q_ref, float* S_out,
                                 cudaStream_t s);
cudaError_t rox_launch_widths(const rox_lines* L, double mass_amu, double P_bar, double T, float* gG,
                              float* gL, cudaStream_t s);
cudaError_t rox_launch_strengths_multi(const rox_lines* L, int n_temps, const double* temps,
                                       const double* q_of_temp, double Q_ref, double* S_T,
                                       unsigned long long* smax_bits, cudaStream_t s);
cudaError_t rox_launch_scale_strengths(const double* S_T, long long n, int n_temps,
                                       const unsigned long long* smax_bits, float* S32, cudaStream_t s);
cudaError_t rox_launch_windows(const double* nu0, long long n_lines, const rox_grid* g, double cutoff,
                               int32_t* jlo, int32_t* jhi, int32_t* k0, float* f, float4* geo,
                               unsigned long long* evals, int32_t* unsorted, int32_t unsorted_value,
                               cudaStream_t s);
cudaError_t rox_launch_tile_ranges(const int32_t* jlo, const int32_t* jhi, long long n_lines, long long n_tiles,
                                   int32_t W, long long* lo, long long* hi, cudaStream_t s);
cudaError_t rox_launch_tile_ranges_geo(const float4* geo, long long n_lines, long long n_tiles, int32_t W,
                                       long long* lo, long long* hi, cudaStream_t s);
size_t rox_sort_ws_bytes(long long n);
cudaError_t rox_launch_sort(const rox_lines* in, const rox_lines_buf* out, int64_t* perm_out, void* ws,
                            cudaStream_t s);
cudaError_t rox_launch_voigt(const RoxVoigtArgs& A, int n_blocks, cudaStream_t s);
cudaError_t rox_voigt_blocks_per_sm(int* nb);
cudaError_t rox_launch_faddeeva(const float* x, const float* y, float* out, long long n, cudaStream_t s);

namespace {

thread_local std::string g_err;
thread_local cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int ok() {
  g_err.clear();
  return ROX_OK;
}

int cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return ROX_OK;
  return fail(ROX_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

int check_lines(const rox_lines* L, bool strengths, bool widths) {
  if (!L) return fail(ROX_EINVAL, "lines is NULL");
  if (L->n < 0) return fail(ROX_EINVAL, "lines->n = %lld < 0", (long long)L->n);
  if (L->n > (int64_t)2000000000) return fail(ROX_ERANGE, "lines->n = %lld above 2e9", (long long)L->n);
  if (L->convention != ROX_HITRAN && L->convention != ROX_EXOMOL)
    return fail(ROX_EINVAL, "lines->convention = %d", L->convention);
  if (L->width_dtype != ROX_WIDTH_F32 && L->width_dtype != ROX_WIDTH_F16)
    return fail(ROX_EINVAL, "lines->width_dtype = %d", L->width_dtype);
  if (L->n == 0) return ROX_OK;
  if (!L->nu0) return fail(ROX_EINVAL, "lines->nu0 is NULL");
  if (strengths) {
    if (!L->s_or_a || !L->e_lower) return fail(ROX_EINVAL, "lines->s_or_a or lines->e_lower is NULL");
    if (L->convention == ROX_EXOMOL && !L->g_up) return fail(ROX_EINVAL, "ExoMol lines need g_up");
  }
  if (widths && (!L->gamma_ref || !L->n_t)) return fail(ROX_EINVAL, "lines->gamma_ref or lines->n_t is NULL");
  return ROX_OK;
}

int check_grid(const rox_grid* g) {
  if (!g) return fail(ROX_EINVAL, "grid is NULL");
  if (!std::isfinite(g->nu_min) || !finite_pos(g->dnu)) return fail(ROX_EINVAL, "grid nu_min/dnu invalid");
  if (g->n <= 0) return fail(ROX_EINVAL, "grid->n = %lld <= 0", (long long)g->n);
  if (g->n > ROX_MAX_GRID) return fail(ROX_ERANGE, "grid->n = %lld above %d", (long long)g->n, ROX_MAX_GRID);
  return ROX_OK;
}

int check_cutoff(double cutoff, const rox_grid* g) {
  if (!finite_pos(cutoff)) return fail(ROX_EINVAL, "cutoff must be > 0");
  if (cutoff > 4000.0) return fail(ROX_ERANGE, "cutoff %g above 4000 cm^-1", cutoff);
  if (cutoff / g->dnu > (double)ROX_MAX_CUTOFF_STEPS)
    return fail(ROX_ERANGE, "cutoff/dnu = %g above %d", cutoff / g->dnu, ROX_MAX_CUTOFF_STEPS);
  return ROX_OK;
}

long long n_tiles_of(long long n_grid) { return (n_grid + ROX_TILE - 1) / ROX_TILE; }

struct WsLayout {
  RoxWsHeader* hdr;
  float4* geo;
  long long* tlo;
  long long* thi;
  double* S_T;
  float* S32;
  size_t bytes;
};

WsLayout ws_layout(void* ws, long long n_lines, long long n_grid, int n_temps) {
  WsLayout w;
  char* base = (char*)ws;
  size_t off = 0;
  w.hdr = (RoxWsHeader*)(base + off);
  off += ROX_WS_HEADER_BYTES;
  w.geo = (float4*)(base + off);
  off += rox_align256((size_t)(n_lines > 0 ? n_lines : 1) * sizeof(float4));
  long long nt = n_tiles_of(n_grid);
  w.tlo = (long long*)(base + off);
  off += rox_align256((size_t)nt * 8);
  w.thi = (long long*)(base + off);
  off += rox_align256((size_t)nt * 8);
  w.S_T = (double*)(base + off);
  off += rox_align256((size_t)n_temps * (size_t)(n_lines > 0 ? n_lines : 1) * 8);
  w.S32 = (float*)(base + off);
  off += rox_align256((size_t)n_temps * (size_t)(n_lines > 0 ? n_lines : 1) * 4);
  w.bytes = off;
  return w;
}

int g_voigt_blocks = 0;
int g_voigt_device = -1;

int voigt_grid(int* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
  if (dev != g_voigt_device) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaDeviceGetAttribute");
    e = rox_voigt_blocks_per_sm(&per);
    if (e != cudaSuccess) return cuda_check(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    g_voigt_blocks = sms * (per > 0 ? per : 1);
    g_voigt_device = dev;
  }
  *out = g_voigt_blocks;
  return ROX_OK;
}

}  // namespace

// sets this thread's error message for entry points defined in other translation units
int rox_set_error(int code, const char* msg) { return fail(code, "%s", msg); }

extern "C" {

const char* rox_last_error(void) { return g_err.c_str(); }

const char* rox_version(void) { return "librox 0.1.0 (sm_103a, FP32 Voigt, FP64 line strengths)"; }

int rox_line_strengths(const rox_lines* lines, double T, double Q_T, double Q_ref, float* S_out, void* stream) {
  int rc = check_lines(lines, true, false);
  if (rc) return rc;
  if (!finite_pos(T) || !finite_pos(Q_T) || !finite_pos(Q_ref)) return fail(ROX_EINVAL, "T, Q_T, Q_ref must be > 0");
  if (lines->n > 0 && !S_out) return fail(ROX_EINVAL, "S_out is NULL");
  if (lines->n == 0) return ok();
  rc = cuda_check(rox_launch_strengths(lines, T, Q_T, Q_ref, S_out, (cudaStream_t)stream), "strengths kernel");
  return rc ? rc : ok();
}

int rox_line_widths(const rox_lines* lines, double mass_amu, double P_bar, double T, float* gamma_G_out,
                    float* gamma_L_out, void* stream) {
  int rc = check_lines(lines, false, true);
  if (rc) return rc;
  if (!finite_pos(mass_amu) || !finite_pos(T) || !std::isfinite(P_bar) || P_bar < 0)
    return fail(ROX_EINVAL, "mass > 0, T > 0, P >= 0 required");
  if (lines->n > 0 && (!gamma_G_out || !gamma_L_out)) return fail(ROX_EINVAL, "output is NULL");
  if (lines->n == 0) return ok();
  rc = cuda_check(rox_launch_widths(lines, mass_amu, P_bar, T, gamma_G_out, gamma_L_out, (cudaStream_t)stream),
                  "widths kernel");
  return rc ? rc : ok();
}

size_t rox_sort_workspace_size(int64_t n) { return n <= 0 ? 256 : rox_sort_ws_bytes(n); }

int rox_sort_lines(const rox_lines* in, const rox_lines_buf* out, int64_t* perm_out, void* ws, size_t ws_bytes,
                   void* stream) {
  int rc = check_lines(in, true, true);
  if (rc) return rc;
  if (!out || !out->nu0 || !out->s_or_a || !out->e_lower || !out->gamma_ref || !out->n_t ||
      (in->convention == ROX_EXOMOL && !out->g_up))
    return fail(ROX_EINVAL, "sort output buffers missing");
  if (in->n == 0) return ok();
  if (!ws || ws_bytes < rox_sort_workspace_size(in->n)) return fail(ROX_ENOMEM, "sort workspace too small");
  rc = cuda_check(rox_launch_sort(in, out, perm_out, ws, (cudaStream_t)stream), "sort");
  return rc ? rc : ok();
}

int rox_line_windows(const double* nu0_sorted, int64_t n_lines, const rox_grid* grid, double cutoff, int32_t* jlo,
                     int32_t* jhi, int32_t* k0, float* f, unsigned long long* evals_out, int32_t* unsorted_out,
                     void* stream) {
  int rc = check_grid(grid);
  if (rc) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  if (n_lines < 0 || (n_lines > 0 && !nu0_sorted)) return fail(ROX_EINVAL, "nu0/n_lines invalid");
  if (n_lines == 0) return ok();
  rc = cuda_check(rox_launch_windows(nu0_sorted, n_lines, grid, cutoff, jlo, jhi, k0, f, nullptr, evals_out,
                                     unsorted_out, 1, (cudaStream_t)stream),
                  "windows kernel");
  return rc ? rc : ok();
}

int rox_tile_ranges(const int32_t* jlo, const int32_t* jhi, int64_t n_lines, int64_t n_grid, int32_t tile_pts,
                    int64_t* lo_out, int64_t* hi_out, void* stream) {
  if (n_lines < 0 || n_grid <= 0 || tile_pts <= 0) return fail(ROX_EINVAL, "sizes invalid");
  if (!lo_out || !hi_out || (n_lines > 0 && (!jlo || !jhi))) return fail(ROX_EINVAL, "NULL pointer");
  long long nt = (n_grid + tile_pts - 1) / tile_pts;
  int rc = cuda_check(rox_launch_tile_ranges(jlo, jhi, n_lines, nt, tile_pts, (long long*)lo_out, (long long*)hi_out,
                                             (cudaStream_t)stream),
                      "tile ranges kernel");
  return rc ? rc : ok();
}

int rox_faddeeva_re(const float* x, const float* y, float* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!x || !y || !out))) return fail(ROX_EINVAL, "invalid arguments");
  if (n == 0) return ok();
  int rc = cuda_check(rox_launch_faddeeva(x, y, out, n, (cudaStream_t)stream), "faddeeva kernel");
  return rc ? rc : ok();
}

size_t rox_xsec_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps) {
  if (!grid || grid->n <= 0 || n_lines < 0 || n_temps <= 0) return 0;
  return ws_layout(nullptr, n_lines, grid->n, n_temps).bytes;
}

int rox_xsec_batch(const rox_lines* lines, const rox_grid* grid, int n_pt, const double* P_bar, const double* T,
                   const double* Q_T, double Q_ref, double mass_amu, double cutoff, unsigned flags, float* sigma_out,
                   void* ws, size_t ws_bytes, void* stream) {
  int rc = check_lines(lines, true, true);
  if (rc) return rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  if (n_pt < 1 || n_pt > ROX_MAX_PT) return fail(ROX_EINVAL, "n_pt = %d outside [1, %d]", n_pt, ROX_MAX_PT);
  if (!P_bar || !T || !Q_T) return fail(ROX_EINVAL, "P_bar, T, Q_T host arrays required");
  if (!finite_pos(Q_ref) || !finite_pos(mass_amu)) return fail(ROX_EINVAL, "Q_ref and mass must be > 0");
  if (flags & ~ROX_ACCUMULATE) return fail(ROX_EINVAL, "unknown flags 0x%x", flags);
  if (!sigma_out) return fail(ROX_EINVAL, "sigma_out is NULL");
  // distinct temperatures (S(T) is computed once per temperature)
  std::vector<double> temps, qs;
  std::vector<int> tidx(n_pt);
  for (int k = 0; k < n_pt; k++) {
    if (!finite_pos(T[k]) || !finite_pos(Q_T[k]) || !std::isfinite(P_bar[k]) || P_bar[k] < 0)
      return fail(ROX_EINVAL, "point %d: T > 0, Q_T > 0, P >= 0 required", k);
    int found = -1;
    for (size_t u = 0; u < temps.size(); u++)
      if (temps[u] == T[k]) { found = (int)u; break; }
    if (found < 0) {
      found = (int)temps.size();
      temps.push_back(T[k]);
      qs.push_back(Q_T[k]);
    } else if (qs[found] != Q_T[k]) {
      return fail(ROX_EINVAL, "point %d: Q_T differs from an earlier point at the same T", k);
    }
    tidx[k] = found;
  }
  const int n_temps = (int)temps.size();
  if (!ws || ((uintptr_t)ws & 255)) return fail(ROX_EINVAL, "workspace NULL or not 256-byte aligned");
  WsLayout w = ws_layout(ws, lines->n, grid->n, n_temps);
  if (ws_bytes < w.bytes) return fail(ROX_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.bytes);

  cudaStream_t s = (cudaStream_t)stream;
  int nblocks = 0;
  if ((rc = voigt_grid(&nblocks))) return rc;
  const long long nt = n_tiles_of(grid->n);
  const long long nl = lines->n;

  static thread_local RoxVoigtArgs A;   // 8 KB of per-point parameters, passed by value
  A.geo = w.geo;
  A.S32 = w.S32;
  A.gamma_ref = lines->gamma_ref;
  A.n_t = lines->n_t;
  A.width_f16 = lines->width_dtype == ROX_WIDTH_F16;
  A.tile_lo = w.tlo;
  A.tile_hi = w.thi;
  A.n_tiles = (int32_t)nt;
  A.n_pt = n_pt;
  A.n_lines = nl;
  A.n_grid = grid->n;
  A.nu_min = grid->nu_min;
  A.dnu_f = (float)grid->dnu;
  A.nu_min_f = (float)grid->nu_min;
  A.hdr = w.hdr;
  A.sigma = sigma_out;
  A.flags = flags;
  for (int k = 0; k < n_pt; k++) {
    A.pt[k].p_fac = (float)(P_bar[k] / ROX_P_REF);
    A.pt[k].gG_fac = (float)(sqrt(2.0 * ROX_KB * T[k] / (mass_amu * ROX_AMU)) / ROX_C_M);
    A.pt[k].l2_ratio = (float)log2(ROX_T_REF / T[k]);
    A.pt[k].t_idx = tidx[k];
  }

  if ((rc = cuda_check(cudaMemsetAsync(w.hdr, 0, sizeof(RoxWsHeader), s), "memset"))) return rc;
  if (nl > 0) {
    if ((rc = cuda_check(rox_launch_windows(lines->nu0, nl, grid, cutoff, nullptr, nullptr, nullptr, nullptr, w.geo,
                                            &w.hdr->evals_lines, &w.hdr->status, ROX_EUNSORTED, s),
                         "windows kernel")))
      return rc;
    if ((rc = cuda_check(rox_launch_strengths_multi(lines, n_temps, temps.data(), qs.data(), Q_ref, w.S_T,
                                                    w.hdr->smax_bits, s),
                         "strengths kernel")))
      return rc;
    if ((rc = cuda_check(rox_launch_scale_strengths(w.S_T, nl, n_temps, w.hdr->smax_bits, w.S32, s),
                         "strength scaling kernel")))
      return rc;
  }
  if ((rc = cuda_check(rox_launch_tile_ranges_geo(w.geo, nl, nt, ROX_TILE, w.tlo, w.thi, s), "tile ranges")))
    return rc;
  long long items = (long long)n_pt * nt;
  int grid_blocks = (int)(items < nblocks ? items : nblocks);
  if (g_prof_start && (rc = cuda_check(cudaEventRecord(g_prof_start, s), "cudaEventRecord"))) return rc;
  if ((rc = cuda_check(rox_launch_voigt(A, grid_blocks, s), "voigt kernel"))) return rc;
  if (g_prof_stop && (rc = cuda_check(cudaEventRecord(g_prof_stop, s), "cudaEventRecord"))) return rc;
  return ok();
}

int rox_xsec(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T, double Q_ref,
             double mass_amu, double cutoff, float* sigma_out, void* ws, size_t ws_bytes, void* stream) {
  return rox_xsec_batch(lines, grid, 1, &P_bar, &T, &Q_T, Q_ref, mass_amu, cutoff, 0u, sigma_out, ws, ws_bytes,
                        stream);
}

int rox_set_profile_events(void* start, void* stop) {
  if ((start == nullptr) != (stop == nullptr)) return fail(ROX_EINVAL, "give both events or neither");
  g_prof_start = (cudaEvent_t)start;
  g_prof_stop = (cudaEvent_t)stop;
  return ok();
}

int rox_ws_status(const void* ws, unsigned long long* evals_out, void* stream) {
  if (!ws) return fail(ROX_EINVAL, "workspace is NULL");
  int rc = cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  if (rc) return rc;
  RoxWsHeader h;
  rc = cuda_check(cudaMemcpy(&h, ws, offsetof(RoxWsHeader, smax_bits), cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (rc) return rc;
  if (evals_out) *evals_out = h.evals_total;
  if (h.status == ROX_EUNSORTED) return fail(ROX_EUNSORTED, "line list is not sorted by ascending nu0");
  if (h.status == ROX_ETIMEOUT) return fail(ROX_ETIMEOUT, "a device-side wait ran out");
  if (h.status != ROX_OK) return fail(h.status, "device status %d", h.status);
  return ok();
}

}  // extern "C"
