// C ABI of librox (include/rox.h): argument checks, workspace layout, launch order.
// Everything after the checks is enqueued on the caller's stream; nothing here
// allocates device memory or synchronises, except rox_ws_status.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include "rox_internal.cuh"

// kernels (rox_params.cu, rox_geometry.cu, rox_voigt.cu)
cudaError_t rox_launch_strengths(const rox_lines* L, double T, double Q_T, double Q_ref, float* S_out,
                                 cudaStream_t s);
cudaError_t rox_launch_strengths_reduced(const rox_lines* L, double T, double Q_T, double Q_ref, double* S_out,
                                         cudaStream_t s);
cudaError_t rox_launch_widths(const rox_lines* L, double mass_amu, double P_bar, double T, float* gG,
                              float* gL, cudaStream_t s);
cudaError_t rox_launch_strengths_multi(const rox_lines* L, int n_temps, const double* temps,
                                       const double* q_of_temp, double Q_ref, double* S_T,
                                       unsigned long long* smax_bits, bool exact, cudaStream_t s);
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
cudaError_t rox_launch_voigt(const RoxVoigtArgs& A, int n_blocks, bool nodes, int extras, int warps, cudaStream_t s);
cudaError_t rox_launch_node_windows(const double* nu0, long long n_lines, const double* nodes, long long n,
                                    double cutoff, int32_t* jlo, int32_t* jhi, float4* geo,
                                    unsigned long long* evals, int32_t* unsorted, int32_t unsorted_value,
                                    cudaStream_t s);
cudaError_t rox_launch_node_offsets(const double* nodes, long long n, long long n_pad, float2* d, float2* base,
                                    int32_t* status, int32_t bad_value, cudaStream_t s);
void rox_fill_strength_consts(int convention, double T, double Q_T, double Q_ref, RoxStrengthJob* jb);
cudaError_t rox_launch_strengths_jobs(const RoxStrengthJobs& J, long long max_count, cudaStream_t s);
cudaError_t rox_voigt_blocks_per_sm(int* nb, bool nodes, bool pre, int warps);
cudaError_t rox_launch_line_params(const RoxListDev& L, const RoxJobDev& J, float4* rec, cudaStream_t s);
cudaError_t rox_launch_select(const double* nu0, const double* S_T, long long n, int n_temps,
                              const unsigned long long* smax_bits, double origin, double width, long long n_bins,
                              double rel, int32_t* bin, unsigned long long* binmax_bits, float* S32, cudaStream_t s);
cudaError_t rox_launch_select_reduced(const rox_lines* L, int n_temps, const double* temps, const double* q_of_temp,
                                      double Q_ref, double* S_T, const unsigned long long* smax_bits, double origin,
                                      double width, long long n_bins, double rel, int32_t* bin,
                                      unsigned long long* binmax_fast, unsigned long long* binmax_exact, float* S32,
                                      cudaStream_t s);
cudaError_t rox_launch_broad_T(const RoxBroadDev& B, const float* a_coef, long long n, int n_temps,
                               const double* temps, float* G, float* gN, cudaStream_t s);
cudaError_t rox_launch_lorentz_out(const RoxBroadDev& B, const float* a_coef, long long n, double P_bar, double T,
                                   float* out, cudaStream_t s);
size_t rox_compact_temp_bytes(long long n);
cudaError_t rox_launch_compact(const float* S32_all, long long n, int n_temps, uint8_t* flags, int32_t* idx,
                               long long* counts, void* temp, size_t temp_bytes, cudaStream_t s);
cudaError_t rox_launch_tile_ranges_idx(const float4* geo, const int32_t* idx, const long long* count, long long n_max,
                                       long long n_tiles, int32_t W, long long* lo, long long* hi, cudaStream_t s);
cudaError_t rox_launch_keep_flags(const double* S_T, const int32_t* bin, const unsigned long long* binmax_bits,
                                  long long n, double rel, uint8_t* keep, cudaStream_t s);
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

int check_nodes(const rox_nodes* g) {
  if (!g || !g->nu) return fail(ROX_EINVAL, "nodes or nodes->nu is NULL");
  if (g->n <= 0) return fail(ROX_EINVAL, "nodes->n = %lld <= 0", (long long)g->n);
  if (g->n > ROX_MAX_GRID) return fail(ROX_ERANGE, "nodes->n = %lld above %d", (long long)g->n, ROX_MAX_GRID);
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
  float* tail_part;
  int32_t* tail_cnt;
  long long tail_cap;
  float2* node_d;      // user-provided nodes only: [n_tiles * ROX_SPAN] offsets, [n_tiles] bases
  float2* span_base;
  int32_t* line_bin;   // main-contributor selection only: [n_lines] bins, [n_temps][n_bins] maxima,
  unsigned long long* binmax;
  unsigned long long* binmax_exact;   // selection on reduced-form strengths: exact bin maxima
  uint8_t* keep_flags; //   per temperature the keep flags, the kept lines' indices and count, the span
  int32_t* keep_idx;   //   ranges over those indices, and the compaction's scratch
  long long* keep_count;
  long long* keep_lo;
  long long* keep_hi;
  void* compact_tmp;
  size_t compact_tmp_bytes;
  float* broad_G;      // broadening descriptions only: [n_temps][n_lines] broadeners' sums, [n_lines]
  float* broad_N;      //   natural widths
  float4* rec;         // one temperature on a uniform grid: per line 3 float4 of per-line constants
  size_t bytes;
};

WsLayout ws_layout(void* ws, long long n_lines, long long n_grid, int n_temps, bool nodes = false,
                   long long n_bins = 0, bool broad = false, long long tail_max = ROX_TAIL_ITEMS_MAX,
                   bool pre = true) {
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
  w.tail_cap = nt < tail_max ? nt : tail_max;
  w.tail_part = (float*)(base + off);
  w.tail_cnt = (int32_t*)(base + off + rox_align256((size_t)w.tail_cap * ROX_PARTS * ROX_SPAN * sizeof(float)));
  off += rox_tail_bytes(w.tail_cap);
  w.node_d = nullptr;
  w.span_base = nullptr;
  if (nodes) {
    w.node_d = (float2*)(base + off);
    off += rox_align256((size_t)nt * ROX_SPAN * sizeof(float2));
    w.span_base = (float2*)(base + off);
    off += rox_align256((size_t)nt * sizeof(float2));
  }
  w.line_bin = nullptr;
  w.binmax = nullptr;
  w.binmax_exact = nullptr;
  w.keep_flags = nullptr;
  w.keep_idx = nullptr;
  w.keep_count = nullptr;
  w.keep_lo = nullptr;
  w.keep_hi = nullptr;
  w.compact_tmp = nullptr;
  w.compact_tmp_bytes = 0;
  if (n_bins > 0) {
    w.line_bin = (int32_t*)(base + off);
    off += rox_align256((size_t)(n_lines > 0 ? n_lines : 1) * 4);
    w.binmax = (unsigned long long*)(base + off);
    off += rox_align256((size_t)n_temps * (size_t)n_bins * 8);
    w.binmax_exact = (unsigned long long*)(base + off);
    off += rox_align256((size_t)n_temps * (size_t)n_bins * 8);
    const size_t nl = (size_t)(n_lines > 0 ? n_lines : 1);
    w.keep_flags = (uint8_t*)(base + off);
    off += rox_align256((size_t)n_temps * nl);
    w.keep_idx = (int32_t*)(base + off);
    off += rox_align256((size_t)n_temps * nl * 4);
    w.keep_count = (long long*)(base + off);
    off += rox_align256((size_t)n_temps * 8);
    w.keep_lo = (long long*)(base + off);
    off += rox_align256((size_t)n_temps * (size_t)nt * 8);
    w.keep_hi = (long long*)(base + off);
    off += rox_align256((size_t)n_temps * (size_t)nt * 8);
    w.compact_tmp_bytes = rox_compact_temp_bytes(n_lines);
    w.compact_tmp = base + off;
    off += rox_align256(w.compact_tmp_bytes);
  }
  w.broad_G = nullptr;
  w.broad_N = nullptr;
  if (broad) {
    const size_t nl = (size_t)(n_lines > 0 ? n_lines : 1);
    w.broad_G = (float*)(base + off);
    off += rox_align256((size_t)n_temps * nl * 4);
    w.broad_N = (float*)(base + off);
    off += rox_align256(nl * 4);
  }
  w.rec = nullptr;
  if (pre && n_temps == 1 && !nodes && n_bins == 0 && !broad) {
    w.rec = (float4*)(base + off);
    off += rox_align256((size_t)(n_lines > 0 ? n_lines : 1) * 3 * sizeof(float4));
  }
  w.bytes = off;
  return w;
}

// a rox_broadening checked and put in kernel form
int check_broadening(const rox_broadening* br, const rox_lines* L, RoxBroadDev* out) {
  if (!br) return fail(ROX_EINVAL, "broadening is NULL");
  if (br->n_broadeners < 1 || br->n_broadeners > ROX_MAX_BROADENERS)
    return fail(ROX_EINVAL, "n_broadeners = %d outside [1, %d]", br->n_broadeners, ROX_MAX_BROADENERS);
  if (br->natural && L->convention != ROX_EXOMOL)
    return fail(ROX_EINVAL, "natural broadening needs Einstein A (ExoMol lists)");
  if (br->natural && L->n > 0 && !L->s_or_a) return fail(ROX_EINVAL, "natural broadening needs lines->s_or_a");
  bool tables = false;
  RoxBroadDev B;
  memset(&B, 0, sizeof B);
  B.n_b = br->n_broadeners;
  B.natural = br->natural ? 1 : 0;
  B.f16 = L->width_dtype == ROX_WIDTH_F16;
  for (int b = 0; b < br->n_broadeners; b++) {
    if (!std::isfinite(br->vmr[b]) || br->vmr[b] < 0.0) return fail(ROX_EINVAL, "broadener %d: vmr must be >= 0", b);
    B.vmr[b] = (float)br->vmr[b];
    if (br->table_gamma[b]) {
      if (!br->table_n[b]) return fail(ROX_EINVAL, "broadener %d: table_n is NULL", b);
      tables = true;
      B.tab_gamma[b] = br->table_gamma[b];
      B.tab_n[b] = br->table_n[b];
    } else {
      if (L->n > 0 && (!br->gamma_ref[b] || !br->n_t[b]))
        return fail(ROX_EINVAL, "broadener %d: gamma_ref / n_t columns or a table required", b);
      B.gamma[b] = br->gamma_ref[b];
      B.n[b] = br->n_t[b];
    }
  }
  if (tables) {
    if (br->table_len < 1) return fail(ROX_EINVAL, "table_len must be >= 1");
    if (L->n > 0 && !br->j_lower) return fail(ROX_EINVAL, "j_lower is required with tables");
    B.j_lower = br->j_lower;
    B.tab_len = br->table_len;
  }
  *out = B;
  return ROX_OK;
}

// main-contributor selection bins of a uniform grid: origin nu_min - cutoff, width B
int select_bins(const rox_select* sel, const rox_grid* g, double cutoff, double* origin, long long* n_bins) {
  if (!sel) return fail(ROX_EINVAL, "selection is NULL");
  if (!std::isfinite(sel->rel) || sel->rel < 0.0) return fail(ROX_EINVAL, "selection rel must be >= 0");
  if (!finite_pos(sel->bin_width)) return fail(ROX_EINVAL, "selection bin_width must be > 0");
  const double nb = std::floor(((double)(g->n - 1) * g->dnu + 2.0 * cutoff) / sel->bin_width) + 1.0;
  if (!(nb <= (double)ROX_MAX_SELECT_BINS))
    return fail(ROX_ERANGE, "%g selection bins above %d (bin_width too small)", nb, ROX_MAX_SELECT_BINS);
  *origin = g->nu_min - cutoff;
  *n_bins = (long long)nb;
  return ROX_OK;
}

// Launch configuration of the Voigt kernel (rox_set_launch_config): warps per CTA, CTAs per SM
// (0: as many as fit), rounds of warps' worth of items split into parts at the end of a launch.
// None of them changes a result.
std::mutex g_cfg_mu;
rox_launch_config g_cfg = {8, 0, 1, 0};
rox_launch_config launch_config() {
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  return g_cfg;
}

// resident CTAs per SM of each instantiation (uniform grid, nodes, precomputed per-line
// constants) and warps per CTA (4, 8) on the current device
int g_voigt_per_sm[3][2] = {{0, 0}, {0, 0}, {0, 0}};
int g_voigt_sms[3][2] = {{0, 0}, {0, 0}, {0, 0}};
int g_voigt_device[3][2] = {{-1, -1}, {-1, -1}, {-1, -1}};

// persistent grid of the Voigt kernel on the current device for the launch configuration cfg
int voigt_grid(int* out, const rox_launch_config& cfg, bool nodes = false, bool pre = false) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(e, "cudaGetDevice");
  const int v = pre ? 2 : (nodes ? 1 : 0), wi = cfg.warps_per_cta == 4 ? 0 : 1;
  if (dev != g_voigt_device[v][wi]) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check(e, "cudaDeviceGetAttribute");
    e = rox_voigt_blocks_per_sm(&per, nodes, pre, cfg.warps_per_cta);
    if (e != cudaSuccess) return cuda_check(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    g_voigt_per_sm[v][wi] = per > 0 ? per : 1;
    g_voigt_sms[v][wi] = sms;
    g_voigt_device[v][wi] = dev;
  }
  int per = g_voigt_per_sm[v][wi];
  if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per) per = cfg.ctas_per_sm;
  *out = g_voigt_sms[v][wi] * per;
  return ROX_OK;
}

// Voigt launches over the jobs, at most ROX_MAX_JOBS per launch; the work counter is reset
// before each launch (the evaluation count keeps adding up). The last items of each launch,
// up to tail_cap and half a round of the launch's warps, are split into their parts.
int launch_voigt_jobs(const RoxListDev* lists, int n_lists, const RoxJobDev* jobs, int n_jobs, RoxWsHeader* hdr,
                      float* tail_part, int32_t* tail_cnt, long long tail_cap, int nblocks, cudaStream_t s,
                      const rox_launch_config& cfg, bool nodes = false, int extras = 0) {
  static thread_local RoxVoigtArgs A;   // ~30 KB of per-job parameters, passed by value
  A.hdr = hdr;
  A.tail_part = tail_part;
  A.tail_cnt = tail_cnt;
  for (int l = 0; l < n_lists; l++) A.list[l] = lists[l];
  for (int j0 = 0; j0 < n_jobs; j0 += ROX_MAX_JOBS) {
    const int nj = (n_jobs - j0) < ROX_MAX_JOBS ? (n_jobs - j0) : ROX_MAX_JOBS;
    int items = 0;
    for (int k = 0; k < nj; k++) {
      A.job[k] = jobs[j0 + k];
      items += A.job[k].n_spans;
      A.item_end[k] = items;
    }
    const int blocks = items < nblocks ? items : nblocks;
    // whole items in complete rounds of the launch's warps, then at least one round of items in
    // parts, so the launch ends in pieces of 1/ROX_PARTS of an item
    const long long warps = (long long)blocks * cfg.warps_per_cta;
    long long split = items <= warps ? items : items % warps + (long long)cfg.split_rounds * warps;
    if (split > items) split = items;
    if (split > tail_cap) split = tail_cap;
    A.n_jobs = nj;
    A.n_items = items;
    A.n_whole = items - (int)split;
    A.n_queue = A.n_whole + (int)split * ROX_PARTS;
    int rc;
    if ((rc = cuda_check(cudaMemsetAsync(&hdr->work_counter, 0, sizeof(int32_t), s), "memset"))) return rc;
    if (split > 0 && (rc = cuda_check(cudaMemsetAsync(tail_cnt, 0, (size_t)split * 4, s), "memset"))) return rc;
    if (j0 == 0 && g_prof_start && (rc = cuda_check(cudaEventRecord(g_prof_start, s), "cudaEventRecord"))) return rc;
    if (items == 0) continue;
    if ((rc = cuda_check(rox_launch_voigt(A, blocks, nodes, extras, cfg.warps_per_cta, s), "voigt kernel"))) return rc;
  }
  if (g_prof_stop) return cuda_check(cudaEventRecord(g_prof_stop, s), "cudaEventRecord");
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

int rox_line_strengths_reduced(const rox_lines* lines, double T, double Q_T, double Q_ref, double* S_out,
                               void* stream) {
  int rc = check_lines(lines, true, false);
  if (rc) return rc;
  if (!finite_pos(T) || !finite_pos(Q_T) || !finite_pos(Q_ref)) return fail(ROX_EINVAL, "T, Q_T, Q_ref must be > 0");
  if (lines->n > 0 && !S_out) return fail(ROX_EINVAL, "S_out is NULL");
  if (lines->n == 0) return ok();
  rc = cuda_check(rox_launch_strengths_reduced(lines, T, Q_T, Q_ref, S_out, (cudaStream_t)stream),
                  "strengths kernel");
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

}  // extern "C"

namespace {
// rox_xsec_batch and rox_xsec_nodes_batch: `grid` (uniform) or `nodes` (user-provided), the
// other NULL; both checked by the caller.
int xsec_batch_impl(const rox_lines* lines, const rox_grid* grid, const rox_nodes* nodes, int n_pt,
                    const double* P_bar, const double* T, const double* Q_T, double Q_ref, double mass_amu,
                    double cutoff, unsigned flags, float* sigma_out, void* ws, size_t ws_bytes, void* stream,
                    const rox_select* sel = nullptr, const rox_broadening* br = nullptr,
                    long long tail_max = ROX_TAIL_ITEMS_MAX, bool allow_pre = true) {
  int rc = check_lines(lines, true, br == nullptr);
  if (rc) return rc;
  RoxBroadDev bdev;
  if (br && (rc = check_broadening(br, lines, &bdev))) return rc;
  const bool on_nodes = nodes != nullptr;
  double sel_origin = 0.0;
  long long n_bins = 0;
  if (sel && (rc = select_bins(sel, grid, cutoff, &sel_origin, &n_bins))) return rc;
  const long long n_grid = on_nodes ? nodes->n : grid->n;
  if (n_pt < 1 || n_pt > ROX_MAX_PT) return fail(ROX_EINVAL, "n_pt = %d outside [1, %d]", n_pt, ROX_MAX_PT);
  if (!P_bar || !T || !Q_T) return fail(ROX_EINVAL, "P_bar, T, Q_T host arrays required");
  if (!finite_pos(Q_ref) || !finite_pos(mass_amu)) return fail(ROX_EINVAL, "Q_ref and mass must be > 0");
  if (flags & ~(ROX_ACCUMULATE | ROX_KAHAN)) return fail(ROX_EINVAL, "unknown flags 0x%x", flags);
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
  WsLayout w = ws_layout(ws, lines->n, n_grid, n_temps, on_nodes, n_bins, br != nullptr, tail_max, allow_pre);
  // one (P,T) point on a uniform grid: the per-line constants once per line (k_line_params)
  const bool pre = w.rec != nullptr && n_pt == 1 && lines->n > 0;
  if (ws_bytes < w.bytes) return fail(ROX_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.bytes);

  cudaStream_t s = (cudaStream_t)stream;
  const rox_launch_config cfg = launch_config();
  int nblocks = 0;
  if ((rc = voigt_grid(&nblocks, cfg, on_nodes, pre))) return rc;
  const long long nt = n_tiles_of(n_grid);
  const long long nl = lines->n;

  if ((rc = cuda_check(cudaMemsetAsync(w.hdr, 0, sizeof(RoxWsHeader), s), "memset"))) return rc;
  if (on_nodes &&
      (rc = cuda_check(rox_launch_node_offsets(nodes->nu, nodes->n, nt * ROX_SPAN, w.node_d, w.span_base,
                                               &w.hdr->status, ROX_EGRID, s),
                       "node offsets kernel")))
    return rc;
  if (nl > 0) {
    const cudaError_t we =
        on_nodes ? rox_launch_node_windows(lines->nu0, nl, nodes->nu, nodes->n, cutoff, nullptr, nullptr, w.geo,
                                           &w.hdr->evals_lines, &w.hdr->status, ROX_EUNSORTED, s)
                 : rox_launch_windows(lines->nu0, nl, grid, cutoff, nullptr, nullptr, nullptr, nullptr, w.geo,
                                      &w.hdr->evals_lines, &w.hdr->status, ROX_EUNSORTED, s);
    if ((rc = cuda_check(we, "windows kernel"))) return rc;
    if ((rc = cuda_check(rox_launch_strengths_multi(lines, n_temps, temps.data(), qs.data(), Q_ref, w.S_T,
                                                    w.hdr->smax_bits, false, s),
                         "strengths kernel")))
      return rc;
    const cudaError_t se =
        sel ? rox_launch_select_reduced(lines, n_temps, temps.data(), qs.data(), Q_ref, w.S_T, w.hdr->smax_bits,
                                        sel_origin, sel->bin_width, n_bins, sel->rel, w.line_bin, w.binmax,
                                        w.binmax_exact, w.S32, s)
            : rox_launch_scale_strengths(w.S_T, nl, n_temps, w.hdr->smax_bits, w.S32, s);
    if ((rc = cuda_check(se, "strength scaling kernel"))) return rc;
    if (sel) {
      // per temperature the kept lines as an index into the sorted list, and span ranges over it
      if ((rc = cuda_check(rox_launch_compact(w.S32, nl, n_temps, w.keep_flags, w.keep_idx, w.keep_count,
                                              w.compact_tmp, w.compact_tmp_bytes, s),
                           "selection compaction")))
        return rc;
      for (int t = 0; t < n_temps; t++)
        if ((rc = cuda_check(rox_launch_tile_ranges_idx(w.geo, w.keep_idx + (size_t)t * nl, w.keep_count + t, nl, nt,
                                                        ROX_TILE, w.keep_lo + (size_t)t * nt,
                                                        w.keep_hi + (size_t)t * nt, s),
                             "selection span ranges")))
          return rc;
    }
    if (br && (rc = cuda_check(rox_launch_broad_T(bdev, lines->s_or_a, nl, n_temps, temps.data(), w.broad_G,
                                                  bdev.natural ? w.broad_N : nullptr, s),
                               "broadening kernel")))
      return rc;
  }
  if ((rc = cuda_check(rox_launch_tile_ranges_geo(w.geo, nl, nt, ROX_TILE, w.tlo, w.thi, s), "tile ranges")))
    return rc;
  RoxListDev L0;
  L0.status = &w.hdr->status;
  L0.geo = w.geo;
  L0.span_lo = w.tlo;
  L0.span_hi = w.thi;
  L0.gamma_ref = lines->gamma_ref;
  L0.n_t = lines->n_t;
  L0.gLT = br ? w.broad_G : nullptr;
  L0.gLT_stride = nl > 0 ? nl : 1;
  L0.gN = (br && bdev.natural) ? w.broad_N : nullptr;
  L0.node_d = w.node_d;
  L0.span_base = w.span_base;
  L0.n_lattice = n_grid;
  L0.dnu_f = on_nodes ? 0.0f : (float)grid->dnu;
  L0.nu_min_f = on_nodes ? 0.0f : (float)grid->nu_min;
  L0.width_f16 = lines->width_dtype == ROX_WIDTH_F16;
  L0.idx = nullptr;
  L0.inv_dnu_f = on_nodes ? 0.0f : (float)(1.0 / grid->dnu);
  L0.rec = pre ? w.rec : nullptr;
  std::vector<RoxJobDev> jobs(n_pt);
  for (int k = 0; k < n_pt; k++) {
    RoxJobDev& J = jobs[k];
    J.S32 = w.S32 + (size_t)tidx[k] * (size_t)(nl > 0 ? nl : 1);
    J.sigma = sigma_out + (size_t)k * (size_t)n_grid;
    J.smax_bits = &w.hdr->smax_bits[tidx[k]];
    J.l0 = 0;
    J.l1 = nl;
    J.first = 0;
    J.n = n_grid;
    J.list = 0;
    J.span_first = 0;
    J.n_spans = (int32_t)nt;
    J.p_fac = (float)(P_bar[k] / ROX_P_REF);
    J.gG_fac = (float)(sqrt(2.0 * ROX_KB * T[k] / (mass_amu * ROX_AMU)) / ROX_C_M);
    J.l2_ratio = (float)log2(ROX_T_REF / T[k]);
    J.flags = flags;
    J.t_row = tidx[k];
  }
  if (sel && nl > 0) {
    // one list per temperature (its kept lines), launches of up to ROX_MAX_LISTS temperatures
    for (int g0 = 0; g0 < n_temps; g0 += ROX_MAX_LISTS) {
      const int ng = (n_temps - g0) < ROX_MAX_LISTS ? (n_temps - g0) : ROX_MAX_LISTS;
      RoxListDev Ls[ROX_MAX_LISTS];
      for (int l = 0; l < ng; l++) {
        Ls[l] = L0;
        Ls[l].idx = w.keep_idx + (size_t)(g0 + l) * nl;
        Ls[l].span_lo = w.keep_lo + (size_t)(g0 + l) * nt;
        Ls[l].span_hi = w.keep_hi + (size_t)(g0 + l) * nt;
      }
      std::vector<RoxJobDev> jg;
      for (int k = 0; k < n_pt; k++)
        if (tidx[k] >= g0 && tidx[k] < g0 + ng) {
          jg.push_back(jobs[k]);
          jg.back().list = tidx[k] - g0;
        }
      if ((rc = launch_voigt_jobs(Ls, ng, jg.data(), (int)jg.size(), w.hdr, w.tail_part, w.tail_cnt, w.tail_cap,
                                  nblocks, s, cfg, false, ROX_VX_INDEX)))
        return rc;
    }
    return ok();
  }
  if (pre && (rc = cuda_check(rox_launch_line_params(L0, jobs[0], w.rec, s), "line parameter kernel"))) return rc;
  const int extras = br ? ROX_VX_BROAD : (pre ? ROX_VX_PRE : 0);
  if ((rc = launch_voigt_jobs(&L0, 1, jobs.data(), n_pt, w.hdr, w.tail_part, w.tail_cnt, w.tail_cap, nblocks, s,
                              cfg, on_nodes, extras)))
    return rc;
  return ok();
}
}  // namespace

extern "C" {

int rox_xsec_batch(const rox_lines* lines, const rox_grid* grid, int n_pt, const double* P_bar, const double* T,
                   const double* Q_T, double Q_ref, double mass_amu, double cutoff, unsigned flags, float* sigma_out,
                   void* ws, size_t ws_bytes, void* stream) {
  int rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  return xsec_batch_impl(lines, grid, nullptr, n_pt, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, flags, sigma_out, ws,
                         ws_bytes, stream);
}

size_t rox_xsec_broadened_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps) {
  if (!grid || grid->n <= 0 || n_lines < 0 || n_temps <= 0) return 0;
  return ws_layout(nullptr, n_lines, grid->n, n_temps, false, 0, true).bytes;
}

int rox_xsec_broadened_batch(const rox_lines* lines, const rox_grid* grid, const rox_broadening* br, int n_pt,
                             const double* P_bar, const double* T, const double* Q_T, double Q_ref, double mass_amu,
                             double cutoff, unsigned flags, float* sigma_out, void* ws, size_t ws_bytes,
                             void* stream) {
  int rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  if (!br) return fail(ROX_EINVAL, "broadening is NULL");
  return xsec_batch_impl(lines, grid, nullptr, n_pt, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, flags, sigma_out, ws,
                         ws_bytes, stream, nullptr, br);
}

int rox_lorentz_widths(const rox_lines* lines, const rox_broadening* br, double P_bar, double T, float* gamma_L_out,
                       void* stream) {
  int rc = check_lines(lines, false, false);
  if (rc) return rc;
  RoxBroadDev B;
  if ((rc = check_broadening(br, lines, &B))) return rc;
  if (!finite_pos(T) || !std::isfinite(P_bar) || P_bar < 0) return fail(ROX_EINVAL, "T > 0 and P >= 0 required");
  if (!gamma_L_out) return fail(ROX_EINVAL, "gamma_L_out is NULL");
  if (lines->n == 0) return ok();
  if ((rc = cuda_check(rox_launch_lorentz_out(B, lines->s_or_a, lines->n, P_bar, T, gamma_L_out,
                                              (cudaStream_t)stream),
                       "Lorentz widths kernel")))
    return rc;
  return ok();
}

size_t rox_xsec_select_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps, double cutoff,
                                      const rox_select* sel) {
  if (!grid || grid->n <= 0 || n_lines < 0 || n_temps <= 0 || !sel || !finite_pos(sel->bin_width) ||
      !finite_pos(cutoff))
    return 0;
  double origin;
  long long n_bins;
  if (select_bins(sel, grid, cutoff, &origin, &n_bins)) return 0;
  return ws_layout(nullptr, n_lines, grid->n, n_temps, false, n_bins).bytes;
}

int rox_xsec_select_batch(const rox_lines* lines, const rox_grid* grid, int n_pt, const double* P_bar,
                          const double* T, const double* Q_T, double Q_ref, double mass_amu, double cutoff,
                          unsigned flags, const rox_select* sel, float* sigma_out, void* ws, size_t ws_bytes,
                          void* stream) {
  int rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  if (!sel) return fail(ROX_EINVAL, "selection is NULL");
  return xsec_batch_impl(lines, grid, nullptr, n_pt, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, flags, sigma_out, ws,
                         ws_bytes, stream, sel);
}

int rox_line_select(const rox_lines* lines, const rox_grid* grid, double cutoff, double T, double Q_T, double Q_ref,
                    const rox_select* sel, uint8_t* keep_out, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_lines(lines, true, false);
  if (rc) return rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  if (!finite_pos(T) || !finite_pos(Q_T) || !finite_pos(Q_ref)) return fail(ROX_EINVAL, "T, Q_T, Q_ref must be > 0");
  if (!keep_out) return fail(ROX_EINVAL, "keep_out is NULL");
  double origin;
  long long n_bins;
  if ((rc = select_bins(sel, grid, cutoff, &origin, &n_bins))) return rc;
  if (!ws || ((uintptr_t)ws & 255)) return fail(ROX_EINVAL, "workspace NULL or not 256-byte aligned");
  WsLayout w = ws_layout(ws, lines->n, grid->n, 1, false, n_bins);
  if (ws_bytes < w.bytes) return fail(ROX_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, w.bytes);
  const long long nl = lines->n;
  if (nl == 0) return ok();
  cudaStream_t s = (cudaStream_t)stream;
  if ((rc = cuda_check(cudaMemsetAsync(w.hdr, 0, sizeof(RoxWsHeader), s), "memset"))) return rc;
  if ((rc = cuda_check(rox_launch_strengths_multi(lines, 1, &T, &Q_T, Q_ref, w.S_T, w.hdr->smax_bits, true, s),
                       "strengths kernel")))
    return rc;
  if ((rc = cuda_check(rox_launch_select(lines->nu0, w.S_T, nl, 1, w.hdr->smax_bits, origin, sel->bin_width, n_bins,
                                         sel->rel, w.line_bin, w.binmax, w.S32, s),
                       "selection kernels")))
    return rc;
  if ((rc = cuda_check(rox_launch_keep_flags(w.S_T, w.line_bin, w.binmax, nl, sel->rel, keep_out, s),
                       "keep flags kernel")))
    return rc;
  return ok();
}

size_t rox_xsec_nodes_workspace_size(int64_t n_lines, int64_t n_nodes, int n_temps) {
  if (n_nodes <= 0 || n_lines < 0 || n_temps <= 0) return 0;
  return ws_layout(nullptr, n_lines, n_nodes, n_temps, true).bytes;
}

int rox_xsec_nodes_batch(const rox_lines* lines, const rox_nodes* nodes, int n_pt, const double* P_bar,
                         const double* T, const double* Q_T, double Q_ref, double mass_amu, double cutoff,
                         unsigned flags, float* sigma_out, void* ws, size_t ws_bytes, void* stream) {
  int rc;
  if ((rc = check_nodes(nodes))) return rc;
  if (!finite_pos(cutoff)) return fail(ROX_EINVAL, "cutoff must be > 0");
  if (cutoff > 4000.0) return fail(ROX_ERANGE, "cutoff %g above 4000 cm^-1", cutoff);
  return xsec_batch_impl(lines, nullptr, nodes, n_pt, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, flags, sigma_out, ws,
                         ws_bytes, stream);
}

int rox_node_windows(const double* nu0_sorted, int64_t n_lines, const rox_nodes* nodes, double cutoff, int32_t* jlo,
                     int32_t* jhi, void* stream) {
  int rc;
  if ((rc = check_nodes(nodes))) return rc;
  if (!nu0_sorted || !jlo || !jhi) return fail(ROX_EINVAL, "nu0, jlo, jhi required");
  if (n_lines < 0) return fail(ROX_EINVAL, "n_lines < 0");
  if (!finite_pos(cutoff)) return fail(ROX_EINVAL, "cutoff must be > 0");
  if (n_lines == 0) return ok();
  return cuda_check(rox_launch_node_windows(nu0_sorted, n_lines, nodes->nu, nodes->n, cutoff, jlo, jhi, nullptr,
                                            nullptr, nullptr, 0, (cudaStream_t)stream),
                    "node windows kernel") ? ROX_ECUDA : ok();
}

}  // extern "C"

// rox_xsec with the tail scratch limited to tail_max items (library-internal, C++ linkage:
// rox_xsec_static runs in a fixed 16 MiB array), and the workspace size that goes with it
size_t rox_xsec_workspace_size_tail(int64_t n_lines, const rox_grid* grid, long long tail_max) {
  if (!grid || grid->n <= 0 || n_lines < 0) return 0;
  return ws_layout(nullptr, n_lines, grid->n, 1, false, 0, false, tail_max, false).bytes;
}
int rox_xsec_tail(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T, double Q_ref,
                  double mass_amu, double cutoff, float* sigma_out, void* ws, size_t ws_bytes, void* stream,
                  long long tail_max) {
  int rc;
  if ((rc = check_grid(grid))) return rc;
  if ((rc = check_cutoff(cutoff, grid))) return rc;
  return xsec_batch_impl(lines, grid, nullptr, 1, &P_bar, &T, &Q_T, Q_ref, mass_amu, cutoff, ROX_KAHAN, sigma_out, ws,
                         ws_bytes, stream, nullptr, nullptr, tail_max, false);
}

extern "C" {

int rox_xsec(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T, double Q_ref,
             double mass_amu, double cutoff, float* sigma_out, void* ws, size_t ws_bytes, void* stream) {
  return rox_xsec_batch(lines, grid, 1, &P_bar, &T, &Q_T, Q_ref, mass_amu, cutoff, ROX_KAHAN, sigma_out, ws, ws_bytes,
                        stream);
}

// ---------------------------------------------------------------- serving path
namespace {
struct PrepLayout {
  RoxWsHeader* hdr;
  float4* geo;
  long long* span_lo;
  long long* span_hi;
  size_t bytes;
};
PrepLayout prep_layout(void* state, long long n_lines, long long n_lattice) {
  PrepLayout p;
  char* base = (char*)state;
  size_t off = 0;
  p.hdr = (RoxWsHeader*)base;
  off += ROX_WS_HEADER_BYTES;
  p.geo = (float4*)(base + off);
  off += rox_align256((size_t)(n_lines > 0 ? n_lines : 1) * sizeof(float4));
  long long ns = n_tiles_of(n_lattice);
  p.span_lo = (long long*)(base + off);
  off += rox_align256((size_t)ns * 8);
  p.span_hi = (long long*)(base + off);
  off += rox_align256((size_t)ns * 8);
  p.bytes = off;
  return p;
}
}  // namespace

size_t rox_prepare_size(int64_t n_lines, const rox_grid* lattice) {
  if (!lattice || lattice->n <= 0 || n_lines < 0) return 0;
  return prep_layout(nullptr, n_lines, lattice->n).bytes;
}

int rox_prepare(const rox_lines* lines, const rox_grid* lattice, double cutoff, void* state, size_t state_bytes,
                rox_prepared* out, void* stream) {
  int rc = check_lines(lines, true, true);
  if (rc) return rc;
  if ((rc = check_grid(lattice))) return rc;
  if ((rc = check_cutoff(cutoff, lattice))) return rc;
  if (!out) return fail(ROX_EINVAL, "out is NULL");
  if (!state || ((uintptr_t)state & 255)) return fail(ROX_EINVAL, "state NULL or not 256-byte aligned");
  PrepLayout p = prep_layout(state, lines->n, lattice->n);
  if (state_bytes < p.bytes) return fail(ROX_ENOMEM, "state %zu bytes < %zu needed", state_bytes, p.bytes);
  cudaStream_t s = (cudaStream_t)stream;
  const long long ns = n_tiles_of(lattice->n);
  if ((rc = cuda_check(cudaMemsetAsync(p.hdr, 0, sizeof(RoxWsHeader), s), "memset"))) return rc;
  if (lines->n > 0 &&
      (rc = cuda_check(rox_launch_windows(lines->nu0, lines->n, lattice, cutoff, nullptr, nullptr, nullptr, nullptr,
                                          p.geo, &p.hdr->evals_lines, &p.hdr->status, ROX_EUNSORTED, s),
                       "windows kernel")))
    return rc;
  if ((rc = cuda_check(rox_launch_tile_ranges_geo(p.geo, lines->n, ns, ROX_SPAN, p.span_lo, p.span_hi, s),
                       "span ranges")))
    return rc;
  out->lines = *lines;
  out->lattice = *lattice;
  out->cutoff = cutoff;
  out->state = state;
  out->span_lo = (const int64_t*)p.span_lo;
  out->span_hi = (const int64_t*)p.span_hi;
  out->n_spans = ns;
  return ok();
}

namespace {
struct JobsTail {
  float* part;
  int32_t* cnt;
  long long cap;
};
size_t jobs_layout(const rox_job* jobs, int n_jobs, void* ws, double** S64, float** S32, JobsTail* tail) {
  size_t off = ROX_WS_HEADER_BYTES;
  long long spans = 0;
  for (int k = 0; k < n_jobs; k++) {
    const size_t c = (size_t)(jobs[k].line_count > 0 ? jobs[k].line_count : 1);
    if (S64) S64[k] = (double*)((char*)ws + off);
    off += rox_align256(c * 8);
    if (S32) S32[k] = (float*)((char*)ws + off);
    off += rox_align256(c * 4);
    if (jobs[k].n > 0 && jobs[k].first >= 0)
      spans += (jobs[k].first + jobs[k].n - 1) / ROX_SPAN - jobs[k].first / ROX_SPAN + 1;
  }
  const long long cap = spans < ROX_TAIL_ITEMS_MAX ? spans : ROX_TAIL_ITEMS_MAX;
  if (tail) {
    tail->cap = cap;
    tail->part = (float*)((char*)ws + off);
    tail->cnt = (int32_t*)((char*)ws + off + rox_align256((size_t)cap * ROX_PARTS * ROX_SPAN * sizeof(float)));
  }
  off += rox_tail_bytes(cap);
  return off;
}
}  // namespace

size_t rox_jobs_workspace_size(const rox_job* jobs, int n_jobs) {
  if (!jobs || n_jobs <= 0) return 0;
  return jobs_layout(jobs, n_jobs, nullptr, nullptr, nullptr, nullptr);
}

int rox_xsec_jobs(const rox_prepared* lists, int n_lists, const rox_job* jobs, int n_jobs, void* ws, size_t ws_bytes,
                  void* stream) {
  if (!lists || n_lists < 1 || n_lists > ROX_MAX_LISTS) return fail(ROX_EINVAL, "n_lists must be 1..%d", ROX_MAX_LISTS);
  if (!jobs || n_jobs < 1 || n_jobs > ROX_MAX_PT) return fail(ROX_EINVAL, "n_jobs must be 1..%d", ROX_MAX_PT);
  int rc;
  for (int l = 0; l < n_lists; l++) {
    if ((rc = check_lines(&lists[l].lines, true, true))) return rc;
    if (!lists[l].state || !lists[l].span_lo || !lists[l].span_hi) return fail(ROX_EINVAL, "list %d not prepared", l);
  }
  for (int k = 0; k < n_jobs; k++) {
    const rox_job& j = jobs[k];
    if (j.list < 0 || j.list >= n_lists) return fail(ROX_EINVAL, "job %d: list %d out of range", k, j.list);
    const rox_prepared& L = lists[j.list];
    if (j.n <= 0 || j.first < 0 || j.first + j.n > L.lattice.n)
      return fail(ROX_EINVAL, "job %d: window [%lld, %lld) outside the lattice", k, (long long)j.first,
                  (long long)(j.first + j.n));
    if (j.line_first < 0 || j.line_count < 0 || j.line_first + j.line_count > L.lines.n)
      return fail(ROX_EINVAL, "job %d: line range outside the list", k);
    if (!finite_pos(j.T) || !finite_pos(j.Q_T) || !finite_pos(j.Q_ref) || !finite_pos(j.mass_amu) ||
        !std::isfinite(j.P_bar) || j.P_bar < 0)
      return fail(ROX_EINVAL, "job %d: T, Q_T, Q_ref, mass > 0 and P >= 0 required", k);
    if (j.flags & ~(ROX_ACCUMULATE | ROX_KAHAN)) return fail(ROX_EINVAL, "job %d: unknown flags", k);
    if (!j.sigma_out) return fail(ROX_EINVAL, "job %d: sigma_out is NULL", k);
  }
  if (!ws || ((uintptr_t)ws & 255)) return fail(ROX_EINVAL, "workspace NULL or not 256-byte aligned");
  const size_t need = jobs_layout(jobs, n_jobs, nullptr, nullptr, nullptr, nullptr);
  if (ws_bytes < need) return fail(ROX_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, need);
  int nblocks = 0;
  const rox_launch_config cfg = launch_config();
  if ((rc = voigt_grid(&nblocks, cfg))) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  RoxWsHeader* hdr = (RoxWsHeader*)ws;
  std::vector<double*> S64(n_jobs);
  std::vector<float*> S32(n_jobs);
  JobsTail tail;
  jobs_layout(jobs, n_jobs, ws, S64.data(), S32.data(), &tail);
  if ((rc = cuda_check(cudaMemsetAsync(hdr, 0, sizeof(RoxWsHeader), s), "memset"))) return rc;

  // strengths of every job's line range at its temperature
  static thread_local RoxStrengthJobs SJ;
  for (int l = 0; l < n_lists; l++) {
    SJ.list[l].nu0 = lists[l].lines.nu0;
    SJ.list[l].s_or_a = lists[l].lines.s_or_a;
    SJ.list[l].g_up = lists[l].lines.g_up;
    SJ.list[l].e_lower = lists[l].lines.e_lower;
    SJ.list[l].convention = lists[l].lines.convention;
    SJ.list[l].pad = 0;
  }
  for (int j0 = 0; j0 < n_jobs; j0 += ROX_MAX_JOBS) {
    const int nj = (n_jobs - j0) < ROX_MAX_JOBS ? (n_jobs - j0) : ROX_MAX_JOBS;
    long long mx = 1;
    for (int q = 0; q < nj; q++) {
      const rox_job& j = jobs[j0 + q];
      RoxStrengthJob& jb = SJ.job[q];
      jb.l0 = j.line_first;
      jb.count = j.line_count;
      jb.S64 = S64[j0 + q];
      jb.S32 = S32[j0 + q];
      jb.smax_bits = &hdr->smax_bits[j0 + q];
      jb.list = j.list;
      jb.pad = 0;
      rox_fill_strength_consts(lists[j.list].lines.convention, j.T, j.Q_T, j.Q_ref, &jb);
      if (j.line_count > mx) mx = j.line_count;
    }
    SJ.n_jobs = nj;
    if ((rc = cuda_check(rox_launch_strengths_jobs(SJ, mx, s), "strengths kernel"))) return rc;
  }

  // one Voigt launch over all (job, span) items
  RoxListDev L[ROX_MAX_LISTS];
  for (int l = 0; l < n_lists; l++) {
    const rox_prepared& P = lists[l];
    L[l].status = &((RoxWsHeader*)P.state)->status;
    L[l].geo = (const float4*)((char*)P.state + ROX_WS_HEADER_BYTES);
    L[l].span_lo = (const long long*)P.span_lo;
    L[l].span_hi = (const long long*)P.span_hi;
    L[l].gamma_ref = P.lines.gamma_ref;
    L[l].n_t = P.lines.n_t;
    L[l].gLT = nullptr;
    L[l].gLT_stride = 0;
    L[l].gN = nullptr;
    L[l].idx = nullptr;
    L[l].node_d = nullptr;
    L[l].span_base = nullptr;
    L[l].n_lattice = P.lattice.n;
    L[l].dnu_f = (float)P.lattice.dnu;
    L[l].nu_min_f = (float)P.lattice.nu_min;
    L[l].width_f16 = P.lines.width_dtype == ROX_WIDTH_F16;
    L[l].inv_dnu_f = (float)(1.0 / P.lattice.dnu);
    L[l].rec = nullptr;
  }
  std::vector<RoxJobDev> J(n_jobs);
  for (int k = 0; k < n_jobs; k++) {
    const rox_job& j = jobs[k];
    RoxJobDev& d = J[k];
    d.S32 = S32[k];
    d.sigma = j.sigma_out;
    d.smax_bits = &hdr->smax_bits[k];
    d.l0 = j.line_first;
    d.l1 = j.line_first + j.line_count;
    d.first = j.first;
    d.n = j.n;
    d.list = j.list;
    d.span_first = (int32_t)(j.first / ROX_SPAN);
    d.n_spans = (int32_t)((j.first + j.n - 1) / ROX_SPAN - j.first / ROX_SPAN + 1);
    d.p_fac = (float)(j.P_bar / ROX_P_REF);
    d.gG_fac = (float)(sqrt(2.0 * ROX_KB * j.T / (j.mass_amu * ROX_AMU)) / ROX_C_M);
    d.l2_ratio = (float)log2(ROX_T_REF / j.T);
    d.flags = j.flags;
    d.t_row = 0;
  }
  if ((rc = launch_voigt_jobs(L, n_lists, J.data(), n_jobs, hdr, tail.part, tail.cnt, tail.cap, nblocks, s, cfg)))
    return rc;
  return ok();
}

int rox_set_launch_config(const rox_launch_config* cfg) {
  rox_launch_config c = {8, 0, 1, 0};
  if (cfg) {
    if (cfg->warps_per_cta != 4 && cfg->warps_per_cta != 8) return fail(ROX_EINVAL, "warps_per_cta must be 4 or 8");
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 64) return fail(ROX_EINVAL, "ctas_per_sm must be 0..64");
    if (cfg->split_rounds < 1 || cfg->split_rounds > 4) return fail(ROX_EINVAL, "split_rounds must be 1..4");
    c = *cfg;
    c.pad = 0;
  }
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  g_cfg = c;
  return ok();
}

int rox_get_launch_config(rox_launch_config* out) {
  if (!out) return fail(ROX_EINVAL, "out is NULL");
  *out = launch_config();
  return ok();
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
  if (h.status != ROX_OK) return fail(h.status, "device status %d", h.status);
  if (h.overflow) return fail(ROX_EOVERFLOW, "a cross-section value is beyond the FP32 range");
  return ok();
}

}  // extern "C"
