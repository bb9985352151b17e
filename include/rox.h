/* rox.h -- C ABI of librox: line-by-line opacity cross-sections on a GB300 (sm_103a).
 *
 * The method is that of the pyROX paper (de Regt, Gandhi, Siebenaler, Gonzalez Picos),
 * section "Functionality of pyROX":
 *   - "Compute line-strengths and -widths": every transition gets a strength and
 *     broadening widths at the requested pressure and temperature;
 *   - "Compute line profiles": a Voigt profile, the real part of the Faddeeva
 *     function (Gandhi et al. 2020, Eq. 12);
 *   - "Combine and save": the profiles are summed into a cross-section sigma(nu)
 *     for each temperature-pressure point.
 * The paper prints no formula. The definitions used (standard HITRAN / ExoMol forms) are:
 *   S(T) HITRAN = S_ref Q(296)/Q(T) exp(-c2 E''(1/T - 1/296)) (1 - e^{-c2 nu0/T})/(1 - e^{-c2 nu0/296})
 *   S(T) ExoMol = g_up A / (8 pi c nu0^2) exp(-c2 E''/T) (1 - e^{-c2 nu0/T}) / Q(T)
 *   gamma_G     = (nu0/c) sqrt(2 k_B T / (m amu))            (1/e Doppler half-width)
 *   gamma_L     = gamma_ref (296/T)^n_T (P / 1.01325 bar)      (Lorentz HWHM)
 *   V(dnu)      = Re w((dnu + i gamma_L)/gamma_G) / (gamma_G sqrt(pi))
 *   sigma_j     = sum over lines with |nu_j - nu0| <= cutoff of S V(nu_j - nu0),
 *                 nu_j = nu_min + j dnu, the cutoff test taken in double precision exactly
 *                 as written (inclusive, no renormalisation).
 * Units: wavenumbers cm^-1, T in K, P in bar, S in cm/molecule, sigma in cm^2/molecule.
 *
 * Conventions for every call:
 *   - returns ROX_OK (0) or an error code below; rox_last_error() gives a message
 *     (thread-local). On an argument error nothing is launched and no output is written.
 *   - array pointers are DEVICE pointers owned by the caller unless stated otherwise;
 *     scalars and small per-point arrays marked "host" are host memory.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). All work is enqueued on
 *     it asynchronously; no call synchronises unless its comment says so.
 *   - scratch memory is a caller-provided device workspace `ws` of `ws_bytes` bytes
 *     (256-byte aligned); the library allocates nothing on the hot path.
 *   - errors found on the device (unsorted input, a bounded wait running out) are
 *     recorded in the workspace and returned by rox_ws_status().
 */
#ifndef ROX_H
#define ROX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define ROX_OK 0
#define ROX_EINVAL 1      /* invalid argument: null pointer, n <= 0, T <= 0, P < 0, Q <= 0, ... */
#define ROX_ENOMEM 2      /* workspace smaller than the matching *_workspace_size() */
#define ROX_ECUDA 3       /* a CUDA runtime call failed (see rox_last_error) */
#define ROX_ETIMEOUT 4    /* reserved for a bounded device-side wait running out; no kernel of this
                             version waits on another, so no call returns it */
#define ROX_EUNSORTED 5   /* line list not in ascending nu0 (reported by rox_ws_status) */
#define ROX_ERANGE 6      /* a size beyond a documented limit */
#define ROX_EGRID 7       /* user-provided nodes not finite or not strictly increasing (rox_ws_status) */
#define ROX_EOVERFLOW 8   /* a cross-section value beyond the FP32 range (inf or NaN) was written
                             (rox_ws_status); the other values of the call are valid */

/* line-list conventions */
#define ROX_HITRAN 0      /* s_or_a = S_ref at 296 K (cm/molecule) */
#define ROX_EXOMOL 1      /* s_or_a = Einstein A (s^-1), g_up required */

/* storage type of the gamma_ref / n_t columns */
#define ROX_WIDTH_F32 0
#define ROX_WIDTH_F16 1

/* flags of rox_xsec_batch (and of the rox_job of rox_xsec_jobs) */
#define ROX_ACCUMULATE 1u /* add into sigma_out instead of overwriting it (chunked line lists) */
#define ROX_KAHAN 2u      /* compensated (Kahan) summation of the per-batch FP32 partial sums of each
                             span part; without it they are added plainly (rox_xsec always sets it) */

/* limits */
#define ROX_MAX_PT 512            /* (P,T) points per rox_xsec_batch call */
#define ROX_MAX_GRID (1 << 23)    /* grid points (line-centre indices are carried exactly in FP32) */
#define ROX_MAX_CUTOFF_STEPS (1 << 21) /* cutoff / dnu */
#define ROX_MAX_SELECT_BINS (1 << 24)  /* bins of a main-contributor selection */

/* A line list as structure-of-arrays, n lines, all DEVICE pointers.
 * nu0       [n] double  line centre (cm^-1), > 0
 * s_or_a    [n] float   HITRAN: S_ref at 296 K (cm/molecule); ExoMol: Einstein A (s^-1)
 * g_up      [n] float   ExoMol upper-state degeneracy (ignored and may be NULL for HITRAN)
 * e_lower   [n] float   lower-state energy E'' (cm^-1)
 * gamma_ref [n] float|half  Lorentz HWHM at 296 K and 1 atm (cm^-1 atm^-1)
 * n_t       [n] float|half  temperature exponent of gamma_L
 * The cross-section calls need the list sorted by ascending nu0 (rox_sort_lines). */
typedef struct rox_lines {
  const double* nu0;
  const float* s_or_a;
  const float* g_up;
  const float* e_lower;
  const void* gamma_ref;
  const void* n_t;
  int64_t n;
  int32_t convention;   /* ROX_HITRAN or ROX_EXOMOL */
  int32_t width_dtype;  /* ROX_WIDTH_F32 or ROX_WIDTH_F16 */
} rox_lines;

/* Writable twin of rox_lines (outputs of rox_sort_lines). */
typedef struct rox_lines_buf {
  double* nu0;
  float* s_or_a;
  float* g_up;
  float* e_lower;
  void* gamma_ref;
  void* n_t;
} rox_lines_buf;

/* Uniform wavenumber grid nu_j = nu_min + j*dnu, j = 0..n-1 (cm^-1). */
typedef struct rox_grid {
  double nu_min;
  double dnu;
  int64_t n;
} rox_grid;

/* User-provided grid (paper, "Similar tools": cross-sections on any wavelength or wavenumber
 * grid, e.g. one of fixed resolution R = lambda/dlambda): n nodes nu[0..n-1] (cm^-1, DEVICE,
 * double), finite and strictly increasing. */
typedef struct rox_nodes {
  const double* nu;
  int64_t n;
} rox_nodes;

/* Message of the last error on this thread ("" if none). Never NULL. */
const char* rox_last_error(void);
/* Library version string. */
const char* rox_version(void);

/* a1 -- line strengths S(T) (cm/molecule) of all lines, FP32 output, FP64 arithmetic
 * for the Boltzmann and stimulated-emission factors and the partition-function ratio.
 * Paper: "Compute line-strengths and -widths".
 * T > 0 (K); Q_T = Q(T) > 0 and Q_ref = Q(296 K) > 0 are computed by the caller (host).
 * S_out [n] float (device). Strengths below the FP32 range round to 0 or a subnormal. */
int rox_line_strengths(const rox_lines* lines, double T, double Q_T, double Q_ref,
                       float* S_out, void* stream);

/* a1 -- the strengths exactly as the cross-section launches compute them (rox_xsec_batch and the
 * calls built on it), in double: the Boltzmann exponent a = -c2 E''(1/T - 1/296) (HITRAN) or
 * -c2 E''/T (ExoMol) in FP64, reduced as a = k ln2 + r (ln 2 in two parts, Cody and Waite);
 * exp(r), the stimulated-emission factor(s) and the prefactor in FP32 on a 2^64 pre-scale, put
 * back by the exact powers 2^-64 and 2^k. Exponents with |a| >= 700 and FP32 products outside
 * [2^-100, 2^100] take the full FP64 form of rox_line_strengths. Relative error below 1e-6 (the
 * sum of the FP32 roundings, the expf and expm1f errors included). Paper: "Compute
 * line-strengths and -widths". Arguments as rox_line_strengths; S_out [n] double (device). */
int rox_line_strengths_reduced(const rox_lines* lines, double T, double Q_T, double Q_ref,
                               double* S_out, void* stream);

/* a2 -- Doppler 1/e half-widths gamma_G and Lorentz HWHM gamma_L (cm^-1), FP32 outputs.
 * Paper: "Compute line-strengths and -widths" (pressure broadening: single power law).
 * mass_amu > 0, P_bar >= 0, T > 0. gamma_G_out, gamma_L_out [n] float (device). */
int rox_line_widths(const rox_lines* lines, double mass_amu, double P_bar, double T,
                    float* gamma_G_out, float* gamma_L_out, void* stream);

/* a3 (sort) -- copy of the line list in ascending nu0 (stable: equal nu0 keep input
 * order) into `out` (device buffers of n elements; g_up may be NULL for HITRAN), and the
 * permutation perm_out[k] = input index of output line k (int64, device, may be NULL).
 * Workspace: rox_sort_workspace_size(n). */
size_t rox_sort_workspace_size(int64_t n);
int rox_sort_lines(const rox_lines* in, const rox_lines_buf* out, int64_t* perm_out,
                   void* ws, size_t ws_bytes, void* stream);

/* a3 (binning) -- per sorted line, the grid-index window and centre decomposition:
 *   jlo[i], jhi[i]: first and last grid index j with |nu_j - nu0_i| <= cutoff, the test
 *                   evaluated in double precision as abs((nu_min + j*dnu) - nu0) <= cutoff;
 *                   jlo clamped to [0, n], jhi to [-1, n-1]; jlo > jhi when no grid point
 *                   is in range (both are non-decreasing along a sorted list);
 *   k0[i], f[i]:    (nu0 - nu_min)/dnu = k0 + f with k0 integer and f in [0, 1).
 * evals_out (device, 1 x uint64): number of (line, grid point) pairs inside the cutoff,
 * added to the value already there. unsorted_out (device, 1 x int32): set to 1 if nu0 is
 * not ascending (left unchanged otherwise). Any output pointer may be NULL. */
int rox_line_windows(const double* nu0_sorted, int64_t n_lines, const rox_grid* grid,
                     double cutoff, int32_t* jlo, int32_t* jhi, int32_t* k0, float* f,
                     unsigned long long* evals_out, int32_t* unsorted_out, void* stream);

/* a3 (prefix) -- per wavenumber tile t (tile_pts grid points, tile t covers grid indices
 * [t*tile_pts, (t+1)*tile_pts)), the range [lo[t], hi[t]) of sorted lines whose window
 * [jlo, jhi] meets the tile. Equivalent to the exclusive prefix sum of the per-tile line
 * histogram; read off the sorted order without atomics. lo_out, hi_out: n_tiles int64. */
int rox_tile_ranges(const int32_t* jlo, const int32_t* jhi, int64_t n_lines, int64_t n_grid,
                    int32_t tile_pts, int64_t* lo_out, int64_t* hi_out, void* stream);

/* FP32 Faddeeva real part used by the Voigt kernel: out[i] = Re w(x[i] + i y[i]), y >= 0.
 * All device arrays of n floats. Max relative error against an FP64 reference about 1.1e-5
 * (values below 1e-15 excepted). */
int rox_faddeeva_re(const float* x, const float* y, float* out, int64_t n, void* stream);

/* a4/a5 -- cross-sections at n_pt (P,T) points in one persistent launch.
 * lines     sorted line list (device)
 * grid      output grid (host struct); n <= ROX_MAX_GRID
 * P_bar, T, Q_T   [n_pt] HOST arrays: pressure (bar, >= 0), temperature (K, > 0),
 *                 partition function Q(T) (> 0); Q_ref = Q(296 K) (> 0)
 * mass_amu  molecular mass (> 0); cutoff  wing cutoff (cm^-1, > 0), cutoff/dnu <= ROX_MAX_CUTOFF_STEPS
 * flags     0, ROX_ACCUMULATE, ROX_KAHAN or both
 * sigma_out [n_pt][grid->n] float (device), point-major; each grid point is written once
 *           per call with a fixed summation order (bitwise reproducible run to run).
 * ws        device workspace of rox_xsec_workspace_size(lines->n, grid, n_temps) bytes, where
 *           n_temps is the number of distinct temperatures among T[0..n_pt-1] (S(T) is
 *           computed once per distinct temperature and kept in the workspace as a double).
 * Voigt profile and tile sums in FP32 (compensated across line chunks). S(T): the Boltzmann
 * exponent and its reduction k ln2 + r in FP64, exp(r), the stimulated-emission factor and the
 * prefactor in FP32 (relative error below 1e-6, against 1e-16 for rox_line_strengths).
 * Line-centre offsets: exact index decomposition in FP64. */
size_t rox_xsec_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps);
int rox_xsec_batch(const rox_lines* lines, const rox_grid* grid, int n_pt,
                   const double* P_bar, const double* T, const double* Q_T, double Q_ref,
                   double mass_amu, double cutoff, unsigned flags, float* sigma_out,
                   void* ws, size_t ws_bytes, void* stream);

/* a4 -- one (P,T) point: rox_xsec_batch with n_pt = 1 and flags = ROX_KAHAN. */
int rox_xsec(const rox_lines* lines, const rox_grid* grid, double P_bar, double T,
             double Q_T, double Q_ref, double mass_amu, double cutoff, float* sigma_out,
             void* ws, size_t ws_bytes, void* stream);

/* a2 pressure-broadening descriptions and natural broadening (paper, "Compute line-strengths
 * and -widths": various pressure-broadening descriptions are supported):
 *   gamma_L = sum_b vmr[b] gamma_ref_b (296/T)^n_b (P / 1.01325 bar) + (natural ? A/(4 pi c) : 0)
 * over n_broadeners broadeners (1..ROX_MAX_BROADENERS), each with per-line columns
 * gamma_ref[b], n_t[b] (DEVICE, float or half as lines->width_dtype) or, where table_gamma[b]
 * is not NULL, values looked up by the line's lower-state J in table_gamma[b][J],
 * table_n[b][J] (DEVICE float, table_len entries; J < 0 takes entry 0, J >= table_len the
 * last one; j_lower [n] int32 DEVICE). natural = 1 adds the Lorentz half-width of the
 * Einstein-A decay, A/(4 pi c) with c in cm/s (ExoMol lists only: s_or_a is A). The list's own
 * gamma_ref / n_t are not used. */
#define ROX_MAX_BROADENERS 4
typedef struct rox_broadening {
  int32_t n_broadeners;
  int32_t natural;
  double vmr[ROX_MAX_BROADENERS];
  const void* gamma_ref[ROX_MAX_BROADENERS];
  const void* n_t[ROX_MAX_BROADENERS];
  const float* table_gamma[ROX_MAX_BROADENERS];
  const float* table_n[ROX_MAX_BROADENERS];
  const int32_t* j_lower;
  int64_t table_len;
} rox_broadening;

/* gamma_L of every line under `br` at (P_bar, T): gamma_L_out [n] float (device). FP32
 * arithmetic (each power as exp2 of n_b log2(296/T)). */
int rox_lorentz_widths(const rox_lines* lines, const rox_broadening* br, double P_bar, double T,
                       float* gamma_L_out, void* stream);

/* rox_xsec_batch with the Lorentz widths of `br`. Per distinct temperature the broadeners' sum
 * sum_b vmr_b gamma_ref_b (296/T)^n_b is computed once per line (FP32, kept in the workspace)
 * and, with natural broadening, A/(4 pi c) once per line; the Voigt kernel then takes
 * gamma_L = that sum * P/P_ref + the natural width. Arguments otherwise as rox_xsec_batch (the
 * list's gamma_ref / n_t may be NULL). ws: rox_xsec_broadened_workspace_size(lines->n, grid,
 * n_temps) bytes. */
size_t rox_xsec_broadened_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps);
int rox_xsec_broadened_batch(const rox_lines* lines, const rox_grid* grid, const rox_broadening* br,
                             int n_pt, const double* P_bar, const double* T, const double* Q_T,
                             double Q_ref, double mass_amu, double cutoff, unsigned flags,
                             float* sigma_out, void* ws, size_t ws_bytes, void* stream);

/* a4/a5 with main-contributor line selection (paper, "Compute line-strengths and -widths": the
 * line-profile step can be sped up by keeping only the main line-strength contributors).
 * At each (P,T) point, with S = S(T) in double precision (as rox_line_strengths; the launch
 * computes the reduced form of rox_xsec_batch and recomputes in double precision every line
 * whose decision it could change, so every decision is the double-precision one), the lines
 * are binned by nu0 into
 * bins of width bin_width (cm^-1) starting at grid->nu_min - cutoff,
 *   bin = floor((nu0 - (nu_min - cutoff)) / bin_width)   (subtraction and division each rounded
 *                                                         once in double precision),
 * n_bins = floor(((grid->n - 1) dnu + 2 cutoff) / bin_width) + 1 (every nu0 that reaches a grid
 * point falls in a bin), and a line is kept iff its bin is in range and
 * S >= rel * (the largest S in its bin at that temperature) (product rounded once). rel = 0
 * keeps every line that reaches the grid; each bin keeps at least its strongest line.
 * sigma_out is the cross-section of the kept lines (R8 over them); dropped lines cost no
 * profile evaluation, and rox_ws_status counts the kept (line, grid point) pairs only.
 * Arguments otherwise as rox_xsec_batch; sel->rel >= 0, sel->bin_width > 0, n_bins <=
 * ROX_MAX_SELECT_BINS. ws: rox_xsec_select_workspace_size(lines->n, grid, n_temps, cutoff, sel)
 * bytes (0 if the selection is invalid). */
typedef struct rox_select {
  double rel;
  double bin_width;
} rox_select;
size_t rox_xsec_select_workspace_size(int64_t n_lines, const rox_grid* grid, int n_temps, double cutoff,
                                      const rox_select* sel);
int rox_xsec_select_batch(const rox_lines* lines, const rox_grid* grid, int n_pt,
                          const double* P_bar, const double* T, const double* Q_T, double Q_ref,
                          double mass_amu, double cutoff, unsigned flags, const rox_select* sel,
                          float* sigma_out, void* ws, size_t ws_bytes, void* stream);

/* The selection of rox_xsec_select_batch at one temperature: keep_out[i] = 1 if line i is
 * kept, else 0 ([lines->n] uint8, device). Widths are not needed (gamma_ref and n_t may be
 * NULL). ws: rox_xsec_select_workspace_size(lines->n, grid, 1, cutoff, sel) bytes. */
int rox_line_select(const rox_lines* lines, const rox_grid* grid, double cutoff, double T,
                    double Q_T, double Q_ref, const rox_select* sel, uint8_t* keep_out,
                    void* ws, size_t ws_bytes, void* stream);

/* a4/a5 on user-provided nodes (paper, "Similar tools": any user-provided wavelength or
 * wavenumber grid, which fixes the resolving power R = lambda/dlambda): rox_xsec_batch with the
 * uniform grid replaced by nodes nu[0..n-1]. A line contributes to node k iff
 * |nu[k] - nu0| <= cutoff, the difference taken once in double precision; sigma_out is
 * [n_pt][nodes->n]. Arguments, flags, ordering and precision as rox_xsec_batch, except that the
 * cutoff only needs 0 < cutoff <= 4000 cm^-1. The nodes are checked on the device: if they are
 * not finite or not strictly increasing, nothing is written and rox_ws_status returns
 * ROX_EGRID. ws: device workspace of rox_xsec_nodes_workspace_size(lines->n, nodes->n,
 * n_temps) bytes (n_temps as for rox_xsec_batch); it includes each node's offset from the
 * first node of its ROX_SPAN-node span, the kernel's exact stand-in for the index
 * decomposition of a uniform grid. */
size_t rox_xsec_nodes_workspace_size(int64_t n_lines, int64_t n_nodes, int n_temps);
int rox_xsec_nodes_batch(const rox_lines* lines, const rox_nodes* nodes, int n_pt,
                         const double* P_bar, const double* T, const double* Q_T, double Q_ref,
                         double mass_amu, double cutoff, unsigned flags, float* sigma_out,
                         void* ws, size_t ws_bytes, void* stream);

/* a3 windows on user-provided nodes: per sorted line, the first node with
 * nu[k] - nu0 >= -cutoff (jlo, in [0, n]) and the last with nu[k] - nu0 <= cutoff (jhi, in
 * [-1, n-1]; jhi < jlo when the line reaches no node), differences rounded once in double
 * precision (binary searches). jlo, jhi: [n_lines] int32 (device). */
int rox_node_windows(const double* nu0_sorted, int64_t n_lines, const rox_nodes* nodes,
                     double cutoff, int32_t* jlo, int32_t* jhi, void* stream);

/* CIA restructuring (paper, "Functionality of pyROX", "Combine and save": for CIA calculations
 * the coefficients read from the input files are restructured into a wavelength- and
 * temperature-dependent grid). Input: n_blocks blocks (1..ROX_CIA_MAX_BLOCKS), block b at
 * temperature T_block[b] (HOST) with samples offset[b] .. offset[b+1]-1 (offset HOST, [n_blocks+1],
 * offset[0] = 0, at least one sample per block) of the DEVICE arrays nu (cm^-1, strictly
 * increasing within a block; not checked) and k (coefficients, any unit). Output: out
 * [n_T][n] double (DEVICE), row t for temperature T_out[t] (HOST, n_T <= ROX_CIA_MAX_TEMPS, finite
 * and distinct) on the
 * grid's points (nu_min + j dnu, one multiply and one add, or the given nodes): at each point
 * the first block (input order) with T_block == T_out[t] whose sample range contains it, linearly
 * interpolated between its bracketing samples, k_i + (k_{i+1} - k_i) (nu - nu_i) / (nu_{i+1} - nu_i),
 * in double precision (within a few ulps of that expression; a sample's own value at a sample),
 * and 0 where no such block covers the point. Nodes may come in any order (ascending is the
 * fast case: each lane walks its intervals forward). On the uniform grid the points of each
 * interval are those the definition assigns to it on the rounded grid values, the value steps
 * from the interval's first point by the constant increment per grid point (within 32 roundings of
 * the expression above, exact at samples); ws: DEVICE scratch of rox_cia_workspace_size(n_blocks,
 * offset[n_blocks]) bytes, 8-byte aligned, not kept between calls. Returns ROX_EINVAL, writing
 * nothing, for a bad block layout or count or a short workspace; launch errors as for the other
 * entry points. */
#define ROX_CIA_MAX_BLOCKS 256
#define ROX_CIA_MAX_TEMPS 4096
typedef struct rox_cia {
  int32_t n_blocks;
  int32_t pad;
  const double* T_block;
  const int64_t* offset;
  const double* nu;
  const double* k;
} rox_cia;
size_t rox_cia_workspace_size(int32_t n_blocks, int64_t n_samples);
int rox_cia_regrid(const rox_cia* cia, const rox_grid* grid, int n_T, const double* T_out,
                   double* out, void* ws, size_t ws_bytes, void* stream);
int rox_cia_regrid_nodes(const rox_cia* cia, const rox_nodes* nodes, int n_T, const double* T_out,
                         double* out, void* stream);

/* Synchronises `stream` and returns the device-side status recorded in `ws` by the last
 * rox_xsec / rox_xsec_batch / rox_xsec_nodes_batch call that used it: ROX_OK, ROX_EUNSORTED
 * (lines not in ascending nu0: no sigma was written), ROX_EGRID (bad nodes: no sigma was
 * written), or ROX_EOVERFLOW (some sigma value is not finite in FP32). If evals_out is not NULL it
 * receives the number of (line, grid point) pairs inside the cutoff summed over the
 * call's (P,T) points (the unit of work of the Voigt kernel). */
int rox_ws_status(const void* ws, unsigned long long* evals_out, void* stream);

/* Serving path, a3 once per list: a sorted line list prepared on a lattice (a grid shared by
 * all requests on it) -- its cutoff windows and its line range per lattice span of ROX_SPAN
 * points -- for any number of rox_xsec_jobs calls with output windows on that lattice.
 * state: device memory of rox_prepare_size(n, lattice) bytes, owned by the caller and kept
 * while `out` is in use. rox_ws_status(state, ...) reports ROX_EUNSORTED if nu0 was not
 * ascending (jobs on such a list then leave their output untouched). */
#define ROX_SPAN 256
typedef struct rox_prepared {
  rox_lines lines;
  rox_grid lattice;
  double cutoff;
  void* state;
  const int64_t* span_lo;   /* device [n_spans]: first line reaching lattice span s */
  const int64_t* span_hi;   /* device [n_spans]: one past the last line reaching span s */
  int64_t n_spans;
} rox_prepared;
size_t rox_prepare_size(int64_t n_lines, const rox_grid* lattice);
int rox_prepare(const rox_lines* lines, const rox_grid* lattice, double cutoff, void* state, size_t state_bytes,
                rox_prepared* out, void* stream);

/* One cross-section request: a window of lattice points on one prepared list at one (P,T).
 * line_first/line_count give the lines that can reach the window, read from a host copy of
 * the list's span tables: line_first = span_lo[first / ROX_SPAN], line_count =
 * span_hi[(first + n - 1) / ROX_SPAN] - line_first; lines outside the range are skipped. */
typedef struct rox_job {
  int32_t list;               /* index into the `lists` of rox_xsec_jobs */
  uint32_t flags;             /* 0, ROX_ACCUMULATE, ROX_KAHAN or both */
  int64_t first, n;           /* lattice points [first, first + n) */
  int64_t line_first, line_count;
  double P_bar, T, Q_T, Q_ref, mass_amu;
  float* sigma_out;           /* [n] float (device) */
} rox_job;

/* a1 + a4 for many requests in one persistent launch (continuous-batching server, batched
 * windows): per job the strengths of its line range at its T (the reduced form of
 * rox_xsec_batch, then scaled to FP32),
 * then one Voigt launch over all (job, span) items. Each job's result is independent of the
 * others in the launch (same summation order as alone). n_jobs <= ROX_MAX_PT,
 * n_lists <= 8. ws: rox_jobs_workspace_size(jobs, n_jobs) bytes. */
size_t rox_jobs_workspace_size(const rox_job* jobs, int n_jobs);
int rox_xsec_jobs(const rox_prepared* lists, int n_lists, const rox_job* jobs, int n_jobs, void* ws, size_t ws_bytes,
                  void* stream);

/* Measurement hook: when start/stop are not NULL (cudaEvent_t handles created by the
 * caller), every following rox_xsec / rox_xsec_batch call on this thread records `start`
 * just before and `stop` just after its Voigt-accumulate kernel launch, on the call's
 * stream. Pass NULL, NULL to stop. Recording is stream-ordered and adds no sync. */
int rox_set_profile_events(void* start, void* stop);

/* Launch configuration of the Voigt kernel, process-wide (the paper has no counterpart; it is a
 * tuning knob of this library, chosen by the autotuner, paper_2510_20870_gb300/autotune.py):
 *   warps_per_cta  4 or 8 (default 8)
 *   ctas_per_sm    CTAs per SM of the persistent grid, 1..the kernel's resident maximum; 0 (default)
 *                  or a larger value: the maximum
 *   split_rounds   1..4 (default 1): after the whole work items, this many rounds of the launch's
 *                  warps worth of items are split into parts, so the launch ends in small pieces
 * No setting changes any result: the summation order of every span is fixed whatever the launch.
 * rox_set_launch_config(NULL) restores the defaults; out-of-range values return ROX_EINVAL and
 * change nothing. Takes effect for the calls that start after it (thread-safe). */
typedef struct rox_launch_config {
  int32_t warps_per_cta;
  int32_t ctas_per_sm;
  int32_t split_rounds;
  int32_t pad;
} rox_launch_config;
int rox_set_launch_config(const rox_launch_config* cfg);
int rox_get_launch_config(rox_launch_config* out);

/* Measurement helper (the paper has no counterpart): the FP32 fused multiply-add rate of this
 * GPU, the denominator of the Voigt kernel's roofline. Launches n_blocks blocks of 256 threads,
 * each thread running 16 independent FMA chains for reps x 8 rounds; out is a DEVICE buffer of
 * at least rox_fp32_probe_out_size(n_blocks) bytes (caller-owned, overwritten with values of no
 * use). *fma_out (host) receives the number of FMAs the launch performs; time the launch with
 * events on `stream` and divide. ROX_EINVAL for n_blocks < 1, reps < 1 or NULL pointers,
 * ROX_ENOMEM for a short buffer. */
size_t rox_fp32_probe_out_size(int n_blocks);
int rox_fp32_probe(int n_blocks, int reps, float* out, size_t out_bytes, double* fma_out, void* stream);

/* Measurement helper: the attainable rate of the Voigt kernel's inner loop. Runs the pass-1
 * pair loop of the cross-section kernel (two lines per reciprocal, far form, no clamp or mask)
 * alone on synthetic far-wing constants, n_blocks blocks of 256 threads (8 warps, as the
 * kernel's default launch), each warp walking 16 pairs reps times over its span of ROX_SPAN
 * points; no line set-up, staging, window edges or slow zones. out as rox_fp32_probe
 * (rox_fp32_probe_out_size(n_blocks) bytes, device). *evals_out (host) receives the
 * (line, point) evaluations the launch performs; time it with events on `stream`. Errors as
 * rox_fp32_probe. */
int rox_pair_loop_probe(int n_blocks, int reps, float* out, size_t out_bytes, double* evals_out, void* stream);

/* Allocation-free variant of rox_xsec (one (P,T) point), for callers that cannot
 * allocate device memory themselves: an application whose own memory manager owns all
 * device memory, a plugin that is not allowed to call cudaMalloc, or an interface that
 * has no way to pass a workspace through. The paper has no counterpart; this is a
 * packaging convenience of this library.
 * The scratch lives in one fixed array inside the library (16 MiB of device memory held on
 * every GPU that loads the library, until the process exits), so sizes are limited to
 * lines->n <= ROX_STATIC_MAX_LINES and grid->n <= ROX_STATIC_MAX_GRID; larger problems
 * return ROX_ERANGE (use rox_xsec with a workspace). Arguments and results are those of
 * rox_xsec; status_out (device, 1 x int32, may be NULL) receives the call's device-side
 * status (ROX_OK, or ROX_EUNSORTED with sigma_out untouched), stream-ordered.
 * No cudaMalloc, cudaFree or other allocation is made. The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture. A cudaDeviceReset unloads the
 * array: after one, restart the process before calling this entry point again. All calls share the one array: calls that overlap on the GPU (different
 * streams, or different host threads, on one device) race and corrupt each other's results;
 * serialise them. Each call clears the parts of the array that must start at zero. */
#define ROX_STATIC_MAX_LINES 262144
#define ROX_STATIC_MAX_GRID (1 << 21)
int rox_xsec_static(const rox_lines* lines, const rox_grid* grid, double P_bar, double T, double Q_T,
                    double Q_ref, double mass_amu, double cutoff, float* sigma_out, int32_t* status_out,
                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ROX_H */
