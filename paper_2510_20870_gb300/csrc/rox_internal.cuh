// Internal definitions shared by the librox translation units (CUDA path only).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "../../include/rox.h"

// Physical constants (CODATA 2018; c, h, k_B exact in SI).
#define ROX_C_CM 2.99792458e10          // speed of light, cm/s
#define ROX_C_M 2.99792458e8            // speed of light, m/s
#define ROX_KB 1.380649e-23             // Boltzmann constant, J/K
#define ROX_HPLANCK 6.62607015e-34      // Planck constant, J s
#define ROX_AMU 1.66053906660e-27       // atomic mass constant, kg
#define ROX_C2 (ROX_HPLANCK * ROX_C_CM / ROX_KB)  // second radiation constant, cm K
#define ROX_T_REF 296.0                 // K, reference temperature of S_ref and gamma_ref
#define ROX_P_REF 1.01325               // bar, 1 atm
#define ROX_PI 3.14159265358979323846

// Voigt work geometry: a warp owns one span of ROX_SPAN = 32*ROX_K consecutive grid points
// (each lane ROX_K points strided by 32) and is its own unit of scheduling; CTAs of
// ROX_WARPS warps only share the Dawson table. Lines reach a warp in batches of 32.
#define ROX_WARPS 8
#define ROX_THREADS (ROX_WARPS * 32)
#define ROX_K (ROX_SPAN / 32)           // ROX_SPAN (include/rox.h) = 256 grid points per span
#define ROX_TILE ROX_SPAN               // grid points per work item (per-item line ranges)

// The far formula (rox_re_w_far in physical units) is used only outside each line's slow
// zone, x^2 + y^2 >= 6.5^2 or 22^2 depending on the line's y. Its per-point offset is
// X_m = X_0 + 32 m dnu with X_0 the offset at the thread's first point, so X_m carries a
// rounding error of 6e-8 (|X_m| + span); the slow zone around each line is therefore at
// least ROX_FAST_MARGIN * span wide, which keeps that error below 2e-6 relative.
#define ROX_FAST_MARGIN 0.032

// Workspace header at the start of every xsec / prepared-list workspace.
struct RoxWsHeader {
  int32_t status;                  // ROX_OK / ROX_EUNSORTED / ROX_EGRID
  int32_t n_pt;
  unsigned long long evals_lines;  // (line, point) pairs inside the cutoff on the whole lattice
  unsigned long long evals_total;  // pairs evaluated by the last Voigt launch(es), all jobs
  int32_t work_counter;            // persistent-kernel work queue
  int32_t overflow;                // set by the Voigt kernel when it writes a non-finite sigma
  unsigned long long smax_bits[ROX_MAX_PT];  // per strength row: max S (double bits)
};
#define ROX_WS_HEADER_BYTES 8192

// Voigt launch: up to ROX_MAX_LISTS prepared line lists and ROX_MAX_JOBS jobs, each job one
// output window on its list's lattice at one (P,T) point; work items are (job, span) pairs.
#define ROX_MAX_JOBS 320
#define ROX_MAX_LISTS 8

struct RoxListDev {
  const int32_t* status;      // the list's preparation status (ROX_OK unless its nu0 was unsorted)
  const float4* geo;          // [n_lines] {k0 (float, exact), f*dnu, jlo (int bits), jhi (int bits)}
  const long long* span_lo;   // per lattice span of ROX_SPAN points: first line reaching it
  const long long* span_hi;   //   and one past the last
  const void* gamma_ref;
  const void* n_t;
  // broadened lists only (else NULL): per line and distinct temperature the broadeners' sum
  // sum_b vmr_b gamma_ref_b (296/T)^n_b, the job's row at gLT + t_row * gLT_stride; per line
  // the natural width (or NULL)
  const float* gLT;
  long long gLT_stride;
  const float* gN;
  // indexed lists only (else NULL): the list's lines as indices into the sorted line arrays, in
  // order (span ranges then count positions in this index)
  const int32_t* idx;
  // user-provided nodes only (NULL on a uniform grid): per node its offset from the first node
  // of its span, per span that first node, both as double-float pairs {hi, lo}; geo then holds
  // {nu0 hi, nu0 lo, jlo, jhi}
  const float2* node_d;
  const float2* span_base;
  // precomputed per-line constants of the launch's one (P,T) point (ROX_VX_PRE lists, else NULL):
  // per line 3 float4, {A, B, P, Q}, {t_z, 1/gamma_G (negative: core-only zone), y, S/(gamma_G
  // sqrt(pi))}, {far form at t_z, zlo (int bits), zhi (int bits), 0}
  const float4* rec;
  long long n_lattice;
  float dnu_f;
  float nu_min_f;
  int32_t width_f16;
  float inv_dnu_f;            // 1/dnu (uniform grid; 0 on nodes)
};

// Lorentz-width description of rox_broadening in kernel parameter form
struct RoxBroadDev {
  int32_t n_b;
  int32_t natural;
  int32_t f16;                 // per-line columns stored as half
  int32_t pad;
  float vmr[ROX_MAX_BROADENERS];
  const void* gamma[ROX_MAX_BROADENERS];
  const void* n[ROX_MAX_BROADENERS];
  const float* tab_gamma[ROX_MAX_BROADENERS];
  const float* tab_n[ROX_MAX_BROADENERS];
  const int32_t* j_lower;
  long long tab_len;
};

// extras of a Voigt launch (kernel instantiations)
#define ROX_VX_INDEX 1    // lists are subsets of the sorted lines given by an index (RoxListDev::idx)
#define ROX_VX_BROAD 2    // widths from the broadening pass (RoxListDev::gLT, gN)
#define ROX_VX_PRE 4      // per-line constants precomputed for the launch's one (P,T) point (RoxListDev::rec)

struct RoxJobDev {
  const float* S32;                      // S * 2^-e of lines l0, l0+1, ... at this job's T
  float* sigma;                          // sigma[j - first] for lattice points j in [first, first + n)
  const unsigned long long* smax_bits;   // this job's largest strength (double bits)
  long long l0;
  long long l1;                          // lines [l0, l1) have strengths (others are skipped)
  long long first;
  long long n;
  int32_t list;
  int32_t span_first;
  int32_t n_spans;
  float p_fac;      // P / P_ref
  float gG_fac;     // sqrt(2 k T / (m amu)) / c  -> gamma_G = nu0 * gG_fac
  float l2_ratio;   // log2(T_ref / T)           -> (T_ref/T)^n_T = exp2(n_T * l2_ratio)
  uint32_t flags;   // ROX_ACCUMULATE, ROX_KAHAN
  int32_t t_row;    // broadened lists: the job's temperature row of the list's gLT
};

// Every span's lines are summed as ROX_PARTS consecutive parts (batch-aligned), each from
// zero, and the part sums are added in part order. A work item is normally a whole span; the
// last items of a launch are split into their parts, taken by different warps: each part stores
// its sum in the tail scratch and the last of them to finish adds the parts in the same order.
// The result is the same either way, so it depends neither on the split nor on the launch grid.
// How many items are split is chosen per launch so that the whole items fill complete rounds of
// the launch's warps and the split ones end the launch in pieces of 1/ROX_PARTS of an item
// (at most ROX_TAIL_ITEMS_MAX items, the size of the workspace's tail scratch).
#define ROX_PARTS 16
#define ROX_TAIL_ITEMS_MAX 8192

struct RoxVoigtArgs {
  RoxWsHeader* hdr;
  float* tail_part;                 // [n_items - n_whole][ROX_PARTS][ROX_SPAN] part sums
  int32_t* tail_cnt;                // [n_items - n_whole] parts finished (zeroed per launch)
  int32_t n_jobs;
  int32_t n_items;                  // items (spans over all jobs); the last n_items - n_whole split
  int32_t n_whole;
  int32_t n_queue;                  // queue entries: n_whole + (n_items - n_whole) * ROX_PARTS
  int32_t item_end[ROX_MAX_JOBS];   // item_end[k] = spans of jobs 0..k
  RoxListDev list[ROX_MAX_LISTS];
  RoxJobDev job[ROX_MAX_JOBS];
};
static_assert(sizeof(RoxVoigtArgs) < 32000, "kernel parameter space");

// Strengths of each job's line range at the job's temperature (rox_xsec_jobs).
struct RoxStrengthList {
  const double* nu0;
  const float* s_or_a;
  const float* g_up;
  const float* e_lower;
  int32_t convention;
  int32_t pad;
};
struct RoxStrengthJob {
  long long l0, count;     // lines [l0, l0 + count) of list `list`
  double* S64;             // [count]
  float* S32;              // [count], S * 2^-e of the job's maximum
  unsigned long long* smax_bits;
  double inv_T, q_ratio, c2_dT;
  int32_t list;
  int32_t pad;
};
struct RoxStrengthJobs {
  int32_t n_jobs;
  int32_t pad;
  RoxStrengthList list[ROX_MAX_LISTS];
  RoxStrengthJob job[ROX_MAX_JOBS];
};
static_assert(sizeof(RoxStrengthJobs) < 32000, "kernel parameter space");

static inline size_t rox_align256(size_t b) { return (b + 255) & ~(size_t)255; }
// tail scratch of a workspace: `cap` items x ROX_PARTS x ROX_SPAN floats, then cap counters
static inline size_t rox_tail_bytes(long long cap) {
  return rox_align256((size_t)cap * ROX_PARTS * ROX_SPAN * sizeof(float)) + rox_align256((size_t)cap * 4);
}
