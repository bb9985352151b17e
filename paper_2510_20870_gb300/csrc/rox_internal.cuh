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
#define ROX_K 8
#define ROX_SPAN (32 * ROX_K)
#define ROX_TILE ROX_SPAN               // grid points per work item (per-item line ranges)

// The far (2-level continued fraction) formula is used only for points with
// x^2 + y^2 >= 22^2. Its per-point offset is X_m = X_0 + 32 m dnu with X_0 the offset at
// the thread's first point, so X_m carries a rounding error of 6e-8 (|X_m| + span); the
// slow zone around each line is therefore at least ROX_FAST_MARGIN * span wide, which
// keeps that error below 2e-6 relative.
#define ROX_FAR_Z2 484.0
#define ROX_FAST_MARGIN 0.032

// Workspace header at the start of every xsec workspace.
struct RoxWsHeader {
  int32_t status;                  // ROX_OK / ROX_EUNSORTED / ROX_ETIMEOUT
  int32_t n_pt;
  unsigned long long evals_lines;  // (line, point) pairs inside the cutoff, one (P,T)
  unsigned long long evals_total;  // evals_lines * n_pt, written by the Voigt kernel
  int32_t work_counter;            // persistent-kernel work queue
  int32_t pad;
  unsigned long long smax_bits[ROX_MAX_PT];  // per distinct temperature: max S (double bits)
};
#define ROX_WS_HEADER_BYTES 8192

// Per (P,T) point parameters of the Voigt kernel.
struct RoxPt {
  float p_fac;      // P / P_ref
  float gG_fac;     // sqrt(2 k T / (m amu)) / c  -> gamma_G = nu0 * gG_fac
  float l2_ratio;   // log2(T_ref / T)           -> (T_ref/T)^n_T = exp2(n_T * l2_ratio)
  int32_t t_idx;    // row of S_T (distinct temperature index)
};

struct RoxVoigtArgs {
  const float4* geo;        // [n_lines] {k0 (float, exact), f*dnu, jlo (int bits), jhi (int bits)}
  const float* S32;         // [n_temps][n_lines] line strength * 2^-e_t (FP32; e_t from smax_bits)
  const void* gamma_ref;
  const void* n_t;
  int32_t width_f16;
  const long long* tile_lo; // [n_tiles]
  const long long* tile_hi;
  int32_t n_tiles;
  int32_t n_pt;
  long long n_lines;
  long long n_grid;
  double nu_min;
  float dnu_f;
  float nu_min_f;
  RoxWsHeader* hdr;
  float* sigma;
  unsigned flags;
  RoxPt pt[ROX_MAX_PT];
};

static inline size_t rox_align256(size_t b) { return (b + 255) & ~(size_t)255; }
