"""FP64 oracle: line strength, widths, Voigt profile and the truncated line sum.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain NumPy/SciPy in float64.

Paper: pyROX (de Regt et al.), section "Functionality of pyROX":
  * "Compute line-strengths and -widths": strength and broadening widths of every
    transition at the user's pressure and temperature. The paper prints no formula;
    the readings below are the standard HITRAN and ExoMol definitions.
  * "Compute line profiles": Voigt profile = real part of the Faddeeva function
    (Gandhi et al. 2020, Eq. 12), computed with scipy.special.wofz. That routine is
    the one used here.
  * "Combine and save": profiles summed into a cross-section per (P,T).
Readings where the paper is silent:
  R1  constants CODATA 2018; T_ref = 296 K; pressures in bar, P_ref = 1 atm = 1.01325 bar.
  R2  HITRAN strength  S(T) = S_ref * Q(T_ref)/Q(T) * exp(-c2 E''(1/T - 1/T_ref))
                             * (1 - exp(-c2 nu0/T)) / (1 - exp(-c2 nu0/T_ref)).
      ExoMol strength  S(T) = g_up A / (8 pi c nu0^2) * exp(-c2 E''/T) * (1 - exp(-c2 nu0/T)) / Q(T).
      Units cm/molecule (nu0 in cm^-1, c in cm/s).
  R3  Doppler 1/e half-width gamma_G = (nu0/c) sqrt(2 k_B T / (m amu)); HWHM = gamma_G sqrt(ln 2).
  R4  Lorentz HWHM gamma_L = gamma_ref (T_ref/T)^n_T (P / P_ref).
  R5  Voigt V(dnu) = Re w((dnu + i gamma_L)/gamma_G) / (gamma_G sqrt(pi)), unit area over dnu.
  R6  Hard wing cutoff, inclusive: a line contributes to grid point j iff
      |nu_j - nu0| <= cutoff, evaluated in float64 as abs((nu_min + j*dnu) - nu0) <= cutoff.
      No renormalisation, no subtraction of the profile value at the cutoff.
  R7  Point sampling at grid nodes nu_j = nu_min + j*dnu, j = 0..n-1 (computed, not accumulated).
  R8  sigma_j = sum over lines in ascending order of S_i V_ij (float64).
  R9  Partition function: analytic Q(T) = a T^1.5, or a 1 K table interpolated linearly.
  R14 User-provided grids (section "Similar tools": any wavelength or wavenumber grid, e.g.
      a fixed resolution R = lambda/dlambda): the nodes nu_k are given as float64 values,
      strictly increasing; R6 and R8 apply with nu_k in place of nu_min + j*dnu, i.e. a line
      contributes to node k iff abs(nu_k - nu0) <= cutoff in float64.
      A fixed-resolution grid has nu_k = nu_lo * (1 + 1/R)^k (constant nu/dnu, hence constant
      lambda/dlambda), k = 0..K with K the largest index keeping nu_k <= nu_hi.
  R15 Main-contributor selection ("Compute line-strengths and -widths": the line-profile step
      can be sped up by keeping only the main line-strength contributors). At each (P,T), with
      S = S(T) in float64: lines are binned by nu0 into n_bins bins of width B starting at
      origin = nu_min - cutoff, bin = floor((nu0 - origin) / B), n_bins =
      floor(((n - 1) dnu + 2 cutoff) / B) + 1, which covers every nu0 that reaches a grid node;
      line i is kept iff its bin is in range and S_i >= rel * max(S over its bin). rel = 0
      keeps every line that can reach the grid; the strongest line of each bin is always kept.
      The cross-section is then R8 over the kept lines.
  R16 Pressure-broadening descriptions ("Compute line-strengths and -widths": various
      descriptions are supported; none is printed) and natural broadening:
        gamma_L = sum_b x_b gamma_ref_b (T_ref/T)^n_b (P / P_ref)  +  [A / (4 pi c)]
      over broadeners b with mixing ratios x_b (up to 4), each broadener's (gamma_ref_b, n_b)
      per line, either given as columns or looked up in a table by the line's lower-state J
      (J beyond the table takes its last entry); the natural term (Lorentz HWHM of the
      Einstein-A decay, c in cm/s) only for ExoMol lists, where s_or_a is A. Lorentz widths
      add, as Lorentzians convolve into one.
  R17 CIA restructuring ("Combine and save": CIA coefficients restructured into a wavelength- and
      temperature-dependent grid): per output temperature, the first input block of that
      temperature covering a node, linear interpolation in wavenumber between its bracketing
      samples (float64, one written order), 0 where no block covers the node (cia_regrid).
"""
import numpy as np
from scipy.special import wofz

__all__ = [
    "C_LIGHT_CM", "C_LIGHT_M", "K_B", "H_PLANCK", "C2", "AMU", "T_REF", "P_REF_BAR",
    "partition_function", "line_strength", "doppler_width", "lorentz_width",
    "voigt_profile", "grid_nodes", "window_indices", "count_evals",
    "xsec_bruteforce", "xsec_windowed", "xsec_points", "xsec_window", "sort_lines",
    "fixed_resolution_nodes", "node_windows", "xsec_nodes", "xsec_nodes_bruteforce",
    "select_bins", "select_mask", "select_lines", "apply_broadening", "lorentz_width_broadened", "cia_regrid",
]

# R1: CODATA 2018 exact SI values where defined
C_LIGHT_M = 2.99792458e8          # m/s
C_LIGHT_CM = 2.99792458e10        # cm/s
K_B = 1.380649e-23                # J/K
H_PLANCK = 6.62607015e-34         # J s
C2 = H_PLANCK * C_LIGHT_CM / K_B  # second radiation constant, cm K
AMU = 1.66053906660e-27           # kg
T_REF = 296.0                     # K
P_REF_BAR = 1.01325               # 1 atm in bar

HITRAN, EXOMOL = 0, 1


def partition_function(q_input, T):
    """R9. q_input is ('analytic', a) or ('table', T_K, Q)."""
    if q_input[0] == "analytic":
        return q_input[1] * np.power(np.asarray(T, dtype=np.float64), 1.5)
    _, tt, qq = q_input
    T = np.asarray(T, dtype=np.float64)
    if np.any(T < tt[0]) or np.any(T > tt[-1]):
        raise ValueError("temperature outside the partition-function table")
    return np.interp(T, tt, qq)


def line_strength(lines, T, Q_T, Q_ref):
    """R2. Strength S(T) in cm/molecule for every line, float64."""
    nu0 = np.asarray(lines["nu0"], dtype=np.float64)
    el = np.asarray(lines["e_lower"], dtype=np.float64)
    s = np.asarray(lines["s_or_a"], dtype=np.float64)
    stim_T = -np.expm1(-C2 * nu0 / T)       # 1 - exp(-c2 nu0 / T)
    if lines["convention"] == HITRAN:
        stim_ref = -np.expm1(-C2 * nu0 / T_REF)
        boltz = np.exp(-C2 * el * (1.0 / T - 1.0 / T_REF))
        return s * (Q_ref / Q_T) * boltz * (stim_T / stim_ref)
    g = np.asarray(lines["g_up"], dtype=np.float64)
    pref = g * s / (8.0 * np.pi * C_LIGHT_CM * nu0 * nu0)
    return pref * np.exp(-C2 * el / T) * stim_T / Q_T


def doppler_width(nu0, T, mass_amu):
    """R3. 1/e Doppler half-width gamma_G (cm^-1)."""
    nu0 = np.asarray(nu0, dtype=np.float64)
    return nu0 / C_LIGHT_M * np.sqrt(2.0 * K_B * T / (mass_amu * AMU))


def lorentz_width(gamma_ref, n_t, P_bar, T):
    """R4. Lorentz HWHM gamma_L (cm^-1)."""
    g = np.asarray(gamma_ref, dtype=np.float64)
    n = np.asarray(n_t, dtype=np.float64)
    return g * np.power(T_REF / T, n) * (P_bar / P_REF_BAR)


def voigt_profile(dnu, gamma_G, gamma_L):
    """R5. Area-normalised Voigt profile (cm) via scipy.special.wofz."""
    z = (np.asarray(dnu, dtype=np.float64) + 1j * np.asarray(gamma_L, dtype=np.float64)) / gamma_G
    return wofz(z).real / (gamma_G * np.sqrt(np.pi))


def grid_nodes(nu_min, dnu, n, j=None):
    """R7. nu_j = nu_min + j*dnu in float64 (one multiply, one add, no accumulation)."""
    if j is None:
        j = np.arange(n, dtype=np.float64)
    return nu_min + np.asarray(j, dtype=np.float64) * dnu


def _inside(nu_min, dnu, j, nu0, cutoff):
    """R6 predicate for integer index arrays j (float64 arithmetic, as written)."""
    return np.abs(grid_nodes(nu_min, dnu, None, j) - nu0) <= cutoff


def window_indices(nu0, nu_min, dnu, n, cutoff):
    """Per line, the first and last grid index (unclipped) satisfying R6.

    With d_j = (nu_min + j*dnu) - nu0 in float64, R6 reads -cutoff <= d_j <= cutoff.
    d_j is non-decreasing in j, so jlo is the first j with d_j >= -cutoff and jhi
    the last j with d_j <= cutoff. A candidate from one division is moved until
    these two tests themselves hold at the ends and fail just outside.
    Returns (jlo, jhi) int64 arrays; jlo > jhi means the line touches no node.
    """
    nu0 = np.asarray(nu0, dtype=np.float64)

    def d(j):
        return grid_nodes(nu_min, dnu, None, j) - nu0

    jlo = np.ceil((nu0 - cutoff - nu_min) / dnu).astype(np.int64)
    jhi = np.floor((nu0 + cutoff - nu_min) / dnu).astype(np.int64)
    for _ in range(8):
        jlo = np.where(d(jlo - 1) >= -cutoff, jlo - 1, jlo)
        jlo = np.where(d(jlo) < -cutoff, jlo + 1, jlo)
        jhi = np.where(d(jhi + 1) <= cutoff, jhi + 1, jhi)
        jhi = np.where(d(jhi) > cutoff, jhi - 1, jhi)
    assert np.all(d(jlo) >= -cutoff) and np.all(d(jlo - 1) < -cutoff)
    assert np.all(d(jhi) <= cutoff) and np.all(d(jhi + 1) > cutoff)
    return jlo, jhi


def count_evals(nu0, nu_min, dnu, n, cutoff):
    """Number of (line, grid node) pairs inside the cutoff (the unit of work)."""
    jlo, jhi = window_indices(nu0, nu_min, dnu, n, cutoff)
    lo = np.maximum(jlo, 0)
    hi = np.minimum(jhi, n - 1)
    return int(np.sum(np.maximum(hi - lo + 1, 0)))


def sort_lines(lines):
    """Lines in ascending nu0 (stable, so equal nu0 keep generation order)."""
    order = np.argsort(np.asarray(lines["nu0"]), kind="stable")
    out = {}
    for k, v in lines.items():
        out[k] = v[order] if isinstance(v, np.ndarray) else v
    return out


def _line_params(lines, P_bar, T, Q_T, Q_ref, mass_amu):
    S = line_strength(lines, T, Q_T, Q_ref)
    gG = doppler_width(lines["nu0"], T, mass_amu)
    if "vmr" in lines:
        gL = lorentz_width_broadened(lines, P_bar, T)
    else:
        gL = lorentz_width(lines["gamma_ref"], lines["n_t"], P_bar, T)
    return S, gG, gL


def apply_broadening(lines, vmr, gamma_ref=None, n_t=None, j_lower=None, table_gamma=None, table_n=None,
                     natural=False):
    """R16: the line dict with per-line columns gamma_b<k>, n_b<k> of each broadener k (from the
    columns gamma_ref[k], n_t[k], or looked up in table_gamma[k], table_n[k] by j_lower, the
    last entry for J beyond the table), the mixing ratios and the natural-broadening switch."""
    out = dict(lines)
    nb = len(vmr)
    for k in range(nb):
        if table_gamma is not None and table_gamma[k] is not None:
            tg = np.asarray(table_gamma[k], dtype=np.float64)
            tn = np.asarray(table_n[k], dtype=np.float64)
            j = np.minimum(np.asarray(j_lower, dtype=np.int64), tg.size - 1)
            out["gamma_b%d" % k] = tg[j]
            out["n_b%d" % k] = tn[j]
        else:
            out["gamma_b%d" % k] = np.asarray(gamma_ref[k], dtype=np.float64)
            out["n_b%d" % k] = np.asarray(n_t[k], dtype=np.float64)
    out["vmr"] = tuple(float(x) for x in vmr)
    out["natural"] = bool(natural)
    return out


def lorentz_width_broadened(lines, P_bar, T):
    """R16. Lorentz HWHM (cm^-1) of a line dict prepared by apply_broadening."""
    g = np.zeros(np.asarray(lines["nu0"]).size, dtype=np.float64)
    for k, x in enumerate(lines["vmr"]):
        g = g + x * lorentz_width(lines["gamma_b%d" % k], lines["n_b%d" % k], P_bar, T)
    if lines["natural"]:
        if lines["convention"] != EXOMOL:
            raise ValueError("natural broadening needs Einstein A (ExoMol lists)")
        g = g + np.asarray(lines["s_or_a"], dtype=np.float64) / (4.0 * np.pi * C_LIGHT_CM)
    return g


def xsec_bruteforce(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff):
    """R8 by brute force: every line against every node, explicit R6 test,
    lines added in the order given. For tiny inputs only (O(lines x nodes))."""
    nu_min, dnu, n = grid
    nu = grid_nodes(nu_min, dnu, n)
    S, gG, gL = _line_params(lines, P_bar, T, Q_T, Q_ref, mass_amu)
    sigma = np.zeros(n, dtype=np.float64)
    nu0 = np.asarray(lines["nu0"], dtype=np.float64)
    for i in range(nu0.size):
        d = nu - nu0[i]
        contrib = S[i] * voigt_profile(d, gG[i], gL[i])
        sigma += np.where(np.abs(d) <= cutoff, contrib, 0.0)
    return sigma


def xsec_windowed(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff):
    """R8, each line touching only its own cutoff window (same order as brute force,
    so the two agree bit for bit: the brute force adds +0.0 elsewhere)."""
    nu_min, dnu, n = grid
    S, gG, gL = _line_params(lines, P_bar, T, Q_T, Q_ref, mass_amu)
    nu0 = np.asarray(lines["nu0"], dtype=np.float64)
    jlo, jhi = window_indices(nu0, nu_min, dnu, n, cutoff)
    sigma = np.zeros(n, dtype=np.float64)
    for i in range(nu0.size):
        a, b = max(int(jlo[i]), 0), min(int(jhi[i]), n - 1)
        if a > b:
            continue
        j = np.arange(a, b + 1)
        d = grid_nodes(nu_min, dnu, n, j) - nu0[i]
        sigma[a:b + 1] += S[i] * voigt_profile(d, gG[i], gL[i])
    return sigma


def xsec_window(lines_sorted, grid, j0, j1, P_bar, T, Q_T, Q_ref, mass_amu, cutoff):
    """sigma at nodes j0..j1-1 exactly (R8), from lines sorted by nu0.

    Only lines with nu0 within cutoff of the window can contribute (R6), so the
    candidate set is cut from the sorted list with a margin and the R6 predicate
    then decides each pair. Lines are added in ascending sorted order, so the
    result equals the full-grid sum at those nodes bit for bit."""
    nu_min, dnu, n = grid
    nu0 = np.asarray(lines_sorted["nu0"], dtype=np.float64)
    lo_nu = grid_nodes(nu_min, dnu, n, j0) - cutoff - 4 * dnu
    hi_nu = grid_nodes(nu_min, dnu, n, j1 - 1) + cutoff + 4 * dnu
    a = int(np.searchsorted(nu0, lo_nu, side="left"))
    b = int(np.searchsorted(nu0, hi_nu, side="right"))
    sub = {k: (v[a:b] if isinstance(v, np.ndarray) else v) for k, v in lines_sorted.items()}
    S, gG, gL = _line_params(sub, P_bar, T, Q_T, Q_ref, mass_amu)
    nu = grid_nodes(nu_min, dnu, n, np.arange(j0, j1))
    sigma = np.zeros(j1 - j0, dtype=np.float64)
    for i in range(b - a):
        d = nu - sub["nu0"][i]
        m = np.abs(d) <= cutoff
        if m.any():
            sigma[m] += S[i] * voigt_profile(d[m], gG[i], gL[i])
    return sigma


def xsec_points(lines_sorted, grid, js, P_bar, T, Q_T, Q_ref, mass_amu, cutoff):
    """sigma at the listed nodes js, one node at a time (exact, same order as R8)."""
    out = np.empty(len(js), dtype=np.float64)
    for k, j in enumerate(js):
        out[k] = xsec_window(lines_sorted, grid, int(j), int(j) + 1, P_bar, T, Q_T, Q_ref, mass_amu, cutoff)[0]
    return out


# ---------------------------------------------------------------- R14: user-provided grids
def fixed_resolution_nodes(nu_lo, nu_hi, R):
    """R14. Nodes nu_k = nu_lo * (1 + 1/R)^k, k = 0..K, K = floor(log(nu_hi/nu_lo)/log(1 + 1/R))
    (each nu_k is one power and one multiply, not accumulated)."""
    q = 1.0 + 1.0 / float(R)
    K = int(np.floor(np.log(float(nu_hi) / float(nu_lo)) / np.log(q)))
    while K >= 0 and nu_lo * q ** K > nu_hi:
        K -= 1
    k = np.arange(K + 1, dtype=np.float64)
    return float(nu_lo) * np.power(q, k)


def node_windows(nu0, nodes, cutoff):
    """R14 windows: per line, the first node k with nodes[k] - nu0 >= -cutoff and the last
    with nodes[k] - nu0 <= cutoff (float64 differences as written; jhi < jlo when the line
    reaches no node). Binary search, valid because the difference is monotone in k."""
    nodes = np.asarray(nodes, dtype=np.float64)
    nu0 = np.atleast_1d(np.asarray(nu0, dtype=np.float64))
    n = nodes.size
    jlo = np.empty(nu0.size, dtype=np.int64)
    jhi = np.empty(nu0.size, dtype=np.int64)
    for i, c in enumerate(nu0):
        a, b = 0, n                       # first k in [0, n] with nodes[k] - c >= -cutoff
        while a < b:
            mid = (a + b) // 2
            if nodes[mid] - c >= -cutoff:
                b = mid
            else:
                a = mid + 1
        jlo[i] = a
        a, b = 0, n                       # first k with nodes[k] - c > cutoff, minus one
        while a < b:
            mid = (a + b) // 2
            if nodes[mid] - c > cutoff:
                b = mid
            else:
                a = mid + 1
        jhi[i] = a - 1
    return jlo, jhi


def xsec_nodes_bruteforce(lines, nodes, P_bar, T, Q_T, Q_ref, mass_amu, cutoff):
    """R8 with R14: every line against every node, explicit cutoff test, lines in the given
    order. Tiny inputs only."""
    nodes = np.asarray(nodes, dtype=np.float64)
    S, gG, gL = _line_params(lines, P_bar, T, Q_T, Q_ref, mass_amu)
    sigma = np.zeros(nodes.size, dtype=np.float64)
    nu0 = np.asarray(lines["nu0"], dtype=np.float64)
    for i in range(nu0.size):
        d = nodes - nu0[i]
        contrib = S[i] * voigt_profile(d, gG[i], gL[i])
        sigma += np.where(np.abs(d) <= cutoff, contrib, 0.0)
    return sigma


def xsec_nodes(lines_sorted, nodes, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, ks=None):
    """R8 with R14 at nodes[ks] (all nodes if ks is None): for each node, the lines whose
    nu0 lies within cutoff (plus a margin) are cut from the sorted list, the cutoff test
    decides each pair, and the lines are added in ascending order (so the result equals the
    brute force on the sorted list bit for bit)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    ks = np.arange(nodes.size) if ks is None else np.asarray(ks)
    nu0 = np.asarray(lines_sorted["nu0"], dtype=np.float64)
    S, gG, gL = _line_params(lines_sorted, P_bar, T, Q_T, Q_ref, mass_amu)
    out = np.zeros(ks.size, dtype=np.float64)
    # lines are sorted, so each node's candidates are one contiguous range
    a_all = np.searchsorted(nu0, nodes[ks] - cutoff * (1 + 1e-12) - 1e-9, side="left")
    b_all = np.searchsorted(nu0, nodes[ks] + cutoff * (1 + 1e-12) + 1e-9, side="right")
    for q, k in enumerate(ks):
        a, b = int(a_all[q]), int(b_all[q])
        if a >= b:
            continue
        d = nodes[k] - nu0[a:b]
        m = np.abs(d) <= cutoff
        contrib = S[a:b][m] * voigt_profile(d[m], gG[a:b][m], gL[a:b][m])
        acc = 0.0
        for v in contrib:                 # ascending line order, one add at a time
            acc += v
        out[q] = acc
    return out


# ---------------------------------------------------------------- R15: main-contributor selection
def select_bins(grid, cutoff, bin_width):
    """R15 bins of a uniform grid: (origin, n_bins)."""
    nu_min, dnu, n = grid
    origin = nu_min - cutoff
    n_bins = int(np.floor(((n - 1) * dnu + 2.0 * cutoff) / bin_width)) + 1
    return origin, n_bins


def select_mask(nu0, S, rel, bin_width, origin, n_bins):
    """R15: boolean mask of the kept lines (S float64 at one temperature)."""
    nu0 = np.asarray(nu0, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    b = np.floor((nu0 - origin) / float(bin_width))
    inr = (b >= 0) & (b < n_bins)
    b = np.where(inr, b, 0).astype(np.int64)
    binmax = {}
    for k, s, ok in zip(b.tolist(), S.tolist(), inr.tolist()):
        if ok and (k not in binmax or s > binmax[k]):
            binmax[k] = s
    thr = np.array([float(rel) * binmax[k] if ok else np.inf for k, ok in zip(b.tolist(), inr.tolist())])
    return inr & (S >= thr)


def select_lines(lines_sorted, grid, cutoff, T, Q_T, Q_ref, rel, bin_width):
    """The kept lines of R15 at temperature T on a uniform grid, as a line dict (same order)."""
    S = line_strength(lines_sorted, T, Q_T, Q_ref)
    origin, n_bins = select_bins(grid, cutoff, bin_width)
    keep = select_mask(lines_sorted["nu0"], S, rel, bin_width, origin, n_bins)
    return {k: (v[keep] if isinstance(v, np.ndarray) else v) for k, v in lines_sorted.items()}, keep


# ---------------------------------------------------------------- R17: CIA restructuring
def cia_regrid(T_block, nu_blocks, k_blocks, T_out, nu_grid):
    """R17 (section "Functionality", "Combine and save": CIA coefficients read from the input
    files are restructured into a wavelength- and temperature-dependent grid). Blocks b hold a
    temperature T_block[b] and strictly increasing wavenumbers nu_blocks[b] with coefficients
    k_blocks[b]. Row t of the result on nodes nu_grid: at each node, the first block (input
    order) with T_block == T_out[t] whose range [nu_first, nu_last] contains the node, linearly
    interpolated between its bracketing samples as
        k_i + (k_{i+1} - k_i) * ((nu - nu_i) / (nu_{i+1} - nu_i))   (float64, in that order),
    the sample's own value at a sample, and 0 where no such block covers the node."""
    nu_grid = np.asarray(nu_grid, dtype=np.float64)
    out = np.zeros((len(T_out), nu_grid.size), dtype=np.float64)
    for t, Tt in enumerate(T_out):
        done = np.zeros(nu_grid.size, dtype=bool)
        for b, Tb in enumerate(T_block):
            if Tb != Tt:
                continue
            x = np.asarray(nu_blocks[b], dtype=np.float64)
            y = np.asarray(k_blocks[b], dtype=np.float64)
            inside = (~done) & (nu_grid >= x[0]) & (nu_grid <= x[-1])
            v = nu_grid[inside]
            i = np.searchsorted(x, v, side="right") - 1          # x[i] <= v < x[i+1], or v == x[-1]
            i = np.minimum(i, x.size - 2) if x.size > 1 else np.zeros_like(i)
            if x.size == 1:
                val = np.full(v.size, y[0])
            else:
                val = y[i] + (y[i + 1] - y[i]) * ((v - x[i]) / (x[i + 1] - x[i]))
                at = v == x[i]
                val[at] = y[i][at]
                last = v == x[-1]
                val[last] = y[-1]
            out[t, inside] = val
            done |= inside
    return out
