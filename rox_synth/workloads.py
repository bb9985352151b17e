"""Synthetic workloads standing in for the paper's line lists (pyROX paper,
"Statement of need" and "Functionality": ExoMol / HITRAN / HITEMP line lists,
cross-sections at each temperature-pressure point).

Five workloads, sized after the configurations this library is measured on:

1. plain     1e4 HITRAN-style lines, one (P,T), 50,001-point grid, 25 cm^-1 wings
2. exomol    1e7 ExoMol-style lines, one (P,T), 2,970,001-point grid
3. batch     1e8 ExoMol-style lines, 15 P x 20 T = 300 (P,T) points
4. large     1e9 HITRAN-style lines (half-precision widths), 100 cm^-1 wings
5. serve     four resident ExoMol-style lists (1e5..1e8 lines) and a Poisson
             request stream of (list, P, T, wavenumber window)

Every column is drawn in FP64 from Philox uniforms and then rounded to its
storage type. Nothing here evaluates any part of the cross-section method.
"""
from dataclasses import dataclass, field
import math
import numpy as np
from .philox import uniform01

HITRAN = 0
EXOMOL = 1

# stream ids of the columns
S_NU0, S_STRENGTH, S_GUP, S_ELOWER, S_GREF, S_NT = 1, 2, 3, 4, 5, 6


@dataclass(frozen=True)
class Workload:
    name: str
    n_lines: int
    seed: int
    convention: int
    nu_lo: float            # nu0 drawn uniform in [nu_lo, nu_hi] (cm^-1)
    nu_hi: float
    strength_lo: float      # S_ref (cm/molecule) or Einstein A (s^-1), log-uniform
    strength_hi: float
    elower_mean: float      # E'' exponential mean (cm^-1)
    mass_amu: float
    grid_lo: float          # uniform output grid, endpoints inclusive
    grid_hi: float
    dnu: float
    cutoff: float           # wing cutoff (cm^-1)
    pts: tuple              # ((P_bar, T_K), ...)
    q_kind: str             # "analytic" (Q = a T^1.5) or "table" (1 K table of a T^1.5, 50-5000 K)
    width_dtype: str = "f32"
    gup_max: int = 100
    gamma_ref_lo: float = 0.02
    gamma_ref_hi: float = 0.1
    n_t_lo: float = 0.4
    n_t_hi: float = 0.8
    q_a: float = 0.05


def _pt_grid(ps, ts):
    return tuple((float(p), float(t)) for p in ps for t in ts)


CONFIGS = {
    1: Workload("plain", 10_000, 1, HITRAN, 2000.0, 2500.0, 1e-30, 1e-19, 3000.0, 18.0,
                2000.0, 2500.0, 0.01, 25.0, ((1.0, 1000.0),), "analytic"),
    2: Workload("exomol", 10_000_000, 2, EXOMOL, 300.0, 30000.0, 1e-8, 1e2, 5000.0, 16.0,
                300.0, 30000.0, 0.01, 25.0, ((0.1, 1500.0),), "table"),
    3: Workload("batch", 100_000_000, 3, EXOMOL, 300.0, 30000.0, 1e-8, 1e2, 5000.0, 16.0,
                300.0, 30000.0, 0.01, 25.0,
                _pt_grid(np.logspace(-5, 2, 15), np.linspace(300.0, 3000.0, 20)), "table"),
    # E'' of the large list is not given by its description; with the HITRAN scaling at 3000 K an
    # exponential of mean 3000 cm^-1 would push the strongest of 1e9 lines to ~1e100 cm/molecule
    # (beyond FP32 cross-sections), so the mean is 1000 cm^-1 (strongest lines ~1e20).
    4: Workload("large", 1_000_000_000, 4, HITRAN, 500.0, 10000.0, 1e-35, 1e-18, 1000.0, 18.0,
                500.0, 10000.0, 0.01, 100.0, ((10.0, 3000.0),), "analytic", width_dtype="f16"),
}

# serving: four resident lists with the exomol distributions
SERVE_LISTS = tuple(
    Workload(f"serve{k}", n, 50 + k, EXOMOL, 300.0, 30000.0, 1e-8, 1e2, 5000.0, 16.0,
             300.0, 30000.0, 0.01, 25.0, (), "table")
    for k, n in enumerate((100_000, 1_000_000, 10_000_000, 100_000_000)))


def grid_of(w: Workload):
    """(nu_min, dnu, n) of the uniform grid nu_j = nu_min + j*dnu, endpoints inclusive."""
    n = int(round((w.grid_hi - w.grid_lo) / w.dnu)) + 1
    return (w.grid_lo, w.dnu, n)


def pt_points(w: Workload):
    return list(w.pts)


def q_table(w: Workload):
    """Partition-function input. 'analytic': returns ('analytic', a) with Q(T) = a*T^1.5.
    'table': returns ('table', T_K, Q) sampled at integer T = 50..5000 K."""
    if w.q_kind == "analytic":
        return ("analytic", w.q_a)
    t = np.arange(50, 5001, dtype=np.float64)
    return ("table", t, w.q_a * t ** 1.5)


def _uniform(w, stream, start, count, lo, hi, idx=None):
    return lo + (hi - lo) * uniform01(w.seed, stream, start, count, idx)


def _loguniform(w, stream, start, count, lo, hi, idx=None):
    u = uniform01(w.seed, stream, start, count, idx)
    return np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)


def _exponential(w, stream, start, count, mean, idx=None):
    return -mean * np.log(uniform01(w.seed, stream, start, count, idx))


def nu0_in_chunks(w: Workload, chunk: int = 10_000_000):
    """Yield (start, nu0) for the whole list, chunk by chunk (line centres only)."""
    for start in range(0, w.n_lines, chunk):
        count = min(chunk, w.n_lines - start)
        yield start, _uniform(w, S_NU0, start, count, w.nu_lo, w.nu_hi)


def make_lines_at(w: Workload, indices):
    """Columns of the lines with the given generation indices (same values as make_lines)."""
    idx = np.asarray(indices, dtype=np.uint64)
    n = idx.size
    wd = np.float16 if w.width_dtype == "f16" else np.float32
    out = {
        "nu0": _uniform(w, S_NU0, 0, n, w.nu_lo, w.nu_hi, idx),
        "s_or_a": _loguniform(w, S_STRENGTH, 0, n, w.strength_lo, w.strength_hi, idx).astype(np.float32),
        "e_lower": _exponential(w, S_ELOWER, 0, n, w.elower_mean, idx).astype(np.float32),
        "gamma_ref": _uniform(w, S_GREF, 0, n, w.gamma_ref_lo, w.gamma_ref_hi, idx).astype(wd),
        "n_t": _uniform(w, S_NT, 0, n, w.n_t_lo, w.n_t_hi, idx).astype(wd),
        "g_up": None,
        "convention": w.convention,
    }
    if w.convention == EXOMOL:
        u = uniform01(w.seed, S_GUP, 0, n, idx)
        out["g_up"] = (1.0 + np.floor(u * w.gup_max)).astype(np.float32)
    return out


def make_lines(w: Workload, start: int = 0, count: int = None):
    """Columns of lines start..start+count-1 (unsorted, in generation order).

    Returns a dict: nu0 float64 (cm^-1); s_or_a float32 (S_ref in cm/molecule at
    296 K for HITRAN, Einstein A in s^-1 for ExoMol); g_up float32 (ExoMol upper-state
    degeneracy, None for HITRAN); e_lower float32 (cm^-1); gamma_ref (cm^-1/atm) and
    n_t as float32 or float16; convention.
    """
    if count is None:
        count = w.n_lines - start
    wd = np.float16 if w.width_dtype == "f16" else np.float32
    out = {
        "nu0": _uniform(w, S_NU0, start, count, w.nu_lo, w.nu_hi),
        "s_or_a": _loguniform(w, S_STRENGTH, start, count, w.strength_lo, w.strength_hi).astype(np.float32),
        "e_lower": _exponential(w, S_ELOWER, start, count, w.elower_mean).astype(np.float32),
        "gamma_ref": _uniform(w, S_GREF, start, count, w.gamma_ref_lo, w.gamma_ref_hi).astype(wd),
        "n_t": _uniform(w, S_NT, start, count, w.n_t_lo, w.n_t_hi).astype(wd),
        "g_up": None,
        "convention": w.convention,
    }
    if w.convention == EXOMOL:
        u = uniform01(w.seed, S_GUP, start, count)
        out["g_up"] = (1.0 + np.floor(u * w.gup_max)).astype(np.float32)
    return out


@dataclass
class Request:
    rid: int
    t_arrival: float     # s
    list_id: int         # index into SERVE_LISTS
    p_bar: float
    t_k: float
    nu_min: float        # window start on the 0.01 cm^-1 lattice of 300-30000
    n: int               # window points


def serve_requests(rate_per_s: float, count: int, seed: int = 5):
    """Poisson request stream: exponential inter-arrival times at the given rate,
    list uniform over the four resident lists, P log-uniform 1e-5..1e2 bar,
    T uniform 300..3000 K, window width uniform 10..5000 cm^-1 on the 0.01 cm^-1
    lattice of 300..30000, start uniform so the window fits."""
    class _W:  # seed holder for the distribution helpers
        pass
    s = _W(); s.seed = seed
    u_gap = uniform01(seed, 101, 0, count)
    u_list = uniform01(seed, 102, 0, count)
    u_p = uniform01(seed, 103, 0, count)
    u_t = uniform01(seed, 104, 0, count)
    u_w = uniform01(seed, 105, 0, count)
    u_s = uniform01(seed, 106, 0, count)
    t = np.cumsum(-np.log(u_gap) / rate_per_s)
    reqs = []
    for i in range(count):
        width = 10.0 + (5000.0 - 10.0) * u_w[i]
        n = int(round(width / 0.01)) + 1
        last_start = int(round((30000.0 - 300.0) / 0.01)) + 1 - n
        k0 = int(math.floor(u_s[i] * (last_start + 1)))
        reqs.append(Request(i, float(t[i]), int(math.floor(u_list[i] * 4)),
                            float(math.exp(math.log(1e-5) + (math.log(1e2) - math.log(1e-5)) * u_p[i])),
                            float(300.0 + 2700.0 * u_t[i]), 300.0 + 0.01 * k0, n))
    return reqs


# User-provided grids (NEXT-1): constant resolving power, and irregular spacing
FIXED_R = 645_000.0        # over 300-30000 cm^-1: 2,970,338 nodes, about the size of config 2's grid


def fixed_resolution_grid(nu_lo: float, nu_hi: float, R: float):
    """Nodes of constant resolving power R = lambda/dlambda: nu_k = nu_lo * (1 + 1/R)^k for
    k = 0..K, K the largest index keeping nu_k <= nu_hi (float64, strictly increasing)."""
    q = 1.0 + 1.0 / float(R)
    K = int(np.floor(np.log(float(nu_hi) / float(nu_lo)) / np.log(q)))
    while K >= 0 and nu_lo * q ** K > nu_hi:
        K -= 1
    return float(nu_lo) * np.power(q, np.arange(K + 1, dtype=np.float64))


def irregular_nodes(seed: int, lo: float, hi: float, n: int):
    """n strictly increasing nodes in [lo, hi] with uneven spacing: half uniform at random,
    half in a few tight clusters (Philox stream 40 of `seed`)."""
    u = uniform01(seed, 40, 0, 2 * n)
    base = lo + (hi - lo) * u[:n // 2]
    centres = lo + (hi - lo) * u[n // 2:n // 2 + 8]
    width = 1e-3 * (hi - lo)
    clus = centres[(np.arange(n - n // 2) % 8)] + width * (u[n:n + n - n // 2] - 0.5)
    nodes = np.unique(np.clip(np.concatenate([base, clus]), lo, hi))
    return nodes.astype(np.float64)


def j_lower_of(w: Workload, start: int = 0, count: int = None):
    """Lower-state rotational quantum number J'' of lines start..start+count-1 (int32, uniform
    0..99; Philox stream 41), the key of J-dependent broadening tables."""
    if count is None:
        count = w.n_lines - start
    return np.floor(100.0 * uniform01(w.seed, 41, start, count)).astype(np.int32)


def cia_blocks(seed: int, temps, lo: float = 20.0, hi: float = 10000.0, samples: int = 4000):
    """Synthetic CIA tables standing in for collision-induced-absorption files (no data files
    are available offline): per temperature one to three blocks covering parts of [lo, hi] with
    irregular, strictly increasing wavenumbers and smooth positive coefficients (cm^5
    molecule^-2 scale). Returns (T_block list, offsets [n_blocks + 1], nu, k) with the blocks
    concatenated (Philox stream 43 of `seed`)."""
    T_block, offsets, nus, ks = [], [0], [], []
    draw = 0
    for T in temps:
        u = uniform01(seed, 43, draw, 4)
        draw += 4
        nb = 1 + int(3 * u[0])
        edges = np.linspace(lo, hi, nb + 1)
        for b in range(nb):
            a, c = edges[b], edges[b + 1]
            m = max(2, samples // nb)
            r = uniform01(seed, 43, draw, m)
            draw += m
            x = np.unique(a + (c - a) * np.sort(r))
            x[0], x[-1] = a, c
            x = np.unique(x)
            centre = lo + (hi - lo) * u[1]
            k = 1e-45 * (float(T) / 300.0) ** 0.5 * (np.exp(-((x - centre) / (0.1 * (hi - lo))) ** 2)
                                                      + 0.3 * np.exp(-((x - lo) / (0.02 * (hi - lo))) ** 2) + 0.01)
            T_block.append(float(T))
            nus.append(x)
            ks.append(k)
            offsets.append(offsets[-1] + x.size)
    return T_block, np.array(offsets, dtype=np.int64), np.concatenate(nus), np.concatenate(ks)
