"""Pins of the FP64 oracle against facts fixed outside it: published constants,
closed forms and limits of the Voigt profile, an independent quadrature of the
Voigt convolution, invariants of the line sum, and brute force on tiny inputs.

Each pin is a plain function taking the oracle module, so the mutation tests at
the end can show that a planted mistake in the oracle (a dropped factor, a wrong
sign, swapped widths) makes a pin fail."""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erfcx, voigt_profile as scipy_voigt

import oracle
import oracle.rox_oracle as orc
import rox_synth as rs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _consts():
    out = {}
    for line in open(os.path.join(GOLDEN, "physical_constants.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


C = _consts()


def _hitran_line(nu0, s_ref, el, gref=0.07, nt=0.75):
    return {"nu0": np.array([nu0]), "s_or_a": np.array([s_ref]), "e_lower": np.array([el]),
            "gamma_ref": np.array([gref]), "n_t": np.array([nt]), "g_up": None, "convention": 0}


def _exomol_line(nu0, a, g, el, gref=0.07, nt=0.75):
    return {"nu0": np.array([nu0]), "s_or_a": np.array([a]), "g_up": np.array([g]),
            "e_lower": np.array([el]), "gamma_ref": np.array([gref]), "n_t": np.array([nt]),
            "convention": 1}


# ---------------------------------------------------------------- strength (a1)
def pin_c2(o):
    assert abs(o.C2 - C["c2_m_K"] * 100.0) < 1e-9 * o.C2


def pin_hitran_at_tref(o):
    rng = np.random.default_rng(0)
    for _ in range(20):
        L = _hitran_line(rng.uniform(100, 30000), 10 ** rng.uniform(-30, -19), rng.exponential(3000))
        s = o.line_strength(L, o.T_REF, 17.3, 17.3)
        assert s[0] == L["s_or_a"][0]


def pin_exomol_from_oscillator_strength(o):
    # S = pi r_e (g_l f / Q) exp(-c2 E''/T) (1 - exp(-c2 nu/T)) with A from f (published coefficient)
    pi_re_cm = math.pi * C["r_e_m"] * 100.0
    for nu, gl, gu, f, el, T, Q in [(2000.0, 3, 5, 1e-3, 500.0, 1000.0, 123.4),
                                    (345.6, 1, 3, 2e-5, 0.0, 300.0, 10.0),
                                    (25000.0, 7, 9, 0.3, 8000.0, 2500.0, 4.2e4)]:
        A = C["a_from_f_coeff"] * nu * nu * gl / gu * f
        c2 = C["c2_m_K"] * 100.0
        expect = pi_re_cm * gl * f / Q * math.exp(-c2 * el / T) * (1 - math.exp(-c2 * nu / T))
        got = o.line_strength(_exomol_line(nu, A, gu, el), T, Q, 1.0)[0]
        assert abs(got / expect - 1) < 1e-3, (got, expect)


def pin_hitran_exomol_consistency(o):
    # an ExoMol line and the HITRAN line built from its 296 K strength agree at every T
    rng = np.random.default_rng(1)
    q = ("table", np.arange(50.0, 5001.0), 0.05 * np.arange(50.0, 5001.0) ** 1.5)
    for _ in range(20):
        nu0, a, g, el = rng.uniform(300, 30000), 10 ** rng.uniform(-8, 2), float(rng.integers(1, 100)), rng.exponential(5000)
        ex = _exomol_line(nu0, a, g, el)
        qref = o.partition_function(q, o.T_REF)
        sref = o.line_strength(ex, o.T_REF, qref, qref)[0]
        hi = _hitran_line(nu0, sref, el)
        for T in [300.0, 777.7, 1500.0, 3000.0]:
            qt = o.partition_function(q, T)
            s1 = o.line_strength(ex, T, qt, qref)[0]
            s2 = o.line_strength(hi, T, qt, qref)[0]
            assert abs(s1 / s2 - 1) < 1e-12


def pin_partition_table(o):
    q = ("table", np.arange(50.0, 5001.0), 0.05 * np.arange(50.0, 5001.0) ** 1.5)
    assert o.partition_function(q, 1000.0) == 0.05 * 1000.0 ** 1.5
    mid = o.partition_function(q, 1000.25)
    assert mid == pytest.approx(0.75 * 0.05 * 1000.0 ** 1.5 + 0.25 * 0.05 * 1001.0 ** 1.5, rel=1e-15)
    with pytest.raises(ValueError):
        o.partition_function(q, 10.0)


# ---------------------------------------------------------------- widths (a2)
def pin_doppler_published(o):
    for nu0, T, M in [(2000.0, 1000.0, 18.0), (300.0, 300.0, 16.0), (30000.0, 3000.0, 2.0)]:
        hwhm = o.doppler_width(nu0, T, M) * math.sqrt(math.log(2.0))
        assert abs(hwhm / (C["doppler_hwhm_coeff"] * nu0 * math.sqrt(T / M)) - 1) < 3e-4


def pin_lorentz_closed_forms(o):
    assert o.lorentz_width(0.07, 0.75, 1.01325, 296.0) == pytest.approx(0.07, rel=1e-15)
    assert o.lorentz_width(0.07, 0.5, 1.01325, 4 * 296.0) == pytest.approx(0.035, rel=1e-15)
    assert o.lorentz_width(0.07, 0.6, 2 * 1.01325, 296.0) == pytest.approx(0.14, rel=1e-15)
    assert o.lorentz_width(0.07, 0.6, 0.0, 700.0) == 0.0


# ---------------------------------------------------------------- Voigt (a4 profile)
def pin_voigt_gaussian_limit(o):
    gG = 0.013
    d = np.linspace(-0.1, 0.1, 101)
    v = o.voigt_profile(d, gG, 0.0)
    assert np.allclose(v, np.exp(-(d / gG) ** 2) / (gG * math.sqrt(math.pi)), rtol=1e-13, atol=0)


def pin_voigt_centre_erfcx(o):
    gG = 0.02
    for y in [1e-6, 0.03, 0.7, 3.0, 40.0]:
        v = o.voigt_profile(0.0, gG, y * gG)
        assert v == pytest.approx(erfcx(y) / (gG * math.sqrt(math.pi)), rel=1e-13)


def pin_voigt_lorentz_limit(o):
    gL = 0.05
    for gG in [1e-5, 1e-4]:
        for d in [0.3, 1.0, 7.0]:
            lor = gL / (math.pi * (d * d + gL * gL))
            assert o.voigt_profile(d, gG, gL) == pytest.approx(lor, rel=10 * (gG / d) ** 2 + 1e-12)


def pin_voigt_convolution_quadrature(o):
    # V = int G(t) L(d - t) dt, G = exp(-t^2/gG^2)/(gG sqrt(pi)), L = gL/(pi(u^2 + gL^2))
    for gG, gL, d in [(0.01, 0.01, 0.0), (0.01, 0.003, 0.02), (0.05, 0.2, 0.7), (0.02, 0.001, 0.05)]:
        def integrand(t):
            return math.exp(-(t / gG) ** 2) / (gG * math.sqrt(math.pi)) * gL / (math.pi * ((d - t) ** 2 + gL ** 2))
        val, err = integrate.quad(integrand, -12 * gG, 12 * gG, points=[d] if abs(d) < 12 * gG else None,
                                  limit=500, epsabs=0, epsrel=1e-12)
        assert o.voigt_profile(d, gG, gL) == pytest.approx(val, rel=1e-8)


def pin_voigt_scipy_profile(o):
    rng = np.random.default_rng(2)
    for _ in range(50):
        gG, gL, d = 10 ** rng.uniform(-4, -0.5), 10 ** rng.uniform(-7, 1), rng.uniform(-30, 30)
        assert o.voigt_profile(d, gG, gL) == pytest.approx(scipy_voigt(d, gG / math.sqrt(2), gL), rel=1e-10)


def pin_voigt_normalisation(o):
    gG, gL, cut = 0.01, 0.002, 20.0
    d = np.linspace(-cut, cut, 4_000_001)
    area = np.trapezoid(o.voigt_profile(d, gG, gL), d)
    tail = 2 * gL / (math.pi * cut)   # Lorentz wing mass beyond +-cut, leading order
    assert area == pytest.approx(1 - tail, abs=1e-6)


# ---------------------------------------------------------------- the line sum (a3/a4/a5)
def _small(seed=7, n=40, conv=0):
    w = rs.CONFIGS[1] if conv == 0 else rs.CONFIGS[2]
    lines = rs.make_lines(w, 1000 * seed, n)
    return orc.sort_lines(lines)


GRID = (2000.0, 0.01, 50001)
ARGS = (1.0, 1000.0, 5.0e3, 255.0, 18.0, 25.0)  # P, T, Q_T, Q_ref, mass, cutoff


def pin_brute_equals_windowed(o):
    L = _small()
    a = o.xsec_bruteforce(L, GRID, *ARGS)
    b = o.xsec_windowed(L, GRID, *ARGS)
    assert np.array_equal(a, b)


def pin_single_line(o):
    L = _small(n=1)
    sig = o.xsec_bruteforce(L, GRID, *ARGS)
    S = o.line_strength(L, ARGS[1], ARGS[2], ARGS[3])[0]
    gG = o.doppler_width(L["nu0"][0], ARGS[1], ARGS[4])
    gL = o.lorentz_width(L["gamma_ref"][0], L["n_t"][0], ARGS[0], ARGS[1])
    nu = 2000.0 + np.arange(GRID[2]) * 0.01
    d = nu - L["nu0"][0]
    m = np.abs(d) <= 25.0
    # independent profile: scipy's own Voigt routine with sigma = gG/sqrt(2)
    expect = np.where(m, S * scipy_voigt(d, gG / math.sqrt(2), gL), 0.0)
    assert np.allclose(sig, expect, rtol=1e-10, atol=0)
    assert m.sum() in (5000, 5001) and np.count_nonzero(sig) == m.sum()


def pin_linearity_and_permutation(o):
    L = _small(n=30)
    A = {k: (v[:12] if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    B = {k: (v[12:] if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    s = o.xsec_windowed(L, GRID, *ARGS)
    sa = o.xsec_windowed(A, GRID, *ARGS)
    sb = o.xsec_windowed(B, GRID, *ARGS)
    assert np.allclose(s, sa + sb, rtol=1e-14, atol=0)
    perm = np.random.default_rng(3).permutation(30)
    P = {k: (v[perm] if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    assert np.allclose(o.xsec_windowed(P, GRID, *ARGS), s, rtol=1e-14, atol=1e-300)


def pin_grid_shift(o):
    # lines on exact binary lattice values: shifting every nu0 by k steps shifts sigma by k nodes
    grid = (2000.0, 0.25, 4001)
    L = _small(n=10)
    L["nu0"] = 2100.0 + 0.25 * np.arange(10) * 7 + 0.0625
    s0 = o.xsec_windowed(L, grid, *ARGS)
    L2 = dict(L); L2["nu0"] = L["nu0"] + 0.25 * 40
    s1 = o.xsec_windowed(L2, grid, *ARGS)
    # the strength depends on nu0 (stimulated emission), so compare profile shapes per line count
    assert np.count_nonzero(s0) == np.count_nonzero(s1)
    assert np.array_equal(np.nonzero(s0)[0] + 40, np.nonzero(s1)[0])


def pin_cutoff_inclusive(o):
    grid = (2000.0, 0.25, 401)         # exact binary values
    L = _small(n=1)
    L["nu0"] = np.array([2050.0])
    sig = o.xsec_bruteforce(L, grid, *ARGS[:5], 1.0)   # cutoff 1.0: nodes 2049.0 .. 2051.0
    nz = np.nonzero(sig)[0]
    assert nz[0] == 196 and nz[-1] == 204 and nz.size == 9
    jlo, jhi = o.window_indices(L["nu0"], *grid, 1.0)
    assert (jlo[0], jhi[0]) == (196, 204)


def pin_count_evals_bruteforce(o):
    rng = np.random.default_rng(4)
    for grid, cut in [((2000.0, 0.01, 50001), 25.0), ((10.0, 0.37, 333), 3.3), ((-5.0, 1.0, 50), 2.0)]:
        nu0 = rng.uniform(grid[0] - 2 * cut, grid[0] + grid[1] * grid[2] + 2 * cut, 60)
        nu = grid[0] + np.arange(grid[2]) * grid[1]
        brute = int(sum(np.count_nonzero(np.abs(nu - x) <= cut) for x in nu0))
        assert o.count_evals(nu0, *grid, cut) == brute


def pin_points_equal_full(o):
    L = _small(n=60)
    full = o.xsec_windowed(L, GRID, *ARGS)
    js = np.array([0, 17, 2500, 2501, 31337, 50000])
    assert np.array_equal(o.xsec_points(L, GRID, js, *ARGS), full[js])
    assert np.array_equal(o.xsec_window(L, GRID, 123, 4567, *ARGS), full[123:4567])


# ---------------------------------------------------------------- user-provided grids (R14)
def pin_nodes_uniform_equals_windowed(o):
    # a uniform grid handed over as explicit nodes gives the windowed sum bit for bit
    L = _small(n=60)
    full = o.xsec_windowed(L, GRID, *ARGS)
    nodes = o.grid_nodes(*GRID)
    ks = np.array([0, 1, 17, 2500, 2501, 9999, 31337, 49999, 50000])
    assert np.array_equal(o.xsec_nodes(L, nodes, *ARGS, ks=ks), full[ks])


def pin_nodes_bruteforce(o):
    # irregular nodes (clusters and gaps), lines inside and outside the node range
    rng = np.random.default_rng(11)
    nodes = np.sort(np.concatenate([rng.uniform(2000, 2500, 700), 2200 + rng.uniform(0, 0.05, 300)]))
    nodes = np.unique(nodes)
    L = _small(n=25)
    cut = 3.0
    brute = o.xsec_nodes_bruteforce(L, nodes, *ARGS[:5], cut)
    assert np.array_equal(o.xsec_nodes(L, nodes, *ARGS[:5], cut), brute)
    assert np.count_nonzero(brute) > 100


def pin_node_windows(o):
    nodes = o.grid_nodes(*GRID)
    rng = np.random.default_rng(12)
    nu0 = np.concatenate([rng.uniform(1950, 2550, 200), [2000.0 - 25.0, 2500.0 + 25.0, 1900.0, 2600.0]])
    jlo, jhi = o.node_windows(nu0, nodes, 25.0)
    ulo, uhi = o.window_indices(nu0, *GRID, 25.0)
    n = GRID[2]
    assert np.array_equal(jlo, np.clip(ulo, 0, n)) and np.array_equal(jhi, np.clip(uhi, -1, n - 1))
    irr = np.unique(rng.uniform(0, 100, 500))
    for c in rng.uniform(-10, 110, 50):
        inside = np.nonzero(np.abs(irr - c) <= 7.5)[0]
        lo, hi = o.node_windows([c], irr, 7.5)
        if inside.size:
            assert (lo[0], hi[0]) == (inside[0], inside[-1])
        else:
            assert hi[0] < lo[0]


def pin_fixed_resolution(o):
    R = 1.0e5
    nodes = o.fixed_resolution_nodes(2000.0, 2500.0, R)
    ratio = nodes[1:] / nodes[:-1]
    assert np.allclose(ratio, 1.0 + 1.0 / R, rtol=1e-14, atol=0)
    lam = 1.0e4 / nodes                      # micron, descending
    res = lam[1:] / (lam[:-1] - lam[1:])     # lambda / dlambda of each neighbouring pair
    assert np.allclose(res, R, rtol=1e-8, atol=0)
    assert nodes[0] == 2000.0 and nodes[-1] <= 2500.0 < nodes[-1] * (1.0 + 1.0 / R)
    assert nodes.size == int(math.floor(math.log(2500.0 / 2000.0) / math.log1p(1.0 / R))) + 1


# ---------------------------------------------------------------- main-contributor selection (R15)
def pin_select_rules(o):
    rng = np.random.default_rng(13)
    nu0 = np.sort(rng.uniform(1000.0, 1100.0, 4000))
    S = 10.0 ** rng.uniform(-30, -18, nu0.size)
    assert o.select_mask(nu0, S, 0.0, 1.0, 990.0, 200).all()           # rel = 0 keeps every line in range
    one = o.select_mask(nu0, S, 1.0, 1e9, 0.0, 1)                      # one bin, rel = 1: the strongest only
    assert one.sum() == 1 and S[one][0] == S.max()
    m = o.select_mask(nu0, S, 1e-3, 1.0, 990.5, 200)
    b = np.floor(nu0 - 990.5).astype(int)
    for k in np.unique(b):                                             # brute force per bin
        sel = b == k
        assert np.array_equal(m[sel], S[sel] >= 1e-3 * S[sel].max())
    assert (o.select_mask(nu0, S, 1e-2, 1.0, 990.5, 200).sum() <= m.sum()
            <= o.select_mask(nu0, S, 1e-4, 1.0, 990.5, 200).sum())
    part = o.select_mask(nu0, S, 0.0, 1.0, 1050.0, 20)                 # bins cover [1050, 1070) only
    assert np.array_equal(part, (nu0 >= 1050.0) & (nu0 < 1070.0))
    assert o.select_bins((2000.0, 0.01, 50001), 25.0, 1.0) == (1975.0, 551)


def pin_select_sum(o):
    # selection with rel = 0 is the full sum bit for bit; otherwise it is the full sum of the kept lines
    L = _small(n=60)
    P, T, Qt, Qr, mass, cut = ARGS
    full = o.xsec_windowed(L, GRID, *ARGS)
    L0, keep0 = o.select_lines(L, GRID, cut, T, Qt, Qr, 0.0, 1.0)
    assert np.array_equal(o.xsec_windowed(L0, GRID, *ARGS), full)
    Lk, keep = o.select_lines(L, GRID, cut, T, Qt, Qr, 1e-3, 5.0)
    assert 0 < keep.sum() < keep.size
    drop = {k: (v[~keep] if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    assert np.allclose(o.xsec_windowed(Lk, GRID, *ARGS) + o.xsec_windowed(drop, GRID, *ARGS), full,
                       rtol=1e-13, atol=1e-300)


# ---------------------------------------------------------------- broadening descriptions (R16)
def pin_broadening_single_equals_power_law(o):
    L = _small(n=50)
    B = o.apply_broadening(L, [1.0], gamma_ref=[L["gamma_ref"]], n_t=[L["n_t"]])
    for P, T in ((1.0, 1000.0), (1e-3, 300.0), (50.0, 3000.0)):
        assert np.array_equal(o.lorentz_width_broadened(B, P, T), o.lorentz_width(L["gamma_ref"], L["n_t"], P, T))
    assert np.array_equal(o.xsec_windowed(B, GRID, *ARGS), o.xsec_windowed(L, GRID, *ARGS))


def pin_broadening_mixture(o):
    L = _small(n=40)
    g1, n1 = np.full(40, 0.08), np.full(40, 0.5)      # e.g. H2
    g2, n2 = np.full(40, 0.03), np.full(40, 0.7)      # e.g. He
    B = o.apply_broadening(L, [0.85, 0.15], gamma_ref=[g1, g2], n_t=[n1, n2])
    P, T = 3.0, 800.0
    expect = (0.85 * 0.08 * (296.0 / 800.0) ** 0.5 + 0.15 * 0.03 * (296.0 / 800.0) ** 0.7) * 3.0 / 1.01325
    assert np.allclose(o.lorentz_width_broadened(B, P, T), expect, rtol=1e-14, atol=0)
    same = o.apply_broadening(L, [0.3, 0.7], gamma_ref=[g1, g1], n_t=[n1, n1])   # split of one broadener
    one = o.apply_broadening(L, [1.0], gamma_ref=[g1], n_t=[n1])
    assert np.allclose(o.lorentz_width_broadened(same, P, T), o.lorentz_width_broadened(one, P, T), rtol=1e-15)


def pin_broadening_table_and_natural(o):
    L = _small(n=30, conv=1)
    J = np.arange(30) * 3                              # 0..87, beyond the 50-entry table from J = 50
    tg = 0.1 - 0.001 * np.arange(50)
    tn = 0.75 - 0.002 * np.arange(50)
    B = o.apply_broadening(L, [1.0], j_lower=J, table_gamma=[tg], table_n=[tn])
    jj = np.minimum(J, 49)
    assert np.array_equal(B["gamma_b0"], tg[jj]) and np.array_equal(B["n_b0"], tn[jj])
    assert B["gamma_b0"][-1] == tg[49]
    L = dict(L)
    L["s_or_a"] = 10.0 ** np.linspace(7.0, 10.0, 30)   # electronic-band Einstein A: natural widths 3e-5..3e-2
    N = o.apply_broadening(L, [1.0], gamma_ref=[L["gamma_ref"]], n_t=[L["n_t"]], natural=True)
    nat = np.asarray(L["s_or_a"], dtype=np.float64) / (4 * math.pi * C["c_m_s"] * 100.0)
    assert np.allclose(o.lorentz_width_broadened(N, 0.0, 1000.0), nat, rtol=1e-15, atol=0)   # P = 0: natural only
    assert np.allclose(o.lorentz_width_broadened(N, 2.0, 1000.0) - o.lorentz_width(L["gamma_ref"], L["n_t"], 2.0,
                       1000.0), nat, rtol=1e-9, atol=1e-300)


# ---------------------------------------------------------------- CIA restructuring (R17)
def _cia_brute(T_block, nu_blocks, k_blocks, T_out, grid_nu):
    out = []
    for Tt in T_out:
        row = []
        for v in grid_nu:
            val = 0.0
            for Tb, x, y in zip(T_block, nu_blocks, k_blocks):
                if Tb != Tt or not (x[0] <= v <= x[-1]):
                    continue
                if len(x) == 1 or v == x[-1]:
                    val = float(y[-1])
                else:
                    i = 0
                    while not (x[i] <= v < x[i + 1]):
                        i += 1
                    val = float(y[i]) if v == x[i] else float(y[i] + (y[i + 1] - y[i]) * ((v - x[i]) / (x[i + 1] - x[i])))
                break
            row.append(val)
        out.append(row)
    return np.array(out)


def pin_cia_regrid(o):
    rng = np.random.default_rng(17)
    xa = np.sort(rng.uniform(10.0, 500.0, 40)); ya = rng.uniform(1e-46, 1e-44, 40)
    xb = np.sort(rng.uniform(300.0, 900.0, 30)); yb = rng.uniform(1e-46, 1e-44, 30)
    xc = np.array([100.0, 250.0]); yc = np.array([3e-45, 5e-45])
    Tb = [300.0, 300.0, 1000.0]
    grid = np.concatenate([np.linspace(0.0, 1000.0, 701), xa[[0, 5, -1]], xb[[0, -1]], [250.0]])
    grid = np.unique(grid)
    got = o.cia_regrid(Tb, [xa, xb, xc], [ya, yb, yc], [300.0, 1000.0, 2000.0], grid)
    assert np.array_equal(got, _cia_brute(Tb, [xa, xb, xc], [ya, yb, yc], [300.0, 1000.0, 2000.0], grid))
    # samples exactly, coverage inclusive, first block wins where two overlap, zero elsewhere
    for x, y in ((xa, ya),):
        for q in (0, 5, -1):
            assert got[0, np.searchsorted(grid, x[q])] == y[q]
    assert got[0, np.searchsorted(grid, xb[-1])] == yb[-1]
    ov = (grid > xb[0]) & (grid < xa[-1])
    ref_a = o.cia_regrid([300.0], [xa], [ya], [300.0], grid[ov])[0]
    assert ov.any() and np.array_equal(got[0, ov], ref_a)
    assert np.all(got[0, grid < xa[0]] == 0.0) and np.all(got[0, grid > xb[-1]] == 0.0)
    assert np.all(got[2] == 0.0)                       # a temperature without blocks
    # linear coefficients are reproduced (closed form)
    xl = np.sort(rng.uniform(50.0, 950.0, 25)); yl = 2e-46 + 3e-48 * xl
    v = np.linspace(xl[0], xl[-1], 333)
    lin = o.cia_regrid([500.0], [xl], [yl], [500.0], v)[0]
    assert np.allclose(lin, 2e-46 + 3e-48 * v, rtol=1e-13, atol=0)


PINS = [pin_c2, pin_hitran_at_tref, pin_exomol_from_oscillator_strength, pin_hitran_exomol_consistency,
        pin_partition_table, pin_doppler_published, pin_lorentz_closed_forms, pin_voigt_gaussian_limit,
        pin_voigt_centre_erfcx, pin_voigt_lorentz_limit, pin_voigt_convolution_quadrature,
        pin_voigt_scipy_profile, pin_voigt_normalisation, pin_brute_equals_windowed, pin_single_line,
        pin_linearity_and_permutation, pin_grid_shift, pin_cutoff_inclusive, pin_count_evals_bruteforce,
        pin_points_equal_full, pin_nodes_uniform_equals_windowed, pin_nodes_bruteforce, pin_node_windows,
        pin_fixed_resolution, pin_select_rules, pin_select_sum, pin_broadening_single_equals_power_law,
        pin_broadening_mixture, pin_broadening_table_and_natural, pin_cia_regrid]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_oracle_pin(pin):
    pin(oracle)


# ---------------------------------------------------------------- planted mistakes
def _fails(pin):
    try:
        pin(orc)
    except AssertionError:
        return True
    return False


def test_mutation_exomol_prefactor(monkeypatch):
    real = orc.line_strength

    def wrong(lines, T, Q_T, Q_ref):  # drops the 8*pi of the ExoMol prefactor
        s = real(lines, T, Q_T, Q_ref)
        return s * (8 * math.pi) if lines["convention"] == 1 else s
    monkeypatch.setattr(orc, "line_strength", wrong)
    assert _fails(pin_exomol_from_oscillator_strength)


def test_mutation_boltzmann_sign(monkeypatch):
    real_exp = np.exp

    class FakeNp:
        def __getattr__(self, k):
            return getattr(np, k)

        @staticmethod
        def exp(x):  # flips the sign of every exponent (Boltzmann factor)
            return real_exp(-np.asarray(x))
    monkeypatch.setattr(orc, "np", FakeNp())
    assert _fails(pin_hitran_exomol_consistency) or _fails(pin_exomol_from_oscillator_strength)


def test_mutation_stimulated_emission_dropped(monkeypatch):
    monkeypatch.setattr(orc.np, "expm1", lambda x: -np.ones_like(np.asarray(x, dtype=float)), raising=True)
    assert _fails(pin_exomol_from_oscillator_strength)


def test_mutation_widths_swapped(monkeypatch):
    real = orc.voigt_profile
    monkeypatch.setattr(orc, "voigt_profile", lambda d, gG, gL: real(d, gL + 1e-300, gG))
    assert _fails(pin_voigt_centre_erfcx) and _fails(pin_voigt_scipy_profile)


def test_mutation_doppler_half_width_convention(monkeypatch):
    real = orc.doppler_width
    monkeypatch.setattr(orc, "doppler_width", lambda nu0, T, m: real(nu0, T, m) * math.sqrt(math.log(2.0)))
    assert _fails(pin_doppler_published)


def test_mutation_cutoff_exclusive(monkeypatch):
    real = orc.window_indices

    def wrong(nu0, nu_min, dnu, n, cutoff):
        jlo, jhi = real(nu0, nu_min, dnu, n, cutoff)
        return jlo + 1, jhi - 1
    monkeypatch.setattr(orc, "window_indices", wrong)
    assert _fails(pin_cutoff_inclusive) and _fails(pin_count_evals_bruteforce)


def test_mutation_sum_order_index(monkeypatch):
    real = orc.grid_nodes
    monkeypatch.setattr(orc, "grid_nodes", lambda nu_min, dnu, n, j=None: real(nu_min, dnu, n, j) + dnu)
    assert _fails(pin_single_line) or _fails(pin_cutoff_inclusive)


def test_mutation_node_cutoff_exclusive(monkeypatch):
    real = orc.node_windows

    def wrong(nu0, nodes, cutoff):
        jlo, jhi = real(nu0, nodes, cutoff * (1 - 1e-9))   # drops nodes exactly at the cutoff
        return jlo, jhi
    monkeypatch.setattr(orc, "node_windows", wrong)
    assert _fails(pin_node_windows)


def test_mutation_nodes_shifted(monkeypatch):
    real = orc.xsec_nodes
    monkeypatch.setattr(orc, "xsec_nodes", lambda L, nodes, *a, **k: real(L, np.asarray(nodes) + 1e-3, *a, **k))
    assert _fails(pin_nodes_uniform_equals_windowed) and _fails(pin_nodes_bruteforce)


def test_mutation_select_threshold_inverted(monkeypatch):
    real = orc.select_mask
    monkeypatch.setattr(orc, "select_mask", lambda nu0, S, rel, b, og, nb: ~real(nu0, S, rel, b, og, nb))
    assert _fails(pin_select_rules)


def test_mutation_natural_width_fwhm(monkeypatch):
    real = orc.lorentz_width_broadened

    def wrong(lines, P, T):   # natural term as a full width (A / (2 pi c)) instead of the half width
        g = real(lines, P, T)
        if lines["natural"]:
            g = g + np.asarray(lines["s_or_a"], dtype=np.float64) / (4.0 * np.pi * orc.C_LIGHT_CM)
        return g
    monkeypatch.setattr(orc, "lorentz_width_broadened", wrong)
    assert _fails(pin_broadening_table_and_natural)


def test_mutation_cia_last_block_wins(monkeypatch):
    real = orc.cia_regrid
    monkeypatch.setattr(orc, "cia_regrid", lambda Tb, xs, ys, To, g: real(Tb[::-1], xs[::-1], ys[::-1], To, g))
    assert _fails(pin_cia_regrid)


def test_mutation_cia_step_instead_of_linear(monkeypatch):
    def wrong(Tb, xs, ys, To, g):   # the lower sample's value instead of the interpolation
        g = np.asarray(g, dtype=np.float64)
        out = np.zeros((len(To), g.size))
        for t, Tt in enumerate(To):
            for T, x, y in zip(Tb, xs, ys):
                if T == Tt:
                    m = (g >= x[0]) & (g <= x[-1]) & (out[t] == 0)
                    out[t, m] = np.asarray(y)[np.searchsorted(x, g[m], side="right") - 1]
        return out
    monkeypatch.setattr(orc, "cia_regrid", wrong)
    assert _fails(pin_cia_regrid)
