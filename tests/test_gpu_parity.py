"""GPU parity: every step of the CUDA path, called through the C ABI, against the FP64
oracle on the same seeded inputs (bit-exact for integer work, the cross-section
tolerance for floating point)."""
import numpy as np
import pytest

import oracle
import rox_synth as rs
from rox_testutil import check_sigma, q_pair, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402


def _run_xsec(dl, grid, pts, q_ref, mass, cutoff, flags=0, sigma=None):
    """pts: list of (P, T, Q_T). Returns sigma [n_pt, n] as numpy float64 and the evals count."""
    n_temps = len(set(t for _, t, _ in pts))
    ws = torch.empty(rox.rox_xsec_workspace_size(dl["nu0"].numel(), grid, n_temps), dtype=torch.uint8, device="cuda")
    if sigma is None:
        sigma = torch.empty((len(pts), grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec_batch(dl, grid, [p for p, _, _ in pts], [t for _, t, _ in pts], [q for _, _, q in pts], q_ref,
                       mass, cutoff, sigma, ws, flags=flags)
    rc, evals = rox.rox_ws_status(ws)
    assert rc == 0, rox.lib.rox_last_error()
    return sigma.double().cpu().numpy(), evals


def _small_lines(conv, n, nu_lo, nu_hi, seed, f16=False):
    w = rs.CONFIGS[1] if conv == 0 else rs.CONFIGS[2]
    from dataclasses import replace
    w = replace(w, nu_lo=nu_lo, nu_hi=nu_hi, seed=seed, width_dtype="f16" if f16 else "f32")
    return w, oracle.sort_lines(rs.make_lines(w, 0, n))


# ------------------------------------------------------------------ a1, a2
@pytest.mark.parametrize("conv,f16", [(0, False), (1, False), (0, True)])
def test_strengths_and_widths(conv, f16):
    w, L = _small_lines(conv, 20000, 300.0, 30000.0, 11 + conv, f16)
    dl = to_device(L, torch)
    for P, T in [(1.0, 1000.0), (1e-5, 300.0), (100.0, 3000.0), (0.0, 296.0)]:
        Qt, Qr = q_pair(w, T)
        S = torch.empty(len(L["nu0"]), dtype=torch.float32, device="cuda")
        rox.rox_line_strengths(dl, T, Qt, Qr, S)
        ref = oracle.line_strength(L, T, Qt, Qr)
        got = S.double().cpu().numpy()
        ok = ref > 1e-37   # FP32 normal range
        assert np.allclose(got[ok], ref[ok], rtol=2e-7, atol=0), T
        gG = torch.empty_like(S)
        gL = torch.empty_like(S)
        rox.rox_line_widths(dl, w.mass_amu, P, T, gG, gL)
        assert np.allclose(gG.double().cpu().numpy(), oracle.doppler_width(L["nu0"], T, w.mass_amu), rtol=2e-7, atol=0)
        refL = oracle.lorentz_width(L["gamma_ref"], L["n_t"], P, T)
        assert np.allclose(gL.double().cpu().numpy(), refL, rtol=1e-6, atol=0)


# ------------------------------------------------------------------ a3
def test_sort_is_stable_and_exact():
    w = rs.CONFIGS[2]
    L = rs.make_lines(w, 0, 300_001)
    L["nu0"][1000:1010] = L["nu0"][5]          # ties keep input order
    dl = to_device(L, torch)
    n = len(L["nu0"])
    out = {k: torch.empty_like(v) for k, v in dl.items() if k != "convention" and v is not None}
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    ws = torch.empty(rox.rox_sort_workspace_size(n), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(dl, out, perm, ws)
    order = np.argsort(L["nu0"], kind="stable")
    assert np.array_equal(perm.cpu().numpy(), order)
    for k in ("nu0", "s_or_a", "g_up", "e_lower", "gamma_ref", "n_t"):
        assert np.array_equal(out[k].cpu().numpy(), L[k][order]), k


@pytest.mark.parametrize("grid,cutoff", [((2000.0, 0.01, 50001), 25.0), ((300.0, 0.01, 2970001), 25.0),
                                         ((10.0, 0.37, 3333), 3.3), ((2000.0, 0.25, 4001), 1.0)])
def test_windows_bit_exact(grid, cutoff):
    rng = np.random.default_rng(5)
    lo, hi = grid[0] - 2 * cutoff, grid[0] + grid[1] * (grid[2] - 1) + 2 * cutoff
    nu0 = np.sort(rng.uniform(lo, hi, 200_000))
    # lines exactly on cutoff boundaries of the lattice
    nu0[:50] = np.sort(grid[0] + grid[1] * rng.integers(0, grid[2], 50) + cutoff)
    nu0 = np.sort(nu0)
    d = torch.from_numpy(nu0).cuda()
    n = len(nu0)
    jlo = torch.empty(n, dtype=torch.int32, device="cuda")
    jhi = torch.empty_like(jlo)
    k0 = torch.empty_like(jlo)
    f = torch.empty(n, dtype=torch.float32, device="cuda")
    ev = torch.zeros(1, dtype=torch.int64, device="cuda")
    uns = torch.zeros(1, dtype=torch.int32, device="cuda")
    rox.rox_line_windows(d, grid, cutoff, jlo, jhi, k0, f, ev, uns)
    rlo, rhi = oracle.window_indices(nu0, *grid, cutoff)
    assert np.array_equal(jlo.cpu().numpy(), np.clip(rlo, 0, grid[2]))
    assert np.array_equal(jhi.cpu().numpy(), np.clip(rhi, -1, grid[2] - 1))
    assert int(ev.item()) == oracle.count_evals(nu0, *grid, cutoff)
    assert uns.item() == 0
    # centre decomposition on lines that reach the grid: k0 + f = (nu0 - nu_min)/dnu, f in [0, 1]
    # (at an exact lattice point either k0 = k, f = 0 or k0 = k - 1, f = 1 may come out)
    reach = np.clip(rhi, -1, grid[2] - 1) >= np.clip(rlo, 0, grid[2])
    u = (nu0 - grid[0]) / grid[1]
    kk = k0.cpu().numpy()[reach].astype(np.float64)
    ff = f.cpu().numpy()[reach].astype(np.float64)
    assert np.all((ff >= 0) & (ff <= 1)) and np.all(np.abs(kk + ff - u[reach]) <= 1e-6)
    # tile ranges: brute force from the oracle's windows
    W = 2048
    nt = (grid[2] + W - 1) // W
    tlo = torch.empty(nt, dtype=torch.int64, device="cuda")
    thi = torch.empty(nt, dtype=torch.int64, device="cuda")
    rox.rox_tile_ranges(jlo, jhi, grid[2], W, tlo, thi)
    cl, ch = np.clip(rlo, 0, grid[2]), np.clip(rhi, -1, grid[2] - 1)
    for t in range(0, nt, max(1, nt // 50)):
        meets = np.nonzero((ch >= t * W) & (cl <= (t + 1) * W - 1))[0]
        if meets.size:
            assert tlo[t].item() <= meets[0] and thi[t].item() >= meets[-1] + 1
            assert np.all(cl[tlo[t].item():thi[t].item()] <= (t + 1) * W - 1)
            assert np.all(ch[tlo[t].item():thi[t].item()] >= t * W)


def test_unsorted_reported():
    w, L = _small_lines(0, 1000, 2000.0, 2100.0, 3)
    L["nu0"] = L["nu0"][::-1].copy()
    dl = to_device(L, torch)
    grid = (2000.0, 0.01, 10001)
    Qt, Qr = q_pair(w, 1000.0)
    ws = torch.empty(rox.rox_xsec_workspace_size(1000, grid, 1), dtype=torch.uint8, device="cuda")
    sigma = torch.full((1, grid[2]), -7.0, device="cuda")
    rox.rox_xsec_batch(dl, grid, [1.0], [1000.0], [Qt], Qr, 18.0, 25.0, sigma, ws)
    rc, _ = rox.rox_ws_status(ws)
    assert rc == 5
    assert torch.all(sigma == -7.0)     # outputs untouched


# ------------------------------------------------------------------ Faddeeva on the device
def test_device_faddeeva_matches_wofz():
    from scipy.special import wofz
    x = np.concatenate([np.linspace(0, 8, 1601), np.linspace(8, 40, 801), np.logspace(np.log10(40), 5, 200)])
    y = np.concatenate([[0.0], np.logspace(-9, 4, 300)])
    X, Y = np.meshgrid(x, y)
    X = X.ravel().astype(np.float32)
    Y = Y.ravel().astype(np.float32)
    out = torch.empty(X.size, dtype=torch.float32, device="cuda")
    rox.rox_faddeeva_re(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), out)
    got = out.double().cpu().numpy()
    ref = wofz(X.astype(np.float64) + 1j * Y.astype(np.float64)).real
    m = ref > 1e-15
    rel = np.abs(got[m] - ref[m]) / ref[m]
    assert rel.max() < 2e-5, rel.max()


# ------------------------------------------------------------------ a4: full cross-sections
def test_config1_full_vs_oracle():
    """Config 1 over its whole grid, with plain and with compensated (ROX_KAHAN) summation of the
    partial sums; M is the oracle's own maximum."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
    dl = to_device(L, torch)
    for flags, label in ((0, "plain sum"), (rox.ROX_KAHAN, "compensated sum")):
        sig, evals = _run_xsec(dl, grid, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff, flags=flags)
        check_sigma(sig[0], ref, label="config 1, " + label)
        assert evals == oracle.count_evals(L["nu0"], *grid, w.cutoff)


def test_overflow_is_reported():
    """A cross-section beyond the FP32 range (S_ref near FLT_MAX) is written as inf and the call's
    status is ROX_EOVERFLOW; a normal call on the same workspace afterwards reports ROX_OK."""
    w, L = _small_lines(0, 200, 1000.0, 1010.0, 5)
    grid = (1000.0, 0.01, 1001)
    Qt, Qr = q_pair(w, 296.0)
    big = dict(L)
    big["s_or_a"] = np.full(len(L["nu0"]), 3.0e38, dtype=np.float32)
    ws = torch.empty(rox.rox_xsec_workspace_size(len(L["nu0"]), grid, 1), dtype=torch.uint8, device="cuda")
    sigma = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec(to_device(big, torch), grid, 1.0, 296.0, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)
    rc, _ = rox.rox_ws_status(ws)
    assert rc == rox.ROX_EOVERFLOW and not torch.isfinite(sigma).all()
    rox.rox_xsec(to_device(L, torch), grid, 1.0, 296.0, Qt, Qr, w.mass_amu, w.cutoff, sigma, ws)
    assert rox.rox_ws_status(ws)[0] == 0 and torch.isfinite(sigma).all()


@pytest.mark.parametrize("case", ["ragged", "pure_doppler", "lorentz_dominated", "narrow_undersampled",
                                  "outside_grid", "single_line", "empty"])
def test_edge_cases_vs_oracle(case):
    grid = (1000.0, 0.01, 3 * 2048 + 517)            # several tiles and a ragged tail
    nu_lo, nu_hi = 990.0, 1000.0 + 0.01 * grid[2] + 10
    conv, n, P, T, mass = 1, 3000, 0.3, 1200.0, 16.0
    if case == "pure_doppler":
        P = 0.0
    elif case == "lorentz_dominated":
        P, T = 100.0, 300.0
    elif case == "narrow_undersampled":
        P, T, mass = 1e-5, 300.0, 200.0
        grid = (1000.0, 0.05, 3 * 2048 + 517)
    elif case == "outside_grid":
        nu_lo, nu_hi = 900.0, 2000.0
    elif case == "single_line":
        n = 1
    elif case == "empty":
        n = 0
    w, L = _small_lines(conv, max(n, 1), nu_lo, nu_hi, 21)
    if n == 0:
        L = {k: (v[:0] if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    if case == "single_line":
        L["nu0"] = np.array([1000.0 + 0.01 * 2047.5])   # straddles a tile boundary
    Qt, Qr = q_pair(w, T)
    cutoff = 7.5
    ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, mass, cutoff)
    sig, _ = _run_xsec(to_device(L, torch), grid, [(P, T, Qt)], Qr, mass, cutoff)
    if n == 0:
        assert np.all(sig == 0)
        return
    check_sigma(sig[0], ref, label=case)


def test_batch_points_vs_oracle():
    w, L = _small_lines(1, 8000, 4990.0, 5110.0, 31)
    grid = (5000.0, 0.01, 10001)
    pts = []
    for P in (1e-5, 0.01, 1.0, 100.0):
        for T in (300.0, 1500.0, 3000.0):
            pts.append((P, T, q_pair(w, T)[0]))
    Qr = q_pair(w, 296.0)[1]
    sig, evals = _run_xsec(to_device(L, torch), grid, pts, Qr, w.mass_amu, 25.0)
    for k, (P, T, Qt) in enumerate(pts):
        ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, w.mass_amu, 25.0)
        check_sigma(sig[k], ref, label="P=%g T=%g" % (P, T))
    assert evals == len(pts) * oracle.count_evals(L["nu0"], *grid, 25.0)


def test_deterministic_and_accumulate():
    w, L = _small_lines(1, 20000, 4990.0, 5110.0, 41)
    grid = (5000.0, 0.01, 10001)
    dl = to_device(L, torch)
    Qt, Qr = q_pair(w, 800.0)
    a, _ = _run_xsec(dl, grid, [(0.5, 800.0, Qt)], Qr, 16.0, 25.0)
    b, _ = _run_xsec(dl, grid, [(0.5, 800.0, Qt)], Qr, 16.0, 25.0)
    assert np.array_equal(a, b)                     # fixed summation order: bitwise run to run
    # the same list in two chunks, accumulated
    h = 8000
    d1 = {k: (v[:h] if hasattr(v, "shape") else v) for k, v in dl.items()}
    d2 = {k: (v[h:].contiguous() if hasattr(v, "shape") else v) for k, v in dl.items()}
    sig = torch.zeros((1, grid[2]), dtype=torch.float32, device="cuda")
    _run_xsec(d1, grid, [(0.5, 800.0, Qt)], Qr, 16.0, 25.0, flags=rox.ROX_ACCUMULATE, sigma=sig)
    c, _ = _run_xsec(d2, grid, [(0.5, 800.0, Qt)], Qr, 16.0, 25.0, flags=rox.ROX_ACCUMULATE, sigma=sig)
    check_sigma(c[0], a[0].astype(np.float64), rel_tol=1e-5, label="chunked")


@pytest.mark.slow
def test_config2_full_size_sampled_windows():
    w = rs.CONFIGS[2]
    L = rs.make_lines(w)
    dl = to_device(L, torch)
    n = len(L["nu0"])
    out = {k: torch.empty_like(v) for k, v in dl.items() if k != "convention" and v is not None}
    out["convention"] = L["convention"]
    ws = torch.empty(rox.rox_sort_workspace_size(n), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(dl, out, None, ws)
    del ws
    Ls = oracle.sort_lines(L)
    grid = rs.grid_of(w)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    sig, evals = _run_xsec(out, grid, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff)
    assert evals == oracle.count_evals(Ls["nu0"], *grid, w.cutoff)
    rng = np.random.default_rng(2)
    starts = [0, grid[2] - 96] + list(rng.integers(0, grid[2] - 96, 48))
    M = float(sig[0].max())   # the oracle's max is not available at full size; GPU max stands in (1e-4 close)
    worst = 0.0
    for s in starts:
        ref = oracle.xsec_window(Ls, grid, int(s), int(s) + 96, P, T, Qt, Qr, w.mass_amu, w.cutoff)
        worst = max(worst, check_sigma(sig[0, s:s + 96], ref, M=M, label="window %d" % s))
    print("PARITY exomol full size, %d windows: worst %.3e" % (len(starts), worst))


# ------------------------------------------------------------------ a4 for many requests (serving path)
def _prepared_setup(n=30000, seed=91):
    w, L = _small_lines(1, n, 295.0, 1330.0, seed)
    lattice = (300.0, 0.01, 100001)
    dl = to_device(L, torch)
    return w, L, lattice, dl, rox.Prepared(dl, lattice, 25.0)


def test_jobs_windows_match_full_xsec_and_oracle():
    w, L, lattice, dl, prep = _prepared_setup()
    assert prep.status()[0] == 0
    Qr = q_pair(w, 296.0)[1]
    reqs = [(0, 100001, 0.1, 1500.0), (12345, 777, 1e-5, 300.0), (40000, 30001, 100.0, 3000.0),
            (99000, 1001, 3.0, 800.0), (256 * 40 + 17, 1, 0.5, 1000.0)]
    outs, jobs = [], []
    for first, n, P, T in reqs:
        o = torch.full((n,), float("nan"), device="cuda")
        outs.append(o)
        jobs.append(rox.make_job(prep, 0, first, n, P, T, q_pair(w, T)[0], Qr, w.mass_amu, o))
    ws = torch.empty(rox.rox_jobs_workspace_size(jobs), dtype=torch.uint8, device="cuda")
    rox.rox_xsec_jobs([prep], jobs, ws)
    rc, evals = rox.rox_ws_status(ws)
    assert rc == 0
    expect_evals = 0
    for (first, n, P, T), o in zip(reqs, outs):
        full, _ = _run_xsec(dl, lattice, [(P, T, q_pair(w, T)[0])], Qr, w.mass_amu, 25.0)
        got = o.double().cpu().numpy()
        # same lines in the same order as the full grid; only the power-of-two strength scale
        # may differ (per-job maximum), which can change nothing but subnormal-range terms
        check_sigma(got, full[0, first:first + n], M=float(full[0].max()), rel_tol=1e-6, label="vs full grid")
        ref = oracle.xsec_window(L, lattice, first, first + n, P, T, q_pair(w, T)[0], Qr, w.mass_amu, 25.0)
        check_sigma(got, ref, M=float(full[0].max()), label="job %d+%d" % (first, n))
        jlo, jhi = oracle.window_indices(L["nu0"], *lattice, 25.0)
        expect_evals += int(np.sum(np.maximum(np.minimum(jhi, first + n - 1) - np.maximum(jlo, first) + 1, 0)))
    assert evals == expect_evals


def test_jobs_alone_equals_in_mix():
    w, L, lattice, dl, prep = _prepared_setup(20000, 93)
    w2, L2 = _small_lines(1, 5000, 295.0, 1330.0, 95)
    dl2 = to_device(L2, torch)
    prep2 = rox.Prepared(dl2, lattice, 25.0)
    Qr = q_pair(w, 296.0)[1]
    rng = np.random.default_rng(7)
    specs = []
    for k in range(24):
        n = int(rng.integers(1, 20000))
        first = int(rng.integers(0, lattice[2] - n))
        specs.append((int(rng.integers(0, 2)), first, n, float(10 ** rng.uniform(-5, 2)), float(rng.uniform(300, 3000))))
    preps = [prep, prep2]

    def run(subset):
        outs, jobs = [], []
        for li, first, n, P, T in subset:
            o = torch.empty(n, device="cuda")
            outs.append(o)
            jobs.append(rox.make_job(preps[li], li, first, n, P, T, q_pair(w, T)[0], Qr, w.mass_amu, o))
        ws = torch.empty(rox.rox_jobs_workspace_size(jobs), dtype=torch.uint8, device="cuda")
        rox.rox_xsec_jobs(preps, jobs, ws)
        assert rox.rox_ws_status(ws)[0] == 0
        return [o.cpu().numpy() for o in outs]

    mixed = run(specs)
    for k, spec in enumerate(specs):
        alone = run([spec])[0]
        assert np.array_equal(alone, mixed[k]), k


def test_shards_on_one_gpu_reassemble_the_unsharded_result():
    """The multi-GPU plan (no exchange): (P,T) shards and wavenumber shards computed separately
    and concatenated give the unsharded cross-sections."""
    from paper_2510_20870_gb300 import dist as rd
    w, L = _small_lines(1, 12000, 4990.0, 5110.0, 51)
    grid = (5000.0, 0.01, 10001)
    dl = to_device(L, torch)
    Qr = q_pair(w, 296.0)[1]
    pts = [(P, T, q_pair(w, T)[0]) for P in (1e-3, 1.0, 30.0) for T in (500.0, 2500.0)]
    full, _ = _run_xsec(dl, grid, pts, Qr, w.mass_amu, 25.0)
    parts = []
    for r in range(3):
        sub, a = rd.point_shard(pts, 3, r)
        parts.append(_run_xsec(dl, grid, sub, Qr, w.mass_amu, 25.0)[0])
    assert np.array_equal(np.concatenate(parts), full)          # same strength scale per T
    prep = rox.Prepared(dl, grid, 25.0)
    for k, (P, T, Qt) in enumerate(pts):
        pieces = []
        for r in range(4):
            first, n = rd.span_shard(grid[2], rox.ROX_SPAN, 4, r)
            o = torch.empty(n, device="cuda")
            job = rox.make_job(prep, 0, first, n, P, T, Qt, Qr, w.mass_amu, o)
            ws = torch.empty(rox.rox_jobs_workspace_size([job]), dtype=torch.uint8, device="cuda")
            rox.rox_xsec_jobs([prep], [job], ws)
            pieces.append(o.double().cpu().numpy())
        check_sigma(np.concatenate(pieces), full[k], rel_tol=1e-6, label="wavenumber shards")


def test_launch_configurations_change_no_result():
    """The autotuner's knobs (warps per CTA, CTAs per SM, split rounds) select other
    instantiations and grids of the Voigt kernel; every one gives the same cross-section bit for
    bit, and it matches the oracle."""
    w, L = _small_lines(1, 30000, 290.0, 1330.0, 41)
    grid = (300.0, 0.01, 100001)
    pts = [(0.1, 1500.0, q_pair(w, 1500.0)[0])]
    Qr = q_pair(w, 296.0)[1]
    dl = to_device(L, torch)
    outs = []
    try:
        for cfg in [(8, 0, 1), (4, 0, 1), (4, 3, 2), (8, 1, 2)]:
            rox.rox_set_launch_config(*cfg)
            assert rox.rox_get_launch_config()["warps_per_cta"] == cfg[0]
            outs.append(_run_xsec(dl, grid, pts, Qr, w.mass_amu, 25.0, flags=rox.ROX_KAHAN)[0])
    finally:
        rox.rox_reset_launch_config()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    ref = oracle.xsec_window(L, grid, 40000, 40200, 0.1, 1500.0, pts[0][2], Qr, w.mass_amu, 25.0)
    check_sigma(outs[0][0, 40000:40200], ref, M=float(outs[0][0].max()), label="launch configurations")


def test_compensated_and_plain_summation_both_in_use():
    """A list of equal strengths and wide (10 bar) lines: every point sums thousands of terms of
    similar size, so ROX_KAHAN and the plain sum round differently somewhere; both match the
    oracle."""
    w, L = _small_lines(0, 60000, 1000.0, 1060.0, 7)
    L = dict(L)
    L["s_or_a"] = np.full(len(L["nu0"]), 1e-20, dtype=np.float32)
    L["e_lower"] = np.zeros(len(L["nu0"]), dtype=np.float32)
    grid = (1000.0, 0.01, 6001)
    Qt, Qr = q_pair(w, 1000.0)
    dl = to_device(L, torch)
    plain = _run_xsec(dl, grid, [(10.0, 1000.0, Qt)], Qr, w.mass_amu, 25.0, flags=0)[0][0]
    comp = _run_xsec(dl, grid, [(10.0, 1000.0, Qt)], Qr, w.mass_amu, 25.0, flags=rox.ROX_KAHAN)[0][0]
    assert np.any(plain != comp)
    for a in (0, 2900, 5937):
        ref = oracle.xsec_window(L, grid, a, a + 64, 10.0, 1000.0, Qt, Qr, w.mass_amu, 25.0)
        M = float(comp.max())
        e_p = check_sigma(plain[a:a + 64], ref, M=M, label="plain sum %d" % a)
        e_c = check_sigma(comp[a:a + 64], ref, M=M, label="compensated sum %d" % a)
        print("PARITY summation window %d: plain %.3e compensated %.3e" % (a, e_p, e_c))
