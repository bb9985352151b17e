"""GPU parity of main-contributor line selection (keep a line iff its strength is at least
rel times the largest strength in its nu0 bin, at each temperature): the kept set bit for bit,
the cross-section of the kept lines within the usual tolerance, through the C ABI."""
from dataclasses import replace

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


def _select_xsec(dl, grid, pts, q_ref, mass, cutoff, rel, bw, sigma=None):
    n_temps = len(set(t for _, t, _ in pts))
    ws = torch.empty(rox.rox_xsec_select_workspace_size(dl["nu0"].numel(), grid, n_temps, cutoff, rel, bw),
                     dtype=torch.uint8, device="cuda")
    if sigma is None:
        sigma = torch.empty((len(pts), grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec_select_batch(dl, grid, [p for p, _, _ in pts], [t for _, t, _ in pts], [q for _, _, q in pts], q_ref,
                              mass, cutoff, rel, bw, sigma, ws)
    rc, evals = rox.rox_ws_status(ws)
    assert rc == 0, rox.lib.rox_last_error()
    return sigma.double().cpu().numpy(), evals


def _gpu_mask(dl, grid, cutoff, T, Qt, Qr, rel, bw):
    n = dl["nu0"].numel()
    ws = torch.empty(rox.rox_xsec_select_workspace_size(n, grid, 1, cutoff, rel, bw), dtype=torch.uint8,
                     device="cuda")
    keep = torch.empty(n, dtype=torch.uint8, device="cuda")
    rox.rox_line_select(dl, grid, cutoff, T, Qt, Qr, rel, bw, keep, ws)
    return keep.cpu().numpy().astype(bool)


@pytest.mark.parametrize("conv", [0, 1])
def test_selection_bit_exact(conv):
    w = rs.CONFIGS[1] if conv == 0 else rs.CONFIGS[2]
    w = replace(w, nu_lo=1950.0, nu_hi=2550.0, seed=31 + conv)
    L = oracle.sort_lines(rs.make_lines(w, 0, 200_000))
    grid = (2000.0, 0.01, 50001)
    dl = to_device(L, torch)
    for T in (300.0, 1500.0):
        Qt, Qr = q_pair(w, T)
        S = oracle.line_strength(L, T, Qt, Qr)
        for rel, bw in ((0.0, 1.0), (1e-3, 1.0), (1e-2, 0.1), (0.5, 5.0), (1e-6, 1e9)):
            got = _gpu_mask(dl, grid, 25.0, T, Qt, Qr, rel, bw)
            origin, nb = oracle.select_bins(grid, 25.0, bw)
            ref = oracle.select_mask(L["nu0"], S, rel, bw, origin, nb)
            assert np.array_equal(got, ref), (T, rel, bw, int((got != ref).sum()))


def test_selected_cross_sections():
    """Config 1's lines, three temperatures in one call (each with its own selection)."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    dl = to_device(L, torch)
    rel, bw = 1e-3, 1.0
    pts = []
    for T in (500.0, 1000.0, 2500.0):
        Qt, Qr = q_pair(w, T)
        pts.append((1.0, T, Qt))
    got, evals = _select_xsec(dl, grid, pts, Qr, w.mass_amu, w.cutoff, rel, bw)
    kept_evals = 0
    for k, (P, T, Qt) in enumerate(pts):
        Lk, keep = oracle.select_lines(L, grid, w.cutoff, T, Qt, Qr, rel, bw)
        assert 0 < keep.sum() < keep.size
        ref = oracle.xsec_windowed(Lk, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
        check_sigma(got[k], ref, label="selected rel=%g T=%g (%d of %d lines)" % (rel, T, keep.sum(), keep.size))
        kept_evals += oracle.count_evals(Lk["nu0"], *grid, w.cutoff)
        full = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
        M = full.max()
        big = full > 1e-3 * M
        print("SELECTION T=%g: kept %d of %d lines; max rel change vs all lines where sigma > 1e-3 max: %.2e" % (
            T, keep.sum(), keep.size, float(np.max(np.abs(ref[big] - full[big]) / full[big]))))
    assert evals == kept_evals


def test_rel_zero_equals_unselected():
    """rel = 0 keeps every line that reaches the grid: the unselected result. The kept-line
    index then lists every line the spans reach, in the same order; a few strengths the
    selection recomputed in the FP64 form (bin maxima) differ from the plain launch's reduced
    form by a few 1e-7, so the check allows rounding."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    dl = to_device(L, torch)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    got, _ = _select_xsec(dl, grid, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff, 0.0, 2.0)
    ws = torch.empty(rox.rox_xsec_workspace_size(L["nu0"].size, grid, 1), dtype=torch.uint8, device="cuda")
    sig = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec(dl, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sig, ws)
    plain = sig[0].double().cpu().numpy()
    check_sigma(got[0], plain, rel_tol=1e-5, label="rel = 0 vs unselected launch")


def test_selection_full_size_sample():
    """Config 2 (1e7 lines, 2,970,001 points) with rel = 1e-3 per 1 cm^-1 bin; the oracle on
    exact 96-point windows from the kept lines."""
    w = rs.CONFIGS[2]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    got, evals = _select_xsec(to_device(L, torch), grid, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff, 1e-3, 1.0)
    Lk, keep = oracle.select_lines(L, grid, w.cutoff, T, Qt, Qr, 1e-3, 1.0)
    M = float(got[0].max())
    rng = np.random.default_rng(9)
    for j0 in rng.integers(0, grid[2] - 96, 8):
        ref = oracle.xsec_window(Lk, grid, int(j0), int(j0) + 96, P, T, Qt, Qr, w.mass_amu, w.cutoff)
        check_sigma(got[0][j0:j0 + 96], ref, M=M, label="selected full size window %d" % j0)
    assert evals == oracle.count_evals(Lk["nu0"], *grid, w.cutoff)
    print("SELECTION config 2: kept %d of %d lines, %d evaluations" % (keep.sum(), keep.size, evals))


def test_selection_more_temperatures_than_one_launch():
    """Ten distinct temperatures: one kept-line list each, grouped eight per launch."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w, 0, 4000))
    grid = (2000.0, 0.02, 25001)
    dl = to_device(L, torch)
    temps = np.linspace(300.0, 3000.0, 10)
    pts = []
    for k, T in enumerate(temps):
        Qt, Qr = q_pair(w, T)
        pts.append((10.0 ** (k / 3.0 - 2.0), float(T), Qt))
    got, evals = _select_xsec(dl, grid, pts, Qr, w.mass_amu, 25.0, 1e-4, 2.0)
    total = 0
    for k, (P, T, Qt) in enumerate(pts):
        Lk, keep = oracle.select_lines(L, grid, 25.0, T, Qt, Qr, 1e-4, 2.0)
        ref = oracle.xsec_windowed(Lk, grid, P, T, Qt, Qr, w.mass_amu, 25.0)
        check_sigma(got[k], ref, label="selected, 10 temperatures, T=%g" % T)
        total += oracle.count_evals(Lk["nu0"], *grid, 25.0)
    assert evals == total
