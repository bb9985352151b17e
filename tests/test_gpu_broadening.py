"""GPU parity of the pressure-broadening descriptions (broadener mixtures, J-dependent tables)
and natural broadening: the Lorentz widths and the cross-sections against the FP64 oracle on
the same seeded inputs, through the C ABI."""
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

# J-dependent table of one broadener (e.g. He): gamma_ref falls and n_T rises slowly with J
TAB_J = np.arange(60)
TAB_GAMMA = (0.09 * np.exp(-TAB_J / 40.0) + 0.01).astype(np.float32)
TAB_N = (0.45 + 0.004 * TAB_J).astype(np.float32)


def _lines(conv, n, nu_lo, nu_hi, seed, big_a=False):
    """Sorted lines with a second broadener's columns (H2-like: 1.3 x gamma_ref, n_T - 0.1) and J."""
    w = rs.CONFIGS[1] if conv == 0 else rs.CONFIGS[2]
    w = replace(w, nu_lo=nu_lo, nu_hi=nu_hi, seed=seed)
    L = rs.make_lines(w, 0, n)
    L["j_lower"] = rs.j_lower_of(w, 0, n)
    L["gamma_h2"] = (L["gamma_ref"].astype(np.float64) * 1.3).astype(np.float32)
    L["n_h2"] = (L["n_t"].astype(np.float64) - 0.1).astype(np.float32)
    if big_a:   # electronic-band Einstein A, so that the natural width shows next to low-pressure widths
        L["s_or_a"] = (10.0 ** (6.0 + 3.0 * rs.uniform01(seed, 42, 0, n))).astype(np.float32)
    return w, oracle.sort_lines(L)


def _descriptions(L, dl, natural):
    """The same description for the oracle (apply_broadening) and the GPU (dict of tensors):
    0.8 H2 (per-line columns) + 0.2 of the J table."""
    ob = oracle.apply_broadening(L, [0.8, 0.2], gamma_ref=[L["gamma_h2"], None], n_t=[L["n_h2"], None],
                                 j_lower=L["j_lower"], table_gamma=[None, TAB_GAMMA], table_n=[None, TAB_N],
                                 natural=natural)
    gb = {"vmr": [0.8, 0.2],
          "gamma_ref": [torch.from_numpy(L["gamma_h2"]).cuda(), None],
          "n_t": [torch.from_numpy(L["n_h2"]).cuda(), None],
          "table_gamma": [None, torch.from_numpy(TAB_GAMMA).cuda()],
          "table_n": [None, torch.from_numpy(TAB_N).cuda()],
          "j_lower": torch.from_numpy(L["j_lower"]).cuda(),
          "natural": natural}
    return ob, gb


@pytest.mark.parametrize("conv,natural", [(0, False), (1, False), (1, True)])
def test_lorentz_widths(conv, natural):
    w, L = _lines(conv, 20_000, 2000.0, 2500.0, 41 + conv, big_a=natural)
    dl = to_device(L, torch)
    ob, gb = _descriptions(L, dl, natural)
    out = torch.empty(L["nu0"].size, dtype=torch.float32, device="cuda")
    for P, T in ((1.0, 296.0), (1e-4, 300.0), (30.0, 2800.0)):
        rox.rox_lorentz_widths(dl, gb, P, T, out)
        ref = oracle.lorentz_width_broadened(ob, P, T)
        got = out.double().cpu().numpy()
        rel = np.abs(got - ref) / ref
        assert rel.max() < 2e-6, (P, T, rel.max())


def test_broadened_cross_sections():
    """Config 1's lines with the two-broadener description, three (P,T) points in one call."""
    w, L = _lines(0, 10_000, 2000.0, 2500.0, 44)
    grid = rs.grid_of(rs.CONFIGS[1])
    dl = to_device(L, torch)
    ob, gb = _descriptions(L, dl, False)
    pts = []
    for P, T in ((1.0, 1000.0), (0.01, 300.0), (50.0, 2500.0)):
        Qt, Qr = q_pair(w, T)
        pts.append((P, T, Qt))
    ws = torch.empty(rox.rox_xsec_broadened_workspace_size(L["nu0"].size, grid, 3), dtype=torch.uint8, device="cuda")
    sig = torch.empty((3, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec_broadened_batch(dl, grid, gb, [p for p, _, _ in pts], [t for _, t, _ in pts], [q for _, _, q in pts],
                                 Qr, w.mass_amu, w.cutoff, sig, ws)
    rc, evals = rox.rox_ws_status(ws)
    assert rc == 0
    got = sig.double().cpu().numpy()
    for k, (P, T, Qt) in enumerate(pts):
        ref = oracle.xsec_windowed(ob, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
        check_sigma(got[k], ref, label="broadened P=%g T=%g" % (P, T))


def test_natural_broadening_low_pressure():
    """ExoMol lines with electronic-band Einstein A at 1e-5 bar: the natural width is comparable
    to (or larger than) the pressure width there."""
    w, L = _lines(1, 3_000, 2000.0, 2500.0, 45, big_a=True)
    grid = (2000.0, 0.005, 100001)
    dl = to_device(L, torch)
    ob, gb = _descriptions(L, dl, True)
    P, T = 1e-5, 1500.0
    Qt, Qr = q_pair(w, T)
    ws = torch.empty(rox.rox_xsec_broadened_workspace_size(L["nu0"].size, grid, 1), dtype=torch.uint8, device="cuda")
    sig = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec_broadened_batch(dl, grid, gb, [P], [T], [Qt], Qr, w.mass_amu, 5.0, sig, ws)
    assert rox.rox_ws_status(ws)[0] == 0
    ref = oracle.xsec_windowed(ob, grid, P, T, Qt, Qr, w.mass_amu, 5.0)
    check_sigma(sig[0].double().cpu().numpy(), ref, label="natural broadening, P=1e-5 bar")
    gl_nat = oracle.lorentz_width_broadened(ob, P, T)
    ob_off = dict(ob)
    ob_off["natural"] = False
    assert np.median(gl_nat / oracle.lorentz_width_broadened(ob_off, P, T)) > 2.0   # natural term dominates


def test_single_broadener_matches_power_law():
    """One broadener with the list's own columns and vmr = 1 is the single power law."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    dl = to_device(L, torch)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    gb = {"vmr": [1.0], "gamma_ref": [dl["gamma_ref"]], "n_t": [dl["n_t"]], "natural": False}
    ws = torch.empty(rox.rox_xsec_broadened_workspace_size(L["nu0"].size, grid, 1), dtype=torch.uint8, device="cuda")
    sig = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec_broadened_batch(dl, grid, gb, [P], [T], [Qt], Qr, w.mass_amu, w.cutoff, sig, ws)
    ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
    check_sigma(sig[0].double().cpu().numpy(), ref, label="one broadener = power law")


def test_bad_descriptions_rejected():
    w, L = _lines(0, 100, 2000.0, 2010.0, 46)
    dl = to_device(L, torch)
    out = torch.empty(100, dtype=torch.float32, device="cuda")
    for bad in ({"vmr": []}, {"vmr": [1.0, 1.0, 1.0, 1.0, 1.0]}, {"vmr": [-1.0], "gamma_ref": [dl["gamma_ref"]],
                                                                  "n_t": [dl["n_t"]]},
                {"vmr": [1.0]}, {"vmr": [1.0], "gamma_ref": [dl["gamma_ref"]], "n_t": [dl["n_t"]], "natural": True}):
        with pytest.raises(rox.RoxError):
            rox.rox_lorentz_widths(dl, bad, 1.0, 300.0, out)
