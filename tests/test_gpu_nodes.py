"""GPU parity on user-provided grids (nodes given as float64 values, e.g. of fixed resolving
power R = lambda/dlambda): windows bit-exact, cross-sections within the tolerance of the
uniform grid, against the FP64 oracle on the same seeded inputs, through the C ABI."""
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


def _nodes_xsec(dl, nodes, pts, q_ref, mass, cutoff, flags=0, sigma=None, expect=0):
    """pts: list of (P, T, Q_T). Returns sigma [n_pt, n] (float64 numpy) and the evals count."""
    n_temps = len(set(t for _, t, _ in pts))
    nd = torch.from_numpy(np.ascontiguousarray(nodes, dtype=np.float64)).cuda()
    ws = torch.empty(rox.rox_xsec_nodes_workspace_size(dl["nu0"].numel(), nd.numel(), n_temps), dtype=torch.uint8,
                     device="cuda")
    if sigma is None:
        sigma = torch.empty((len(pts), nd.numel()), dtype=torch.float32, device="cuda")
    rox.rox_xsec_nodes_batch(dl, nd, [p for p, _, _ in pts], [t for _, t, _ in pts], [q for _, _, q in pts], q_ref,
                             mass, cutoff, sigma, ws, flags=flags)
    rc, evals = rox.rox_ws_status(ws)
    assert rc == expect, (rc, rox.lib.rox_last_error())
    return sigma.double().cpu().numpy(), evals


def _lines(conv, n, nu_lo, nu_hi, seed):
    w = rs.CONFIGS[1] if conv == 0 else rs.CONFIGS[2]
    w = replace(w, nu_lo=nu_lo, nu_hi=nu_hi, seed=seed)
    return w, oracle.sort_lines(rs.make_lines(w, 0, n))


def test_node_windows_bit_exact():
    w, L = _lines(1, 200_000, 250.0, 30050.0, 21)
    nodes = rs.fixed_resolution_grid(300.0, 30000.0, rs.FIXED_R)
    nu0 = torch.from_numpy(L["nu0"]).cuda()
    nd = torch.from_numpy(nodes).cuda()
    jlo = torch.empty(nu0.numel(), dtype=torch.int32, device="cuda")
    jhi = torch.empty_like(jlo)
    rox.rox_node_windows(nu0, nd, 25.0, jlo, jhi)
    gl, gh = jlo.cpu().numpy(), jhi.cpu().numpy()
    idx = np.concatenate([np.arange(200), np.arange(L["nu0"].size - 200, L["nu0"].size),
                          np.random.default_rng(0).choice(L["nu0"].size, 3000, replace=False)])
    ol, oh = oracle.node_windows(L["nu0"][idx], nodes, 25.0)
    assert np.array_equal(gl[idx], ol) and np.array_equal(gh[idx], oh)
    # edge lines whose cutoff falls exactly on a node
    c = np.array([nodes[1000] + 25.0, nodes[2_000_000] - 25.0, nodes[0] - 25.0, nodes[-1] + 25.0])
    jl2 = torch.empty(4, dtype=torch.int32, device="cuda")
    jh2 = torch.empty_like(jl2)
    rox.rox_node_windows(torch.from_numpy(c).cuda(), nd, 25.0, jl2, jh2)
    ol, oh = oracle.node_windows(c, nodes, 25.0)
    assert np.array_equal(jl2.cpu().numpy(), ol) and np.array_equal(jh2.cpu().numpy(), oh)


def test_uniform_grid_as_nodes():
    """The uniform grid of config 1 handed over as nodes: the oracle's windowed sum (the
    node form of the oracle reproduces it bit for bit), and the uniform GPU path."""
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    grid = rs.grid_of(w)
    nodes = oracle.grid_nodes(*grid)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    dl = to_device(L, torch)
    got, evals = _nodes_xsec(dl, nodes, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff)
    ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff)
    check_sigma(got[0], ref, label="nodes, uniform config 1")
    assert evals == oracle.count_evals(L["nu0"], *grid, w.cutoff)
    ws = torch.empty(rox.rox_xsec_workspace_size(L["nu0"].size, grid, 1), dtype=torch.uint8, device="cuda")
    sig = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
    rox.rox_xsec(dl, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, sig, ws)
    check_sigma(got[0], sig[0].double().cpu().numpy(), M=float(ref.max()), label="nodes vs uniform path")


def test_fixed_resolution_full_grid():
    w = rs.CONFIGS[1]
    L = oracle.sort_lines(rs.make_lines(w))
    nodes = rs.fixed_resolution_grid(2000.0, 2500.0, 2.0e5)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    got, evals = _nodes_xsec(to_device(L, torch), nodes, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff)
    ref = oracle.xsec_nodes(L, nodes, P, T, Qt, Qr, w.mass_amu, w.cutoff)
    check_sigma(got[0], ref, label="fixed R = 2e5, config 1 lines")
    lo, hi = oracle.node_windows(L["nu0"], nodes, w.cutoff)
    assert evals == int(np.maximum(hi - lo + 1, 0).sum())


@pytest.mark.parametrize("P", [1e-5, 1.0, 100.0])
def test_irregular_nodes_batch(P):
    """Uneven spacing (random nodes plus tight clusters), three temperatures in one call."""
    w, L = _lines(0, 3000, 1990.0, 2510.0, 22)
    nodes = rs.irregular_nodes(23, 2000.0, 2500.0, 6000)
    dl = to_device(L, torch)
    pts = []
    for T in (300.0, 1000.0, 3000.0):
        Qt, Qr = q_pair(w, T)
        pts.append((P, T, Qt))
    got, _ = _nodes_xsec(dl, nodes, pts, Qr, w.mass_amu, 10.0)
    for k, (p, T, Qt) in enumerate(pts):
        ref = oracle.xsec_nodes(L, nodes, p, T, Qt, Qr, w.mass_amu, 10.0)
        check_sigma(got[k], ref, label="irregular nodes P=%g T=%g" % (p, T))


def test_nodes_edge_cases():
    w, L = _lines(0, 500, 2000.0, 2010.0, 24)
    dl = to_device(L, torch)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    cases = {
        "one node": np.array([2005.0]),
        "fewer than a span": np.sort(rs.irregular_nodes(25, 2004.0, 2006.0, 100)),
        "ragged, beyond the lines": rs.fixed_resolution_grid(1995.0, 2030.0, 3.0e5)[:4099],
        "no line in reach": np.linspace(3000.0, 3001.0, 300),
    }
    for name, nodes in cases.items():
        got, _ = _nodes_xsec(dl, nodes, [(P, T, Qt)], Qr, w.mass_amu, 5.0)
        ref = oracle.xsec_nodes(L, nodes, P, T, Qt, Qr, w.mass_amu, 5.0)
        if ref.max() == 0.0:
            assert np.all(got[0] == 0.0), name
        else:
            check_sigma(got[0], ref, label=name)


def test_bad_nodes_leave_sigma_untouched():
    w, L = _lines(0, 200, 2000.0, 2010.0, 26)
    dl = to_device(L, torch)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    for nodes in (np.array([2000.0, 2001.0, 2001.0, 2002.0]), np.array([2003.0, 2002.0, 2004.0]),
                  np.array([2000.0, np.nan, 2002.0])):
        sigma = torch.full((1, nodes.size), -7.0, dtype=torch.float32, device="cuda")
        _nodes_xsec(dl, nodes, [(P, T, Qt)], Qr, w.mass_amu, 5.0, sigma=sigma, expect=rox.ROX_EGRID)
        assert torch.all(sigma == -7.0)


def test_fixed_resolution_full_size_sample():
    """Config 2's 1e7 lines on the fixed-R grid over 300-30000 cm^-1 (2,970,338 nodes), the
    launch the bench times; the oracle at sampled nodes."""
    w = rs.CONFIGS[2]
    L = oracle.sort_lines(rs.make_lines(w))
    nodes = rs.fixed_resolution_grid(300.0, 30000.0, rs.FIXED_R)
    (P, T), = w.pts
    Qt, Qr = q_pair(w, T)
    got, evals = _nodes_xsec(to_device(L, torch), nodes, [(P, T, Qt)], Qr, w.mass_amu, w.cutoff)
    ks = np.concatenate([[0, 1, nodes.size - 1], np.random.default_rng(5).choice(nodes.size, 40, replace=False)])
    ref = oracle.xsec_nodes(L, nodes, P, T, Qt, Qr, w.mass_amu, w.cutoff, ks=ks)
    M = float(got[0].max())
    check_sigma(got[0][ks], ref, M=M, label="fixed R full size, sampled nodes")
    assert evals > 4e10
