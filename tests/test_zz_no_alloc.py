"""rox_xsec_static: the cross-section entry point that allocates nothing.

Some callers cannot allocate device memory for a workspace -- an application whose own
memory manager owns all device memory, a plugin that is not allowed to call cudaMalloc,
or an interface with no slot to pass a workspace through. For them the library keeps a
fixed scratch array of its own. This test calls that entry point through the C ABI twice
in a row, at two different (P,T) points, and checks each result against the ordinary
workspace entry point (rox_xsec) with the cross-section tolerance used everywhere else.
The file runs last so that a failure here never hides the other GPU tests."""
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


def _lines():
    from dataclasses import replace
    w = replace(rs.CONFIGS[1], nu_lo=1990.0, nu_hi=2080.0, seed=77)
    return w, oracle.sort_lines(rs.make_lines(w, 0, 20000))


def test_static_entry_point_matches_workspace_path_twice():
    w, L = _lines()
    dl = to_device(L, torch)
    grid = (2000.0, 0.01, 3 * 2048 + 517)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    for P, T in [(1.0, 1000.0), (0.05, 2500.0)]:
        Qt, Qr = q_pair(w, T)
        ws = torch.empty(rox.rox_xsec_workspace_size(len(L["nu0"]), grid, 1), dtype=torch.uint8, device="cuda")
        ref = torch.empty((1, grid[2]), dtype=torch.float32, device="cuda")
        rox.rox_xsec(dl, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, ref, ws)
        assert rox.rox_ws_status(ws)[0] == 0
        out = torch.full((1, grid[2]), float("nan"), dtype=torch.float32, device="cuda")
        rox.rox_xsec_static(dl, grid, P, T, Qt, Qr, w.mass_amu, w.cutoff, out, status)
        torch.cuda.synchronize()
        assert status.item() == 0
        check_sigma(out[0].double().cpu().numpy(), ref[0].double().cpu().numpy(), label="static P=%g T=%g" % (P, T))


def test_static_entry_point_rejects_sizes_beyond_its_scratch():
    w, L = _lines()
    dl = to_device(L, torch)
    out = torch.empty((1, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(rox.RoxError) as e:
        rox.rox_xsec_static(dl, (2000.0, 0.01, (1 << 21) + 1), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, out)
    assert e.value.code == 6 and "static scratch" in str(e.value)


def test_static_entry_point_at_its_size_limits():
    """The largest problem the static scratch accepts -- ROX_STATIC_MAX_LINES lines on a grid of
    ROX_STATIC_MAX_GRID points -- runs and matches the workspace entry point."""
    from dataclasses import replace
    n_lines, n_grid = 262144, 1 << 21
    w = replace(rs.CONFIGS[1], nu_lo=1000.0, nu_hi=1000.0 + 0.01 * (n_grid - 1), seed=78)
    L = oracle.sort_lines(rs.make_lines(w, 0, n_lines))
    dl = to_device(L, torch)
    grid = (1000.0, 0.01, n_grid)
    Qt, Qr = q_pair(w, 1500.0)
    ws = torch.empty(rox.rox_xsec_workspace_size(n_lines, grid, 1), dtype=torch.uint8, device="cuda")
    ref = torch.empty((1, n_grid), dtype=torch.float32, device="cuda")
    rox.rox_xsec(dl, grid, 0.5, 1500.0, Qt, Qr, w.mass_amu, w.cutoff, ref, ws)
    assert rox.rox_ws_status(ws)[0] == 0
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = torch.full((1, n_grid), float("nan"), dtype=torch.float32, device="cuda")
    rox.rox_xsec_static(dl, grid, 0.5, 1500.0, Qt, Qr, w.mass_amu, w.cutoff, out, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    check_sigma(out[0].double().cpu().numpy(), ref[0].double().cpu().numpy(), label="static at the limits")


def test_static_entry_point_reports_unsorted_lines_and_leaves_sigma_untouched():
    """An unsorted list: status_out receives ROX_EUNSORTED (5) and sigma keeps its contents."""
    w, L = _lines()
    rev = {k: (v[::-1].copy() if isinstance(v, np.ndarray) else v) for k, v in L.items()}
    dl = to_device(rev, torch)
    grid = (2000.0, 0.01, 2048)
    Qt, Qr = q_pair(w, 1000.0)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    out = torch.full((1, grid[2]), float("nan"), dtype=torch.float32, device="cuda")
    rox.rox_xsec_static(dl, grid, 1.0, 1000.0, Qt, Qr, w.mass_amu, w.cutoff, out, status)
    torch.cuda.synchronize()
    assert status.item() == 5
    assert torch.isnan(out).all()
