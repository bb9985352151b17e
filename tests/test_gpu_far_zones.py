"""The Voigt kernel's slow-zone boundaries, line by line, against the FP64 oracle.

Each line's far form (rox_faddeeva.cuh) holds only outside its slow zone: the per-line Pade
approximant for y < 0.75 and 0.95 <= y < 11.5 beyond |z|^2 = max(6.5^2, 42 y), the 2-level
continued fraction otherwise beyond |z| = 22. Here one isolated line sits at each side of every
range boundary (and inside each range), broad enough (gamma_G ~ 0.33 cm^-1: mass 2 amu, 3000 K,
near 20,000 cm^-1) that its zone spans hundreds of grid points and the uniform grid's precision
margin does not cover the boundary. Each line's profile must match the oracle within 2e-5
relative: the forms' own bounds (core forms 1.1e-5, Pade 3.5e-6, 2-level fraction 1.1e-5) plus
FP32 accumulation. A zone drawn too small for its form would show errors of 1e-4 and more (the
Pade form at |z| = 8 for y = 4: 1.4e-4)."""
import numpy as np
import pytest

import oracle
from rox_testutil import check_sigma, q_pair, to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402
from test_gpu_parity import _run_xsec, _small_lines  # noqa: E402

Y_VALUES = (0.3, 0.7, 0.7499, 0.75, 0.866, 0.9499, 0.95, 1.0, 1.006, 1.5, 2.0, 4.0, 8.0, 11.49, 11.5, 16.0)
SPACING = 60.0        # cm^-1 between lines: windows (cutoff 25) never overlap
NU_FIRST = 20000.0
P, T, MASS, CUTOFF = 1.0, 3000.0, 2.0, 25.0
PER_LINE_TOL = 2e-5


def test_zone_boundaries_line_by_line():
    n = len(Y_VALUES)
    w, L = _small_lines(1, n, NU_FIRST - 1.0, NU_FIRST + SPACING * n, 7)
    nu0 = NU_FIRST + SPACING * np.arange(n, dtype=np.float64)
    gG = oracle.doppler_width(nu0, T, MASS)
    unit_gl = oracle.lorentz_width(np.ones(n, dtype=np.float64), np.full(n, 0.5), P, T)   # gamma_L per gamma_ref
    L["nu0"] = nu0
    L["n_t"] = np.full(n, 0.5, dtype=np.float32)
    L["gamma_ref"] = (np.asarray(Y_VALUES) * gG / unit_gl).astype(np.float32)
    L["e_lower"] = np.zeros(n, dtype=np.float32)
    y = oracle.lorentz_width(L["gamma_ref"].astype(np.float64), L["n_t"].astype(np.float64), P, T) / gG
    assert np.allclose(y, Y_VALUES, rtol=1e-6)
    assert np.all(gG > 0.3)                          # zones of 6.5 gG and more: hundreds of points
    grid = (NU_FIRST - 30.0, 0.01, int(round((SPACING * n + 30.0) / 0.01)))
    Qt, Qr = q_pair(w, T)
    ref = oracle.xsec_windowed(L, grid, P, T, Qt, Qr, MASS, CUTOFF)
    sig, evals = _run_xsec(to_device(L, torch), grid, [(P, T, Qt)], Qr, MASS, CUTOFF)
    jlo, jhi = oracle.window_indices(nu0, grid[0], grid[1], grid[2], CUTOFF)
    assert evals == int(np.sum(jhi - jlo + 1))
    nu = grid[0] + grid[1] * np.arange(grid[2])
    for i, yv in enumerate(Y_VALUES):
        seg = np.abs(nu - nu0[i]) <= CUTOFF + 0.5
        check_sigma(sig[0][seg], ref[seg], rel_tol=PER_LINE_TOL, label="line y=%g" % yv)
