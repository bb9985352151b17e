"""The seeded input generator: Philox known answers and the workload shapes."""
import os

import numpy as np

import rox_synth as rs
from rox_synth.philox import philox4x32_10


def test_philox_known_answers():
    path = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = philox4x32_10(*v[:6])
        assert [int(x) for x in out] == v[6:]
        n += 1
    assert n == 3


def test_uniform_open_interval_and_subsets():
    u = rs.uniform01(9, 1, 0, 100000)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.01
    assert np.array_equal(rs.uniform01(9, 1, 500, 100), u[500:600])


def test_workload_columns_and_ranges():
    for cid in (1, 2, 4):
        w = rs.CONFIGS[cid]
        L = rs.make_lines(w, 123, 5000)
        assert L["nu0"].dtype == np.float64 and L["s_or_a"].dtype == np.float32
        assert L["nu0"].min() >= w.nu_lo and L["nu0"].max() <= w.nu_hi
        assert L["s_or_a"].min() >= np.float32(w.strength_lo) * 0.999
        assert L["gamma_ref"].dtype == (np.float16 if w.width_dtype == "f16" else np.float32)
        if w.convention == rs.workloads.EXOMOL:
            g = L["g_up"]
            assert g.min() >= 1 and g.max() <= 100 and np.all(g == np.round(g))
        # any slice regenerates identically
        L2 = rs.make_lines(w, 123 + 1000, 10)
        assert np.array_equal(L2["nu0"], L["nu0"][1000:1010])


def test_grids():
    assert rs.grid_of(rs.CONFIGS[1]) == (2000.0, 0.01, 50001)
    assert rs.grid_of(rs.CONFIGS[2]) == (300.0, 0.01, 2970001)
    assert rs.grid_of(rs.CONFIGS[4]) == (500.0, 0.01, 950001)
    assert len(rs.pt_points(rs.CONFIGS[3])) == 300


def test_requests_fit_the_lattice():
    reqs = rs.serve_requests(200.0, 500)
    t = np.array([r.t_arrival for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(len(reqs) / t[-1] - 200.0) < 30
    for r in reqs:
        assert 300.0 <= r.nu_min and r.nu_min + (r.n - 1) * 0.01 <= 30000.0 + 1e-6
        assert 1e-5 <= r.p_bar <= 1e2 and 300 <= r.t_k <= 3000 and 0 <= r.list_id < 4


def test_lines_at_indices_match_ranges():
    w = rs.CONFIGS[4]
    a = rs.make_lines(w, 5000, 300)
    idx = np.arange(5000, 5300)[::-1]
    b = rs.make_lines_at(w, idx)
    for k in ("nu0", "s_or_a", "e_lower", "gamma_ref", "n_t"):
        assert np.array_equal(a[k][::-1], b[k])
