"""GPU CIA restructuring against the FP64 oracle through the C ABI. Both sides interpolate
in float64 and pick the same interval for every point; the kernels multiply by an interval's
reciprocal width where the oracle divides, and on the uniform grid step from point to point
by the constant increment (k_{i+1} - k_i) dnu / h_i, i.e. they evaluate at the exact grid
point where the oracle evaluates at its rounded value. So the rows agree to 64 roundings of
the values along a lane's run (at most 64 points) plus 4 ulps of nu times the local slope, exactly at
samples, and are zero exactly where the oracle's are."""
import numpy as np
import pytest

import oracle
import rox_synth as rs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402


def _same(got, ref, nu_pts):
    """got == ref within 128 eps (|ref| + 64 gap |slope|) + 4 ulp(nu) |slope|, the slope taken
    from neighbouring covered points of ref; zero exactly where ref is zero."""
    assert got.shape == ref.shape
    assert np.array_equal(got == 0.0, ref == 0.0)
    nu_pts = np.asarray(nu_pts, dtype=np.float64)
    gap = np.diff(nu_pts)
    d = np.abs(np.diff(ref, axis=1)) / gap
    d[(ref[:, 1:] == 0.0) | (ref[:, :-1] == 0.0)] = 0.0      # no slope across a coverage edge
    slope = np.zeros_like(ref)
    slope[:, 1:] = d
    slope[:, :-1] = np.maximum(slope[:, :-1], d)
    # the stepped value carries up to 64 roundings of the largest value along a lane's run
    near = np.abs(ref) + 64 * np.concatenate([gap, gap[-1:]]) * slope if gap.size else np.abs(ref)
    tol = 128 * np.finfo(np.float64).eps * near + 4 * np.spacing(np.abs(nu_pts)) * slope
    err = np.abs(got - ref)
    assert np.all(err <= tol), float(np.max(err / np.maximum(tol, 1e-300)))
    nz = ref != 0.0
    return float(np.max(err[nz] / np.abs(ref[nz]))) if nz.any() else 0.0


def _regrid(Tb, off, nu, k, grid, T_out, out, ws_bytes=None):
    need = rox.rox_cia_workspace_size(len(Tb), int(off[-1]))
    ws = torch.empty(need if ws_bytes is None else ws_bytes, dtype=torch.uint8, device="cuda")
    rox.rox_cia_regrid(Tb, off, nu, k, grid, T_out, out, ws)


def _blocks(seed, temps, samples):
    Tb, off, nu, k = rs.cia_blocks(seed, temps, samples=samples)
    per_nu = [nu[off[b]:off[b + 1]] for b in range(len(Tb))]
    per_k = [k[off[b]:off[b + 1]] for b in range(len(Tb))]
    return Tb, off, torch.from_numpy(nu).cuda(), torch.from_numpy(k).cuda(), per_nu, per_k


def test_cia_uniform_grid():
    temps = [200.0, 300.0, 400.0, 700.0, 1000.0, 2000.0, 3000.0]
    Tb, off, nu, k, pn, pk = _blocks(7, temps, 3000)
    grid = (10.0, 0.37, 30001)                 # starts below and ends beyond the blocks' coverage
    T_out = [3000.0, 300.0, 250.0, 200.0]     # any order; 250 K has no block
    out = torch.empty((len(T_out), grid[2]), dtype=torch.float64, device="cuda")
    _regrid(Tb, off, nu, k, grid, T_out, out)
    pts = oracle.grid_nodes(*grid)
    ref = oracle.cia_regrid(Tb, pn, pk, T_out, pts)
    got = out.cpu().numpy()
    print("CIA uniform grid: max relative difference %.2e" % _same(got, ref, pts))
    assert np.all(got[2] == 0.0) and np.count_nonzero(got[0]) > 20000


def test_cia_nodes():
    temps = [250.0, 600.0]
    Tb, off, nu, k, pn, pk = _blocks(8, temps, 800)
    # fixed-R nodes plus every block sample and both block edges exactly
    nodes = np.unique(np.concatenate([rs.fixed_resolution_grid(15.0, 10005.0, 2000.0), pn[0], pn[-1]]))
    out = torch.empty((2, nodes.size), dtype=torch.float64, device="cuda")
    rox.rox_cia_regrid_nodes(Tb, off, nu, k, torch.from_numpy(nodes).cuda(), [250.0, 600.0], out)
    ref = oracle.cia_regrid(Tb, pn, pk, [250.0, 600.0], nodes)
    got = out.cpu().numpy()
    print("CIA nodes: max relative difference %.2e" % _same(got, ref, nodes))
    for b in (0, len(Tb) - 1):          # every block sample is reproduced exactly
        row = 0 if Tb[b] == 250.0 else 1
        idx = np.searchsorted(nodes, pn[b])
        first = [oracle.cia_regrid(Tb, pn, pk, [Tb[b]], pn[b][q:q + 1])[0, 0] for q in range(0, pn[b].size, 97)]
        assert np.array_equal(got[row, idx[::97]], np.array(first))


def test_cia_overlapping_blocks_and_single_sample():
    # hand-made blocks at one temperature: an overlap (first wins) and a one-sample block
    x1 = np.array([100.0, 200.0, 300.0]); y1 = np.array([1.0, 2.0, 4.0])
    x2 = np.array([250.0, 400.0]); y2 = np.array([10.0, 20.0])
    x3 = np.array([500.0]); y3 = np.array([7.0])
    nu = torch.from_numpy(np.concatenate([x1, x2, x3])).cuda()
    k = torch.from_numpy(np.concatenate([y1, y2, y3])).cuda()
    Tb, off = [300.0, 300.0, 300.0], [0, 3, 5, 6]
    grid = (0.0, 12.5, 49)
    out = torch.empty((1, 49), dtype=torch.float64, device="cuda")
    _regrid(Tb, off, nu, k, grid, [300.0], out)
    pts = oracle.grid_nodes(*grid)
    ref = oracle.cia_regrid(Tb, [x1, x2, x3], [y1, y2, y3], [300.0], pts)
    got = out.cpu().numpy()
    _same(got, ref, pts)
    # 200: a sample; 250: inside the first block (its value wins over the second's); 300: the
    # first block's last sample; 350: the second block only; 500: the one-sample block
    assert got[0, 16] == 2.0 and got[0, 20] == 3.0 and got[0, 24] == 4.0
    assert abs(got[0, 28] - (10.0 + 10.0 * (100.0 / 150.0))) < 1e-12 and got[0, 40] == 7.0
    assert got[0, 0] == 0.0 and got[0, 36] == 0.0


def test_cia_rejects_bad_input():
    nu = torch.zeros(4, dtype=torch.float64, device="cuda")
    k = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.empty((1, 10), dtype=torch.float64, device="cuda")
    for Tb, off in (([], [0]), ([300.0], [0, 0]), ([300.0], [1, 4])):
        with pytest.raises(rox.RoxError):
            _regrid(Tb, off, nu, k, (0.0, 1.0, 10), [300.0], out)
    with pytest.raises(rox.RoxError):   # workspace one element short
        _regrid([300.0], [0, 4], nu, k, (0.0, 1.0, 10), [300.0], out,
                ws_bytes=rox.rox_cia_workspace_size(1, 4) - 8)


def test_cia_nodes_out_of_order():
    """Shuffled nodes give the shuffled row (the kernel searches again when a node goes backwards)."""
    Tb, off, nu, k, pn, pk = _blocks(9, [500.0], 600)
    nodes = rs.irregular_nodes(27, 0.0, 10100.0, 5000)
    perm = np.random.default_rng(3).permutation(nodes.size)
    out = torch.empty((1, nodes.size), dtype=torch.float64, device="cuda")
    rox.rox_cia_regrid_nodes(Tb, off, nu, k, torch.from_numpy(nodes[perm]).cuda(), [500.0], out)
    ref = oracle.cia_regrid(Tb, pn, pk, [500.0], nodes)
    got = np.empty_like(ref)
    got[:, perm] = out.cpu().numpy()
    _same(got, ref, nodes)


def test_cia_grid_runs_and_edges():
    """Uniform grids whose coverage edges, samples and tile ends fall in every position of a
    lane's run: tiny and ragged grids, a grid point on every sample of a block (dnu dividing
    the sample spacing), samples closer than dnu (intervals holding no point) and one row per
    temperature of several blocks each."""
    x = np.arange(50.0, 250.0, 2.5)              # every sample on a grid point of dnu = 0.5
    y = 1.0 + 0.01 * (x - 150.0) ** 2
    xd = np.sort(np.concatenate([np.linspace(300.0, 310.0, 400), [305.0001, 305.0002]]))
    yd = np.cos(xd)
    blocks = [(500.0, x, y), (500.0, xd, yd), (900.0, x[::3], y[::3] * 2.0), (900.0, xd, yd + 3.0)]
    Tb = [b[0] for b in blocks]
    nu = torch.from_numpy(np.concatenate([b[1] for b in blocks])).cuda()
    k = torch.from_numpy(np.concatenate([b[2] for b in blocks])).cuda()
    off = np.cumsum([0] + [b[1].size for b in blocks])
    for grid in ((40.0, 0.5, 1), (40.0, 0.5, 63), (40.0, 0.5, 2049), (0.0, 0.5, 1000), (49.75, 0.5, 4500),
                 (120.0, 0.013, 70001)):
        out = torch.empty((2, grid[2]), dtype=torch.float64, device="cuda")
        _regrid(Tb, off, nu, k, grid, [900.0, 500.0], out)
        pts = oracle.grid_nodes(*grid)
        ref = oracle.cia_regrid(Tb, [b[1] for b in blocks], [b[2] for b in blocks], [900.0, 500.0], pts)
        got = out.cpu().numpy()
        _same(got, ref, pts)
        on = np.isin(pts, x)                      # grid points on samples of the 500 K block: exact
        assert np.array_equal(got[1, on], ref[1, on])


def test_cia_unsorted_samples_stay_in_bounds():
    """Samples out of order break the documented precondition (the result is then unspecified),
    but every index the kernels form stays inside its block: both paths run and write finite
    values."""
    rng = np.random.default_rng(4)
    x = rng.uniform(100.0, 900.0, 500)                    # not sorted
    y = rng.uniform(1.0, 2.0, 500)
    nu, k = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    out = torch.empty((1, 20001), dtype=torch.float64, device="cuda")
    _regrid([300.0], [0, 500], nu, k, (0.0, 0.05, 20001), [300.0], out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    nodes = torch.from_numpy(np.linspace(0.0, 1000.0, 20001)).cuda()
    rox.rox_cia_regrid_nodes([300.0], [0, 500], nu, k, nodes, [300.0], out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
