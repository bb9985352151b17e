"""GPU CIA restructuring against the FP64 oracle through the C ABI: float64 linear
interpolation (the kernel multiplies by each interval's reciprocal width where the oracle
divides), so rows agree to a few ulps, exactly at samples, and zero where no block covers."""
import numpy as np
import pytest

import oracle
import rox_synth as rs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402


def _same(got, ref):
    """Equal to 1e-14 relative, and exactly where the oracle gives 0 or a block sample."""
    assert got.shape == ref.shape
    assert np.array_equal(got == 0.0, ref == 0.0)
    nz = ref != 0.0
    rel = np.abs(got[nz] - ref[nz]) / np.abs(ref[nz])
    assert rel.max() < 1e-14, rel.max()
    return rel.max()


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
    rox.rox_cia_regrid(Tb, off, nu, k, grid, T_out, out)
    ref = oracle.cia_regrid(Tb, pn, pk, T_out, oracle.grid_nodes(*grid))
    got = out.cpu().numpy()
    _same(got, ref)
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
    _same(got, ref)
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
    rox.rox_cia_regrid(Tb, off, nu, k, grid, [300.0], out)
    ref = oracle.cia_regrid(Tb, [x1, x2, x3], [y1, y2, y3], [300.0], oracle.grid_nodes(*grid))
    got = out.cpu().numpy()
    _same(got, ref)
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
            rox.rox_cia_regrid(Tb, off, nu, k, (0.0, 1.0, 10), [300.0], out)


def test_cia_nodes_out_of_order():
    """Shuffled nodes give the shuffled row (the kernel searches again when a node goes backwards)."""
    Tb, off, nu, k, pn, pk = _blocks(9, [500.0], 600)
    nodes = rs.irregular_nodes(27, 0.0, 10100.0, 5000)
    perm = np.random.default_rng(3).permutation(nodes.size)
    out = torch.empty((1, nodes.size), dtype=torch.float64, device="cuda")
    rox.rox_cia_regrid_nodes(Tb, off, nu, k, torch.from_numpy(nodes[perm]).cuda(), [500.0], out)
    ref = oracle.cia_regrid(Tb, pn, pk, [500.0], nodes)
    _same(out.cpu().numpy(), ref[:, perm])
