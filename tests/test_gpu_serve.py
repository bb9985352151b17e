"""The continuous-batching server: four resident line lists (1e5 to 1e8 lines), a Poisson
request stream, batches launched while others are still running; every result equals the
same request served alone (bit for bit) and the oracle on sampled windows."""
import numpy as np
import pytest

import oracle
import rox_synth as rs
from rox_testutil import check_sigma, q_pair

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402
from paper_2510_20870_gb300 import serve  # noqa: E402
from rox_synth.device import make_lines_device  # noqa: E402

LATTICE = (300.0, 0.01, 2970001)


def _sorted_device(w):
    raw = make_lines_device(w, 0, w.n_lines)
    out = {k: (torch.empty_like(v) if isinstance(v, torch.Tensor) else v) for k, v in raw.items()}
    ws = torch.empty(rox.rox_sort_workspace_size(w.n_lines), dtype=torch.uint8, device="cuda")
    rox.rox_sort_lines(raw, out, None, ws)
    return out


@pytest.fixture(scope="module")
def server():
    lists = [_sorted_device(w) for w in rs.SERVE_LISTS]
    w0 = rs.SERVE_LISTS[0]
    return serve.Server(lists, LATTICE, w0.cutoff, w0.mass_amu, rs.q_table(w0), max_inflight=3, max_batch=16)


def _lines_near(w, lo, hi):
    """Host-generated, nu0-sorted lines of list w with nu0 in [lo, hi] (scanned chunk by chunk)."""
    found = []
    for start, nu0 in rs.nu0_in_chunks(w):
        found.append(start + np.nonzero((nu0 >= lo) & (nu0 <= hi))[0])
    return oracle.sort_lines(rs.make_lines_at(w, np.concatenate(found)))


def test_results_alone_equal_results_in_the_mix(server):
    reqs = serve.requests_from_stream(rs.serve_requests(400.0, 40, seed=11), LATTICE)
    mixed = server.run(reqs, realtime=True)
    assert len(mixed) == len(reqs)
    assert server.max_inflight_seen >= 2 and server.max_batch_seen >= 2   # batches overlapped, mixes formed
    for r, m in zip(reqs, mixed):
        alone = server.run([r], realtime=False, one_per_launch=True)[0]
        assert np.array_equal(alone.sigma, m.sigma), r.rid
    stats = serve.latency_stats(mixed)
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    # the oracle on 3 of the 40 served requests (7.5%), one per list of 1e6, 1e7 and 1e8 lines,
    # on 64 points in the middle of each window
    w0 = rs.SERVE_LISTS[0]
    Qr = q_pair(w0, 296.0)[1]
    nu_min, dnu, _ = LATTICE
    for lid in (1, 2, 3):
        k = next(i for i, r in enumerate(reqs) if r.list_id == lid)
        r, m = reqs[k], mixed[k]
        s0 = r.first + max(0, r.n // 2 - 32)
        n = min(64, r.n)
        w = rs.SERVE_LISTS[lid]
        L = _lines_near(w, nu_min + dnu * s0 - w.cutoff - 0.05, nu_min + dnu * (s0 + n - 1) + w.cutoff + 0.05)
        Qt = q_pair(w, r.t_k)[0]
        ref = oracle.xsec_window(L, LATTICE, s0, s0 + n, r.p_bar, r.t_k, Qt, Qr, w.mass_amu, w.cutoff)
        check_sigma(m.sigma[s0 - r.first:s0 - r.first + n], ref, M=float(m.sigma.max()),
                    label="served request %d (list %d)" % (r.rid, lid))


def test_served_windows_match_the_oracle(server):
    w = rs.SERVE_LISTS[1]                         # 1e6-line list, regenerated on the host
    L = oracle.sort_lines(rs.make_lines(w))
    reqs = [serve.Request(0, 0.0, 1, 0.02, 700.0, 150_000, 40_000),
            serve.Request(1, 0.0, 1, 50.0, 2900.0, 2_000_000, 5_000),
            serve.Request(2, 0.0, 1, 1e-5, 300.0, 0, 1_001)]
    res = server.run(reqs, realtime=False)
    Qr = q_pair(w, 296.0)[1]
    for r, out in zip(reqs, res):
        Qt = q_pair(w, r.t_k)[0]
        s0 = r.first + r.n // 2 - 48
        ref = oracle.xsec_window(L, LATTICE, s0, s0 + 96, r.p_bar, r.t_k, Qt, Qr, w.mass_amu, w.cutoff)
        got = out.sigma[s0 - r.first:s0 - r.first + 96]
        check_sigma(got, ref, M=float(out.sigma.max()), label="request %d" % r.rid)
