"""The C-ABI library loads without a GPU, exports every entry point declared in
include/rox.h, and rejects invalid arguments on the host before any CUDA call.

The refusal tests pass placeholder device pointers that must never be dereferenced. They run
only where no GPU is visible: there, a call that got past the host checks by mistake fails at
its first CUDA call instead of launching on a bad address."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "rox.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rox_[a-z0-9_]+)\s*\(", src)))


def _gpu_visible():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


host_only = pytest.mark.skipif(_gpu_visible(), reason="placeholder device pointers: runs only without a GPU")


@pytest.fixture(scope="module")
def lib():
    import paper_2510_20870_gb300._binding as b
    return b


def test_every_declared_symbol_is_exported(lib):
    names = _header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib.lib, n), n


def test_version(lib):
    assert "sm_103a" in lib.version()


@host_only
def test_invalid_arguments_rejected_on_host(lib):
    L = lib.lib
    G = lib.RoxGrid(2000.0, 0.01, 50001)
    rc = L.rox_xsec(None, ctypes.byref(G), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, None, None, 0, None)
    assert rc == lib.ROX_EINVAL and b"NULL" in L.rox_last_error()
    lines = lib.RoxLines(nu0=8, s_or_a=8, g_up=None, e_lower=8, gamma_ref=8, n_t=8, n=10, convention=0,
                         width_dtype=0)
    bad_grid = lib.RoxGrid(2000.0, -0.01, 50001)
    rc = L.rox_xsec(ctypes.byref(lines), ctypes.byref(bad_grid), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, 8, 256, 1 << 30,
                    None)
    assert rc == lib.ROX_EINVAL
    big_grid = lib.RoxGrid(2000.0, 0.01, 1 << 24)
    rc = L.rox_xsec(ctypes.byref(lines), ctypes.byref(big_grid), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, 8, 256, 1 << 30,
                    None)
    assert rc == lib.ROX_ERANGE
    for args in [(1.0, -5.0, 1.0), (1.0, 1000.0, 0.0), (-1.0, 1000.0, 1.0)]:   # (P = 0 is valid)
        rc = L.rox_xsec(ctypes.byref(lines), ctypes.byref(G), args[0], args[1], args[2],
                        1.0, 18.0, 25.0, 8, 256, 1 << 30, None)
        assert rc == lib.ROX_EINVAL, args
    # ExoMol without g_up
    ex = lib.RoxLines(nu0=8, s_or_a=8, g_up=None, e_lower=8, gamma_ref=8, n_t=8, n=10, convention=1, width_dtype=0)
    assert L.rox_xsec(ctypes.byref(ex), ctypes.byref(G), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, 8, 256, 1 << 30,
                      None) == lib.ROX_EINVAL
    # workspace too small
    assert L.rox_xsec(ctypes.byref(lines), ctypes.byref(G), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, 8, 256, 16,
                      None) == lib.ROX_ENOMEM
    # cutoff
    assert L.rox_xsec(ctypes.byref(lines), ctypes.byref(G), 1.0, 1000.0, 1.0, 1.0, 18.0, 0.0, 8, 256, 1 << 30,
                      None) == lib.ROX_EINVAL
    # flags: ROX_ACCUMULATE | ROX_KAHAN are the only ones (an unknown bit is refused before any launch)
    one = (ctypes.c_double * 1)
    for bad in (4, 8, 0x100):
        rc = L.rox_xsec_batch(ctypes.byref(lines), ctypes.byref(G), 1, one(1.0), one(1000.0), one(1.0), 1.0, 18.0,
                              25.0, bad, 8, 256, 1 << 30, None)
        assert rc == lib.ROX_EINVAL and b"flags" in L.rox_last_error(), bad


def test_workspace_size_is_host_only(lib):
    G = lib.RoxGrid(300.0, 0.01, 2970001)
    one = lib.lib.rox_xsec_workspace_size(10_000_000, ctypes.byref(G), 1)
    a = lib.lib.rox_xsec_workspace_size(10_000_000, ctypes.byref(G), 2)
    b = lib.lib.rox_xsec_workspace_size(10_000_000, ctypes.byref(G), 20)
    assert a > 10_000_000 * (16 + 2 * 12) and b - a == 18 * 10_000_000 * 12   # FP64 + scaled FP32 strengths
    # one temperature: plus 48 bytes per line of per-line constants, minus one strength row
    assert one - a == 10_000_000 * (48 - 12)
    assert lib.lib.rox_xsec_workspace_size(10, ctypes.byref(G), 0) == 0


def test_partition_function_host_helper():
    from paper_2510_20870_gb300.partition import PartitionFunction
    q = PartitionFunction(("table", [50.0, 51.0, 52.0], [1.0, 3.0, 7.0]))
    assert q(50.0) == 1.0 and q(51.5) == 5.0 and q(52.0) == 7.0
    with pytest.raises(ValueError):
        q(49.0)
    assert PartitionFunction(("analytic", 0.05))(400.0) == pytest.approx(0.05 * 8000.0)


@host_only
def test_static_scratch_holds_the_largest_static_problem(lib):
    """rox_xsec_static runs the cross-section in a fixed 16 MiB array: its largest accepted
    problem (ROX_STATIC_MAX_LINES lines, ROX_STATIC_MAX_GRID points) passes the size checks and
    only then meets the missing GPU (ROX_ECUDA); one line more is refused with ROX_ERANGE. The
    pointers are placeholders that are never dereferenced."""
    from paper_2510_20870_gb300 import _binding as b
    fn = b.lib.rox_xsec_static
    grid = b.grid_struct((0.0, 0.01, 1 << 21))
    for n, want in ((262144, b.ROX_ECUDA), (262145, b.ROX_ERANGE)):
        L = b.RoxLines(ctypes.c_void_p(256), ctypes.c_void_p(512), None, ctypes.c_void_p(768), ctypes.c_void_p(1024),
                       ctypes.c_void_p(1280), n, 0, 0)
        rc = fn(ctypes.byref(L), ctypes.byref(grid), 1.0, 1000.0, 1.0, 1.0, 18.0, 25.0, ctypes.c_void_p(2048), None,
                None)
        assert rc == want, (n, rc, b.lib.rox_last_error())


@host_only
def test_cia_arguments_rejected_on_host(lib):
    """CIA restructuring: every malformed layout is refused before anything reaches the GPU
    (the device pointers here are placeholders that are never dereferenced)."""
    L = lib.lib
    assert L.rox_cia_workspace_size(2, 10) == 8 * (4 * 10 + 2)

    def call(T_block, offset, T_out, grid=(0.0, 1.0, 10), ws=256, ws_bytes=1 << 20, nodes=None):
        tb = (ctypes.c_double * max(1, len(T_block)))(*T_block)
        off = (ctypes.c_int64 * len(offset))(*offset)
        to = (ctypes.c_double * max(1, len(T_out)))(*T_out)
        C = lib.RoxCia(len(T_block), 0, ctypes.cast(tb, ctypes.c_void_p), ctypes.cast(off, ctypes.c_void_p), 8, 8)
        if nodes is not None:
            N = lib.RoxNodes(*nodes)
            return L.rox_cia_regrid_nodes(ctypes.byref(C), ctypes.byref(N), len(T_out), to, 8, None)
        G = lib.RoxGrid(*grid)
        return L.rox_cia_regrid(ctypes.byref(C), ctypes.byref(G), len(T_out), to, 8, ws, ws_bytes, None)

    E = lib.ROX_EINVAL
    assert call([], [0], [300.0]) == E                                   # no block
    assert call([300.0], [1, 4], [300.0]) == E                           # offset[0] != 0
    assert call([300.0, 500.0], [0, 3, 3], [300.0]) == E                 # an empty block
    assert call([300.0], [0, 4], [300.0, 300.0]) == E and b"twice" in L.rox_last_error()
    assert call([300.0], [0, 4], [float("nan")]) == E
    assert call([300.0], [0, 4], []) == E                                # no output row
    assert call([300.0], [0, 4], [float(t) for t in range(1, 4098)]) == E   # more rows than ROX_CIA_MAX_TEMPS
    assert call([300.0], [0, 4], [300.0], grid=(0.0, -1.0, 10)) == E     # dnu <= 0
    assert call([300.0], [0, 4], [300.0], grid=(0.0, 1.0, 0)) == E       # no point
    need = L.rox_cia_workspace_size(1, 4)
    assert call([300.0], [0, 4], [300.0], ws_bytes=need - 8) == E        # workspace one element short
    assert call([300.0], [0, 4], [300.0], ws=260, ws_bytes=need) == E    # workspace not 8-byte aligned
    assert call([300.0], [0, 4], [300.0], ws=None, ws_bytes=need) == E   # no workspace
    assert call([300.0], [0, 4], [300.0], nodes=(None, 10)) == E         # nodes missing


@host_only
def test_extension_arguments_rejected_on_host(lib):
    """Selection, broadening descriptions and user-provided nodes: malformed arguments are
    refused on the host with the documented codes (device pointers are placeholders)."""
    L = lib.lib
    by = ctypes.byref
    G = lib.RoxGrid(2000.0, 0.01, 50001)
    hit = lib.RoxLines(nu0=8, s_or_a=8, g_up=None, e_lower=8, gamma_ref=8, n_t=8, n=10, convention=0, width_dtype=0)
    exo = lib.RoxLines(nu0=8, s_or_a=8, g_up=8, e_lower=8, gamma_ref=8, n_t=8, n=10, convention=1, width_dtype=0)
    P, T, Q = (ctypes.c_double * 1)(1.0), (ctypes.c_double * 1)(1000.0), (ctypes.c_double * 1)(1.0)
    E = lib.ROX_EINVAL

    # main-contributor selection: rel >= 0, bin_width > 0, bins within ROX_MAX_SELECT_BINS
    for rel, bw in ((-1.0, 1.0), (float("nan"), 1.0), (1e-3, 0.0), (1e-3, -2.0), (1e-3, 1e-9)):
        sel = lib.RoxSelect(rel, bw)
        assert L.rox_xsec_select_workspace_size(10, by(G), 1, 25.0, by(sel)) == 0, (rel, bw)
        rc = L.rox_xsec_select_batch(by(hit), by(G), 1, P, T, Q, 1.0, 18.0, 25.0, 0, by(sel), 8, 256, 1 << 30, None)
        assert rc in (E, lib.ROX_ERANGE), (rel, bw, rc)
    assert L.rox_xsec_select_batch(by(hit), by(G), 1, P, T, Q, 1.0, 18.0, 25.0, 0, None, 8, 256, 1 << 30, None) == E

    # broadening descriptions
    def broad(n_b, vmr=(1.0,), cols=True, natural=0, table=False, j_lower=None, table_len=0):
        br = lib.RoxBroadening()
        br.n_broadeners, br.natural, br.table_len = n_b, natural, table_len
        br.j_lower = j_lower
        for b in range(min(n_b, 4)):
            br.vmr[b] = vmr[b] if b < len(vmr) else 0.5
            if table:
                br.table_gamma[b], br.table_n[b] = 8, 8
            elif cols:
                br.gamma_ref[b], br.n_t[b] = 8, 8
        return br

    def xsec(lines, br):
        return L.rox_xsec_broadened_batch(by(lines), by(G), by(br), 1, P, T, Q, 1.0, 18.0, 25.0, 0, 8, 256, 1 << 30,
                                          None)
    assert L.rox_xsec_broadened_batch(by(hit), by(G), None, 1, P, T, Q, 1.0, 18.0, 25.0, 0, 8, 256, 1 << 30,
                                      None) == E
    assert xsec(hit, broad(0)) == E                                  # no broadener
    assert xsec(hit, broad(5)) == E                                  # more than ROX_MAX_BROADENERS
    assert xsec(hit, broad(1, vmr=(-0.5,))) == E                     # negative mixing ratio
    assert xsec(hit, broad(1, cols=False)) == E                      # neither columns nor a table
    assert xsec(hit, broad(1, natural=1)) == E                       # natural width needs Einstein A
    assert xsec(exo, broad(1, table=True, table_len=0, j_lower=8)) == E    # empty J table
    assert xsec(exo, broad(1, table=True, table_len=60, j_lower=None)) == E  # table without J''
    out = (ctypes.c_float * 10)()
    assert L.rox_lorentz_widths(by(hit), by(broad(1, cols=False)), 1.0, 300.0, out, None) == E

    # user-provided nodes
    N = lib.RoxNodes(8, 1000)
    args = (1, P, T, Q, 1.0, 18.0)
    assert L.rox_xsec_nodes_batch(by(hit), by(lib.RoxNodes(None, 1000)), *args, 25.0, 0, 8, 256, 1 << 30, None) == E
    assert L.rox_xsec_nodes_batch(by(hit), by(lib.RoxNodes(8, 0)), *args, 25.0, 0, 8, 256, 1 << 30, None) == E
    assert L.rox_xsec_nodes_batch(by(hit), by(N), *args, 0.0, 0, 8, 256, 1 << 30, None) == E
    assert L.rox_xsec_nodes_batch(by(hit), by(N), *args, 5000.0, 0, 8, 256, 1 << 30, None) == lib.ROX_ERANGE
    assert L.rox_xsec_nodes_batch(by(hit), by(N), *args, 25.0, 0, 8, 256, 16, None) == lib.ROX_ENOMEM


def test_launch_config_validation(lib):
    """rox_set_launch_config refuses out-of-range knobs and changes nothing then; NULL restores
    the defaults (host-only calls)."""
    import paper_2510_20870_gb300 as rox
    rox.rox_set_launch_config(4, 2, 3)
    assert rox.rox_get_launch_config() == {"warps_per_cta": 4, "ctas_per_sm": 2, "split_rounds": 3}
    for bad in [(6, 0, 1), (8, -1, 1), (8, 0, 0), (8, 0, 5)]:
        with pytest.raises(rox.RoxError):
            rox.rox_set_launch_config(*bad)
        assert rox.rox_get_launch_config()["warps_per_cta"] == 4
    rox.rox_reset_launch_config()
    assert rox.rox_get_launch_config() == {"warps_per_cta": 8, "ctas_per_sm": 0, "split_rounds": 1}
