"""The C-ABI library loads without a GPU, exports every entry point declared in
include/rox.h, and rejects invalid arguments on the host before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "rox.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rox_[a-z0-9_]+)\s*\(", src)))


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
    for args in [(0.0, 1000.0, 1.0), (1.0, -5.0, 1.0), (1.0, 1000.0, 0.0), (-1.0, 1000.0, 1.0)]:
        rc = L.rox_xsec(ctypes.byref(lines), ctypes.byref(G), args[0] if args[0] >= 0 else -1.0, args[1], args[2],
                        1.0, 18.0, 25.0, 8, 256, 1 << 30, None)
        if args == (0.0, 1000.0, 1.0):
            continue  # P = 0 is valid (pure Doppler); reaching the launch needs a GPU
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


def test_workspace_size_is_host_only(lib):
    G = lib.RoxGrid(300.0, 0.01, 2970001)
    a = lib.lib.rox_xsec_workspace_size(10_000_000, ctypes.byref(G), 1)
    b = lib.lib.rox_xsec_workspace_size(10_000_000, ctypes.byref(G), 20)
    assert a > 10_000_000 * (16 + 12) and b - a == 19 * 10_000_000 * 12   # FP64 + scaled FP32 strengths
    assert lib.lib.rox_xsec_workspace_size(10, ctypes.byref(G), 0) == 0


def test_partition_function_host_helper():
    from paper_2510_20870_gb300.partition import PartitionFunction
    q = PartitionFunction(("table", [50.0, 51.0, 52.0], [1.0, 3.0, 7.0]))
    assert q(50.0) == 1.0 and q(51.5) == 5.0 and q(52.0) == 7.0
    with pytest.raises(ValueError):
        q(49.0)
    assert PartitionFunction(("analytic", 0.05))(400.0) == pytest.approx(0.05 * 8000.0)


def test_static_scratch_holds_the_largest_static_problem():
    """rox_xsec_static runs rox_xsec in a fixed 16 MiB array: the workspace of its largest
    accepted problem (ROX_STATIC_MAX_LINES lines, ROX_STATIC_MAX_GRID points, one T) fits."""
    from paper_2510_20870_gb300 import _binding as b
    need = b.rox_xsec_workspace_size(262144, (0.0, 0.01, 1 << 21), 1)
    assert 0 < need <= 16 << 20, need


def test_cia_arguments_rejected_on_host(lib):
    """CIA restructuring: every malformed layout is refused before anything reaches the GPU
    (the device pointers here are placeholders that are never dereferenced)."""
    L = lib.lib
    assert L.rox_cia_workspace_size(2, 10) == 8 * (3 * 10 + 2)

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
