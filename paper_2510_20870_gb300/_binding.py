"""ctypes binding of librox (include/rox.h): argument marshalling only.

Every function here takes torch CUDA tensors (device memory) and host scalars, builds
the C structs and calls the C entry point of the same name. Nothing is computed here:
each step of the cross-section path runs in the library's CUDA kernels. A non-zero
status raises RoxError with the library's message.
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librox.so")

ROX_OK, ROX_EINVAL, ROX_ENOMEM, ROX_ECUDA, ROX_ETIMEOUT, ROX_EUNSORTED, ROX_ERANGE, ROX_EGRID, ROX_EOVERFLOW = range(9)
ROX_HITRAN, ROX_EXOMOL = 0, 1
ROX_WIDTH_F32, ROX_WIDTH_F16 = 0, 1
ROX_ACCUMULATE = 1
ROX_KAHAN = 2
ROX_MAX_PT = 512
ROX_TILE = 256  # grid points per Voigt work item (one warp: 32 lanes x ROX_K points)


class RoxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("librox error %d: %s" % (code, msg))
        self.code = code


class RoxLines(ctypes.Structure):
    _fields_ = [("nu0", ctypes.c_void_p), ("s_or_a", ctypes.c_void_p), ("g_up", ctypes.c_void_p),
                ("e_lower", ctypes.c_void_p), ("gamma_ref", ctypes.c_void_p), ("n_t", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("convention", ctypes.c_int32), ("width_dtype", ctypes.c_int32)]


class RoxLinesBuf(ctypes.Structure):
    _fields_ = [("nu0", ctypes.c_void_p), ("s_or_a", ctypes.c_void_p), ("g_up", ctypes.c_void_p),
                ("e_lower", ctypes.c_void_p), ("gamma_ref", ctypes.c_void_p), ("n_t", ctypes.c_void_p)]


class RoxGrid(ctypes.Structure):
    _fields_ = [("nu_min", ctypes.c_double), ("dnu", ctypes.c_double), ("n", ctypes.c_int64)]


class RoxNodes(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_void_p), ("n", ctypes.c_int64)]


class RoxSelect(ctypes.Structure):
    _fields_ = [("rel", ctypes.c_double), ("bin_width", ctypes.c_double)]


ROX_MAX_BROADENERS = 4


class RoxBroadening(ctypes.Structure):
    _fields_ = [("n_broadeners", ctypes.c_int32), ("natural", ctypes.c_int32),
                ("vmr", ctypes.c_double * ROX_MAX_BROADENERS), ("gamma_ref", ctypes.c_void_p * ROX_MAX_BROADENERS),
                ("n_t", ctypes.c_void_p * ROX_MAX_BROADENERS), ("table_gamma", ctypes.c_void_p * ROX_MAX_BROADENERS),
                ("table_n", ctypes.c_void_p * ROX_MAX_BROADENERS), ("j_lower", ctypes.c_void_p),
                ("table_len", ctypes.c_int64)]


class RoxCia(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("pad", ctypes.c_int32), ("T_block", ctypes.c_void_p),
                ("offset", ctypes.c_void_p), ("nu", ctypes.c_void_p), ("k", ctypes.c_void_p)]


class RoxPrepared(ctypes.Structure):
    _fields_ = [("lines", RoxLines), ("lattice", RoxGrid), ("cutoff", ctypes.c_double), ("state", ctypes.c_void_p),
                ("span_lo", ctypes.c_void_p), ("span_hi", ctypes.c_void_p), ("n_spans", ctypes.c_int64)]


class RoxLaunchConfig(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("split_rounds", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class RoxJob(ctypes.Structure):
    _fields_ = [("list", ctypes.c_int32), ("flags", ctypes.c_uint32), ("first", ctypes.c_int64), ("n", ctypes.c_int64),
                ("line_first", ctypes.c_int64), ("line_count", ctypes.c_int64), ("P_bar", ctypes.c_double),
                ("T", ctypes.c_double), ("Q_T", ctypes.c_double), ("Q_ref", ctypes.c_double),
                ("mass_amu", ctypes.c_double), ("sigma_out", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("librox.so is not built: run `python -c \"import __graft_entry__ as g; g.build()\"` "
                          "(or python -m paper_2510_20870_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I64, I32, D, U = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_uint
    sig = {
        "rox_last_error": (ctypes.c_char_p, []),
        "rox_version": (ctypes.c_char_p, []),
        "rox_line_strengths": (ctypes.c_int, [P, D, D, D, P, P]),
        "rox_line_widths": (ctypes.c_int, [P, D, D, D, P, P, P]),
        "rox_line_strengths_reduced": (ctypes.c_int, [P, D, D, D, P, P]),
        "rox_sort_workspace_size": (ctypes.c_size_t, [I64]),
        "rox_sort_lines": (ctypes.c_int, [P, P, P, P, ctypes.c_size_t, P]),
        "rox_line_windows": (ctypes.c_int, [P, I64, P, D, P, P, P, P, P, P, P]),
        "rox_tile_ranges": (ctypes.c_int, [P, P, I64, I64, I32, P, P, P]),
        "rox_faddeeva_re": (ctypes.c_int, [P, P, P, I64, P]),
        "rox_xsec_workspace_size": (ctypes.c_size_t, [I64, P, ctypes.c_int]),
        "rox_xsec_batch": (ctypes.c_int, [P, P, ctypes.c_int, P, P, P, D, D, D, U, P, P, ctypes.c_size_t, P]),
        "rox_xsec": (ctypes.c_int, [P, P, D, D, D, D, D, D, P, P, ctypes.c_size_t, P]),
        "rox_ws_status": (ctypes.c_int, [P, P, P]),
        "rox_set_profile_events": (ctypes.c_int, [P, P]),
        "rox_xsec_static": (ctypes.c_int, [P, P, D, D, D, D, D, D, P, P, P]),
        "rox_prepare_size": (ctypes.c_size_t, [I64, P]),
        "rox_prepare": (ctypes.c_int, [P, P, D, P, ctypes.c_size_t, P, P]),
        "rox_jobs_workspace_size": (ctypes.c_size_t, [P, ctypes.c_int]),
        "rox_xsec_jobs": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_size_t, P]),
        "rox_xsec_nodes_workspace_size": (ctypes.c_size_t, [I64, I64, ctypes.c_int]),
        "rox_xsec_nodes_batch": (ctypes.c_int, [P, P, ctypes.c_int, P, P, P, D, D, D, U, P, P, ctypes.c_size_t, P]),
        "rox_node_windows": (ctypes.c_int, [P, I64, P, D, P, P, P]),
        "rox_xsec_select_workspace_size": (ctypes.c_size_t, [I64, P, ctypes.c_int, D, P]),
        "rox_xsec_select_batch": (ctypes.c_int, [P, P, ctypes.c_int, P, P, P, D, D, D, U, P, P, P, ctypes.c_size_t,
                                                 P]),
        "rox_line_select": (ctypes.c_int, [P, P, D, D, D, D, P, P, P, ctypes.c_size_t, P]),
        "rox_lorentz_widths": (ctypes.c_int, [P, P, D, D, P, P]),
        "rox_cia_workspace_size": (ctypes.c_size_t, [ctypes.c_int32, ctypes.c_int64]),
        "rox_cia_regrid": (ctypes.c_int, [P, P, ctypes.c_int, P, P, P, ctypes.c_size_t, P]),
        "rox_cia_regrid_nodes": (ctypes.c_int, [P, P, ctypes.c_int, P, P, P]),
        "rox_xsec_broadened_workspace_size": (ctypes.c_size_t, [I64, P, ctypes.c_int]),
        "rox_fp32_probe_out_size": (ctypes.c_size_t, [ctypes.c_int]),
        "rox_set_launch_config": (ctypes.c_int, [P]),
        "rox_get_launch_config": (ctypes.c_int, [P]),
        "rox_fp32_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P, P]),
        "rox_pair_loop_probe": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, P, ctypes.c_size_t, P, P]),
        "rox_xsec_broadened_batch": (ctypes.c_int, [P, P, P, ctypes.c_int, P, P, P, D, D, D, U, P, P,
                                                    ctypes.c_size_t, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def version():
    return lib.rox_version().decode()


def _check(rc):
    if rc != ROX_OK:
        raise RoxError(rc, lib.rox_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda):
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def lines_struct(lines):
    """rox_lines from a dict of CUDA tensors: nu0 float64, s_or_a/e_lower (g_up) float32,
    gamma_ref/n_t float32 or float16; 'convention' 0 (HITRAN) or 1 (ExoMol)."""
    gref = lines["gamma_ref"]
    wd = ROX_WIDTH_F16 if gref.dtype == torch.float16 else ROX_WIDTH_F32
    L = RoxLines(nu0=_ptr(lines["nu0"]).value, s_or_a=_ptr(lines["s_or_a"]).value,
                 g_up=(_ptr(lines["g_up"]).value if lines.get("g_up") is not None else None),
                 e_lower=_ptr(lines["e_lower"]).value, gamma_ref=_ptr(gref).value,
                 n_t=_ptr(lines["n_t"]).value, n=lines["nu0"].numel(),
                 convention=int(lines["convention"]), width_dtype=wd)
    return L


def grid_struct(grid):
    nu_min, dnu, n = grid
    return RoxGrid(float(nu_min), float(dnu), int(n))


def rox_line_strengths(lines, T, Q_T, Q_ref, S_out, stream=None):
    L = lines_struct(lines)
    _check(lib.rox_line_strengths(ctypes.byref(L), T, Q_T, Q_ref, _ptr(S_out), _stream(stream)))


def rox_line_strengths_reduced(lines, T, Q_T, Q_ref, S_out, stream=None):
    """S(T) as the cross-section launches compute it (reduced form), float64 CUDA tensor S_out."""
    L = lines_struct(lines)
    _check(lib.rox_line_strengths_reduced(ctypes.byref(L), T, Q_T, Q_ref, _ptr(S_out), _stream(stream)))


def rox_line_widths(lines, mass_amu, P_bar, T, gamma_G_out, gamma_L_out, stream=None):
    L = lines_struct(lines)
    _check(lib.rox_line_widths(ctypes.byref(L), mass_amu, P_bar, T, _ptr(gamma_G_out), _ptr(gamma_L_out),
                               _stream(stream)))


def rox_sort_workspace_size(n):
    return lib.rox_sort_workspace_size(n)


def rox_sort_lines(lines, out, perm_out, ws, stream=None):
    L = lines_struct(lines)
    B = RoxLinesBuf(nu0=_ptr(out["nu0"]).value, s_or_a=_ptr(out["s_or_a"]).value,
                    g_up=(_ptr(out["g_up"]).value if out.get("g_up") is not None else None),
                    e_lower=_ptr(out["e_lower"]).value, gamma_ref=_ptr(out["gamma_ref"]).value,
                    n_t=_ptr(out["n_t"]).value)
    _check(lib.rox_sort_lines(ctypes.byref(L), ctypes.byref(B), _ptr(perm_out), _ptr(ws), ws.numel(),
                              _stream(stream)))


def rox_line_windows(nu0, grid, cutoff, jlo=None, jhi=None, k0=None, f=None, evals=None, unsorted=None,
                     stream=None):
    G = grid_struct(grid)
    _check(lib.rox_line_windows(_ptr(nu0), nu0.numel(), ctypes.byref(G), cutoff, _ptr(jlo), _ptr(jhi), _ptr(k0),
                                _ptr(f), _ptr(evals), _ptr(unsorted), _stream(stream)))


def rox_tile_ranges(jlo, jhi, n_grid, tile_pts, lo_out, hi_out, stream=None):
    _check(lib.rox_tile_ranges(_ptr(jlo), _ptr(jhi), jlo.numel(), n_grid, tile_pts, _ptr(lo_out), _ptr(hi_out),
                               _stream(stream)))


def rox_faddeeva_re(x, y, out, stream=None):
    _check(lib.rox_faddeeva_re(_ptr(x), _ptr(y), _ptr(out), x.numel(), _stream(stream)))


def rox_xsec_workspace_size(n_lines, grid, n_temps):
    G = grid_struct(grid)
    return lib.rox_xsec_workspace_size(n_lines, ctypes.byref(G), n_temps)


def rox_xsec_batch(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, ws, flags=0, stream=None):
    n_pt = len(P_bar)
    arr = ctypes.c_double * n_pt
    L = lines_struct(lines)
    G = grid_struct(grid)
    _check(lib.rox_xsec_batch(ctypes.byref(L), ctypes.byref(G), n_pt, arr(*P_bar), arr(*T), arr(*Q_T), Q_ref,
                              mass_amu, cutoff, flags, _ptr(sigma_out), _ptr(ws), ws.numel(), _stream(stream)))


def nodes_struct(nodes):
    """rox_nodes from a CUDA float64 tensor of strictly increasing nodes (cm^-1)."""
    if nodes.dtype != torch.float64:
        raise TypeError("nodes must be float64")
    return RoxNodes(_ptr(nodes).value, nodes.numel())


def rox_xsec_nodes_workspace_size(n_lines, n_nodes, n_temps):
    return lib.rox_xsec_nodes_workspace_size(n_lines, n_nodes, n_temps)


def rox_xsec_nodes_batch(lines, nodes, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, ws, flags=0, stream=None):
    """Cross-sections on user-provided nodes (float64 CUDA tensor); sigma_out [n_pt][n_nodes]."""
    n_pt = len(P_bar)
    arr = ctypes.c_double * n_pt
    L = lines_struct(lines)
    N = nodes_struct(nodes)
    _check(lib.rox_xsec_nodes_batch(ctypes.byref(L), ctypes.byref(N), n_pt, arr(*P_bar), arr(*T), arr(*Q_T), Q_ref,
                                    mass_amu, cutoff, flags, _ptr(sigma_out), _ptr(ws), ws.numel(), _stream(stream)))


def rox_node_windows(nu0, nodes, cutoff, jlo, jhi, stream=None):
    N = nodes_struct(nodes)
    _check(lib.rox_node_windows(_ptr(nu0), nu0.numel(), ctypes.byref(N), cutoff, _ptr(jlo), _ptr(jhi),
                                _stream(stream)))


def rox_xsec_select_workspace_size(n_lines, grid, n_temps, cutoff, rel, bin_width):
    G = grid_struct(grid)
    S = RoxSelect(float(rel), float(bin_width))
    return lib.rox_xsec_select_workspace_size(n_lines, ctypes.byref(G), n_temps, cutoff, ctypes.byref(S))


def rox_xsec_select_batch(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, rel, bin_width, sigma_out, ws, flags=0,
                          stream=None):
    """rox_xsec_batch keeping only the main line-strength contributors (rel, bin_width)."""
    n_pt = len(P_bar)
    arr = ctypes.c_double * n_pt
    L = lines_struct(lines)
    G = grid_struct(grid)
    S = RoxSelect(float(rel), float(bin_width))
    _check(lib.rox_xsec_select_batch(ctypes.byref(L), ctypes.byref(G), n_pt, arr(*P_bar), arr(*T), arr(*Q_T), Q_ref,
                                     mass_amu, cutoff, flags, ctypes.byref(S), _ptr(sigma_out), _ptr(ws), ws.numel(),
                                     _stream(stream)))


def rox_line_select(lines, grid, cutoff, T, Q_T, Q_ref, rel, bin_width, keep_out, ws, stream=None):
    L = lines_struct(lines)
    G = grid_struct(grid)
    S = RoxSelect(float(rel), float(bin_width))
    _check(lib.rox_line_select(ctypes.byref(L), ctypes.byref(G), cutoff, T, Q_T, Q_ref, ctypes.byref(S),
                               _ptr(keep_out), _ptr(ws), ws.numel(), _stream(stream)))


def broadening_struct(br):
    """rox_broadening from a dict: vmr (list), and per broadener either gamma_ref / n_t (lists of
    CUDA tensors, dtype of the list's widths) or table_gamma / table_n (lists of float32 CUDA tensors)
    with j_lower (int32 CUDA tensor); natural (bool)."""
    vmr = list(br["vmr"])
    nb = len(vmr)
    B = RoxBroadening()
    B.n_broadeners = nb
    B.natural = 1 if br.get("natural") else 0
    tabs = list(br.get("table_gamma") or [None] * nb) + [None] * nb
    tabn = list(br.get("table_n") or [None] * nb) + [None] * nb
    gref = list(br.get("gamma_ref") or [None] * nb) + [None] * nb
    nts = list(br.get("n_t") or [None] * nb) + [None] * nb
    for k in range(min(nb, ROX_MAX_BROADENERS)):     # the library rejects more than ROX_MAX_BROADENERS
        B.vmr[k] = float(vmr[k])
        B.gamma_ref[k] = _ptr(gref[k]).value if gref[k] is not None else None
        B.n_t[k] = _ptr(nts[k]).value if nts[k] is not None else None
        B.table_gamma[k] = _ptr(tabs[k]).value if tabs[k] is not None else None
        B.table_n[k] = _ptr(tabn[k]).value if tabn[k] is not None else None
    tl = [t.numel() for t in tabs if t is not None]
    B.table_len = tl[0] if tl else 0
    B.j_lower = _ptr(br["j_lower"]).value if br.get("j_lower") is not None else None
    return B


def rox_lorentz_widths(lines, br, P_bar, T, gamma_L_out, stream=None):
    L = lines_struct(lines)
    B = broadening_struct(br)
    _check(lib.rox_lorentz_widths(ctypes.byref(L), ctypes.byref(B), P_bar, T, _ptr(gamma_L_out), _stream(stream)))


def rox_xsec_broadened_workspace_size(n_lines, grid, n_temps):
    G = grid_struct(grid)
    return lib.rox_xsec_broadened_workspace_size(n_lines, ctypes.byref(G), n_temps)


def rox_xsec_broadened_batch(lines, grid, br, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, ws, flags=0,
                             stream=None):
    """rox_xsec_batch with the Lorentz widths of the broadening description `br` (see broadening_struct)."""
    n_pt = len(P_bar)
    arr = ctypes.c_double * n_pt
    L = lines_struct(lines)
    G = grid_struct(grid)
    B = broadening_struct(br)
    _check(lib.rox_xsec_broadened_batch(ctypes.byref(L), ctypes.byref(G), ctypes.byref(B), n_pt, arr(*P_bar), arr(*T),
                                        arr(*Q_T), Q_ref, mass_amu, cutoff, flags, _ptr(sigma_out), _ptr(ws),
                                        ws.numel(), _stream(stream)))


def _cia_call(fn, grid_arg, T_block, offset, nu, k, T_out, out, stream, ws=None):
    nb = len(T_block)
    tb = (ctypes.c_double * nb)(*[float(x) for x in T_block])
    off = (ctypes.c_int64 * (nb + 1))(*[int(x) for x in offset])
    to = (ctypes.c_double * len(T_out))(*[float(x) for x in T_out])
    C = RoxCia(nb, 0, ctypes.cast(tb, ctypes.c_void_p), ctypes.cast(off, ctypes.c_void_p), _ptr(nu).value, _ptr(k).value)
    if ws is None:
        _check(fn(ctypes.byref(C), ctypes.byref(grid_arg), len(T_out), to, _ptr(out), _stream(stream)))
    else:
        _check(fn(ctypes.byref(C), ctypes.byref(grid_arg), len(T_out), to, _ptr(out), _ptr(ws), ws.numel(),
                  _stream(stream)))


def rox_cia_workspace_size(n_blocks, n_samples):
    return int(lib.rox_cia_workspace_size(int(n_blocks), int(n_samples)))


def rox_cia_regrid(T_block, offset, nu, k, grid, T_out, out, ws, stream=None):
    """CIA blocks (temperatures and offsets on the host; nu, k float64 CUDA tensors, blocks
    concatenated) onto the uniform grid: out [len(T_out)][n] float64; ws: uint8 CUDA tensor of
    rox_cia_workspace_size(len(T_block), offset[-1]) bytes."""
    _cia_call(lib.rox_cia_regrid, grid_struct(grid), T_block, offset, nu, k, T_out, out, stream, ws=ws)


def rox_cia_regrid_nodes(T_block, offset, nu, k, nodes, T_out, out, stream=None):
    _cia_call(lib.rox_cia_regrid_nodes, nodes_struct(nodes), T_block, offset, nu, k, T_out, out, stream)


def rox_xsec(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, ws, stream=None):
    L = lines_struct(lines)
    G = grid_struct(grid)
    _check(lib.rox_xsec(ctypes.byref(L), ctypes.byref(G), P_bar, T, Q_T, Q_ref, mass_amu, cutoff, _ptr(sigma_out),
                        _ptr(ws), ws.numel(), _stream(stream)))


def rox_set_profile_events(start=None, stop=None):
    """start/stop: torch.cuda.Event (enable_timing=True, already recorded once so that the
    CUDA event exists) or None to disable."""
    h = (lambda e: None if e is None else ctypes.c_void_p(e.cuda_event))
    _check(lib.rox_set_profile_events(h(start), h(stop)))


def rox_xsec_static(lines, grid, P_bar, T, Q_T, Q_ref, mass_amu, cutoff, sigma_out, status_out=None, stream=None):
    """rox_xsec without a workspace (scratch held by the library; see include/rox.h)."""
    L = lines_struct(lines)
    G = grid_struct(grid)
    _check(lib.rox_xsec_static(ctypes.byref(L), ctypes.byref(G), P_bar, T, Q_T, Q_ref, mass_amu, cutoff,
                               _ptr(sigma_out), _ptr(status_out), _stream(stream)))


ROX_SPAN = 256


class Prepared:
    """A sorted line list prepared on a lattice for rox_xsec_jobs (keeps its buffers alive).
    span_lo / span_hi: host copies of the per-span line ranges (numpy int64)."""

    def __init__(self, lines, lattice, cutoff, stream=None):
        import numpy as np
        self.lines = lines
        self.lattice = tuple(lattice)
        self.cutoff = float(cutoff)
        n = lines["nu0"].numel()
        G = grid_struct(lattice)
        self.state = torch.empty(lib.rox_prepare_size(n, ctypes.byref(G)), dtype=torch.uint8,
                                 device=lines["nu0"].device)
        self.struct = RoxPrepared()
        L = lines_struct(lines)
        _check(lib.rox_prepare(ctypes.byref(L), ctypes.byref(G), self.cutoff, _ptr(self.state), self.state.numel(),
                               ctypes.byref(self.struct), _stream(stream)))
        ns = self.struct.n_spans
        lo = torch.empty(ns, dtype=torch.int64, device=self.state.device)
        hi = torch.empty(ns, dtype=torch.int64, device=self.state.device)
        dev = self.state.device
        # copy the device span tables (views of the state buffer) to host once
        off_lo = self.struct.span_lo - self.state.data_ptr()
        off_hi = self.struct.span_hi - self.state.data_ptr()
        lo.copy_(self.state[off_lo:off_lo + 8 * ns].view(torch.int64))
        hi.copy_(self.state[off_hi:off_hi + 8 * ns].view(torch.int64))
        self.span_lo = lo.cpu().numpy()
        self.span_hi = hi.cpu().numpy()
        self.n_lines = n

    def line_range(self, first, n):
        s0, s1 = first // ROX_SPAN, (first + n - 1) // ROX_SPAN
        l0 = int(self.span_lo[s0])
        return l0, max(0, int(self.span_hi[s1]) - l0)

    def status(self, stream=None):
        return rox_ws_status(self.state, stream)


def make_job(prepared, list_index, first, n, P_bar, T, Q_T, Q_ref, mass_amu, sigma_out, flags=0):
    l0, cnt = prepared.line_range(first, n)
    return RoxJob(list=list_index, flags=flags, first=first, n=n, line_first=l0, line_count=cnt, P_bar=P_bar, T=T,
                  Q_T=Q_T, Q_ref=Q_ref, mass_amu=mass_amu, sigma_out=_ptr(sigma_out).value)


def rox_jobs_workspace_size(jobs):
    arr = (RoxJob * len(jobs))(*jobs)
    return lib.rox_jobs_workspace_size(arr, len(jobs))


def rox_xsec_jobs(prepared_lists, jobs, ws, stream=None):
    lists = (RoxPrepared * len(prepared_lists))(*[p.struct for p in prepared_lists])
    arr = (RoxJob * len(jobs))(*jobs)
    _check(lib.rox_xsec_jobs(lists, len(prepared_lists), arr, len(jobs), _ptr(ws), ws.numel(), _stream(stream)))


def rox_fp32_probe(n_blocks, reps, out, stream=None):
    """Launch the FP32 FMA-rate probe (include/rox.h); returns the number of FMAs it performs."""
    fma = ctypes.c_double(0.0)
    _check(lib.rox_fp32_probe(int(n_blocks), int(reps), _ptr(out), out.numel() * out.element_size(),
                              ctypes.byref(fma), _stream(stream)))
    return fma.value


def rox_fp32_probe_out_size(n_blocks):
    return int(lib.rox_fp32_probe_out_size(int(n_blocks)))


def rox_pair_loop_probe(n_blocks, reps, out, stream=None):
    """Launch the Voigt pair-loop probe (include/rox.h); returns the (line, point) evaluations it performs."""
    ev = ctypes.c_double(0.0)
    _check(lib.rox_pair_loop_probe(int(n_blocks), int(reps), _ptr(out), out.numel() * out.element_size(),
                                   ctypes.byref(ev), _stream(stream)))
    return ev.value


def rox_set_launch_config(warps_per_cta=8, ctas_per_sm=0, split_rounds=1):
    """Launch configuration of the Voigt kernel (include/rox.h); changes no result."""
    c = RoxLaunchConfig(int(warps_per_cta), int(ctas_per_sm), int(split_rounds), 0)
    _check(lib.rox_set_launch_config(ctypes.byref(c)))


def rox_reset_launch_config():
    _check(lib.rox_set_launch_config(None))


def rox_get_launch_config():
    c = RoxLaunchConfig()
    _check(lib.rox_get_launch_config(ctypes.byref(c)))
    return {"warps_per_cta": c.warps_per_cta, "ctas_per_sm": c.ctas_per_sm, "split_rounds": c.split_rounds}


def rox_ws_status(ws, stream=None):
    """Synchronises the stream; returns (status code, evals) and does not raise."""
    ev = ctypes.c_ulonglong(0)
    rc = lib.rox_ws_status(_ptr(ws), ctypes.byref(ev), _stream(stream))
    return rc, ev.value
