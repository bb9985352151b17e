"""Device-side generation of the synthetic line lists (same values as make_lines, on the GPU).

Used for the line lists too large to generate on the host in reasonable time (1e8 and 1e9
lines). The CUDA source is rox_synth/csrc/synth_gen.cu, built in-tree by build()."""
import ctypes
import math
import os

from .workloads import EXOMOL, Workload

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librox_synth.so")


class _Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint32), ("exomol", ctypes.c_int32), ("nu_lo", ctypes.c_double),
                ("nu_span", ctypes.c_double), ("log_s_lo", ctypes.c_double), ("log_s_span", ctypes.c_double),
                ("el_mean", ctypes.c_double), ("gref_lo", ctypes.c_double), ("gref_span", ctypes.c_double),
                ("nt_lo", ctypes.c_double), ("nt_span", ctypes.c_double), ("gup_max", ctypes.c_int32),
                ("width_f16", ctypes.c_int32)]


def build(nvcc="/usr/local/cuda/bin/nvcc"):
    import subprocess
    src = os.path.join(_HERE, "csrc", "synth_gen.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC", "-shared",
                    "-o", LIB_PATH, src], check=True, capture_output=True)
    return LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librox_synth.so is not built (run __graft_entry__.build())")
        _lib = ctypes.CDLL(LIB_PATH)
        _lib.rox_synth_lines.restype = ctypes.c_int
        _lib.rox_synth_lines.argtypes = [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong] + [ctypes.c_void_p] * 7
    return _lib


def alloc_lines(w: Workload, count, device="cuda"):
    import torch
    wd = torch.float16 if w.width_dtype == "f16" else torch.float32
    out = {"nu0": torch.empty(count, dtype=torch.float64, device=device),
           "s_or_a": torch.empty(count, dtype=torch.float32, device=device),
           "e_lower": torch.empty(count, dtype=torch.float32, device=device),
           "gamma_ref": torch.empty(count, dtype=wd, device=device),
           "n_t": torch.empty(count, dtype=wd, device=device),
           "g_up": torch.empty(count, dtype=torch.float32, device=device) if w.convention == EXOMOL else None,
           "convention": w.convention}
    return out


def make_lines_device(w: Workload, start=0, count=None, out=None, stream=None):
    """Columns of lines start..start+count-1 generated on the current CUDA device (torch tensors)."""
    import torch
    if count is None:
        count = w.n_lines - start
    if out is None:
        out = alloc_lines(w, count)
    p = _Params(seed=w.seed, exomol=int(w.convention == EXOMOL), nu_lo=w.nu_lo, nu_span=w.nu_hi - w.nu_lo,
                log_s_lo=math.log(w.strength_lo), log_s_span=math.log(w.strength_hi) - math.log(w.strength_lo),
                el_mean=w.elower_mean, gref_lo=w.gamma_ref_lo, gref_span=w.gamma_ref_hi - w.gamma_ref_lo,
                nt_lo=w.n_t_lo, nt_span=w.n_t_hi - w.n_t_lo, gup_max=w.gup_max, width_f16=int(w.width_dtype == "f16"))
    s = stream if stream is not None else torch.cuda.current_stream()
    ptr = (lambda t: None if t is None else ctypes.c_void_p(t.data_ptr()))
    rc = _load().rox_synth_lines(ctypes.byref(p), start, count, ptr(out["nu0"]), ptr(out["s_or_a"]), ptr(out["g_up"]),
                                 ptr(out["e_lower"]), ptr(out["gamma_ref"]), ptr(out["n_t"]),
                                 ctypes.c_void_p(s.cuda_stream))
    if rc != 0:
        raise RuntimeError("rox_synth_lines failed (%d)" % rc)
    return out
