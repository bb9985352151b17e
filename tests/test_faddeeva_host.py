"""Accuracy of the kernels' FP32 Faddeeva code, compiled for the host CPU (same source
as the device code, rox_faddeeva.cuh), against scipy.special.wofz in FP64."""
import ctypes

import numpy as np
import pytest
from scipy.special import wofz


@pytest.fixture(scope="module")
def host_re_w():
    import __graft_entry__
    path = __graft_entry__._build_module().build_host_lib()
    lib = ctypes.CDLL(path)
    f = lib.rox_host_re_w
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]

    def call(x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        out = np.empty_like(x)
        f(x.ctypes.data, y.ctypes.data, out.ctypes.data, x.size)
        return out
    return call


def _grid():
    x = np.concatenate([np.linspace(0, 8, 1601), np.linspace(8, 40, 801), np.logspace(np.log10(40), 5, 200),
                        [4.5, 6.0, 10.0, 22.0]])
    y = np.concatenate([[0.0, 1e-30], np.logspace(-9, 4, 400), [0.1, 1.0]])
    X, Y = np.meshgrid(x, y)
    return X.ravel().astype(np.float32), Y.ravel().astype(np.float32)


def test_relative_accuracy_everywhere(host_re_w):
    X, Y = _grid()
    got = host_re_w(X, Y).astype(np.float64)
    ref = wofz(X.astype(np.float64) + 1j * Y.astype(np.float64)).real
    m = ref > 1e-15            # below 1e-15 of the line peak nothing can reach the tolerance
    rel = np.abs(got[m] - ref[m]) / ref[m]
    assert rel.max() < 2e-5, rel.max()
    assert np.all(np.abs(got[~m]) < 2e-15)


def test_special_cases(host_re_w):
    from scipy.special import erfcx
    y = np.logspace(-8, 3, 200).astype(np.float32)
    got = host_re_w(np.zeros_like(y), y).astype(np.float64)
    assert np.allclose(got, erfcx(y.astype(np.float64)), rtol=1e-5, atol=0)
    x = np.linspace(0, 6, 601).astype(np.float32)
    got = host_re_w(x, np.zeros_like(x)).astype(np.float64)
    g = np.exp(-x.astype(np.float64) ** 2)
    assert np.allclose(got, g, rtol=2e-5, atol=1e-16)
    # symmetric in x
    xs = np.linspace(-30, 30, 241).astype(np.float32)
    ys = np.full_like(xs, 0.37)
    assert np.array_equal(host_re_w(xs, ys), host_re_w(-xs, ys))
