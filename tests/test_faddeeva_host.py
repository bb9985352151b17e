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


@pytest.fixture(scope="module")
def host_far():
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build_host_lib())
    f = lib.rox_host_re_w_far
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    r2 = lib.rox_host_far_r2
    r2.argtypes = [ctypes.c_float]
    r2.restype = ctypes.c_float

    def call(x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        out = np.empty_like(x)
        f(x.ctypes.data, y.ctypes.data, out.ctypes.data, x.size)
        return out
    return call, r2


def test_far_form_accuracy_outside_its_zone(host_far):
    """The Voigt kernel's pair formula, against wofz: the per-line Pade form from |z|^2 = 6.5^2
    (y < 0.75), 6.5^2 + 3.5 / |4 y^2 - 3| (0.75 <= y < 0.95, around its coefficients' pole at
    y = 0.866) and max(6.5^2, 42 y) (0.95 <= y < 11.5) outward; the 2-level fraction from |z| = 22
    outward where the Pade boundary would pass 22 (next to the pole, and y >= 11.5)."""
    far, r2 = host_far
    worst = {}
    pade_ys = set()
    for y in np.concatenate([[0.0, 1e-12], np.logspace(-9, np.log10(0.4999), 120),
                             [0.5, 0.6, 0.7, 0.7499, 0.75, 0.8, 0.866, 0.9, 0.9499, 0.95, 1.0, 1.5, 11.49, 11.5],
                             np.linspace(0.75, 0.95, 81), 0.8660254 + np.linspace(-0.004, 0.004, 33),
                             np.linspace(1.0, 11.4, 53), np.logspace(0, 3, 40)]).astype(np.float32):
        R2 = r2(float(y))
        if y < 0.75:
            want = 42.25
        elif y < 0.95:
            g = abs(float(np.float32(4.0) * y * y - np.float32(3.0)))
            want = 42.25 + 3.5 / g if g > 0 else np.inf
        elif y < 11.5:
            want = max(42.25, float(np.float32(42.0) * y))
        else:
            want = np.inf
        want = want if want < 484.0 else 484.0
        assert abs(R2 - want) <= 1e-5 * want, (y, R2, want)
        if R2 < 484.0:
            pade_ys.add(float(y))
        x0 = np.sqrt(max(0.0, R2 - float(y) ** 2))
        x = np.concatenate([x0 + np.linspace(0, 2, 401), x0 + np.logspace(0.31, 5, 400)]).astype(np.float32)
        x = x[x.astype(np.float64) ** 2 + float(y) ** 2 >= R2]
        got = far(x, np.full_like(x, y)).astype(np.float64)
        ref = wofz(x.astype(np.float64) + 1j * float(y)).real
        if R2 < 484.0 and y < 1e-9:
            # the form omits e^{-x^2} <= e^{-42.25} = 4.5e-19 (of the line peak, Re w(0, y) ~ 1);
            # below y = 1e-9 that part is no longer small next to the Lorentz wing itself
            assert np.all(np.abs(got - ref) < 5e-19)
            continue
        m = ref > 1e-15
        if m.any():
            rel = np.abs(got[m] - ref[m]) / ref[m]
            worst[float(y)] = rel.max()
        assert np.all(np.abs(got[~m]) < 2e-15)
    pade = max(v for k, v in worst.items() if k in pade_ys)
    cf2 = max(v for k, v in worst.items() if k not in pade_ys)
    print("far form: Pade worst %.2e, 2-level fraction worst %.2e" % (pade, cf2))
    assert pade < 6e-6, pade      # 3.4e-6 in exact arithmetic, plus FP32 rounding
    assert cf2 < 2e-5, cf2


def test_far_form_pade_reduces_to_series(host_far):
    """At y -> 0 the Pade form is (y/sqrt(pi)) (u - 7/2)/(u^2 - 5u + 15/4); its expansion must
    reproduce 1/u + 3/(2u^2) + 15/(4u^3) + 105/(8u^4) (the asymptotic series of Re w / y at y = 0)."""
    far, _ = host_far
    y = 1e-6
    for u in (60.0, 200.0, 1000.0):
        x = np.float32(np.sqrt(u))
        got = float(far(np.array([x]), np.array([y], dtype=np.float32))[0]) * np.sqrt(np.pi) / y
        uu = float(x) ** 2
        series = 1 / uu + 1.5 / uu**2 + 3.75 / uu**3 + 13.125 / uu**4
        assert abs(got - series) / series < 2e-6 + 100 / uu**4, (u, got, series)   # next term O(u^-5)


def test_core_forms_to_radius_7():
    """rox_re_w_core (Dawson-Taylor for y < 0.1, Weideman above) stands alone in the Voigt
    kernel's |z| < 6.5 zone of lines with the Pade far form and the boundary 6.5^2 (y < 0.75 and
    0.95 <= y < 1.006): it must hold out to |z| = 7.1 there."""
    import __graft_entry__
    lib = ctypes.CDLL(__graft_entry__._build_module().build_host_lib())
    f = lib.rox_host_re_w_core
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64]
    worst = 0.0
    for y in np.concatenate([[0.0, 1e-9], np.logspace(-7, np.log10(0.4999), 150), np.linspace(0.5, 0.75, 11),
                             np.linspace(0.95, 1.01, 7)]):
        x = np.linspace(0, np.sqrt(max(0.0, 7.1 ** 2 - y * y)), 1500).astype(np.float32)
        yy = np.full_like(x, np.float32(y))
        out = np.empty_like(x)
        f(x.ctypes.data, yy.ctypes.data, out.ctypes.data, x.size)
        ref = wofz(x.astype(np.float64) + 1j * float(yy[0])).real
        m = ref > 1e-15
        worst = max(worst, float((np.abs(out.astype(np.float64) - ref)[m] / ref[m]).max()))
    assert worst < 1.5e-5, worst
