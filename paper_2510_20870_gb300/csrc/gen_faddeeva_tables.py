"""Generate rox_faddeeva_tables.h: the constants of the FP32 Faddeeva kernel code.

Run: python gen_faddeeva_tables.py > rox_faddeeva_tables.h  (build() checks it is current)

Everything is derived here from mathematics, with exact rational arithmetic where
it matters; no special-function library is called:
  * Taylor coefficients of Dawson's integral F(x) = exp(-x^2) int_0^x exp(t^2) dt
    around nodes x_c = 0, 0.125, ..., 6.0, from its Maclaurin series
    F(x) = sum_k (-1)^k 2^k x^(2k+1) / (2k+1)!!  (exact rationals, summed to 1e-60)
    and the ODE F' = 1 - 2 x F, which gives (n+1) d_{n+1} = [n=0] - 2 x_c d_n - 2 d_{n-1}.
  * Weideman's rational approximation (J.A.C. Weideman, SIAM J. Numer. Anal. 31 (1994)
    1497-1518): w(z) ~ 1/(sqrt(pi)(L - iz)) + 2/(L - iz)^2 sum_{n=0}^{N-1} a_{n+1} Z^n,
    Z = (L + iz)/(L - iz), L = 2^(-1/4) sqrt(N); a_n are the Fourier coefficients of
    (L^2 + t^2) exp(-t^2) in theta with t = L tan(theta/2), here by a 4N-point
    trapezoid rule (FFT).
  * Numerator and denominator polynomials of the n-level truncation of the Laplace
    continued fraction w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - (2/2)/(z - (3/2)/(z - ...)))).
"""
from fractions import Fraction as Fr
import numpy as np

DAW_STEP = Fr(1, 8)      # node spacing
DAW_NODES = 59           # x_c = 0 .. 7.25
DAW_DEG = 7
WEI_N = 20


def dawson_taylor(xc, deg):
    s = Fr(0)
    term = xc
    k = 0
    while True:
        s += term
        k += 1
        term = term * (-2) * xc * xc / (2 * k + 1)
        if k > 8 and abs(term) < Fr(1, 10 ** 60):
            break
    d = [s]
    for n in range(deg):
        prev = d[n - 1] if n >= 1 else Fr(0)
        d.append(((1 if n == 0 else 0) - 2 * xc * d[n] - 2 * prev) / (n + 1))
    return d


def weideman(N):
    L = 2 ** -0.25 * np.sqrt(N)
    M = 2 * N
    k = np.arange(-M + 1, M)
    theta = k * np.pi / M
    t = L * np.tan(theta / 2)
    f = np.concatenate([[0.0], np.exp(-t * t) * (L * L + t * t)])
    a = np.real(np.fft.fft(np.fft.fftshift(f))) / (2 * M)
    return L, list(np.flipud(a[1:N + 1]))   # a_N .. a_1 (Horner order)


def cf_polys(n):
    """w ~ (i/sqrt(pi)) A(z)/B(z); returns coefficient dicts power -> Fraction."""
    def mul(a, b):
        r = {}
        for i, x in a.items():
            for j, y in b.items():
                r[i + j] = r.get(i + j, 0) + x * y
        return r

    def sub(a, b):
        r = dict(a)
        for j, y in b.items():
            r[j] = r.get(j, 0) - y
        return r
    z = {1: Fr(1)}
    num, den = dict(z), {0: Fr(1)}
    for k in range(n - 1, 0, -1):
        num, den = sub(mul(z, num), {p: Fr(k, 2) * c for p, c in den.items()}), num
    return den, num   # A, B


def even_part_in_zeta(P):
    """P(z) with only even (or only odd) powers -> coefficients in zeta = z^2, highest first, and parity."""
    deg = max(P)
    parity = deg % 2
    assert all(p % 2 == parity for p in P if P[p] != 0)
    return [P.get(p, Fr(0)) for p in range(deg, -1, -2)], parity


def f32(v):
    return "%.9ef" % float(np.float32(float(v)))


def main():
    out = []
    out.append("/* Generated by gen_faddeeva_tables.py -- do not edit. Constants of the FP32")
    out.append("   Faddeeva evaluation (see that script for their mathematical definitions). */")
    out.append("#pragma once")
    out.append("#define ROX_DAW_NODES %d" % DAW_NODES)
    out.append("#define ROX_DAW_DEG %d" % DAW_DEG)
    out.append("#define ROX_DAW_STEP %sf" % float(DAW_STEP))
    out.append("#define ROX_DAW_INV_STEP %sf" % float(1 / DAW_STEP))
    out.append("/* d[node][n] = F^(n)(x_c)/n!, x_c = node * ROX_DAW_STEP, n = 0..ROX_DAW_DEG; rows padded with a")
    out.append("   zero to an odd stride so that lanes reading consecutive nodes hit distinct shared-memory banks */")
    out.append("#define ROX_DAW_STRIDE %d" % (DAW_DEG + 2))
    out.append("ROX_TABLE float rox_daw_taylor[ROX_DAW_NODES][ROX_DAW_STRIDE] = {")
    for i in range(DAW_NODES):
        d = dawson_taylor(i * DAW_STEP, DAW_DEG) + [0]
        out.append("  {" + ", ".join(f32(v) for v in d) + "},")
    out.append("};")
    L, a = weideman(WEI_N)
    out.append("#define ROX_WEI_N %d" % WEI_N)
    out.append("#define ROX_WEI_L %s" % f32(L))
    out.append("/* a_N .. a_1 (Horner order) */")
    out.append("ROX_TABLE float rox_wei_a[ROX_WEI_N] = {" + ", ".join(f32(v) for v in a) + "};")
    for n in (5,):
        A, B = cf_polys(n)
        ca, pa = even_part_in_zeta(A)
        cb, pb = even_part_in_zeta(B)
        out.append("/* CF%d: w ~ (i/sqrt(pi)) A(z)/B(z); A = z^%d a(z^2), B = z^%d b(z^2); coefficients highest first */" % (n, pa, pb))
        out.append("#define ROX_CF%d_A_ODD %d" % (n, pa))
        out.append("ROX_TABLE float rox_cf%d_a[%d] = {%s};" % (n, len(ca), ", ".join(f32(v) for v in ca)))
        out.append("ROX_TABLE float rox_cf%d_b[%d] = {%s};" % (n, len(cb), ", ".join(f32(v) for v in cb)))
    print("\n".join(out))


if __name__ == "__main__":
    main()
