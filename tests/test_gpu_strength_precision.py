"""The strengths the cross-section launches use, read back per line.

The cross-section path computes S(T) in a reduced form (FP64 Boltzmann exponent and its
reduction, FP32 exp of the reduced argument, FP32 stimulated-emission factors and prefactor;
paper, "Compute line-strengths and -widths"). rox_line_strengths_reduced returns exactly those
values; here they are compared line by line with the FP64 oracle for HITRAN- and ExoMol-style
lists at 100-3000 K, including lines around the FP64 fallbacks: Boltzmann exponents near
|a| = 700 and FP32 products near 2^-100 and 2^100 (extreme S_ref or A). The bound, 1e-6
relative, is the sum of the FP32 roundings and of the expf / expm1f errors of the form."""
import numpy as np
import pytest

import oracle
import rox_synth as rs
from rox_testutil import to_device

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2510_20870_gb300 as rox  # noqa: E402

HITRAN, EXOMOL = 0, 1     # line-list conventions (include/rox.h)
REL_BOUND = 1e-6
TEMPS = (100.0, 296.0, 700.0, 1500.0, 3000.0)


def _lines(convention, n=200_000, n_extreme=4_000, seed=31):
    rng = np.random.default_rng(seed + convention)
    nu0 = np.sort(rng.uniform(20.0, 30000.0, n + 2 * n_extreme))
    m = nu0.size
    if convention == HITRAN:
        s = np.exp(rng.uniform(np.log(1e-30), np.log(1e-19), m))
        el = rng.exponential(3000.0, m)
    else:
        s = np.exp(rng.uniform(np.log(1e-8), np.log(1e2), m))
        el = rng.exponential(5000.0, m)
    pick = rng.permutation(m)
    ext_s, ext_e = pick[:n_extreme], pick[n_extreme:2 * n_extreme]
    # strengths (or Einstein A) over the whole FP32 range: products near 2^-100 and 2^100
    s[ext_s] = np.exp(rng.uniform(np.log(1e-44), np.log(1e37), n_extreme))
    # lower-state energies around |a| = 700 at 3000 K (HITRAN: a = c2 E'' (1/296 - 1/T))
    el[ext_e] = rng.uniform(1.50e5, 1.70e5, n_extreme)
    out = {"nu0": nu0, "s_or_a": s.astype(np.float32), "e_lower": el.astype(np.float32),
           "gamma_ref": np.full(m, 0.05, np.float32), "n_t": np.full(m, 0.5, np.float32), "convention": convention,
           "g_up": None}
    if convention == EXOMOL:
        out["g_up"] = (1.0 + np.floor(rng.uniform(0.0, 100.0, m))).astype(np.float32)
    return out


@pytest.mark.parametrize("convention", [HITRAN, EXOMOL])
def test_reduced_strengths_match_the_oracle_per_line(convention):
    L = _lines(convention)
    dl = to_device(L, torch)
    w = rs.CONFIGS[1] if convention == HITRAN else rs.CONFIGS[2]
    qi = rs.q_table(w)
    Qr = float(oracle.partition_function(qi, oracle.T_REF))
    S = torch.empty(len(L["nu0"]), dtype=torch.float64, device="cuda")
    near = 0
    for T in TEMPS:
        Qt = float(oracle.partition_function(qi, T))
        rox.rox_line_strengths_reduced(dl, T, Qt, Qr, S)
        got = S.cpu().numpy()
        with np.errstate(over="ignore"):          # lines beyond |a| ~ 709 overflow the oracle's exp
            ref = oracle.line_strength(L, T, Qt, Qr)
        ok = (ref > 1e-290) & (ref < 1e290)
        rel = np.abs(got[ok] - ref[ok]) / ref[ok]
        worst = float(rel.max())
        # the exponent a of each line, and how many lines sit near the fallback thresholds
        c2 = oracle.C2
        el = L["e_lower"].astype(np.float64)
        a = -c2 * el * (1.0 / T - 1.0 / oracle.T_REF) if convention == HITRAN else -c2 * el / T
        near += int(np.sum(np.abs(np.abs(a[ok]) - 700.0) < 20.0))
        assert np.all(np.abs(got[ref == 0.0]) < 1e-300)   # underflow on both sides
        print("PARITY reduced strengths conv %d T=%g: max rel err %.3e over %d lines" % (convention, T, worst, ok.sum()))
        assert worst <= REL_BOUND, (convention, T, worst)
    if convention == HITRAN:
        assert near > 100          # lines on both sides of |a| = 700 were checked
