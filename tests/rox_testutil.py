"""Shared helpers of the test suite: device copies of synthetic line lists, the
tolerance of the cross-section parity checks, and oracle shortcuts."""
import numpy as np

import oracle
import rox_synth as rs

# Parity tolerance for a cross-section (per (P,T) point), M = max of the oracle's sigma:
# |gpu - oracle| / oracle <= 1e-4 where oracle > 1e-6 M, and |gpu - oracle| <= 1e-8 M elsewhere.
REL_TOL = 1e-4
REL_FLOOR = 1e-6
ABS_FLOOR = 1e-8


def check_sigma(gpu, ref, M=None, rel_tol=REL_TOL, label=""):
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert gpu.shape == ref.shape
    if M is None:
        M = float(ref.max()) if ref.size else 0.0
    big = ref > REL_FLOOR * M
    err = np.abs(gpu - ref)
    rel = np.where(big, err / np.where(big, ref, 1.0), 0.0)
    worst_rel = float(rel.max()) if rel.size else 0.0
    small_err = float(err[~big].max()) if (~big).any() else 0.0
    assert np.all(np.isfinite(gpu)), label + ": non-finite output"
    assert worst_rel <= rel_tol, "%s: max rel err %.3e at %d (gpu %r ref %r)" % (
        label, worst_rel, int(rel.argmax()), gpu[rel.argmax()], ref[rel.argmax()])
    assert small_err <= ABS_FLOOR * M + 1e-300, "%s: abs err %.3e > %.3e" % (label, small_err, ABS_FLOOR * M)
    print("PARITY %s: max rel err %.3e over %d points (abs err below the floor %.3e of M)" % (
        label, worst_rel, int(big.sum()), small_err / M if M > 0 else 0.0))
    return worst_rel


def q_pair(w, T):
    qi = rs.q_table(w)
    return float(oracle.partition_function(qi, T)), float(oracle.partition_function(qi, oracle.T_REF))


def to_device(lines, torch):
    out = {"convention": lines["convention"]}
    for k in ("nu0", "s_or_a", "g_up", "e_lower", "gamma_ref", "n_t"):
        v = lines.get(k)
        out[k] = None if v is None else torch.from_numpy(np.ascontiguousarray(v)).cuda()
    return out
