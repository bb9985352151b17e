"""The measurement probes of include/rox.h (the roofline's denominators): they launch, report the
work they do, refuse bad arguments, and the pair loop's rate stays below the FMA peak."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2510_20870_gb300 import _binding as rb  # noqa: E402

SPAN = rb.ROX_SPAN


def _rate(launch, n=3):
    launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    work = sum(launch() for _ in range(n))
    e1.record()
    torch.cuda.synchronize()
    return work / (e0.elapsed_time(e1) * 1e-3)


def test_probe_work_counts_and_refusals():
    nb = 8
    out = torch.empty(rb.rox_fp32_probe_out_size(nb) // 4, dtype=torch.float32, device="cuda")
    assert rb.rox_fp32_probe(nb, 3, out) == nb * 256 * 3 * 8 * 16
    # per thread: reps x 16 pairs x 2 lines x (ROX_SPAN / 32) points
    assert rb.rox_pair_loop_probe(nb, 3, out) == nb * 256 * 3 * 16 * 2 * (SPAN // 32)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    with pytest.raises(rb.RoxError):
        rb.rox_pair_loop_probe(nb + 1, 3, out)          # buffer too small
    with pytest.raises(rb.RoxError):
        rb.rox_pair_loop_probe(nb, 0, out)


def test_pair_loop_rate_below_the_fma_peak():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nb = sms * 4
    out = torch.empty(rb.rox_fp32_probe_out_size(nb) // 4, dtype=torch.float32, device="cuda")
    peak = _rate(lambda: rb.rox_fp32_probe(nb, 2_000, out))
    loop = _rate(lambda: rb.rox_pair_loop_probe(sms * 3, 200, out))
    print("PROBES FMA peak %.3e FMA/s; pair loop %.3e evals/s" % (peak, loop))
    # the pair loop does 11 flops (about 6 FMA-pipe operations) per evaluation: below the FMA peak
    assert loop * 6.0 <= 1.05 * peak
