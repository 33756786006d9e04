"""The device-rate micro-benchmarks return plausible, ordered rates: shared
memory above L2, FP32 FMA above FP64 FMA, all positive and finite."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_measured_rates_are_plausible():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03812_gb300 as P
    from paper_1512_03812_gb300 import binding
    P.build()
    r = binding.measure_peaks(l2_bytes=16 << 20, l2_passes=8)
    for k in ("fp64_tflops", "fp32_tflops", "l2_read_gbs", "smem_read_gbs"):
        assert math.isfinite(r[k]) and r[k] > 0, (k, r[k])
    assert r["fp32_tflops"] > 4 * r["fp64_tflops"]
    assert r["smem_read_gbs"] > r["l2_read_gbs"] > 1000.0
