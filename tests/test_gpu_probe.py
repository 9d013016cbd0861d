"""The FP64 FMA-rate probe behind the FP64 roofline: every variant runs,
keeps its work observable (finite sums) and counts its flops; the fastest
stays within the unit-count rate (SMs x max clock x 2 FMA/clk x 2 flop),
within timing noise."""
import json
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2511_21268_gb300 import amg as A  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_probe_variants_run_and_stay_below_the_unit_count_rate():
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = 2070.0
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mhz = float(json.load(open(path)).get("sm_max_mhz", mhz))
    derived = sms * mhz * 1e6 * 4 / 1e12
    nv = A.amg_dfma_probe_variants()
    assert nv >= 2
    best = 0.0
    for v in range(nv):
        th = A.amg_dfma_probe_threads(v)
        assert th in (128, 256)
        blocks = sms * 4
        out = torch.empty(blocks * th, dtype=torch.float64, device="cuda")
        A.amg_dfma_probe(v, blocks, 64, out)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fl = A.amg_dfma_probe(v, blocks, 4096, out)
        e1.record()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert fl == 2.0 * 16 * 4096 * blocks * th * {0: 8, 1: 4, 2: 2, 3: 8}[v]
        best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    assert 0.3 * derived < best < 1.05 * derived, (best, derived)
    with pytest.raises(A.AmgError):
        A.amg_dfma_probe(nv, 1, 1, out)
