"""Autotuning of the finest level's layout (opts.autotune): the setup
times the candidate layouts / launch shapes of the q = K p pass and keeps
the fastest; the choice is cached per process by matrix shape.  Whatever
it picks, the V-cycle and the solve stay within the parity tolerances of
the oracle, and a second setup of the same shape reuses the choice without
timing."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [A.AMG_FP64, A.AMG_FP32_BF16FINE])
def test_autotuned_layout_keeps_parity_and_is_cached(prec):
    prob = I.poisson_box(3, 20, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    H1 = A.Hierarchy(*args, precision=prec, autotune=1)
    H2 = A.Hierarchy(*args, precision=prec, autotune=1)
    assert H2.info.tune_ms == 0.0  # cached
    assert H1.info.staged_passes == H2.info.staged_passes and H1.info.sell64_warps == H2.info.sell64_warps
    print(f"precision {prec}: layout {H1.info.staged_passes}, warps {H1.info.sell64_warps}, "
          f"tuning {H1.info.tune_ms:.1f} ms")
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    r = np.random.default_rng(3).standard_normal(prob.n)
    z = H1.vcycle(dev(r)).cpu().numpy()
    zo = Ho.vcycle(r)
    tol = 1e-12 if prec == A.AMG_FP64 else 1e-2
    assert np.linalg.norm(z - zo) <= tol * np.linalg.norm(zo)
    g = H1.solve(dev(prob.F), rtol=1e-8)
    ref = Ho.pcg(prob.F, rtol=1e-8, flexible=prec != A.AMG_FP64)
    assert g["status"] == 0
    u = g["u"].cpu().numpy()
    if prec == A.AMG_FP64:
        assert abs(g["iters"] - ref["iters"]) <= 1
    assert np.linalg.norm(u - ref["u"]) <= 1e-7 * np.linalg.norm(ref["u"])
