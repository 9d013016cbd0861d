"""Mixed-precision solve (FP32 V-cycle, optionally BF16 finest-level values;
FP32 outer SpMV; FP64 flexible-CG recurrences with FP64 true-residual
replacement) against the FP64 CPU oracle.

Bars: the hierarchy is the FP64 one (bit-exact); the solve reaches the
requested rtol on the FP64 true residual; the solution's relative error
against the FP64 oracle solution is at most 1e-7 at rtol 1e-8 (printed);
iteration counts stay within 1.3x + 5 of the FP64 ones (the FP32 outer
operator can cost a few extra iterations before the FP64 true residual
confirms convergence).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402

MIXED_SOL_RTOL = 1e-7
VCYCLE_ERR = {A.AMG_FP32: 1e-5, A.AMG_FP32_BF16FINE: 3e-2}


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("prec", [A.AMG_FP32, A.AMG_FP32_BF16FINE])
@pytest.mark.parametrize("d,n,p", [(3, 14, 3), (2, 40, 2), (3, 10, 4)])
def test_mixed_solve_error_vs_fp64_oracle(prec, d, n, p):
    prob = I.poisson_box(d, n, p)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    ref = Ho.pcg(prob.F, rtol=1e-8, flexible=True)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=prec)
    g = H.solve(gpu(prob.F), rtol=1e-8)
    assert g["status"] == 0
    assert g["relres"] <= 1e-8  # FP64 true residual
    err = np.linalg.norm(g["u"].cpu().numpy() - ref["u"]) / np.linalg.norm(ref["u"])
    print(f"precision={prec} d={d} n={n} p={p}: iters {g['iters']} (fp64 oracle {ref['iters']}), "
          f"relative error vs FP64 oracle {err:.2e}")
    assert err <= MIXED_SOL_RTOL
    assert g["iters"] <= int(1.3 * ref["iters"]) + 5


@pytest.mark.parametrize("prec", [A.AMG_FP32, A.AMG_FP32_BF16FINE])
def test_mixed_hierarchy_is_the_fp64_one_and_vcycle_error(prec):
    prob = I.poisson_box(3, 9, 3)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=prec)
    for l in range(H.num_levels):
        rp, ci, v = Ho.level_csr(l)
        g = H.export_level(l)
        assert np.array_equal(g["val"].view(np.uint64), v.view(np.uint64))
    r = np.random.default_rng(3).standard_normal(prob.n)
    z = H.vcycle(gpu(r)).cpu().numpy()
    zo = Ho.vcycle(r)
    err = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    print(f"precision={prec}: V-cycle relative error vs FP64 oracle {err:.2e}")
    assert err <= VCYCLE_ERR[prec]


def test_mixed_replacement_only_at_convergence_and_itmax():
    prob = I.poisson_box(3, 12, 3)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=A.AMG_FP32_BF16FINE,
                    resid_replace_every=0)
    g = H.solve(gpu(prob.F), rtol=1e-8)
    assert g["status"] == 0 and g["relres"] <= 1e-8
    c = H.solve(gpu(prob.F), rtol=1e-12, itmax=7)
    assert c["status"] == A.AMG_ERR_NOT_CONVERGED and c["iters"] == 7
    z = H.solve(torch.zeros(prob.n, dtype=torch.float64, device="cuda"), rtol=1e-8)
    assert z["iters"] == 0 and z["status"] == 0


def _expected_staged_kind(prob):
    """Sliced lane-per-row slabs (2) when the 32-row slabs average at least
    16 run slots (the largest run count of their rows), else lane-per-run
    slabs (1); runs are maximal sequences of consecutive columns."""
    rp, ci = prob.rowptr, prob.col
    runs = np.array([1 + np.count_nonzero(np.diff(ci[rp[i]:rp[i + 1]]) != 1) for i in range(prob.n)])
    nsl = (prob.n + 31) // 32
    pad = np.zeros(nsl * 32, dtype=runs.dtype)
    pad[:prob.n] = runs
    return 2 if pad.reshape(nsl, 32).max(axis=1).mean() >= 16 else 1


@pytest.mark.parametrize("prec", [A.AMG_FP32, A.AMG_FP32_BF16FINE])
@pytest.mark.parametrize("d,n,p", [(3, 14, 3), (3, 16, 2), (3, 10, 4), (2, 40, 2)])
def test_staged_finest_passes_kind_and_vcycle(prec, d, n, p):
    """Both staged finest-level layouts (sliced slabs with LM = 5, 7, 9 and
    lane-per-run slabs), with level 1 sliced too where it applies, give the
    FP64 oracle's V-cycle within the precision's bound, and the layout follows
    the slab run-count rule."""
    prob = I.poisson_box(d, n, p)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=prec)
    kind = _expected_staged_kind(prob)
    assert H.info.level_format[0] == 1
    assert H.info.staged_passes == kind
    if kind == 2:
        assert H.info.staged_slots >= prob.nnz
    # level 1 (plain CSR) is sliced as well when the finest level is and it
    # has at least 16 slabs of rows above a coarser level
    expect1 = int(kind == 2 and H.num_levels >= 3 and H.info.n[1] >= 16 * 32)
    assert H.info.staged_level1 == expect1
    r = np.random.default_rng(5).standard_normal(prob.n)
    z = H.vcycle(gpu(r)).cpu().numpy()
    zo = Ho.vcycle(r)
    err = np.linalg.norm(z - zo) / np.linalg.norm(zo)
    print(f"precision={prec} d={d} n={n} p={p}: staged kind {kind}, V-cycle error vs FP64 oracle {err:.2e}")
    assert err <= VCYCLE_ERR[prec]
    g = H.solve(gpu(prob.F), rtol=1e-8)
    assert g["status"] == 0 and g["relres"] <= 1e-8


def test_staged_wait_expires_and_context_stays_usable():
    """The bounded mbarrier wait of the staged passes gives up on a barrier
    that nothing completes (status, no hang) and returns on a completed one;
    the device is usable afterwards."""
    import time
    t0 = time.perf_counter()
    timed_out, completed = A.amg_staged_wait_selftest(2.0)
    assert timed_out == 1 and completed == 1
    assert time.perf_counter() - t0 < 5.0
    prob = I.poisson_box(3, 9, 3)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=A.AMG_FP32_BF16FINE)
    g = H.solve(gpu(prob.F), rtol=1e-8)
    assert g["status"] == 0 and g["relres"] <= 1e-8
