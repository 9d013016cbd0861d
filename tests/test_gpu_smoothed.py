"""Smoothed prolongator on the GPU (Sec. 3.1 "Variants": P_bar = (I -
omega D^-1 K) P) against the oracle, through the C ABI.

* Hierarchies with smoothed prolongators on the first level and on every
  level: P_bar and every coarse matrix P_bar^T K P_bar bit for bit (same
  summation order on both sides), per-row theta on level 0 included.
* The V-cycle within 1e-12 and the PCG solve within 1e-10 (iterations +-1)
  of the oracle's, FP64; mixed precision reaches the FP64 true residual and
  stays within 1e-7 of the FP64 solution.
* Multi-system solves refuse a smoothed hierarchy (their V-cycle uses the
  tentative prolongator's member lists).
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


CASES = [(2, 24, 2, 1), (2, 20, 3, -1), (3, 8, 2, -1), (3, 7, 3, 1), (3, 6, 4, 2)]


@pytest.mark.parametrize("d,n,p,levels", CASES, ids=lambda c: str(c))
def test_smoothed_hierarchy_bit_exact(d, n, p, levels):
    prob = I.poisson_box(d, n, p)
    kw = dict(coarse_max=30, smooth_levels=levels)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, **kw)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), **kw)
    assert H.num_levels == Ho.num_levels >= 2
    for l in range(H.num_levels):
        g = H.export_level(l)
        rp, ci, v = Ho.level_csr(l)
        assert np.array_equal(g["rowptr"], rp) and np.array_equal(g["col"], ci), l
        assert np.array_equal(bits(g["val"]), bits(v)), l
        if l < H.num_levels - 1:
            smoothed = levels < 0 or l < levels
            assert H.info.smoothed[l] == int(smoothed)
            grp, gci, gv = H.export_prolongator(l)
            orp, oci, ov = Ho.prolongator(l)
            assert np.array_equal(grp, orp) and np.array_equal(gci, oci), l
            assert np.array_equal(bits(gv), bits(ov)), l
            assert H.info.p_nnz[l] == len(ov)
    assert abs(H.info.opc - Ho.opc) <= 1e-15


def test_per_row_theta_on_level0_bit_exact():
    prob = I.poisson_box(2, 20, 3)
    theta = 0.4 + I.rng_u01(77, prob.n)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30, smooth_levels=1, theta0=theta)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=30, smooth_levels=1,
                    smooth_theta=dev(theta))
    grp, gci, gv = H.export_prolongator(0)
    orp, oci, ov = Ho.prolongator(0)
    assert np.array_equal(gci, oci) and np.array_equal(bits(gv), bits(ov))
    g = H.export_level(1)
    assert np.array_equal(bits(g["val"]), bits(Ho.level_csr(1)[2]))


@pytest.mark.parametrize("d,n,p,levels", [(2, 32, 3, -1), (3, 10, 3, 1), (3, 9, 2, -1)])
def test_smoothed_vcycle_and_solve_match_oracle(d, n, p, levels):
    prob = I.poisson_box(d, n, p)
    kw = dict(coarse_max=40, smooth_levels=levels)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, **kw)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), **kw)
    r = np.random.default_rng(11).standard_normal(prob.n)
    z = H.vcycle(dev(r)).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    g = H.solve(dev(prob.F), rtol=1e-10)
    ref = Ho.pcg(prob.F, rtol=1e-10)
    assert g["status"] == 0 and abs(g["iters"] - ref["iters"]) <= 1
    u = g["u"].cpu().numpy()
    if g["iters"] != ref["iters"]:
        u = H.solve(dev(prob.F), rtol=0.0, itmax=ref["iters"])["u"].cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-10 * np.linalg.norm(ref["u"])
    plain = Ho.__class__(prob.rowptr, prob.col, prob.val, coarse_max=40).pcg(prob.F, rtol=1e-10)
    print(f"d={d} n={n} p={p} smooth_levels={levels}: iterations {g['iters']} (tentative P: {plain['iters']}), "
          f"OPC {H.info.opc:.2f}")


@pytest.mark.parametrize("prec", [A.AMG_FP32, A.AMG_FP32_BF16FINE])
def test_smoothed_mixed_precision(prec):
    prob = I.poisson_box(3, 14, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    u64 = A.Hierarchy(*args, smooth_levels=-1).solve(dev(prob.F), rtol=1e-8)["u"].cpu().numpy()
    g = A.Hierarchy(*args, smooth_levels=-1, precision=prec).solve(dev(prob.F), rtol=1e-8)
    assert g["status"] == 0
    u = g["u"].cpu().numpy()
    K = sp.csr_matrix((prob.val, prob.col, prob.rowptr))
    assert np.linalg.norm(prob.F - K @ u) <= 1e-8 * 1.0001 * np.linalg.norm(prob.F)
    assert np.linalg.norm(u - u64) <= 1e-7 * np.linalg.norm(u64)


def test_multi_system_solves_refuse_smoothed_hierarchy():
    prob = I.poisson_box(2, 16, 2)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), smooth_levels=1, coarse_max=20)
    F = dev(np.stack([prob.F, prob.F]))
    with pytest.raises(A.AmgError):
        H.solve_multi(F)
