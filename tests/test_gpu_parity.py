"""GPU path vs the CPU oracle, through the C ABI (arXiv 2511.21268 Sec. 3-4).

Setup results must be bit-exact (matchings, aggregates, prolongator
values, Galerkin matrices, l1 diagonals, test vectors).  The FP64 solve
must agree with the oracle within 1e-10 relative at equal iteration counts,
with iteration counts within +-1; the V-cycle and level SpMVs within
1e-12 / 1e-13 relative (summation order is the only difference).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402

VCYCLE_RTOL = 1e-12
SPMV_RTOL = 1e-13
SOLVE_RTOL = 1e-10

CASES = [
    (2, 32, 2),   # 2-D p=2 n=32: N = 1,024 (the small plain-method workload)
    (2, 21, 4),   # ragged 2-D, p=4
    (3, 9, 3),    # 3-D p=3, several levels
    (3, 13, 2),   # 3-D p=2, ragged group tails
]


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def setup_both(prob, **opts):
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, **opts)
    okw = {k: v for k, v in opts.items() if k in ("nu_pre", "nu_post", "match_passes", "coarse_max", "max_levels",
                                                   "testvec_sweeps", "testvec_kind", "seed", "stag", "dense_max")}
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, **okw)
    return H, Ho


def assert_setup_identical(H, Ho):
    assert H.num_levels == Ho.num_levels
    for l in range(H.num_levels):
        g = H.export_level(l)
        rp, ci, v = Ho.level_csr(l)
        assert np.array_equal(g["rowptr"], rp), f"level {l} rowptr"
        assert np.array_equal(g["col"], ci), f"level {l} col"
        assert np.array_equal(g["val"].view(np.uint64), v.view(np.uint64)), f"level {l} values not bit-exact"
        d, w = Ho.level_vectors(l)
        assert np.array_equal(g["dl1"].view(np.uint64), d.view(np.uint64)), f"level {l} l1 diagonal"
        if g["w"] is not None:
            assert np.array_equal(g["w"].view(np.uint64), w.view(np.uint64)), f"level {l} test vector"
        if l < H.num_levels - 1:
            agg, pv = Ho.level_map(l)
            assert np.array_equal(g["agg"], agg), f"level {l} aggregates"
            assert np.array_equal(g["pval"].view(np.uint64), pv.view(np.uint64)), f"level {l} prolongator"
            for s in range(Ho.level_npass(l)):
                mg, ag, pg = H.export_pass(l, s)
                mo, ao, po = Ho.pass_map(l, s)
                assert np.array_equal(mg, mo), f"level {l} pass {s} matching"
                assert np.array_equal(ag, ao)
                assert np.array_equal(pg.view(np.uint64), po.view(np.uint64))
    # a9: the coarsest level's Cholesky factor bit for bit (same operation
    # order, each product and difference rounded once), its inverse against
    # numpy's inverse of the coarse matrix
    Lg, Ai = H.export_coarse()
    Lo = Ho.coarse_chol()
    assert np.array_equal(Lg.view(np.uint64), Lo.view(np.uint64)), "coarse Cholesky factor"
    rp, ci, v = Ho.level_csr(H.num_levels - 1)
    nc = len(rp) - 1
    Kc = np.zeros((nc, nc))
    for i in range(nc):
        Kc[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    inv = np.linalg.inv(Kc)
    assert np.abs(Ai - inv).max() <= 1e-11 * np.abs(inv).max(), "coarse inverse"


@pytest.mark.parametrize("d,n,p", CASES)
def test_setup_bit_exact(d, n, p):
    prob = I.poisson_box(d, n, p)
    H, Ho = setup_both(prob, coarse_max=20)
    assert H.num_levels >= 3
    assert_setup_identical(H, Ho)
    assert abs(H.info.opc - Ho.opc) < 1e-15


@pytest.mark.parametrize("opts", [dict(match_passes=1), dict(match_passes=3), dict(testvec_kind=1),
                                  dict(testvec_sweeps=0), dict(seed=7, coarse_max=50)])
def test_setup_bit_exact_options(opts):
    prob = I.poisson_box(3, 8, 3)
    H, Ho = setup_both(prob, **opts)
    assert_setup_identical(H, Ho)


def test_setup_bit_exact_variable_coefficient_annulus():
    prob = I.annulus_kappa(6, 2, kappa_seed=3)
    H, Ho = setup_both(prob, coarse_max=30)
    assert_setup_identical(H, Ho)


def _symmetry_variant(prob, lower_ulps):
    """The input with every lower entry set to its upper mirror's bits, moved
    by `lower_ulps` ulps: 0 gives a matrix symmetric in every bit, 1 one that
    is symmetric only up to rounding."""
    import types
    rp, ci = prob.rowptr, prob.col
    v = prob.val.copy()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    low = np.nonzero(ci < rows)[0]
    for k in low:
        i, j = rows[k], ci[k]
        m = rp[j] + np.searchsorted(ci[rp[j]:rp[j + 1]], i)
        v[k] = v[m]
    if lower_ulps:
        v[low] = np.nextafter(v[low], np.inf)
    return types.SimpleNamespace(rowptr=rp, col=ci, val=v)


@pytest.mark.parametrize("lower_ulps", [0, 1])
def test_setup_bit_exact_bit_symmetric_and_rounding_symmetric_input(lower_ulps):
    """The Galerkin values kernel computes the lower triangle in place when
    the level matrix is symmetric in every bit (0) and leaves it to the
    mirror pass when it is symmetric only up to rounding (1); the oracle
    takes K_c(I,J), J < I, from K_c(J,I) in both cases."""
    prob = _symmetry_variant(I.annulus_kappa(6, 2, kappa_seed=3), lower_ulps)
    H, Ho = setup_both(prob, coarse_max=30)
    assert_setup_identical(H, Ho)


@pytest.mark.parametrize("d,n,p", CASES)
def test_level_spmv_matches_oracle(d, n, p):
    prob = I.poisson_box(d, n, p)
    H, Ho = setup_both(prob, coarse_max=20)
    rng = np.random.default_rng(0)
    for l in range(H.num_levels):
        x = rng.standard_normal(H.level_n(l))
        y = H.spmv(l, gpu(x)).cpu().numpy()
        rp, ci, v = Ho.level_csr(l)
        yo = O.spmv(rp, ci, v, x)
        assert np.abs(y - yo).max() <= SPMV_RTOL * np.abs(yo).max() * 10


def sliced_fp64_expected(prob):
    """The FP64 sliced passes (staged_passes 3) apply when the 32-row slabs
    average at least 16 run slots (the largest run count of their rows)."""
    rp, ci = prob.rowptr, prob.col
    runs = np.array([1 + np.count_nonzero(np.diff(ci[rp[i]:rp[i + 1]]) != 1) for i in range(prob.n)])
    nsl = (prob.n + 31) // 32
    pad = np.zeros(nsl * 32, dtype=runs.dtype)
    pad[:prob.n] = runs
    return pad.reshape(nsl, 32).max(axis=1).mean() >= 16


@pytest.mark.parametrize("d,n,p", CASES)
@pytest.mark.parametrize("nu", [(1, 1), (2, 3)])
@pytest.mark.parametrize("fmt", [0, 1, 2], ids=["csr", "runs", "sliced"])
def test_vcycle_matches_oracle(d, n, p, nu, fmt):
    prob = I.poisson_box(d, n, p)
    H, Ho = setup_both(prob, coarse_max=20, nu_pre=nu[0], nu_post=nu[1], matrix_format=fmt)
    # tensor-product rows: equal runs of consecutive columns
    assert H.info.level_format[0] == min(fmt, 1)
    sliced = fmt == 2 and H.num_levels > 1 and sliced_fp64_expected(prob)
    assert H.info.staged_passes == (3 if sliced else 0)
    if sliced:
        assert H.info.staged_slots >= prob.nnz and H.info.staged_window_bytes > 0
    assert H.info.staged_level1 == 0  # level 1 runs sliced only in mixed precision
    rng = np.random.default_rng(1)
    for _ in range(3):
        r = rng.standard_normal(prob.n)
        z = H.vcycle(gpu(r)).cpu().numpy()
        zo = Ho.vcycle(r)
        assert np.linalg.norm(z - zo) <= VCYCLE_RTOL * np.linalg.norm(zo)


@pytest.mark.parametrize("d,n,p", [(3, 16, 3), (3, 14, 2)])
def test_fp64_sliced_finest_passes_match_oracle(d, n, p):
    """FP64 sliced passes on the finest level (run slots of LM values, a warp
    per slab), on hierarchies with several blocks' worth of slabs: the
    V-cycle and the solve against the oracle."""
    prob = I.poisson_box(d, n, p)
    H, Ho = setup_both(prob, coarse_max=20)
    assert H.info.staged_passes == 3 and H.info.staged_level1 == 0
    rng = np.random.default_rng(4)
    for _ in range(2):
        r = rng.standard_normal(prob.n)
        z = H.vcycle(gpu(r)).cpu().numpy()
        zo = Ho.vcycle(r)
        assert np.linalg.norm(z - zo) <= VCYCLE_RTOL * np.linalg.norm(zo)
    compare_solves(prob, 1e-8, coarse_max=20)


def compare_solves(prob, rtol, flexible=False, **opts):
    H, Ho = setup_both(prob, flexible=int(flexible), **opts)
    go = Ho.pcg(prob.F, rtol=rtol, flexible=flexible)
    gg = H.solve(gpu(prob.F), rtol=rtol)
    assert gg["status"] == 0 and go["status"] == 0
    assert abs(gg["iters"] - go["iters"]) <= 1, (gg["iters"], go["iters"])
    ug = gg["u"].cpu().numpy()
    if gg["iters"] != go["iters"]:  # compare at equal iteration counts
        ug = H.solve(gpu(prob.F), rtol=0.0, itmax=go["iters"])["u"].cpu().numpy()
    err = np.linalg.norm(ug - go["u"]) / np.linalg.norm(go["u"])
    assert err <= SOLVE_RTOL, err
    assert gg["relres"] <= rtol * 1.0001
    return H, Ho, gg, go


@pytest.mark.parametrize("d,n,p", CASES)
@pytest.mark.parametrize("fmt", [0, 1], ids=["csr", "runs"])
def test_pcg_matches_oracle(d, n, p, fmt):
    compare_solves(I.poisson_box(d, n, p), 1e-8, coarse_max=20, matrix_format=fmt)


def test_pcg_small_plain_method_config():
    """2-D p=2 n=32 (N=1,024), defaults (coarsest <= 200 rows), rtol 1e-6."""
    prob = I.poisson_box(2, 32, 2)
    H, Ho, gg, go = compare_solves(prob, 1e-6)
    assert H.level_n(H.num_levels - 1) <= 200


def test_flexible_cg_matches_oracle():
    compare_solves(I.poisson_box(3, 8, 3), 1e-9, flexible=True, coarse_max=20)


def test_random_rhs_and_host_buffers():
    prob = I.poisson_box_random_rhs(2, 24, 3, seed=11)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val)
    u = np.zeros(prob.n)
    st, it, rr = A.amg_pcg_solve(H._h, prob.F, u, 1e-10, 500)  # host pointers
    assert st == 0 and rr <= 1e-10
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    go = Ho.pcg(prob.F, rtol=1e-10)
    assert abs(it - go["iters"]) <= 1
    # discretisation-independent check: F = K u_true exactly solvable
    assert np.linalg.norm(u - prob.u_true) <= 1e-6 * np.linalg.norm(prob.u_true)


def test_single_level_hierarchy_is_exact_solve():
    prob = I.poisson_box(2, 8, 2)  # 64 rows <= coarse_max
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val)
    assert H.num_levels == 1
    g = H.solve(gpu(prob.F), rtol=1e-12)
    assert g["iters"] == 1 and g["relres"] < 1e-12


def test_warm_start_zero_rhs_and_itmax():
    prob = I.poisson_box(2, 16, 2)
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    a = H.solve(gpu(prob.F), rtol=1e-10)
    b = H.solve(gpu(prob.F), u=a["u"].clone(), rtol=1e-10)
    assert b["iters"] == 0
    z = H.solve(torch.zeros(prob.n, dtype=torch.float64, device="cuda"), rtol=1e-10)
    assert z["iters"] == 0 and z["status"] == 0 and not z["u"].any()
    c = H.solve(gpu(prob.F), rtol=1e-14, itmax=3)
    assert c["status"] == A.AMG_ERR_NOT_CONVERGED and c["iters"] == 3
    e = H.solve(gpu(prob.F), rtol=1e-10, itmax=0)
    assert e["status"] == A.AMG_ERR_NOT_CONVERGED and e["iters"] == 0


def test_iterates_match_oracle_step_by_step():
    prob = I.poisson_box(3, 10, 3)
    H, Ho = setup_both(prob, coarse_max=20)
    for k in (1, 2, 5, 9):
        go = Ho.pcg(prob.F, rtol=0.0, itmax=k)
        gg = H.solve(gpu(prob.F), rtol=0.0, itmax=k)
        assert gg["iters"] == go["iters"] == k
        err = np.linalg.norm(gg["u"].cpu().numpy() - go["u"]) / np.linalg.norm(go["u"])
        assert err <= 1e-12


# ------------------------------------------------------------- error paths
def test_errors_are_reported_not_trapped():
    prob = I.poisson_box(2, 10, 2)
    rp, ci, v = prob.rowptr.copy(), prob.col.copy(), prob.val.copy()
    # unsorted columns
    bad = ci.copy()
    bad[rp[5]], bad[rp[5] + 1] = bad[rp[5] + 1], bad[rp[5]]
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, bad, v)
    assert e.value.code == A.AMG_ERR_ARG
    # column out of range
    bad = ci.copy()
    bad[rp[3]] = prob.n + 5
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, bad, v)
    assert e.value.code == A.AMG_ERR_ARG
    # NaN value
    vv = v.copy()
    vv[7] = np.nan
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, ci, vv)
    assert e.value.code == A.AMG_ERR_NAN
    # zero diagonal
    vv = v.copy()
    for k in range(rp[4], rp[5]):
        if ci[k] == 4:
            vv[k] = 0.0
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, ci, vv)
    assert e.value.code == A.AMG_ERR_NOT_SPD
    # structurally unsymmetric: drop entry (5, j) for its first off-diagonal j, keep (j, 5)
    k_drop = next(k for k in range(rp[5], rp[6]) if ci[k] != 5)
    rp2 = rp.copy()
    rp2[6:] -= 1
    ci2 = np.delete(ci, k_drop)
    v2 = np.delete(v, k_drop)
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp2, ci2, v2, coarse_max=10)
    assert e.value.code == A.AMG_ERR_ARG
    # matching round budget
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, ci, v, max_match_rounds=1, coarse_max=10)
    assert e.value.code == A.AMG_ERR_TIMEOUT
    # coarsest too large for the dense solve
    with pytest.raises(A.AmgError) as e:
        A.Hierarchy(rp, ci, v, dense_max=10, coarse_max=50)
    assert e.value.code == A.AMG_ERR_COARSE_TOO_LARGE
    # NaN right-hand side
    H = A.Hierarchy(rp, ci, v, coarse_max=20)
    F = prob.F.copy()
    F[3] = np.nan
    g = H.solve(gpu(F), rtol=1e-8)
    assert g["status"] == A.AMG_ERR_NAN
    # the hierarchy still works afterwards
    g = H.solve(gpu(prob.F), rtol=1e-8)
    assert g["status"] == 0
    # bad arguments
    with pytest.raises(A.AmgError):
        A.Hierarchy(rp, ci, v, nu_pre=0)
    with pytest.raises(A.AmgError):
        A.Hierarchy(rp, ci, v, match_passes=9)


def test_device_resident_input_and_determinism():
    prob = I.poisson_box(3, 8, 2)
    H1 = A.Hierarchy(gpu(prob.rowptr), gpu(prob.col), gpu(prob.val), coarse_max=20)
    H2 = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    for l in range(H1.num_levels):
        a, b = H1.export_level(l), H2.export_level(l)
        for k in ("rowptr", "col", "val"):
            assert np.array_equal(a[k], b[k])
    r1 = H1.solve(gpu(prob.F), rtol=1e-9)
    r2 = H1.solve(gpu(prob.F), rtol=1e-9)
    assert torch.equal(r1["u"], r2["u"])  # deterministic reductions
