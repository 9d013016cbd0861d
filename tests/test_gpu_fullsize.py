"""Full-size checks on the workloads' own sizes, in the configuration bench.py
times (device-resident inputs, default options).

* 3-D Poisson p=3 n=64 (N=274,625, 86.9 M nonzeros), FP64: the whole
  hierarchy bit-exact against the oracle, the V-cycle within 1e-12, and the
  complete PCG solve at rtol 1e-8 against the oracle's (iterations +-1,
  solution 1e-10).
* Precision sweep p = 2/3/4 at n = 96/64/48: the GPU FP64 solve against
  the oracle's FP64 solve of the same system (iterations +-1, 1e-10); the
  mixed-precision solves reach the FP64 true residual 1e-8 (recomputed here
  with scipy) and stay within 1e-7 of the oracle's solution; the errors
  are printed.  The oracle's solve runs its row loops on all host cores
  (results independent of the thread count).
* The 48-system batch of 2-D problems (p in {2,3,4}, n in 32..256, seeded)
  and 16 right-hand sides on 3-D p=3 n=48: every system's true residual
  (scipy) meets rtol 1e-8; one right-hand side is compared with the oracle.
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


def true_relres(prob_or_csr, F, u):
    rp, ci, v = prob_or_csr
    K = sp.csr_matrix((v, ci, rp), shape=(len(rp) - 1,) * 2)
    return np.linalg.norm(F - K @ u) / np.linalg.norm(F)


@pytest.fixture(scope="module")
def cube64():
    prob = I.poisson_box(3, 64, 3)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    return prob, Ho


def test_fullsize_fp64_hierarchy_bit_exact(cube64):
    prob, Ho = cube64
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val))
    assert H.num_levels == Ho.num_levels
    for l in range(H.num_levels):
        g = H.export_level(l)
        rp, ci, v = Ho.level_csr(l)
        assert np.array_equal(g["rowptr"], rp) and np.array_equal(g["col"], ci)
        assert np.array_equal(g["val"].view(np.uint64), v.view(np.uint64))
        d, w = Ho.level_vectors(l)  # l1 diagonal and test vector (the wide-level folds)
        assert np.array_equal(g["dl1"].view(np.uint64), d.view(np.uint64))
        if g["w"] is not None:
            assert np.array_equal(g["w"].view(np.uint64), w.view(np.uint64))
        if l < H.num_levels - 1:
            agg, pv = Ho.level_map(l)
            assert np.array_equal(g["agg"], agg) and np.array_equal(g["pval"].view(np.uint64), pv.view(np.uint64))
    r = np.random.default_rng(5).standard_normal(prob.n)
    z = H.vcycle(dev(r)).cpu().numpy()
    zo = Ho.vcycle(r)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)


def test_fullsize_fp64_solve_matches_oracle(cube64):
    prob, Ho = cube64
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val))
    g = H.solve(dev(prob.F), rtol=1e-8)
    ref = Ho.pcg(prob.F, rtol=1e-8)
    assert g["status"] == 0 and ref["status"] == 0
    assert abs(g["iters"] - ref["iters"]) <= 1
    u = g["u"].cpu().numpy()
    if g["iters"] != ref["iters"]:
        u = H.solve(dev(prob.F), rtol=0.0, itmax=ref["iters"])["u"].cpu().numpy()
    assert np.linalg.norm(u - ref["u"]) <= 1e-10 * np.linalg.norm(ref["u"])
    assert true_relres((prob.rowptr, prob.col, prob.val), prob.F, g["u"].cpu().numpy()) <= 1e-8 * 1.0001


@pytest.mark.parametrize("p,n", [(2, 96), (3, 64), (4, 48)])
def test_fullsize_precision_sweep(p, n):
    import os

    prob = I.poisson_box(3, n, p)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    F = dev(prob.F)
    O.set_threads(os.cpu_count() or 1)
    try:
        oref = O.Hierarchy(prob.rowptr, prob.col, prob.val).pcg(prob.F, rtol=1e-8)
    finally:
        O.set_threads(1)
    assert oref["status"] == 0
    uo = oref["u"]
    ref = A.Hierarchy(*args).solve(F, rtol=1e-8)
    assert ref["status"] == 0 and abs(ref["iters"] - oref["iters"]) <= 1
    u64 = ref["u"].cpu().numpy()
    if ref["iters"] != oref["iters"]:
        u64 = A.Hierarchy(*args).solve(F, rtol=0.0, itmax=oref["iters"])["u"].cpu().numpy()
    assert np.linalg.norm(u64 - uo) <= 1e-10 * np.linalg.norm(uo)
    for prec, name in [(A.AMG_FP32, "fp32"), (A.AMG_FP32_BF16FINE, "bf16-fine")]:
        g = A.Hierarchy(*args, precision=prec).solve(F, rtol=1e-8)
        assert g["status"] == 0
        u = g["u"].cpu().numpy()
        rr = true_relres((prob.rowptr, prob.col, prob.val), prob.F, u)
        err = np.linalg.norm(u - uo) / np.linalg.norm(uo)
        print(f"p={p} n={n} N={prob.n} {name}: iters {g['iters']} (fp64 {ref['iters']}, oracle {oref['iters']}), "
              f"true relres {rr:.2e}, error vs the FP64 oracle {err:.2e}")
        assert rr <= 1e-8 * 1.0001
        assert err <= 1e-7


def test_fullsize_batch_of_48():
    probs = I.batch_instances(seed=20251126, count=48)
    systems = [(dev(q.rowptr), dev(q.col), dev(q.val)) for q in probs]
    B = A.BatchHierarchy(systems, precision=A.AMG_FP32)
    out = B.solve_batch([dev(q.F) for q in probs], rtol=1e-8)
    assert out["status"] == 0
    worst = 0.0
    for k, q in enumerate(probs):
        u = out["u"][k].cpu().numpy()
        rr = true_relres((q.rowptr, q.col, q.val), q.F, u)
        worst = max(worst, rr)
        assert rr <= 1e-8 * 1.0001, (k, rr)
    print(f"48-system batch: N={sum(q.n for q in probs)}, iterations {int(out['iters'].min())}.."
          f"{int(out['iters'].max())}, worst true relres {worst:.2e}")


def test_fullsize_sixteen_rhs():
    prob = I.poisson_box_random_rhs(3, 48, 3, seed=16, nrhs=16)
    F = np.ascontiguousarray(prob.F.reshape(16, prob.n))
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), precision=A.AMG_FP32)
    out = H.solve_multi(dev(F), rtol=1e-8)
    assert out["status"] == 0
    U = out["u"].cpu().numpy()
    for c in range(16):
        assert true_relres((prob.rowptr, prob.col, prob.val), F[c], U[c]) <= 1e-8 * 1.0001
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    ref = Ho.pcg(F[0], rtol=1e-8, flexible=True)
    err = np.linalg.norm(U[0] - ref["u"]) / np.linalg.norm(ref["u"])
    print(f"16 RHS, 3-D p=3 n=48: iterations {out['iters'].tolist()}, column 0 error vs FP64 oracle {err:.2e}")
    assert err <= 1e-7


def _oracle_omega_at(prob, rows, w64):
    """Oracle omega of level 0 at a few rows, from the sub-matrix on their
    3-hop neighbourhood (the network reads 2 hops; the third keeps every
    needed row complete), with the level's damping cap from the oracle's
    Lanczos estimate on the whole matrix.  Returns (omega, omega_max)."""
    from oracle import mpnn as M

    K = sp.csr_matrix((prob.val, prob.col, prob.rowptr), shape=(prob.n, prob.n))
    d, rc = O.l1_diag(prob.rowptr, prob.col, prob.val)
    assert rc == 0
    omax = 2.0 / M.lanczos_bound(K, d, seed=M.LANCZOS_SEED)
    S = np.asarray(rows)
    ring = S
    for _ in range(3):
        ring = np.unique(np.concatenate([ring, K[ring].indices]))
    sub = K[ring][:, ring].tocsr()
    sub.sort_indices()
    om, _ = M.forward(w64, *M.features(sub.indptr.astype(np.int64), sub.indices.astype(np.int32), sub.data), omax)
    return om[np.searchsorted(ring, S)], omax


def test_fullsize_learned_damping_mixed_precision(cube64):
    """Network trained on 3-D p in {2,3,4} n=16 cubes, applied to the 3-D p=3
    n=64 workload: omega at sampled rows against the oracle (BF16 weights),
    then the mixed-precision learned solve meets rtol 1e-8 (true FP64
    residual), stays within 1e-7 of the FP64 solution and needs fewer
    iterations than the plain mixed-precision solve."""
    prob, Ho = cube64
    train = []
    for pp in (2, 3, 4):
        q = I.poisson_box(3, 16, pp)
        train.append(A.Hierarchy(dev(q.rowptr), dev(q.col), dev(q.val)))
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    hist = train[0].mpnn_train(w, steps=60, nprobe=4, seed=1000, lr=1e-2, others=train[1:])
    assert hist[-10:].mean() < hist[0]
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    F = dev(prob.F)
    u64 = A.Hierarchy(*args).solve(F, rtol=1e-8)["u"].cpu().numpy()
    H = A.Hierarchy(*args, precision=A.AMG_FP32_BF16FINE)
    plain = H.solve(F, rtol=1e-8)
    H.mpnn_apply(w, bf16_weights=True)
    om = H.mpnn_omega(0).cpu().numpy().astype(np.float64)
    rows = np.random.default_rng(9).choice(prob.n, 5, replace=False)
    rows = np.sort(np.concatenate([rows, [0, prob.n // 2]]))

    def bf16(a):
        b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
        return ((((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16).astype(np.uint32)).view(np.float32)

    ref, omax = _oracle_omega_at(prob, rows, bf16(w.cpu().numpy()).astype(np.float64))
    assert abs(2.0 / H.smoother_bound(0) - omax) <= 1e-10 * omax
    assert np.max(np.abs(om[rows] - ref)) <= 2e-5
    g = H.solve(F, rtol=1e-8)
    assert g["status"] == 0
    u = g["u"].cpu().numpy()
    rr = true_relres((prob.rowptr, prob.col, prob.val), prob.F, u)
    err = np.linalg.norm(u - u64) / np.linalg.norm(u64)
    print(f"learned + mixed, 3-D p=3 n=64: iterations {g['iters']} (plain mixed {plain['iters']}), "
          f"true relres {rr:.2e}, error vs FP64 {err:.2e}, omega mean {om.mean():.3f} std {om.std():.3f} "
          f"[{om.min():.3f}, {om.max():.3f}], cap {omax:.3f}, at the cap {np.mean(om >= 0.999 * omax):.2f}")
    # rows may sit at the cap (the interior), but omega varies over the rows
    assert om.std() > 0.02 and np.mean(om >= 0.999 * omax) < 0.95
    assert rr <= 1e-8 * 1.0001 and err <= 1e-7
    assert g["iters"] < plain["iters"]


def test_fullsize_annulus_learned_mixed_precision():
    """The learned-damping workload: quarter annulus (NURBS geometry) p=3
    n=64 with a random log-normal coefficient.  Network trained on annulus
    hierarchies p in {2,3,4}, n in {16,32} with four other coefficient
    fields each; the mixed-precision learned
    solve meets rtol 1e-8 on the FP64 true residual, stays within 1e-7 of
    the FP64 solution and needs fewer iterations than plain FP64 AMG."""
    prob = I.annulus_kappa(64, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    F = dev(prob.F)
    train = []  # p in {2,3,4} x n in {16,32} x 4 coefficient fields (not the evaluated one, seed 7)
    for n in (16, 32):
        for pp in (2, 3, 4):
            for ks in (101, 102, 103, 104):
                q = I.annulus_kappa(n, pp, kappa_seed=ks)
                train.append(A.Hierarchy(dev(q.rowptr), dev(q.col), dev(q.val)))
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    hist = train[0].mpnn_train(w, steps=60, nprobe=4, seed=2000, lr=1e-2, others=train[1:])
    ref = A.Hierarchy(*args).solve(F, rtol=1e-8)
    assert ref["status"] == 0
    u64 = ref["u"].cpu().numpy()
    H = A.Hierarchy(*args, precision=A.AMG_FP32_BF16FINE)
    H.mpnn_apply(w, bf16_weights=True)
    g = H.solve(F, rtol=1e-8)
    assert g["status"] == 0
    u = g["u"].cpu().numpy()
    rr = true_relres((prob.rowptr, prob.col, prob.val), prob.F, u)
    err = np.linalg.norm(u - u64) / np.linalg.norm(u64)
    om = H.mpnn_omega(0).cpu().numpy()
    print(f"annulus p=3 n=64: FP64 plain {ref['iters']} iterations, mixed + learned {g['iters']}; true relres "
          f"{rr:.2e}, error vs FP64 {err:.2e}; loss {hist[0]:.3f} -> {hist[-1]:.3f}; omega [{om.min():.3f}, "
          f"{om.max():.3f}]")
    assert rr <= 1e-8 * 1.0001 and err <= 1e-7
    assert g["iters"] < ref["iters"]
