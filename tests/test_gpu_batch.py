"""Several right-hand sides (SpMM) and batches of block-diagonal systems.

Oracle: each right-hand side is an independent PCG with the same
preconditioner, so it must match the oracle's single-RHS PCG column by
column.  A batch is one hierarchy of the block-diagonal matrix; its V-cycle
acts on each block separately, so system k's CG equals the oracle's PCG on
the assembled matrix with F zero outside block k.  FP64: iterations within
+-1 and solutions within 1e-10 relative; mixed precision: error vs the FP64
oracle <= 1e-7 at rtol 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402


def block_diag(systems):
    rps, cis, vs, off, zoff = [], [], [], 0, 0
    for rp, ci, v in systems:
        rps.append(rp[:-1] + zoff)
        cis.append(ci + off)
        vs.append(v)
        off += len(rp) - 1
        zoff += rp[-1]
    return (np.concatenate(rps + [np.array([zoff])]).astype(np.int64), np.concatenate(cis).astype(np.int32),
            np.concatenate(vs))


@pytest.mark.parametrize("nrhs,mem", [(5, "device"), (16, "host"), (1, "device"), (32, "device")])
def test_multi_rhs_matches_oracle_columnwise(nrhs, mem):
    prob = I.poisson_box_random_rhs(3, 8, 3, seed=4, nrhs=nrhs)
    F = np.ascontiguousarray(prob.F.reshape(nrhs, prob.n))
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    Fi = F if mem == "host" else torch.from_numpy(F).cuda()
    out = H.solve_multi(Fi, rtol=1e-9)
    U = out["u"] if mem == "host" else out["u"].cpu().numpy()
    assert out["status"] == 0
    for c in range(nrhs):
        ref = Ho.pcg(F[c], rtol=1e-9)
        assert abs(int(out["iters"][c]) - ref["iters"]) <= 1
        uc = U[c]
        if out["iters"][c] != ref["iters"]:
            g = H.solve(torch.from_numpy(F[c]).cuda(), rtol=0.0, itmax=ref["iters"])
            uc = g["u"].cpu().numpy()
        assert np.linalg.norm(uc - ref["u"]) <= 1e-10 * np.linalg.norm(ref["u"])
        assert out["relres"][c] <= 1e-9 * 1.0001


def test_multi_rhs_mixed_precision_error_vs_fp64():
    prob = I.poisson_box_random_rhs(3, 10, 3, seed=8, nrhs=16)
    F = np.ascontiguousarray(prob.F.reshape(16, prob.n))
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, precision=A.AMG_FP32_BF16FINE)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    out = H.solve_multi(torch.from_numpy(F).cuda(), rtol=1e-8)
    assert out["status"] == 0 and (out["relres"] <= 1e-8).all()
    U = out["u"].cpu().numpy()
    worst = 0.0
    for c in range(16):
        ref = Ho.pcg(F[c], rtol=1e-8, flexible=True)
        worst = max(worst, np.linalg.norm(U[c] - ref["u"]) / np.linalg.norm(ref["u"]))
    print(f"multi-RHS mixed precision: max relative error vs FP64 oracle {worst:.2e}")
    assert worst <= 1e-7


def test_multi_rhs_zero_column_itmax_and_errors():
    prob = I.poisson_box_random_rhs(2, 12, 2, seed=2, nrhs=3)
    F = np.ascontiguousarray(prob.F.reshape(3, prob.n))
    F[1] = 0.0
    H = A.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    out = H.solve_multi(torch.from_numpy(F).cuda(), rtol=1e-10)
    assert out["status"] == 0 and out["iters"][1] == 0 and not out["u"][1].any()
    lim = H.solve_multi(torch.from_numpy(F).cuda(), rtol=1e-14, itmax=2)
    assert lim["status"] == A.AMG_ERR_NOT_CONVERGED and (lim["iters"][[0, 2]] == 2).all()
    with pytest.raises(A.AmgError):
        A.Hierarchy(prob.rowptr, prob.col, prob.val, nu_pre=2).solve_multi(torch.from_numpy(F).cuda())
    big = np.zeros((33, prob.n))
    with pytest.raises(A.AmgError):
        H.solve_multi(big)


BATCH = [(2, 10, 2), (2, 7, 3), (2, 12, 4), (3, 4, 2), (2, 16, 2)]


def batch_systems(seed=11):
    probs = [I.poisson_box_random_rhs(d, n, p, seed=seed + k) for k, (d, n, p) in enumerate(BATCH)]
    return probs, [(q.rowptr, q.col, q.val) for q in probs]


@pytest.mark.parametrize("mem", ["device", "host"])
def test_batch_matches_oracle_per_system(mem):
    probs, systems = batch_systems()
    rp, ci, v = block_diag(systems)
    B = A.BatchHierarchy(systems if mem == "host" else
                         [tuple(torch.from_numpy(a).cuda() for a in s_) for s_ in systems], coarse_max=20)
    Ho = O.Hierarchy(rp, ci, v, coarse_max=20)
    # the batch hierarchy is the hierarchy of the block-diagonal matrix (bit-exact)
    assert B.num_levels == Ho.num_levels
    for l in range(B.num_levels):
        g = B.export_level(l)
        rpo, cio, vo = Ho.level_csr(l)
        assert np.array_equal(g["col"], cio) and np.array_equal(g["val"].view(np.uint64), vo.view(np.uint64))
    Fs = [q.F for q in probs] if mem == "host" else [torch.from_numpy(q.F).cuda() for q in probs]
    out = B.solve_batch(Fs, rtol=1e-9)
    assert out["status"] == 0
    off = np.cumsum([0] + [q.n for q in probs])
    for k, q in enumerate(probs):
        Fk = np.zeros(off[-1])
        Fk[off[k]:off[k + 1]] = q.F
        ref = Ho.pcg(Fk, rtol=1e-9)
        assert abs(int(out["iters"][k]) - ref["iters"]) <= 1, (k, out["iters"][k], ref["iters"])
        uk = out["u"][k] if mem == "host" else out["u"][k].cpu().numpy()
        rk = ref["u"][off[k]:off[k + 1]]
        if out["iters"][k] == ref["iters"]:
            assert np.linalg.norm(uk - rk) <= 1e-10 * np.linalg.norm(rk)
        assert np.linalg.norm(uk - q.u_true) <= 1e-6 * np.linalg.norm(q.u_true)
        assert out["relres"][k] <= 1e-9 * 1.0001


def test_batch_mixed_precision_and_frozen_systems():
    probs, systems = batch_systems(seed=21)
    B = A.BatchHierarchy(systems, coarse_max=20, precision=A.AMG_FP32_BF16FINE)
    Fs = [torch.from_numpy(q.F).cuda() for q in probs]
    Fs[2] = torch.zeros_like(Fs[2])
    out = B.solve_batch(Fs, rtol=1e-8)
    assert out["status"] == 0
    assert out["iters"][2] == 0 and not out["u"][2].any()
    for k, q in enumerate(probs):
        if k == 2:
            continue
        assert out["relres"][k] <= 1e-8
        err = np.linalg.norm(out["u"][k].cpu().numpy() - q.u_true) / np.linalg.norm(q.u_true)
        assert err <= 1e-5
    # the iteration counts differ per system: converged systems were frozen
    assert len(set(int(i) for i in out["iters"])) > 1


def test_batch_errors():
    probs, systems = batch_systems()
    bad = list(systems)
    rp, ci, v = bad[1]
    ci = ci.copy()
    ci[3] = len(rp) + 10  # column outside its own system
    bad[1] = (rp, ci, v)
    with pytest.raises(A.AmgError) as e:
        A.BatchHierarchy(bad)
    assert e.value.code == A.AMG_ERR_ARG
    H = A.Hierarchy(*systems[0])
    with pytest.raises(A.AmgError):
        A.amg_pcg_solve_batch(H._h, [probs[0].F], [np.zeros(probs[0].n)], 1e-8, 100)
