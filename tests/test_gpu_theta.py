"""Learned prolongator-smoothing weights theta (the network's second head)
on the GPU against the oracle (oracle/mpnn.py), through the C ABI.

* theta of the second head on level 0 against the oracle's FP64 forward
  (|diff| <= 2e-5 with FP32 weights; theta in (0, omega_max)).
* The two-grid loss of the smoothing weights and its gradient with respect
  to the weights on two-level hierarchies with a smoothed level 0: loss and
  gradient within 1e-5 relative of the oracle's (FP32 network).
* A setup given the weights and smooth_levels = 1 smooths level 0 with the
  network's theta: its P_bar and coarse matrix are bit for bit the oracle's
  for that theta.
* Training on theta hierarchies lowers the two-grid loss; the learned
  weights against the constant 4/3 and the tentative prolongator in PCG
  iterations (printed).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from oracle import mpnn as M  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def theta_weights(seed):
    d = M.unpack(I.mpnn_init_weights(seed))
    d["qt"] = d["qt"] * 10
    d["b2"] = np.full(M.HIDDEN, 0.05)
    return M.pack(d).astype(np.float32)


CASES = [(2, 12, 3), (3, 6, 2)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "d%d_n%d_p%d" % c)
def case(request):
    d, n, p = request.param
    prob = I.poisson_box(d, n, p)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=20, smooth_levels=1, max_levels=2)
    assert H.num_levels == 2 and H.info.smoothed[0] == 1
    return prob, Ho, H, M.TwoGrid(Ho)


def test_theta_head_and_twogrid_loss_match_oracle(case):
    prob, Ho, H, tg = case
    w32 = theta_weights(3)
    loss, g = H.mpnn_theta_loss_grad(dev(w32), nprobe=3, seed=17)
    g = g.cpu().numpy()
    th = H.mpnn_theta().cpu().numpy().astype(np.float64)
    L_ref, g_ref, th_ref = M.theta_loss_and_grad(tg, w32.astype(np.float64), nprobe=3, seed=17)
    assert np.max(np.abs(th - th_ref)) <= 2e-5
    assert th.std() > 1e-3 and 0 < th.min() and th.max() < tg.omax
    assert abs(loss - L_ref) <= 1e-5 * abs(L_ref)
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print(f"N={prob.n}: theta loss {loss:.6f} (oracle {L_ref:.6f}), gradient relative error {err:.2e}")
    assert err <= 1e-5
    for name, blk in M.unpack(g_ref).items():
        if name in ("q", "c"):
            assert np.all(M.unpack(g)[name] == 0)  # omega is held fixed in this loss
            continue
        assert np.linalg.norm(M.unpack(g)[name] - blk) <= 1e-5 * np.linalg.norm(blk) + 1e-7 * np.linalg.norm(g_ref)
    # the network's theta is installed: P_bar and K_c are the oracle's for it
    Hs = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, smooth_levels=1, max_levels=2, theta0=th)
    grp, gci, gv = H.export_prolongator(0)
    assert np.array_equal(bits(gv), bits(Hs.prolongator(0)[2]))
    assert np.array_equal(bits(H.export_level(1)["val"]), bits(Hs.level_csr(1)[2]))


def test_setup_with_weights_smooths_level0_with_the_network_theta():
    prob = I.poisson_box(3, 8, 3)
    w = dev(theta_weights(5))
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=30, smooth_levels=1,
                    mpnn_weights=w, mpnn_bf16=1)
    th = H.mpnn_theta().cpu().numpy().astype(np.float64)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30, smooth_levels=1, theta0=th)
    assert H.num_levels == Ho.num_levels
    assert np.array_equal(bits(H.export_prolongator(0)[2]), bits(Ho.prolongator(0)[2]))
    for l in range(H.num_levels):
        assert np.array_equal(bits(H.export_level(l)["val"]), bits(Ho.level_csr(l)[2]))
    g = H.solve(dev(prob.F), rtol=1e-8)
    assert g["status"] == 0


def test_training_theta_lowers_loss_and_compare_iterations():
    """Joint training on damping hierarchies (V-cycle loss of omega) and
    two-level smoothed hierarchies (two-grid loss of theta); then PCG on a
    3-D p=3 n=12 cube with the learned theta against theta = 4/3 and the
    tentative prolongator (plain smoother in all three)."""
    dmp, sm = [], []
    for pp in (2, 3, 4):
        q = I.poisson_box(3, 8, pp)
        args = (dev(q.rowptr), dev(q.col), dev(q.val))
        dmp.append(A.Hierarchy(*args))
        sm.append(A.Hierarchy(*args, smooth_levels=1, max_levels=2, coarse_max=20))
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    l0 = [h.mpnn_theta_loss_grad(w, nprobe=4, seed=500)[0] for h in sm]
    hist = dmp[0].mpnn_train(w, steps=40, nprobe=4, seed=1000, lr=1e-2, others=dmp[1:] + sm)
    assert np.all(np.isfinite(hist))
    l1 = [h.mpnn_theta_loss_grad(w, nprobe=4, seed=500)[0] for h in sm]
    print("two-grid theta loss before/after training", np.round(l0, 4), np.round(l1, 4))
    assert np.mean(l1) < np.mean(l0)
    prob = I.poisson_box(3, 12, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    F = dev(prob.F)
    it_t = A.Hierarchy(*args).solve(F, rtol=1e-8)["iters"]
    it_c = A.Hierarchy(*args, smooth_levels=1).solve(F, rtol=1e-8)["iters"]
    Hl = A.Hierarchy(*args, smooth_levels=1, mpnn_weights=w, mpnn_bf16=1)
    Hl.mpnn_apply(None)  # plain smoother: compare the prolongators alone
    gl = Hl.solve(F, rtol=1e-8)
    th = Hl.mpnn_theta().cpu().numpy()
    print(f"3-D p=3 n=12 PCG iterations: tentative P {it_t}, theta 4/3 {it_c}, learned theta {gl['iters']} "
          f"(theta [{th.min():.3f}, {th.max():.3f}], std {th.std():.3f}; OPC {Hl.info.opc:.3f})")
    assert gl["status"] == 0 and gl["iters"] <= it_t
