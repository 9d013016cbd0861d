"""Learned smoother damping on the GPU against the oracle (oracle/mpnn.py).

* The damping cap: the Lanczos estimate lam_hat of lambda_max(D^-1 K) per
  level against the oracle's (1e-10 relative).
* omega of the network on every level: FP32 weights and BF16-rounded
  weights, against the oracle's FP64 forward with the same weights
  (|diff| <= 2e-5; omega is in (0, omega_max), omega_max = 2 / lam_hat <
  2.9, and the GPU computes in FP32).
* The installed damping is what the V-cycle runs: GPU V-cycle vs the
  oracle's damped V-cycle with the GPU's omega (1e-12), and restoring the
  plain smoother is bitwise.
* Loss and gradient: the loss with the GPU's omega equals the oracle's
  FP64 loss for that omega (1e-10); against the oracle's end-to-end
  loss/gradient for the same weights, loss 1e-5 and gradient 1e-5 relative
  (FP32 network and FP32 weights; every parameter block 1e-5 of its own
  norm).  Two runs are bitwise identical.
* Adam step against the textbook update; training lowers the loss and the
  PCG iteration count; the fallback rule keeps the reference smoother when
  the learned one is worse.
* Constant damping (amg_set_damping): the V-cycle against the oracle's
  damped V-cycle, omega = 1 restores the plain smoother bit for bit.
* The trained network against the best constant damping of a sweep:
  iterations, spread of omega, no saturation at the cap.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from oracle import mpnn as M  # noqa: E402
from paper_2511_21268_gb300 import amg as A  # noqa: E402
from paper_2511_21268_gb300 import inputs as I  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), as FP32."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def varied_weights(seed):
    """Initial weights with a larger output layer, so omega varies over
    the rows and spans much of (0, 2)."""
    d = M.unpack(I.mpnn_init_weights(seed))
    d["q"] = d["q"] * 20
    d["c"] = np.array([0.3])
    d["b1"] = np.full(M.HIDDEN, 0.05)
    return M.pack(d).astype(np.float32)


CASES = [(2, 32, 3), (3, 10, 3)]  # 3-D rows hold up to 343 entries (several 32-entry chunks)


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "d%d_n%d_p%d" % c)
def case(request):
    d, n, p = request.param
    prob = I.poisson_box(d, n, p)
    Ho = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=50)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=50)
    assert H.num_levels == Ho.num_levels >= 3
    return prob, Ho, H, M.Levels(Ho)


@pytest.mark.parametrize("bf16", [False, True])
def test_omega_matches_oracle(case, bf16):
    prob, Ho, H, lv = case
    w32 = varied_weights(5)
    H.mpnn_apply(dev(w32), bf16_weights=bf16)
    wref = (bf16_round(w32) if bf16 else w32).astype(np.float64)
    spread = 0.0
    for l in range(H.num_levels - 1):
        om = H.mpnn_omega(l).cpu().numpy().astype(np.float64)
        ref, _ = M.forward(wref, *M.features(*lv.csr[l]), lv.omax[l])
        assert np.max(np.abs(om - ref)) <= 2e-5, (l, np.max(np.abs(om - ref)))
        spread = max(spread, ref.max() - ref.min())
    assert spread > 0.1
    H.mpnn_apply(None)


def test_damped_vcycle_matches_oracle_and_restore_is_bitwise(case):
    prob, Ho, H, lv = case
    r = np.random.default_rng(3).standard_normal(prob.n)
    z_plain = H.vcycle(dev(r)).cpu().numpy()
    H.mpnn_apply(dev(varied_weights(7)), bf16_weights=True)
    omegas = [H.mpnn_omega(l).cpu().numpy().astype(np.float64) for l in range(H.num_levels - 1)]
    omegas.append(np.ones(H.level_n(H.num_levels - 1)))
    z = H.vcycle(dev(r)).cpu().numpy()
    zo = M.vcycle_omega(lv, omegas, r)
    assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    assert np.linalg.norm(z - z_plain) > 1e-3 * np.linalg.norm(z_plain)
    H.mpnn_apply(None)
    z_back = H.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(z_back.view(np.uint64), z_plain.view(np.uint64))


def test_loss_and_gradient_match_oracle(case):
    prob, Ho, H, lv = case
    w32 = varied_weights(11)
    loss, g = H.mpnn_loss_grad(dev(w32), nprobe=3, seed=11)
    g = g.cpu().numpy()
    # the V-cycle part in FP64: the oracle's loss for the GPU's omega
    omegas = [H.mpnn_omega(l).cpu().numpy().astype(np.float64) for l in range(H.num_levels - 1)]
    omegas.append(np.ones(H.level_n(H.num_levels - 1)))
    lo, _ = M.loss_and_domega(lv, omegas, M.probes(11, 3, prob.n))
    assert abs(loss - lo) <= 1e-10 * abs(lo)
    # end to end, FP64 oracle with the same weights
    L_ref, g_ref, _ = M.loss_and_grad(Ho, w32.astype(np.float64), nprobe=3, seed=11)
    assert abs(loss - L_ref) <= 1e-5 * abs(L_ref)
    err = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    print(f"N={prob.n}: loss {loss:.6f} (oracle {L_ref:.6f}), gradient relative error {err:.2e}")
    assert err <= 1e-5
    # every parameter block receives its gradient
    for name, blk in M.unpack(g_ref).items():
        gb = M.unpack(g)[name]
        assert np.linalg.norm(gb - blk) <= 1e-5 * np.linalg.norm(blk) + 1e-7 * np.linalg.norm(g_ref), name
    loss2, g2 = H.mpnn_loss_grad(dev(w32), nprobe=3, seed=11)
    assert loss2 == loss and np.array_equal(g2.cpu().numpy(), g)


def test_smoother_bound_matches_oracle(case):
    prob, Ho, H, lv = case
    for l in range(H.num_levels - 1):
        lam = H.smoother_bound(l)
        assert abs(2.0 / lam - lv.omax[l]) <= 1e-10 * lv.omax[l], (l, 2.0 / lam, lv.omax[l])
        assert 0.6 < lam <= 1.0


def test_constant_damping_matches_oracle_and_one_is_plain(case):
    prob, Ho, H, lv = case
    r = np.random.default_rng(4).standard_normal(prob.n)
    z_plain = H.vcycle(dev(r)).cpu().numpy()
    for om in (1.7, 2.2):
        H.set_damping(om)
        z = H.vcycle(dev(r)).cpu().numpy()
        zo = M.vcycle_omega(lv, [np.full(lv.K[l].shape[0], om) for l in range(lv.L)], r)
        assert np.linalg.norm(z - zo) <= 1e-12 * np.linalg.norm(zo)
    H.set_damping(1.0)
    z_back = H.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(z_back.view(np.uint64), z_plain.view(np.uint64))
    with pytest.raises(A.AmgError):
        H.set_damping(0.0)


def test_adam_step_matches_textbook():
    prob = I.poisson_box(2, 16, 2)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=20)
    rng = np.random.default_rng(0)
    w = rng.standard_normal(A.AMG_MPNN_NPARAM).astype(np.float32)
    m = (rng.standard_normal(A.AMG_MPNN_NPARAM) * 0.1).astype(np.float32)
    v = (rng.random(A.AMG_MPNN_NPARAM) * 0.01).astype(np.float32)
    g = rng.standard_normal(A.AMG_MPNN_NPARAM)
    wd, md, vd, gd = dev(w), dev(m), dev(v), dev(g)
    A.amg_mpnn_adam(H._h, wd, gd, md, vd, 3, 1e-2)
    # the kernel's constants are FP32: 1 - beta2 = 1 - fl32(0.999) differs
    # from 0.001 by 1.3e-5 relative, so the reference uses the same values
    f = np.float32
    b1, b2 = float(f(0.9)), float(f(0.999))
    c1, c2 = float(f(1) - f(b1)), float(f(1) - f(b2))
    m1 = b1 * m + c1 * g
    v1 = b2 * v + c2 * g * g
    w1 = w - 1e-2 * (m1 / (1 - b1 ** 3)) / (np.sqrt(v1 / (1 - b2 ** 3)) + 1e-8)
    assert np.allclose(md.cpu().numpy(), m1, rtol=1e-5, atol=1e-7)
    assert np.allclose(vd.cpu().numpy(), v1, rtol=1e-5, atol=1e-9)
    assert np.allclose(wd.cpu().numpy(), w1, rtol=1e-5, atol=1e-6)


def test_training_reduces_loss_and_iterations():
    prob = I.poisson_box(2, 32, 3)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=50)
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    hist = H.mpnn_train(w, steps=40, nprobe=4, seed=1000, lr=1e-2)
    assert np.all(np.isfinite(hist))
    assert hist[-10:].mean() < hist[0] - 0.5
    used, ip, il = H.mpnn_select(w, dev(prob.F), rtol=1e-8)
    print(f"2-D p=3 n=32: loss {hist[0]:.3f} -> {hist[-1]:.3f}; PCG iterations plain {ip}, learned {il}")
    assert used and il <= 0.9 * ip
    g = H.solve(dev(prob.F), rtol=1e-8)
    assert g["status"] == 0 and g["iters"] == il
    K = sp.csr_matrix((prob.val, prob.col, prob.rowptr))
    u = g["u"].cpu().numpy()
    assert np.linalg.norm(prob.F - K @ u) <= 1e-8 * 1.0001 * np.linalg.norm(prob.F)


def test_fallback_keeps_plain_smoother_when_learned_is_worse():
    prob = I.poisson_box(2, 32, 3)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val), coarse_max=50)
    r = np.random.default_rng(1).standard_normal(prob.n)
    z_plain = H.vcycle(dev(r)).cpu().numpy()
    d = M.unpack(I.mpnn_init_weights(2))
    d["c"] = np.array([-6.0])  # omega about 0.005: a very weak smoother
    used, ip, il = H.mpnn_select(dev(M.pack(d).astype(np.float32)), dev(prob.F), rtol=1e-8, itmax=2000)
    assert not used and il > ip
    z = H.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(z.view(np.uint64), z_plain.view(np.uint64))
    # against a constant reference damping: that damping stays installed
    used, ic, il = H.mpnn_select(dev(M.pack(d).astype(np.float32)), dev(prob.F), rtol=1e-8, itmax=2000,
                                 omega_ref=1.8)
    assert not used and ic < ip
    H.set_damping(1.8)
    z18 = H.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(H.vcycle(dev(r)).cpu().numpy().view(np.uint64), z18.view(np.uint64))


@pytest.mark.parametrize("prec", [A.AMG_FP32, A.AMG_FP32_BF16FINE])
def test_learned_damping_in_mixed_precision(prec):
    prob = I.poisson_box(3, 16, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    A.Hierarchy(*args).mpnn_train(w, steps=30, nprobe=4, seed=500, lr=1e-2)
    H = A.Hierarchy(*args, precision=prec)
    plain = H.solve(dev(prob.F), rtol=1e-8)
    H.mpnn_apply(w, bf16_weights=True)
    g = H.solve(dev(prob.F), rtol=1e-8)
    K = sp.csr_matrix((prob.val, prob.col, prob.rowptr))
    u = g["u"].cpu().numpy()
    print(f"3-D p=3 n=16 precision {prec}: iterations plain {plain['iters']}, learned {g['iters']}")
    assert g["status"] == 0 and g["iters"] < plain["iters"]
    assert np.linalg.norm(prob.F - K @ u) <= 1e-8 * 1.0001 * np.linalg.norm(prob.F)


def test_training_over_several_hierarchies_uses_the_mean_loss():
    probs = [I.poisson_box(2, 16, 3), I.poisson_box(2, 24, 2)]
    Hs = [A.Hierarchy(dev(q.rowptr), dev(q.col), dev(q.val), coarse_max=20) for q in probs]
    w0 = I.mpnn_init_weights(4).astype(np.float32)
    losses, grads = zip(*[H.mpnn_loss_grad(dev(w0), nprobe=2, seed=77) for H in Hs])
    w = dev(w0)
    hist = Hs[0].mpnn_train(w, steps=1, nprobe=2, seed=77, lr=1e-3, others=Hs[1:])
    assert abs(hist[0] - 0.5 * (losses[0] + losses[1])) <= 1e-14 * abs(hist[0])
    # first Adam step: w - lr g / (|g| + eps) elementwise (bias-corrected moments)
    g = 0.5 * (grads[0].cpu().numpy() + grads[1].cpu().numpy())
    f = np.float32
    c1, c2 = float(f(1) - f(0.9)), float(f(1) - f(0.999))
    mh = c1 * g / (1 - float(f(0.9)))
    vh = c2 * g * g / (1 - float(f(0.999)))
    expect = w0 - 1e-3 * mh / (np.sqrt(vh) + 1e-8)
    assert np.allclose(w.cpu().numpy(), expect, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("prec,bf16", [(A.AMG_FP64, False), (A.AMG_FP32_BF16FINE, True)])
def test_weights_at_setup_install_the_apply_damping_bit_for_bit(prec, bf16):
    """Setup given the network weights (the finest level's network running on
    a second stream alongside the coarse-level setup) installs exactly the
    damping that amg_mpnn_apply installs after a plain setup: omega, the
    V-cycle and the solve are bitwise equal, and w = NULL restores the plain
    smoother bit for bit."""
    prob = I.poisson_box(3, 14, 3)
    args = (dev(prob.rowptr), dev(prob.col), dev(prob.val))
    w = dev(varied_weights(9))
    H1 = A.Hierarchy(*args, coarse_max=50, precision=prec)
    r = np.random.default_rng(21).standard_normal(prob.n)
    z_plain = H1.vcycle(dev(r)).cpu().numpy()
    H1.mpnn_apply(w, bf16_weights=bf16)
    H2 = A.Hierarchy(*args, coarse_max=50, precision=prec, mpnn_weights=w, mpnn_bf16=int(bf16))
    assert H2.num_levels == H1.num_levels >= 3
    assert H2.info.setup_phase_ms[9] > 0
    for l in range(H1.num_levels - 1):
        o1, o2 = H1.mpnn_omega(l).cpu().numpy(), H2.mpnn_omega(l).cpu().numpy()
        assert np.array_equal(o1.view(np.uint32), o2.view(np.uint32)), l
    z1, z2 = H1.vcycle(dev(r)).cpu().numpy(), H2.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(z1.view(np.uint64), z2.view(np.uint64))
    assert np.linalg.norm(z2 - z_plain) > 1e-3 * np.linalg.norm(z_plain)
    g1, g2 = H1.solve(dev(prob.F), rtol=1e-8), H2.solve(dev(prob.F), rtol=1e-8)
    assert g2["status"] == 0 and g1["iters"] == g2["iters"]
    assert np.array_equal(g1["u"].cpu().numpy().view(np.uint64), g2["u"].cpu().numpy().view(np.uint64))
    H2.mpnn_apply(None)
    z_back = H2.vcycle(dev(r)).cpu().numpy()
    assert np.array_equal(z_back.view(np.uint64), z_plain.view(np.uint64))
    with pytest.raises(A.AmgError):
        A.Hierarchy(*args, coarse_max=50, mpnn_weights=w, mpnn_bf16=2)



def test_trained_network_against_the_best_constant_damping():
    """The question the learned part has to answer: does a per-row damping
    beat the best single damping value?  Train on 3-D cubes p in {2, 3, 4},
    n = 10 (FP64 hierarchies), then on a 3-D p=3 n=16 cube compare PCG
    iterations with the network against a sweep of constants.  The trained
    omega must vary over the rows (rows may sit at the level's cap 2 /
    lam_hat, the edge of the range where the smoother is guaranteed to
    converge, but not all of them); the fallback rule against the best
    constant keeps whichever is better, so the installed smoother is never
    worse than that constant."""
    train = []
    for pp in (2, 3, 4):
        q = I.poisson_box(3, 10, pp)
        train.append(A.Hierarchy(dev(q.rowptr), dev(q.col), dev(q.val)))
    w = dev(I.mpnn_init_weights(1).astype(np.float32))
    hist = train[0].mpnn_train(w, steps=60, nprobe=4, seed=1000, lr=1e-2, others=train[1:])
    assert hist[-10:].mean() < hist[0] - 0.3
    prob = I.poisson_box(3, 16, 3)
    H = A.Hierarchy(dev(prob.rowptr), dev(prob.col), dev(prob.val))
    F = dev(prob.F)
    its = {}
    for om in (1.0, 1.5, 1.8, 2.0, 2.2, 2.4):
        H.set_damping(om)
        g = H.solve(F, rtol=1e-8, itmax=2000)
        if g["status"] == 0:
            its[om] = g["iters"]
    best = min(its, key=lambda o: (its[o], o))
    H.mpnn_apply(w, bf16_weights=True)
    g = H.solve(F, rtol=1e-8)
    assert g["status"] == 0
    stats = []
    for l in range(H.num_levels - 1):
        om = H.mpnn_omega(l).cpu().numpy()
        omax = 2.0 / H.smoother_bound(l)
        at_cap = float(np.mean(om >= 0.999 * omax))
        stats.append((l, om.min(), om.max(), om.std(), omax, at_cap))
        assert at_cap < 0.95
    print("constant sweep", its, "best", best, "learned", g["iters"],
          "omega per level (min, max, std, cap, fraction at the cap)",
          [tuple(round(float(x), 3) for x in s_) for s_ in stats])
    assert stats[0][3] > 1e-2  # omega varies over the rows of the finest level
    assert g["iters"] < its[1.0]
    used, ic, il = H.mpnn_select(w, F, rtol=1e-8, omega_ref=best)
    assert ic == its[best] and il == g["iters"]
    assert used == (il <= ic)
    final = H.solve(F, rtol=1e-8)
    assert final["iters"] == min(il, ic)
