"""Pins for the learned-damping oracle (oracle/mpnn.py).

Independent checks: central finite differences of the loss (w.r.t. the
per-row damping and w.r.t. the network weights), reduction to the C
oracle's plain V-cycle when omega = 1, symmetry of the damped V-cycle,
scale invariance and permutation equivariance of the network.
"""
import numpy as np
import pytest

import oracle as O
from oracle import mpnn as M
from paper_2511_21268_gb300 import inputs as I


@pytest.fixture(scope="module")
def small():
    prob = I.poisson_box(2, 10, 3)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    return prob, H, M.Levels(H)


def unit_omega_weights():
    d = M.unpack(M.init_weights(3))
    d["q"] = np.zeros(M.HIDDEN)
    d["c"] = np.zeros(1)  # 2 sigmoid(0) = 1
    return M.pack(d)


def test_nparam_and_layout():
    assert M.NPARAM == 4386
    w = M.init_weights(2)
    assert np.array_equal(M.pack(M.unpack(w)), w)


def test_unit_omega_reduces_to_plain_vcycle(small):
    prob, H, lv = small
    w = unit_omega_weights()
    omegas = [M.forward(w, *M.features(*lv.csr[l]))[0] for l in range(lv.L)]
    assert all(np.allclose(o, 1.0, rtol=0, atol=1e-15) for o in omegas)
    r = np.random.default_rng(0).standard_normal(prob.n)
    z = M.vcycle_omega(lv, omegas, r)
    assert np.linalg.norm(z - H.vcycle(r)) <= 1e-13 * np.linalg.norm(z)


def test_damped_vcycle_symmetric(small):
    prob, H, lv = small
    rng = np.random.default_rng(1)
    omegas = [rng.uniform(0.2, 1.9, lv.K[l].shape[0]) for l in range(lv.L)]
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    bx, by = M.vcycle_omega(lv, omegas, x), M.vcycle_omega(lv, omegas, y)
    assert abs(x @ by - y @ bx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(bx)
    assert x @ bx > 0


def test_loss_gradient_wrt_omega_finite_differences(small):
    prob, H, lv = small
    rng = np.random.default_rng(2)
    omegas = [rng.uniform(0.5, 1.8, lv.K[l].shape[0]) for l in range(lv.L)]
    X = M.probes(7, 3, prob.n)
    L0, g = M.loss_and_domega(lv, omegas, X)
    dirs = [rng.standard_normal(len(o)) for o in omegas]
    h = 1e-6
    Lp, _ = M.loss_and_domega(lv, [o + h * d for o, d in zip(omegas, dirs)], X)
    Lm, _ = M.loss_and_domega(lv, [o - h * d for o, d in zip(omegas, dirs)], X)
    fd = (Lp - Lm) / (2 * h)
    an = sum(gl @ dl for gl, dl in zip(g, dirs))
    assert abs(fd - an) <= 1e-6 * abs(an)
    assert L0 < 0  # the V-cycle reduces the error


def test_loss_gradient_wrt_weights_finite_differences(small):
    prob, H, lv = small
    w = M.init_weights(5)
    d = M.unpack(w)
    d["c"] = np.array([0.3])
    d["b1"] = np.full(M.HIDDEN, 0.05)
    w = M.pack(d)
    L0, g, _ = M.loss_and_grad(H, w, nprobe=2, seed=11)
    rng = np.random.default_rng(3)
    for _ in range(3):
        v = rng.standard_normal(M.NPARAM)
        h = 1e-6
        Lp, _, _ = M.loss_and_grad(H, w + h * v, nprobe=2, seed=11)
        Lm, _, _ = M.loss_and_grad(H, w - h * v, nprobe=2, seed=11)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g @ v) <= 1e-5 * max(abs(fd), 1e-8), (fd, g @ v)


def test_network_scale_invariance_and_permutation_equivariance(small):
    prob, H, lv = small
    w = M.init_weights(9)
    d = M.unpack(w)
    d["q"] = d["q"] * 20
    w = M.pack(d)
    om, _ = M.forward(w, *M.features(prob.rowptr, prob.col, prob.val))
    om2, _ = M.forward(w, *M.features(prob.rowptr, prob.col, prob.val * 37.5))
    assert np.allclose(om, om2, rtol=1e-12, atol=0)
    assert om.std() > 1e-3  # the network output varies over the nodes
    # relabel the unknowns: outputs are relabelled the same way
    K = prob.to_scipy()
    perm = np.random.default_rng(4).permutation(prob.n)
    Kp = K[perm][:, perm].tocsr()
    Kp.sort_indices()
    omp, _ = M.forward(w, *M.features(Kp.indptr.astype(np.int64), Kp.indices.astype(np.int32), Kp.data))
    assert np.allclose(omp, om[perm], rtol=1e-12, atol=1e-14)


def test_damping_range_keeps_smoother_convergent(small):
    prob, H, lv = small
    K = lv.K[0].toarray()
    rng = np.random.default_rng(5)
    om = rng.uniform(0.01, 1.99, prob.n)
    E = np.eye(prob.n) - (om / lv.d[0])[:, None] * K
    Lk = np.linalg.cholesky(K)
    assert np.linalg.norm(Lk.T @ E @ np.linalg.inv(Lk.T), 2) < 1


# ---------------------------------------------------------- damping cap ----
def test_lanczos_bound_exact_on_diagonal_matrices():
    """For diagonal K the spectrum of D^-1 K is k_i / d_i: Lanczos with as
    many steps as rows spans the whole space, so the estimate is the exact
    maximum; with K = D it is 1 (the cap)."""
    rng = np.random.default_rng(8)
    k = rng.uniform(1.0, 3.0, 9)
    d = k / rng.uniform(0.2, 0.95, 9)
    import scipy.sparse as sp

    lam = M.lanczos_bound(sp.diags(k).tocsr(), d, steps=20)
    assert abs(lam - (k / d).max()) <= 1e-12
    assert M.lanczos_bound(sp.diags(d).tocsr(), d) == 1.0


@pytest.mark.parametrize("d,n,p", [(2, 10, 3), (3, 6, 2), (3, 5, 3)])
def test_lanczos_bound_is_a_close_upper_estimate(d, n, p):
    """Against the dense spectrum: lambda_max(D^-1 K) <= lam_hat <= 1.03
    lambda_max on every level of IgA hierarchies (the residual term
    beta_k |s_k| lifts the Ritz value over the eigenvalue)."""
    prob = I.poisson_box(d, n, p)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    lv = M.Levels(H)
    for l in range(lv.L - 1):
        K = lv.K[l].toarray()
        dl = lv.d[l]
        lam = np.linalg.eigvalsh(K / np.sqrt(dl)[:, None] / np.sqrt(dl)[None, :]).max()
        est = M.lanczos_bound(lv.K[l], dl, seed=M.LANCZOS_SEED + l)
        assert lam <= est <= min(1.0, 1.03 * lam), (l, lam, est)
        assert abs(lv.omax[l] - 2.0 / est) <= 1e-15 * lv.omax[l]
        assert 0.6 < lam < 0.95  # IgA levels: the admissible damping reaches past 2


def test_damping_below_the_cap_keeps_smoother_convergent(small):
    """Every omega_i in (0, 2 / lam_hat) gives a K-norm contraction: the
    cap enlarges the admissible range past 2 without losing convergence."""
    prob, H, lv = small
    K = lv.K[0].toarray()
    rng = np.random.default_rng(6)
    om = rng.uniform(0.01, 0.999 * lv.omax[0], prob.n)
    om[:5] = 0.999 * lv.omax[0]
    assert om.max() > 2.0
    E = np.eye(prob.n) - (om / lv.d[0])[:, None] * K
    Lk = np.linalg.cholesky(K)
    assert np.linalg.norm(Lk.T @ E @ np.linalg.inv(Lk.T), 2) < 1


def test_capped_output_gradient_finite_differences(small):
    """The loss gradient through omega = omega_max sigmoid(z) (per-level
    omega_max) against central differences of the weights."""
    prob, H, lv = small
    w = M.init_weights(12)
    dd = M.unpack(w)
    dd["q"] = dd["q"] * 10
    dd["c"] = np.array([2.5])
    w = M.pack(dd)
    L0, g, om = M.loss_and_grad(lv, w, nprobe=2, seed=13)
    assert max(o.max() for o in om[:-1]) > 2.0  # past the old (0, 2) range
    v = np.random.default_rng(14).standard_normal(M.NPARAM)
    h = 1e-6
    Lp, _, _ = M.loss_and_grad(lv, w + h * v, nprobe=2, seed=13)
    Lm, _, _ = M.loss_and_grad(lv, w - h * v, nprobe=2, seed=13)
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - g @ v) <= 1e-5 * max(abs(fd), 1e-8)


# --------------------------------------------- prolongator smoothing theta ----
@pytest.fixture(scope="module")
def twogrid():
    prob = I.poisson_box(2, 12, 3)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    return prob, M.TwoGrid(H)


def test_twogrid_theta_gradient_finite_differences(twogrid):
    """d L_theta / d theta against central differences of the per-row
    smoothing weights (the two-grid loss rebuilds P_bar and K_c)."""
    prob, tg = twogrid
    rng = np.random.default_rng(21)
    theta = rng.uniform(0.4, 1.6, prob.n)
    m = rng.uniform(0.8, 2.0, prob.n) / tg.d
    X = M.probes(5, 2, prob.n)
    L0, g = M.twogrid_theta_loss(tg, m, theta, X)
    v = rng.standard_normal(prob.n)
    h = 1e-6
    Lp, _ = M.twogrid_theta_loss(tg, m, theta + h * v, X)
    Lm, _ = M.twogrid_theta_loss(tg, m, theta - h * v, X)
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - g @ v) <= 1e-6 * abs(fd)
    assert L0 < 0


def test_twogrid_theta_zero_is_the_tentative_two_grid(twogrid):
    """theta = 0 gives the two-grid operator with the tentative P: the loss
    equals the textbook E = (I - MK)(I - P K_c^-1 P^T K)(I - MK) applied
    densely."""
    prob, tg = twogrid
    m = np.full(prob.n, 1.0) / tg.d
    X = M.probes(6, 2, prob.n)
    L0, _ = M.twogrid_theta_loss(tg, m, np.zeros(prob.n), X)
    K = tg.K.toarray()
    P = tg.P.toarray()
    S = np.eye(prob.n) - m[:, None] * K
    E = S @ (np.eye(prob.n) - P @ np.linalg.solve(P.T @ K @ P, P.T @ K)) @ S
    ref = np.mean([np.log((E @ x) @ K @ (E @ x)) - np.log(x @ K @ x) for x in X])
    assert abs(L0 - ref) <= 1e-12 * abs(ref)


def test_theta_head_gradient_finite_differences(twogrid):
    """The whole chain: network (second head) -> theta -> P_bar, K_c ->
    two-grid loss, against central differences of the weights."""
    prob, tg = twogrid
    w = M.init_weights(8)
    dd = M.unpack(w)
    dd["qt"] = dd["qt"] * 10
    dd["b2"] = np.full(M.HIDDEN, 0.05)
    w = M.pack(dd)
    L0, g, theta = M.theta_loss_and_grad(tg, w, nprobe=2, seed=3)
    assert theta.std() > 1e-3 and 0 < theta.min() and theta.max() < tg.omax
    assert np.all(M.unpack(g)["q"] == 0) and M.unpack(g)["c"][0] == 0  # omega is held fixed
    om0, _ = M.forward(w, *M.features(*tg.csr), tg.omax)
    rng = np.random.default_rng(9)
    for _ in range(2):
        v = rng.standard_normal(M.NPARAM)
        h = 1e-6
        Lp, _, _ = M.theta_loss_and_grad(tg, w + h * v, nprobe=2, seed=3, omega_fixed=om0)
        Lm, _, _ = M.theta_loss_and_grad(tg, w - h * v, nprobe=2, seed=3, omega_fixed=om0)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g @ v) <= 1e-5 * max(abs(fd), 1e-8), (fd, g @ v)
