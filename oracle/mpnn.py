"""CPU ORACLE (test infrastructure) for the learned smoother damping.

The paper's l1-Jacobi smoother (Sec. 3.2) uses x <- x + D^-1 (f - K x)
with the l1 diagonal D.  The learned variant scales it per row,
x <- x + diag(omega_i / d_i) (f - K x), 0 < omega_i < omega_max.  The
smoother converges in the K-norm when 2 diag(d / omega) - K is positive
definite, which holds for every omega_i < 2 / lambda_max(D^-1 K); the l1
diagonal gives lambda_max <= 1, so (0, 2) is always admissible, and the IgA
levels have lambda_max of 0.7-0.9, so the admissible range reaches 2.2-2.8.
omega_max = 2 / lam_hat per level, lam_hat = min(1, Lanczos upper estimate
of lambda_max(D^-1 K)) (lanczos_bound below).  omega is produced by a small
message-passing network over the matrix graph and trained to minimise the
error reduction of the V-cycle (Sec. 3, two-level correction applied
recursively) used as CG preconditioner.  The paper has no learned
component; this file is the plain FP64 statement of what the GPU kernels
compute, written out step by step.

Network (hidden width 32, two message-passing layers):
  node features  x_i = [rho_i, sig_i, log2(nnz_i) / 8, 1] with
                 rho_i = sum_{j != i} |k_ij| / k_ii,
                 sig_i = sum_{j != i} k_ij / k_ii
  edge weights   a_ij = k_ij / sqrt(k_ii k_jj), j != i   (a_ii = 0)
  h0  = relu(W0 x + b0)
  m_l = sum_j a_ij h_{l-1, j}
  h_l = relu(U_l m_l + V_l h_{l-1} + b_l),      l = 1, 2
  omega = omega_max sigmoid(q . h2 + c)
  theta = theta_max sigmoid(qt . h2 + ct)     (second head, level 0 only)
applied to every level's matrix with the same weights (omega_max per level).
theta is the per-row weight of the smoothed prolongator of level 0,
P_bar = (I - diag(theta) D^-1 K) P (the paper's Sec. 3.1 "Variants" with a
per-row weight), theta_max = omega_max of level 0.

Loss for probe vectors x_k (SplitMix64 uniform in (-1, 1)):
  L = (1/m) sum_k log( y_k^T K y_k / x_k^T K x_k ),  y_k = x_k - B_omega K x_k
with B_omega the V-cycle (one pre- and one post-sweep, exact coarsest
solve).  The gradient is obtained by reverse-mode differentiation of the
V-cycle steps and of the network, written out by hand below.

Loss of the smoothing weights (two-grid, level 0, exact coarse solve):
  L_theta = (1/m) sum_k log( y_k^T K y_k / x_k^T K x_k ),
  y_k = (I - M K)(I - P_bar K_c^-1 P_bar^T K)(I - M K) x_k,
  K_c = P_bar^T K P_bar, M = diag(omega / d) (omega of the first head, held
  fixed in this loss), with its gradient with respect to theta (hence to
  qt, ct and the shared layers).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp

LANCZOS_STEPS = 15
LANCZOS_SEED = 0x4C414E43  # start vector of level l: SplitMix64(LANCZOS_SEED + l)

HIDDEN = 32
NFEAT = 4
# flat parameter layout (name, shape)
LAYOUT = [("W0", (HIDDEN, NFEAT)), ("b0", (HIDDEN,)), ("U1", (HIDDEN, HIDDEN)), ("V1", (HIDDEN, HIDDEN)),
          ("b1", (HIDDEN,)), ("U2", (HIDDEN, HIDDEN)), ("V2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("q", (HIDDEN,)), ("c", (1,)), ("qt", (HIDDEN,)), ("ct", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in LAYOUT)


def unpack(w):
    out, o = {}, 0
    for name, shape in LAYOUT:
        k = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + k], np.float64).reshape(shape)
        o += k
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in LAYOUT])


def init_weights(seed=1):
    """Seeded initial weights: the shared input generator's recipe (scaled
    uniform SplitMix64 draws, zero biases, q scaled by 0.1, so that omega
    starts near 1)."""
    from paper_2511_21268_gb300 import inputs as I

    w = I.mpnn_init_weights(seed)
    assert len(w) == NPARAM
    return w


# ---------------------------------------------------------------- features
def features(rowptr, col, val):
    """Node features x (N, 4) and the normalised off-diagonal matrix A'."""
    n = len(rowptr) - 1
    K = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    kii = K.diagonal()
    off = K - sp.diags(kii)
    off.eliminate_zeros()
    rho = np.asarray(abs(off).sum(axis=1)).ravel() / kii
    sig = np.asarray(off.sum(axis=1)).ravel() / kii
    nnz = np.diff(rowptr).astype(np.float64)
    x = np.stack([rho, sig, np.log2(nnz) / 8.0, np.ones(n)], axis=1)
    s = 1.0 / np.sqrt(kii)
    Ap = sp.diags(s) @ off @ sp.diags(s)
    return x, sp.csr_matrix(Ap)


# ----------------------------------------------------------------- network
def lanczos_bound(K, d, steps=LANCZOS_STEPS, seed=LANCZOS_SEED):
    """Upper estimate lam_hat of lambda_max(D^-1 K) for SPD K and positive d.

    Lanczos (no reorthogonalisation) on the symmetric S = D^-1/2 K D^-1/2,
    which has the spectrum of D^-1 K, from q_1 = x / ||x||, x_i = 2 U_i - 1
    with U_i draw i of SplitMix64(seed) on 53 bits:
        w = S q_j - beta_{j-1} q_{j-1}; alpha_j = q_j . w;
        w = w - alpha_j q_j; beta_j = ||w||; q_{j+1} = w / beta_j.
    The largest eigenvalue theta of the tridiagonal T = tridiag(beta,
    alpha, beta) is a Ritz value of S, and some eigenvalue of S lies within
    beta_k |s_k| of it (s the unit eigenvector of T for theta, k the last
    step); theta + beta_k |s_k| is returned, capped at 1 (the l1 diagonal
    bounds lambda_max by 1).  A zero beta_j ends the recurrence: the Krylov
    space is invariant and theta is exact."""
    n = K.shape[0]
    isd = 1.0 / np.sqrt(d)
    x = probes(seed, 1, n)[0]
    q = x / np.sqrt(x @ x)
    qp = np.zeros(n)
    bprev = 0.0
    alpha, beta = [], []
    for _ in range(min(steps, n)):
        w = isd * (K @ (isd * q)) - bprev * qp
        a = q @ w
        w = w - a * q
        b = np.sqrt(w @ w)
        alpha.append(a)
        beta.append(b)
        if b == 0.0:
            break
        qp, q, bprev = q, w / b, b
    ev, S = sl.eigh_tridiagonal(np.array(alpha), np.array(beta[:-1]))
    bound = ev[-1] + beta[-1] * abs(S[-1, -1])
    return min(1.0, bound)


def forward(w, x, Ap, omax=2.0, tmax=2.0):
    """omega (N,) of the first head and the tape; the tape also holds the
    second head's theta = tmax sigmoid(qt . h2 + ct)."""
    p = unpack(w)
    u0 = x @ p["W0"].T + p["b0"]
    h0 = np.maximum(u0, 0.0)
    m1 = Ap @ h0
    u1 = m1 @ p["U1"].T + h0 @ p["V1"].T + p["b1"]
    h1 = np.maximum(u1, 0.0)
    m2 = Ap @ h1
    u2 = m2 @ p["U2"].T + h1 @ p["V2"].T + p["b2"]
    h2 = np.maximum(u2, 0.0)
    z = h2 @ p["q"] + p["c"][0]
    sg = 1.0 / (1.0 + np.exp(-z))
    zt = h2 @ p["qt"] + p["ct"][0]
    sgt = 1.0 / (1.0 + np.exp(-zt))
    return omax * sg, dict(x=x, u0=u0, h0=h0, m1=m1, u1=u1, h1=h1, m2=m2, u2=u2, h2=h2, z=z, sg=sg, zt=zt, sgt=sgt,
                           theta=tmax * sgt)


def backward(w, tape, Ap, domega, omax=2.0, dtheta=None, tmax=2.0):
    """Gradient of the loss w.r.t. the flat weights given d loss / d omega
    (and d loss / d theta of the second head, if any)."""
    p = unpack(w)
    dz = domega * omax * tape["sg"] * (1.0 - tape["sg"])
    g = {"q": tape["h2"].T @ dz, "c": np.array([dz.sum()])}
    dh2 = np.outer(dz, p["q"])
    if dtheta is None:
        g["qt"], g["ct"] = np.zeros(HIDDEN), np.zeros(1)
    else:
        dzt = dtheta * tmax * tape["sgt"] * (1.0 - tape["sgt"])
        g["qt"], g["ct"] = tape["h2"].T @ dzt, np.array([dzt.sum()])
        dh2 = dh2 + np.outer(dzt, p["qt"])
    du2 = dh2 * (tape["u2"] > 0)
    g["U2"] = du2.T @ tape["m2"]
    g["V2"] = du2.T @ tape["h1"]
    g["b2"] = du2.sum(axis=0)
    dh1 = du2 @ p["V2"] + Ap.T @ (du2 @ p["U2"])
    du1 = dh1 * (tape["u1"] > 0)
    g["U1"] = du1.T @ tape["m1"]
    g["V1"] = du1.T @ tape["h0"]
    g["b1"] = du1.sum(axis=0)
    dh0 = du1 @ p["V1"] + Ap.T @ (du1 @ p["U1"])
    du0 = dh0 * (tape["u0"] > 0)
    g["W0"] = du0.T @ tape["x"]
    g["b0"] = du0.sum(axis=0)
    return pack(g)


# ------------------------------------------------------------ V-cycle with omega
class Levels:
    """Hierarchy data of an oracle Hierarchy as scipy operators."""

    def __init__(self, H):
        self.L = H.num_levels
        self.K, self.d, self.P = [], [], []
        for l in range(self.L):
            rp, ci, v = H.level_csr(l)
            n = len(rp) - 1
            self.K.append(sp.csr_matrix((v, ci, rp), shape=(n, n)))
            self.d.append(H.level_vectors(l)[0])
            if l < self.L - 1:
                agg, pv = H.level_map(l)
                self.P.append(sp.csr_matrix((pv, (np.arange(n), agg)), shape=(n, H.level_n(l + 1))))
        self.chol = H.coarse_chol()
        self.csr = [(H.level_csr(l)) for l in range(self.L)]
        # damping cap of every smoothed level: omega_max = 2 / lam_hat
        self.omax = [2.0 / lanczos_bound(self.K[l], self.d[l], seed=LANCZOS_SEED + l) for l in range(self.L - 1)]

    def coarse_solve(self, f):
        y = sl.solve_triangular(self.chol, f, lower=True)
        return sl.solve_triangular(self.chol.T, y, lower=False)


def vcycle_omega(lv: Levels, omegas, f, l=0, tape=None):
    """B_omega f from level l: x1 = Dw f, r1 = f - K x1, e = V_{l+1}(P^T r1),
    x2 = x1 + P e, r2 = f - K x2, x3 = x2 + Dw r2 (Dw = diag(omega / d))."""
    if l == lv.L - 1:
        return lv.coarse_solve(f)
    K, P, Dw = lv.K[l], lv.P[l], omegas[l] / lv.d[l]
    x1 = Dw * f
    r1 = f - K @ x1
    e = vcycle_omega(lv, omegas, P.T @ r1, l + 1, tape)
    x2 = x1 + P @ e
    r2 = f - K @ x2
    if tape is not None:
        tape[l] = (f, r2)
    return x2 + Dw * r2


def vcycle_omega_backward(lv: Levels, omegas, gbar, tape, domegas, l=0):
    """Reverse of vcycle_omega: given d loss / d x3 at level l, accumulate
    d loss / d omega_l into domegas[l] and return d loss / d f."""
    if l == lv.L - 1:
        return lv.coarse_solve(gbar)
    K, P, d = lv.K[l], lv.P[l], lv.d[l]
    Dw = omegas[l] / d
    f, r2 = tape[l]
    # x3 = x2 + Dw r2
    dx2 = gbar.copy()
    dr2 = Dw * gbar
    domegas[l] += gbar * r2 / d
    # r2 = f - K x2
    df = dr2.copy()
    dx2 -= K @ dr2
    # x2 = x1 + P e
    dx1 = dx2.copy()
    de = P.T @ dx2
    # e = V_{l+1}(fc), fc = P^T r1
    dfc = vcycle_omega_backward(lv, omegas, de, tape, domegas, l + 1)
    dr1 = P @ dfc
    # r1 = f - K x1
    df += dr1
    dx1 -= K @ dr1
    # x1 = Dw f
    df += Dw * dx1
    domegas[l] += dx1 * f / d
    return df


def probes(seed, m, n):
    """Probe k, entry i: 2 U - 1 with U draw (k n + i) of SplitMix64(seed)."""
    from paper_2511_21268_gb300 import inputs as I

    return (I.rng_u01(seed, m * n) * 2.0 - 1.0).reshape(m, n)


def loss_and_domega(lv: Levels, omegas, X):
    """Mean over probes of log(y^T K y / x^T K x), y = x - B K x, and its
    gradient with respect to every level's omega."""
    K = lv.K[0]
    total = 0.0
    domegas = [np.zeros(lv.K[l].shape[0]) for l in range(lv.L)]
    for x in X:
        Kx = K @ x
        tape = {}
        z = vcycle_omega(lv, omegas, Kx, 0, tape)
        y = x - z
        Ky = K @ y
        yKy, xKx = y @ Ky, x @ Kx
        total += np.log(yKy) - np.log(xKx)
        gbar = -2.0 * Ky / yKy  # d/dz of log(y^T K y), y = x - z
        vcycle_omega_backward(lv, omegas, gbar, tape, domegas, 0)
    m = len(X)
    return total / m, [g / m for g in domegas]


def loss_and_grad(H, w, nprobe=4, seed=99):
    """Loss of the network's damping on hierarchy H (an oracle Hierarchy or
    its Levels) and its gradient with respect to the flat weights (network
    applied to every smoothed level, omega_max of each level)."""
    lv = H if isinstance(H, Levels) else Levels(H)
    feats = [features(*lv.csr[l]) for l in range(lv.L - 1)]
    outs = [forward(w, x, Ap, lv.omax[l]) for l, (x, Ap) in enumerate(feats)]
    # the coarsest level is solved exactly: it has no smoother
    omegas = [o[0] for o in outs] + [np.ones(lv.K[lv.L - 1].shape[0])]
    X = probes(seed, nprobe, lv.K[0].shape[0])
    loss, domegas = loss_and_domega(lv, omegas, X)
    grad = np.zeros(NPARAM)
    for l in range(lv.L - 1):
        grad += backward(w, outs[l][1], feats[l][1], domegas[l], lv.omax[l])
    return loss, grad, omegas


# ----------------------------------------------- smoothing weights theta
class TwoGrid:
    """Level 0 of an oracle hierarchy with the pieces of the smoothed
    prolongator: K, d, the tentative P (agg, pval), the product K P (its
    values are what theta scales) and the cap omega_max of level 0."""

    def __init__(self, H):
        import oracle as O

        self.O = O
        rp, ci, v = H.level_csr(0)
        n = len(rp) - 1
        self.csr = (rp, ci, v)
        self.K = sp.csr_matrix((v, ci, rp), shape=(n, n))
        self.d = H.level_vectors(0)[0]
        self.agg, self.pval = H.level_map(0)
        self.nc = H.level_n(1)
        self.P = sp.csr_matrix((self.pval, (np.arange(n), self.agg)), shape=(n, self.nc))
        self.KP = (self.K @ self.P).tocsr()
        self.omax = 2.0 / lanczos_bound(self.K, self.d, seed=LANCZOS_SEED)

    def pbar(self, theta):
        """P_bar and K_c = P_bar^T K P_bar in the oracle's own arithmetic."""
        rp, ci, v = self.csr
        prp, pci, pv = self.O.smooth_prolongator(rp, ci, v, self.d, theta, self.agg, self.pval, self.nc)
        crp, cci, cv = self.O.galerkin_general(rp, ci, v, prp, pci, pv, self.nc)
        Pb = sp.csr_matrix((pv, pci, prp), shape=(len(rp) - 1, self.nc))
        Kc = sp.csr_matrix((cv, cci, crp), shape=(self.nc, self.nc)).toarray()
        return Pb, Kc


def twogrid_theta_loss(tg: TwoGrid, m, theta, X):
    """L_theta (see the module header) for per-row smoothing weights theta
    and smoother diagonal m = omega / d, and d L_theta / d theta.

    Reverse pass for one probe x (K, M, K_c symmetric):
      x1 = x - M K x; g = P_bar^T K x1; e = K_c^-1 g; x2 = x1 - P_bar e;
      y = x2 - M K x2; L = log(y'Ky) - log(x'Kx)
      ybar = 2 K y / y'Ky; x2bar = ybar - K M ybar; ebar = -P_bar^T x2bar;
      gbar = K_c^-1 ebar;  d L / d P_bar = -a e' + b gbar' with
      a = x2bar + K P_bar gbar, b = K x1 - K P_bar e = K x2;
    and P_bar(i, J) = P(i, J) - (theta_i / d_i) (K P)(i, J) gives
      d L / d theta_i = (a_i (K P e)_i - b_i (K P gbar)_i) / d_i."""
    Pb, Kc = tg.pbar(theta)
    L = sl.cho_factor(Kc)
    K = tg.K
    total = 0.0
    dth = np.zeros(K.shape[0])
    for x in X:
        Kx = K @ x
        x1 = x - m * Kx
        Kx1 = K @ x1
        e = sl.cho_solve(L, Pb.T @ Kx1)
        x2 = x1 - Pb @ e
        Kx2 = K @ x2
        y = x2 - m * Kx2
        Ky = K @ y
        yKy, xKx = y @ Ky, x @ Kx
        total += np.log(yKy) - np.log(xKx)
        ybar = 2.0 * Ky / yKy
        x2bar = ybar - K @ (m * ybar)
        gbar = sl.cho_solve(L, -(Pb.T @ x2bar))
        a = x2bar + K @ (Pb @ gbar)
        b = Kx2
        dth += (a * (tg.KP @ e) - b * (tg.KP @ gbar)) / tg.d
    return total / len(X), dth / len(X)


def theta_loss_and_grad(tg: TwoGrid, w, nprobe=4, seed=99, omega_fixed=None):
    """L_theta of the network's two heads on level 0 (omega held fixed: the
    first head's, or omega_fixed when given) and its gradient with respect
    to the flat weights; returns (loss, grad, theta)."""
    x, Ap = features(*tg.csr)
    omega, tape = forward(w, x, Ap, tg.omax, tg.omax)
    if omega_fixed is not None:
        omega = omega_fixed
    X = probes(seed, nprobe, tg.K.shape[0])
    loss, dth = twogrid_theta_loss(tg, omega / tg.d, tape["theta"], X)
    grad = backward(w, tape, Ap, np.zeros_like(omega), tg.omax, dth, tg.omax)
    return loss, grad, tape["theta"]
