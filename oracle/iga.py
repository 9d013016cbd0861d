"""CPU ORACLE (test infrastructure) for the IgA assembly of K u = F.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA
library or with the input generator's C assembly.

What it computes (arXiv 2511.21268, Sec. 2.2, single-patch discretization):
the stiffness entries of -div(kappa grad u) = f pulled back to the
parametric cube,

    k_ij = int_[0,1]^3 kappa(F(xi)) (grad_xi N_j)^T J^-1 J^-T (grad_xi N_i) |det J| dxi,
    f_i  = int_[0,1]^3 f(F(xi)) N_i |det J| dxi,

J = dF/dxi, by the standard element loop of that section: for every knot
span element, the element matrix and vector by Gauss quadrature (nq points
per direction), added into the global entries through the local-to-global
index map.  kappa = 1 is the paper's Laplacian; the variable kappa is the
learned-damping workload's coefficient.

Basis (Sec. 2.1): tensor products N_i(xi) = B_i1(xi1) B_i2(xi2) B_i3(xi3) of
the degree-p B-splines on the open uniform knot vector with n elements (p+1
zeros, the interior knots 1/n .. (n-1)/n, p+1 ones), evaluated by the
Cox-de Boor recursion.  The discrete space is the B-spline space on the
parametric cube for both geometries (non-isoparametric in the annulus case,
Sec. 2.4).

Geometries:
  "cube"    F(xi) = xi on [0,1]^3;
  "annulus" the quarter annulus of radii 1 and 2 extruded over z in [0,1]:
            F(xi) = (1 + xi1) c(xi2) + xi3 e_z, with c the quadratic NURBS
            arc (Sec. 2.1's rational form) through control points (1,0),
            (1,1), (0,1) with weights 1, sqrt(2)/2, 1 -- the exact quarter
            circle.

Coefficient: kappa(x) = exp(sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m))
(M random Fourier features of a Gaussian field; omega and phi are inputs),
kappa = 1 for M = 0.

Unknowns: all (n+p)^3 functions (with_boundary=True), or the interior ones
after eliminating the functions that are nonzero on the boundary
(homogeneous Dirichlet data on the whole boundary): per direction the
functions 1 .. n+p-2, numbered i1 + m (i2 + m i3).

Sources: "one" (f = 1) or "sine" (f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)).
"""
from __future__ import annotations

import math

import numpy as np

WMID = math.sqrt(0.5)  # weight of the arc's middle control point


# ------------------------------------------------------------- B-splines
def knots(n: int, p: int) -> np.ndarray:
    """Open uniform knot vector on [0, 1]: n + 2p + 1 knots."""
    return np.concatenate([np.zeros(p + 1), np.arange(1, n) / n, np.ones(p + 1)])


def bspline(n: int, p: int, x: float) -> tuple[np.ndarray, np.ndarray]:
    """Values and first derivatives of all n+p B-splines of degree p at x in
    [0, 1], by the Cox-de Boor recursion
        N_{i,0} = 1 on [u_i, u_{i+1}) (the last non-empty span is closed),
        N_{i,k} = (x - u_i)/(u_{i+k} - u_i) N_{i,k-1}
                + (u_{i+k+1} - x)/(u_{i+k+1} - u_{i+1}) N_{i+1,k-1},
        N'_{i,p} = p N_{i,p-1}/(u_{i+p} - u_i) - p N_{i+1,p-1}/(u_{i+p+1} - u_{i+1}),
    with every term whose denominator is 0 left out."""
    u = knots(n, p)
    nk = len(u)
    N = np.zeros(nk - 1)
    span = min(int(math.floor(x * n)), n - 1) + p  # knot span [u_span, u_span+1) holding x
    N[span] = 1.0
    prev = N
    for k in range(1, p + 1):
        cur = np.zeros(nk - 1 - k)
        for i in range(nk - 1 - k):
            a = 0.0
            if u[i + k] > u[i]:
                a += (x - u[i]) / (u[i + k] - u[i]) * prev[i]
            if u[i + k + 1] > u[i + 1]:
                a += (u[i + k + 1] - x) / (u[i + k + 1] - u[i + 1]) * prev[i + 1]
            cur[i] = a
        if k == p:
            d = np.zeros(nk - 1 - k)
            for i in range(nk - 1 - k):
                if u[i + p] > u[i]:
                    d[i] += p * prev[i] / (u[i + p] - u[i])
                if u[i + p + 1] > u[i + 1]:
                    d[i] -= p * prev[i + 1] / (u[i + p + 1] - u[i + 1])
            return cur, d
        prev = cur
    return prev, np.zeros_like(prev)  # p = 0


def gauss(nq: int) -> tuple[np.ndarray, np.ndarray]:
    """Gauss-Legendre nodes and weights on [-1, 1]."""
    return np.polynomial.legendre.leggauss(nq)


# --------------------------------------------------------------- geometry
def arc(t: float) -> tuple[np.ndarray, np.ndarray]:
    """The quadratic NURBS quarter arc c(t) and c'(t): Bernstein basis
    B0 = (1-t)^2, B1 = 2t(1-t), B2 = t^2, weights (1, WMID, 1), control
    points (1,0), (1,1), (0,1); c = sum w_k B_k P_k / sum w_k B_k."""
    B = np.array([(1 - t) ** 2, 2 * t * (1 - t), t * t])
    dB = np.array([-2 * (1 - t), 2 - 4 * t, 2 * t])
    w = np.array([1.0, WMID, 1.0])
    P = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    W = w @ B
    dW = w @ dB
    A = (w * B) @ P
    dA = (w * dB) @ P
    return A / W, (dA * W - A * dW) / (W * W)


def geometry(kind: str, xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """x = F(xi) and J = dF/dxi (J[a, b] = dx_a / dxi_b)."""
    if kind == "cube":
        return xi.copy(), np.eye(3)
    if kind != "annulus":
        raise ValueError(kind)
    c, dc = arc(xi[1])
    r = 1.0 + xi[0]
    x = np.array([r * c[0], r * c[1], xi[2]])
    J = np.array([[c[0], r * dc[0], 0.0], [c[1], r * dc[1], 0.0], [0.0, 0.0, 1.0]])
    return x, J


def kappa(x: np.ndarray, omega: np.ndarray | None, phi: np.ndarray | None, sigma: float) -> float:
    """exp(sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m)); 1 without features.
    omega is (M, 3), phi (M,)."""
    if omega is None or len(phi) == 0:
        return 1.0
    M = len(phi)
    return math.exp(sigma * math.sqrt(2.0 / M) * float(np.sum(np.cos(omega @ x + phi))))


def source(kind: str, x: np.ndarray) -> float:
    if kind == "one":
        return 1.0
    if kind == "sine":
        return 3.0 * math.pi ** 2 * math.sin(math.pi * x[0]) * math.sin(math.pi * x[1]) * math.sin(math.pi * x[2])
    raise ValueError(kind)


# ----------------------------------------------------------- element loop
class Patch:
    """One tensor-product patch with its data; unknown numbering as in the
    module docstring."""

    def __init__(self, n: int, p: int, nq: int | None = None, geom: str = "cube", with_boundary: bool = False,
                 omega=None, phi=None, sigma: float = 0.0, src: str = "one"):
        self.n, self.p, self.nq = n, p, nq or p + 1
        self.geom, self.with_boundary, self.src = geom, with_boundary, src
        self.omega = None if omega is None else np.asarray(omega, np.float64).reshape(-1, 3)
        self.phi = None if phi is None else np.asarray(phi, np.float64)
        self.sigma = sigma
        self.off = 0 if with_boundary else 1
        self.m = n + p if with_boundary else n + p - 2
        self.N = self.m ** 3
        self.gx, self.gw = gauss(self.nq)
        self._cache: dict[int, tuple[np.ndarray, np.ndarray]] = {}

    def dof(self, g1: int, g2: int, g3: int) -> int:
        """Unknown index of the global function (g1, g2, g3), or -1 when it
        is eliminated."""
        i = [g - self.off for g in (g1, g2, g3)]
        if min(i) < 0 or max(i) >= self.m:
            return -1
        return i[0] + self.m * (i[1] + self.m * i[2])

    def basis_1d(self, e: int) -> tuple[np.ndarray, np.ndarray]:
        """V[q, a], D[q, a]: values and derivatives of the p+1 functions
        e .. e+p at the nq Gauss points of element e of one direction."""
        if e not in self._cache:
            n, p, h = self.n, self.p, 1.0 / self.n
            V = np.zeros((self.nq, p + 1))
            D = np.zeros((self.nq, p + 1))
            for q in range(self.nq):
                v, d = bspline(n, p, (e + 0.5 * (self.gx[q] + 1.0)) * h)
                V[q] = v[e:e + p + 1]
                D[q] = d[e:e + p + 1]
            self._cache[e] = (V, D)
        return self._cache[e]

    def element(self, e: tuple[int, int, int]) -> tuple[np.ndarray, np.ndarray]:
        """Element matrix k^e_ab and vector f^e_a of the (p+1)^3 functions
        nonzero on element e (local a = a1 + (p+1)(a2 + (p+1) a3), global
        function e_k + a_k per direction): sum over the element's Gauss
        points of kappa w |det J| (J^-T grad N_a) . (J^-T grad N_b) and
        f w |det J| N_a."""
        n, p, nq = self.n, self.p, self.nq
        P1 = p + 1
        h = 1.0 / n
        ke = np.zeros((P1 ** 3, P1 ** 3))
        fe = np.zeros(P1 ** 3)
        (V1, D1), (V2, D2), (V3, D3) = (self.basis_1d(e[k]) for k in range(3))
        for q3 in range(nq):
            for q2 in range(nq):
                for q1 in range(nq):
                    q = (q1, q2, q3)
                    xi = np.array([(e[k] + 0.5 * (self.gx[q[k]] + 1.0)) * h for k in range(3)])
                    w = (0.5 * h) ** 3 * self.gw[q1] * self.gw[q2] * self.gw[q3]
                    # N_a and grad_xi N_a, a = a1 + P1 (a2 + P1 a3)
                    Nv = np.kron(V3[q3], np.kron(V2[q2], V1[q1]))
                    G = np.stack([np.kron(V3[q3], np.kron(V2[q2], D1[q1])),
                                  np.kron(V3[q3], np.kron(D2[q2], V1[q1])),
                                  np.kron(D3[q3], np.kron(V2[q2], V1[q1]))], axis=1)
                    x, J = geometry(self.geom, xi)
                    detJ = np.linalg.det(J)
                    grad = G @ np.linalg.inv(J)  # row a: (J^-T grad_xi N_a)^T
                    kap = kappa(x, self.omega, self.phi, self.sigma)
                    ke += kap * w * abs(detJ) * (grad @ grad.T)
                    fe += source(self.src, x) * w * abs(detJ) * Nv
        return ke, fe

    def local_dofs(self, e: tuple[int, int, int]) -> list[int]:
        P1 = self.p + 1
        return [self.dof(e[0] + a1, e[1] + a2, e[2] + a3) for a3 in range(P1) for a2 in range(P1) for a1 in range(P1)]

    def assemble(self) -> tuple[np.ndarray, np.ndarray]:
        """Dense K and F by the element loop (small patches only)."""
        K = np.zeros((self.N, self.N))
        F = np.zeros(self.N)
        for e3 in range(self.n):
            for e2 in range(self.n):
                for e1 in range(self.n):
                    e = (e1, e2, e3)
                    ke, fe = self.element(e)
                    loc = self.local_dofs(e)
                    for a, I in enumerate(loc):
                        if I < 0:
                            continue
                        F[I] += fe[a]
                        for b, Jd in enumerate(loc):
                            if Jd >= 0:
                                K[I, Jd] += ke[a, b]
        return K, F

    def row(self, I: int) -> tuple[dict[int, float], float]:
        """Row I of K (column -> value) and F[I], from the elements in the
        support of unknown I only."""
        m, p, n = self.m, self.p, self.n
        i = (I % m, (I // m) % m, I // (m * m))
        g = [ik + self.off for ik in i]
        out: dict[int, float] = {}
        f = 0.0
        P1 = p + 1
        for e3 in range(max(0, g[2] - p), min(n - 1, g[2]) + 1):
            for e2 in range(max(0, g[1] - p), min(n - 1, g[1]) + 1):
                for e1 in range(max(0, g[0] - p), min(n - 1, g[0]) + 1):
                    e = (e1, e2, e3)
                    ke, fe = self.element(e)
                    a = (g[0] - e1) + P1 * ((g[1] - e2) + P1 * (g[2] - e3))
                    f += fe[a]
                    for b, Jd in enumerate(self.local_dofs(e)):
                        if Jd >= 0:
                            out[Jd] = out.get(Jd, 0.0) + ke[a, b]
        return out, f


def greville(n: int, p: int) -> np.ndarray:
    """Greville abscissae (mean of p consecutive interior knots) of the n+p
    functions: sum_i gamma_i B_i(x) = x for p >= 1."""
    u = knots(n, p)
    return np.array([u[i + 1:i + p + 1].mean() for i in range(n + p)])
