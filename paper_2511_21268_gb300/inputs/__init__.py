"""Seeded synthetic inputs: IgA stiffness systems K u = F and random vectors.

This module is the only code shared by the CPU oracle and the GPU path.  It
builds the *inputs* of the AMG-PCG method (the matrix, the right-hand side,
seeded random fields) and holds none of the method's arithmetic.  The
numerical work happens in ``iga_gen.c`` (plain C, FP64, no FMA contraction).

Workload recipes (arXiv 2511.21268, Sec. 2 and Sec. 5 for the problem class):

* ``poisson_box(d, n, p)`` -- -Laplace u = f on the unit square/cube, B-splines
  of degree p, C^{p-1}, n elements per direction, homogeneous Dirichlet data
  eliminated, f from the manufactured solution u = prod sin(pi x_k).
  N = (n+p-2)^d.
* ``poisson_box_random_rhs`` -- same matrix, F = K u_true with u_true ~ N(0,1).
* ``batch_instances`` -- the mixed batch of 2-D instances with p drawn from
  {2,3,4} and n from {32..256} by a seeded SplitMix64 stream.
* ``annulus_kappa`` -- NURBS quarter annulus extruded in z with a log-normal
  coefficient kappa = exp(g), g a seeded Gaussian field.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field

import numpy as np

from .. import _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build_inputs()
        L = ctypes.CDLL(path)
        i32, i64, u64, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        P = ctypes.c_void_p
        L.iga_rng_u01.argtypes = [u64, i64, P]
        L.iga_rng_normal.argtypes = [u64, i64, P]
        L.iga_gauss_legendre.argtypes = [i32, P, P]
        L.iga_gauss_legendre.restype = i32
        L.iga_bspline_local.argtypes = [i32, i32, i32, dbl, P, P]
        L.iga_bspline_all.argtypes = [i32, i32, dbl, P, P]
        L.iga_1d_matrices.argtypes = [i32, i32, i32, P, P]
        L.iga_1d_matrices.restype = i32
        L.iga_num_dofs.argtypes = [i32, i32, i32, i32]
        L.iga_num_dofs.restype = i64
        L.iga_nnz.argtypes = [i32, i32, i32, i32]
        L.iga_nnz.restype = i64
        L.iga_assemble_kron.argtypes = [i32, i32, i32, i32, P, P, P]
        L.iga_assemble_kron.restype = i32
        L.iga_kron_box_nnz.argtypes = [i32, i32, P, P, P]
        L.iga_kron_box_nnz.restype = i32
        L.iga_assemble_kron_box.argtypes = [i32, i32, P, P, P, P, P]
        L.iga_assemble_kron_box.restype = i32
        L.iga_assemble_lshape.argtypes = [i32, i32, P, i32, i32, P, P, P, i64]
        L.iga_assemble_lshape.restype = i32
        L.iga_load_sine.argtypes = [i32, i32, i32, i32, i32, P]
        L.iga_load_sine.restype = i32
        L.iga_assemble_elem.argtypes = [i32, i32, i32, i32, i32, i32, i32, dbl, dbl, u64, i32, P, P, P, P]
        L.iga_assemble_elem.restype = i32
        L.iga_l2_error_sine.argtypes = [i32, i32, i32, i32, P]
        L.iga_l2_error_sine.restype = dbl
        L.iga_csr_apply.argtypes = [i64, P, P, P, P, P]
        L.iga_kappa_points.argtypes = [i32, dbl, dbl, u64, i64, P, P]
        L.iga_geom_points.argtypes = [i32, i32, i64, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------- RNG ----
def rng_u01(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    lib().iga_rng_u01(seed & 0xFFFFFFFFFFFFFFFF, count, _p(out))
    return out


def rng_normal(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, np.float64)
    lib().iga_rng_normal(seed & 0xFFFFFFFFFFFFFFFF, count, _p(out))
    return out


def splitmix64(seed: int, count: int) -> list[int]:
    """Raw 64-bit SplitMix64 outputs (pure Python; used only to draw workload
    parameters such as the batch's (p, n) pairs)."""
    M = 0xFFFFFFFFFFFFFFFF
    out = []
    for k in range(count):
        z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return out


# ----------------------------------------------------- basis / quadrature ----
def gauss_legendre(q: int) -> tuple[np.ndarray, np.ndarray]:
    x = np.empty(q)
    w = np.empty(q)
    if lib().iga_gauss_legendre(q, _p(x), _p(w)) != 0:
        raise ValueError("bad quadrature order")
    return x, w


def bspline_all(n: int, p: int, xi: float) -> tuple[np.ndarray, np.ndarray]:
    v = np.empty(n + p)
    d = np.empty(n + p)
    lib().iga_bspline_all(n, p, float(xi), _p(v), _p(d))
    return v, d


def one_d_matrices(n: int, p: int, nq: int | None = None) -> tuple[np.ndarray, np.ndarray]:
    nb = n + p
    K1 = np.empty((nb, nb))
    M1 = np.empty((nb, nb))
    if lib().iga_1d_matrices(n, p, nq or p + 1, _p(K1), _p(M1)) != 0:
        raise ValueError("bad arguments")
    return K1, M1


def num_dofs(d: int, n: int, p: int, with_boundary: bool = False) -> int:
    return int(lib().iga_num_dofs(d, n, p, int(with_boundary)))


def nnz(d: int, n: int, p: int, with_boundary: bool = False) -> int:
    return int(lib().iga_nnz(d, n, p, int(with_boundary)))


# ------------------------------------------------------------ problems ----
@dataclass
class Problem:
    """A CSR system K u = F (FP64, int64 row offsets, int32 sorted columns)."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    F: np.ndarray
    meta: dict = field(default_factory=dict)
    u_true: np.ndarray | None = None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def assemble_kron(d: int, n: int, p: int, with_boundary: bool = False):
    N = num_dofs(d, n, p, with_boundary)
    Z = nnz(d, n, p, with_boundary)
    rowptr = np.empty(N + 1, np.int64)
    col = np.empty(Z, np.int32)
    val = np.empty(Z, np.float64)
    if lib().iga_assemble_kron(d, n, p, int(with_boundary), _p(rowptr), _p(col), _p(val)) != 0:
        raise ValueError("bad arguments")
    return rowptr, col, val


def load_sine(d: int, n: int, p: int, nq: int | None = None, with_boundary: bool = False) -> np.ndarray:
    F = np.empty(num_dofs(d, n, p, with_boundary))
    if lib().iga_load_sine(d, n, p, nq or p + 1, int(with_boundary), _p(F)) != 0:
        raise ValueError("bad arguments")
    return F


def assemble_elem(d, n, p, nq=None, geom=0, with_boundary=False, kappa=None, fkind=0):
    """Element-loop assembly. kappa = (M, ell, sigma, seed) or None (kappa=1).
    fkind 0: f = 1; fkind 1: f = d pi^2 prod sin(pi x_k)."""
    N = num_dofs(d, n, p, with_boundary)
    Z = nnz(d, n, p, with_boundary)
    rowptr = np.empty(N + 1, np.int64)
    col = np.empty(Z, np.int32)
    val = np.empty(Z, np.float64)
    F = np.empty(N)
    M, ell, sigma, seed = kappa if kappa is not None else (0, 1.0, 0.0, 0)
    rc = lib().iga_assemble_elem(d, n, p, nq or p + 1, geom, int(with_boundary), M, ell, sigma, seed, fkind,
                                 _p(rowptr), _p(col), _p(val), _p(F))
    if rc != 0:
        raise ValueError("bad arguments")
    return rowptr, col, val, F


def l2_error_sine(d: int, n: int, p: int, coef: np.ndarray, nq: int | None = None) -> float:
    coef = np.ascontiguousarray(coef, np.float64)
    return float(lib().iga_l2_error_sine(d, n, p, nq or p + 3, _p(coef)))


def csr_apply(rowptr, col, val, x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    y = np.empty(len(rowptr) - 1)
    lib().iga_csr_apply(len(rowptr) - 1, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def kappa_points(M, ell, sigma, seed, pts: np.ndarray) -> np.ndarray:
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    out = np.empty(len(pts))
    lib().iga_kappa_points(M, ell, sigma, seed, len(pts), _p(pts), _p(out))
    return out


def geom_points(geom: int, d: int, xi: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    xi = np.ascontiguousarray(xi, np.float64).reshape(-1, d)
    x = np.empty_like(xi)
    det = np.empty(len(xi))
    lib().iga_geom_points(geom, d, len(xi), _p(xi), _p(x), _p(det))
    return x, det


def poisson_box(d: int, n: int, p: int) -> Problem:
    """-Laplace u = d pi^2 prod sin(pi x_k) on the unit box, Dirichlet u = 0."""
    rowptr, col, val = assemble_kron(d, n, p)
    F = load_sine(d, n, p)
    return Problem(len(rowptr) - 1, rowptr, col, val, F,
                   {"kind": "poisson_box", "d": d, "n": n, "p": p, "rhs": "sine"})


def poisson_box_random_rhs(d: int, n: int, p: int, seed: int, nrhs: int = 1) -> Problem:
    """Same matrix with F = K u_true, u_true ~ N(0,1) (column-major N x nrhs)."""
    rowptr, col, val = assemble_kron(d, n, p)
    N = len(rowptr) - 1
    U = rng_normal(seed, N * nrhs).reshape(nrhs, N)
    F = np.stack([csr_apply(rowptr, col, val, U[k]) for k in range(nrhs)])
    prob = Problem(N, rowptr, col, val, F[0] if nrhs == 1 else F,
                   {"kind": "poisson_box", "d": d, "n": n, "p": p, "rhs": "random", "seed": seed, "nrhs": nrhs})
    prob.u_true = U[0] if nrhs == 1 else U
    return prob


def batch_params(seed: int, count: int, degrees=(2, 3, 4), n_lo: int = 32, n_hi: int = 256) -> list[tuple[int, int]]:
    """(p, n) for each batch instance: p = degrees[z_{2k} mod 3],
    n = n_lo + z_{2k+1} mod (n_hi - n_lo + 1), z the SplitMix64(seed) stream."""
    z = splitmix64(seed, 2 * count)
    return [(degrees[z[2 * k] % len(degrees)], n_lo + z[2 * k + 1] % (n_hi - n_lo + 1)) for k in range(count)]


def batch_instances(seed: int = 20251126, count: int = 48, d: int = 2) -> list[Problem]:
    out = []
    for k, (p, n) in enumerate(batch_params(seed, count)):
        out.append(poisson_box_random_rhs(d, n, p, seed=seed + 1 + k))
        out[-1].meta["instance"] = k
    return out


# ------------------------------------- cube with mixed boundary conditions
def assemble_kron_box(n: int, p: int, lo, hi):
    """3-D unit cube stiffness restricted to the DOFs lo[k] <= i_k < hi[k]
    (full tensor indices per direction, x fastest)."""
    lo = np.ascontiguousarray(lo, np.int32)
    hi = np.ascontiguousarray(hi, np.int32)
    z = ctypes.c_int64()
    if lib().iga_kron_box_nnz(n, p, _p(lo), _p(hi), ctypes.byref(z)) != 0:
        raise ValueError("bad arguments")
    N = int(np.prod(hi - lo))
    rowptr = np.empty(N + 1, np.int64)
    col = np.empty(z.value, np.int32)
    val = np.empty(z.value, np.float64)
    if lib().iga_assemble_kron_box(n, p, _p(lo), _p(hi), _p(rowptr), _p(col), _p(val)) != 0:
        raise ValueError("assembly failed")
    return rowptr, col, val


def load_1d(n: int, p: int, g, nq: int | None = None) -> np.ndarray:
    """b_a = integral over [0, 1] of g(x) N_a(x) (Gauss, nq points per element)."""
    q = nq or p + 3
    gx, gw = gauss_legendre(q)
    b = np.zeros(n + p)
    for e in range(n):
        for t in range(q):
            x = (e + 0.5 * (gx[t] + 1.0)) / n
            v, _ = bspline_all(n, p, x)
            b += v * (g(x) * 0.5 * gw[t] / n)
    return b


def _apply_kron3(A, B, C, v):
    """(A (x) B (x) C) v for v indexed [z][y][x] (C acts on x, B on y, A on z)."""
    return np.einsum("ai,bj,ck,ijk->abc", A, B, C, v, optimize=True)


def cube_mixed_bc(n: int, p: int) -> Problem:
    """The paper's cube test case (Sec. 5): -Laplace u = f on [0,1]^3 with
    f = -exp(x+z) sin(y), Dirichlet data g_D = exp(x+z) sin(y) on x = 0,
    x = 1, y = 0 and Neumann data on y = 1 (exp(x+z) cos(y)), z = 0
    (-exp(x+z) sin(y)) and z = 1 (exp(x+z) sin(y)); exact solution
    u = exp(x+z) sin(y).  B-splines of degree p, maximal regularity, n
    elements per direction: (n+p-2)(n+p-1)(n+p) unknowns (x: both ends
    eliminated, y: one, z: none), the paper's matrix sizes.

    Non-homogeneous Dirichlet data by lifting: u_D = the L2 projection of
    g_D onto the tensor spline space (g_D is separable, so it is the tensor
    product of the 1-D projections), kept on the Dirichlet DOFs; the system
    is K_ff u_f = F_f - K_fD u_D with F = the load plus the Neumann face
    integrals (all separable products of 1-D integrals)."""
    nb = n + p
    K1, M1 = one_d_matrices(n, p)
    ex = load_1d(n, p, math.exp)
    sn = load_1d(n, p, math.sin)
    e_first, e_last = np.zeros(nb), np.zeros(nb)
    e_first[0], e_last[-1] = 1.0, 1.0  # the only basis functions nonzero at 0 and 1
    # load (f = -exp(x) sin(y) exp(z)) and Neumann terms; tensors indexed [z][y][x]
    F = -np.einsum("a,b,c->abc", ex, sn, ex)
    F += math.cos(1.0) * np.einsum("a,b,c->abc", ex, e_last, ex)       # y = 1: exp(x+z) cos(1)
    F += -np.einsum("a,b,c->abc", e_first, sn, ex)                    # z = 0: -exp(x) sin(y)
    F += math.e * np.einsum("a,b,c->abc", e_last, sn, ex)             # z = 1: exp(x+1) sin(y)
    # lifting: L2 projection of g_D = exp(x) sin(y) exp(z), kept on the Dirichlet DOFs
    import scipy.linalg as sl

    Px = sl.solve(M1, ex, assume_a="pos")
    Py = sl.solve(M1, sn, assume_a="pos")
    U = np.einsum("a,b,c->abc", Px, Py, Px)
    dmask = np.zeros((nb, nb, nb), bool)
    dmask[:, :, 0] = dmask[:, :, -1] = True  # x = 0, x = 1
    dmask[:, 0, :] = True                    # y = 0
    uD = np.where(dmask, U, 0.0)
    KuD = (_apply_kron3(M1, M1, K1, uD) + _apply_kron3(M1, K1, M1, uD)) + _apply_kron3(K1, M1, M1, uD)
    R = F - KuD
    lo, hi = (1, 1, 0), (nb - 1, nb, nb)  # kept index ranges in x, y, z
    rowptr, col, val = assemble_kron_box(n, p, lo, hi)
    Ff = np.ascontiguousarray(R[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].reshape(-1))
    prob = Problem(len(rowptr) - 1, rowptr, col, val, Ff,
                   {"kind": "cube_mixed_bc", "d": 3, "n": n, "p": p})
    prob.lift = uD
    prob.free = (lo, hi)
    return prob


def cube_mixed_bc_l2_error(prob: Problem, u_free: np.ndarray, nq: int | None = None) -> float:
    """||u_h - u||_L2 on the cube for u = exp(x+z) sin(y), u_h the spline
    with the free coefficients u_free and the lifting on the Dirichlet DOFs."""
    n, p = prob.meta["n"], prob.meta["p"]
    nb = n + p
    lo, hi = prob.free
    C = prob.lift.copy()
    C[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = np.asarray(u_free).reshape(hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])
    q = nq or p + 3
    gx, gw = gauss_legendre(q)
    pts = np.array([(e + 0.5 * (gx[t] + 1.0)) / n for e in range(n) for t in range(q)])
    wts = np.array([0.5 * gw[t] / n for e in range(n) for t in range(q)])
    B = np.stack([bspline_all(n, p, x)[0] for x in pts])  # [point][basis]
    uh = np.einsum("ai,bj,ck,ijk->abc", B, B, B, C, optimize=True)
    ue = np.einsum("a,b,c->abc", np.exp(pts), np.sin(pts), np.exp(pts))
    w3 = np.einsum("a,b,c->abc", wts, wts, wts)
    return float(np.sqrt(np.sum(w3 * (uh - ue) ** 2)))


# ----------------------------------------------- three-patch L-shape
# Patches (x offset, y offset) of the L-shaped cross-section: A = [0,1]^2,
# B = [-1,0]x[0,1], C = [0,1]x[-1,0]; each times [0,1] in z.
LSHAPE_PATCHES = ((0.0, 0.0), (-1.0, 0.0), (0.0, -1.0))


def _lshape_lattice_offsets(m):
    """Lattice offsets (gx, gy) of the patches A, B, C (see iga_gen.c)."""
    return ((m - 1, m - 1), (0, m - 1), (m - 1, 0))


def _lshape_u(x, y, z):
    return np.exp(x) * np.sin(x * y) * np.cos(z)


def _lshape_f(x, y, z):
    return np.exp(x) * np.cos(z) * (-2.0 * np.cos(x * y) * y + np.sin(x * y) * (y * y + x * x))


def _quad_1d(n, p, nq=None):
    q = nq or p + 3
    gx, gw = gauss_legendre(q)
    pts = np.array([(e + 0.5 * (gx[t] + 1.0)) / n for e in range(n) for t in range(q)])
    wts = np.array([0.5 * gw[t] / n for e in range(n) for t in range(q)])
    B = np.stack([bspline_all(n, p, x)[0] for x in pts])  # [point][basis]
    return pts, wts, B


def lshape_mixed_bc(n: int, p: int) -> Problem:
    """The paper's multipatch L-shaped test case (Sec. 2.3, Sec. 5): three
    conforming unit-cube patches forming an L in (x, y) (A = [0,1]^2,
    B = [-1,0]x[0,1], C = [0,1]x[-1,0]) times [0,1] in z, -Laplace u = f with
    the exact solution u = exp(x) sin(xy) cos(z); Dirichlet data on the four
    outer lateral faces and on z = 0, z = 1, Neumann data on the two
    re-entrant faces (x = 0 for y < 0: -du/dx; y = 0 for x < 0: -du/dy).
    Maximal regularity inside each patch, C^0 across the patch interfaces
    (shared interface functions).  Unknowns (m-2)(m-1)(3m-5), m = n + p: the
    paper's matrix sizes.  Dirichlet data by lifting (per-patch L2
    projection of g_D, kept on the Dirichlet functions)."""
    import scipy.linalg as sl

    m = n + p
    Lg = 2 * m - 1
    offs = _lshape_lattice_offsets(m)
    # lattice membership and the Dirichlet set (outer lateral edges; z = 0, 1)
    inL = np.zeros((Lg, Lg), bool)
    for ox, oy in offs:
        inL[oy:oy + m, ox:ox + m] = True
    keep2 = inL.copy()
    keep2[:, 0] = keep2[:, Lg - 1] = False   # x = -1 (B), x = 1 (A, C)
    keep2[0, :] = keep2[Lg - 1, :] = False   # y = -1 (C), y = 1 (A, B)
    # stiffness of the free functions
    nfree2 = int(keep2.sum())
    N = nfree2 * (m - 2)
    cap = N * (2 * p + 1) ** 3
    rowptr = np.empty(N + 1, np.int64)
    col = np.empty(cap, np.int32)
    val = np.empty(cap, np.float64)
    k2 = np.ascontiguousarray(keep2.astype(np.uint8).reshape(-1))
    if lib().iga_assemble_lshape(n, p, _p(k2), 1, m - 1, _p(rowptr), _p(col), _p(val), cap) != 0:
        raise ValueError("assembly failed")
    z = int(rowptr[-1])
    col, val = col[:z].copy(), val[:z].copy()
    # per-patch load of f and L2 projection of g_D; global tensors [z][gy][gx]
    K1, M1 = one_d_matrices(n, p)
    Minv = sl.inv(M1)
    pts, wts, B = _quad_1d(n, p)
    Fg = np.zeros((m, Lg, Lg))
    Ug = np.zeros((m, Lg, Lg))
    seen = np.zeros((m, Lg, Lg), bool)
    for (wx, wy), (ox, oy) in zip(LSHAPE_PATCHES, offs):
        X, Y, Z = np.meshgrid(pts + wx, pts + wy, pts, indexing="ij")  # [x][y][z]
        W = np.einsum("a,b,c->abc", wts, wts, wts)
        fq = np.transpose(_lshape_f(X, Y, Z) * W, (2, 1, 0))  # [z][y][x]
        gq = np.transpose(_lshape_u(X, Y, Z) * W, (2, 1, 0))
        Fg[:, oy:oy + m, ox:ox + m] += np.einsum("ci,bj,ak,ijk->cba", B.T, B.T, B.T, fq, optimize=True)
        proj = np.einsum("ci,bj,ak,ijk->cba", B.T, B.T, B.T, gq, optimize=True)
        proj = _apply_kron3(Minv, Minv, Minv, proj)
        sl_ = (slice(None), slice(oy, oy + m), slice(ox, ox + m))
        new = ~seen[sl_]
        Ug[sl_][new] = proj[new]
        seen[sl_] = True
    # Neumann data on the re-entrant faces
    Y2, Z2 = np.meshgrid(pts - 1.0, pts, indexing="ij")  # C's face x = 0: world y in [-1, 0]
    W2 = np.einsum("a,b->ab", wts, wts)
    gN = (-(Y2) * np.cos(Z2)) * W2                          # -du/dx at x = 0
    ox, oy = offs[2]
    Fg[:, oy:oy + m, ox] += np.einsum("cj,bi,ij->cb", B.T, B.T, gN, optimize=True)
    X2, Z2 = np.meshgrid(pts - 1.0, pts, indexing="ij")  # B's face y = 0: world x in [-1, 0]
    gN = (-X2 * np.exp(X2) * np.cos(Z2)) * W2                # -du/dy at y = 0
    ox, oy = offs[1]
    Fg[:, oy, ox:ox + m] += np.einsum("cj,ai,ij->ca", B.T, B.T, gN, optimize=True)
    # lifting: K u_D through the patches, then the free rows
    free = np.zeros((m, Lg, Lg), bool)
    free[1:m - 1] = keep2[None, :, :]
    uD = np.where(inL[None, :, :] & ~free, Ug, 0.0)
    KuD = np.zeros_like(uD)
    for ox, oy in offs:
        t = uD[:, oy:oy + m, ox:ox + m]
        KuD[:, oy:oy + m, ox:ox + m] += ((_apply_kron3(M1, M1, K1, t) + _apply_kron3(M1, K1, M1, t))
                                        + _apply_kron3(K1, M1, M1, t))
    R = Fg - KuD
    Ff = np.ascontiguousarray(R[free])  # z outermost, then y, then x: the assembly's numbering
    prob = Problem(N, rowptr, col, val, Ff, {"kind": "lshape_mixed_bc", "d": 3, "n": n, "p": p})
    prob.lift = uD
    prob.free_mask = free
    return prob


def lshape_mixed_bc_l2_error(prob: Problem, u_free: np.ndarray) -> float:
    """||u_h - u||_L2 over the three patches, u = exp(x) sin(xy) cos(z)."""
    n, p = prob.meta["n"], prob.meta["p"]
    m = n + p
    C = prob.lift.copy()
    C[prob.free_mask] = np.asarray(u_free)
    pts, wts, B = _quad_1d(n, p)
    W = np.einsum("a,b,c->abc", wts, wts, wts)
    err = 0.0
    for (wx, wy), (ox, oy) in zip(LSHAPE_PATCHES, _lshape_lattice_offsets(m)):
        uh = np.einsum("ai,bj,ck,ijk->abc", B, B, B, C[:, oy:oy + m, ox:ox + m], optimize=True)  # [z][y][x]
        Z, Y, X = np.meshgrid(pts, pts + wy, pts + wx, indexing="ij")
        err += float(np.sum(np.transpose(W, (2, 1, 0)) * (uh - _lshape_u(X, Y, Z)) ** 2))
    return math.sqrt(err)


ANNULUS_KAPPA = dict(M=256, ell=0.2, sigma=1.0)


def annulus_kappa(n: int, p: int, kappa_seed: int = 7, nq: int | None = None) -> Problem:
    """-div(kappa grad u) = 1 on the quarter annulus (radii 1, 2) x [0,1],
    homogeneous Dirichlet, kappa = exp(g) with g of correlation length 0.2,
    sigma = 1 (random Fourier features, M = 256)."""
    k = ANNULUS_KAPPA
    rowptr, col, val, F = assemble_elem(3, n, p, nq, geom=1, kappa=(k["M"], k["ell"], k["sigma"], kappa_seed), fkind=0)
    return Problem(len(rowptr) - 1, rowptr, col, val, F,
                   {"kind": "annulus_kappa", "d": 3, "n": n, "p": p, "kappa_seed": kappa_seed})


def annulus_volume() -> float:
    return 0.75 * math.pi


# ------------------------------------------------------------ network weights
# Block layout of the learned-damping network's flat weight vector (hidden
# width 32, 4 node features): (name, shape) in storage order.
MPNN_LAYOUT = [("W0", (32, 4)), ("b0", (32,)), ("U1", (32, 32)), ("V1", (32, 32)), ("b1", (32,)),
               ("U2", (32, 32)), ("V2", (32, 32)), ("b2", (32,)), ("q", (32,)), ("c", (1,)),
               ("qt", (32,)), ("ct", (1,))]
MPNN_NPARAM = sum(int(np.prod(s)) for _, s in MPNN_LAYOUT)


def mpnn_init_weights(seed: int = 1) -> np.ndarray:
    """Seeded initial weights (FP64): entry k of the flat vector is
    (2 U_k - 1) sqrt(3 / fan_in) with U_k draw k of SplitMix64(seed), fan_in
    the block's column count (32 for vectors); biases and c are zero and
    the output weights q and qt are scaled by 0.1, so omega starts near half
    its cap; ct = ln 2, so that the prolongator-smoothing weight theta
    starts near two thirds of its cap."""
    u = rng_u01(seed, MPNN_NPARAM) * 2.0 - 1.0
    out, o = [], 0
    for name, shape in MPNN_LAYOUT:
        k = int(np.prod(shape))
        fan = shape[1] if len(shape) == 2 else 32
        blk = u[o:o + k] * np.sqrt(3.0 / fan)
        if name in ("b0", "b1", "b2", "c"):
            blk = np.zeros(k)
        elif name == "ct":
            blk = np.full(k, np.log(2.0))
        elif name in ("q", "qt"):
            blk = blk * 0.1
        out.append(blk)
        o += k
    return np.concatenate(out)
