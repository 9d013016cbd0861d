"""Pins for the seeded input generator (IgA assembly, arXiv 2511.21268 Sec. 2).

Each check compares against something fixed independently of the code under
test: closed-form integrals, scipy's B-spline routines, partition of unity,
published RNG outputs, the O(h^{p+1}) approximation order.
"""
import math

import numpy as np
import pytest
import scipy.interpolate as si
import scipy.linalg as sl
import scipy.sparse.linalg as spl

from paper_2511_21268_gb300 import inputs as I
from tests.conftest import read_golden


def test_splitmix64_published_outputs():
    for seed, idx, val in read_golden("splitmix64.txt"):
        seed, idx = int(seed), int(idx)
        assert I.splitmix64(seed, idx + 1)[idx] == int(val, 16)
    # the C generator draws the same stream: u = (z >> 11) 2^-53
    z = I.splitmix64(1234567, 5)
    u = I.rng_u01(1234567, 5)
    assert np.array_equal(u, np.array([(v >> 11) * 2.0**-53 for v in z]))


def test_normal_draws_statistics():
    x = I.rng_normal(99, 200000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert abs(np.mean(x**4) - 3.0) < 0.05  # Gaussian kurtosis


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8])
def test_gauss_legendre_exact_degree(q):
    x, w = I.gauss_legendre(q)
    for k in range(2 * q):  # exact up to degree 2q-1
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x**k) - exact) < 1e-13
    # and not for degree 2q
    k = 2 * q
    assert abs(np.dot(w, x**k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("n,p", [(1, 1), (4, 2), (7, 3), (5, 4), (3, 6)])
def test_bspline_basis_matches_scipy(n, p):
    t = np.r_[np.zeros(p + 1), np.arange(1, n) / n, np.ones(p + 1)]
    rng = np.random.default_rng(n * 10 + p)
    for xi in rng.uniform(0, 1, 25):
        v, d = I.bspline_all(n, p, xi)
        ref_v = np.array([si.BSpline(t, np.eye(n + p)[i], p)(xi) for i in range(n + p)])
        ref_d = np.array([si.BSpline(t, np.eye(n + p)[i], p).derivative()(xi) for i in range(n + p)])
        assert np.allclose(v, ref_v, atol=1e-14)
        assert np.allclose(d, ref_d, atol=1e-11 * max(1, n * p))
        assert abs(v.sum() - 1.0) < 1e-14 and abs(d.sum()) < 1e-11 * n * p  # partition of unity
        assert (v >= -1e-15).all()


@pytest.mark.parametrize("n,p", [(6, 2), (9, 3), (5, 4)])
def test_1d_matrices_closed_forms(n, p):
    K1, M1 = I.one_d_matrices(n, p)
    t = np.r_[np.zeros(p + 1), np.arange(1, n) / n, np.ones(p + 1)]
    # int N_i = (t_{i+p+1} - t_i) / (p+1); sum_j M_ij = int N_i
    integrals = (t[p + 1:] - t[: n + p]) / (p + 1)
    assert np.allclose(M1.sum(axis=1), integrals, atol=1e-15)
    assert abs(M1.sum() - 1.0) < 1e-14
    assert np.abs(K1.sum(axis=1)).max() < 1e-12 * np.abs(K1).max()  # derivative of a constant
    assert np.array_equal(K1, K1.T) and np.array_equal(M1, M1.T)
    # exact quadrature: more points change nothing
    K2, M2 = I.one_d_matrices(n, p, nq=p + 4)
    assert np.allclose(K1, K2, rtol=0, atol=1e-13 * np.abs(K1).max())
    assert np.allclose(M1, M2, rtol=0, atol=1e-15)
    # bandwidth
    ii, jj = np.nonzero(M1)
    assert np.abs(ii - jj).max() == p


def test_sizes_closed_form():
    # N = (n+p-2)^d after eliminating the Dirichlet functions
    assert I.num_dofs(2, 32, 2) == 1024
    assert I.num_dofs(3, 64, 3) == 274625
    assert I.num_dofs(3, 96, 2) == 884736 and I.num_dofs(3, 48, 4) == 125000 and I.num_dofs(3, 48, 3) == 117649
    # nnz = (1-D band count)^d, band count m(2p+1) - p(p+1)
    for d, n, p in [(2, 32, 2), (3, 64, 3), (3, 96, 2), (3, 48, 4), (2, 256, 4)]:
        m = n + p - 2
        assert I.nnz(d, n, p) == (m * (2 * p + 1) - p * (p + 1)) ** d
    assert I.nnz(2, 32, 2) == 23716 and I.nnz(3, 64, 3) == 86938307
    # bandwidth statement: at most (2p+1)^d nonzeros per row
    rp, ci, v = I.assemble_kron(3, 8, 3)
    assert np.diff(rp).max() == 7**3


@pytest.mark.parametrize("d,n,p", [(2, 6, 2), (2, 5, 4), (3, 4, 2), (3, 3, 3)])
def test_assembly_symmetry_rowsums_spd(d, n, p):
    rp, ci, v = I.assemble_kron(d, n, p, with_boundary=True)
    A = np.zeros((len(rp) - 1,) * 2)
    for i in range(len(rp) - 1):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.array_equal(A, A.T)  # bitwise symmetric
    # pre-BC Laplacian annihilates constants (partition of unity)
    assert np.abs(A.sum(axis=1)).max() <= 1e-12 * np.abs(A).max()
    # after elimination: SPD (Cholesky succeeds)
    rp, ci, v = I.assemble_kron(d, n, p)
    B = np.zeros((len(rp) - 1,) * 2)
    for i in range(len(rp) - 1):
        B[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    assert np.array_equal(B, B.T)
    sl.cholesky(B)
    assert np.linalg.eigvalsh(B).min() > 0


@pytest.mark.parametrize("d,n,p", [(2, 5, 2), (2, 4, 3), (3, 3, 2), (3, 3, 3)])
def test_element_loop_equals_kronecker(d, n, p):
    rp, ci, v = I.assemble_kron(d, n, p)
    rp2, ci2, v2, F2 = I.assemble_elem(d, n, p)
    assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
    assert np.abs(v - v2).max() <= 1e-13 * np.abs(v).max()
    # load f = 1 before BCs integrates to the volume
    _, _, _, F = I.assemble_elem(d, n, p, with_boundary=True)
    assert abs(F.sum() - 1.0) < 1e-13


def test_annulus_geometry_and_volume():
    rng = np.random.default_rng(1)
    xi = rng.uniform(0, 1, (200, 3))
    x, det = I.geom_points(1, 3, xi)
    r = np.hypot(x[:, 0], x[:, 1])
    assert np.allclose(r, 1 + xi[:, 0], atol=1e-14)  # exact circle from the NURBS arc
    assert (x[:, :2] >= -1e-15).all() and (det > 0).all()
    assert np.allclose(x[:, 2], xi[:, 2])
    # |Omega| = 3 pi / 4: f = 1 load before BCs sums to the volume
    _, _, _, F = I.assemble_elem(3, 3, 2, nq=6, geom=1, with_boundary=True)
    assert abs(F.sum() - 0.75 * math.pi) < 1e-11
    # zero row sums survive the geometry map and a variable coefficient
    rp, ci, v, _ = I.assemble_elem(3, 3, 2, geom=1, with_boundary=True, kappa=(16, 0.2, 1.0, 7))
    rs = np.add.reduceat(v, rp[:-1])
    assert np.abs(rs).max() < 1e-12 * np.abs(v).max()


def test_kappa_field_statistics():
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, (4000, 3)) * 50.0  # far apart -> nearly independent samples
    g = np.log(I.kappa_points(256, 0.2, 1.0, 7, pts))
    assert abs(g.mean()) < 0.1 and abs(g.std() - 1.0) < 0.1
    # correlation length: nearby points are strongly correlated
    a = rng.uniform(0, 1, (2000, 3))
    b = a + np.array([0.02, 0, 0])
    ga = np.log(I.kappa_points(256, 0.2, 1.0, 7, a))
    gb = np.log(I.kappa_points(256, 0.2, 1.0, 7, b))
    assert np.corrcoef(ga, gb)[0, 1] > 0.95


@pytest.mark.parametrize("d,p,ns", [(2, 2, (8, 16, 32)), (2, 3, (8, 16, 32)), (3, 2, (4, 8, 12))])
def test_l2_convergence_order(d, p, ns):
    """Manufactured u = prod sin(pi x_k): ||u - u_h||_L2 = O(h^{p+1})."""
    errs = []
    for n in ns:
        prob = I.poisson_box(d, n, p)
        u = spl.spsolve(prob.to_scipy().tocsc(), prob.F)
        errs.append(I.l2_error_sine(d, n, p, u))
    slope = np.polyfit(np.log(1.0 / np.array(ns)), np.log(errs), 1)[0]
    assert abs(slope - (p + 1)) < 0.3, (errs, slope)


def test_batch_params_seeded():
    pn = I.batch_params(20251126, 48)
    assert len(pn) == 48
    assert all(p in (2, 3, 4) and 32 <= n <= 256 for p, n in pn)
    assert pn == I.batch_params(20251126, 48)
    assert len(set(p for p, _ in pn)) == 3


# ------------------------------------------------ mixed-BC cube (Sec. 5) ----
def test_cube_mixed_bc_sizes_are_the_papers():
    """(k+p)(k+p-1)(k+p-2) unknowns: the matrix sizes of the paper's Table 1
    (tests/golden/cube_table1.txt), computed without assembling."""
    from tests.conftest import read_golden

    for k, p, size, _, _ in read_golden("cube_table1.txt"):
        k, p, size = int(k), int(p), int(size)
        assert (k + p) * (k + p - 1) * (k + p - 2) == size
    prob = I.cube_mixed_bc(12, 3)
    assert prob.n == 2730
    K = prob.to_scipy()
    assert (K != K.T).nnz == 0  # bitwise symmetric
    assert np.all(np.diff(prob.rowptr) > 0)


@pytest.mark.parametrize("p", [2, 3])
def test_cube_mixed_bc_converges_at_order_p_plus_1(p):
    """The discrete solution (direct solve) approaches u = exp(x+z) sin(y)
    in L2 at rate p+1: the load, the three Neumann face integrals and the
    Dirichlet lifting are all right (a wrong sign or face breaks the rate)."""
    import scipy.sparse.linalg as spl

    errs = []
    ns = [4, 8, 16]
    for n in ns:
        prob = I.cube_mixed_bc(n, p)
        u = spl.spsolve(prob.to_scipy().tocsc(), prob.F)
        errs.append(I.cube_mixed_bc_l2_error(prob, u))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert errs[-1] < 1e-4
    assert abs(rates[-1] - (p + 1)) < 0.4, (errs, rates)


# --------------------------------------------- multipatch L-shape (Sec. 5) ----
def test_lshape_sizes_are_the_papers():
    """(m-2)(m-1)(3m-5) unknowns, m = k + p: the matrix sizes of the
    paper's multipatch L-shaped table (tests/golden/lshape_table2.txt)."""
    from tests.conftest import read_golden

    for row in read_golden("lshape_table2.txt"):
        k, p, size = int(row[0]), int(row[1]), int(row[2])
        m = k + p
        ours = (m - 2) * (m - 1) * (3 * m - 5)
        if len(row) > 5 and row[5] == "misprint":
            # printed value off in at most two digits of the same length
            a, b = str(ours), str(size)
            assert len(a) == len(b) and sum(x != y for x, y in zip(a, b)) <= 2, (k, p, size, ours)
        else:
            assert ours == size, (k, p, size, ours)
    prob = I.lshape_mixed_bc(12, 2)
    assert prob.n == 5772
    K = prob.to_scipy()
    assert (K != K.T).nnz == 0
    # SPD: the smallest eigenvalue of a small case is positive
    small = I.lshape_mixed_bc(3, 2).to_scipy().toarray()
    assert np.linalg.eigvalsh(small).min() > 0


@pytest.mark.parametrize("p", [2, 3])
def test_lshape_converges_at_order_p_plus_1(p):
    """Three conforming patches with shared interface functions (C^0 across
    the interfaces), Dirichlet lifting, Neumann data on the re-entrant
    faces: the discrete solution approaches exp(x) sin(xy) cos(z) in L2 at
    rate p+1 (a wrong interface identification, face or sign breaks it)."""
    errs = []
    for n in (4, 8, 16):
        prob = I.lshape_mixed_bc(n, p)
        u = spl.spsolve(prob.to_scipy().tocsc(), prob.F)
        errs.append(I.lshape_mixed_bc_l2_error(prob, u))
    rate = np.log2(errs[-2] / errs[-1])
    assert abs(rate - (p + 1)) < 0.4, (errs, rate)
