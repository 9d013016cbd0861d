"""Pins of the assembly oracle (oracle/iga.py) against facts the paper and
the mathematics fix: a library B-spline routine, the closed-form trilinear
element, the Kronecker structure of the cube, partition of unity, exactly
represented linear fields, the exact quarter circle, and an independent
polar-coordinate quadrature of the coefficient."""
import math

import numpy as np
import pytest

from oracle import iga


@pytest.mark.parametrize("n,p", [(1, 1), (3, 2), (5, 3), (4, 4)])
def test_bspline_matches_scipy(n, p):
    from scipy.interpolate import BSpline

    t = iga.knots(n, p)
    rng = np.random.default_rng(3)
    for x in np.concatenate([rng.uniform(0, 1, 9), [0.0, 0.5, 0.999999]]):
        v, d = iga.bspline(n, p, float(x))
        for i in range(n + p):
            c = np.zeros(n + p)
            c[i] = 1.0
            s = BSpline(t, c, p)
            assert abs(v[i] - s(x)) < 1e-14
            assert abs(d[i] - s.derivative()(x)) < 1e-12 * max(1, n * p)


def test_trilinear_element_closed_form():
    """n = 1, p = 1 on the unit cube: the trilinear Laplacian element,
    1/3 on the diagonal, 0 between edge neighbours, -1/12 between face- and
    body-diagonal corners; f = 1 loads 1/8 per corner."""
    K, F = iga.Patch(1, 1, geom="cube", with_boundary=True).assemble()
    for a in range(8):
        for b in range(8):
            ham = bin(a ^ b).count("1")
            want = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[ham]
            assert abs(K[a, b] - want) < 1e-15
    assert np.allclose(F, 1 / 8, rtol=0, atol=1e-16)


def _scipy_1d(n, p):
    """1-D stiffness and mass of the n+p B-splines from scipy's B-splines and
    a 20-point Gauss rule per element (exact for these polynomials)."""
    from scipy.interpolate import BSpline

    t = iga.knots(n, p)
    x, w = np.polynomial.legendre.leggauss(20)
    A = np.zeros((n + p, n + p))
    M = np.zeros((n + p, n + p))
    fns = []
    for i in range(n + p):
        c = np.zeros(n + p)
        c[i] = 1.0
        s = BSpline(t, c, p)
        fns.append((s, s.derivative()))
    for e in range(n):
        xe = (e + 0.5 * (x + 1)) / n
        we = 0.5 * w / n
        V = np.array([f(xe) for f, _ in fns])
        D = np.array([g(xe) for _, g in fns])
        A += (D * we) @ D.T
        M += (V * we) @ V.T
    return A, M


@pytest.mark.parametrize("n,p", [(2, 1), (3, 2), (2, 3)])
def test_cube_equals_kronecker_sum(n, p):
    K, F = iga.Patch(n, p, geom="cube", with_boundary=True).assemble()
    A, M = _scipy_1d(n, p)
    Kk = np.kron(M, np.kron(M, A)) + np.kron(M, np.kron(A, M)) + np.kron(A, np.kron(M, M))
    assert np.abs(K - Kk).max() < 1e-13 * np.abs(Kk).max()
    m1 = M.sum(axis=1)  # int B_i
    assert np.abs(F - np.kron(m1, np.kron(m1, m1))).max() < 1e-15


def test_arc_is_the_exact_quarter_circle():
    for t in np.linspace(0, 1, 17):
        c, dc = iga.arc(float(t))
        assert abs(np.hypot(*c) - 1.0) < 1e-15
        assert abs(c @ dc) < 1e-14  # tangent
    assert np.allclose(iga.arc(0.0)[0], [1, 0], atol=0)
    assert np.allclose(iga.arc(1.0)[0], [0, 1], atol=0)
    assert np.allclose(iga.arc(0.5)[0], [math.sqrt(0.5)] * 2, atol=1e-16)
    # length of the arc: int_0^1 |c'(t)| dt = pi / 2
    x, w = np.polynomial.legendre.leggauss(40)
    L = sum(0.5 * wi * np.hypot(*iga.arc(0.5 * (xi + 1))[1]) for xi, wi in zip(x, w))
    assert abs(L - math.pi / 2) < 1e-13


def _kappa_params(M, seed=5, ell=0.2):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(M, 3)) / ell, rng.uniform(0, 2 * math.pi, M)


@pytest.mark.parametrize("geom,M", [("cube", 0), ("annulus", 0), ("annulus", 6)])
def test_partition_of_unity_zero_row_sums(geom, M):
    om, ph = _kappa_params(M) if M else (None, None)
    P = iga.Patch(2, 2, geom=geom, with_boundary=True, omega=om, phi=ph, sigma=1.0)
    K, F = P.assemble()
    assert np.abs(K.sum(axis=1)).max() < 1e-13 * np.abs(K).max()
    assert np.array_equal(K, K.T)
    vol = 1.0 if geom == "cube" else 0.75 * math.pi
    if M == 0:
        assert abs(F.sum() - vol) < 1e-6 * vol


def test_annulus_linear_fields_energy():
    """xi1 (the radius minus 1) and xi3 (= z) are in the space (Greville
    coefficients); with kappa = 1 their energies are the volume 3 pi / 4 and
    their gradients are orthogonal."""
    n, p = 3, 3
    K, _ = iga.Patch(n, p, geom="annulus", with_boundary=True).assemble()
    g = iga.greville(n, p)
    one = np.ones(n + p)
    c1 = np.kron(one, np.kron(one, g))
    c3 = np.kron(g, np.kron(one, one))
    vol = 0.75 * math.pi
    assert abs(c1 @ K @ c1 - vol) < 1e-7 * vol  # Gauss error of int |c'(t)| dt only
    assert abs(c3 @ K @ c3 - vol) < 1e-7 * vol
    assert abs(c1 @ K @ c3) < 1e-13


def test_annulus_kappa_integral_against_polar_quadrature():
    """u = z has energy int kappa dOmega; compare with a tensor Gauss rule
    in polar coordinates (r, angle, z), which does not use the NURBS map.
    With 8 Gauss points per element direction the NURBS-side rule is within
    1e-9 (its error falls from 1e-5 at 4 points to 2e-10 at 8)."""
    om, ph = _kappa_params(4, seed=11, ell=0.5)
    n, p = 4, 3
    P = iga.Patch(n, p, nq=8, geom="annulus", with_boundary=True, omega=om, phi=ph, sigma=0.5)
    K, _ = P.assemble()
    g = iga.greville(n, p)
    one = np.ones(n + p)
    c3 = np.kron(g, np.kron(one, one))
    x, w = np.polynomial.legendre.leggauss(24)
    tot = 0.0
    for r, wr in zip(1.5 + 0.5 * x, 0.5 * w):
        for a, wa in zip(math.pi / 4 * (x + 1), math.pi / 4 * w):
            for z, wz in zip(0.5 * (x + 1), 0.5 * w):
                tot += wr * wa * wz * r * iga.kappa(np.array([r * math.cos(a), r * math.sin(a), z]), om, ph, 0.5)
    assert abs(c3 @ K @ c3 - tot) < 1e-8 * tot


def test_elimination_and_rows_agree_with_full_matrix():
    om, ph = _kappa_params(3)
    kw = dict(geom="annulus", omega=om, phi=ph, sigma=1.0)
    Kb, Fb = iga.Patch(3, 2, with_boundary=True, **kw).assemble()
    P = iga.Patch(3, 2, with_boundary=False, **kw)
    K, F = P.assemble()
    m, mb = P.m, 5
    keep = [i1 + mb * (i2 + mb * i3) for i3 in range(1, 4) for i2 in range(1, 4) for i1 in range(1, 4)]
    assert np.array_equal(K, Kb[np.ix_(keep, keep)])
    assert np.array_equal(F, Fb[keep])
    for I in (0, 13, m ** 3 - 1):
        row, f = P.row(I)
        dense = np.zeros(m ** 3)
        for j, v in row.items():
            dense[j] = v
        assert np.abs(dense - K[I]).max() < 1e-15 * np.abs(K[I]).max()
        assert abs(f - F[I]) < 1e-16


def test_sine_source_integral():
    """sum_i F_i with all functions kept is int f = 3 pi^2 (2 / pi)^3 = 24 / pi."""
    _, F = iga.Patch(3, 3, nq=8, geom="cube", with_boundary=True, src="sine").assemble()
    assert abs(F.sum() - 24 / math.pi) < 1e-9


def test_oracle_matches_the_input_generators_element_loop():
    """Two independent element loops (the oracle here, the input generator's
    C code) on the annulus with the generator's random Fourier features."""
    from paper_2511_21268_gb300 import inputs

    n, p, seed = 3, 2, 7
    M, ell, sigma = 16, 0.2, 1.0
    om = inputs.rng_normal(seed, 3 * M).reshape(M, 3) / ell
    ph = inputs.rng_u01(seed + 1, M) * 2 * math.pi
    rp, ci, va, F = inputs.assemble_elem(3, n, p, geom=1, kappa=(M, ell, sigma, seed), fkind=0)
    K, Fo = iga.Patch(n, p, geom="annulus", omega=om, phi=ph, sigma=sigma).assemble()
    dense = np.zeros_like(K)
    for i in range(len(rp) - 1):
        dense[i, ci[rp[i]:rp[i + 1]]] = va[rp[i]:rp[i + 1]]
    assert np.array_equal(dense != 0, K != 0)
    assert np.abs(dense - K).max() < 1e-13 * np.abs(K).max()
    assert np.abs(F - Fo).max() < 1e-15
