"""Pins for the CPU oracle (arXiv 2511.21268, Sec. 3, 3.1, 3.2).

The oracle is checked against facts fixed outside it: the paper's worked
matching example (Fig. 2), brute force on tiny graphs, the characterisation
of the greedy matching under a strict order, Cauchy-Schwarz bounds on c_ij,
orthonormality of the tentative prolongator, dense linear algebra from
numpy/scipy, the textbook two-grid error propagator and V-cycle symmetry.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spl

import oracle as O
from paper_2511_21268_gb300 import inputs as I
from tests.conftest import read_golden


def dense(rp, ci, v):
    n = len(rp) - 1
    A = np.zeros((n, n))
    for i in range(n):
        A[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
    return A


def to_csr(A):
    rp, ci, v = [0], [], []
    for i in range(A.shape[0]):
        nz = np.nonzero(A[i])[0]
        ci += list(nz)
        v += list(A[i, nz])
        rp.append(len(ci))
    return np.array(rp, np.int64), np.array(ci, np.int32), np.array(v)


def brute_force_max_product(n, edges):
    """All matchings of a tiny graph; returns (best product, best edge set)."""
    best = (1.0, ())
    for r in range(1, n // 2 + 1):
        for sub in itertools.combinations(range(len(edges)), r):
            verts = [v for e in sub for v in edges[e][:2]]
            if len(set(verts)) < len(verts):
                continue
            prod = np.prod([edges[e][2] for e in sub])
            if prod > best[0]:
                best = (prod, tuple(sorted((edges[e][0], edges[e][1]) for e in sub)))
    return best


def order_key(c, lo, hi):
    return (-c, lo, hi)


def is_greedy_matching(n, edges, mate):
    """Greedy matching under a strict order <=> (1) valid matching and
    (2) every unmatched edge touches a heavier matched edge."""
    for i in range(n):
        if mate[i] >= 0 and mate[mate[i]] != i:
            return False
    matched = {(min(i, mate[i]), max(i, mate[i])) for i in range(n) if mate[i] >= 0}
    wt = {(lo, hi): c for lo, hi, c in edges}
    for lo, hi in matched:
        if (lo, hi) not in wt:
            return False
    for lo, hi, c in edges:
        if (lo, hi) in matched:
            continue
        ok = False
        for v in (lo, hi):
            if mate[v] >= 0:
                e = (min(v, mate[v]), max(v, mate[v]))
                if order_key(wt[e], *e) < order_key(c, lo, hi):
                    ok = True
        if not ok:
            return False
    return True


# ------------------------------------------------------------ Fig. 2 ----
def test_fig2_worked_example():
    rows = read_golden("fig2_matching.txt")
    edges = [(int(r[0]), int(r[1]), float(r[2])) for r in rows if r[0].isdigit()]
    exp = {r[0]: r[1:] for r in rows if not r[0].isdigit()}
    best, M = brute_force_max_product(4, edges)
    assert best == float(exp["max_product_matching"][-1])
    assert M == tuple(tuple(int(x) for x in s.split("-")) for s in exp["max_product_matching"][:-1])
    lo, hi, c = zip(*edges)
    mate = O.match_greedy_edges(4, lo, hi, c)
    got = sorted({(min(i, int(mate[i])), max(i, int(mate[i]))) for i in range(4)})
    want = [tuple(int(x) for x in s.split("-")) for s in exp["greedy_matching"][:-1]]
    assert got == want
    assert np.prod([dict(((a, b), w) for a, b, w in edges)[e] for e in got]) == float(exp["greedy_matching"][-1])


@pytest.mark.parametrize("seed", range(12))
def test_greedy_matching_properties_random_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 9))
    edges = [(i, j, float(rng.choice([0.5, 1.0, 1.5, 2.0, rng.uniform(0.1, 3)])))
             for i in range(n) for j in range(i + 1, n) if rng.random() < 0.6]
    if not edges:
        return
    lo, hi, c = zip(*edges)
    mate = O.match_greedy_edges(n, lo, hi, c)
    assert is_greedy_matching(n, edges, mate)
    # maximal: no edge with both ends free
    assert all(mate[a] >= 0 or mate[b] >= 0 for a, b, _ in edges)
    # 1/2-approximation of the maximum weight (sum of log c for log c >= 0)
    pos = [(a, b, w) for a, b, w in edges if w >= 1.0]
    if pos:
        lo, hi, c = zip(*pos)
        m2 = O.match_greedy_edges(n, lo, hi, c)
        got = sum(np.log(w) for a, b, w in pos if m2[a] == b)
        best = np.log(brute_force_max_product(n, pos)[0])
        assert got >= 0.5 * best - 1e-12


# ------------------------------------------------------- edge weights ----
def test_edge_weight_closed_forms():
    # K_e = [[2,-1],[-1,2]], w = (1,1): c = 1 - 2(-1)/(2+2) = 3/2
    assert O.edge_weight(-1.0, 2.0, 2.0, 1.0, 1.0) == 1.5
    # w orthogonal-ish: w = (1,-1) -> c = 1 - 2(-1)(-1)/4 = 1/2
    assert O.edge_weight(-1.0, 2.0, 2.0, 1.0, -1.0) == 0.5
    # unequal diagonals: k=-1, k_lolo=2, k_hihi=4, w=(1,2): 1 - (-4)/(2 + 16) = 11/9
    assert abs(O.edge_weight(-1.0, 2.0, 4.0, 1.0, 2.0) - 11.0 / 9.0) < 1e-16
    # w_j = 0 -> c = 1
    assert O.edge_weight(-1.0, 2.0, 2.0, 1.0, 0.0) == 1.0
    # explicit zero coupling and w = 0 are not edges
    assert O.edge_weight(0.0, 2.0, 2.0, 1.0, 1.0) is None
    assert O.edge_weight(-1.0, 2.0, 2.0, 0.0, 0.0) is None


def test_edge_weight_cauchy_schwarz_on_iga():
    prob = I.poisson_box(2, 8, 3)
    w = O.test_vector(prob.rowptr, prob.col, prob.val)
    dg = prob.to_scipy().diagonal()
    cs = []
    for i in range(prob.n):
        for k in range(prob.rowptr[i], prob.rowptr[i + 1]):
            j = prob.col[k]
            if j > i:
                c = O.edge_weight(prob.val[k], dg[i], dg[j], w[i], w[j])
                if c is not None:
                    cs.append(c)
    cs = np.array(cs)
    assert (cs > 0).all() and (cs < 2).all()  # |k_ij| < sqrt(k_ii k_jj) for SPD K
    assert (cs > 1).any() and (cs < 1).any()  # IgA matrices have couplings of both signs


# ----------------------------------------------------- l1 / smoother ----
def test_l1_diag_dominates_and_smoother_contracts():
    prob = I.poisson_box(2, 6, 3)
    K = prob.to_scipy().toarray()
    d, rc = O.l1_diag(prob.rowptr, prob.col, prob.val)
    assert rc == 0
    # D - K is positive semidefinite (weak diagonal dominance) -> eig(D^-1 K) in (0, 1]
    ev = np.linalg.eigvals(K / d[:, None]).real
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12
    # error propagator I - D^-1 K has K-norm < 1
    E = np.eye(len(d)) - K / d[:, None]
    Lk = np.linalg.cholesky(K)
    assert np.linalg.norm(Lk.T @ E @ np.linalg.inv(Lk.T), 2) < 1
    # a nonpositive diagonal is reported
    v = prob.val.copy()
    v[prob.rowptr[3] + list(prob.col[prob.rowptr[3]:prob.rowptr[4]]).index(3)] = 0.0
    assert O.l1_diag(prob.rowptr, prob.col, v)[1] == -2


def tridiag(n):
    """CSR of tridiag(-1, 2, -1) (1-D linear finite elements, h = 1)."""
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return to_csr(T)


def test_l1_diag_closed_forms():
    """d_i = k_ii + sum_{j != i} |k_ij| (Sec. 3.2) on matrices whose l1
    diagonal is known by hand: tridiag(-1, 2, -1) gives (3, 4, ..., 4, 3);
    the 5-point Laplacian on a 3 x 3 grid gives 6 at corners, 7 on edges,
    8 in the centre; a row with entries of both signs adds their moduli
    (a double-counted k_ii or a signed sum would fail each of these)."""
    d, rc = O.l1_diag(*tridiag(7))
    assert rc == 0 and np.array_equal(d, [3.0, 4.0, 4.0, 4.0, 4.0, 4.0, 3.0])
    T = 2.0 * np.eye(3) - np.eye(3, k=1) - np.eye(3, k=-1)
    L2 = np.kron(T, np.eye(3)) + np.kron(np.eye(3), T)
    d, rc = O.l1_diag(*to_csr(L2))
    assert rc == 0 and np.array_equal(d, [6.0, 7.0, 6.0, 7.0, 8.0, 7.0, 6.0, 7.0, 6.0])
    A = np.array([[4.0, -0.5, 0.25, -1.0], [-0.5, 3.0, 0.0, 0.125], [0.25, 0.0, 2.0, 0.0], [-1.0, 0.125, 0.0, 5.0]])
    d, rc = O.l1_diag(*to_csr(A))
    assert rc == 0 and np.array_equal(d, [5.75, 3.625, 2.25, 6.125])


def test_test_vector_sweeps_closed_form():
    """Test-vector relaxation w <- w - D_l1^-1 K w (Sec. 3.1 with the
    smoother of Sec. 3.2) from w0 = 1 on tridiag(-1, 2, -1): K w0 =
    (1, 0, ..., 0, 1), so one sweep gives (2/3, 1, ..., 1, 2/3); the second
    gives (5/9, 11/12, 1, ..., 1, 11/12, 5/9).  Dividing by k_ii = 2 instead
    of d_i, or sweeping in place (Gauss-Seidel order), changes both."""
    rp, ci, v = tridiag(8)
    w1 = O.test_vector(rp, ci, v, kind=1, sweeps=1)
    assert np.allclose(w1, [2 / 3, 1, 1, 1, 1, 1, 1, 2 / 3], rtol=0, atol=1e-15)
    w2 = O.test_vector(rp, ci, v, kind=1, sweeps=2)
    assert np.allclose(w2, [5 / 9, 11 / 12, 1, 1, 1, 1, 11 / 12, 5 / 9], rtol=0, atol=1e-15)
    # 2-D: the 5-point Laplacian on a 4 x 4 grid from w0 = 1.  (K 1)_i is
    # the number of eliminated neighbours: 2 at corners (d = 6), 1 on edges
    # (d = 7), 0 inside, so w1 = 1 - 2/6 at corners and 1 - 1/7 on edges.
    T = 2.0 * np.eye(4) - np.eye(4, k=1) - np.eye(4, k=-1)
    L2 = np.kron(T, np.eye(4)) + np.kron(np.eye(4), T)
    w1 = O.test_vector(*to_csr(L2), kind=1, sweeps=1).reshape(4, 4)
    expect = np.array([[2 / 3, 6 / 7, 6 / 7, 2 / 3], [6 / 7, 1, 1, 6 / 7], [6 / 7, 1, 1, 6 / 7],
                       [2 / 3, 6 / 7, 6 / 7, 2 / 3]])
    assert np.allclose(w1, expect, rtol=0, atol=1e-15)


def test_test_vector_start_and_smoothing():
    prob = I.poisson_box(2, 10, 2)
    w0 = O.test_vector(prob.rowptr, prob.col, prob.val, seed=5, sweeps=0)
    assert np.array_equal(w0, I.rng_u01(5, prob.n))  # SplitMix64 draws, independent implementation
    K = prob.to_scipy()
    energies = []
    for s in range(5):
        w = O.test_vector(prob.rowptr, prob.col, prob.val, seed=5, sweeps=s)
        energies.append(w @ (K @ w) / (w @ w))
    assert all(a > b for a, b in zip(energies, energies[1:]))  # Rayleigh quotient drops: smoother w
    assert np.array_equal(O.test_vector(prob.rowptr, prob.col, prob.val, kind=1, sweeps=0), np.ones(prob.n))


# --------------------------------------------------- aggregation / P ----
@pytest.mark.parametrize("d,n,p", [(2, 10, 2), (3, 5, 3)])
def test_prolongator_orthonormal_and_galerkin(d, n, p):
    prob = I.poisson_box(d, n, p)
    w = O.test_vector(prob.rowptr, prob.col, prob.val)
    mate = O.match_greedy(prob.rowptr, prob.col, prob.val, w)
    assert all(mate[mate[i]] == i for i in range(prob.n) if mate[i] >= 0)
    agg, pval, nc = O.aggregate(mate, w)
    P = np.zeros((prob.n, nc))
    P[np.arange(prob.n), agg] = pval
    assert np.abs(P.T @ P - np.eye(nc)).max() < 1e-15  # orthonormal columns
    assert np.bincount(agg).max() <= 2
    wc = O.restrict(agg, pval, w, nc)
    assert np.abs(P @ wc - w).max() < 1e-15 * np.abs(w).max() * 4  # w lies in range(P)
    # coarse numbering by the smallest fine index
    first = np.full(nc, -1)
    for i in range(prob.n - 1, -1, -1):
        first[agg[i]] = i
    assert (np.diff(first) > 0).all()
    # Galerkin product equals the dense triple product, bitwise symmetric
    rpc, cic, vc = O.galerkin(prob.rowptr, prob.col, prob.val, agg, pval, nc)
    Kc = dense(rpc, cic, vc)
    K = prob.to_scipy().toarray()
    assert np.array_equal(Kc, Kc.T)
    assert np.abs(Kc - P.T @ K @ P).max() < 1e-13 * np.abs(K).max()
    x = np.random.default_rng(0).standard_normal(nc)
    assert abs(x @ Kc @ x - (P @ x) @ K @ (P @ x)) < 1e-12 * abs(x @ Kc @ x)
    np.linalg.cholesky(Kc)  # SPD


def test_hierarchy_levels_spd_and_opc():
    prob = I.poisson_box(3, 8, 2)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    sizes = [H.level_n(l) for l in range(H.num_levels)]
    assert sizes[0] == prob.n and sizes[-1] <= 20
    assert all(b * 4 >= a for a, b in zip(sizes, sizes[1:]))  # two passes: aggregates of <= 4
    nnzs = [H.level_nnz(l) for l in range(H.num_levels)]
    assert abs(H.opc - sum(nnzs) / nnzs[0]) < 1e-15
    for l in range(H.num_levels):
        A = dense(*H.level_csr(l))
        assert np.array_equal(A, A.T)
        np.linalg.cholesky(A)
    for l in range(H.num_levels - 1):
        agg, pv = H.level_map(l)
        assert np.bincount(agg).max() <= 4
        P = np.zeros((sizes[l], sizes[l + 1]))
        P[np.arange(sizes[l]), agg] = pv
        assert np.abs(P.T @ P - np.eye(sizes[l + 1])).max() < 1e-14
        A, Ac = dense(*H.level_csr(l)), dense(*H.level_csr(l + 1))
        assert np.abs(Ac - P.T @ A @ P).max() < 1e-12 * np.abs(A).max()
    L = H.coarse_chol()
    Ac = dense(*H.level_csr(H.num_levels - 1))
    assert np.allclose(L, np.linalg.cholesky(Ac), rtol=0, atol=1e-13 * np.abs(Ac).max())


def test_cholesky_against_numpy():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 30 * np.eye(30)
    L, rc = O.cholesky(A)
    assert rc == 0 and np.allclose(L, np.linalg.cholesky(A), atol=1e-13)
    b = rng.standard_normal(30)
    assert np.allclose(O.chol_solve(L, b), np.linalg.solve(A, b), atol=1e-13)
    A[5, 5] = -1.0
    assert O.cholesky(A)[1] == -2


# ------------------------------------------------------------ V-cycle ----
def test_two_grid_matches_textbook_error_propagator():
    """B = (I - E) K^-1 with E = (I - M K)(I - P Kc^-1 P^T K)(I - M K)."""
    prob = I.poisson_box(2, 7, 2)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=prob.n - 1, max_levels=2)
    assert H.num_levels == 2
    K = prob.to_scipy().toarray()
    d, _ = H.level_vectors(0)
    agg, pv = H.level_map(0)
    nc = H.level_n(1)
    P = np.zeros((prob.n, nc))
    P[np.arange(prob.n), agg] = pv
    Kc = P.T @ K @ P
    M = np.diag(1.0 / d)
    Id = np.eye(prob.n)
    S = Id - M @ K
    E = S @ (Id - P @ np.linalg.solve(Kc, P.T @ K)) @ S
    B = (Id - E) @ np.linalg.inv(K)
    Bo = np.column_stack([H.vcycle(e) for e in np.eye(prob.n)])
    assert np.abs(Bo - B).max() < 1e-11 * np.abs(B).max()


@pytest.mark.parametrize("d,n,p", [(2, 12, 2), (3, 6, 3)])
def test_vcycle_symmetric_positive_definite(d, n, p):
    prob = I.poisson_box(d, n, p)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30)
    assert H.num_levels >= 3
    rng = np.random.default_rng(1)
    for _ in range(5):
        x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
        bx, by = H.vcycle(x), H.vcycle(y)
        assert abs(x @ by - y @ bx) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(bx) * 10
        assert x @ bx > 0


# -------------------------------------------------------------- Krylov ----
def test_pcg_against_direct_solve():
    prob = I.poisson_box(3, 5, 3)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=10)
    out = H.pcg(prob.F, rtol=1e-14, itmax=500)
    u = spl.spsolve(prob.to_scipy().tocsc(), prob.F)
    assert out["status"] == 0
    assert np.linalg.norm(out["u"] - u) <= 1e-11 * np.linalg.norm(u)
    fl = H.pcg(prob.F, rtol=1e-14, itmax=500, flexible=True)
    assert np.linalg.norm(fl["u"] - u) <= 1e-11 * np.linalg.norm(u)


def test_pcg_exact_preconditioner_one_iteration():
    prob = I.poisson_box(2, 8, 2)  # 64 unknowns, coarsest level = the matrix itself
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=1000)
    assert H.num_levels == 1
    out = H.pcg(prob.F, rtol=1e-12)
    assert out["iters"] == 1 and out["relres"] < 1e-13


def test_pcg_and_fcg_same_iterates_for_fixed_preconditioner():
    prob = I.poisson_box(2, 20, 3)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    a = H.pcg(prob.F, rtol=1e-10, history=True)
    b = H.pcg(prob.F, rtol=1e-10, flexible=True, history=True)
    assert abs(a["iters"] - b["iters"]) <= 1
    k = min(a["iters"], b["iters"])
    assert np.allclose(a["history"][:k], b["history"][:k], rtol=1e-6)
    assert a["relres"] <= 1e-10 * 1.01 and b["relres"] <= 1e-10 * 1.01


def test_pcg_warm_start_and_zero_rhs():
    prob = I.poisson_box(2, 10, 2)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val)
    a = H.pcg(prob.F, rtol=1e-10)
    b = H.pcg(prob.F, x0=a["u"], rtol=1e-10)
    assert b["iters"] == 0
    z = H.pcg(np.zeros(prob.n), rtol=1e-10)
    assert z["iters"] == 0 and not z["u"].any()


def test_full_pipeline_discretisation_order():
    """PCG-AMG solutions converge like O(h^{p+1}) to the manufactured solution."""
    errs, ns = [], (6, 12, 24)
    for n in ns:
        prob = I.poisson_box(2, n, 2)
        H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
        out = H.pcg(prob.F, rtol=1e-12)
        errs.append(I.l2_error_sine(2, n, 2, out["u"]))
    slope = np.polyfit(np.log(1.0 / np.array(ns)), np.log(errs), 1)[0]
    assert abs(slope - 3) < 0.3


def test_setup_deterministic():
    prob = I.poisson_box(3, 6, 2)
    A = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    B = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20)
    for l in range(A.num_levels):
        for a, b in zip(A.level_csr(l), B.level_csr(l)):
            assert np.array_equal(a, b)


def test_solve_phase_threads_do_not_change_results():
    """The solve phase's row loops may run on several threads; each row's
    sum and every dot product are evaluated as in the sequential code, so
    the iterates are bitwise the same."""
    prob = I.poisson_box(3, 8, 3)
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30)
    O.set_threads(1)
    a = H.pcg(prob.F, rtol=1e-10)
    got = O.set_threads(4)
    try:
        b = H.pcg(prob.F, rtol=1e-10)
    finally:
        O.set_threads(1)
    assert got in (1, 4)
    assert a["iters"] == b["iters"] and np.array_equal(a["u"].view(np.uint64), b["u"].view(np.uint64))


# ------------------------------------------------- smoothed prolongator ----
def _tentative(prob, **kw):
    H = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, **kw)
    d, _ = H.level_vectors(0)
    agg, pv = H.level_map(0)
    return H, d, agg, pv


@pytest.mark.parametrize("d,n,p", [(2, 8, 2), (2, 6, 3), (3, 4, 2)])
def test_smoothed_prolongator_and_galerkin_against_dense(d, n, p):
    """P_bar = (I - diag(theta) D^-1 K) P (Sec. 3.1 "Variants") and K_c =
    P_bar^T K P_bar against dense numpy products, per-row theta; the pattern
    of P_bar is every aggregate a row's stored columns reach; K_c is
    bitwise symmetric and positive definite."""
    prob = I.poisson_box(d, n, p)
    H, dl1, agg, pv = _tentative(prob)
    nc = H.level_n(1)
    K = prob.to_scipy().toarray()
    P = np.zeros((prob.n, nc))
    P[np.arange(prob.n), agg] = pv
    theta = np.random.default_rng(d * 10 + p).uniform(0.3, 1.6, prob.n)
    rp, ci, v = O.smooth_prolongator(prob.rowptr, prob.col, prob.val, dl1, theta, agg, pv, nc)
    Pb = np.zeros((prob.n, nc))
    for i in range(prob.n):
        Pb[i, ci[rp[i]:rp[i + 1]]] = v[rp[i]:rp[i + 1]]
        want = sorted({int(agg[j]) for j in prob.col[prob.rowptr[i]:prob.rowptr[i + 1]]})
        assert list(ci[rp[i]:rp[i + 1]]) == want
    ref = P - (theta / dl1)[:, None] * (K @ P)
    assert np.abs(Pb - ref).max() <= 1e-14 * np.abs(ref).max()
    crp, cci, cv = O.galerkin_general(prob.rowptr, prob.col, prob.val, rp, ci, v, nc)
    Kc = np.zeros((nc, nc))
    for I_ in range(nc):
        Kc[I_, cci[crp[I_]:crp[I_ + 1]]] = cv[crp[I_]:crp[I_ + 1]]
    Kref = ref.T @ K @ ref
    assert np.abs(Kc - Kref).max() <= 1e-13 * np.abs(Kref).max()
    assert np.array_equal(Kc, Kc.T)
    np.linalg.cholesky(Kc)
    # theta = 0 gives back the tentative prolongator (with explicit zeros)
    rp0, ci0, v0 = O.smooth_prolongator(prob.rowptr, prob.col, prob.val, dl1, np.zeros(prob.n), agg, pv, nc)
    P0 = np.zeros((prob.n, nc))
    for i in range(prob.n):
        P0[i, ci0[rp0[i]:rp0[i + 1]]] = v0[rp0[i]:rp0[i + 1]]
    assert np.array_equal(P0, P)


def test_smoothed_hierarchy_vcycle_symmetric_and_faster():
    """With smoothed prolongators on every level the V-cycle stays symmetric
    and positive (restriction = P_bar^T), the hierarchy's coarse matrices
    are the general Galerkin products, and PCG needs fewer iterations than
    with the tentative prolongators on a 2-D p=3 problem."""
    prob = I.poisson_box(2, 24, 3)
    Hs = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30, smooth_levels=-1)
    Ht = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30)
    rp, ci, v = Hs.prolongator(0)
    crp, cci, cv = O.galerkin_general(prob.rowptr, prob.col, prob.val, rp, ci, v, Hs.level_n(1))
    g = Hs.level_csr(1)
    assert np.array_equal(g[0], crp) and np.array_equal(g[1], cci) and np.array_equal(g[2], cv)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    bx, by = Hs.vcycle(x), Hs.vcycle(y)
    assert abs(x @ by - y @ bx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(bx)
    assert x @ bx > 0
    its_s = Hs.pcg(prob.F, rtol=1e-8)["iters"]
    its_t = Ht.pcg(prob.F, rtol=1e-8)["iters"]
    assert its_s < its_t
    assert Hs.opc > Ht.opc  # the price: wider coarse operators


def test_smoothed_level0_takes_per_row_theta():
    """theta0 replaces smooth_omega on level 0 only; a constant theta0 equal
    to smooth_omega reproduces the default hierarchy bit for bit."""
    prob = I.poisson_box(2, 16, 2)
    a = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, smooth_levels=1)
    b = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, smooth_levels=1,
                    theta0=np.full(prob.n, 4.0 / 3.0))
    for l in range(a.num_levels):
        for x, y in zip(a.level_csr(l), b.level_csr(l)):
            assert np.array_equal(x, y)
    c = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=20, smooth_levels=1,
                    theta0=np.linspace(0.5, 1.5, prob.n))
    assert not np.array_equal(c.level_csr(1)[2], a.level_csr(1)[2])
    assert c.prolongator(1)[0][-1] == c.level_n(1)  # level 1 keeps the tentative prolongator


# ------------------------------------------------ Chebyshev smoother ----
def cheb4_poly(lam, k):
    """(-1)^k T_{2k+1}(sqrt(lam)) / ((2k+1) sqrt(lam)): the error polynomial
    of k steps of the 4th-kind Chebyshev smoother (rho = 1)."""
    from numpy.polynomial import chebyshev as C

    s = np.sqrt(lam)
    return (-1) ** k * C.chebval(s, [0] * (2 * k + 1) + [1]) / ((2 * k + 1) * s)


@pytest.mark.parametrize("k", [1, 2, 3, 8])
def test_chebyshev_smoother_closed_form_on_diagonal_matrix(k):
    """On K = diag(k_i) with l1 diagonal d = k / lam (lam in (0, 1]) the
    error after k steps from x0 is p_k(lam) (x0 - x*), p_k the 4th-kind
    polynomial in closed form; from zero, r = f - K x."""
    rng = np.random.default_rng(k)
    n = 40
    kk = rng.uniform(1.0, 3.0, n)
    lam = np.concatenate([[1.0, 1e-3], rng.uniform(0.01, 1.0, n - 2)])
    d = kk / lam
    rp, ci = np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32)
    xs = rng.standard_normal(n)
    f = kk * xs
    x0 = rng.standard_normal(n)
    x, _ = O.cheb4_smooth(rp, ci, kk, d, f, x0=x0, degree=k)
    assert np.allclose(x - xs, cheb4_poly(lam, k) * (x0 - xs), rtol=0, atol=1e-12)
    x, r = O.cheb4_smooth(rp, ci, kk, d, f, degree=k)
    assert np.allclose(x - xs, cheb4_poly(lam, k) * (-xs), rtol=0, atol=1e-12)
    assert np.allclose(r, f - kk * x, rtol=0, atol=1e-12)
    # the min-max property: |sqrt(lam) p_k(lam)| <= 1 / (2k + 1) on (0, 1]
    grid = np.linspace(1e-6, 1, 2001)
    assert np.max(np.abs(np.sqrt(grid) * cheb4_poly(grid, k))) <= 1 / (2 * k + 1) + 1e-12


def test_chebyshev_vcycle_symmetric_positive_and_faster():
    """With Chebyshev smoothing (same polynomial before and after the coarse
    correction) the V-cycle stays symmetric and positive, and degree 4
    needs fewer PCG iterations than one l1-Jacobi sweep on a 3-D p=3 cube."""
    prob = I.poisson_box(3, 8, 3)
    Hc = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30, cheb_degree=4)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal(prob.n), rng.standard_normal(prob.n)
    bx, by = Hc.vcycle(x), Hc.vcycle(y)
    assert abs(x @ by - y @ bx) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(bx)
    assert x @ bx > 0
    Hj = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=30)
    assert Hc.pcg(prob.F, rtol=1e-8)["iters"] < Hj.pcg(prob.F, rtol=1e-8)["iters"]


def test_coarse_cg_against_textbook_and_dense():
    """The coarse CG (Sec. 5: Jacobi-preconditioned CG to a relative
    tolerance or an iteration cap) reaches the dense solution when run to a
    tight tolerance, stops at the cap otherwise, and the V-cycle with it
    still solves the system under flexible CG."""
    prob = I.poisson_box(2, 12, 2)
    Hd = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=60)
    Hc = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=60, coarse_solver=1, coarse_tol=1e-14,
                     coarse_maxit=1000)
    r = np.random.default_rng(4).standard_normal(prob.n)
    zd, zc = Hd.vcycle(r), Hc.vcycle(r)
    assert np.linalg.norm(zd - zc) <= 1e-10 * np.linalg.norm(zd)
    H4 = O.Hierarchy(prob.rowptr, prob.col, prob.val, coarse_max=60, coarse_solver=1)
    g = H4.pcg(prob.F, rtol=1e-8, flexible=True)
    assert g["status"] == 0 and g["relres"] <= 1e-8 * 1.0001
    # one iteration of the coarse CG is the Jacobi-preconditioned steepest-descent step
    L = Hd.num_levels - 1
    rp, ci, v = Hd.level_csr(L)
    Kc = dense(rp, ci, v)
    f = np.random.default_rng(5).standard_normal(len(rp) - 1)
    z = f / np.diag(Kc)
    x1 = (f @ z) / (z @ Kc @ z) * z
    assert np.allclose(O.coarse_cg(rp, ci, v, f, 1e-4, 1), x1, rtol=1e-13, atol=0)
    # to a tight tolerance it is the dense solve
    assert np.allclose(O.coarse_cg(rp, ci, v, f, 1e-13, 500), np.linalg.solve(Kc, f), rtol=1e-10, atol=0)
