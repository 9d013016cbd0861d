/*
 * CPU ORACLE -- test infrastructure only.
 *
 * A plain, slow, sequential FP64 implementation of the matching-based
 * aggregation AMG preconditioned conjugate gradient method of
 * arXiv 2511.21268.  It is the reference the CUDA path is checked against
 * and shares no code with it.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Built with -O2 -ffp-contract=off: every floating-point operation below is
 * one IEEE-754 double operation in program order, so the setup results
 * (test vector, edge weights, matching, aggregates, Galerkin values) are
 * reproducible bit for bit.
 *
 * Passages followed (section / equation of the paper):
 *   l1 diagonal d_i = k_ii + sum_{j!=i} |k_ij|          Sec. 3.2
 *   l1-Jacobi sweep x <- x + D^-1 (f - K x)             Sec. 3.2, Eq. (smoother)
 *   test vector: relaxation on K w = 0 from a random
 *     start, restricted to coarse levels                Sec. 3.1 ("Edge weights")
 *   compatibility weight c_ij                           Sec. 3.1, Eq. (cij)
 *   maximum product matching, approximated greedily     Sec. 3.1, Eq. (maxprod)
 *   pair / singleton prolongator                        Sec. 3.1, Eq. (prolongation)
 *   m-step aggregation P = P_1 ... P_m                  Sec. 3.1 ("Variants")
 *   Galerkin coarse matrix K_c = P^T K P                Sec. 3, Eq. (galerkin_matrix_projection)
 *   operator complexity                                 Sec. 3.1, Eq. (OPC)
 *   smoothed prolongator P_bar = (I - w D^-1 K) P       Sec. 3.1 ("Variants")
 *   two-level correction / V-cycle                      Sec. 3 (steps 1-5)
 *   conjugate gradients, flexible CG                    Sec. 3, Sec. 4 ("Solver invocation"),
 *                                                       Sec. 5 (flexible CG, x0 = 0)
 *
 * Readings where the paper is silent (each applied identically on the GPU):
 *   - test vector: w0_i = U[0,1) from draw i of SplitMix64(seed); `s`
 *     l1-Jacobi sweeps w <- w - D^-1 (K w) on the finest level; coarse
 *     levels get w_c = P^T w.  All sums run left to right in CSR order.
 *   - edges: stored off-diagonal entries with k_ij != 0; an edge is
 *     eligible iff the denominator of c_ij and w_lo^2 + w_hi^2 are > 0.
 *   - c_ij evaluated with lo = min(i,j), hi = max(i,j):
 *       num = ((2 k) w_lo) w_hi
 *       den = k_lolo (w_lo w_lo) + k_hihi (w_hi w_hi)
 *       c   = 1 - num / den
 *   - the matching maximises the product (Eq. maxprod governs); since log
 *     is monotone the greedy algorithm ranks edges by c directly, under
 *     the strict total order (c desc, lo asc, hi asc).
 *   - coarse index of an aggregate = rank of its smallest fine index.
 *   - pair (i<j): nrm = sqrt(w_i w_i + w_j w_j), p_i = w_i/nrm,
 *     p_j = w_j/nrm; singleton s: p_s = w_s/|w_s|, or +1 if w_s = 0.
 *   - Galerkin: for coarse I <= J, K_c(I,J) = sum over fine a in I
 *     (ascending), then stored (a,b) with b in J (ascending b), of
 *     (p_a k_ab) p_b, added left to right starting from +0.0;
 *     K_c(J,I) := K_c(I,J).
 *   - coarsening stops when N_l <= coarse_max, when a new level would keep
 *     more than `stag` of the rows (it is then discarded) or at max_levels.
 *     The coarsest matrix is factorised by dense Cholesky.
 *   - smoothed prolongator (option smooth_levels): on the first
 *     smooth_levels levels (-1: all) the composite tentative P (one entry per
 *     row) becomes P_bar = (I - diag(theta) D^-1 K) P, D the l1 diagonal,
 *     theta_i = smooth_omega (default 4/3: the classical 4 / (3 rho(D^-1 K))
 *     with rho <= 1, which the l1 diagonal guarantees), or on level 0 a
 *     per-row theta given by the caller.  Row i of P_bar holds the coarse
 *     columns {agg(j) : j stored in row i} in ascending order, exact zeros
 *     included; with t = theta_i / d_i and kp_J = sum over stored j of row i
 *     in ascending order with agg(j) = J of k_ij p_j (from +0.0):
 *       P_bar(i, J) = (J == agg(i) ? p_i : 0.0) - t kp_J.
 *     Coarse matrix K_c = P_bar^T (K P_bar): T = K P_bar with T(i, J) = sum
 *     over stored j of row i in ascending order of k_ij P_bar(j, J) (from
 *     +0.0); for I <= J, K_c(I, J) = sum over the rows a of P_bar's column I
 *     in ascending order of P_bar(a, I) T(a, J) (from +0.0);
 *     K_c(J, I) := K_c(I, J).  Both patterns are structural.  The coarse
 *     test vector stays w_c = P_tent^T w from the matching passes.
 *   - V-cycle with nu1 pre- and nu2 post-sweeps of l1-Jacobi from x = 0;
 *     restriction f_c = P^T r, prolongation x += P e (P_bar where smoothed).
 *   - Chebyshev acceleration of l1-Jacobi (option cheb_degree = k >= 1,
 *     Sec. 3.2 and Sec. 5: polynomial smoothers of the 4th kind), taking
 *     rho(D^-1 K) <= 1 from the l1 diagonal instead of a spectral estimate:
 *       r_0 = f - K x_0, d_0 = (4/3) D^-1 r_0, x_1 = x_0 + d_0, and for
 *       i = 1 .. k-1:  r_i = r_{i-1} - K d_{i-1},
 *       d_i = (2i-1)/(2i+3) d_{i-1} + (8i+4)/(2i+3) D^-1 r_i,
 *       x_{i+1} = x_i + d_i.
 *     Its error polynomial is p_k(l) = (-1)^k T_{2k+1}(sqrt l) /
 *     ((2k+1) sqrt l), l in the spectrum of D^-1 K, the degree-k polynomial
 *     with p(0) = 1 of least max |sqrt(l) p(l)| on [0, 1].  Pre-smoothing
 *     starts from x_0 = 0 (r_0 = f) and hands r_k = r_{k-1} - K d_{k-1} to
 *     the restriction; post-smoothing starts from the prolongated x.  The
 *     paper's "optimized" variant scales the steps by tabulated weights
 *     that are not used here.
 *   - coarsest solve (option coarse_solver = 1, Sec. 5): CG preconditioned
 *     by Jacobi (z = r / k_ii) from x = 0, stopping once ||r|| <= coarse_tol
 *     ||f|| (recursive residual) or after coarse_maxit iterations; the
 *     default is the exact dense Cholesky solve.
 *   - PCG stops when ||r_k||_2 <= rtol ||F||_2 on the recursive residual.
 *
 * Threads: the solve phase (V-cycle and CG) may run its row loops -- each
 * row's sum evaluated exactly as in the sequential code -- on several
 * OpenMP threads (orc_set_threads); restrictions, which add into shared
 * coarse entries, and every dot product stay sequential, so the results do
 * not depend on the thread count.  The setup is always sequential (the
 * greedy matching is defined by its sequential scan).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* threads of the solve phase's row loops (1 = sequential) */
static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t < 1 ? 1 : t; }

int orc_get_threads(void) { return g_threads; }

/* 1 if this build runs the row loops on OpenMP threads */
int orc_have_openmp(void) {
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

#define ORC_MAX_LEVELS 32
#define ORC_MAX_PASSES 4

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NOT_SPD = -2, ORC_ERR_BREAKDOWN = -3, ORC_ERR_NOT_CONVERGED = -4,
       ORC_ERR_NAN = -7, ORC_ERR_COARSE_TOO_LARGE = -8, ORC_ERR_NOMEM = -9 };

typedef struct {
    int nu_pre, nu_post;
    int match_passes;
    int coarse_max;
    int max_levels;
    int testvec_sweeps;
    int testvec_kind; /* 0 = smoothed random, 1 = ones */
    uint64_t seed;
    double stag;      /* stop coarsening if n_{l+1} > stag * n_l */
    int dense_max;    /* largest coarsest level factorised densely */
    int smooth_levels;   /* smoothed prolongator on the first levels (-1 = all, 0 = none) */
    double smooth_omega; /* theta of the smoothed levels (4/3) */
    int cheb_degree;     /* 0: nu_pre / nu_post l1-Jacobi sweeps; k >= 1: 4th-kind Chebyshev of degree k */
    int coarse_solver;   /* 0: dense Cholesky; 1: CG with Jacobi preconditioning */
    double coarse_tol;   /* coarse CG: stop at ||r|| <= coarse_tol ||f|| (1e-4) */
    int coarse_maxit;    /* coarse CG: at most this many iterations (30) */
} orc_opts;

typedef struct {
    int64_t n, nnz;
    int64_t* rowptr;
    int32_t* col;
    double* val;
    double* dl1;
    double* w;
    /* map to level l+1: composite aggregate map and prolongator values */
    int32_t* agg;
    double* pval;
    /* smoothed prolongator (NULL when the level uses the tentative P) */
    int64_t* sp_rp;
    int32_t* sp_ci;
    double* sp_v;
    /* per matching pass: mates, pass aggregate maps, pass values */
    int npass;
    int64_t pass_n[ORC_MAX_PASSES + 1];
    int32_t* pass_mate[ORC_MAX_PASSES];
    int32_t* pass_agg[ORC_MAX_PASSES];
    double* pass_pval[ORC_MAX_PASSES];
} orc_level;

typedef struct {
    orc_opts o;
    int nlev;
    orc_level lev[ORC_MAX_LEVELS];
    double* chol; /* dense lower Cholesky factor of the coarsest matrix, row-major */
    int64_t nc;
} orc_hier;

/* ------------------------------------------------------------- RNG ---- */
/* SplitMix64 (Steele, Lea, Flood 2014); draw k of the stream seeded `seed`. */
static uint64_t orc_sm64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------ basic kernels ---- */
/* d_i = k_ii + sum_{j != i} |k_ij| (Sec. 3.2); the off-diagonal sum runs in
 * CSR order from +0.0.  Returns ORC_ERR_NOT_SPD if some k_ii <= 0. */
int orc_l1_diag(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, double* d) {
    int rc = ORC_OK;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0, kii = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            if (ci[k] == i) kii = v[k];
            else s = s + fabs(v[k]);
        }
        if (!(kii > 0.0)) rc = ORC_ERR_NOT_SPD;
        d[i] = kii + s;
    }
    return rc;
}

static double row_dot(const int64_t* rp, const int32_t* ci, const double* v, int64_t i, const double* x) {
    double s = 0.0;
    for (int64_t k = rp[i]; k < rp[i + 1]; k++) s = s + v[k] * x[ci[k]];
    return s;
}

void orc_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int64_t i = 0; i < n; i++) y[i] = row_dot(rp, ci, v, i, x);
}

/* r = f - K x, row by row */
static void residual(const int64_t* rp, const int32_t* ci, const double* v, int64_t n, const double* f,
                     const double* x, double* r) {
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
    for (int64_t i = 0; i < n; i++) r[i] = f[i] - row_dot(rp, ci, v, i, x);
}

static double dot(int64_t n, const double* a, const double* b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s = s + a[i] * b[i];
    return s;
}

static double diag_of(const int64_t* rp, const int32_t* ci, const double* v, int64_t i) {
    for (int64_t k = rp[i]; k < rp[i + 1]; k++)
        if (ci[k] == i) return v[k];
    return 0.0;
}

/* Test vector (Sec. 3.1): w0 random, then `sweeps` l1-Jacobi sweeps on
 * K w = 0:  w_i <- w_i - (K w)_i / d_i, all rows from the previous iterate. */
int orc_test_vector(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* dl1, int kind,
                    uint64_t seed, int sweeps, double* w) {
    for (int64_t i = 0; i < n; i++) w[i] = kind == 1 ? 1.0 : (double)(orc_sm64(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
    double* t = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    if (!t) return ORC_ERR_NOMEM;
    for (int s = 0; s < sweeps; s++) {
        orc_spmv(n, rp, ci, v, w, t);
        for (int64_t i = 0; i < n; i++) w[i] = w[i] - t[i] / dl1[i];
    }
    free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------- matching ---- */
typedef struct {
    double c;
    int32_t lo, hi;
} orc_edge;

/* Compatibility weight, Eq. (cij), in the canonical (lo, hi) order.
 * Returns 1 and sets *c if the edge is eligible. */
int orc_edge_weight(double k, double klo, double khi, double wlo, double whi, double* c) {
    if (k == 0.0) return 0;
    double num = ((2.0 * k) * wlo) * whi;
    double den = klo * (wlo * wlo) + khi * (whi * whi);
    double nrm2 = wlo * wlo + whi * whi;
    if (!(den > 0.0) || !(nrm2 > 0.0)) return 0;
    *c = 1.0 - num / den;
    return 1;
}

/* strict total order: a before b iff a is heavier */
static int edge_cmp(const void* A, const void* B) {
    const orc_edge* a = (const orc_edge*)A;
    const orc_edge* b = (const orc_edge*)B;
    if (a->c > b->c) return -1;
    if (a->c < b->c) return 1;
    if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;
    if (a->hi != b->hi) return a->hi < b->hi ? -1 : 1;
    return 0;
}

/* Sort the edges by the strict order and keep each edge whose two ends are
 * still free. */
static int64_t greedy_scan(int64_t n, orc_edge* E, int64_t m, int32_t* mate) {
    qsort(E, (size_t)m, sizeof(orc_edge), edge_cmp);
    for (int64_t i = 0; i < n; i++) mate[i] = -1;
    int64_t pairs = 0;
    for (int64_t e = 0; e < m; e++)
        if (mate[E[e].lo] < 0 && mate[E[e].hi] < 0) {
            mate[E[e].lo] = E[e].hi;
            mate[E[e].hi] = E[e].lo;
            pairs++;
        }
    return pairs;
}

/* Greedy approximation of the maximum product matching (Sec. 3.1): visit
 * the eligible edges from heaviest to lightest and keep an edge when both
 * ends are still free.  mate[i] = partner, or -1 for a singleton.
 * Returns the number of pairs (or a negative error). */
int64_t orc_match_greedy(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* w,
                         int32_t* mate) {
    double* dg = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
    int64_t ne = 0;
    for (int64_t i = 0; i < n; i++) {
        dg[i] = diag_of(rp, ci, v, i);
        for (int64_t k = rp[i]; k < rp[i + 1]; k++)
            if (ci[k] > i) ne++;
    }
    orc_edge* E = (orc_edge*)malloc(sizeof(orc_edge) * (ne > 0 ? ne : 1));
    if (!dg || !E) { free(dg); free(E); return ORC_ERR_NOMEM; }
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            int64_t j = ci[k];
            if (j <= i) continue;
            double c;
            if (orc_edge_weight(v[k], dg[i], dg[j], w[i], w[j], &c)) {
                E[m].c = c;
                E[m].lo = (int32_t)i;
                E[m].hi = (int32_t)j;
                m++;
            }
        }
    int64_t pairs = greedy_scan(n, E, m, mate);
    free(E);
    free(dg);
    return pairs;
}

/* Greedy matching on an explicit weighted edge list (lo[e] < hi[e]). */
int64_t orc_match_greedy_edges(int64_t n, int64_t m, const int32_t* lo, const int32_t* hi, const double* c,
                               int32_t* mate) {
    orc_edge* E = (orc_edge*)malloc(sizeof(orc_edge) * (m > 0 ? m : 1));
    if (!E) return ORC_ERR_NOMEM;
    for (int64_t e = 0; e < m; e++) {
        E[e].c = c[e];
        E[e].lo = lo[e];
        E[e].hi = hi[e];
    }
    int64_t pairs = greedy_scan(n, E, m, mate);
    free(E);
    return pairs;
}

/* Aggregates from a matching (Eq. prolongation): one coarse unknown per pair
 * and per singleton, numbered by the aggregate's smallest fine index. */
int64_t orc_aggregate(int64_t n, const int32_t* mate, const double* w, int32_t* agg, double* pval) {
    int64_t nc = 0;
    for (int64_t i = 0; i < n; i++) {
        int32_t j = mate[i];
        if (j < 0) {
            agg[i] = (int32_t)nc++;
            pval[i] = w[i] < 0.0 ? -1.0 : 1.0; /* w_s/|w_s|, +1 for w_s = 0 */
        } else if (j > i) {
            double nrm = sqrt(w[i] * w[i] + w[j] * w[j]);
            agg[i] = agg[j] = (int32_t)nc++;
            pval[i] = w[i] / nrm;
            pval[j] = w[j] / nrm;
        }
    }
    return nc;
}

/* w_c = P^T w: w_c[I] = sum over a in I ascending of p_a w_a. */
void orc_restrict(int64_t n, const int32_t* agg, const double* pval, const double* x, int64_t nc, double* xc) {
    for (int64_t I = 0; I < nc; I++) xc[I] = 0.0;
    for (int64_t i = 0; i < n; i++) xc[agg[i]] = xc[agg[i]] + pval[i] * x[i];
}

/* Galerkin product K_c = P^T K P for a prolongator with one nonzero per row
 * (value pval[i] in column agg[i]).  Output CSR with sorted columns. */
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

int orc_galerkin(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const int32_t* agg,
                 const double* pval, int64_t nc, int64_t** out_rp, int32_t** out_ci, double** out_v) {
    /* members of each aggregate in ascending fine order */
    int64_t* mp = (int64_t*)calloc(nc + 1, sizeof(int64_t));
    int32_t* mi = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; i++) mp[agg[i] + 1]++;
    for (int64_t I = 0; I < nc; I++) mp[I + 1] += mp[I];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nc + 1));
    memcpy(fill, mp, sizeof(int64_t) * (nc + 1));
    for (int64_t i = 0; i < n; i++) mi[fill[agg[i]]++] = (int32_t)i;

    /* upper triangle (J >= I), Gustavson-style dense accumulator */
    double* acc = (double*)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    for (int64_t I = 0; I < nc; I++) mark[I] = -1;
    int64_t cap = 1024, used = 0;
    int64_t* urp = (int64_t*)malloc(sizeof(int64_t) * (nc + 1));
    int32_t* uci = (int32_t*)malloc(sizeof(int32_t) * cap);
    double* uv = (double*)malloc(sizeof(double) * cap);
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (nc > 0 ? nc : 1));
    urp[0] = 0;
    for (int64_t I = 0; I < nc; I++) {
        int64_t nl = 0;
        for (int64_t t = mp[I]; t < mp[I + 1]; t++) {
            int64_t a = mi[t];
            for (int64_t k = rp[a]; k < rp[a + 1]; k++) {
                int64_t b = ci[k];
                int32_t J = agg[b];
                if (J < I) continue;
                if (mark[J] != I) {
                    mark[J] = I;
                    acc[J] = 0.0;
                    list[nl++] = J;
                }
                acc[J] = acc[J] + (pval[a] * v[k]) * pval[b];
            }
        }
        qsort(list, (size_t)nl, sizeof(int32_t), cmp_i32);
        if (used + nl > cap) {
            while (used + nl > cap) cap *= 2;
            uci = (int32_t*)realloc(uci, sizeof(int32_t) * cap);
            uv = (double*)realloc(uv, sizeof(double) * cap);
        }
        for (int64_t t = 0; t < nl; t++) {
            uci[used] = list[t];
            uv[used] = acc[list[t]];
            used++;
        }
        urp[I + 1] = used;
    }
    /* full matrix: row I = {J < I : I in upper row J} then upper row I */
    int64_t* rp_c = (int64_t*)calloc(nc + 1, sizeof(int64_t));
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            rp_c[I + 1]++;
            if (uci[t] != I) rp_c[uci[t] + 1]++;
        }
    for (int64_t I = 0; I < nc; I++) rp_c[I + 1] += rp_c[I];
    int64_t nnzc = rp_c[nc];
    int32_t* ci_c = (int32_t*)malloc(sizeof(int32_t) * (nnzc > 0 ? nnzc : 1));
    double* v_c = (double*)malloc(sizeof(double) * (nnzc > 0 ? nnzc : 1));
    memcpy(fill, rp_c, sizeof(int64_t) * (nc + 1));
    /* lower parts first: rows J receive (I, value) in increasing I */
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            int32_t J = uci[t];
            if (J == I) continue;
            ci_c[fill[J]] = (int32_t)I;
            v_c[fill[J]] = uv[t];
            fill[J]++;
        }
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            ci_c[fill[I]] = uci[t];
            v_c[fill[I]] = uv[t];
            fill[I]++;
        }
    free(mp); free(mi); free(fill); free(acc); free(mark); free(urp); free(uci); free(uv); free(list);
    *out_rp = rp_c;
    *out_ci = ci_c;
    *out_v = v_c;
    return ORC_OK;
}

/* --------------------------------------------- smoothed prolongator ---- */
/* P_bar = (I - diag(theta) D^-1 K) P for the tentative P (value pval[i] in
 * column agg[i]), Sec. 3.1 ("Variants"); theta[i] per row.  Output CSR
 * (n rows, nc columns) in the order and with the values stated at the top. */
int orc_smooth_prolongator(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* dl1,
                           const double* theta, const int32_t* agg, const double* pval, int64_t nc,
                           int64_t** out_rp, int32_t** out_ci, double** out_v) {
    int64_t* prp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (nc > 0 ? nc : 1));
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    double* acc = (double*)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    if (!prp || !list || !mark || !acc) { free(prp); free(list); free(mark); free(acc); return ORC_ERR_NOMEM; }
    for (int64_t J = 0; J < nc; J++) mark[J] = -1;
    /* pattern: distinct agg(j) over the stored j of each row */
    prp[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t cnt = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            int32_t J = agg[ci[k]];
            if (mark[J] != i) { mark[J] = i; cnt++; }
        }
        prp[i + 1] = prp[i] + cnt;
    }
    int64_t nnz = prp[n];
    int32_t* pci = (int32_t*)malloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    double* pv = (double*)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    if (!pci || !pv) { free(prp); free(list); free(mark); free(acc); free(pci); free(pv); return ORC_ERR_NOMEM; }
    for (int64_t J = 0; J < nc; J++) mark[J] = -1;
    for (int64_t i = 0; i < n; i++) {
        int64_t nl = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            int32_t j = ci[k], J = agg[j];
            if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list[nl++] = J; }
            acc[J] = acc[J] + v[k] * pval[j];
        }
        qsort(list, (size_t)nl, sizeof(int32_t), cmp_i32);
        const double t = theta[i] / dl1[i];
        for (int64_t q = 0; q < nl; q++) {
            int32_t J = list[q];
            pci[prp[i] + q] = J;
            pv[prp[i] + q] = (J == agg[i] ? pval[i] : 0.0) - t * acc[J];
        }
    }
    free(list); free(mark); free(acc);
    *out_rp = prp;
    *out_ci = pci;
    *out_v = pv;
    return ORC_OK;
}

/* K_c = P^T (K P) for a general prolongator P (CSR, n x nc, sorted columns):
 * T = K P row by row (for each coarse column, terms in ascending fine
 * column order), then for I <= J the sum over the rows a of column I of P
 * in ascending order of P(a, I) T(a, J), mirrored to J < I.  Output CSR with
 * sorted columns. */
int orc_galerkin_general(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const int64_t* prp,
                         const int32_t* pci, const double* pv, int64_t nc, int64_t** out_rp, int32_t** out_ci,
                         double** out_v) {
    double* acc = (double*)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (nc > 0 ? nc : 1));
    int64_t* trp = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    if (!acc || !mark || !list || !trp) { free(acc); free(mark); free(list); free(trp); return ORC_ERR_NOMEM; }
    /* T = K P */
    int64_t cap = 1024, used = 0;
    int32_t* tci = (int32_t*)malloc(sizeof(int32_t) * cap);
    double* tv = (double*)malloc(sizeof(double) * cap);
    for (int64_t J = 0; J < nc; J++) mark[J] = -1;
    trp[0] = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t nl = 0;
        for (int64_t k = rp[i]; k < rp[i + 1]; k++) {
            int64_t j = ci[k];
            for (int64_t q = prp[j]; q < prp[j + 1]; q++) {
                int32_t J = pci[q];
                if (mark[J] != i) { mark[J] = i; acc[J] = 0.0; list[nl++] = J; }
                acc[J] = acc[J] + v[k] * pv[q];
            }
        }
        qsort(list, (size_t)nl, sizeof(int32_t), cmp_i32);
        if (used + nl > cap) {
            while (used + nl > cap) cap *= 2;
            tci = (int32_t*)realloc(tci, sizeof(int32_t) * cap);
            tv = (double*)realloc(tv, sizeof(double) * cap);
        }
        for (int64_t q = 0; q < nl; q++) { tci[used] = list[q]; tv[used] = acc[list[q]]; used++; }
        trp[i + 1] = used;
    }
    /* columns of P: rows a ascending within each column */
    int64_t* cp = (int64_t*)calloc(nc + 1, sizeof(int64_t));
    int32_t* crow = (int32_t*)malloc(sizeof(int32_t) * (prp[n] > 0 ? prp[n] : 1));
    double* cval = (double*)malloc(sizeof(double) * (prp[n] > 0 ? prp[n] : 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nc + 1));
    for (int64_t q = 0; q < prp[n]; q++) cp[pci[q] + 1]++;
    for (int64_t J = 0; J < nc; J++) cp[J + 1] += cp[J];
    memcpy(fill, cp, sizeof(int64_t) * (nc + 1));
    for (int64_t a = 0; a < n; a++)
        for (int64_t q = prp[a]; q < prp[a + 1]; q++) {
            crow[fill[pci[q]]] = (int32_t)a;
            cval[fill[pci[q]]] = pv[q];
            fill[pci[q]]++;
        }
    /* upper triangle of P^T T */
    int64_t ucap = 1024, uused = 0;
    int64_t* urp = (int64_t*)malloc(sizeof(int64_t) * (nc + 1));
    int32_t* uci = (int32_t*)malloc(sizeof(int32_t) * ucap);
    double* uv = (double*)malloc(sizeof(double) * ucap);
    for (int64_t J = 0; J < nc; J++) mark[J] = -1;
    urp[0] = 0;
    for (int64_t I = 0; I < nc; I++) {
        int64_t nl = 0;
        for (int64_t q = cp[I]; q < cp[I + 1]; q++) {
            int64_t a = crow[q];
            for (int64_t t = trp[a]; t < trp[a + 1]; t++) {
                int32_t J = tci[t];
                if (J < I) continue;
                if (mark[J] != I) { mark[J] = I; acc[J] = 0.0; list[nl++] = J; }
                acc[J] = acc[J] + cval[q] * tv[t];
            }
        }
        qsort(list, (size_t)nl, sizeof(int32_t), cmp_i32);
        if (uused + nl > ucap) {
            while (uused + nl > ucap) ucap *= 2;
            uci = (int32_t*)realloc(uci, sizeof(int32_t) * ucap);
            uv = (double*)realloc(uv, sizeof(double) * ucap);
        }
        for (int64_t t = 0; t < nl; t++) { uci[uused] = list[t]; uv[uused] = acc[list[t]]; uused++; }
        urp[I + 1] = uused;
    }
    /* full symmetric matrix: row I = {J < I : I in upper row J} then upper row I */
    int64_t* rp_c = (int64_t*)calloc(nc + 1, sizeof(int64_t));
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            rp_c[I + 1]++;
            if (uci[t] != I) rp_c[uci[t] + 1]++;
        }
    for (int64_t I = 0; I < nc; I++) rp_c[I + 1] += rp_c[I];
    int64_t nnzc = rp_c[nc];
    int32_t* ci_c = (int32_t*)malloc(sizeof(int32_t) * (nnzc > 0 ? nnzc : 1));
    double* v_c = (double*)malloc(sizeof(double) * (nnzc > 0 ? nnzc : 1));
    memcpy(fill, rp_c, sizeof(int64_t) * (nc + 1));
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            int32_t J = uci[t];
            if (J == I) continue;
            ci_c[fill[J]] = (int32_t)I;
            v_c[fill[J]] = uv[t];
            fill[J]++;
        }
    for (int64_t I = 0; I < nc; I++)
        for (int64_t t = urp[I]; t < urp[I + 1]; t++) {
            ci_c[fill[I]] = uci[t];
            v_c[fill[I]] = uv[t];
            fill[I]++;
        }
    free(acc); free(mark); free(list); free(trp); free(tci); free(tv); free(cp); free(crow); free(cval);
    free(fill); free(urp); free(uci); free(uv);
    *out_rp = rp_c;
    *out_ci = ci_c;
    *out_v = v_c;
    return ORC_OK;
}

/* -------------------------------------------------------- dense Cholesky ---- */
/* A = L L^T, L lower, row-major in place (upper part zeroed). */
int orc_cholesky(int64_t n, double* A) {
    for (int64_t j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; k++) s = s - A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return ORC_ERR_NOT_SPD;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; k++) t = t - A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
        for (int64_t i = 0; i < j; i++) A[i * n + j] = 0.0;
    }
    return ORC_OK;
}

/* x = L^-T L^-1 b */
void orc_chol_solve(int64_t n, const double* L, const double* b, double* x) {
    for (int64_t i = 0; i < n; i++) {
        double t = b[i];
        for (int64_t k = 0; k < i; k++) t = t - L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (int64_t k = i + 1; k < n; k++) t = t - L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* ------------------------------------------------------------- setup ---- */
void orc_opts_default(orc_opts* o) {
    o->nu_pre = 1;
    o->nu_post = 1;
    o->match_passes = 2;
    o->coarse_max = 200;
    o->max_levels = 30;
    o->testvec_sweeps = 4;
    o->testvec_kind = 0;
    o->seed = 20251126ULL;
    o->stag = 0.9;
    o->dense_max = 4096;
    o->smooth_levels = 0;
    o->smooth_omega = 4.0 / 3.0;
    o->cheb_degree = 0;
    o->coarse_solver = 0;
    o->coarse_tol = 1e-4;
    o->coarse_maxit = 30;
}

static void level_free(orc_level* L) {
    free(L->rowptr); free(L->col); free(L->val); free(L->dl1); free(L->w); free(L->agg); free(L->pval);
    free(L->sp_rp); free(L->sp_ci); free(L->sp_v);
    for (int s = 0; s < ORC_MAX_PASSES; s++) { free(L->pass_mate[s]); free(L->pass_agg[s]); free(L->pass_pval[s]); }
    memset(L, 0, sizeof(*L));
}

void orc_free(orc_hier* h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; l++) level_free(&h->lev[l]);
    free(h->chol);
    free(h);
}

orc_hier* orc_setup_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const orc_opts* opts,
                       const double* theta0, int* status);

orc_hier* orc_setup(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const orc_opts* opts,
                    int* status) {
    return orc_setup_ex(n, rp, ci, v, opts, NULL, status);
}

/* As orc_setup; theta0 (n entries, or NULL) replaces smooth_omega on level
 * 0 when level 0's prolongator is smoothed. */
orc_hier* orc_setup_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const orc_opts* opts,
                       const double* theta0, int* status) {
    orc_hier* h = (orc_hier*)calloc(1, sizeof(orc_hier));
    if (opts) h->o = *opts;
    else orc_opts_default(&h->o);
    *status = ORC_OK;
    if (n <= 0 || h->o.match_passes < 1 || h->o.match_passes > ORC_MAX_PASSES || h->o.max_levels < 1 ||
        h->o.max_levels > ORC_MAX_LEVELS) {
        *status = ORC_ERR_ARG;
        free(h);
        return NULL;
    }
    /* level 0 = copy of the input */
    orc_level* L0 = &h->lev[0];
    L0->n = n;
    L0->nnz = rp[n];
    L0->rowptr = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
    L0->col = (int32_t*)malloc(sizeof(int32_t) * (L0->nnz > 0 ? L0->nnz : 1));
    L0->val = (double*)malloc(sizeof(double) * (L0->nnz > 0 ? L0->nnz : 1));
    memcpy(L0->rowptr, rp, sizeof(int64_t) * (n + 1));
    memcpy(L0->col, ci, sizeof(int32_t) * L0->nnz);
    memcpy(L0->val, v, sizeof(double) * L0->nnz);
    h->nlev = 1;
    L0->dl1 = (double*)malloc(sizeof(double) * n);
    if (orc_l1_diag(n, rp, ci, v, L0->dl1) != ORC_OK) { *status = ORC_ERR_NOT_SPD; orc_free(h); return NULL; }
    L0->w = (double*)malloc(sizeof(double) * n);
    orc_test_vector(n, rp, ci, v, L0->dl1, h->o.testvec_kind, h->o.seed, h->o.testvec_sweeps, L0->w);

    while (h->nlev < h->o.max_levels && h->lev[h->nlev - 1].n > h->o.coarse_max) {
        orc_level* F = &h->lev[h->nlev - 1];
        /* m matching passes */
        int64_t cn = F->n;
        int64_t* crp = F->rowptr;
        int32_t* cci = F->col;
        double* cv = F->val;
        double* cw = F->w;
        int own = 0;
        F->npass = h->o.match_passes;
        F->pass_n[0] = cn;
        for (int s = 0; s < h->o.match_passes; s++) {
            int32_t* mate = (int32_t*)malloc(sizeof(int32_t) * cn);
            int32_t* agg = (int32_t*)malloc(sizeof(int32_t) * cn);
            double* pv = (double*)malloc(sizeof(double) * cn);
            orc_match_greedy(cn, crp, cci, cv, cw, mate);
            int64_t nn = orc_aggregate(cn, mate, cw, agg, pv);
            int64_t* nrp;
            int32_t* nci;
            double* nv;
            orc_galerkin(cn, crp, cci, cv, agg, pv, nn, &nrp, &nci, &nv);
            double* nw = (double*)malloc(sizeof(double) * (nn > 0 ? nn : 1));
            orc_restrict(cn, agg, pv, cw, nn, nw);
            if (own) { free(crp); free(cci); free(cv); free(cw); }
            F->pass_mate[s] = mate;
            F->pass_agg[s] = agg;
            F->pass_pval[s] = pv;
            F->pass_n[s + 1] = nn;
            cn = nn; crp = nrp; cci = nci; cv = nv; cw = nw;
            own = 1;
        }
        if ((double)cn > h->o.stag * (double)F->n) { /* stagnation: discard */
            free(crp); free(cci); free(cv); free(cw);
            for (int s = 0; s < ORC_MAX_PASSES; s++) {
                free(F->pass_mate[s]); free(F->pass_agg[s]); free(F->pass_pval[s]);
                F->pass_mate[s] = NULL; F->pass_agg[s] = NULL; F->pass_pval[s] = NULL;
            }
            F->npass = 0;
            break;
        }
        /* composite map P = P_1 ... P_m */
        F->agg = (int32_t*)malloc(sizeof(int32_t) * F->n);
        F->pval = (double*)malloc(sizeof(double) * F->n);
        for (int64_t i = 0; i < F->n; i++) {
            int32_t a = F->pass_agg[0][i];
            double pv = F->pass_pval[0][i];
            for (int s = 1; s < F->npass; s++) {
                pv = pv * F->pass_pval[s][a];
                a = F->pass_agg[s][a];
            }
            F->agg[i] = a;
            F->pval[i] = pv;
        }
        const int lf = h->nlev - 1;
        if (h->o.smooth_levels < 0 || lf < h->o.smooth_levels) {
            /* smoothed prolongator and its Galerkin product replace the
             * tentative P's coarse matrix */
            double* th = (double*)malloc(sizeof(double) * F->n);
            for (int64_t i = 0; i < F->n; i++) th[i] = (lf == 0 && theta0) ? theta0[i] : h->o.smooth_omega;
            int rs = orc_smooth_prolongator(F->n, F->rowptr, F->col, F->val, F->dl1, th, F->agg, F->pval, cn,
                                            &F->sp_rp, &F->sp_ci, &F->sp_v);
            free(th);
            int64_t* grp;
            int32_t* gci;
            double* gv;
            if (rs == ORC_OK)
                rs = orc_galerkin_general(F->n, F->rowptr, F->col, F->val, F->sp_rp, F->sp_ci, F->sp_v, cn, &grp,
                                          &gci, &gv);
            if (rs != ORC_OK) {
                free(crp); free(cci); free(cv); free(cw);
                *status = rs;
                orc_free(h);
                return NULL;
            }
            free(crp); free(cci); free(cv);
            crp = grp;
            cci = gci;
            cv = gv;
        }
        orc_level* C = &h->lev[h->nlev];
        C->n = cn;
        C->nnz = crp[cn];
        C->rowptr = crp;
        C->col = cci;
        C->val = cv;
        C->w = cw;
        C->dl1 = (double*)malloc(sizeof(double) * (cn > 0 ? cn : 1));
        if (orc_l1_diag(cn, crp, cci, cv, C->dl1) != ORC_OK) {
            h->nlev++;
            *status = ORC_ERR_NOT_SPD;
            orc_free(h);
            return NULL;
        }
        h->nlev++;
    }
    /* dense Cholesky of the coarsest level */
    orc_level* Lc = &h->lev[h->nlev - 1];
    if (Lc->n > h->o.dense_max) { *status = ORC_ERR_COARSE_TOO_LARGE; orc_free(h); return NULL; }
    h->nc = Lc->n;
    h->chol = (double*)calloc((size_t)(h->nc * h->nc), sizeof(double));
    for (int64_t i = 0; i < h->nc; i++)
        for (int64_t k = Lc->rowptr[i]; k < Lc->rowptr[i + 1]; k++) h->chol[i * h->nc + Lc->col[k]] = Lc->val[k];
    if (orc_cholesky(h->nc, h->chol) != ORC_OK) { *status = ORC_ERR_NOT_SPD; orc_free(h); return NULL; }
    return h;
}

/* ------------------------------------------------ Chebyshev smoother ---- */
/* k steps of the 4th-kind Chebyshev acceleration of l1-Jacobi (see the top
 * of the file) on K x = f.  zero_start: x_0 = 0 (x is overwritten) and on
 * return r holds r_k = r_{k-1} - K d_{k-1} (= f - K x_k); otherwise x holds
 * x_0 and r is workspace.  d, t: workspace of n entries. */
void orc_cheb4_smooth(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* dl1,
                      const double* f, double* x, double* r, double* d, double* t, int degree, int zero_start) {
    if (zero_start) {
        for (int64_t i = 0; i < n; i++) {
            x[i] = 0.0;
            r[i] = f[i];
        }
    } else {
        residual(rp, ci, v, n, f, x, r);
    }
    for (int64_t i = 0; i < n; i++) d[i] = (4.0 / 3.0) * (r[i] / dl1[i]);
    for (int64_t i = 0; i < n; i++) x[i] = x[i] + d[i];
    for (int s = 1; s < degree; s++) {
        const double a = (double)(2 * s - 1) / (double)(2 * s + 3);
        const double b = (double)(8 * s + 4) / (double)(2 * s + 3);
        orc_spmv(n, rp, ci, v, d, t);
        for (int64_t i = 0; i < n; i++) r[i] = r[i] - t[i];
        for (int64_t i = 0; i < n; i++) d[i] = a * d[i] + b * (r[i] / dl1[i]);
        for (int64_t i = 0; i < n; i++) x[i] = x[i] + d[i];
    }
    if (zero_start) { /* the residual for the restriction */
        orc_spmv(n, rp, ci, v, d, t);
        for (int64_t i = 0; i < n; i++) r[i] = r[i] - t[i];
    }
}

/* Jacobi-preconditioned CG on K x = f from x = 0 (coarsest level, Sec. 5):
 * at most maxit iterations, stopping when ||r||_2 <= tol ||f||_2. */
void orc_coarse_cg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* f, double tol,
                   int maxit, double* x) {
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    double* dg = (double*)malloc(sizeof(double) * n);
    for (int64_t i = 0; i < n; i++) {
        x[i] = 0.0;
        r[i] = f[i];
        dg[i] = diag_of(rp, ci, v, i);
        z[i] = r[i] / dg[i];
        p[i] = z[i];
    }
    const double stop = tol * sqrt(dot(n, f, f));
    double rho = dot(n, r, z);
    for (int it = 0; it < maxit && sqrt(dot(n, r, r)) > stop; it++) {
        orc_spmv(n, rp, ci, v, p, q);
        const double pq = dot(n, p, q);
        if (!(pq > 0.0)) break;
        const double alpha = rho / pq;
        for (int64_t i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
        for (int64_t i = 0; i < n; i++) z[i] = r[i] / dg[i];
        const double rho1 = dot(n, r, z);
        const double beta = rho1 / rho;
        rho = rho1;
        for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
    }
    free(r); free(z); free(p); free(q); free(dg);
}

/* ------------------------------------------------------------- V-cycle ---- */
/* Two-level correction applied recursively (Sec. 3, steps 1-5), l1-Jacobi
 * smoothing from x = 0, exact coarsest solve. */
static void vcycle(const orc_hier* h, int l, const double* f, double* x) {
    const orc_level* L = &h->lev[l];
    const int64_t n = L->n;
    if (l == h->nlev - 1) {
        if (h->o.coarse_solver == 1 && h->nlev > 1)
            orc_coarse_cg(n, L->rowptr, L->col, L->val, f, h->o.coarse_tol, h->o.coarse_maxit, x);
        else
            orc_chol_solve(n, h->chol, f, x);
        return;
    }
    double* r = (double*)malloc(sizeof(double) * n);
    const int cheb = h->o.cheb_degree;
    double* d = cheb > 0 ? (double*)malloc(sizeof(double) * n) : NULL;
    double* t = cheb > 0 ? (double*)malloc(sizeof(double) * n) : NULL;
    if (cheb > 0) {
        orc_cheb4_smooth(n, L->rowptr, L->col, L->val, L->dl1, f, x, r, d, t, cheb, 1);
    } else {
        for (int64_t i = 0; i < n; i++) x[i] = 0.0;
        for (int s = 0; s < h->o.nu_pre; s++) {
            residual(L->rowptr, L->col, L->val, n, f, x, r);
            for (int64_t i = 0; i < n; i++) x[i] = x[i] + r[i] / L->dl1[i];
        }
        residual(L->rowptr, L->col, L->val, n, f, x, r);
    }
    const int64_t nc = h->lev[l + 1].n;
    double* fc = (double*)malloc(sizeof(double) * nc);
    double* ec = (double*)malloc(sizeof(double) * nc);
    if (L->sp_rp) { /* f_c = P_bar^T r, column by column in ascending row order */
        for (int64_t J = 0; J < nc; J++) fc[J] = 0.0;
        for (int64_t i = 0; i < n; i++)
            for (int64_t q = L->sp_rp[i]; q < L->sp_rp[i + 1]; q++) fc[L->sp_ci[q]] = fc[L->sp_ci[q]] + L->sp_v[q] * r[i];
    } else {
        orc_restrict(n, L->agg, L->pval, r, nc, fc);
    }
    vcycle(h, l + 1, fc, ec);
    if (L->sp_rp) { /* x += P_bar e */
        for (int64_t i = 0; i < n; i++) {
            double t = 0.0;
            for (int64_t q = L->sp_rp[i]; q < L->sp_rp[i + 1]; q++) t = t + L->sp_v[q] * ec[L->sp_ci[q]];
            x[i] = x[i] + t;
        }
    } else {
        for (int64_t i = 0; i < n; i++) x[i] = x[i] + L->pval[i] * ec[L->agg[i]];
    }
    if (cheb > 0) {
        orc_cheb4_smooth(n, L->rowptr, L->col, L->val, L->dl1, f, x, r, d, t, cheb, 0);
    } else {
        for (int s = 0; s < h->o.nu_post; s++) {
            residual(L->rowptr, L->col, L->val, n, f, x, r);
            for (int64_t i = 0; i < n; i++) x[i] = x[i] + r[i] / L->dl1[i];
        }
    }
    free(d);
    free(t);
    free(r);
    free(fc);
    free(ec);
}

void orc_vcycle_apply(const orc_hier* h, const double* r, double* z) { vcycle(h, 0, r, z); }

/* ----------------------------------------------------------- Krylov ---- */
/* Preconditioned CG (flexible = 0) or Notay's flexible CG with one stored
 * direction (flexible = 1).  u holds x0 on input and the solution on output.
 * Convergence: ||r_k||_2 <= rtol ||F||_2 on the recursive residual;
 * *relres receives ||F - K u||_2 / ||F||_2 recomputed at the end.
 * history (optional, itmax+1 entries) receives ||r_k|| / ||F||. */
int orc_pcg(const orc_hier* h, const double* Fv, double* u, double rtol, int itmax, int flexible, int* iters,
            double* relres, double* history) {
    const orc_level* L = &h->lev[0];
    const int64_t n = L->n;
    double* r = (double*)malloc(sizeof(double) * n);
    double* z = (double*)malloc(sizeof(double) * n);
    double* p = (double*)malloc(sizeof(double) * n);
    double* q = (double*)malloc(sizeof(double) * n);
    int rc = ORC_OK, it = 0;
    const double nF = sqrt(dot(n, Fv, Fv));
    residual(L->rowptr, L->col, L->val, n, Fv, u, r);
    double nr = sqrt(dot(n, r, r));
    if (history) history[0] = nF > 0.0 ? nr / nF : 0.0;
    if (!(nF > 0.0)) {
        for (int64_t i = 0; i < n; i++) u[i] = 0.0;
        nr = 0.0;
    }
    if (isnan(nr)) rc = ORC_ERR_NAN;
    if (rc == ORC_OK && nr > rtol * nF) {
        vcycle(h, 0, r, z);
        for (int64_t i = 0; i < n; i++) p[i] = z[i];
        double rho = dot(n, r, z);
        for (it = 0; it < itmax;) {
            orc_spmv(n, L->rowptr, L->col, L->val, p, q);
            double pq = dot(n, p, q);
            if (!(pq > 0.0)) { rc = isnan(pq) ? ORC_ERR_NAN : ORC_ERR_BREAKDOWN; break; }
            double alpha = (flexible ? dot(n, p, r) : rho) / pq;
            for (int64_t i = 0; i < n; i++) u[i] = u[i] + alpha * p[i];
            for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
            it++;
            nr = sqrt(dot(n, r, r));
            if (history) history[it] = nr / nF;
            if (isnan(nr)) { rc = ORC_ERR_NAN; break; }
            if (nr <= rtol * nF) break;
            vcycle(h, 0, r, z);
            double beta;
            if (flexible) {
                beta = -dot(n, z, q) / pq;
            } else {
                double rho1 = dot(n, r, z);
                beta = rho1 / rho;
                rho = rho1;
            }
            for (int64_t i = 0; i < n; i++) p[i] = z[i] + beta * p[i];
        }
        if (rc == ORC_OK && nr > rtol * nF) rc = ORC_ERR_NOT_CONVERGED;
    }
    residual(L->rowptr, L->col, L->val, n, Fv, u, r);
    *relres = nF > 0.0 ? sqrt(dot(n, r, r)) / nF : 0.0;
    *iters = it;
    free(r); free(z); free(p); free(q);
    return rc;
}

/* ---------------------------------------------------------- accessors ---- */
int orc_num_levels(const orc_hier* h) { return h->nlev; }
int64_t orc_level_n(const orc_hier* h, int l) { return h->lev[l].n; }
int64_t orc_level_nnz(const orc_hier* h, int l) { return h->lev[l].nnz; }
int orc_level_npass(const orc_hier* h, int l) { return h->lev[l].npass; }
int64_t orc_level_pass_n(const orc_hier* h, int l, int s) { return h->lev[l].pass_n[s]; }
void orc_level_csr(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v) {
    const orc_level* L = &h->lev[l];
    memcpy(rp, L->rowptr, sizeof(int64_t) * (L->n + 1));
    memcpy(ci, L->col, sizeof(int32_t) * L->nnz);
    memcpy(v, L->val, sizeof(double) * L->nnz);
}
void orc_level_vectors(const orc_hier* h, int l, double* dl1, double* w) {
    const orc_level* L = &h->lev[l];
    if (dl1) memcpy(dl1, L->dl1, sizeof(double) * L->n);
    if (w) memcpy(w, L->w, sizeof(double) * L->n);
}
/* composite map (s < 0) or pass s map */
void orc_level_map(const orc_hier* h, int l, int s, int32_t* agg, double* pval, int32_t* mate) {
    const orc_level* L = &h->lev[l];
    if (s < 0) {
        memcpy(agg, L->agg, sizeof(int32_t) * L->n);
        memcpy(pval, L->pval, sizeof(double) * L->n);
        return;
    }
    int64_t n = L->pass_n[s];
    if (agg) memcpy(agg, L->pass_agg[s], sizeof(int32_t) * n);
    if (pval) memcpy(pval, L->pass_pval[s], sizeof(double) * n);
    if (mate) memcpy(mate, L->pass_mate[s], sizeof(int32_t) * n);
}
/* stored entries of level l's smoothed prolongator (0 when tentative) */
int64_t orc_level_sp_nnz(const orc_hier* h, int l) {
    const orc_level* L = &h->lev[l];
    return L->sp_rp ? L->sp_rp[L->n] : 0;
}

void orc_level_sp(const orc_hier* h, int l, int64_t* rp, int32_t* ci, double* v) {
    const orc_level* L = &h->lev[l];
    memcpy(rp, L->sp_rp, sizeof(int64_t) * (L->n + 1));
    memcpy(ci, L->sp_ci, sizeof(int32_t) * L->sp_rp[L->n]);
    memcpy(v, L->sp_v, sizeof(double) * L->sp_rp[L->n]);
}

void orc_coarse_chol(const orc_hier* h, double* L) { memcpy(L, h->chol, sizeof(double) * h->nc * h->nc); }

double orc_opc(const orc_hier* h) {
    double s = 0.0;
    for (int l = 0; l < h->nlev; l++) s += (double)h->lev[l].nnz;
    return s / (double)h->lev[0].nnz;
}
