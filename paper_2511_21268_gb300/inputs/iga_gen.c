/*
 * Seeded input generator: IgA stiffness systems K u = F for the Poisson
 * problem -div(kappa grad u) = f with homogeneous Dirichlet data on the whole
 * boundary, discretised with tensor-product B-splines of degree p and maximal
 * regularity C^{p-1} on n uniform elements per direction.
 *
 * This module produces the INPUTS of the AMG-PCG path (matrix K in CSR, load
 * vector F, seeded random vectors). It contains none of the solver's
 * arithmetic and is shared by the CPU oracle and the GPU path.
 *
 * Paper passages followed (arXiv 2511.21268):
 *   Sec. 2 (Poisson weak form, eq. "poisson"), Sec. 2.1 (B-spline / NURBS
 *   bases, geometry map), Sec. 2.2 (stiffness pull-back
 *   k_ij = int (grad R_j)^T J^-T J^-1 grad R_i det J, element loop and
 *   local-to-global scatter, Dirichlet DOFs fixed by elimination),
 *   Sec. 2.4 (non-isoparametric: NURBS geometry, B-spline solution space).
 *
 * Two assembly routes:
 *   - iga_assemble_kron: unit square / unit cube with kappa = 1.  The
 *     stiffness matrix of a tensor-product space on a Cartesian box is the
 *     sum over directions of Kronecker products of 1-D stiffness and mass
 *     matrices; the 1-D matrices are computed by (p+1)-point Gauss
 *     quadrature, which is exact for these polynomial integrands.
 *   - iga_assemble_elem: the plain element loop with Gauss quadrature on any
 *     of the supported geometry maps (identity box, NURBS quarter annulus
 *     extruded in z) and a variable coefficient kappa(x).
 * Both return a bitwise symmetric K: every (i,j) and (j,i) entry is produced
 * by the same floating-point expression.
 *
 * Compiled with -ffp-contract=off so that results are identical on x86-64
 * and aarch64 hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IGA_MAXP 8
#define IGA_MAXQ 16

/* ---------------------------------------------------------------- RNG ---- */
/* SplitMix64 (Steele, Lea, Flood 2014): the k-th output (k = 0, 1, ...) of
 * the stream seeded with `seed` is mix(seed + (k+1) * golden). */
static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}
static uint64_t sm64_at(uint64_t seed, uint64_t k) {
    return sm64_mix(seed + (k + 1) * 0x9e3779b97f4a7c15ULL);
}
static double u01_from(uint64_t z) { return (double)(z >> 11) * 0x1.0p-53; }

/* out[k] = U[0,1) draw k of SplitMix64(seed). */
void iga_rng_u01(uint64_t seed, int64_t count, double* out) {
    for (int64_t k = 0; k < count; k++) out[k] = u01_from(sm64_at(seed, (uint64_t)k));
}

/* out[k] ~ N(0,1) by the Box-Muller transform of the uniform pair
 * (u_{2m}, u_{2m+1}) of SplitMix64(seed): z_{2m} = R cos(2 pi u'), z_{2m+1} =
 * R sin(2 pi u'), R = sqrt(-2 ln(1 - u)). */
void iga_rng_normal(uint64_t seed, int64_t count, double* out) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t m = 0; 2 * m < count; m++) {
        double u = u01_from(sm64_at(seed, (uint64_t)(2 * m)));
        double v = u01_from(sm64_at(seed, (uint64_t)(2 * m + 1)));
        double R = sqrt(-2.0 * log(1.0 - u));
        out[2 * m] = R * cos(two_pi * v);
        if (2 * m + 1 < count) out[2 * m + 1] = R * sin(two_pi * v);
    }
}

/* --------------------------------------------------------- quadrature ---- */
/* q-point Gauss-Legendre rule on [-1,1]: nodes are the roots of P_q found by
 * Newton's method on the three-term recurrence; w = 2 / ((1-x^2) P_q'(x)^2). */
static void legendre_eval(int q, double t, double* pq, double* dpq) {
    double pk = t, pkm1 = 1.0;
    for (int k = 2; k <= q; k++) {
        double pn = ((2.0 * k - 1.0) * t * pk - (k - 1.0) * pkm1) / k;
        pkm1 = pk;
        pk = pn;
    }
    if (q == 1) { pk = t; pkm1 = 1.0; }
    *pq = pk;
    *dpq = q * (t * pk - pkm1) / (t * t - 1.0);
}

int iga_gauss_legendre(int q, double* x, double* w) {
    const double pi = 3.14159265358979323846264338328;
    if (q < 1 || q > IGA_MAXQ) return -1;
    for (int i = 0; i < q; i++) {
        double t = cos(pi * (i + 0.75) / (q + 0.5)), pq, dp;
        for (int it = 0; it < 100; it++) {
            legendre_eval(q, t, &pq, &dp);
            double dt = pq / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        legendre_eval(q, t, &pq, &dp);
        x[q - 1 - i] = t; /* ascending */
        w[q - 1 - i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
    return 0;
}

/* --------------------------------------------------------- B-splines ---- */
/* Open uniform knot vector on [0,1] with n elements, degree p: p+1 zeros,
 * the interior knots 1/n..(n-1)/n, p+1 ones (n + 2p + 1 knots, n + p basis
 * functions, maximal regularity C^{p-1}). */
static double knot(int n, int p, int i) {
    if (i <= p) return 0.0;
    if (i >= n + p) return 1.0;
    return (double)(i - p) / (double)n;
}

/* Values and first derivatives of the p+1 B-splines that are nonzero on
 * element e (functions e..e+p) at the point xi of that element, by the
 * Cox-de Boor recursion
 *   N_{i,0} = 1 on [u_i, u_{i+1}),
 *   N_{i,k} = (xi-u_i)/(u_{i+k}-u_i) N_{i,k-1}
 *           + (u_{i+k+1}-xi)/(u_{i+k+1}-u_{i+1}) N_{i+1,k-1}   (0/0 := 0),
 *   N'_{i,p} = p N_{i,p-1}/(u_{i+p}-u_i) - p N_{i+1,p-1}/(u_{i+p+1}-u_{i+1}).
 * vals[a], ders[a] belong to global function e+a. */
void iga_bspline_local(int n, int p, int e, double xi, double* vals, double* ders) {
    /* B[k][a]: degree-k function with global index e + p - k + a, a = 0..k */
    double B[IGA_MAXP + 1][IGA_MAXP + 2];
    memset(B, 0, sizeof(B));
    const int s = e + p; /* knot span index */
    B[0][0] = 1.0;
    for (int k = 1; k <= p; k++) {
        for (int a = 0; a <= k; a++) {
            int i = s - k + a;
            double left = 0.0, right = 0.0;
            /* N_{i,k-1} has index a-1 in row k-1 (global s-(k-1)+(a-1) = i) */
            if (a >= 1) {
                double den = knot(n, p, i + k) - knot(n, p, i);
                if (den > 0.0) left = (xi - knot(n, p, i)) / den * B[k - 1][a - 1];
            }
            /* N_{i+1,k-1} has index a in row k-1 */
            if (a <= k - 1) {
                double den = knot(n, p, i + k + 1) - knot(n, p, i + 1);
                if (den > 0.0) right = (knot(n, p, i + k + 1) - xi) / den * B[k - 1][a];
            }
            B[k][a] = left + right;
        }
    }
    for (int a = 0; a <= p; a++) vals[a] = B[p][a];
    if (p == 0) {
        ders[0] = 0.0;
        return;
    }
    for (int a = 0; a <= p; a++) {
        int i = s - p + a;
        double d = 0.0;
        if (a >= 1) {
            double den = knot(n, p, i + p) - knot(n, p, i);
            if (den > 0.0) d += p * B[p - 1][a - 1] / den;
        }
        if (a <= p - 1) {
            double den = knot(n, p, i + p + 1) - knot(n, p, i + 1);
            if (den > 0.0) d -= p * B[p - 1][a] / den;
        }
        ders[a] = d;
    }
}

/* All n+p basis functions at xi in [0,1] (dense output, for tests). */
void iga_bspline_all(int n, int p, double xi, double* vals, double* ders) {
    int e = (int)floor(xi * n);
    if (e >= n) e = n - 1;
    if (e < 0) e = 0;
    double v[IGA_MAXP + 1], d[IGA_MAXP + 1];
    iga_bspline_local(n, p, e, xi, v, d);
    for (int i = 0; i < n + p; i++) { vals[i] = 0.0; ders[i] = 0.0; }
    for (int a = 0; a <= p; a++) { vals[e + a] = v[a]; ders[e + a] = d[a]; }
}

/* 1-D stiffness K1_ij = int_0^1 N_i' N_j' dx and mass M1_ij = int N_i N_j dx
 * over all n+p functions (dense row-major (n+p)^2), nq-point Gauss rule per
 * element.  Each entry is accumulated in the order (element asc, point asc)
 * from the commutative product N_i N_j, so K1, M1 are bitwise symmetric. */
int iga_1d_matrices(int n, int p, int nq, double* K1, double* M1) {
    if (p < 1 || p > IGA_MAXP || nq < 1 || nq > IGA_MAXQ || n < 1) return -1;
    const int nb = n + p;
    double gx[IGA_MAXQ], gw[IGA_MAXQ];
    iga_gauss_legendre(nq, gx, gw);
    memset(K1, 0, sizeof(double) * nb * nb);
    memset(M1, 0, sizeof(double) * nb * nb);
    const double h = 1.0 / n;
    for (int e = 0; e < n; e++) {
        for (int q = 0; q < nq; q++) {
            double xi = (e + 0.5 * (gx[q] + 1.0)) * h;
            double wq = 0.5 * h * gw[q];
            double v[IGA_MAXP + 1], d[IGA_MAXP + 1];
            iga_bspline_local(n, p, e, xi, v, d);
            for (int a = 0; a <= p; a++)
                for (int b = 0; b <= p; b++) {
                    int i = e + a, j = e + b;
                    K1[i * nb + j] += (d[a] * d[b]) * wq;
                    M1[i * nb + j] += (v[a] * v[b]) * wq;
                }
        }
    }
    return 0;
}

/* ------------------------------------------------------ CSR structure ---- */
/* DOFs: per direction, functions `off .. off+m-1` where off = 1, m = n+p-2
 * after eliminating the Dirichlet functions (the first and last function of
 * each direction are the only ones nonzero on the boundary), or off = 0,
 * m = n+p for the matrix before boundary conditions.  Global DOF index
 * I = i1 + m (i2 + m i3), x fastest.  Row I couples to every J with
 * |i_k - j_k| <= p in each direction; columns sorted ascending. */
static int64_t band_count(int m, int p) {
    int64_t c = 0;
    for (int i = 0; i < m; i++) {
        int lo = i - p < 0 ? 0 : i - p, hi = i + p > m - 1 ? m - 1 : i + p;
        c += hi - lo + 1;
    }
    return c;
}

int64_t iga_num_dofs(int d, int n, int p, int with_boundary) {
    int64_t m = with_boundary ? n + p : n + p - 2;
    return d == 2 ? m * m : m * m * m;
}

int64_t iga_nnz(int d, int n, int p, int with_boundary) {
    int m = with_boundary ? n + p : n + p - 2;
    int64_t c = band_count(m, p);
    return d == 2 ? c * c : c * c * c;
}

/* Fill rowptr / col for the tensor band pattern. */
static void build_pattern(int d, int m, int p, int64_t* rowptr, int32_t* col) {
    int64_t N = (d == 2) ? (int64_t)m * m : (int64_t)m * m * m;
    int64_t pos = 0;
    rowptr[0] = 0;
    for (int64_t I = 0; I < N; I++) {
        int i1 = (int)(I % m), i2 = (int)((I / m) % m), i3 = (d == 3) ? (int)(I / ((int64_t)m * m)) : 0;
        int lo1 = i1 - p < 0 ? 0 : i1 - p, hi1 = i1 + p > m - 1 ? m - 1 : i1 + p;
        int lo2 = i2 - p < 0 ? 0 : i2 - p, hi2 = i2 + p > m - 1 ? m - 1 : i2 + p;
        int lo3 = 0, hi3 = 0;
        if (d == 3) { lo3 = i3 - p < 0 ? 0 : i3 - p; hi3 = i3 + p > m - 1 ? m - 1 : i3 + p; }
        for (int j3 = lo3; j3 <= hi3; j3++)
            for (int j2 = lo2; j2 <= hi2; j2++)
                for (int j1 = lo1; j1 <= hi1; j1++)
                    col[pos++] = (int32_t)(j1 + (int64_t)m * (j2 + (int64_t)m * j3));
        rowptr[I + 1] = pos;
    }
}

/* Position of column (j1,j2,j3) inside row (i1,i2,i3). */
static inline int64_t pat_pos(int d, int m, int p, int i1, int i2, int i3, int j1, int j2, int j3) {
    int lo1 = i1 - p < 0 ? 0 : i1 - p, hi1 = i1 + p > m - 1 ? m - 1 : i1 + p;
    int lo2 = i2 - p < 0 ? 0 : i2 - p;
    int w1 = hi1 - lo1 + 1;
    int64_t r = (int64_t)(j2 - lo2) * w1 + (j1 - lo1);
    if (d == 3) {
        int lo3 = i3 - p < 0 ? 0 : i3 - p;
        int hi2 = i2 + p > m - 1 ? m - 1 : i2 + p;
        int w2 = hi2 - lo2 + 1;
        r += (int64_t)(j3 - lo3) * w2 * w1;
    }
    return r;
}

/* ------------------------------------------ box with per-direction DOFs ---- */
/* 3-D unit cube, K restricted to the DOFs (i1, i2, i3) with lo[k] <= i_k <
 * hi[k] (indices of the full tensor space of n + p functions per direction,
 * x fastest): the system of a box whose faces carry Dirichlet data on some
 * sides only (the eliminated faces are the excluded index planes).  Same
 * entry expression as iga_assemble_kron; rows and columns numbered
 * (i1 - lo1) + m1 ((i2 - lo2) + m2 (i3 - lo3)), columns sorted. */
int iga_kron_box_nnz(int n, int p, const int* lo, const int* hi, int64_t* nnz) {
    if (p < 1 || p > IGA_MAXP || n < 1) return -1;
    const int nb = n + p;
    int64_t prod = 1;
    for (int k = 0; k < 3; k++) {
        if (lo[k] < 0 || hi[k] > nb || hi[k] <= lo[k]) return -1;
        const int m = hi[k] - lo[k];
        int64_t c = 0;
        for (int i = 0; i < m; i++) {
            const int a = i - p < 0 ? 0 : i - p, b = i + p > m - 1 ? m - 1 : i + p;
            c += b - a + 1;
        }
        prod *= c;
    }
    *nnz = prod;
    return 0;
}

int iga_assemble_kron_box(int n, int p, const int* lo, const int* hi, int64_t* rowptr, int32_t* col, double* val) {
    int64_t z;
    if (iga_kron_box_nnz(n, p, lo, hi, &z) != 0) return -1;
    const int nb = n + p;
    const int m1 = hi[0] - lo[0], m2 = hi[1] - lo[1], m3 = hi[2] - lo[2];
    double* K1 = (double*)malloc(sizeof(double) * nb * nb);
    double* M1 = (double*)malloc(sizeof(double) * nb * nb);
    if (!K1 || !M1) { free(K1); free(M1); return -2; }
    iga_1d_matrices(n, p, p + 1, K1, M1);
    const int64_t N = (int64_t)m1 * m2 * m3;
    int64_t pos = 0;
    rowptr[0] = 0;
    for (int64_t I = 0; I < N; I++) {
        const int i1 = (int)(I % m1), i2 = (int)((I / m1) % m2), i3 = (int)(I / ((int64_t)m1 * m2));
        const int a1 = i1 - p < 0 ? 0 : i1 - p, b1 = i1 + p > m1 - 1 ? m1 - 1 : i1 + p;
        const int a2 = i2 - p < 0 ? 0 : i2 - p, b2 = i2 + p > m2 - 1 ? m2 - 1 : i2 + p;
        const int a3 = i3 - p < 0 ? 0 : i3 - p, b3 = i3 + p > m3 - 1 ? m3 - 1 : i3 + p;
        const int g1 = i1 + lo[0], g2 = i2 + lo[1], g3 = i3 + lo[2];
        for (int j3 = a3; j3 <= b3; j3++)
            for (int j2 = a2; j2 <= b2; j2++)
                for (int j1 = a1; j1 <= b1; j1++) {
                    const int h1 = j1 + lo[0], h2 = j2 + lo[1], h3 = j3 + lo[2];
                    const double kx = K1[g1 * nb + h1], mx = M1[g1 * nb + h1];
                    const double ky = K1[g2 * nb + h2], my = M1[g2 * nb + h2];
                    const double kz = K1[g3 * nb + h3], mz = M1[g3 * nb + h3];
                    col[pos] = (int32_t)(j1 + (int64_t)m1 * (j2 + (int64_t)m2 * j3));
                    val[pos] = ((kx * my) * mz + (mx * ky) * mz) + (mx * my) * kz;
                    pos++;
                }
        rowptr[I + 1] = pos;
    }
    free(K1);
    free(M1);
    return pos == z ? 0 : -3;
}

/* ------------------------------------------------ three-patch L-shape ---- */
/* Three unit-cube patches with the same open knot vectors (n elements,
 * degree p, m = n + p functions per direction), conforming along their
 * shared faces: A = [0,1]x[0,1], B = [-1,0]x[0,1], C = [0,1]x[-1,0] in
 * (x, y), each times [0,1] in z.  Their functions sit on a (2m-1) x (2m-1)
 * lattice in (x, y) (B: gx < m, A and C: gx >= m-1; C: gy < m, A and B:
 * gy >= m-1), the quadrant gx < m-1, gy < m-1 being absent; a function on
 * an interface line belongs to both patches (C^0 coupling).  Two functions
 * couple through every patch that holds both; the entry is the sum over
 * those patches (in the order A, B, C) of the unit-cube Kronecker entry
 * ((kx my) mz + (mx ky) mz) + (mx my) kz in patch-local indices.  The
 * kept functions are the lattice points with keep2[gy (2m-1) + gx] != 0
 * times the z indices [z0, z1), numbered x fastest, then y, then z; columns
 * sorted; cap bounds the stored entries. */
static int lshape_patch_has(int m, int pidx, int gx, int gy) {
    switch (pidx) {
        case 0: return gx >= m - 1 && gy >= m - 1;  /* A */
        case 1: return gx <= m - 1 && gy >= m - 1;  /* B */
        default: return gx >= m - 1 && gy <= m - 1; /* C */
    }
}
static int lshape_off(int m, int pidx, int axis) {
    if (axis == 0) return pidx == 1 ? 0 : m - 1;
    return pidx == 2 ? 0 : m - 1;
}

int iga_assemble_lshape(int n, int p, const uint8_t* keep2, int z0, int z1, int64_t* rowptr, int32_t* col,
                        double* val, int64_t cap) {
    if (p < 1 || p > IGA_MAXP || n < 1 || z0 < 0 || z1 > n + p || z1 <= z0) return -1;
    const int m = n + p, L = 2 * m - 1, mz = z1 - z0;
    double* K1 = (double*)malloc(sizeof(double) * m * m);
    double* M1 = (double*)malloc(sizeof(double) * m * m);
    int64_t* idx2 = (int64_t*)malloc(sizeof(int64_t) * L * L);
    if (!K1 || !M1 || !idx2) { free(K1); free(M1); free(idx2); return -2; }
    iga_1d_matrices(n, p, p + 1, K1, M1);
    int64_t n2 = 0;
    for (int gy = 0; gy < L; gy++)
        for (int gx = 0; gx < L; gx++) {
            const int in = lshape_patch_has(m, 0, gx, gy) || lshape_patch_has(m, 1, gx, gy) ||
                           lshape_patch_has(m, 2, gx, gy);
            idx2[gy * L + gx] = (in && keep2[gy * L + gx]) ? n2++ : -1;
        }
    int64_t pos = 0, row = 0;
    rowptr[0] = 0;
    for (int iz = z0; iz < z1; iz++)
        for (int gy = 0; gy < L; gy++)
            for (int gx = 0; gx < L; gx++) {
                if (idx2[gy * L + gx] < 0) continue;
                for (int jz = (iz - p > z0 ? iz - p : z0); jz <= (iz + p < z1 - 1 ? iz + p : z1 - 1); jz++)
                    for (int hy = (gy - p > 0 ? gy - p : 0); hy <= (gy + p < L - 1 ? gy + p : L - 1); hy++)
                        for (int hx = (gx - p > 0 ? gx - p : 0); hx <= (gx + p < L - 1 ? gx + p : L - 1); hx++) {
                            const int64_t j2 = idx2[hy * L + hx];
                            if (j2 < 0) continue;
                            double v = 0.0;
                            int any = 0;
                            for (int P = 0; P < 3; P++) {
                                if (!lshape_patch_has(m, P, gx, gy) || !lshape_patch_has(m, P, hx, hy)) continue;
                                const int ax = gx - lshape_off(m, P, 0), bx = hx - lshape_off(m, P, 0);
                                const int ay = gy - lshape_off(m, P, 1), by = hy - lshape_off(m, P, 1);
                                const double kx = K1[ax * m + bx], mx = M1[ax * m + bx];
                                const double ky = K1[ay * m + by], my = M1[ay * m + by];
                                const double kz = K1[iz * m + jz], mzz = M1[iz * m + jz];
                                const double e = ((kx * my) * mzz + (mx * ky) * mzz) + (mx * my) * kz;
                                v = any ? v + e : e;
                                any = 1;
                            }
                            if (!any) continue;
                            if (pos >= cap) { free(K1); free(M1); free(idx2); return -3; }
                            col[pos] = (int32_t)(j2 + n2 * (int64_t)(jz - z0));
                            val[pos] = v;
                            pos++;
                        }
                rowptr[++row] = pos;
            }
    (void)mz;
    free(K1);
    free(M1);
    free(idx2);
    return 0;
}

/* ------------------------------------------------- Kronecker assembly ---- */
/* K = K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1 on the unit cube
 * (two terms on the unit square), restricted to the DOF set.  The entry for
 * (I,J) is ((t1 + t2) + t3) with t1 = (K1x * M1y) * M1z, etc. */
int iga_assemble_kron(int d, int n, int p, int with_boundary, int64_t* rowptr, int32_t* col, double* val) {
    if ((d != 2 && d != 3) || p < 1 || p > IGA_MAXP || n < 1) return -1;
    const int nb = n + p, off = with_boundary ? 0 : 1, m = with_boundary ? nb : nb - 2;
    if (m < 1) return -1;
    double* K1 = (double*)malloc(sizeof(double) * nb * nb);
    double* M1 = (double*)malloc(sizeof(double) * nb * nb);
    if (!K1 || !M1) { free(K1); free(M1); return -2; }
    iga_1d_matrices(n, p, p + 1, K1, M1);
    build_pattern(d, m, p, rowptr, col);
    const int64_t N = (d == 2) ? (int64_t)m * m : (int64_t)m * m * m;
    for (int64_t I = 0; I < N; I++) {
        int i1 = (int)(I % m) + off, i2 = (int)((I / m) % m) + off;
        int i3 = (d == 3) ? (int)(I / ((int64_t)m * m)) + off : 0;
        for (int64_t k = rowptr[I]; k < rowptr[I + 1]; k++) {
            int64_t J = col[k];
            int j1 = (int)(J % m) + off, j2 = (int)((J / m) % m) + off;
            int j3 = (d == 3) ? (int)(J / ((int64_t)m * m)) + off : 0;
            double kx = K1[i1 * nb + j1], mx = M1[i1 * nb + j1];
            double ky = K1[i2 * nb + j2], my = M1[i2 * nb + j2];
            if (d == 2) {
                val[k] = kx * my + mx * ky;
            } else {
                double kz = K1[i3 * nb + j3], mz = M1[i3 * nb + j3];
                double t1 = (kx * my) * mz, t2 = (mx * ky) * mz, t3 = (mx * my) * kz;
                val[k] = (t1 + t2) + t3;
            }
        }
    }
    free(K1);
    free(M1);
    return 0;
}

/* Load vector for the manufactured solution u = prod_k sin(pi x_k) on the
 * unit box: f = d pi^2 u, separable, F_I = d pi^2 prod_k b_{i_k} with
 * b_i = int_0^1 sin(pi x) N_i(x) dx by an nq-point Gauss rule per element. */
int iga_load_sine(int d, int n, int p, int nq, int with_boundary, double* F) {
    const double pi = 3.14159265358979323846264338328;
    if ((d != 2 && d != 3) || p < 1 || p > IGA_MAXP || nq < 1 || nq > IGA_MAXQ) return -1;
    const int nb = n + p, off = with_boundary ? 0 : 1, m = with_boundary ? nb : nb - 2;
    double* b = (double*)calloc(nb, sizeof(double));
    double gx[IGA_MAXQ], gw[IGA_MAXQ];
    iga_gauss_legendre(nq, gx, gw);
    const double h = 1.0 / n;
    for (int e = 0; e < n; e++)
        for (int q = 0; q < nq; q++) {
            double xi = (e + 0.5 * (gx[q] + 1.0)) * h, wq = 0.5 * h * gw[q];
            double v[IGA_MAXP + 1], dd[IGA_MAXP + 1];
            iga_bspline_local(n, p, e, xi, v, dd);
            double s = sin(pi * xi);
            for (int a = 0; a <= p; a++) b[e + a] += (s * v[a]) * wq;
        }
    const double c = d * pi * pi;
    const int64_t N = (d == 2) ? (int64_t)m * m : (int64_t)m * m * m;
    for (int64_t I = 0; I < N; I++) {
        int i1 = (int)(I % m) + off, i2 = (int)((I / m) % m) + off;
        double v = (c * b[i1]) * b[i2];
        if (d == 3) v = v * b[(int)(I / ((int64_t)m * m)) + off];
        F[I] = v;
    }
    free(b);
    return 0;
}

/* ------------------------------------------------- geometry + kappa ---- */
/* geom 0: identity map on [0,1]^d.
 * geom 1 (d = 3 only): quarter annulus of radii 1 and 2 extruded over
 *   z in [0,1]: xi1 -> radius r = 1 + xi1 (linear), xi2 -> the exact quarter
 *   circle given by the quadratic NURBS arc with control points (1,0), (1,1),
 *   (0,1) and weights 1, sqrt(2)/2, 1, xi3 -> z.  The solution space stays
 *   the B-spline space on the parametric cube (non-isoparametric, Sec. 2.4). */
static void geom_eval(int geom, int d, const double* xi, double* x, double J[3][3]) {
    if (geom == 0) {
        for (int a = 0; a < d; a++) {
            x[a] = xi[a];
            for (int b = 0; b < d; b++) J[a][b] = (a == b) ? 1.0 : 0.0;
        }
        return;
    }
    /* quadratic NURBS arc */
    const double t = xi[1];
    const double wmid = 0.70710678118654752440084436210;
    const double B0 = (1 - t) * (1 - t), B1 = 2 * t * (1 - t), B2 = t * t;
    const double dB0 = -2 * (1 - t), dB1 = 2 - 4 * t, dB2 = 2 * t;
    const double W = B0 + wmid * B1 + B2, dW = dB0 + wmid * dB1 + dB2;
    const double Ax = B0 * 1.0 + wmid * B1 * 1.0 + B2 * 0.0;
    const double Ay = B0 * 0.0 + wmid * B1 * 1.0 + B2 * 1.0;
    const double dAx = dB0 + wmid * dB1, dAy = wmid * dB1 + dB2;
    const double cx = Ax / W, cy = Ay / W;
    const double dcx = (dAx * W - Ax * dW) / (W * W), dcy = (dAy * W - Ay * dW) / (W * W);
    const double r = 1.0 + xi[0];
    x[0] = r * cx;
    x[1] = r * cy;
    x[2] = xi[2];
    J[0][0] = cx;  J[0][1] = r * dcx; J[0][2] = 0.0;
    J[1][0] = cy;  J[1][1] = r * dcy; J[1][2] = 0.0;
    J[2][0] = 0.0; J[2][1] = 0.0;     J[2][2] = 1.0;
}

/* kappa(x) = exp(g(x)), g a Gaussian random field of correlation length ell
 * and standard deviation sigma sampled by M random Fourier features:
 *   g(x) = sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m),
 *   omega_m ~ N(0, ell^-2 I) (normals 3m..3m+2 of stream `seed`),
 *   phi_m ~ U[0, 2 pi) (uniform m of stream seed + 1).
 * M = 0 gives kappa = 1. */
typedef struct {
    int M;
    double sigma;
    double* omega; /* 3M */
    double* phi;   /* M */
} kappa_field;

static void kappa_init(kappa_field* k, int M, double ell, double sigma, uint64_t seed) {
    const double two_pi = 6.283185307179586476925286766559;
    k->M = M;
    k->sigma = sigma;
    k->omega = NULL;
    k->phi = NULL;
    if (M <= 0) return;
    k->omega = (double*)malloc(sizeof(double) * 3 * M);
    k->phi = (double*)malloc(sizeof(double) * M);
    iga_rng_normal(seed, 3 * (int64_t)M, k->omega);
    for (int i = 0; i < 3 * M; i++) k->omega[i] /= ell;
    iga_rng_u01(seed + 1, M, k->phi);
    for (int i = 0; i < M; i++) k->phi[i] *= two_pi;
}
static void kappa_free(kappa_field* k) { free(k->omega); free(k->phi); }
static double kappa_eval(const kappa_field* k, int d, const double* x) {
    if (k->M <= 0) return 1.0;
    double g = 0.0;
    for (int m = 0; m < k->M; m++) {
        double a = k->phi[m];
        for (int c = 0; c < d; c++) a += k->omega[3 * m + c] * x[c];
        g += cos(a);
    }
    return exp(k->sigma * sqrt(2.0 / k->M) * g);
}

/* Exposed for tests: kappa at a list of points (npts x 3). */
void iga_kappa_points(int M, double ell, double sigma, uint64_t seed, int64_t npts, const double* x, double* out) {
    kappa_field kf;
    kappa_init(&kf, M, ell, sigma, seed);
    for (int64_t i = 0; i < npts; i++) out[i] = kappa_eval(&kf, 3, x + 3 * i);
    kappa_free(&kf);
}

/* Geometry map exposed for tests: x and det J at parametric points. */
void iga_geom_points(int geom, int d, int64_t npts, const double* xi, double* x, double* detJ) {
    for (int64_t i = 0; i < npts; i++) {
        double J[3][3];
        geom_eval(geom, d, xi + d * i, x + d * i, J);
        if (d == 2) detJ[i] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        else
            detJ[i] = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                      J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    }
}

/* ---------------------------------------------------- element loop ---- */
/* k_ij = sum_e sum_q kappa(x_q) w_q |det J| (J^-T grad_xi N_i) . (J^-T grad_xi N_j),
 * F_i = sum_e sum_q f(x_q) N_i |det J| w_q, with f = 1 (fkind 0) or the
 * manufactured source d pi^2 prod sin(pi x_k) (fkind 1, identity geometry);
 * nq Gauss points per direction.
 *
 * Element matrices: with B_q = sqrt(kappa w |det J|) J^-T grad_xi N (d x nloc),
 * k^e = sum_q B_q^T B_q (upper triangle, in that order).  Elements are
 * processed plane by plane (fixed e3): the element matrices of a plane are
 * computed in parallel, then scattered into the upper triangle of K in
 * parallel by ranges of the second row index, each entry receiving the
 * element contributions in lexicographic element order (x fastest) -- the
 * order of a sequential element loop, so the result does not depend on the
 * thread count.  The lower triangle is mirrored at the end.
 *
 * kappa = exp(g), g = sigma sqrt(2/M) sum_m cos(w_m . x + phi_m): with
 * x = (x(xi1, xi2), y(xi1, xi2), z(xi3)) (both geometries are extruded in
 * z), cos(a + b) = cos a cos b - sin a sin b separates the (xi1, xi2) and
 * xi3 parts, so kappa at all quadrature points costs M sines and cosines
 * per point of each factor plus an M-term product sum per point. */
#include <pthread.h>
#include <unistd.h>

typedef struct {
    int d, n, p, nq, geom, off, m, P1, nloc, nqe, fkind, e3;
    double h;
    const double *V, *D, *gx, *gw;
    const double* kap;  /* [z point][2-D point] or NULL (kappa = 1) */
    double* ke;         /* [n^(d-1) elements of the plane][nloc (nloc+1) / 2] */
    double* fe;         /* [elements][nloc] */
    const int64_t* rowptr;
    const int32_t* col;
    double* val;
    double* F;
    int nthreads;
} elem_ctx;

typedef struct {
    elem_ctx* c;
    int t;
} elem_job;

static int num_threads(void) {
    long t = sysconf(_SC_NPROCESSORS_ONLN);
    if (t < 1) t = 1;
    if (t > 32) t = 32;
    return (int)t;
}

/* Run fn(job) on nthreads threads (thread t gets job t; a job whose thread
 * cannot be created runs on the calling thread). */
static void run_parallel(void* (*fn)(void*), elem_ctx* c) {
    pthread_t th[32];
    elem_job jobs[32];
    int joined[32];
    for (int t = 0; t < c->nthreads; t++) {
        jobs[t].c = c;
        jobs[t].t = t;
        joined[t] = 0;
        if (t > 0) {
            if (pthread_create(&th[t], NULL, fn, &jobs[t]) == 0) joined[t] = 1;
            else fn(&jobs[t]);
        }
    }
    fn(&jobs[0]);
    for (int t = 1; t < c->nthreads; t++)
        if (joined[t]) pthread_join(th[t], NULL);
}

/* element matrix and load vector of element (e1, e2, c->e3) */
static void element(const elem_ctx* c, int e1, int e2, double* ke, double* fe) {
    const double pi = 3.14159265358979323846264338328;
    const int d = c->d, nq = c->nq, P1 = c->P1, nloc = c->nloc, n = c->n, e3 = c->e3;
    const double h = c->h;
    double B[3][729]; /* nloc <= (IGA_MAXP + 1)^3 = 729 */
    double N[729];
    memset(ke, 0, sizeof(double) * nloc * (nloc + 1) / 2);
    memset(fe, 0, sizeof(double) * nloc);
    for (int qq = 0; qq < c->nqe; qq++) {
        const int q1 = qq % nq, q2 = (qq / nq) % nq, q3 = (d == 3) ? qq / (nq * nq) : 0;
        const double xi[3] = {(e1 + 0.5 * (c->gx[q1] + 1.0)) * h, (e2 + 0.5 * (c->gx[q2] + 1.0)) * h,
                              (d == 3) ? (e3 + 0.5 * (c->gx[q3] + 1.0)) * h : 0.0};
        double wq = (0.5 * h * c->gw[q1]) * (0.5 * h * c->gw[q2]);
        if (d == 3) wq *= 0.5 * h * c->gw[q3];
        double x[3] = {0, 0, 0}, J[3][3];
        geom_eval(c->geom, d, xi, x, J);
        double inv[3][3], detJ;
        if (d == 2) {
            detJ = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            inv[0][0] = J[1][1] / detJ;
            inv[0][1] = -J[0][1] / detJ;
            inv[1][0] = -J[1][0] / detJ;
            inv[1][1] = J[0][0] / detJ;
        } else {
            const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            detJ = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
            inv[0][0] = c00 / detJ;
            inv[1][0] = c01 / detJ;
            inv[2][0] = c02 / detJ;
            inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / detJ;
            inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / detJ;
            inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / detJ;
            inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / detJ;
            inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / detJ;
            inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / detJ;
        }
        double kap = 1.0;
        if (c->kap) {
            const int nqn = n * nq;
            const int64_t ip2 = (int64_t)(e2 * nq + q2) * nqn + (e1 * nq + q1);
            const int64_t iz = (d == 3) ? (int64_t)(e3 * nq + q3) : 0;
            kap = c->kap[iz * (int64_t)nqn * nqn + ip2];
        }
        double fval = 1.0;
        if (c->fkind == 1) {
            fval = d * pi * pi;
            for (int k = 0; k < d; k++) fval *= sin(pi * x[k]);
        }
        const double sc = sqrt(kap * wq * fabs(detJ));
        const double* v1 = c->V + (e1 * nq + q1) * P1;
        const double* d1 = c->D + (e1 * nq + q1) * P1;
        const double* v2 = c->V + (e2 * nq + q2) * P1;
        const double* d2 = c->D + (e2 * nq + q2) * P1;
        const double* v3 = c->V + (e3 * nq + q3) * P1;
        const double* d3 = c->D + (e3 * nq + q3) * P1;
        for (int l = 0; l < nloc; l++) {
            const int a1 = l % P1, a2 = (l / P1) % P1, a3 = (d == 3) ? l / (P1 * P1) : 0;
            double g[3];
            if (d == 2) {
                g[0] = d1[a1] * v2[a2];
                g[1] = v1[a1] * d2[a2];
                g[2] = 0.0;
                N[l] = v1[a1] * v2[a2];
            } else {
                g[0] = d1[a1] * v2[a2] * v3[a3];
                g[1] = v1[a1] * d2[a2] * v3[a3];
                g[2] = v1[a1] * v2[a2] * d3[a3];
                N[l] = v1[a1] * v2[a2] * v3[a3];
            }
            /* physical gradient J^-T g, scaled */
            for (int r = 0; r < d; r++) {
                double t = 0.0;
                for (int k = 0; k < d; k++) t += inv[k][r] * g[k];
                B[r][l] = sc * t;
            }
        }
        const double fw = fval * fabs(detJ) * wq;
        int64_t pos = 0;
        for (int a = 0; a < nloc; a++) {
            double* row = ke + pos - a; /* row[b] for b >= a */
            const double b0 = B[0][a], b1 = B[1][a], b2 = d == 3 ? B[2][a] : 0.0;
            if (d == 3) {
                for (int b = a; b < nloc; b++) row[b] += (b0 * B[0][b] + b1 * B[1][b]) + b2 * B[2][b];
            } else {
                for (int b = a; b < nloc; b++) row[b] += b0 * B[0][b] + b1 * B[1][b];
            }
            pos += nloc - a;
            fe[a] += fw * N[a];
        }
    }
}

static void* compute_job(void* arg) {
    elem_job* j = (elem_job*)arg;
    elem_ctx* c = j->c;
    const int n = c->n, nel = n * n;
    const int64_t kes = (int64_t)c->nloc * (c->nloc + 1) / 2;
    for (int el = j->t; el < nel; el += c->nthreads) {
        const int e1 = el % n, e2 = el / n;
        element(c, e1, e2, c->ke + el * kes, c->fe + (int64_t)el * c->nloc);
    }
    return NULL;
}

/* scatter the plane's element matrices into rows whose second index lies in
 * this thread's range [lo, hi) of i2 (element order e2, e1 ascending) */
static void* scatter_job(void* arg) {
    elem_job* j = (elem_job*)arg;
    elem_ctx* c = j->c;
    const int n = c->n, m = c->m, p = c->p, P1 = c->P1, nloc = c->nloc, d = c->d, off = c->off, e3 = c->e3;
    const int lo = (int)((int64_t)m * j->t / c->nthreads), hi = (int)((int64_t)m * (j->t + 1) / c->nthreads);
    const int64_t kes = (int64_t)nloc * (nloc + 1) / 2;
    int e2a = lo + off - p, e2b = hi - 1 + off;
    if (e2a < 0) e2a = 0;
    if (e2b > n - 1) e2b = n - 1;
    for (int e2 = e2a; e2 <= e2b; e2++)
        for (int e1 = 0; e1 < n; e1++) {
            const int el = e2 * n + e1;
            const double* ke = c->ke + el * kes;
            const double* fe = c->fe + (int64_t)el * nloc;
            for (int a = 0; a < nloc; a++) {
                const int a1 = a % P1, a2 = (a / P1) % P1, a3 = (d == 3) ? a / (P1 * P1) : 0;
                const int i1 = e1 + a1 - off, i2 = e2 + a2 - off, i3 = (d == 3) ? e3 + a3 - off : 0;
                if (i2 < lo || i2 >= hi) continue;
                if (i1 < 0 || i1 >= m || i2 < 0 || i3 < 0 || i3 >= m) continue;
                const int64_t I = i1 + (int64_t)m * (i2 + (int64_t)m * i3);
                if (c->F) c->F[I] += fe[a];
                for (int b = 0; b < nloc; b++) {
                    const int b1 = b % P1, b2 = (b / P1) % P1, b3 = (d == 3) ? b / (P1 * P1) : 0;
                    const int j1 = e1 + b1 - off, j2 = e2 + b2 - off, j3 = (d == 3) ? e3 + b3 - off : 0;
                    if (j1 < 0 || j1 >= m || j2 < 0 || j2 >= m || j3 < 0 || j3 >= m) continue;
                    const int64_t Jg = j1 + (int64_t)m * (j2 + (int64_t)m * j3);
                    if (Jg < I) continue;
                    const int lo_ab = a <= b ? a : b, hi_ab = a <= b ? b : a;
                    const double kab = ke[(int64_t)lo_ab * nloc - (int64_t)lo_ab * (lo_ab - 1) / 2 + (hi_ab - lo_ab)];
                    c->val[c->rowptr[I] + pat_pos(d, m, p, i1, i2, i3, j1, j2, j3)] += kab;
                }
            }
        }
    return NULL;
}

/* lower triangle := mirror of the upper one, rows [N t / T, N (t+1) / T) */
static void* mirror_job(void* arg) {
    elem_job* j = (elem_job*)arg;
    elem_ctx* c = j->c;
    const int d = c->d, m = c->m, p = c->p;
    const int64_t N = (d == 2) ? (int64_t)m * m : (int64_t)m * m * m;
    const int64_t I0 = N * j->t / c->nthreads, I1 = N * (j->t + 1) / c->nthreads;
    for (int64_t I = I0; I < I1; I++) {
        int i1 = (int)(I % m), i2 = (int)((I / m) % m), i3 = (d == 3) ? (int)(I / ((int64_t)m * m)) : 0;
        for (int64_t k = c->rowptr[I]; k < c->rowptr[I + 1]; k++) {
            int64_t Jg = c->col[k];
            if (Jg >= I) continue;
            int j1 = (int)(Jg % m), j2 = (int)((Jg / m) % m), j3 = (d == 3) ? (int)(Jg / ((int64_t)m * m)) : 0;
            c->val[k] = c->val[c->rowptr[Jg] + pat_pos(d, m, p, j1, j2, j3, i1, i2, i3)];
        }
    }
    return NULL;
}

/* kappa at every quadrature point: [iz][ip2], iz = e3 nq + q3 (one z point
 * in 2-D), ip2 = (e2 nq + q2) (n nq) + e1 nq + q1. */
typedef struct {
    const kappa_field* kf;
    int d, n, nq, geom, nthreads, t;
    const double *gx, *zc, *zs;  /* cos / sin of w_m3 z for every z point: [iz][M] */
    double* out;
} kappa_job;

static void* kappa_worker(void* arg) {
    kappa_job* j = (kappa_job*)arg;
    const kappa_field* kf = j->kf;
    const int M = kf->M, n = j->n, nq = j->nq, nqn = n * nq, nz = (j->d == 3) ? nqn : 1;
    const double h = 1.0 / n, amp = kf->sigma * sqrt(2.0 / M);
    double* ac = (double*)malloc(sizeof(double) * M);
    double* as = (double*)malloc(sizeof(double) * M);
    for (int64_t ip2 = j->t; ip2 < (int64_t)nqn * nqn; ip2 += j->nthreads) {
        const int i1 = (int)(ip2 % nqn), i2 = (int)(ip2 / nqn);
        const double xi[3] = {((i1 / nq) + 0.5 * (j->gx[i1 % nq] + 1.0)) * h,
                              ((i2 / nq) + 0.5 * (j->gx[i2 % nq] + 1.0)) * h, 0.0};
        double x[3] = {0, 0, 0}, J[3][3];
        geom_eval(j->geom, j->d, xi, x, J);
        for (int m = 0; m < M; m++) {
            const double a = kf->phi[m] + kf->omega[3 * m] * x[0] + kf->omega[3 * m + 1] * x[1];
            ac[m] = cos(a);
            as[m] = sin(a);
        }
        for (int iz = 0; iz < nz; iz++) {
            const double* zc = j->zc + (int64_t)iz * M;
            const double* zs = j->zs + (int64_t)iz * M;
            double g = 0.0;
            for (int m = 0; m < M; m++) g += ac[m] * zc[m] - as[m] * zs[m];
            j->out[(int64_t)iz * nqn * nqn + ip2] = exp(amp * g);
        }
    }
    free(ac);
    free(as);
    return NULL;
}

static double* kappa_table(const kappa_field* kf, int d, int n, int nq, int geom, const double* gx, int nthreads) {
    const int M = kf->M, nqn = n * nq, nz = (d == 3) ? nqn : 1;
    double* out = (double*)malloc(sizeof(double) * (size_t)nz * nqn * nqn);
    double* zc = (double*)malloc(sizeof(double) * (size_t)nz * M);
    double* zs = (double*)malloc(sizeof(double) * (size_t)nz * M);
    if (!out || !zc || !zs) {
        free(out); free(zc); free(zs);
        return NULL;
    }
    for (int iz = 0; iz < nz; iz++) {
        const double z = (d == 3) ? ((iz / nq) + 0.5 * (gx[iz % nq] + 1.0)) / n : 0.0;
        for (int m = 0; m < M; m++) {
            const double b = kf->omega[3 * m + 2] * z;
            zc[(int64_t)iz * M + m] = cos(b);
            zs[(int64_t)iz * M + m] = sin(b);
        }
    }
    pthread_t th[32];
    kappa_job jobs[32];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = (kappa_job){kf, d, n, nq, geom, nthreads, t, gx, zc, zs, out};
        if (t > 0 && pthread_create(&th[t], NULL, kappa_worker, &jobs[t]) != 0) {
            kappa_worker(&jobs[t]);
            jobs[t].t = -1;
        }
    }
    kappa_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++)
        if (jobs[t].t >= 0) pthread_join(th[t], NULL);
    free(zc);
    free(zs);
    return out;
}

int iga_assemble_elem(int d, int n, int p, int nq, int geom, int with_boundary, int kappa_M, double kappa_ell,
                      double kappa_sigma, uint64_t kappa_seed, int fkind, int64_t* rowptr, int32_t* col, double* val,
                      double* F) {
    if ((d != 2 && d != 3) || p < 1 || p > IGA_MAXP || nq < 1 || nq > IGA_MAXQ) return -1;
    if (geom == 1 && d != 3) return -1;
    const int nb = n + p, off = with_boundary ? 0 : 1, m = with_boundary ? nb : nb - 2;
    const int P1 = p + 1;
    const int nloc = (d == 2) ? P1 * P1 : P1 * P1 * P1;
    if (nloc > 729) return -1;
    build_pattern(d, m, p, rowptr, col);
    const int64_t N = (d == 2) ? (int64_t)m * m : (int64_t)m * m * m;
    memset(val, 0, sizeof(double) * rowptr[N]);
    if (F) memset(F, 0, sizeof(double) * N);

    elem_ctx c;
    memset(&c, 0, sizeof(c));
    c.d = d; c.n = n; c.p = p; c.nq = nq; c.geom = geom; c.off = off; c.m = m; c.P1 = P1; c.nloc = nloc;
    c.nqe = (d == 2) ? nq * nq : nq * nq * nq;
    c.fkind = fkind;
    c.h = 1.0 / n;
    c.rowptr = rowptr; c.val = val; c.F = F;
    c.nthreads = num_threads();

    double gx[IGA_MAXQ], gw[IGA_MAXQ];
    iga_gauss_legendre(nq, gx, gw);
    c.gx = gx; c.gw = gw;
    double* V = (double*)malloc(sizeof(double) * n * nq * P1);
    double* D = (double*)malloc(sizeof(double) * n * nq * P1);
    for (int e = 0; e < n; e++)
        for (int q = 0; q < nq; q++)
            iga_bspline_local(n, p, e, (e + 0.5 * (gx[q] + 1.0)) * c.h, V + (e * nq + q) * P1, D + (e * nq + q) * P1);
    c.V = V; c.D = D;

    kappa_field kf;
    kappa_init(&kf, kappa_M, kappa_ell, kappa_sigma, kappa_seed);
    double* kap = NULL;
    if (kf.M > 0) {
        kap = kappa_table(&kf, d, n, nq, geom, gx, c.nthreads);
        if (!kap) { free(V); free(D); kappa_free(&kf); return -2; }
    }
    c.kap = kap;

    const int nel = n * n; /* elements of a plane (of the whole square in 2-D) */
    const int64_t kes = (int64_t)nloc * (nloc + 1) / 2;
    c.ke = (double*)malloc(sizeof(double) * (size_t)nel * kes);
    c.fe = (double*)malloc(sizeof(double) * (size_t)nel * nloc);
    if (!c.ke || !c.fe) {
        free(c.ke); free(c.fe); free(V); free(D); free(kap); kappa_free(&kf);
        return -2;
    }
    const int ne3 = (d == 3) ? n : 1;
    for (int e3 = 0; e3 < ne3; e3++) {
        c.e3 = e3;
        run_parallel(compute_job, &c);
        run_parallel(scatter_job, &c);
    }
    /* mirror the upper triangle (rows in parallel; reads only upper entries) */
    c.col = col;
    run_parallel(mirror_job, &c);
    free(c.ke); free(c.fe); free(V); free(D); free(kap);
    kappa_free(&kf);
    return 0;
}

/* ----------------------------------------------------- post-processing ---- */
/* L2 error || u - u_h ||_{L2(0,1)^d} for u = prod sin(pi x_k), u_h the
 * B-spline field with interior coefficients `coef` (zero on the eliminated
 * boundary functions), by an nq-point rule per element and direction. */
double iga_l2_error_sine(int d, int n, int p, int nq, const double* coef) {
    const double pi = 3.14159265358979323846264338328;
    const int nb = n + p, m = nb - 2, P1 = p + 1;
    double gx[IGA_MAXQ], gw[IGA_MAXQ];
    iga_gauss_legendre(nq, gx, gw);
    const double h = 1.0 / n;
    double err2 = 0.0;
    const int ne3 = (d == 3) ? n : 1, nq3 = (d == 3) ? nq : 1;
    for (int e3 = 0; e3 < ne3; e3++)
        for (int e2 = 0; e2 < n; e2++)
            for (int e1 = 0; e1 < n; e1++)
                for (int q3 = 0; q3 < nq3; q3++)
                    for (int q2 = 0; q2 < nq; q2++)
                        for (int q1 = 0; q1 < nq; q1++) {
                            double xi[3] = {(e1 + 0.5 * (gx[q1] + 1.0)) * h, (e2 + 0.5 * (gx[q2] + 1.0)) * h,
                                            (d == 3) ? (e3 + 0.5 * (gx[q3] + 1.0)) * h : 0.0};
                            double w = (0.5 * h * gw[q1]) * (0.5 * h * gw[q2]);
                            if (d == 3) w *= 0.5 * h * gw[q3];
                            double v1[IGA_MAXP + 1], v2[IGA_MAXP + 1], v3[IGA_MAXP + 1], dd[IGA_MAXP + 1];
                            iga_bspline_local(n, p, e1, xi[0], v1, dd);
                            iga_bspline_local(n, p, e2, xi[1], v2, dd);
                            if (d == 3) iga_bspline_local(n, p, e3, xi[2], v3, dd);
                            else v3[0] = 1.0;
                            double uh = 0.0;
                            for (int a3 = 0; a3 < ((d == 3) ? P1 : 1); a3++)
                                for (int a2 = 0; a2 < P1; a2++)
                                    for (int a1 = 0; a1 < P1; a1++) {
                                        int i1 = e1 + a1 - 1, i2 = e2 + a2 - 1, i3 = (d == 3) ? e3 + a3 - 1 : 0;
                                        if (i1 < 0 || i1 >= m || i2 < 0 || i2 >= m || i3 < 0 || i3 >= m) continue;
                                        int64_t I = i1 + (int64_t)m * (i2 + (int64_t)m * i3);
                                        uh += coef[I] * v1[a1] * v2[a2] * v3[a3];
                                    }
                            double u = sin(pi * xi[0]) * sin(pi * xi[1]);
                            if (d == 3) u *= sin(pi * xi[2]);
                            err2 += (u - uh) * (u - uh) * w;
                        }
    return sqrt(err2);
}

/* y = K x in CSR, rows summed left to right in column order (input recipe
 * F = K u_true for the random-solution workloads). */
void iga_csr_apply(int64_t N, const int64_t* rowptr, const int32_t* col, const double* val, const double* x, double* y) {
    for (int64_t i = 0; i < N; i++) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) s += val[k] * x[col[k]];
        y[i] = s;
    }
}
