// IgA assembly on the GPU by sum factorization (arXiv 2511.21268, Sec. 2.2).
//
// Stiffness entries of -div(kappa grad u) = f on one tensor-product B-spline
// patch, pulled back to the parametric cube and summed over the Gauss
// points q = (q1, q2, q3) of all elements:
//   k_ij = sum_q sum_{a,b} C_ab(q) d_a N_i(q) d_b N_j(q),
//   C = kappa(F(xi_q)) w_q |det J| J^-1 J^-T,        f_i = sum_q f w_q |det J| N_i(q),
// with N_i = b_i1(xi1) b_i2(xi2) b_i3(xi3) and d_a the parametric derivative
// in direction a.  Each term (a, b) factors into 1-D pair weights
//   W^{xy}_{i, delta}(q) = b^x_i(q) b^y_{i+delta}(q),   x, y in {value, derivative},
// one per direction, so the 3-D sum is contracted one direction at a time
// (sum factorization, the tensor-product alternative to the element loop
// that Sec. 2.2 points to):
//   A(r3, q2, q1) = sum_q3 W3(r3, q3) C(q3, q2, q1)
//   B(r3, r2, q1) = sum_q2 W2(r2, q2) A(r3, q2, q1)
//   K(r3, r2, r1) = sum_q1 W1(r1, q1) B(r3, r2, q1)
// with r_k = (i_k, delta_k) the 1-D pairs of the band |i_k - j_k| <= p.  The
// weight of a pair is nonzero on the Gauss points of the elements where both
// functions live, (p + 1 - |delta|) nq consecutive points, stored from the
// first of them.
//
// The geometries are extruded in xi3 (F_3 = xi3, F_1 and F_2 independent of
// xi3): J = [J2 0; 0 1], so C_02 = C_12 = 0 and C_22 = kappa w |det J2|.
// The five terms (0,0), (0,1), (1,0), (1,1), (2,2) have 1-D weight types
//   direction 3: vv vv vv vv dd;  direction 2: vv vd dv dd vv;
//   direction 1: dd dv vd vv vv,
// so after direction 3 there are four distinct arrays (C00, C01, C11 with
// vv; C22 with dd) and after direction 2 four groups by direction-1 type.
//
// kappa = exp(g), g = sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m) with
// x = (x(xi1, xi2), y(xi1, xi2), z(xi3)): cos(a + b) = cos a cos b - sin a sin b
// separates the plane and z parts, so g at all Q^3 points is the product of
// a Q^2 x 2M matrix [cos a, -sin a] and a 2M x Q matrix [cos b; sin b] -- an
// FP64 GEMM (register-tiled, below) whose epilogue forms the coefficients.
//
// Everything is FP64.  The sums run in a different order than an element
// loop's, so results agree with one to rounding, not bit for bit.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "amg_gb300.h"
#include "amg_internal.cuh"

namespace amg {
namespace {

constexpr int kMaxDeg = 8;       // largest degree p
constexpr int kMaxNq = 16;       // most Gauss points per element and direction
constexpr int kMaxQ = 768;       // most Gauss points per direction (n nq): the contraction's staging
constexpr int kCtIn = 32;        // inner positions per block of the contractions
constexpr int kCtWarps = 8;      // warps per block of the contractions
constexpr int kInRows = 8;       // rows per block of the last contraction
constexpr int kGT = 64;          // GEMM tile (plane points x z points)
constexpr int kGK = 16;          // GEMM depth per stage

struct IgaDims {
    int n, p, nq, m, off, Q, B, R, Lmax, R1, L1max;
};

__host__ __device__ inline double knot(int n, int p, int i) {
    return i <= p ? 0.0 : (i >= n + p ? 1.0 : (double)(i - p) / (double)n);
}

// Gauss-Legendre nodes and weights on [-1, 1], ascending: Newton's method on
// P_nq (three-term recurrence) from the starting guess cos(pi (k+3/4)/(nq+1/2)),
// w = 2 / ((1 - t^2) P_nq'(t)^2).
__global__ void k_iga_gauss(int nq, double* gx, double* gw) {
    const int k = threadIdx.x;
    if (k >= nq) return;
    const double pi = 3.14159265358979323846;
    double t = cos(pi * (k + 0.75) / (nq + 0.5)), pn = 0.0, dp = 1.0;
    for (int it = 0; it < 100; it++) {
        double p0 = 1.0, p1 = t;
        for (int j = 2; j <= nq; j++) {
            const double p2 = ((2 * j - 1) * t * p1 - (j - 1) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        pn = nq == 1 ? t : p1;
        const double pm = nq == 1 ? 1.0 : p0;
        dp = nq * (t * pn - pm) / (t * t - 1.0);
        const double dt = pn / dp;
        t -= dt;
        if (fabs(dt) < 1e-16) break;
    }
    {
        double p0 = 1.0, p1 = t;
        for (int j = 2; j <= nq; j++) {
            const double p2 = ((2 * j - 1) * t * p1 - (j - 1) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        pn = nq == 1 ? t : p1;
        dp = nq == 1 ? 1.0 : nq * (t * pn - p0) / (t * t - 1.0);
    }
    gx[nq - 1 - k] = t;
    gw[nq - 1 - k] = 2.0 / ((1.0 - t * t) * dp * dp);
}

// Values V[q][a] and derivatives D[q][a] of the p+1 B-splines e..e+p that
// live on element e = q / nq, at its Gauss point q % nq: the span recursion
// for the nonzero functions of a knot span (degree 0 -> p, each step mixing
// neighbours with the weights (xi - u_i) / (u_{i+k} - u_i)), and
// N'_{i,p} = p (N_{i,p-1} / (u_{i+p} - u_i) - N_{i+1,p-1} / (u_{i+p+1} - u_{i+1})).
__global__ void k_iga_basis(int n, int p, int nq, const double* __restrict__ gx, double* V, double* D) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * nq) return;
    const int e = q / nq, s = e + p;
    const double xi = (e + 0.5 * (gx[q % nq] + 1.0)) / n;
    double N[kMaxDeg + 1], Np[kMaxDeg + 1], left[kMaxDeg + 1], right[kMaxDeg + 1];
    N[0] = 1.0;
    Np[0] = 1.0;
    for (int k = 1; k <= p; k++) {
        if (k == p)
            for (int a = 0; a < p; a++) Np[a] = N[a];
        left[k] = xi - knot(n, p, s + 1 - k);
        right[k] = knot(n, p, s + k) - xi;
        double saved = 0.0;
        for (int r = 0; r < k; r++) {
            const double tmp = N[r] / (right[r + 1] + left[k - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[k - r] * tmp;
        }
        N[k] = saved;
    }
    const int P1 = p + 1;
    for (int a = 0; a <= p; a++) {
        const int i = e + a;
        double d = 0.0;
        if (a >= 1) d += Np[a - 1] / (knot(n, p, i + p) - knot(n, p, i));
        if (a <= p - 1) d -= Np[a] / (knot(n, p, i + p + 1) - knot(n, p, i + 1));
        V[(int64_t)q * P1 + a] = N[a];
        D[(int64_t)q * P1 + a] = p * d;
    }
}

// 1-D pair tables: r = i B + (delta + p), j = i + delta (kept functions,
// global index g = i + off).  s[r], L[r]: first Gauss point and count of the
// elements where both live (L = 0 when j is not kept); W_xy[r][k] the
// products of value/derivative at point s[r] + k.
__global__ void k_iga_pairs(IgaDims d, const double* __restrict__ V, const double* __restrict__ D, int* s, int* L,
                            double* Wvv, double* Wvd, double* Wdv, double* Wdd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)d.R * d.Lmax) return;
    const int r = (int)(idx / d.Lmax), k = (int)(idx % d.Lmax);
    const int i = r / d.B, delta = r % d.B - d.p, j = i + delta;
    const int gi = i + d.off, gj = j + d.off;
    const int e0 = max(max(gi, gj) - d.p, 0), e1 = min(min(gi, gj), d.n - 1);
    const bool ok = j >= 0 && j < d.m && e0 <= e1;
    const int len = ok ? (e1 - e0 + 1) * d.nq : 0;
    if (k == 0) {
        s[r] = ok ? e0 * d.nq : 0;
        L[r] = len;
    }
    double vv = 0.0, vd = 0.0, dv = 0.0, dd = 0.0;
    if (k < len) {
        const int q = e0 * d.nq + k, e = q / d.nq, P1 = d.p + 1;
        const double vi = V[(int64_t)q * P1 + gi - e], di = D[(int64_t)q * P1 + gi - e];
        const double vj = V[(int64_t)q * P1 + gj - e], dj = D[(int64_t)q * P1 + gj - e];
        vv = vi * vj;
        vd = vi * dj;
        dv = di * vj;
        dd = di * dj;
    }
    Wvv[idx] = vv;
    Wvd[idx] = vd;
    Wdv[idx] = dv;
    Wdd[idx] = dd;
}

// Single-function table of the load vector: r = i, the Gauss points of the
// elements where function g = i + off lives, W1[i][k] its values there.
__global__ void k_iga_single(IgaDims d, const double* __restrict__ V, int* s, int* L, double* W) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)d.R1 * d.L1max) return;
    const int i = (int)(idx / d.L1max), k = (int)(idx % d.L1max);
    const int g = i + d.off, e0 = max(g - d.p, 0), e1 = min(g, d.n - 1);
    const int len = (e1 - e0 + 1) * d.nq;
    if (k == 0) {
        s[i] = e0 * d.nq;
        L[i] = len;
    }
    double v = 0.0;
    if (k < len) {
        const int q = e0 * d.nq + k, e = q / d.nq;
        v = V[(int64_t)q * (d.p + 1) + g - e];
    }
    W[idx] = v;
}

// Plane data per point (q2, q1) of the (xi1, xi2) plane, p2 = q2 Q + q1:
// x, y, the 2x2 block G = J2^-1 J2^-T (g00, g01, g11) and |det J2| w1 w2 (h/2)^2.
// geometry 0: identity; 1: quarter annulus, (1 + xi1) c(xi2) with c the
// quadratic NURBS arc through (1,0), (1,1), (0,1), weights 1, sqrt(1/2), 1.
__global__ void k_iga_plane(int geometry, int n, int nq, const double* __restrict__ gx,
                            const double* __restrict__ gw, double* plane) {
    const int Q = n * nq;
    const int64_t p2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p2 >= (int64_t)Q * Q) return;
    const int q1 = (int)(p2 % Q), q2 = (int)(p2 / Q);
    const double h = 1.0 / n;
    const double xi1 = (q1 / nq + 0.5 * (gx[q1 % nq] + 1.0)) * h;
    const double xi2 = (q2 / nq + 0.5 * (gx[q2 % nq] + 1.0)) * h;
    const double w = (0.5 * h * gw[q1 % nq]) * (0.5 * h * gw[q2 % nq]);
    double x, y, j00, j01, j10, j11;
    if (geometry == AMG_GEOM_ANNULUS) {
        const double t = xi2, wm = 0.70710678118654752440;
        const double b0 = (1 - t) * (1 - t), b1 = 2 * t * (1 - t), b2 = t * t;
        const double d0 = -2 * (1 - t), d1 = 2 - 4 * t, d2 = 2 * t;
        const double W = b0 + wm * b1 + b2, dW = d0 + wm * d1 + d2;
        const double ax = b0 + wm * b1, ay = wm * b1 + b2;
        const double dax = d0 + wm * d1, day = wm * d1 + d2;
        const double cx = ax / W, cy = ay / W;
        const double dcx = (dax * W - ax * dW) / (W * W), dcy = (day * W - ay * dW) / (W * W);
        const double r = 1.0 + xi1;
        x = r * cx;
        y = r * cy;
        j00 = cx;
        j01 = r * dcx;
        j10 = cy;
        j11 = r * dcy;
    } else {
        x = xi1;
        y = xi2;
        j00 = 1.0;
        j01 = 0.0;
        j10 = 0.0;
        j11 = 1.0;
    }
    const double det = j00 * j11 - j01 * j10;
    // J2^-1 = [j11 -j01; -j10 j00] / det; G = J2^-1 J2^-T (rows of J2^-1 dotted)
    const double a = j11 / det, b = -j01 / det, c = -j10 / det, dd = j00 / det;
    double* o = plane + p2 * 6;
    o[0] = x;
    o[1] = y;
    o[2] = a * a + b * b;
    o[3] = a * c + b * dd;
    o[4] = c * c + dd * dd;
    o[5] = fabs(det) * w;
}

// z and w3 (h/2) per z point.
__global__ void k_iga_zline(int n, int nq, const double* __restrict__ gx, const double* __restrict__ gw,
                            double* zl) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * nq) return;
    const double h = 1.0 / n;
    zl[2 * q] = (q / nq + 0.5 * (gx[q % nq] + 1.0)) * h;
    zl[2 * q + 1] = 0.5 * h * gw[q % nq];
}

// GEMM operands of kappa: Ak[p2][k] = cos(a_m) (k = m < M), -sin(a_m)
// (k = M + m), zero padding up to K2; Bk[k][q3] = cos(b_m), sin(b_m).
// a_m = omega_m,x x + omega_m,y y + phi_m, b_m = omega_m,z z.
__global__ void k_iga_kappa_plane(int64_t P2, int M, int K2, const double* __restrict__ plane,
                                  const double* __restrict__ om, const double* __restrict__ ph, double* Ak) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P2 * K2) return;
    const int64_t p2 = idx / K2;
    const int k = (int)(idx % K2);
    double v = 0.0;
    if (k < 2 * M) {
        const int mm = k % M;
        const double a = om[3 * mm] * plane[p2 * 6] + om[3 * mm + 1] * plane[p2 * 6 + 1] + ph[mm];
        v = k < M ? cos(a) : -sin(a);
    }
    Ak[idx] = v;
}

__global__ void k_iga_kappa_z(int Q, int M, int K2, const double* __restrict__ zl, const double* __restrict__ om,
                              double* Bk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K2 * Q) return;
    const int k = idx / Q, q3 = idx % Q;
    double v = 0.0;
    if (k < 2 * M) {
        const int mm = k % M;
        const double b = om[3 * mm + 2] * zl[2 * q3];
        v = k < M ? cos(b) : sin(b);
    }
    Bk[idx] = v;
}

struct CoefOut {
    double *c00, *c01, *c11, *c22, *e;
};

// Coefficients at point (q3, p2) from g (kappa = exp(amp g); amp = 0: kappa = 1).
__device__ __forceinline__ void coef_store(const CoefOut& o, int64_t P2, int64_t p2, int q3, double g, double amp,
                                           const double* __restrict__ plane, const double* __restrict__ zl,
                                           int source) {
    const double* pl = plane + p2 * 6;
    const double dw = pl[5] * zl[2 * q3 + 1];
    const double cw = (amp != 0.0 ? exp(amp * g) : 1.0) * dw;
    const int64_t at = (int64_t)q3 * P2 + p2;
    o.c00[at] = cw * pl[2];
    if (o.c01) o.c01[at] = cw * pl[3];
    o.c11[at] = cw * pl[4];
    o.c22[at] = cw;
    if (o.e) {
        double f = 1.0;
        if (source == AMG_SRC_SINE) {
            const double pi = 3.14159265358979323846;
            f = 3.0 * pi * pi * sin(pi * pl[0]) * sin(pi * pl[1]) * sin(pi * zl[2 * q3]);
        }
        o.e[at] = f * dw;
    }
}

// Coefficients without kappa (thread per point).
__global__ void k_iga_coef_const(int64_t P2, int Q, const double* __restrict__ plane, const double* __restrict__ zl,
                                 int source, CoefOut o) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P2 * Q) return;
    coef_store(o, P2, idx % P2, (int)(idx / P2), 0.0, 0.0, plane, zl, source);
}

// g[q3][p2] = sum_k Ak[p2][k] Bk[k][q3] on 64 x 64 tiles (256 threads, 4 x 4
// accumulators each: rows tx + 16 a, columns ty + 16 b), then the
// coefficients.  K2 is a multiple of kGK.
__global__ void __launch_bounds__(256) k_iga_coef_gemm(int64_t P2, int Q, int K2, const double* __restrict__ Ak,
                                                      const double* __restrict__ Bk, double amp,
                                                      const double* __restrict__ plane,
                                                      const double* __restrict__ zl, int source, CoefOut o) {
    __shared__ double As[kGK][kGT + 1];
    __shared__ double Bs[kGK][kGT];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t r0 = (int64_t)blockIdx.x * kGT;
    const int c0 = blockIdx.y * kGT;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < K2; k0 += kGK) {
#pragma unroll
        for (int u = 0; u < (kGT * kGK) / 256; u++) {
            const int e = tid + 256 * u;
            const int row = e / kGK, kk = e % kGK;
            As[kk][row] = r0 + row < P2 ? Ak[(r0 + row) * K2 + k0 + kk] : 0.0;
            const int kb = e / kGT, col = e % kGT;
            Bs[kb][col] = c0 + col < Q ? Bk[(int64_t)(k0 + kb) * Q + c0 + col] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                a[u] = As[kk][tx + 16 * u];
                b[u] = Bs[kk][ty + 16 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++)
#pragma unroll
                for (int v = 0; v < 4; v++) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const int64_t p2 = r0 + tx + 16 * u;
            const int q3 = c0 + ty + 16 * v;
            if (p2 < P2 && q3 < Q) coef_store(o, P2, p2, q3, acc[u][v], amp, plane, zl, source);
        }
}

// Contraction of the middle (outer-major) axis: Y[o][r][c] (+)= sum_{k < L[r]}
// W[r][k] X[o][s[r] + k][c], c < IN, r < R.  Block (tile of 32 c, o): X's
// Q x 32 slab in shared memory, warps over r, lanes over c.
__global__ void __launch_bounds__(32 * kCtWarps) k_iga_outer(int64_t IN, int Q, int R, const double* __restrict__ X,
                                                             const int* __restrict__ s, const int* __restrict__ L,
                                                             const double* __restrict__ W, int Lmax, double* Y,
                                                             int accumulate) {
    extern __shared__ double xs[];  // [Q][kCtIn]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int64_t c0 = (int64_t)blockIdx.x * kCtIn;
    const int64_t o = blockIdx.y;
    const double* Xo = X + o * Q * IN;
    for (int q = ty; q < Q; q += kCtWarps) xs[q * kCtIn + tx] = c0 + tx < IN ? Xo[(int64_t)q * IN + c0 + tx] : 0.0;
    __syncthreads();
    if (c0 + tx >= IN) return;
    double* Yo = Y + o * R * IN + c0 + tx;
    for (int r = ty; r < R; r += kCtWarps) {
        const int st = s[r], len = L[r];
        const double* w = W + (int64_t)r * Lmax;
        double acc = 0.0;
        for (int k = 0; k < len; k++) acc = fma(w[k], xs[(st + k) * kCtIn + tx], acc);
        double* y = Yo + (int64_t)r * IN;
        *y = accumulate ? *y + acc : acc;
    }
}

// Last contraction (the innermost axis, q1) and the CSR scatter: rows
// o = r3 R + r2 of the ng direction-1 groups X_g[o][q1];
// K(I, J) = sum_g sum_k W_g[r1][k] X_g[o][s[r1] + k] goes to the position of
// J in row I (columns in (delta3, delta2, delta1) order).  A block stages
// `rows` consecutive rows of every group in shared memory (row stride Q + 1);
// thread t takes row t % rows and every (256 / rows)-th pair from t / rows on,
// so the lanes that share a pair read the same weights (a broadcast) and rows
// a padded stride apart.
struct InnerGroups {
    const double* X[4];
    const double* W[4];
    int ng;
};

__device__ __forceinline__ void band_range(int i, int m, int p, int& lo, int& nv) {
    lo = max(-p, -i);
    nv = min(p, m - 1 - i) - lo + 1;
}

constexpr int kInThreads = 256;

template <int NG>
__global__ void __launch_bounds__(kInThreads) k_iga_inner_csr(IgaDims d, InnerGroups G, int rows,
                                                              const int* __restrict__ s, const int* __restrict__ L,
                                                              const int64_t* __restrict__ rowptr, double* val) {
    extern __shared__ double xs[];  // [NG][rows][Q + 1]
    const int64_t O = (int64_t)d.R * d.R;
    const int64_t o0 = (int64_t)blockIdx.x * rows;
    const int Qp = d.Q + 1;
#pragma unroll
    for (int g = 0; g < NG; g++)
        for (int t = threadIdx.x; t < rows * d.Q; t += blockDim.x) {
            const int row = t / d.Q, q = t % d.Q;
            xs[((int64_t)g * rows + row) * Qp + q] = o0 + row < O ? G.X[g][(o0 + row) * d.Q + q] : 0.0;
        }
    __syncthreads();
    const int row = threadIdx.x % rows, slot = threadIdx.x / rows, nslot = kInThreads / rows;
    const int64_t o = o0 + row;
    if (o >= O) return;
    const int r3 = (int)(o / d.R), r2 = (int)(o % d.R);
    const int i3 = r3 / d.B, d3 = r3 % d.B - d.p, i2 = r2 / d.B, d2 = r2 % d.B - d.p;
    const int j3 = i3 + d3, j2 = i2 + d2;
    if (j3 < 0 || j3 >= d.m || j2 < 0 || j2 >= d.m) return;
    int lo3, nv3, lo2, nv2;
    band_range(i3, d.m, d.p, lo3, nv3);
    band_range(i2, d.m, d.p, lo2, nv2);
    const double* xr = xs + (int64_t)row * Qp;
    // pairs in delta-major order: the pairs a warp shares have the same
    // delta, hence the same number of common Gauss points (no divergence)
    for (int u = slot; u < d.R; u += nslot) {
        const int r1 = (u % d.m) * d.B + u / d.m;
        const int i1 = r1 / d.B, d1 = r1 % d.B - d.p, j1 = i1 + d1;
        if (j1 < 0 || j1 >= d.m) continue;
        const int st = s[r1], len = L[r1];
        double acc = 0.0;
#pragma unroll
        for (int g = 0; g < NG; g++) {
            const double* x = xr + (int64_t)g * rows * Qp + st;
            const double* wt = G.W[g] + (int64_t)r1 * d.Lmax;
            for (int k = 0; k < len; k++) acc = fma(__ldg(wt + k), x[k], acc);
        }
        int lo1, nv1;
        band_range(i1, d.m, d.p, lo1, nv1);
        const int64_t I = i1 + (int64_t)d.m * (i2 + (int64_t)d.m * i3);
        val[rowptr[I] + ((int64_t)(d3 - lo3) * nv2 + (d2 - lo2)) * nv1 + (d1 - lo1)] = acc;
    }
}

// Load vector's last contraction: F[o m + i1] = sum_k W1[i1][k] X[o][s1[i1] + k].
__global__ void __launch_bounds__(32 * kInRows) k_iga_inner_dense(IgaDims d, const double* __restrict__ X,
                                                                  const int* __restrict__ s,
                                                                  const int* __restrict__ L,
                                                                  const double* __restrict__ W, double* F) {
    extern __shared__ double xs[];  // [kInRows][Q + 1]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t O = (int64_t)d.m * d.m;
    const int64_t o0 = (int64_t)blockIdx.x * kInRows;
    const int Qp = d.Q + 1;
    for (int t = threadIdx.x; t < kInRows * d.Q; t += blockDim.x) {
        const int row = t / d.Q, q = t % d.Q;
        xs[(int64_t)row * Qp + q] = o0 + row < O ? X[(o0 + row) * d.Q + q] : 0.0;
    }
    __syncthreads();
    const int64_t o = o0 + w;
    if (o >= O) return;
    for (int i1 = lane; i1 < d.m; i1 += 32) {
        const int st = s[i1], len = L[i1];
        const double* x = xs + (int64_t)w * Qp + st;
        const double* wt = W + (int64_t)i1 * d.L1max;
        double acc = 0.0;
        for (int k = 0; k < len; k++) acc = fma(wt[k], x[k], acc);
        F[o * d.m + i1] = acc;
    }
}

// sum_{x < i} nv(x), nv(x) = min(p, m-1-x) - max(-p, -x) + 1 (band count of
// index x), in closed form: i + f(i) + f(m) - f(m - i), f(i) = sum_{x<i} min(p, x).
__host__ __device__ inline int64_t band_prefix(int64_t i, int64_t m, int64_t p) {
    auto f = [p](int64_t k) -> int64_t { return k <= p ? k * (k - 1) / 2 : p * (p + 1) / 2 + p * (k - p - 1); };
    return i + f(i) + f(m) - f(m - i);
}

// CSR pattern (warp per row): rowptr in closed form, columns in ascending
// order (delta3, delta2, delta1); rowptr[N] by the last row's warp.
__global__ void k_iga_pattern(int m, int p, int64_t* rowptr, int32_t* col) {
    const int lane = threadIdx.x & 31;
    const int64_t N = (int64_t)m * m * m;
    const int64_t T = band_prefix(m, m, p);
    for (int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < N;
         I += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int i1 = (int)(I % m), i2 = (int)((I / m) % m), i3 = (int)(I / ((int64_t)m * m));
        int lo1, nv1, lo2, nv2, lo3, nv3;
        band_range(i1, m, p, lo1, nv1);
        band_range(i2, m, p, lo2, nv2);
        band_range(i3, m, p, lo3, nv3);
        const int64_t base = band_prefix(i3, m, p) * T * T +
                             (int64_t)nv3 * (band_prefix(i2, m, p) * T + (int64_t)nv2 * band_prefix(i1, m, p));
        if (lane == 0) {
            rowptr[I] = base;
            if (I == N - 1) rowptr[N] = T * T * T;
        }
        const int cnt = nv1 * nv2 * nv3;
        for (int t = lane; t < cnt; t += 32) {
            const int c1 = t % nv1, c2 = (t / nv1) % nv2, c3 = t / (nv1 * nv2);
            const int j1 = i1 + lo1 + c1, j2 = i2 + lo2 + c2, j3 = i3 + lo3 + c3;
            col[base + t] = j1 + m * (j2 + m * j3);
        }
    }
}

inline int nblk(int64_t work, int threads) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, (int64_t)1 << 30));
}

int check_patch(const amg_iga_patch* P, IgaDims& d) {
    if (!P) return AMG_ERR_ARG;
    const int nq = P->nq == 0 ? P->p + 1 : P->nq;
    if (P->n < 1 || P->p < 1 || P->p > kMaxDeg || nq < 1 || nq > kMaxNq) return AMG_ERR_ARG;
    if ((int64_t)P->n * nq > kMaxQ) return AMG_ERR_ARG;
    if (P->geometry != AMG_GEOM_CUBE && P->geometry != AMG_GEOM_ANNULUS) return AMG_ERR_ARG;
    if (P->with_boundary != 0 && P->with_boundary != 1) return AMG_ERR_ARG;
    if (P->source != AMG_SRC_ONE && P->source != AMG_SRC_SINE) return AMG_ERR_ARG;
    if (P->kappa_m < 0 || P->kappa_m > 65536) return AMG_ERR_ARG;
    if (P->kappa_m > 0 && (!P->kappa_omega || !P->kappa_phi || !std::isfinite(P->kappa_sigma))) return AMG_ERR_ARG;
    d.n = P->n;
    d.p = P->p;
    d.nq = nq;
    d.off = P->with_boundary ? 0 : 1;
    d.m = P->with_boundary ? P->n + P->p : P->n + P->p - 2;
    d.Q = P->n * nq;
    d.B = 2 * P->p + 1;
    d.R = d.m * d.B;
    d.Lmax = (P->p + 1) * nq;
    d.R1 = d.m;
    d.L1max = (P->p + 1) * nq;
    if (d.m > 0 && (int64_t)d.m * d.m * d.m > 0x7fffffffLL) return AMG_ERR_ARG;
    return AMG_OK;
}

}  // namespace
}  // namespace amg

using namespace amg;

extern "C" int amg_iga_size(const amg_iga_patch* P, int64_t* n, int64_t* nnz) {
    IgaDims d;
    const int rc = check_patch(P, d);
    if (rc != AMG_OK) return rc;
    if (!n || !nnz) return AMG_ERR_ARG;
    const int64_t m = std::max(d.m, 0);
    const int64_t T = m > 0 ? band_prefix(m, m, d.p) : 0;
    *n = m * m * m;
    *nnz = T * T * T;
    return AMG_OK;
}

extern "C" int amg_iga_assemble(const amg_iga_patch* P, int64_t* rowptr, int32_t* col, double* val, double* F,
                                void* cuda_stream, double* flops) {
    IgaDims d;
    int rc = check_patch(P, d);
    if (rc != AMG_OK) return rc;
    if (!rowptr || !col || !val) return AMG_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int m = std::max(d.m, 0);
    if (m == 0) {  // nothing kept: rowptr = {0}
        cudaError_t e = cudaMemsetAsync(rowptr, 0, sizeof(int64_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (flops) *flops = 0.0;
        return e == cudaSuccess ? AMG_OK : report_cuda(e, "amg_iga_assemble");
    }
    const int Q = d.Q;
    const int64_t P2 = (int64_t)Q * Q, P3 = P2 * Q, R = d.R, R2 = R * R;
    const int M = P->kappa_m;
    const int K2 = M > 0 ? ((2 * M + kGK - 1) / kGK) * kGK : 0;
    const bool has01 = P->geometry != AMG_GEOM_CUBE;
    std::vector<void*> bufs;
    struct Free {
        std::vector<void*>* b;
        cudaStream_t s;
        ~Free() {
            for (void* p : *b)
                if (p) cudaFreeAsync(p, s);
        }
    } guard{&bufs, s};
    cudaError_t err = cudaSuccess;
    auto get = [&](auto** p, size_t count) {
        *p = nullptr;
        if (err != cudaSuccess) return;
        void* q = nullptr;
        err = dev_alloc(&q, std::max<size_t>(count, 1) * sizeof(**p), s);
        if (err == cudaSuccess) {
            bufs.push_back(q);
            *p = reinterpret_cast<std::remove_reference_t<decltype(*p)>>(q);
        }
    };
    auto release = [&](void* p) {
        auto it = std::find(bufs.begin(), bufs.end(), p);
        if (it != bufs.end()) {
            cudaFreeAsync(p, s);
            bufs.erase(it);
        }
    };
    double *gx, *gw, *V, *D, *plane, *zl, *Wt[4], *W1;
    int *sp, *Lp, *s1, *L1;
    get(&gx, d.nq);
    get(&gw, d.nq);
    get(&V, (size_t)Q * (d.p + 1));
    get(&D, (size_t)Q * (d.p + 1));
    get(&plane, (size_t)P2 * 6);
    get(&zl, (size_t)Q * 2);
    for (auto& w : Wt) get(&w, (size_t)R * d.Lmax);
    get(&W1, (size_t)d.R1 * d.L1max);
    get(&sp, R);
    get(&Lp, R);
    get(&s1, d.R1);
    get(&L1, d.R1);
    if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble workspace");
    double *const Wvv = Wt[0], *const Wvd = Wt[1], *const Wdv = Wt[2], *const Wdd = Wt[3];
    k_iga_gauss<<<AMG_GRID(1), 32, 0, s>>>(d.nq, gx, gw);
    k_iga_basis<<<AMG_GRID(nblk(Q, 128)), 128, 0, s>>>(d.n, d.p, d.nq, gx, V, D);
    k_iga_pairs<<<AMG_GRID(nblk(R * d.Lmax, 256)), 256, 0, s>>>(d, V, D, sp, Lp, Wvv, Wvd, Wdv, Wdd);
    k_iga_single<<<AMG_GRID(nblk((int64_t)d.R1 * d.L1max, 256)), 256, 0, s>>>(d, V, s1, L1, W1);
    k_iga_plane<<<AMG_GRID(nblk(P2, 256)), 256, 0, s>>>(P->geometry, d.n, d.nq, gx, gw, plane);
    k_iga_zline<<<AMG_GRID(nblk(Q, 128)), 128, 0, s>>>(d.n, d.nq, gx, gw, zl);
    k_iga_pattern<<<AMG_GRID(nblk((int64_t)m * m * m * 32, 256)), 256, 0, s>>>(m, d.p, rowptr, col);
    // coefficients at every Gauss point
    CoefOut co{};
    get(&co.c00, (size_t)P3);
    if (has01) get(&co.c01, (size_t)P3);
    get(&co.c11, (size_t)P3);
    get(&co.c22, (size_t)P3);
    if (F) get(&co.e, (size_t)P3);
    if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble coefficients");
    double gemm_fma = 0.0;
    if (M > 0) {
        double *Ak, *Bk;
        get(&Ak, (size_t)P2 * K2);
        get(&Bk, (size_t)K2 * Q);
        if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble kappa");
        k_iga_kappa_plane<<<AMG_GRID(nblk(P2 * K2, 256)), 256, 0, s>>>(P2, M, K2, plane, P->kappa_omega,
                                                                          P->kappa_phi, Ak);
        k_iga_kappa_z<<<AMG_GRID(nblk((int64_t)K2 * Q, 256)), 256, 0, s>>>(Q, M, K2, zl, P->kappa_omega, Bk);
        const double amp = P->kappa_sigma * sqrt(2.0 / M);
        dim3 grid((unsigned)((P2 + kGT - 1) / kGT), (unsigned)((Q + kGT - 1) / kGT));
        k_iga_coef_gemm<<<AMG_GRID(grid), 256, 0, s>>>(P2, Q, K2, Ak, Bk, amp, plane, zl, P->source, co);
        gemm_fma = (double)P2 * Q * (2.0 * M);
        release(Ak);
        release(Bk);
    } else {
        k_iga_coef_const<<<AMG_GRID(nblk(P3, 256)), 256, 0, s>>>(P2, Q, plane, zl, P->source, co);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return report_cuda(err, "amg_iga_assemble launch");
    // contractions: Q x 32 staging per block
    const size_t smo = (size_t)Q * kCtIn * sizeof(double);
    if ((err = cudaFuncSetAttribute(k_iga_outer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smo)) !=
        cudaSuccess)
        return report_cuda(err, "amg_iga_assemble smem");
    auto outer = [&](const double* X, int64_t O, int64_t IN, int Rr, const int* ss, const int* LL, const double* W,
                     int Lm, double* Y, int accumulate) {
        dim3 grid((unsigned)((IN + kCtIn - 1) / kCtIn), (unsigned)O);
        k_iga_outer<<<AMG_GRID(grid), 32 * kCtWarps, smo, s>>>(IN, Q, Rr, X, ss, LL, W, Lm, Y, accumulate);
    };
    // direction 3
    double *A00, *A01 = nullptr, *A11, *A22;
    get(&A00, (size_t)R * P2);
    if (has01) get(&A01, (size_t)R * P2);
    get(&A11, (size_t)R * P2);
    get(&A22, (size_t)R * P2);
    if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble direction 3");
    outer(co.c00, 1, P2, d.R, sp, Lp, Wvv, d.Lmax, A00, 0);
    if (has01) outer(co.c01, 1, P2, d.R, sp, Lp, Wvv, d.Lmax, A01, 0);
    outer(co.c11, 1, P2, d.R, sp, Lp, Wvv, d.Lmax, A11, 0);
    outer(co.c22, 1, P2, d.R, sp, Lp, Wdd, d.Lmax, A22, 0);
    double *fa = nullptr, *fb = nullptr;
    if (F) {
        get(&fa, (size_t)m * P2);
        if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble load");
        outer(co.e, 1, P2, d.R1, s1, L1, W1, d.L1max, fa, 0);
    }
    release(co.c00);
    release(co.c01);
    release(co.c11);
    release(co.c22);
    release(co.e);
    // direction 2, grouped by the direction-1 type
    double *Gdd, *Gdv = nullptr, *Gvd = nullptr, *Gvv;
    get(&Gdd, (size_t)R2 * Q);
    if (has01) {
        get(&Gdv, (size_t)R2 * Q);
        get(&Gvd, (size_t)R2 * Q);
    }
    get(&Gvv, (size_t)R2 * Q);
    if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble direction 2");
    outer(A00, R, Q, d.R, sp, Lp, Wvv, d.Lmax, Gdd, 0);
    if (has01) {
        outer(A01, R, Q, d.R, sp, Lp, Wvd, d.Lmax, Gdv, 0);
        outer(A01, R, Q, d.R, sp, Lp, Wdv, d.Lmax, Gvd, 0);
    }
    outer(A11, R, Q, d.R, sp, Lp, Wdd, d.Lmax, Gvv, 0);
    outer(A22, R, Q, d.R, sp, Lp, Wvv, d.Lmax, Gvv, 1);
    if (F) {
        get(&fb, (size_t)m * m * Q);
        if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble load");
        outer(fa, m, Q, d.R1, s1, L1, W1, d.L1max, fb, 0);
        release(fa);
    }
    release(A00);
    release(A01);
    release(A11);
    release(A22);
    // direction 1 and the scatter
    InnerGroups G{};
    G.X[G.ng] = Gdd;
    G.W[G.ng++] = Wdd;
    if (has01) {
        G.X[G.ng] = Gdv;
        G.W[G.ng++] = Wdv;
        G.X[G.ng] = Gvd;
        G.W[G.ng++] = Wvd;
    }
    G.X[G.ng] = Gvv;
    G.W[G.ng++] = Wvv;
    // rows per block of the last contraction: 8 (four pairs per warp), so
    // that several blocks share an SM (16 rows left one block, 8 warps, per
    // SM: 12 % of the warp slots); fewer when the staged rows do not fit
    int optin = 0, devi = 0;
    if ((err = cudaGetDevice(&devi)) != cudaSuccess ||
        (err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, devi)) != cudaSuccess)
        return report_cuda(err, "amg_iga_assemble device");
    int rows = 8;
    while (rows > 1 && (size_t)G.ng * rows * (Q + 1) * sizeof(double) > (size_t)optin / 2) rows >>= 1;
    const size_t smi = (size_t)G.ng * rows * (Q + 1) * sizeof(double);
    if (smi > (size_t)optin) return AMG_ERR_ARG;
    auto inner = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
        if (e != cudaSuccess) return e;
        kern<<<AMG_GRID(nblk(R2, rows)), kInThreads, smi, s>>>(d, G, rows, sp, Lp, rowptr, val);
        return cudaGetLastError();
    };
    err = G.ng == 4 ? inner(k_iga_inner_csr<4>) : inner(k_iga_inner_csr<2>);
    if (err != cudaSuccess) return report_cuda(err, "amg_iga_assemble last contraction");
    if (F) {
        const size_t smf = (size_t)kInRows * (Q + 1) * sizeof(double);
        if ((err = cudaFuncSetAttribute(k_iga_inner_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smf)) != cudaSuccess)
            return report_cuda(err, "amg_iga_assemble smem");
        k_iga_inner_dense<<<AMG_GRID(nblk((int64_t)m * m, kInRows)), 32 * kInRows, smf, s>>>(d, fb, s1, L1, W1, F);
    }
    if ((err = cudaGetLastError()) != cudaSuccess) return report_cuda(err, "amg_iga_assemble launch");
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return report_cuda(err, "amg_iga_assemble");
    if (flops) {
        // FMAs of the GEMM and of the contractions (sums over the pair tables' lengths)
        std::vector<int> Lh(d.R), L1h(d.R1);
        if ((err = cudaMemcpy(Lh.data(), Lp, sizeof(int) * d.R, cudaMemcpyDeviceToHost)) != cudaSuccess ||
            (err = cudaMemcpy(L1h.data(), L1, sizeof(int) * d.R1, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return report_cuda(err, "amg_iga_assemble flops");
        double sl = 0.0, sl1 = 0.0;
        for (int v : Lh) sl += v;
        for (int v : L1h) sl1 += v;
        // pairs whose second function is kept (the others are zero rows)
        double rows_ok = 0.0;
        for (int r = 0; r < d.R; r++) rows_ok += Lh[r] > 0 ? 1.0 : 0.0;
        const int na = has01 ? 4 : 3, nb = has01 ? 5 : 3;
        double fma_k = na * sl * (double)P2 + nb * rows_ok * sl * Q + G.ng * rows_ok * rows_ok * sl;
        double fma_f = F ? sl1 * (double)P2 + (double)m * sl1 * Q + (double)m * m * sl1 : 0.0;
        *flops = 2.0 * (gemm_fma + fma_k + fma_f);
    }
    return AMG_OK;
}
