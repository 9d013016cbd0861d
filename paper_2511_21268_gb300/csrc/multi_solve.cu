// Multi-system CG: S independent CG iterations sharing one AMG hierarchy,
// run in one graph-captured loop (arXiv 2511.21268 Sec. 3 V-cycle and CG;
// the batching is this library's design).
//
//   * R right-hand sides of one matrix: vectors interleaved as [N][R]; a
//     matrix pass reads each matrix entry once for all R vectors (SpMM):
//     R lanes (rounded up to a power of two) share a row, every lane owns
//     one right-hand side, the entry value and column are broadcast and
//     the R vector values of a column are one coalesced load.  System s =
//     right-hand side s.
//   * a batch of independent matrices assembled block-diagonally into one
//     hierarchy (there are no coupling entries, so matchings, aggregates and
//     Galerkin products never cross blocks and every level operator is
//     block diagonal): R = 1, system of row i = seg[i].
//
// Each system has its own CG scalars and convergence test; the dot products
// are per-system sums in a fixed order (deterministic).  Converged systems
// are frozen while the others iterate.  The V-cycle uses one pre- and one
// post-smoothing sweep.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
enum { D_RR = 0, D_FF, D_PQ, D_PR, D_RZ, D_ZQ, D_RR2, D_COUNT };

__device__ __forceinline__ double ldm(const double* v, int64_t k) { return __ldg(v + k); }
__device__ __forceinline__ float ldm(const float* v, int64_t k) { return __ldg(v + k); }
__device__ __forceinline__ float ldm(const __nv_bfloat16* v, int64_t k) { return __bfloat162float(v[k]); }

// Element (row i, vector c) handled by this thread; false when outside.
#define MULTI_ELEM(n, R, Rp)                                      \
    const int64_t g__ = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; \
    const int i = (int)(g__ / (Rp)), c = (int)(g__ % (Rp));       \
    if (i >= (n) || c >= (R)) return;

__device__ __forceinline__ int sys_of(const int32_t* seg, int i, int c) { return seg ? seg[i] : c; }

// sum_k v_k X[col_k][c] over row i (values V, vectors X, accumulation A)
template <typename A, typename V, typename X>
__device__ __forceinline__ A row_dot_m(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                       const V* __restrict__ v, const X* __restrict__ x, int i, int R, int c) {
    const int64_t b = rp[i], e = rp[i + 1];
    A acc = A(0);
    int64_t k = b;
    for (; k + 3 < e; k += 4) {
        const A v0 = (A)ldm(v, k), v1 = (A)ldm(v, k + 1), v2 = (A)ldm(v, k + 2), v3 = (A)ldm(v, k + 3);
        const int c0 = __ldg(ci + k), c1 = __ldg(ci + k + 1), c2 = __ldg(ci + k + 2), c3 = __ldg(ci + k + 3);
        const A x0 = (A)x[(int64_t)c0 * R + c], x1 = (A)x[(int64_t)c1 * R + c];
        const A x2 = (A)x[(int64_t)c2 * R + c], x3 = (A)x[(int64_t)c3 * R + c];
        acc = fma(v0, x0, acc);
        acc = fma(v1, x1, acc);
        acc = fma(v2, x2, acc);
        acc = fma(v3, x3, acc);
    }
    for (; k < e; k++) acc = fma((A)ldm(v, k), (A)x[(int64_t)__ldg(ci + k) * R + c], acc);
    return acc;
}

// ----------------------------------------------------------------- kernels
// FP64 residual r = F - K x; x0 = r / d (V-cycle precision); products r^2
// and F^2.  gate: only systems whose replacement is due.
template <typename X0>
__global__ void k_m_residual(int n, int R, int Rp, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const double* __restrict__ v, const double* __restrict__ x, const double* __restrict__ F,
                             const X0* __restrict__ invd, double* r, X0* x0, double* pa, double* pb,
                             const MultiState* gate, const int32_t* seg) {
    MULTI_ELEM(n, R, Rp)
    const int64_t e = (int64_t)i * R + c;
    if (gate) {
        const MultiState& s = gate[sys_of(seg, i, c)];
        if (s.done || !s.replace_now) return;
    }
    const double fi = F[e];
    const double ri = fi - row_dot_m<double>(rp, ci, v, x, i, R, c);
    r[e] = ri;
    if (x0) x0[e] = (X0)ri * invd[i];
    pa[e] = ri * ri;
    if (pb) pb[e] = fi * fi;
}

// Outer q = K p; products p.q and (flexible) p.r.
template <typename A, typename V, typename PX>
__global__ void k_m_spmv_pq(int n, int R, int Rp, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const V* __restrict__ v, const PX* __restrict__ pg, const double* __restrict__ p,
                            const double* __restrict__ r, double* q, double* pa, double* pb, int flexible,
                            const MultiState* st, const int32_t* seg, const int* active) {
    if (*active == 0) return;
    MULTI_ELEM(n, R, Rp)
    if (st[sys_of(seg, i, c)].done) return;
    const int64_t e = (int64_t)i * R + c;
    const double qs = (double)row_dot_m<A>(rp, ci, v, pg, i, R, c);
    q[e] = qs;
    pa[e] = p[e] * qs;
    if (flexible) pb[e] = p[e] * r[e];
}

// V-cycle down-sweep residual rbuf = f - K x.
template <typename A, typename V, typename FT>
__global__ void k_m_resid(int n, int R, int Rp, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const V* __restrict__ v, const FT* __restrict__ f, const A* __restrict__ x, A* rbuf,
                          const int* active) {
    if (*active == 0) return;
    MULTI_ELEM(n, R, Rp)
    const int64_t e = (int64_t)i * R + c;
    rbuf[e] = (A)f[e] - row_dot_m<A>(rp, ci, v, x, i, R, c);
}

template <typename A>
__global__ void k_m_restrict(int nc, int R, const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                             const double* __restrict__ pval, const A* __restrict__ rbuf, A* fc, A* xc,
                             const A* __restrict__ invdc, const int* active) {
    if (*active == 0) return;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)nc * R) return;
    const int I = (int)(g / R), c = (int)(g % R);
    A acc = A(0);
    for (int m = mptr[I]; m < mptr[I + 1]; m++) {
        const int a = midx[m];
        acc = fma((A)pval[a], rbuf[(int64_t)a * R + c], acc);
    }
    fc[g] = acc;
    if (xc) xc[g] = acc * invdc[I];
}

// Coarsest level, e = A^-1 f per vector; prolongation into the finer level,
// or (single-level hierarchy) z = e with the products r.z and z.q.
template <typename FT, typename XT>
__global__ void k_m_coarse(int nd, int R, const double* __restrict__ Ainv, const FT* __restrict__ f,
                           const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                           const double* __restrict__ pvalf, XT* xf, double* z, const double* __restrict__ q,
                           double* pa, double* pb, int flexible, const int* active) {
    if (*active == 0) return;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)nd * R) return;
    const int I = (int)(g / R), c = (int)(g % R);
    const double* row = Ainv + (int64_t)I * nd;
    double s = 0.0;
    for (int j = 0; j < nd; j++) s = fma(row[j], (double)f[(int64_t)j * R + c], s);
    if (z) {
        z[g] = s;
        pa[g] = (double)f[g] * s;
        if (flexible) pb[g] = s * q[g];
    } else {
        for (int m = mptr[I]; m < mptr[I + 1]; m++) {
            const int a = midx[m];
            const int64_t e = (int64_t)a * R + c;
            xf[e] = (XT)fma(pvalf[a], s, (double)xf[e]);
        }
    }
}

template <typename A, typename V>
__global__ void k_m_up(int n, int R, int Rp, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const V* __restrict__ v, const A* __restrict__ f, const A* __restrict__ x,
                       const A* __restrict__ invd, const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                       const double* __restrict__ pvalf, A* xf, const int* active) {
    if (*active == 0) return;
    MULTI_ELEM(n, R, Rp)
    const int64_t e = (int64_t)i * R + c;
    const A y = fma(invd[i], f[e] - row_dot_m<A>(rp, ci, v, x, i, R, c), x[e]);
    for (int m = mptr[i]; m < mptr[i + 1]; m++) {
        const int a = midx[m];
        const int64_t ea = (int64_t)a * R + c;
        xf[ea] = fma((A)pvalf[a], y, xf[ea]);
    }
}

template <typename A, typename V>
__global__ void k_m_up0(int n, int R, int Rp, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                        const V* __restrict__ v, const double* __restrict__ r, const A* __restrict__ x,
                        const A* __restrict__ invd, double* z, const double* __restrict__ q, double* pa, double* pb,
                        int flexible, const int* active) {
    if (*active == 0) return;
    MULTI_ELEM(n, R, Rp)
    const int64_t e = (int64_t)i * R + c;
    const double ra = r[e];
    const double za = (double)fma(invd[i], (A)ra - row_dot_m<A>(rp, ci, v, x, i, R, c), x[e]);
    z[e] = za;
    pa[e] = ra * za;
    if (flexible) pb[e] = za * q[e];
}

// x += alpha p, r -= alpha q, x0 = r / d, product r^2 (systems not done).
template <typename X0>
__global__ void k_m_update(int n, int R, double* x, double* r, const double* __restrict__ p,
                           const double* __restrict__ q, const X0* __restrict__ invd, X0* x0, double* pa,
                           const MultiState* st, const int32_t* seg, const int* active) {
    if (*active == 0) return;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * R) return;
    const int i = (int)(g / R), c = (int)(g % R);
    const MultiState& s = st[sys_of(seg, i, c)];
    if (s.done) return;
    const double alpha = s.alpha;
    x[g] = fma(alpha, p[g], x[g]);
    const double ri = fma(-alpha, q[g], r[g]);
    r[g] = ri;
    if (x0) x0[g] = (X0)ri * invd[i];
    pa[g] = ri * ri;
}

__global__ void k_m_pupdate(int n, int R, double* p, const double* __restrict__ z, float* p32, int first,
                            const MultiState* st, const int32_t* seg, const int* active) {
    if (*active == 0) return;
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * R) return;
    const int i = (int)(g / R), c = (int)(g % R);
    const MultiState& s = st[sys_of(seg, i, c)];
    if (s.done) return;
    const double pi = first ? z[g] : fma(s.beta, p[g], z[g]);
    p[g] = pi;
    if (p32) p32[g] = __double2float_rn(pi);
}

// dots[s * D_COUNT + slot] = sum over the elements of system s (fixed order);
// one block per system.
__global__ void k_m_sys_sum(int n, int R, const int64_t* __restrict__ segoff, const double* __restrict__ pa, int sa,
                            const double* __restrict__ pb, int sb, double* dots, const int* active) {
    if (active && *active == 0) return;
    const int s = blockIdx.x;
    int64_t lo, hi, stride, off;
    if (segoff) {
        lo = segoff[s];
        hi = segoff[s + 1];
        stride = 1;
        off = 0;
    } else {
        lo = 0;
        hi = n;
        stride = R;
        off = s;
    }
    double a = 0.0, b = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        a += pa[i * stride + off];
        if (pb) b += pb[i * stride + off];
    }
    __shared__ double sha[32], shb[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL, a, o);
        b += __shfl_xor_sync(FULL, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sha[threadIdx.x >> 5] = a;
        shb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            ta += sha[w];
            tb += shb[w];
        }
        dots[s * D_COUNT + sa] = ta;
        if (pb) dots[s * D_COUNT + sb] = tb;
    }
}

// ------------------------------------------------------------------ scalars
// One block, one thread per system; *active = number of systems not done.
__device__ void count_active(int S, const MultiState* st, int* active) {
    __shared__ int cnt;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < S; s += blockDim.x)
        if (!st[s].done) atomicAdd(&cnt, 1);
    __syncthreads();
    if (threadIdx.x == 0) *active = cnt;
}

__global__ void k_m_scal_init(int S, const double* dots, double rtol, int itmax, int repl, MultiState* st,
                              int* active, int* itmax_out) {
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        MultiState& m = st[s];
        const double nF = sqrt(dots[s * D_COUNT + D_FF]), nr = sqrt(dots[s * D_COUNT + D_RR]);
        m.nF = nF;
        m.tol = rtol * nF;
        m.nr = nr;
        m.iters = 0;
        m.status = AMG_OK;
        m.done = 0;
        m.replace_now = 0;
        if (isnan(nr) || isnan(nF) || isinf(nr) || isinf(nF)) {
            m.status = AMG_ERR_NAN;
            m.done = 1;
        } else if (!(nF > 0.0) || nr <= m.tol) {
            m.done = 1;
        } else if (itmax <= 0) {
            m.status = AMG_ERR_NOT_CONVERGED;
            m.done = 1;
        }
    }
    if (threadIdx.x == 0) {
        itmax_out[0] = itmax;
        itmax_out[1] = repl;
    }
    count_active(S, st, active);
}

__global__ void k_m_scal_alpha(int S, const double* dots, int flexible, MultiState* st, int* active) {
    if (*active == 0) return;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        MultiState& m = st[s];
        if (m.done) continue;
        const double pq = dots[s * D_COUNT + D_PQ];
        const double num = flexible ? dots[s * D_COUNT + D_PR] : m.rho;
        m.pq = pq;
        if (!(pq > 0.0)) {
            m.status = (isnan(pq) || isnan(num)) ? AMG_ERR_NAN : AMG_ERR_BREAKDOWN;
            m.done = 1;
        } else {
            m.alpha = num / pq;
        }
    }
    count_active(S, st, active);
}

__global__ void k_m_scal_conv(int S, const double* dots, int mixed, const int* params, MultiState* st, int* active) {
    if (*active == 0) return;
    const int itmax = params[0], repl = params[1];
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        MultiState& m = st[s];
        if (m.done) continue;
        const double nr = sqrt(dots[s * D_COUNT + D_RR]);
        const int it = m.iters + 1;
        m.iters = it;
        m.nr = nr;
        if (isnan(nr) || isinf(nr)) {
            m.status = AMG_ERR_NAN;
            m.done = 1;
        } else if (mixed && (nr <= m.tol || it >= itmax || (repl > 0 && it % repl == 0))) {
            m.replace_now = 1;
        } else if (nr <= m.tol) {
            m.done = 1;
        } else if (it >= itmax) {
            m.status = AMG_ERR_NOT_CONVERGED;
            m.done = 1;
        }
    }
    count_active(S, st, active);
}

__global__ void k_m_scal_replaced(int S, const double* dots, const int* params, MultiState* st, int* active) {
    if (*active == 0) return;
    const int itmax = params[0];
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        MultiState& m = st[s];
        if (m.done || !m.replace_now) continue;
        const double nr = sqrt(dots[s * D_COUNT + D_RR2]);
        m.nr = nr;
        m.replace_now = 0;
        if (isnan(nr) || isinf(nr)) {
            m.status = AMG_ERR_NAN;
            m.done = 1;
        } else if (nr <= m.tol) {
            m.done = 1;
        } else if (m.iters >= itmax) {
            m.status = AMG_ERR_NOT_CONVERGED;
            m.done = 1;
        }
    }
    count_active(S, st, active);
}

__global__ void k_m_scal_beta(int S, const double* dots, int flexible, int first, MultiState* st, int* active) {
    if (*active == 0) return;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        MultiState& m = st[s];
        if (m.done) continue;
        const double rz = dots[s * D_COUNT + D_RZ];
        const double zq = dots[s * D_COUNT + D_ZQ];
        if (isnan(rz) || (flexible && !first && isnan(zq))) {
            m.status = AMG_ERR_NAN;
            m.done = 1;
            continue;
        }
        m.beta = first ? 0.0 : (flexible ? -zq / m.pq : rz / m.rho);
        m.rho = rz;
    }
    count_active(S, st, active);
}

// [N][R] <-> column-major (leading dimension ld) copies
__global__ void k_interleave(int n, int R, int64_t ld, const double* __restrict__ src, double* dst) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * R) return;
    const int i = (int)(g / R), c = (int)(g % R);
    dst[g] = src[(int64_t)c * ld + i];
}

__global__ void k_deinterleave(int n, int R, int64_t ld, const double* __restrict__ src, double* dst) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)n * R) return;
    const int i = (int)(g % n), c = (int)(g / n);
    dst[(int64_t)c * ld + i] = src[(int64_t)i * R + c];
}

// ----------------------------------------------------------------- host side
inline int elem_blocks(int64_t count) { return (int)((count + 255) / 256 > 0 ? (count + 255) / 256 : 1); }

template <typename A>
struct MView;

template <>
struct MView<double> {
    static double* f(MultiWork& w, int l) { return static_cast<double*>(w.lf[l]); }
    static double* x(MultiWork& w, int l) { return static_cast<double*>(w.lx[l]); }
    static double* t(MultiWork& w, int l) { return static_cast<double*>(w.lt[l]); }
    static const double* invd(Level& L) { return L.invd; }
    template <typename Fn>
    static void vals(Level& L, int, Fn&& fn) { fn(static_cast<const double*>(L.A.val)); }
};

template <>
struct MView<float> {
    static float* f(MultiWork& w, int l) { return static_cast<float*>(w.lf[l]); }
    static float* x(MultiWork& w, int l) { return static_cast<float*>(w.lx[l]); }
    static float* t(MultiWork& w, int l) { return static_cast<float*>(w.lt[l]); }
    static const float* invd(Level& L) { return L.invd32; }
    template <typename Fn>
    static void vals(Level& L, int l, Fn&& fn) {
        if (l == 0 && L.val16) fn(static_cast<const __nv_bfloat16*>(L.val16));
        else fn(static_cast<const float*>(L.val32));
    }
};

template <typename T>
using vt = std::remove_cv_t<std::remove_pointer_t<T>>;

template <typename A>
cudaError_t m_vcycle(amg_hierarchy* h, cudaStream_t s) {
    using Vw = MView<A>;
    MultiWork& w = *h->mw;
    const int L = h->nlev, R = w.R, Rp = w.Rp, flex = h->o.flexible;
    const int* act = w.active;
    if (L == 1) {
        k_m_coarse<double, A><<<AMG_GRID(elem_blocks((int64_t)h->ndense * R)), 256, 0, s>>>(
            h->ndense, R, h->Ainv, w.r, nullptr, nullptr, nullptr, nullptr, w.z, w.q, w.pa, w.pb, flex, act);
        return cudaGetLastError();
    }
    for (int l = 0; l < L - 1; l++) {
        Level& F = h->lev[l];
        Level& C = h->lev[l + 1];
        const int n = F.A.n;
        const int nb = elem_blocks((int64_t)n * Rp);
        Vw::vals(F, l, [&](auto vp) {
            using V = vt<decltype(vp)>;
            if (l == 0)
                k_m_resid<A, V, double><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, F.A.rowptr, F.A.col, vp, w.r,
                                                                     Vw::x(w, 0), Vw::t(w, 0), act);
            else
                k_m_resid<A, V, A><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, F.A.rowptr, F.A.col, vp, Vw::f(w, l),
                                                                Vw::x(w, l), Vw::t(w, l), act);
        });
        const bool coarsest = (l + 1 == L - 1);
        k_m_restrict<A><<<AMG_GRID(elem_blocks((int64_t)C.A.n * R)), 256, 0, s>>>(
            C.A.n, R, F.mem_ptr, F.mem_idx, F.pval, Vw::t(w, l), Vw::f(w, l + 1), coarsest ? nullptr : Vw::x(w, l + 1),
            Vw::invd(C), act);
    }
    {
        Level& F = h->lev[L - 2];
        Level& C = h->lev[L - 1];
        k_m_coarse<A, A><<<AMG_GRID(elem_blocks((int64_t)C.A.n * R)), 256, 0, s>>>(
            C.A.n, R, h->Ainv, Vw::f(w, L - 1), F.mem_ptr, F.mem_idx, F.pval, Vw::x(w, L - 2), nullptr, nullptr,
            nullptr, nullptr, 0, act);
    }
    for (int l = L - 2; l >= 0; l--) {
        Level& F = h->lev[l];
        const int n = F.A.n;
        const int nb = elem_blocks((int64_t)n * Rp);
        Vw::vals(F, l, [&](auto vp) {
            using V = vt<decltype(vp)>;
            if (l == 0) {
                k_m_up0<A, V><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, F.A.rowptr, F.A.col, vp, w.r, Vw::x(w, 0),
                                                           Vw::invd(F), w.z, w.q, w.pa, w.pb, flex, act);
            } else {
                Level& G = h->lev[l - 1];
                k_m_up<A, V><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, F.A.rowptr, F.A.col, vp, Vw::f(w, l),
                                                          Vw::x(w, l), Vw::invd(F), G.mem_ptr, G.mem_idx, G.pval,
                                                          Vw::x(w, l - 1), act);
            }
        });
    }
    return cudaGetLastError();
}

cudaError_t m_vcycle_any(amg_hierarchy* h, cudaStream_t s) {
    return h->mixed ? m_vcycle<float>(h, s) : m_vcycle<double>(h, s);
}

cudaError_t m_residual(amg_hierarchy* h, double* r, bool x0, bool ff, const MultiState* gate, cudaStream_t s) {
    MultiWork& w = *h->mw;
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int nb = elem_blocks((int64_t)n * w.Rp);
    const bool want = x0 && h->nlev > 1;
    if (h->mixed)
        k_m_residual<float><<<AMG_GRID(nb), 256, 0, s>>>(n, w.R, w.Rp, L0.A.rowptr, L0.A.col, L0.A.val, w.x, w.F,
                                                         L0.invd32, r, want ? static_cast<float*>(w.lx[0]) : nullptr,
                                                         w.pa, ff ? w.pb : nullptr, gate, w.seg);
    else
        k_m_residual<double><<<AMG_GRID(nb), 256, 0, s>>>(n, w.R, w.Rp, L0.A.rowptr, L0.A.col, L0.A.val, w.x, w.F,
                                                          L0.invd, r, want ? static_cast<double*>(w.lx[0]) : nullptr,
                                                          w.pa, ff ? w.pb : nullptr, gate, w.seg);
    return cudaGetLastError();
}

void m_sum(amg_hierarchy* h, const double* pa, int sa, const double* pb, int sb, const int* act, cudaStream_t s) {
    MultiWork& w = *h->mw;
    k_m_sys_sum<<<AMG_GRID(w.S), 256, 0, s>>>(h->lev[0].A.n, w.R, w.segoff, pa, sa, pb, sb, w.dots, act);
}

void m_pupdate(amg_hierarchy* h, int first, cudaStream_t s) {
    MultiWork& w = *h->mw;
    const int64_t cnt = (int64_t)h->lev[0].A.n * w.R;
    k_m_pupdate<<<AMG_GRID(elem_blocks(cnt)), 256, 0, s>>>(h->lev[0].A.n, w.R, w.p, w.z, h->mixed ? w.p32 : nullptr,
                                                           first, w.st, w.seg, w.active);
}

}  // namespace

cudaError_t enqueue_multi_start(amg_hierarchy* h, cudaStream_t s) {
    MultiWork& w = *h->mw;
    AMG_TRY(m_residual(h, w.r, true, true, nullptr, s));
    m_sum(h, w.pa, D_RR, w.pb, D_FF, nullptr, s);
    k_m_scal_init<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, h->rtol, h->itmax,
                                               h->mixed ? h->o.resid_replace_every : 0, w.st, w.active, w.params);
    AMG_TRY(cudaGetLastError());
    AMG_TRY(m_vcycle_any(h, s));
    m_sum(h, w.pa, D_RZ, h->o.flexible ? w.pb : nullptr, D_ZQ, w.active, s);
    k_m_scal_beta<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, h->o.flexible, 1, w.st, w.active);
    m_pupdate(h, 1, s);
    return cudaGetLastError();
}

cudaError_t enqueue_multi_iteration(amg_hierarchy* h, cudaStream_t s) {
    MultiWork& w = *h->mw;
    Level& L0 = h->lev[0];
    const int n = L0.A.n, R = w.R, Rp = w.Rp, flex = h->o.flexible;
    const int nb = elem_blocks((int64_t)n * Rp);
    if (h->mixed)
        k_m_spmv_pq<float, float, float><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, L0.A.rowptr, L0.A.col, L0.val32,
                                                                      w.p32, w.p, w.r, w.q, w.pa, w.pb, flex, w.st,
                                                                      w.seg, w.active);
    else
        k_m_spmv_pq<double, double, double><<<AMG_GRID(nb), 256, 0, s>>>(n, R, Rp, L0.A.rowptr, L0.A.col, L0.A.val,
                                                                         w.p, w.p, w.r, w.q, w.pa, w.pb, flex, w.st,
                                                                         w.seg, w.active);
    m_sum(h, w.pa, D_PQ, flex ? w.pb : nullptr, D_PR, w.active, s);
    k_m_scal_alpha<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, flex, w.st, w.active);
    const int64_t cnt = (int64_t)n * R;
    const bool x0 = h->nlev > 1;
    if (h->mixed)
        k_m_update<float><<<AMG_GRID(elem_blocks(cnt)), 256, 0, s>>>(
            n, R, w.x, w.r, w.p, w.q, L0.invd32, x0 ? static_cast<float*>(w.lx[0]) : nullptr, w.pa, w.st, w.seg,
            w.active);
    else
        k_m_update<double><<<AMG_GRID(elem_blocks(cnt)), 256, 0, s>>>(
            n, R, w.x, w.r, w.p, w.q, L0.invd, x0 ? static_cast<double*>(w.lx[0]) : nullptr, w.pa, w.st, w.seg,
            w.active);
    m_sum(h, w.pa, D_RR, nullptr, 0, w.active, s);
    k_m_scal_conv<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, h->mixed, w.params, w.st, w.active);
    if (h->mixed) {
        AMG_TRY(m_residual(h, w.r, true, false, w.st, s));
        m_sum(h, w.pa, D_RR2, nullptr, 0, w.active, s);
        k_m_scal_replaced<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, w.params, w.st, w.active);
    }
    AMG_TRY(cudaGetLastError());
    AMG_TRY(m_vcycle_any(h, s));
    m_sum(h, w.pa, D_RZ, flex ? w.pb : nullptr, D_ZQ, w.active, s);
    k_m_scal_beta<<<AMG_GRID(1), 1024, 0, s>>>(w.S, w.dots, flex, 0, w.st, w.active);
    m_pupdate(h, 0, s);
    return cudaGetLastError();
}

// ||F_s - K x_s|| and ||F_s|| per system into dots[s][RR], dots[s][FF].
cudaError_t enqueue_multi_final(amg_hierarchy* h, cudaStream_t s) {
    MultiWork& w = *h->mw;
    AMG_TRY(m_residual(h, w.q, false, true, nullptr, s));
    m_sum(h, w.pa, D_RR, w.pb, D_FF, nullptr, s);
    return cudaGetLastError();
}

int multi_dot_stride() { return D_COUNT; }

cudaError_t launch_interleave(int n, int R, int64_t ld, const double* src, double* dst, cudaStream_t s) {
    k_interleave<<<AMG_GRID(elem_blocks((int64_t)n * R)), 256, 0, s>>>(n, R, ld, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_deinterleave(int n, int R, int64_t ld, const double* src, double* dst, cudaStream_t s) {
    k_deinterleave<<<AMG_GRID(elem_blocks((int64_t)n * R)), 256, 0, s>>>(n, R, ld, src, dst);
    return cudaGetLastError();
}

}  // namespace amg
