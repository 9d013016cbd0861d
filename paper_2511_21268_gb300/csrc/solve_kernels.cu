// Solve-phase kernels: CG recurrences, V-cycle with l1-Jacobi smoothing,
// aggregate restriction/prolongation and the coarsest dense solve
// (arXiv 2511.21268, Sec. 3 two-level correction steps 1-5 applied
// recursively, Sec. 3.2 l1-Jacobi, Sec. 4 CG invocation).
//
// Matrix passes use one kernel shape: a warp owns a group of RPW
// consecutive rows.  For each row every lane accumulates the entries
// k = start + lane + 32 t (coalesced value/column loads, the vector gathered
// through L2), the 32 lane partials go to a shared-memory tile, and the row
// total is finished by 32/RPW lanes with one short sequential sum and
// log2(32/RPW) shuffles.  On GB300, where an SM issues about two FP64 FMAs
// per clock, this keeps the FP64 work per row close to nnz/32 warp
// instructions and runs each row's epilogue on RPW rows per instruction.
//
// Precision: every kernel is templated on the accumulation type A, the
// stored value type V and the vector types.  FP64 mode instantiates them
// with double everywhere.  Mixed mode runs the V-cycle in FP32 (values FP32,
// or BF16 on the finest level; FP32 vectors and 1/dl1), the outer SpMV with
// FP32 values and FP32 accumulation, and keeps FP64 for the CG vectors and
// recurrences, the dot products, the coarsest solve and a true-residual
// replacement r = F - K x with the FP64 matrix (periodic, and before any
// convergence is declared).
//
// Fusions:
//   * pre-smoothing from x = 0 is x = D^-1 f, written by whoever produces f
//     (the CG update for level 0, the restriction for level l+1);
//   * down sweep: r = f - K x into a scratch vector, then restriction
//     f_{l+1}[I] = sum_{a in I} p_a r_a and x_{l+1} = f_{l+1} / d;
//   * up sweep of level l: y = x + (f - K x) / d, prolongated at once into
//     the finer level, x_{l-1}[c] += p_c y_a for the members c of a; on
//     level 0 it writes z and the partial sums of r.z (and z.q);
//   * coarsest solve: dense FP64 GEMV with the precomputed inverse, followed
//     by the same prolongation.
// Reductions are deterministic: fixed grids, fixed lane/warp/block order and
// a single-block final sum.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "amg_internal.cuh"
#include "row_kernels.cuh"

namespace amg {

namespace {

// Deterministic single-block sum of nb partials (result on every thread).
// The warp totals are combined by thread 0 only: GB300's FP64 rate makes
// redundant per-thread FP64 adds costly.
__device__ double sum_partials(const double* __restrict__ part, int nb, double* sh) {
    double s = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s += part[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += sh[w];
        sh[32] = tot;
    }
    __syncthreads();
    const double tot = sh[32];
    __syncthreads();
    return tot;
}

// Restriction f_c[I] = sum_{a in I, ascending} p_a r_a, x_c = f_c / d_c.
// GS lanes per coarse row load its members in parallel (members GS apart);
// the group's first lane then folds the terms in member order, so the sum
// is the same FMA chain as a sequential loop.
template <typename A, int GS>
__global__ void k_restrict(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                           const double* __restrict__ pval, const A* __restrict__ rbuf, A* fc, A* xc,
                           const A* __restrict__ invdc, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    constexpr int G = 32 / GS;  // coarse rows per warp
    const int lane = threadIdx.x & 31, q = lane % GS, gbase = lane - q;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int I0 = warp * G; I0 < nc; I0 += nwarps * G) {  // warp-uniform
        const int I = I0 + lane / GS;
        const bool valid = I < nc;
        const int m0 = valid ? mptr[I] : 0, cnt = valid ? mptr[I + 1] - m0 : 0;
        const int cmax = __reduce_max_sync(FULL, cnt);
        A acc = A(0);
        for (int base = 0; base < cmax; base += GS) {
            A pa = A(0), ra = A(0);
            if (base + q < cnt) {
                const int a = midx[m0 + base + q];
                pa = (A)pval[a];
                ra = rbuf[a];
            }
#pragma unroll
            for (int j = 0; j < GS; j++) {
                const A pj = __shfl_sync(FULL, pa, gbase + j), rj = __shfl_sync(FULL, ra, gbase + j);
                if (base + j < cnt) acc = fma(pj, rj, acc);
            }
        }
        if (valid && q == 0) {
            fc[I] = acc;
            if (xc) xc[I] = acc * invdc[I];
        }
    }
}

// Prolongation as a gather over the finer level's rows: x_f[c] +=
// p_c y[agg[c]] (the same FMA per row as scattering y over the aggregates'
// members).
template <typename A>
__global__ void k_prolong(int n, const int32_t* __restrict__ agg, const double* __restrict__ pval,
                          const A* __restrict__ y, A* xf, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
        xf[c] = fma((A)pval[c], y[agg[c]], xf[c]);
}

// Coarsest level: e = A^-1 f with the dense FP64 symmetric inverse
// (row-major), then prolongation into the finer level, or (single-level
// hierarchy) z = e with the partial r.z (and z.q).
template <typename FT, typename XT>
__global__ void __launch_bounds__(kBlock) k_coarse(int n, const double* __restrict__ Ainv, const FT* __restrict__ f,
                                                    const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                                                    const double* __restrict__ pvalf, XT* xf, double* z,
                                                    const double* __restrict__ q, double* part_rz, double* part_zq,
                                                    int flexible, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[kWarpsPerBlock];
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double rz = 0.0, zq = 0.0;
    if (I < n) {
        const double* row = Ainv + (int64_t)I * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s = fma(row[j], (double)f[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (z) {
            if (lane == 0) {
                z[I] = s;
                rz = (double)f[I] * s;
                if (flexible) zq = s * q[I];
            }
        } else {  // the aggregate's members, one per lane
            const int m1 = mptr[I + 1];
            for (int m = mptr[I] + lane; m < m1; m += 32) {
                const int c = midx[m];
                xf[c] = (XT)fma(pvalf[c], s, (double)xf[c]);
            }
        }
    }
    if (z) {
        block_partial(rz, sh, part_rz + blockIdx.x);
        if (flexible) block_partial(zq, sh, part_zq + blockIdx.x);
    }
}

// ------------------------------------------------- coarsest level by CG
// Fixed-order sum over one block of 1024 threads (result on every thread).
__device__ __forceinline__ double block_sum1024(double t, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) u += red[w];
        red[32] = u;
    }
    __syncthreads();
    return red[32];
}

// Coarsest level by Jacobi-preconditioned CG from x = 0 (Sec. 5's coarse
// solver): at most maxit iterations, stop once ||r|| <= tol ||f||.  One
// block; FP64 work vectors r, z, p, q, x in global memory (4 n + n doubles);
// the result goes to e in the V-cycle precision.
template <typename A>
__global__ void __launch_bounds__(1024) k_coarse_cg(int n, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                     const double* __restrict__ kii, const A* __restrict__ f, A* e,
                                                     double* work, double tol, int maxit, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double red[33];
    double *r = work, *z = work + n, *p = work + 2 * (int64_t)n, *q = work + 3 * (int64_t)n,
           *x = work + 4 * (int64_t)n;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwp = blockDim.x >> 5;
    double ff = 0.0, rz = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double fi = (double)f[i], zi = fi / kii[i];
        x[i] = 0.0;
        r[i] = fi;
        z[i] = zi;
        p[i] = zi;
        ff = fma(fi, fi, ff);
        rz = fma(fi, zi, rz);
    }
    ff = block_sum1024(ff, red);
    double rho = block_sum1024(rz, red);
    double rr = ff;
    const double stop = tol * sqrt(ff);
    for (int it = 0; it < maxit && sqrt(rr) > stop; it++) {
        for (int i = wid; i < n; i += nwp) {  // q = K p, a warp per row
            double acc = 0.0;
            for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) acc = fma(v[k], p[ci[k]], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
            if (lane == 0) q[i] = acc;
        }
        __syncthreads();
        double t = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) t = fma(p[i], q[i], t);
        const double pq = block_sum1024(t, red);
        if (!(pq > 0.0)) break;
        const double alpha = rho / pq;
        double t1 = 0.0, t2 = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            x[i] = fma(alpha, p[i], x[i]);
            const double ri = fma(-alpha, q[i], r[i]);
            const double zi = ri / kii[i];
            r[i] = ri;
            z[i] = zi;
            t1 = fma(ri, zi, t1);
            t2 = fma(ri, ri, t2);
        }
        const double rho1 = block_sum1024(t1, red);
        rr = block_sum1024(t2, red);
        const double beta = rho1 / rho;
        rho = rho1;
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = fma(beta, p[i], z[i]);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) e[i] = (A)x[i];
}

// ------------------------------------------- Chebyshev smoothing (4th kind)
// 4th-kind Chebyshev acceleration of l1-Jacobi with rho(D^-1 K) <= 1 (the l1
// diagonal's bound): d_0 = (4/3) D^-1 r_0; r_i = r_{i-1} - K d_{i-1},
// d_i = a_i d_{i-1} + b_i D^-1 r_i, a_i = (2i-1)/(2i+3), b_i = (8i+4)/(2i+3);
// x advances by each d.  The x update of a step is deferred to the next
// kernel, whose matrix pass reads d, not x (x stays row-local).

// pre-smoothing from x = 0: x = 0, d = c0 D^-1 f
template <typename A, typename FT>
__global__ void k_cheb_start(int n, const FT* __restrict__ f, const A* __restrict__ invd, A c0, A* x, A* d,
                             const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = A(0);
        d[i] = c0 * invd[i] * (A)f[i];
    }
}

// x += dprev; r = rprev - K dprev; dnew = a dprev + b D^-1 r (r may be rprev)
template <int RPW, typename A, typename M, typename FT>
__global__ void __launch_bounds__(kBlock) k_cheb_step(int n, M mat, const A* __restrict__ dprev, const FT* rprev,
                                                       A* r, const A* __restrict__ invd, A a, A b, A* dnew, A* x,
                                                       const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, dprev, row0, n, lane, tiles[wid]);
    if (owner) {
        const A ri = (A)rprev[myrow] - s;
        const A dp = dprev[myrow];
        r[myrow] = ri;
        dnew[myrow] = fma(b, invd[myrow] * ri, a * dp);
        x[myrow] += dp;
    }
}

// end of pre-smoothing: x += dprev; r = rprev - K dprev (the residual)
template <int RPW, typename A, typename M, typename FT>
__global__ void __launch_bounds__(kBlock) k_cheb_resid(int n, M mat, const A* __restrict__ dprev, const FT* rprev,
                                                        A* r, A* x, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, dprev, row0, n, lane, tiles[wid]);
    if (owner) {
        r[myrow] = (A)rprev[myrow] - s;
        x[myrow] += dprev[myrow];
    }
}

// start of post-smoothing: r = f - K x, d = c0 D^-1 r (x unchanged)
template <int RPW, typename A, typename M, typename FT>
__global__ void __launch_bounds__(kBlock) k_cheb_post0(int n, M mat, const FT* __restrict__ f,
                                                        const A* __restrict__ x, const A* __restrict__ invd, A c0,
                                                        A* r, A* d, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, x, row0, n, lane, tiles[wid]);
    if (owner) {
        const A ri = (A)f[myrow] - s;
        r[myrow] = ri;
        d[myrow] = c0 * invd[myrow] * ri;
    }
}

// x += d
template <typename A>
__global__ void k_cheb_add(int n, const A* __restrict__ d, A* x, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] += d[i];
}

// level 0 after post-smoothing: z = x + d (FP64); block partials r.z and
// (flexible) z.q over a grid-stride loop
template <typename A>
__global__ void __launch_bounds__(kBlock) k_cheb_z(int n, const A* __restrict__ x, const A* __restrict__ d,
                                                    const double* __restrict__ r, double* z,
                                                    const double* __restrict__ q, double* part_rz, double* part_zq,
                                                    int flexible, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[kWarpsPerBlock];
    double rz = 0.0, zq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double zi = (double)(x[i] + d[i]);
        z[i] = zi;
        rz = fma(r[i], zi, rz);
        if (flexible) zq = fma(zi, q[i], zq);
    }
    block_partial(rz, sh, part_rz + blockIdx.x);
    if (flexible) block_partial(zq, sh, part_zq + blockIdx.x);
}

// ------------------------------------------------------------ CG scalars
__global__ void k_scal_init(const double* part_rr, const double* part_ff, int nb, double rtol, int itmax,
                            int repl_every, double* hist, SolveState* st) {
    pdl_entry();
    // every field a later kernel reads is (re)set here
    __shared__ double sh[33];
    const double rr = sum_partials(part_rr, nb, sh);
    const double ff = sum_partials(part_ff, nb, sh);
    if (threadIdx.x == 0) {
        const double nF = sqrt(ff), nr = sqrt(rr);
        st->nF = nF;
        st->tol = rtol * nF;
        st->nr = nr;
        st->iters = 0;
        st->itmax = itmax;
        st->replace_now = 0;
        st->repl_every = repl_every;
        st->status = AMG_OK;
        st->done = 0;
        if (hist) hist[0] = nF > 0.0 ? nr / nF : 0.0;
        if (isnan(nr) || isnan(nF) || isinf(nr) || isinf(nF)) {
            st->status = AMG_ERR_NAN;
            st->done = 1;
        } else if (!(nF > 0.0) || nr <= st->tol) {
            st->done = 1;
        } else if (itmax <= 0) {
            st->status = AMG_ERR_NOT_CONVERGED;
            st->done = 1;
        }
    }
}

__global__ void k_scal_alpha(const double* part_pq, const double* part_pr, int nb, int flexible, SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[33];
    const double pq = sum_partials(part_pq, nb, sh);
    const double num = flexible ? sum_partials(part_pr, nb, sh) : st->rho;
    if (threadIdx.x == 0) {
        st->pq = pq;
        if (!(pq > 0.0)) {
            st->status = (isnan(pq) || isnan(num)) ? AMG_ERR_NAN : AMG_ERR_BREAKDOWN;
            st->done = 1;
        } else {
            st->alpha = num / pq;
        }
    }
}

// Convergence test on the recursive residual.  mixed = 1: convergence is
// only declared on an FP64 true residual, so a replacement is requested
// instead (also every repl_every iterations).
__global__ void k_scal_conv(const double* part_rr, int nb, double* hist, int hist_cap, int mixed, SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[33];
    const double rr = sum_partials(part_rr, nb, sh);
    if (threadIdx.x == 0) {
        const double nr = sqrt(rr);
        const int it = st->iters + 1;
        st->iters = it;
        st->nr = nr;
        if (hist && it < hist_cap) hist[it] = nr / st->nF;
        if (isnan(nr) || isinf(nr)) {
            st->status = AMG_ERR_NAN;
            st->done = 1;
        } else if (mixed && (nr <= st->tol || it >= st->itmax || (st->repl_every > 0 && it % st->repl_every == 0))) {
            st->replace_now = 1;
        } else if (nr <= st->tol) {
            st->done = 1;
        } else if (it >= st->itmax) {
            st->status = AMG_ERR_NOT_CONVERGED;
            st->done = 1;
        }
    }
}

// After a residual replacement: test the FP64 true residual.
__global__ void k_scal_replaced(const double* part_rr, int nb, double* hist, int hist_cap, SolveState* st) {
    pdl_entry();
    if (st->done || !st->replace_now) return;
    __shared__ double sh[33];
    const double rr = sum_partials(part_rr, nb, sh);
    if (threadIdx.x == 0) {
        const double nr = sqrt(rr);
        const int it = st->iters;
        st->nr = nr;
        st->replace_now = 0;
        if (hist && it < hist_cap) hist[it] = nr / st->nF;
        if (isnan(nr) || isinf(nr)) {
            st->status = AMG_ERR_NAN;
            st->done = 1;
        } else if (nr <= st->tol) {
            st->done = 1;
        } else if (it >= st->itmax) {
            st->status = AMG_ERR_NOT_CONVERGED;
            st->done = 1;
        }
    }
}

// rho = r.z; beta = rho_new / rho (PCG) or -z.q / p.q (flexible); first: beta = 0.
__global__ void k_scal_beta(const double* part_rz, const double* part_zq, int nb, int flexible, int first,
                            SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[33];
    const double rz = sum_partials(part_rz, nb, sh);
    const double zq = (flexible && !first) ? sum_partials(part_zq, nb, sh) : 0.0;
    if (threadIdx.x == 0) {
        if (isnan(rz) || isnan(zq)) {
            st->status = AMG_ERR_NAN;
            st->done = 1;
            return;
        }
        if (first) st->beta = 0.0;
        else st->beta = flexible ? -zq / st->pq : rz / st->rho;
        st->rho = rz;
    }
}

// x += alpha p, r -= alpha q, x0 = r / d (in X0), partial ||r||^2.
template <typename X0>
__global__ void k_update(int n, double* x, double* r, const double* __restrict__ p, const double* __restrict__ q,
                         const X0* __restrict__ invd, X0* x0, double* part_rr, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    __shared__ double sh[kWarpsPerBlock];
    const double alpha = st->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        if (x0) x0[i] = (X0)ri * invd[i];
        rr = fma(ri, ri, rr);
    }
    block_partial(rr, sh, part_rr + blockIdx.x);
}

// p = z + beta p (first direction: p = z); p32 = FP32 copy (mixed).
__global__ void k_pupdate(int n, double* p, const double* __restrict__ z, float* p32, int first, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    const double beta = st->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double pi = first ? z[i] : fma(beta, p[i], z[i]);
        p[i] = pi;
        if (p32) p32[i] = __double2float_rn(pi);
    }
}

template <typename X0>
__global__ void k_scale(int n, const double* __restrict__ a, const X0* __restrict__ b, X0* out) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (X0)a[i] * b[i];
}

__global__ void k_sqrt_sum(const double* part, int nb, double* out) {
    pdl_entry();
    __shared__ double sh[33];
    const double s = sum_partials(part, nb, sh);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// ----------------------------------------------------------------- dispatch
template <typename F>
inline void with_rpw(int rpw, F&& f) {
    if (rpw == 8) f(std::integral_constant<int, 8>{});
    else f(std::integral_constant<int, 1>{});
}

}  // namespace

int rows_per_warp(int n, int num_sms) {
    // 8-row groups once there are enough of them to fill the GPU several times
    return ((int64_t)n >= (int64_t)num_sms * kWarpsPerBlock * 8 * 4) ? 8 : 1;
}

int row_blocks(int n, int rpw) {
    return (int)(((int64_t)n + (int64_t)rpw * kWarpsPerBlock - 1) / ((int64_t)rpw * kWarpsPerBlock));
}

int vec_blocks(int n, int num_sms) {
    int64_t b = ((int64_t)n + kBlock - 1) / kBlock;
    const int cap = num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

// blocks of the restriction: 4 lanes per coarse row
static int restrict_blocks(int nc, int num_sms) {
    return vec_blocks((int)std::min<int64_t>((int64_t)nc * 4, INT32_MAX), num_sms);
}

cudaError_t launch_spmv(const DevCSR& A, const double* x, double* y, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rpw = rows_per_warp(A.n, sms);
    const int nb = row_blocks(A.n, rpw);
    if (A.n == 0) return cudaSuccess;
    with_rpw(rpw, [&](auto R) {
        launch_pdl(k_spmv<decltype(R)::value, CsrM<double>>, nb, kBlock, 0, s, A.n, CsrM<double>{A.rowptr, A.col, A.val}, x, y);
    });
    return cudaGetLastError();
}

// Event-record node around a timed fine-level kernel (only while the
// iteration graph is being captured with profiling on).
static void prof_mark(amg_hierarchy* h, int k, int side, cudaStream_t s) {
    if (h->prof && h->prof_slot >= 0)
        cudaEventRecordWithFlags(h->prof_ev[h->prof_slot][k][side], s, cudaEventRecordExternal);
}

// Partial-sum slots inside h->partials (h->npart doubles each).
static double* slot(amg_hierarchy* h, int k) { return h->partials + (int64_t)k * h->npart; }
enum { S_RR = 0, S_FF, S_PQ, S_PR, S_RZ, S_ZQ, S_OUT, S_RR2, S_COUNT };

// ---------------------------------------------------------- per-mode views
// Matrix view of level L with values v: run-encoded columns when the level
// has them, plain CSR otherwise.
template <typename V, typename Fn>
static void with_mat(const Level& L, const V* v, Fn&& fn) {
    if (L.run_ptr) fn(RunM<V>{L.A.rowptr, L.run_ptr, L.run_len, L.run_start, v});
    else fn(CsrM<V>{L.A.rowptr, L.A.col, v});
}

// Vectors and values of a level in the V-cycle precision A.
template <typename A>
struct View;

template <>
struct View<double> {
    static double* f(Level& L) { return L.f; }
    static double* x(Level& L) { return L.x; }
    static double* t(Level& L) { return L.t; }
    static const double* invd(Level& L) { return L.invd; }
    template <typename Fn>
    static void vals(Level& L, int, Fn&& fn) { with_mat(L, static_cast<const double*>(L.A.val), fn); }
};

template <>
struct View<float> {
    static float* f(Level& L) { return L.f32; }
    static float* x(Level& L) { return L.x32; }
    static float* t(Level& L) { return L.t32; }
    static const float* invd(Level& L) { return L.invd32; }
    template <typename Fn>
    static void vals(Level& L, int l, Fn&& fn) {
        if (l == 0 && L.val16) with_mat(L, static_cast<const __nv_bfloat16*>(L.val16), fn);
        else with_mat(L, static_cast<const float*>(L.val32), fn);
    }
};

template <typename T>
using vtype = std::remove_cv_t<std::remove_pointer_t<T>>;

// Coarsest level of a hierarchy with at least two levels: e = A^-1 f
// (dense inverse, or CG when coarse_solver = 1), prolongated into x of
// level L - 2 (tentative P fused with the dense solve, or a gather).
template <typename A>
static void coarsest_solve(amg_hierarchy* h, A* xF, cudaStream_t s) {
    using Vw = View<A>;
    const int L = h->nlev;
    Level& F = h->lev[L - 2];
    Level& C = h->lev[L - 1];
    const SolveState* st = h->st;
    if (h->o.coarse_solver == 1) {
        A* e = Vw::x(C);
        launch_pdl(k_coarse_cg<A>, 1, 1024, 0, s, C.A.n, C.A.rowptr, C.A.col, C.A.val, C.kii,
                   static_cast<const A*>(Vw::f(C)), e, h->ccg, h->o.coarse_tol, h->o.coarse_maxit, st);
        if (F.smoothed)
            sp_prolong<A>(F, static_cast<const A*>(e), xF, st, s);
        else
            launch_pdl(k_prolong<A>, vec_blocks(F.A.n, h->num_sms), kBlock, 0, s, F.A.n, F.agg, F.pval,
                       static_cast<const A*>(e), xF, st);
    } else if (F.smoothed) {
        sp_coarse<A>(C.A.n, h->Ainv, Vw::f(C), Vw::x(C), st, s);
        sp_prolong<A>(F, Vw::x(C), xF, st, s);
    } else {
        launch_pdl(k_coarse<A, A>, row_blocks(C.A.n, 1), kBlock, 0, s, C.A.n, h->Ainv, Vw::f(C), F.mem_ptr,
                   F.mem_idx, F.pval, xF, nullptr, nullptr, nullptr, nullptr, 0, st);
    }
}

// V-cycle on r (= f_0); the pre-smoothed level-0 iterate is already in x_0.
// Writes z (FP64) and the partial sums of r.z (and z.q).
template <typename A>
static cudaError_t vcycle_impl(amg_hierarchy* h, cudaStream_t s) {
    using Vw = View<A>;
    const int L = h->nlev;
    const int sms = h->num_sms;
    const int flex = h->o.flexible;
    const SolveState* st = h->st;
    if (L == 1) {
        launch_pdl(k_coarse<double, A>, row_blocks(h->ndense, 1), kBlock, 0, s,
            h->ndense, h->Ainv, h->r, nullptr, nullptr, nullptr, nullptr, h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ),
            flex, st);
        return cudaGetLastError();
    }
    A* xcur[AMG_MAX_LEVELS];
    A* xalt[AMG_MAX_LEVELS];
    for (int l = 0; l < L; l++) {
        xcur[l] = Vw::x(h->lev[l]);
        xalt[l] = Vw::t(h->lev[l]);
    }
    // down
    for (int l = 0; l < L - 1; l++) {
        Level& F = h->lev[l];
        Level& C = h->lev[l + 1];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw);
        Vw::vals(F, l, [&](auto mat) {
            using M = decltype(mat);
            auto sweep_and_resid = [&](auto fp) {
                using FT = vtype<decltype(fp)>;
                for (int sw = 1; sw < h->o.nu_pre; sw++) {
                    A* xo = xcur[l];
                    A* xn = xalt[l];
                    with_rpw(rpw, [&](auto R) {
                        launch_pdl(k_sweep<decltype(R)::value, A, M, FT>, nb, kBlock, 0, s,
                            n, mat, fp, xo, Vw::invd(F), xn, st);
                    });
                    xcur[l] = xn;
                    xalt[l] = xo;
                }
                A* rb = xalt[l];  // free buffer of this level holds the residual
                const A* xc = xcur[l];
                if (l == 0) prof_mark(h, 1, 0, s);
                if constexpr (std::is_same_v<A, double>) {
                    if (l == 0 && h->sell64) {
                        sell64_resid(h, h->r, xc, rb, s);
                        prof_mark(h, 1, 1, s);
                        return;
                    }
                }
                if constexpr (std::is_same_v<A, float>) {
                    if (l == 0 && h->stream) {
                        launch_stream_resid(h, h->r, xc, rb, s);
                        prof_mark(h, 1, 1, s);
                        return;
                    }
                    if (l == 1 && h->sell[1].on) {
                        sell_resid1(h, static_cast<const float*>(Vw::f(F)), xc, rb, s);
                        return;
                    }
                }
                with_rpw(rpw, [&](auto R) {
                    launch_pdl(k_resid<decltype(R)::value, A, M, FT, A>, nb, kBlock, 0, s, n, mat, fp, xc, rb, st);
                });
                if (l == 0) prof_mark(h, 1, 1, s);
            };
            if (l == 0) sweep_and_resid(static_cast<const double*>(h->r));
            else sweep_and_resid(static_cast<const A*>(Vw::f(F)));
        });
        const bool coarsest = (l + 1 == L - 1);
        if (F.smoothed)  // f_c = P_bar^T r
            sp_restrict<A>(F, C, xalt[l], Vw::f(C), coarsest ? nullptr : xcur[l + 1], Vw::invd(C), st, s);
        else
            launch_pdl(k_restrict<A, 4>, restrict_blocks(C.A.n, sms), kBlock, 0, s, C.A.n, F.mem_ptr, F.mem_idx,
                       F.pval, xalt[l], Vw::f(C), coarsest ? nullptr : xcur[l + 1], Vw::invd(C), st);
    }
    // coarsest
    coarsest_solve<A>(h, xcur[L - 2], s);
    // up
    for (int l = L - 2; l >= 0; l--) {
        Level& F = h->lev[l];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw);
        Vw::vals(F, l, [&](auto mat) {
            using M = decltype(mat);
            auto sweeps = [&](auto fp) {
                using FT = vtype<decltype(fp)>;
                for (int sw = 1; sw < h->o.nu_post; sw++) {
                    A* xo = xcur[l];
                    A* xn = xalt[l];
                    with_rpw(rpw, [&](auto R) {
                        launch_pdl(k_sweep<decltype(R)::value, A, M, FT>, nb, kBlock, 0, s,
                            n, mat, fp, xo, Vw::invd(F), xn, st);
                    });
                    xcur[l] = xn;
                    xalt[l] = xo;
                }
            };
            if (l == 0) sweeps(static_cast<const double*>(h->r));
            else sweeps(static_cast<const A*>(Vw::f(F)));
            const A* xc = xcur[l];
            if (l == 0) {
                prof_mark(h, 2, 0, s);
                if constexpr (std::is_same_v<A, double>) {
                    if (h->sell64) {
                        sell64_up0(h, h->r, xc, Vw::invd(F), h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ), flex, s);
                        prof_mark(h, 2, 1, s);
                        return;
                    }
                }
                if constexpr (std::is_same_v<A, float>) {
                    if (h->stream) {
                        launch_stream_up0(h, h->r, xc, Vw::invd(F), h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ), flex,
                                          s);
                        prof_mark(h, 2, 1, s);
                        return;
                    }
                }
                with_rpw(rpw, [&](auto R) {
                    launch_pdl(k_up0<decltype(R)::value, A, M>, nb, kBlock, 0, s,
                        n, mat, h->r, xc, Vw::invd(F), h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ), flex, st);
                });
                prof_mark(h, 2, 1, s);
            } else {
                Level& G = h->lev[l - 1];
                A* xf = xcur[l - 1];
                if constexpr (std::is_same_v<A, float>) {
                    if (l == 1 && h->sell[1].on) {  // y = smoothed level 1, then the gather into level 0
                        A* y = xalt[1];
                        sell_upy1(h, static_cast<const float*>(Vw::f(F)), xc, Vw::invd(F), y, s);
                        if (G.smoothed)
                            sp_prolong<A>(G, y, xf, st, s);
                        else
                            launch_pdl(k_prolong<A>, vec_blocks(G.A.n, sms), kBlock, 0, s, G.A.n, G.agg, G.pval, y,
                                       xf, st);
                        return;
                    }
                }
                if (G.smoothed) {  // y = x + (f - K x) / d, then x_f += P_bar y
                    A* y = xalt[l];
                    with_rpw(rpw, [&](auto R) {
                        launch_pdl(k_sweep<decltype(R)::value, A, M, A>, nb, kBlock, 0, s, n, mat,
                                   static_cast<const A*>(Vw::f(F)), xc, Vw::invd(F), y, st);
                    });
                    sp_prolong<A>(G, y, xf, st, s);
                    return;
                }
                with_rpw(rpw, [&](auto R) {
                    launch_pdl(k_up<decltype(R)::value, A, M>, nb, kBlock, 0, s,
                        n, mat, Vw::f(F), xc, Vw::invd(F), G.mem_ptr, G.mem_idx, G.pval, xf, st);
                });
            }
        });
    }
    return cudaGetLastError();
}

// V-cycle with the Chebyshev smoother of degree cheb_degree on every level
// (plain row-group matrix passes on every level, tentative or smoothed
// prolongators); the coarsest solve and the CG interface as vcycle_impl.
template <typename A>
static cudaError_t vcycle_cheb(amg_hierarchy* h, cudaStream_t s) {
    using Vw = View<A>;
    const int L = h->nlev;
    const int sms = h->num_sms;
    const int k = h->o.cheb_degree;
    const int flex = h->o.flexible;
    const SolveState* st = h->st;
    if (L == 1) {
        launch_pdl(k_coarse<double, A>, row_blocks(h->ndense, 1), kBlock, 0, s,
            h->ndense, h->Ainv, h->r, nullptr, nullptr, nullptr, nullptr, h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ),
            flex, st);
        return cudaGetLastError();
    }
    const A c0 = A(4.0 / 3.0);
    auto coef_a = [](int i) { return A((double)(2 * i - 1) / (double)(2 * i + 3)); };
    auto coef_b = [](int i) { return A((double)(8 * i + 4) / (double)(2 * i + 3)); };
    // down: pre-smoothing from zero, residual, restriction
    for (int l = 0; l < L - 1; l++) {
        Level& F = h->lev[l];
        Level& C = h->lev[l + 1];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw), nv = vec_blocks(n, sms);
        A* x = Vw::x(F);
        A* r = Vw::t(F);
        A* d0 = static_cast<A*>(F.cd[0]);
        A* d1 = static_cast<A*>(F.cd[1]);
        auto run = [&](auto fp) {
            using FT = vtype<decltype(fp)>;
            launch_pdl(k_cheb_start<A, FT>, nv, kBlock, 0, s, n, fp, Vw::invd(F), c0, x, d0, st);
            Vw::vals(F, l, [&](auto mat) {
                using M = decltype(mat);
                A* dp = d0;
                A* dn = d1;
                for (int i = 1; i < k; i++) {
                    with_rpw(rpw, [&](auto R) {
                        if (i == 1)
                            launch_pdl(k_cheb_step<decltype(R)::value, A, M, FT>, nb, kBlock, 0, s, n, mat,
                                       static_cast<const A*>(dp), fp, r, Vw::invd(F), coef_a(i), coef_b(i), dn, x,
                                       st);
                        else
                            launch_pdl(k_cheb_step<decltype(R)::value, A, M, A>, nb, kBlock, 0, s, n, mat,
                                       static_cast<const A*>(dp), static_cast<const A*>(r), r, Vw::invd(F),
                                       coef_a(i), coef_b(i), dn, x, st);
                    });
                    std::swap(dp, dn);
                }
                with_rpw(rpw, [&](auto R) {
                    if (k == 1)
                        launch_pdl(k_cheb_resid<decltype(R)::value, A, M, FT>, nb, kBlock, 0, s, n, mat,
                                   static_cast<const A*>(dp), fp, r, x, st);
                    else
                        launch_pdl(k_cheb_resid<decltype(R)::value, A, M, A>, nb, kBlock, 0, s, n, mat,
                                   static_cast<const A*>(dp), static_cast<const A*>(r), r, x, st);
                });
            });
        };
        bool sliced = false;
        if constexpr (std::is_same_v<A, double>) {
            if (l == 0 && h->sell64) {  // the finest level's matrix passes on its sliced FP64 copy
                const double* f0 = h->r;
                launch_pdl(k_cheb_start<double, double>, nv, kBlock, 0, s, n, f0, Vw::invd(F), c0, x, d0, st);
                A* dp = d0;
                A* dn = d1;
                for (int i = 1; i < k; i++) {
                    sell64_cheb_step(h, dp, i == 1 ? f0 : r, r, Vw::invd(F), coef_a(i), coef_b(i), dn, x, s);
                    std::swap(dp, dn);
                }
                sell64_cheb_resid(h, dp, k == 1 ? f0 : r, r, x, s);
                sliced = true;
            }
        }
        if (!sliced) {
            if (l == 0) run(static_cast<const double*>(h->r));
            else run(static_cast<const A*>(Vw::f(F)));
        }
        if (F.smoothed)
            sp_restrict<A>(F, C, r, Vw::f(C), static_cast<A*>(nullptr), Vw::invd(C), st, s);
        else
            launch_pdl(k_restrict<A, 4>, restrict_blocks(C.A.n, sms), kBlock, 0, s, C.A.n, F.mem_ptr, F.mem_idx,
                       F.pval, static_cast<const A*>(r), Vw::f(C), static_cast<A*>(nullptr), Vw::invd(C), st);
    }
    // coarsest, prolongated into level L-2
    coarsest_solve<A>(h, Vw::x(h->lev[L - 2]), s);
    // up: post-smoothing from the corrected x, then prolongation to the finer level
    for (int l = L - 2; l >= 0; l--) {
        Level& F = h->lev[l];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw), nv = vec_blocks(n, sms);
        A* x = Vw::x(F);
        A* r = Vw::t(F);
        A* d0 = static_cast<A*>(F.cd[0]);
        A* d1 = static_cast<A*>(F.cd[1]);
        A* dlast = d0;
        auto run = [&](auto fp) {
            using FT = vtype<decltype(fp)>;
            Vw::vals(F, l, [&](auto mat) {
                using M = decltype(mat);
                with_rpw(rpw, [&](auto R) {
                    launch_pdl(k_cheb_post0<decltype(R)::value, A, M, FT>, nb, kBlock, 0, s, n, mat, fp,
                               static_cast<const A*>(x), Vw::invd(F), c0, r, d0, st);
                });
                A* dp = d0;
                A* dn = d1;
                for (int i = 1; i < k; i++) {
                    with_rpw(rpw, [&](auto R) {
                        launch_pdl(k_cheb_step<decltype(R)::value, A, M, A>, nb, kBlock, 0, s, n, mat,
                                   static_cast<const A*>(dp), static_cast<const A*>(r), r, Vw::invd(F), coef_a(i),
                                   coef_b(i), dn, x, st);
                    });
                    std::swap(dp, dn);
                }
                dlast = dp;
            });
        };
        bool sliced = false;
        if constexpr (std::is_same_v<A, double>) {
            if (l == 0 && h->sell64) {  // the finest level's matrix passes on its sliced FP64 copy
                sell64_cheb_post0(h, x, h->r, Vw::invd(F), c0, r, d0, s);
                A* dp = d0;
                A* dn = d1;
                for (int i = 1; i < k; i++) {
                    sell64_cheb_step(h, dp, r, r, Vw::invd(F), coef_a(i), coef_b(i), dn, x, s);
                    std::swap(dp, dn);
                }
                dlast = dp;
                sliced = true;
            }
        }
        if (!sliced) {
            if (l == 0) run(static_cast<const double*>(h->r));
            else run(static_cast<const A*>(Vw::f(F)));
        }
        if (l == 0) {
            const int nbz0 = (h->stream || h->sell64) ? h->stream_blocks : row_blocks(n, rows_per_warp(n, sms));
            launch_pdl(k_cheb_z<A>, nbz0, kBlock, 0, s, n, static_cast<const A*>(x), static_cast<const A*>(dlast),
                       static_cast<const double*>(h->r), h->z, static_cast<const double*>(h->q), slot(h, S_RZ),
                       slot(h, S_ZQ), flex, st);
        } else {
            launch_pdl(k_cheb_add<A>, nv, kBlock, 0, s, n, static_cast<const A*>(dlast), x, st);
            Level& G = h->lev[l - 1];
            if (G.smoothed)
                sp_prolong<A>(G, static_cast<const A*>(x), Vw::x(G), st, s);
            else
                launch_pdl(k_prolong<A>, vec_blocks(G.A.n, sms), kBlock, 0, s, G.A.n, G.agg, G.pval,
                           static_cast<const A*>(x), Vw::x(G), st);
        }
    }
    return cudaGetLastError();
}

cudaError_t enqueue_vcycle(amg_hierarchy* h, cudaStream_t s) {
    if (h->o.cheb_degree > 0) return h->mixed ? vcycle_cheb<float>(h, s) : vcycle_cheb<double>(h, s);
    return h->mixed ? vcycle_impl<float>(h, s) : vcycle_impl<double>(h, s);
}

// blocks of the level-0 row kernels, of the vector kernels, and of the
// kernel that produces z (level-0 up sweep or single-level coarse solve)
static int nb0(amg_hierarchy* h) { return row_blocks(h->lev[0].A.n, rows_per_warp(h->lev[0].A.n, h->num_sms)); }
static int nbv(amg_hierarchy* h) { return vec_blocks(h->lev[0].A.n, h->num_sms); }
// blocks (= partial sums) of the FP64 residual kernel
static int nb_res(amg_hierarchy* h) {
    const int b = nb0(h), cap = h->num_sms * 4;
    return b < cap ? b : cap;
}
// partial sums written by the level-0 q = K p and up-sweep kernels
static int nb_fine(amg_hierarchy* h) { return (h->stream || h->sell64) ? h->stream_blocks : nb0(h); }
static int nbz(amg_hierarchy* h) { return h->nlev > 1 ? nb_fine(h) : row_blocks(h->ndense, 1); }

size_t partial_slot_size(int n0, int num_sms) {
    const int a = row_blocks(n0, rows_per_warp(n0, num_sms));
    const int b = vec_blocks(n0, num_sms);
    const int m = a > b ? a : b;
    return (size_t)((m > num_sms ? m : num_sms) + 2);
}

size_t partial_slot_count() { return S_COUNT; }

// FP64 residual r = F - K x (K the FP64 finest matrix) with x0 = r / d for
// the V-cycle in its precision; partials into rr_slot (and ||F||^2 if ff).
static cudaError_t launch_residual(amg_hierarchy* h, double* r, bool want_x0, int rr_slot, bool ff,
                                   const SolveState* gate, cudaStream_t s) {
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int rpw = rows_per_warp(n, h->num_sms), nb = nb_res(h);
    const bool x0 = want_x0 && h->nlev > 1;
    double* pff = ff ? slot(h, S_FF) : nullptr;
    with_rpw(rpw, [&](auto R) {
        constexpr int RPW = decltype(R)::value;
        with_mat(L0, static_cast<const double*>(L0.A.val), [&](auto mat) {
            using M = decltype(mat);
            if (h->mixed)
                launch_pdl(k_residual0<RPW, float, M>, nb, kBlock, 0, s, n, mat, h->x, h->F, L0.invd32, r,
                                                                           x0 ? L0.x32 : nullptr, slot(h, rr_slot),
                                                                           pff, gate);
            else
                launch_pdl(k_residual0<RPW, double, M>, nb, kBlock, 0, s, n, mat, h->x, h->F, L0.invd, r,
                                                                            x0 ? L0.x : nullptr, slot(h, rr_slot),
                                                                            pff, gate);
        });
    });
    return cudaGetLastError();
}

static void launch_pupdate(amg_hierarchy* h, int first, cudaStream_t s) {
    launch_pdl(k_pupdate, nbv(h), kBlock, 0, s, h->lev[0].A.n, h->p, h->z, h->mixed ? h->p32 : nullptr, first,
                                                  h->st);
}

// r = F - K x, ||F||, ||r||, first V-cycle, p = z, rho = r.z.
cudaError_t enqueue_pcg_start(amg_hierarchy* h, cudaStream_t s) {
    AMG_TRY(launch_residual(h, h->r, true, S_RR, true, nullptr, s));
    launch_pdl(k_scal_init, 1, 256, 0, s, slot(h, S_RR), slot(h, S_FF), nb_res(h), h->rtol, h->itmax,
                                            h->mixed ? h->o.resid_replace_every : 0, h->hist, h->st);
    AMG_TRY(cudaGetLastError());
    AMG_TRY(enqueue_vcycle(h, s));
    launch_pdl(k_scal_beta, 1, 256, 0, s, slot(h, S_RZ), slot(h, S_ZQ), nbz(h), h->o.flexible, 1, h->st);
    launch_pupdate(h, 1, s);
    return cudaGetLastError();
}

cudaError_t enqueue_pcg_iteration(amg_hierarchy* h, cudaStream_t s) {
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int flex = h->o.flexible;
    const int rpw = rows_per_warp(n, h->num_sms), nb = row_blocks(n, rpw);
    prof_mark(h, 0, 0, s);
    with_rpw(rpw, [&](auto R) {
        constexpr int RPW = decltype(R)::value;
        if (h->mixed && h->stream)
            launch_stream_spmv_pq(h, h->p32, h->p, h->r, h->q, slot(h, S_PQ), slot(h, S_PR), flex, s);
        else if (h->sell64)
            sell64_spmv_pq(h, h->p, h->r, h->q, slot(h, S_PQ), slot(h, S_PR), flex, s);
        else if (h->mixed)
            with_mat(L0, static_cast<const float*>(L0.val32), [&](auto mat) {
                launch_pdl(k_spmv_pq<RPW, float, decltype(mat), float>, nb, kBlock, 0, s,
                    n, mat, h->p32, h->p, h->r, h->q, slot(h, S_PQ), slot(h, S_PR), flex, h->st);
            });
        else
            with_mat(L0, static_cast<const double*>(L0.A.val), [&](auto mat) {
                launch_pdl(k_spmv_pq<RPW, double, decltype(mat), double>, nb, kBlock, 0, s,
                    n, mat, h->p, h->p, h->r, h->q, slot(h, S_PQ), slot(h, S_PR), flex, h->st);
            });
    });
    prof_mark(h, 0, 1, s);
    launch_pdl(k_scal_alpha, 1, 256, 0, s, slot(h, S_PQ), slot(h, S_PR), nb_fine(h), flex, h->st);
    const bool x0 = h->nlev > 1;
    if (h->mixed)
        launch_pdl(k_update<float>, nbv(h), kBlock, 0, s, n, h->x, h->r, h->p, h->q, L0.invd32, x0 ? L0.x32 : nullptr,
                                                            slot(h, S_RR), h->st);
    else
        launch_pdl(k_update<double>, nbv(h), kBlock, 0, s, n, h->x, h->r, h->p, h->q, L0.invd, x0 ? L0.x : nullptr,
                                                             slot(h, S_RR), h->st);
    launch_pdl(k_scal_conv, 1, 256, 0, s, slot(h, S_RR), nbv(h), h->hist, h->hist_cap, h->mixed, h->st);
    if (h->mixed) {  // FP64 true-residual replacement, when due
        AMG_TRY(launch_residual(h, h->r, true, S_RR2, false, h->st, s));
        launch_pdl(k_scal_replaced, 1, 256, 0, s, slot(h, S_RR2), nb_res(h), h->hist, h->hist_cap, h->st);
    }
    AMG_TRY(cudaGetLastError());
    AMG_TRY(enqueue_vcycle(h, s));
    launch_pdl(k_scal_beta, 1, 256, 0, s, slot(h, S_RZ), slot(h, S_ZQ), nbz(h), flex, 0, h->st);
    launch_pupdate(h, 0, s);
    return cudaGetLastError();
}

// The row-group q = K p pass of the finest level (the layout used when no
// sliced or staged copy is in use), for the setup's autotuning.
cudaError_t launch_rowgroup_pq(amg_hierarchy* h, cudaStream_t s) {
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int rpw = rows_per_warp(n, h->num_sms), nb = row_blocks(n, rpw);
    with_rpw(rpw, [&](auto R) {
        constexpr int RPW = decltype(R)::value;
        if (h->mixed)
            with_mat(L0, static_cast<const float*>(L0.val32), [&](auto mat) {
                launch_pdl(k_spmv_pq<RPW, float, decltype(mat), float>, nb, kBlock, 0, s, n, mat, h->p32, h->p,
                           h->r, h->q, slot(h, S_PQ), slot(h, S_PR), 0, h->st);
            });
        else
            with_mat(L0, static_cast<const double*>(L0.A.val), [&](auto mat) {
                launch_pdl(k_spmv_pq<RPW, double, decltype(mat), double>, nb, kBlock, 0, s, n, mat, h->p, h->p,
                           h->r, h->q, slot(h, S_PQ), slot(h, S_PR), 0, h->st);
            });
    });
    return cudaGetLastError();
}

// ||F - K x|| and ||F|| into slot(S_OUT)[0..1] (FP64, recomputed).
cudaError_t launch_final_residual(amg_hierarchy* h, cudaStream_t s) {
    AMG_TRY(launch_residual(h, h->q, false, S_RR, true, nullptr, s));
    launch_pdl(k_sqrt_sum, 1, 256, 0, s, slot(h, S_RR), nb_res(h), slot(h, S_OUT));
    launch_pdl(k_sqrt_sum, 1, 256, 0, s, slot(h, S_FF), nb_res(h), slot(h, S_OUT) + 1);
    return cudaGetLastError();
}

double* final_residual_slot(amg_hierarchy* h) { return slot(h, S_OUT); }

// z = B r for r already in h->r (state must not be "done").
cudaError_t enqueue_vcycle_standalone(amg_hierarchy* h, cudaStream_t s) {
    if (h->nlev > 1) {
        Level& L0 = h->lev[0];
        if (h->mixed)
            launch_pdl(k_scale<float>, nbv(h), kBlock, 0, s, L0.A.n, h->r, L0.invd32, L0.x32);
        else
            launch_pdl(k_scale<double>, nbv(h), kBlock, 0, s, L0.A.n, h->r, L0.invd, L0.x);
    }
    AMG_TRY(cudaGetLastError());
    return enqueue_vcycle(h, s);
}

}  // namespace amg
