// Matrix-pass building blocks and the row-group kernels of the solve
// phase (included by solve_kernels.cu): matrix views (plain CSR, and CSR
// values with run-encoded columns), the warp row-group reduction and the
// kernels that make one pass over a level matrix with their fused
// epilogues -- q = K p with p.q, residuals, smoothing sweeps, the up sweep
// with prolongation, the level-0 up sweep with r.z -- and the FP64
// residual.  Arithmetic of arXiv 2511.21268, Sec. 3 (two-level correction
// steps applied recursively) and Sec. 3.2 (l1-Jacobi).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double ldv(const double* v, int64_t k) { return __ldg(v + k); }
__device__ __forceinline__ float ldv(const float* v, int64_t k) { return __ldg(v + k); }
__device__ __forceinline__ float ldv(const __nv_bfloat16* v, int64_t k) { return __bfloat162float(v[k]); }

// Lane partial of row i: sum over k = b + lane + 32 t of v_k x_{c_k}, in A.
// The rows this runs on (levels with few rows, a warp per row) are
// latency-bound: each chunk of U entries per lane loads all its values and
// columns, then all its x entries, then runs the FMA chain in entry order,
// and the last partial chunk does the same with predicated loads, so a row
// of up to 32 U entries costs two dependent round trips.
template <typename A, typename V, typename X>
__device__ __forceinline__ A lane_partial(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                          const V* __restrict__ v, const X* __restrict__ x, int i, int lane) {
    constexpr int U = sizeof(A) == 4 ? 16 : 8;
    const int64_t b = rp[i], e = rp[i + 1];
    A acc = A(0);
    int64_t k = b + lane;
    for (; k + 32 * (U - 1) < e; k += 32 * U) {
        A vv[U], xx[U];
        int cc[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            vv[u] = (A)ldv(v, k + 32 * u);
            cc[u] = __ldg(ci + k + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < U; u++) xx[u] = (A)x[cc[u]];
#pragma unroll
        for (int u = 0; u < U; u++) acc = fma(vv[u], xx[u], acc);
    }
    if (k < e) {  // fewer than U entries left on this lane
        A vv[U - 1], xx[U - 1];
        int cc[U - 1];
#pragma unroll
        for (int u = 0; u < U - 1; u++) {
            const bool in = k + 32 * u < e;
            vv[u] = in ? (A)ldv(v, k + 32 * u) : A(0);
            cc[u] = in ? __ldg(ci + k + 32 * u) : -1;
        }
#pragma unroll
        for (int u = 0; u < U - 1; u++) xx[u] = cc[u] >= 0 ? (A)x[cc[u]] : A(0);
#pragma unroll
        for (int u = 0; u < U - 1; u++)
            if (cc[u] >= 0) acc = fma(vv[u], xx[u], acc);
    }
    return acc;
}

// Matrix views of the row-group kernels.  CsrM: plain CSR.  RunM: CSR
// values with run-encoded columns (every row a sequence of equal runs of L
// consecutive columns): one 4-byte start column per run replaces the run's
// column indices, so a pass reads s_v + 4/L bytes per entry from HBM
// instead of s_v + 4.  The lanes keep the CSR order (lane t reads entries
// b + t + 32 j, coalesced); entry b + u lies in run u / L at offset u % L,
// the quotient taken as __umulhi(u, ceil(2^32 / L)) (exact for u < 2^16),
// and the run's start column is an L1-resident load shared by the L lanes
// of the run.
__constant__ uint32_t kRunMagic[kMaxRunLen + 1] = {0u,          0u,          2147483648u, 1431655766u, 1073741824u,
                                                   858993460u,  715827883u,  613566757u,  536870912u,  477218589u};

template <typename V>
struct CsrM {
    static constexpr bool kFlat = true;
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ ci;
    const V* __restrict__ v;
    template <typename A, typename X>
    __device__ __forceinline__ A partial(const X* __restrict__ x, int i, int lane) const {
        return lane_partial<A>(rp, ci, v, x, i, lane);
    }
    // Lane partials of the RPW rows row0 .. row0+RPW-1 into tile[r][lane]:
    // the warp streams the rows' contiguous entries, lane t taking entries
    // e0 + t + 32 j in order with four loads in flight, so no row waits for
    // the previous one.  A lane keeps one running sum and stores it to
    // tile[r][t] when its next entry lies past row r (rows it never
    // touches keep 0).
    template <int RPW, typename A, typename X>
    __device__ __forceinline__ void flat(const X* __restrict__ x, int row0, int n, int lane, A (*tile)[33]) const {
        const int64_t myb = lane <= RPW ? rp[min(row0 + lane, n)] : 0;
        const int64_t e0 = __shfl_sync(FULL, myb, 0);
        const int rel = (int)(myb - e0);  // row bound j on lane j, relative to e0
        int bnd[RPW + 1];
#pragma unroll
        for (int j = 0; j <= RPW; j++) bnd[j] = __shfl_sync(FULL, rel, j);
#pragma unroll
        for (int r = 0; r < RPW; r++) tile[r][lane] = A(0);
        const int len = bnd[RPW];
        const V* __restrict__ vr = v + e0;
        const int32_t* __restrict__ cr = ci + e0;
        int r = 0, nb = bnd[1];
        A acc = A(0);
        auto take = [&](int k, A val, A xv) {
            while (k >= nb) {  // rows ending before entry k
                tile[r][lane] = acc;
                acc = A(0);
                r++;
#pragma unroll
                for (int j = 1; j <= RPW; j++)
                    if (j == r + 1) nb = bnd[j];
            }
            acc = fma(val, xv, acc);
        };
        for (int k0 = lane; k0 < len; k0 += 128) {
            const int k1 = k0 + 32, k2 = k0 + 64, k3 = k0 + 96;
            const A v0 = (A)ldv(vr, k0);
            const A v1 = k1 < len ? (A)ldv(vr, k1) : A(0);
            const A v2 = k2 < len ? (A)ldv(vr, k2) : A(0);
            const A v3 = k3 < len ? (A)ldv(vr, k3) : A(0);
            const int c0 = __ldg(cr + k0);
            const int c1 = k1 < len ? __ldg(cr + k1) : 0;
            const int c2 = k2 < len ? __ldg(cr + k2) : 0;
            const int c3 = k3 < len ? __ldg(cr + k3) : 0;
            const A x0 = (A)x[c0];
            const A x1 = k1 < len ? (A)x[c1] : A(0);
            const A x2 = k2 < len ? (A)x[c2] : A(0);
            const A x3 = k3 < len ? (A)x[c3] : A(0);
            take(k0, v0, x0);
            if (k1 < len) take(k1, v1, x1);
            if (k2 < len) take(k2, v2, x2);
            if (k3 < len) take(k3, v3, x3);
        }
        if (r < RPW) tile[r][lane] = acc;
    }
};

template <typename V>
struct RunM {
    static constexpr bool kFlat = false;
    const int64_t* __restrict__ rp;
    const int32_t* __restrict__ rptr;
    const uint8_t* __restrict__ rlen;
    const int32_t* __restrict__ rst;
    const V* __restrict__ v;
    template <typename A, typename X>
    __device__ __forceinline__ A partial(const X* __restrict__ x, int i, int lane) const {
        const int64_t b = __ldg(rp + i), e = __ldg(rp + i + 1);
        const uint32_t L = rlen[i];
        const uint32_t mg = kRunMagic[L];
        const int32_t* __restrict__ rs = rst + __ldg(rptr + i);
        const uint32_t len = (uint32_t)(e - b);
        const V* __restrict__ vr = v + b;
        A acc = A(0);
        uint32_t u = lane;
        auto col = [&](uint32_t w) {
            const uint32_t q = __umulhi(w, mg);
            return __ldg(rs + q) + (int)(w - q * L);
        };
        for (; u + 96 < len; u += 128) {
            const A v0 = (A)ldv(vr, u), v1 = (A)ldv(vr, u + 32), v2 = (A)ldv(vr, u + 64), v3 = (A)ldv(vr, u + 96);
            const int c0 = col(u), c1 = col(u + 32), c2 = col(u + 64), c3 = col(u + 96);
            const A x0 = (A)x[c0], x1 = (A)x[c1], x2 = (A)x[c2], x3 = (A)x[c3];
            acc = fma(v0, x0, acc);
            acc = fma(v1, x1, acc);
            acc = fma(v2, x2, acc);
            acc = fma(v3, x3, acc);
        }
        for (; u < len; u += 32) acc = fma((A)ldv(vr, u), (A)x[col(u)], acc);
        return acc;
    }
};

// Row totals for the RPW rows row0 .. row0+RPW-1 (rows >= n give 0).
// Returns the total of row `row0 + lane / (32/RPW)` on every lane.
template <int RPW, typename A, typename M, typename X>
__device__ __forceinline__ A group_rows(const M& mat, const X* __restrict__ x, int row0, int n, int lane,
                                        A (*tile)[33]) {
    if constexpr (RPW == 1) {
        A s = row0 < n ? mat.template partial<A>(x, row0, lane) : A(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        return s;
    } else {
        constexpr int LPR = 32 / RPW;  // lanes per row in the finishing step
        if constexpr (M::kFlat) {
            mat.template flat<RPW, A>(x, row0, n, lane, tile);
        } else {
#pragma unroll 1
            for (int r = 0; r < RPW; r++) {
                const int i = row0 + r;
                tile[r][lane] = i < n ? mat.template partial<A>(x, i, lane) : A(0);
            }
        }
        __syncwarp();
        const int r = lane / LPR, q = lane % LPR;
        A s = A(0);
#pragma unroll
        for (int t = 0; t < RPW; t++) s += tile[r][q * RPW + t];
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        __syncwarp();
        return s;
    }
}

// Deterministic sum of one value per lane over the block -> *out (thread 0).
__device__ __forceinline__ void block_partial(double tv, double* sh, double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tv += __shfl_xor_sync(FULL, tv, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = tv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
        *out = s;
    }
}

#define DONE_GUARD(st)                  \
    do {                                \
        if ((st) && (st)->done) return; \
    } while (0)

// Common prologue of the row-group kernels.
#define ROWGROUP_PROLOGUE(A)                                           \
    __shared__ A tiles[kWarpsPerBlock][RPW][33];                       \
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;         \
    const int row0 = (blockIdx.x * kWarpsPerBlock + wid) * RPW;        \
    constexpr int LPR = 32 / RPW;                                      \
    const int myrow = row0 + lane / LPR;                               \
    const bool owner = (lane % LPR) == 0 && myrow < n;                 \
    (void)owner;

// ----------------------------------------------------------------- kernels
template <int RPW, typename M>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, M mat, const double* __restrict__ x, double* y) {
    pdl_entry();
    ROWGROUP_PROLOGUE(double)
    const double s = group_rows<RPW, double>(mat, x, row0, n, lane, tiles[wid]);
    if (owner) y[myrow] = s;
}

// FP64: r = F - K x, x0 = r / d (optional, in X0), partials ||r||^2, ||F||^2.
// `gate` (optional): run only while the solve is not done and a
// residual replacement is due.
template <int RPW, typename X0, typename M>
__global__ void __launch_bounds__(kBlock) k_residual0(int n, M mat, const double* __restrict__ x,
                                                       const double* __restrict__ F,
                                                       const X0* __restrict__ invd, double* r, X0* x0,
                                                       double* part_rr, double* part_ff, const SolveState* gate) {
    pdl_entry();
    // grid-stride over row groups (a small grid: the gated launch of every
    // mixed-precision iteration returns at once unless a replacement is due)
    if (gate && (gate->done || !gate->replace_now)) return;
    __shared__ double tiles[kWarpsPerBlock][RPW][33];
    __shared__ double sh[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int LPR = 32 / RPW;
    double rr = 0.0, ff = 0.0;
    const int ngroups = (n + RPW - 1) / RPW;
    for (int g = blockIdx.x * kWarpsPerBlock + wid; g - wid < ngroups; g += gridDim.x * kWarpsPerBlock) {
        const int row0 = g * RPW;  // groups past the end give zero rows (uniform per block)
        const double s = group_rows<RPW, double>(mat, x, row0, n, lane, tiles[wid]);
        const int myrow = row0 + lane / LPR;
        if ((lane % LPR) == 0 && myrow < n) {
            const double fi = F[myrow], ri = fi - s;
            r[myrow] = ri;
            if (x0) x0[myrow] = (X0)ri * invd[myrow];
            rr += ri * ri;
            ff += fi * fi;
        }
    }
    block_partial(rr, sh, part_rr + blockIdx.x);
    if (part_ff) block_partial(ff, sh, part_ff + blockIdx.x);
}

// Outer SpMV q = K p (values V, gathered vector PX, accumulation A; q FP64),
// partials p.q and (flexible) p.r with the FP64 p.
template <int RPW, typename A, typename M, typename PX>
__global__ void __launch_bounds__(kBlock) k_spmv_pq(int n, M mat, const PX* __restrict__ pg,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ r, double* q, double* part_pq,
                                                     double* part_pr, int flexible, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    __shared__ double sh[kWarpsPerBlock];
    const A s = group_rows<RPW, A>(mat, pg, row0, n, lane, tiles[wid]);
    double pq = 0.0, pr = 0.0;
    if (owner) {
        const double qs = (double)s;
        q[myrow] = qs;
        const double pi = p[myrow];
        pq = pi * qs;
        if (flexible) pr = pi * r[myrow];
    }
    block_partial(pq, sh, part_pq + blockIdx.x);
    if (flexible) block_partial(pr, sh, part_pr + blockIdx.x);
}

// rbuf = f - K x (down-sweep residual of one level).
template <int RPW, typename A, typename M, typename FT, typename XT>
__global__ void __launch_bounds__(kBlock) k_resid(int n, M mat, const FT* __restrict__ f, const XT* __restrict__ x,
                                                   A* rbuf, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, x, row0, n, lane, tiles[wid]);
    if (owner) rbuf[myrow] = (A)f[myrow] - s;
}

// t = x + (f - K x) / d (extra smoothing sweep).
template <int RPW, typename A, typename M, typename FT>
__global__ void __launch_bounds__(kBlock) k_sweep(int n, M mat, const FT* __restrict__ f, const A* __restrict__ x,
                                                   const A* __restrict__ invd, A* t, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, x, row0, n, lane, tiles[wid]);
    if (owner) t[myrow] = fma(invd[myrow], (A)f[myrow] - s, x[myrow]);
}

// Up sweep of level l >= 1: y_a = x_a + (f_a - (K x)_a) / d_a, then
// x_{l-1}[c] += p_c y_a for the members c of a (one member per lane of the
// row's lane group).
template <int RPW, typename A, typename M>
__global__ void __launch_bounds__(kBlock) k_up(int n, M mat, const A* __restrict__ f, const A* __restrict__ x,
                                                const A* __restrict__ invd,
                                                const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                                                const double* __restrict__ pvalf, A* xf, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    const A s = group_rows<RPW, A>(mat, x, row0, n, lane, tiles[wid]);
    // every lane of the row's group has the total; the aggregate's members
    // (independent fine rows) are spread over those LPR lanes
    if (myrow < n) {
        const A y = fma(invd[myrow], f[myrow] - s, x[myrow]);
        const int m1 = mptr[myrow + 1];
        for (int m = mptr[myrow] + lane % LPR; m < m1; m += LPR) {
            const int c = midx[m];
            xf[c] = fma((A)pvalf[c], y, xf[c]);
        }
    }
}

// Up sweep of level 0: z = x + (r - K x) / d (z FP64); partials r.z and
// (flexible) z.q.
template <int RPW, typename A, typename M>
__global__ void __launch_bounds__(kBlock) k_up0(int n, M mat, const double* __restrict__ r,
                                                 const A* __restrict__ x, const A* __restrict__ invd, double* z,
                                                 const double* __restrict__ q, double* part_rz, double* part_zq,
                                                 int flexible, const SolveState* st) {
    pdl_entry();
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE(A)
    __shared__ double sh[kWarpsPerBlock];
    const A s = group_rows<RPW, A>(mat, x, row0, n, lane, tiles[wid]);
    double rz = 0.0, zq = 0.0;
    if (owner) {
        const double ra = r[myrow];
        const double za = (double)fma(invd[myrow], (A)ra - s, x[myrow]);
        z[myrow] = za;
        rz = ra * za;
        if (flexible) zq = za * q[myrow];
    }
    block_partial(rz, sh, part_rz + blockIdx.x);
    if (flexible) block_partial(zq, sh, part_zq + blockIdx.x);
}

}  // namespace
}  // namespace amg
