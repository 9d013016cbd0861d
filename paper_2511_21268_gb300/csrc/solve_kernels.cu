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
// Fusions:
//   * pre-smoothing from x = 0 is x = D^-1 f, written by whoever produces f
//     (the CG update for level 0, the restriction for level l+1);
//   * down sweep: r = f - K x into a scratch vector, then restriction
//     f_{l+1}[I] = sum_{a in I} p_a r_a and x_{l+1} = f_{l+1} / d;
//   * up sweep of level l: y = x + (f - K x) / d, prolongated at once into
//     the finer level, x_{l-1}[c] += p_c y_a for the members c of a; on
//     level 0 it writes z and the partial sums of r.z (and z.q);
//   * coarsest solve: dense GEMV with the precomputed inverse, followed by
//     the same prolongation.
// Reductions are deterministic: fixed grids, fixed lane/warp/block order and
// a single-block final sum.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// Lane partial of row i: sum over k = b + lane + 32 t of v_k x_{c_k}.
__device__ __forceinline__ double lane_partial(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                               const double* __restrict__ v, const double* __restrict__ x, int i,
                                               int lane) {
    const int64_t b = rp[i], e = rp[i + 1];
    double acc = 0.0;
    int64_t k = b + lane;
    for (; k + 96 < e; k += 128) {
        const double v0 = __ldg(v + k), v1 = __ldg(v + k + 32), v2 = __ldg(v + k + 64), v3 = __ldg(v + k + 96);
        const int c0 = __ldg(ci + k), c1 = __ldg(ci + k + 32), c2 = __ldg(ci + k + 64), c3 = __ldg(ci + k + 96);
        const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
        acc = fma(v0, x0, acc);
        acc = fma(v1, x1, acc);
        acc = fma(v2, x2, acc);
        acc = fma(v3, x3, acc);
    }
    for (; k < e; k += 32) acc = fma(__ldg(v + k), x[__ldg(ci + k)], acc);
    return acc;
}

// Row totals for the RPW rows row0 .. row0+RPW-1 (rows >= n give 0).
// Returns the total of row `row0 + lane / (32/RPW)` on every lane.
template <int RPW>
__device__ __forceinline__ double group_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                             const double* __restrict__ v, const double* __restrict__ x, int row0,
                                             int n, int lane, double (*tile)[33]) {
    if constexpr (RPW == 1) {
        double s = row0 < n ? lane_partial(rp, ci, v, x, row0, lane) : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        return s;
    } else {
        constexpr int LPR = 32 / RPW;  // lanes per row in the finishing step
#pragma unroll 1
        for (int r = 0; r < RPW; r++) {
            const int i = row0 + r;
            tile[r][lane] = i < n ? lane_partial(rp, ci, v, x, i, lane) : 0.0;
        }
        __syncwarp();
        const int r = lane / LPR, q = lane % LPR;
        double s = 0.0;
#pragma unroll
        for (int t = 0; t < RPW; t++) s += tile[r][q * RPW + t];
#pragma unroll
        for (int o = LPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        __syncwarp();
        return s;
    }
}

// Deterministic sum of one value per owner lane over the block -> out.
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

// Deterministic single-block sum of nb partials (all threads get it).
__device__ double sum_partials(const double* __restrict__ part, int nb, double* sh) {
    double s = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) s += part[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) tot += sh[w];
    __syncthreads();
    return tot;
}

#define DONE_GUARD(st)                  \
    do {                                \
        if ((st) && (st)->done) return; \
    } while (0)

// Common prologue of the row-group kernels.
#define ROWGROUP_PROLOGUE                                              \
    __shared__ double tiles[kWarpsPerBlock][RPW][33];                  \
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;         \
    const int row0 = (blockIdx.x * kWarpsPerBlock + wid) * RPW;        \
    constexpr int LPR = 32 / RPW;                                      \
    const int myrow = row0 + lane / LPR;                               \
    const bool owner = (lane % LPR) == 0 && myrow < n;                 \
    (void)owner;

// ----------------------------------------------------------------- kernels
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                  const double* __restrict__ v, const double* __restrict__ x,
                                                  double* y) {
    ROWGROUP_PROLOGUE
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    if (owner) y[myrow] = s;
}

// r = F - K x, x0 = r / d (optional), partials ||r||^2 and ||F||^2.
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_residual0(int n, const int64_t* __restrict__ rp,
                                                       const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                       const double* __restrict__ x, const double* __restrict__ F,
                                                       const double* __restrict__ invd, double* r, double* x0,
                                                       double* part_rr, double* part_ff) {
    ROWGROUP_PROLOGUE
    __shared__ double sh[kWarpsPerBlock];
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    double rr = 0.0, ff = 0.0;
    if (owner) {
        const double fi = F[myrow], ri = fi - s;
        r[myrow] = ri;
        if (x0) x0[myrow] = ri * invd[myrow];
        rr = ri * ri;
        ff = fi * fi;
    }
    block_partial(rr, sh, part_rr + blockIdx.x);
    block_partial(ff, sh, part_ff + blockIdx.x);
}

// q = K p, partials p.q and (flexible) p.r.
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_spmv_pq(int n, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                     const double* __restrict__ p, const double* __restrict__ r,
                                                     double* q, double* part_pq, double* part_pr, int flexible,
                                                     const SolveState* st) {
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE
    __shared__ double sh[kWarpsPerBlock];
    const double s = group_rows<RPW>(rp, ci, v, p, row0, n, lane, tiles[wid]);
    double pq = 0.0, pr = 0.0;
    if (owner) {
        q[myrow] = s;
        const double pi = p[myrow];
        pq = pi * s;
        if (flexible) pr = pi * r[myrow];
    }
    block_partial(pq, sh, part_pq + blockIdx.x);
    if (flexible) block_partial(pr, sh, part_pr + blockIdx.x);
}

// rbuf = f - K x (down sweep residual of one level).
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_resid(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const double* __restrict__ v, const double* __restrict__ f,
                                                   const double* __restrict__ x, double* rbuf, const SolveState* st) {
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    if (owner) rbuf[myrow] = f[myrow] - s;
}

// t = x + (f - K x) / d (extra smoothing sweep).
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_sweep(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const double* __restrict__ v, const double* __restrict__ f,
                                                   const double* __restrict__ x, const double* __restrict__ invd,
                                                   double* t, const SolveState* st) {
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    if (owner) t[myrow] = fma(invd[myrow], f[myrow] - s, x[myrow]);
}

// Up sweep of level l >= 1: y_a = x_a + (f_a - (K x)_a) / d_a, then
// x_{l-1}[c] += p_c y_a for the members c of a.
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_up(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                const double* __restrict__ v, const double* __restrict__ f,
                                                const double* __restrict__ x, const double* __restrict__ invd,
                                                const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                                                const double* __restrict__ pvalf, double* xf, const SolveState* st) {
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    if (owner) {
        const double y = fma(invd[myrow], f[myrow] - s, x[myrow]);
        for (int m = mptr[myrow]; m < mptr[myrow + 1]; m++) {
            const int c = midx[m];
            xf[c] = fma(pvalf[c], y, xf[c]);
        }
    }
}

// Up sweep of level 0: z = x + (r - K x) / d; partials r.z and (flexible) z.q.
template <int RPW>
__global__ void __launch_bounds__(kBlock) k_up0(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                 const double* __restrict__ v, const double* __restrict__ r,
                                                 const double* __restrict__ x, const double* __restrict__ invd,
                                                 double* z, const double* __restrict__ q, double* part_rz,
                                                 double* part_zq, int flexible, const SolveState* st) {
    DONE_GUARD(st);
    ROWGROUP_PROLOGUE
    __shared__ double sh[kWarpsPerBlock];
    const double s = group_rows<RPW>(rp, ci, v, x, row0, n, lane, tiles[wid]);
    double rz = 0.0, zq = 0.0;
    if (owner) {
        const double ra = r[myrow];
        const double za = fma(invd[myrow], ra - s, x[myrow]);
        z[myrow] = za;
        rz = ra * za;
        if (flexible) zq = za * q[myrow];
    }
    block_partial(rz, sh, part_rz + blockIdx.x);
    if (flexible) block_partial(zq, sh, part_zq + blockIdx.x);
}

// Restriction f_c[I] = sum_{a in I, ascending} p_a r_a, x_c = f_c / d_c.
__global__ void k_restrict(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                           const double* __restrict__ pval, const double* __restrict__ rbuf, double* fc, double* xc,
                           const double* __restrict__ invdc, const SolveState* st) {
    DONE_GUARD(st);
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int m = mptr[I]; m < mptr[I + 1]; m++) {
            const int a = midx[m];
            acc = fma(pval[a], rbuf[a], acc);
        }
        fc[I] = acc;
        if (xc) xc[I] = acc * invdc[I];
    }
}

// Coarsest level: e = A^-1 f with the dense symmetric inverse (row-major),
// then prolongation into the finer level, or (single-level hierarchy) z = e
// with the partial r.z (and z.q).
__global__ void __launch_bounds__(kBlock) k_coarse(int n, const double* __restrict__ Ainv, const double* __restrict__ f,
                                                    const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                                                    const double* __restrict__ pvalf, double* xf, double* z,
                                                    const double* __restrict__ q, double* part_rz, double* part_zq,
                                                    int flexible, const SolveState* st) {
    DONE_GUARD(st);
    __shared__ double sh[kWarpsPerBlock];
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double rz = 0.0, zq = 0.0;
    if (I < n) {
        const double* row = Ainv + (int64_t)I * n;
        double s = 0.0;
        for (int j = lane; j < n; j += 32) s = fma(row[j], f[j], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (z) {
            if (lane == 0) {
                z[I] = s;
                rz = f[I] * s;
                if (flexible) zq = s * q[I];
            }
        } else if (lane == 0) {
            for (int m = mptr[I]; m < mptr[I + 1]; m++) {
                const int c = midx[m];
                xf[c] = fma(pvalf[c], s, xf[c]);
            }
        }
    }
    if (z) {
        block_partial(rz, sh, part_rz + blockIdx.x);
        if (flexible) block_partial(zq, sh, part_zq + blockIdx.x);
    }
}

// ------------------------------------------------------------ CG scalars
__global__ void k_scal_init(const double* part_rr, const double* part_ff, int nb, double rtol, int itmax,
                            double* hist, SolveState* st) {
    // every field a later kernel reads is (re)set here
    __shared__ double sh[32];
    const double rr = sum_partials(part_rr, nb, sh);
    const double ff = sum_partials(part_ff, nb, sh);
    if (threadIdx.x == 0) {
        const double nF = sqrt(ff), nr = sqrt(rr);
        st->nF = nF;
        st->tol = rtol * nF;
        st->nr = nr;
        st->iters = 0;
        st->itmax = itmax;
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
    DONE_GUARD(st);
    __shared__ double sh[32];
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

__global__ void k_scal_conv(const double* part_rr, int nb, double* hist, int hist_cap, SolveState* st) {
    DONE_GUARD(st);
    __shared__ double sh[32];
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
    DONE_GUARD(st);
    __shared__ double sh[32];
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

// x += alpha p, r -= alpha q, x0 = r / d, partial ||r||^2.
__global__ void k_update(int n, double* x, double* r, const double* __restrict__ p, const double* __restrict__ q,
                         const double* __restrict__ invd, double* x0, double* part_rr, const SolveState* st) {
    DONE_GUARD(st);
    __shared__ double sh[kWarpsPerBlock];
    const double alpha = st->alpha;
    double rr = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = fma(alpha, p[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        if (x0) x0[i] = ri * invd[i];
        rr = fma(ri, ri, rr);
    }
    block_partial(rr, sh, part_rr + blockIdx.x);
}

// p = z + beta p (first direction: p = z).
__global__ void k_pupdate(int n, double* p, const double* __restrict__ z, int first, const SolveState* st) {
    DONE_GUARD(st);
    const double beta = st->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        p[i] = first ? z[i] : fma(beta, p[i], z[i]);
}

__global__ void k_scale(int n, const double* __restrict__ a, const double* __restrict__ b, double* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = a[i] * b[i];
}

__global__ void k_sqrt_sum(const double* part, int nb, double* out) {
    __shared__ double sh[32];
    const double s = sum_partials(part, nb, sh);
    if (threadIdx.x == 0) *out = sqrt(s);
}

// ----------------------------------------------------------------- dispatch
template <typename K1, typename K8>
inline void pick(int rpw, K1 k1, K8 k8) {
    if (rpw == 8) k8();
    else k1();
}

}  // namespace

int rows_per_warp(int n, int num_sms) {
    // 8-row groups once there are enough of them to fill the GPU several times
    return ((int64_t)n >= (int64_t)num_sms * kWarpsPerBlock * 8 * 4) ? 8 : 1;
}

int row_blocks(int n, int rpw) { return (int)(((int64_t)n + (int64_t)rpw * kWarpsPerBlock - 1) / ((int64_t)rpw * kWarpsPerBlock)); }

int vec_blocks(int n, int num_sms) {
    int64_t b = ((int64_t)n + kBlock - 1) / kBlock;
    const int cap = num_sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

int grid_for_rows(int, int n, int num_sms) { return row_blocks(n, rows_per_warp(n, num_sms)); }

cudaError_t launch_spmv(const DevCSR& A, const double* x, double* y, cudaStream_t s) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int rpw = rows_per_warp(A.n, sms);
    const int nb = row_blocks(A.n, rpw);
    if (A.n == 0) return cudaSuccess;
    pick(rpw, [&] { k_spmv<1><<<AMG_GRID(nb), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, x, y); },
         [&] { k_spmv<8><<<AMG_GRID(nb), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, x, y); });
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
enum { S_RR = 0, S_FF, S_PQ, S_PR, S_RZ, S_ZQ, S_OUT };

// V-cycle on r (= f_0); the pre-smoothed level-0 iterate is already in lev[0].x.
// Writes z and the partial sums of r.z (and z.q).
cudaError_t enqueue_vcycle(amg_hierarchy* h, cudaStream_t s) {
    const int L = h->nlev;
    const int sms = h->num_sms;
    const int flex = h->o.flexible;
    const SolveState* st = h->st;
    if (L == 1) {
        k_coarse<<<AMG_GRID(row_blocks(h->ndense, 1)), kBlock, 0, s>>>(h->ndense, h->Ainv, h->r, nullptr, nullptr, nullptr,
                                                             nullptr, h->z, h->q, slot(h, S_RZ), slot(h, S_ZQ), flex,
                                                             st);
        return cudaGetLastError();
    }
    double* xcur[AMG_MAX_LEVELS];
    double* xalt[AMG_MAX_LEVELS];
    for (int l = 0; l < L; l++) {
        xcur[l] = h->lev[l].x;
        xalt[l] = h->lev[l].t;
    }
    // down
    for (int l = 0; l < L - 1; l++) {
        Level& F = h->lev[l];
        Level& C = h->lev[l + 1];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw);
        const double* f = (l == 0) ? h->r : F.f;
        for (int sw = 1; sw < h->o.nu_pre; sw++) {
            double* xo = xcur[l];
            double* xn = xalt[l];
            pick(rpw,
                 [&] { k_sweep<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xo, F.invd, xn, st); },
                 [&] { k_sweep<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xo, F.invd, xn, st); });
            xcur[l] = xn;
            xalt[l] = xo;
        }
        double* rb = xalt[l];  // free buffer of this level holds the residual
        const double* xc = xcur[l];
        if (l == 0) prof_mark(h, 1, 0, s);
        pick(rpw, [&] { k_resid<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xc, rb, st); },
             [&] { k_resid<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xc, rb, st); });
        if (l == 0) prof_mark(h, 1, 1, s);
        const bool coarsest = (l + 1 == L - 1);
        k_restrict<<<AMG_GRID(vec_blocks(C.A.n, sms)), kBlock, 0, s>>>(C.A.n, F.mem_ptr, F.mem_idx, F.pval, rb, C.f,
                                                             coarsest ? nullptr : xcur[l + 1], C.invd, st);
    }
    // coarsest
    {
        Level& F = h->lev[L - 2];
        Level& C = h->lev[L - 1];
        k_coarse<<<AMG_GRID(row_blocks(C.A.n, 1)), kBlock, 0, s>>>(C.A.n, h->Ainv, C.f, F.mem_ptr, F.mem_idx, F.pval,
                                                         xcur[L - 2], nullptr, nullptr, nullptr, nullptr, 0, st);
    }
    // up
    for (int l = L - 2; l >= 0; l--) {
        Level& F = h->lev[l];
        const int n = F.A.n;
        const int rpw = rows_per_warp(n, sms), nb = row_blocks(n, rpw);
        const double* f = (l == 0) ? h->r : F.f;
        for (int sw = 1; sw < h->o.nu_post; sw++) {
            double* xo = xcur[l];
            double* xn = xalt[l];
            pick(rpw,
                 [&] { k_sweep<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xo, F.invd, xn, st); },
                 [&] { k_sweep<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, f, xo, F.invd, xn, st); });
            xcur[l] = xn;
            xalt[l] = xo;
        }
        const double* xc = xcur[l];
        if (l == 0) {
            prof_mark(h, 2, 0, s);
            pick(rpw,
                 [&] {
                     k_up0<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, h->r, xc, F.invd, h->z, h->q,
                                                    slot(h, S_RZ), slot(h, S_ZQ), flex, st);
                 },
                 [&] {
                     k_up0<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, h->r, xc, F.invd, h->z, h->q,
                                                    slot(h, S_RZ), slot(h, S_ZQ), flex, st);
                 });
            prof_mark(h, 2, 1, s);
        } else {
            Level& G = h->lev[l - 1];
            double* xf = xcur[l - 1];
            pick(rpw,
                 [&] {
                     k_up<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, F.f, xc, F.invd, G.mem_ptr,
                                                   G.mem_idx, G.pval, xf, st);
                 },
                 [&] {
                     k_up<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, F.A.rowptr, F.A.col, F.A.val, F.f, xc, F.invd, G.mem_ptr,
                                                   G.mem_idx, G.pval, xf, st);
                 });
        }
    }
    return cudaGetLastError();
}

// blocks of the level-0 row kernels, of the vector kernels, and of the
// kernel that produces z (level-0 up sweep or single-level coarse solve)
static int nb0(amg_hierarchy* h) { return row_blocks(h->lev[0].A.n, rows_per_warp(h->lev[0].A.n, h->num_sms)); }
static int nbv(amg_hierarchy* h) { return vec_blocks(h->lev[0].A.n, h->num_sms); }
static int nbz(amg_hierarchy* h) { return h->nlev > 1 ? nb0(h) : row_blocks(h->ndense, 1); }

size_t partial_slot_size(int n0, int num_sms) {
    const int a = row_blocks(n0, rows_per_warp(n0, num_sms));
    const int b = vec_blocks(n0, num_sms);
    return (size_t)((a > b ? a : b) + 2);
}

static cudaError_t launch_residual(amg_hierarchy* h, double* r, double* x0, cudaStream_t s) {
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int rpw = rows_per_warp(n, h->num_sms), nb = row_blocks(n, rpw);
    pick(rpw,
         [&] {
             k_residual0<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, h->x, h->F, L0.invd, r, x0,
                                                  slot(h, S_RR), slot(h, S_FF));
         },
         [&] {
             k_residual0<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, h->x, h->F, L0.invd, r, x0,
                                                  slot(h, S_RR), slot(h, S_FF));
         });
    return cudaGetLastError();
}

// r = F - K x, ||F||, ||r||, first V-cycle, p = z, rho = r.z.
cudaError_t enqueue_pcg_start(amg_hierarchy* h, cudaStream_t s) {
    const int n = h->lev[0].A.n;
    AMG_TRY(launch_residual(h, h->r, h->nlev > 1 ? h->lev[0].x : nullptr, s));
    k_scal_init<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_RR), slot(h, S_FF), nb0(h), h->rtol, h->itmax, h->hist, h->st);
    AMG_TRY(cudaGetLastError());
    AMG_TRY(enqueue_vcycle(h, s));
    k_scal_beta<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_RZ), slot(h, S_ZQ), nbz(h), h->o.flexible, 1, h->st);
    k_pupdate<<<AMG_GRID(nbv(h)), kBlock, 0, s>>>(n, h->p, h->z, 1, h->st);
    return cudaGetLastError();
}

cudaError_t enqueue_pcg_iteration(amg_hierarchy* h, cudaStream_t s) {
    Level& L0 = h->lev[0];
    const int n = L0.A.n;
    const int flex = h->o.flexible;
    const int rpw = rows_per_warp(n, h->num_sms), nb = row_blocks(n, rpw);
    prof_mark(h, 0, 0, s);
    pick(rpw,
         [&] {
             k_spmv_pq<1><<<AMG_GRID(nb), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, h->p, h->r, h->q, slot(h, S_PQ),
                                                slot(h, S_PR), flex, h->st);
         },
         [&] {
             k_spmv_pq<8><<<AMG_GRID(nb), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, h->p, h->r, h->q, slot(h, S_PQ),
                                                slot(h, S_PR), flex, h->st);
         });
    prof_mark(h, 0, 1, s);
    k_scal_alpha<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_PQ), slot(h, S_PR), nb, flex, h->st);
    k_update<<<AMG_GRID(nbv(h)), kBlock, 0, s>>>(n, h->x, h->r, h->p, h->q, L0.invd, h->nlev > 1 ? L0.x : nullptr,
                                       slot(h, S_RR), h->st);
    k_scal_conv<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_RR), nbv(h), h->hist, h->hist_cap, h->st);
    AMG_TRY(cudaGetLastError());
    AMG_TRY(enqueue_vcycle(h, s));
    k_scal_beta<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_RZ), slot(h, S_ZQ), nbz(h), flex, 0, h->st);
    k_pupdate<<<AMG_GRID(nbv(h)), kBlock, 0, s>>>(n, h->p, h->z, 0, h->st);
    return cudaGetLastError();
}

// ||F - K x|| and ||F|| into slot(S_OUT)[0..1] (FP64, recomputed).
cudaError_t launch_final_residual(amg_hierarchy* h, cudaStream_t s) {
    AMG_TRY(launch_residual(h, h->q, nullptr, s));
    k_sqrt_sum<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_RR), nb0(h), slot(h, S_OUT));
    k_sqrt_sum<<<AMG_GRID(1), 1024, 0, s>>>(slot(h, S_FF), nb0(h), slot(h, S_OUT) + 1);
    return cudaGetLastError();
}

double* final_residual_slot(amg_hierarchy* h) { return slot(h, S_OUT); }

// z = B r for r already in h->r (state must not be "done").
cudaError_t enqueue_vcycle_standalone(amg_hierarchy* h, cudaStream_t s) {
    if (h->nlev > 1)
        k_scale<<<AMG_GRID(nbv(h)), kBlock, 0, s>>>(h->lev[0].A.n, h->r, h->lev[0].invd, h->lev[0].x);
    AMG_TRY(cudaGetLastError());
    return enqueue_vcycle(h, s);
}

}  // namespace amg
