// Smoothed prolongator P_bar = (I - diag(theta) D^-1 K) P (arXiv 2511.21268,
// Sec. 3.1 "Variants", D the l1 diagonal of Sec. 3.2) and its Galerkin
// product K_c = P_bar^T (K P_bar), on the GPU, bit for bit as the oracle
// defines them:
//   * P_bar row i holds the coarse columns {agg(j) : j stored in row i},
//     ascending; with kp_J = sum over the stored j of row i in ascending order
//     with agg(j) = J of k_ij p_j and t = theta_i / d_i,
//     P_bar(i, J) = (J == agg(i) ? p_i : 0) - t kp_J;
//   * T = K P_bar, T(i, J) = sum over the stored j of row i in ascending
//     order of k_ij P_bar(j, J);
//   * K_c(I, J), I <= J, = sum over the rows a of column I of P_bar in
//     ascending order of P_bar(a, I) T(a, J); K_c(J, I) := K_c(I, J).
// Every sum starts from +0.0 and adds one correctly rounded product at a time
// (__dmul_rn / __dadd_rn, no contraction).
//
// All three products are row-merge SpGEMMs C = A B with one warp per output
// row.  The warp marks the output columns of its row in a shared-memory
// bitmap over the row's column span (bounded by the first and last column of
// every B row it reads), and prefix popcounts of the bitmap words give each
// column its rank in the sorted row: no sorting and no atomics on values.
// Two kernels walk a row's items -- the pairs (t, q) of an entry t of A's row
// and an entry q of B's row aci[t], t ascending, then q:
//   * short B rows (the tentative P, one entry per row): one warp per output
//     row takes 32 consecutive items per round, with the loads of kSpBatch
//     rounds in flight together (A's entries 32 at a time; a scan of their
//     B-row lengths places each item).  In the numeric pass the items of a
//     round that hit the same output column come from different t (a B row
//     has distinct columns) and are added in lane order, i.e. in ascending t;
//   * long B rows (K, P_bar, K P_bar): one block per output row shares one
//     accumulator (a warp's share of shared memory would leave the SM a few
//     warps); its threads split B's row of one t at a time (distinct columns,
//     no conflicts) and a block barrier separates successive t.
// Either way every output entry's sum runs in ascending order of A's column.
//
// The transpose P_bar^T needs no sort either: with K structurally symmetric,
// column J of P_bar holds exactly the rows that K's rows of J's members
// reach, i.e. the pattern of P^T K row J, which the same bitmap pass lists in
// ascending order; its values are found by a binary search in P_bar's rows.
//
// The V-cycle kernels for smoothed levels: restriction f_c = P_bar^T r (warp
// per coarse row over P_bar^T), prolongation x += P_bar y (warp per fine row),
// and the coarsest level's dense solve without the fused prolongation.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kSpWarps = 8;  // warps per block of the SpGEMM row kernels (fewer if shared memory is short)
constexpr int kSpBatch = 8;  // rounds of 32 items whose loads a warp keeps in flight together
constexpr int kSpUnroll = 4;  // B entries a thread of the block-per-row kernel loads before it accumulates them
constexpr double kSpMidRow = 16.0;    // average B row length from which the block-per-row kernel (64 threads) runs
constexpr double kSpLongRow = 256.0;  // ... and from which it runs with 256 threads
constexpr size_t kSpBitsBudget = (size_t)4 << 30;  // bytes of stored row bitmaps, at most

enum SpMode { SP_COUNT = 0, SP_COLS = 1, SP_VALUES = 2, SP_UPPER = 3 };

// Column span [lo, hi] of output row i of C = A B: bounded by the first and
// last stored column of every B row that A's row i reaches.
__device__ __forceinline__ void row_span(const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                                         const int64_t* __restrict__ brp, const int32_t* __restrict__ bci, int i,
                                         int lane, int& lo, int& hi) {
    int l = 0x7fffffff, h = -1;
    for (int64_t t = arp[i] + lane; t < arp[i + 1]; t += 32) {
        const int k = aci[t];
        const int64_t b0 = brp[k], b1 = brp[k + 1];
        if (b1 > b0) {
            l = min(l, bci[b0]);
            h = max(h, bci[b1 - 1]);
        }
    }
    lo = __reduce_min_sync(FULL, l);
    hi = __reduce_max_sync(FULL, h);
}

// A chunk of A's row: lane l takes entry tb + l (when < a1): the range
// [q0, q0 + len) of B's row aci[t] -- from its first column >= cfirst when
// cfirst >= 0 -- and the value a = av[t] (0 without values).  incl is the
// inclusive scan of len over the lanes, tot the chunk's item count.
__device__ __forceinline__ void chunk_open(const int32_t* __restrict__ aci, const double* __restrict__ av,
                                           const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                           int64_t tb, int64_t a1, int lane, int cfirst, int64_t& q0, int& len,
                                           int& incl, int& tot, double& a) {
    q0 = 0;
    len = 0;
    a = 0.0;
    const int64_t t = tb + lane;
    if (t < a1) {
        const int k = aci[t];
        int64_t b0 = brp[k];
        const int64_t b1 = brp[k + 1];
        if (cfirst >= 0) {
            int64_t hi = b1;
            while (b0 < hi) {
                const int64_t mid = (b0 + hi) >> 1;
                if (bci[mid] < cfirst) b0 = mid + 1;
                else hi = mid;
            }
        }
        q0 = b0;
        len = (int)(b1 - b0);
        if (av) a = av[t];
    }
    incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
    }
    tot = __shfl_sync(FULL, incl, 31);
}

// Item f of the chunk (0 <= f < tot): it belongs to the first lane s whose
// running length exceeds f; returns its B position q and A value a_s.  All
// lanes take part (lanes with f >= tot get a position they must not use).
__device__ __forceinline__ int64_t chunk_item(int f, int64_t q0, int len, int incl, double a, double& as) {
    int s = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(FULL, incl, s + step - 1);
        if (v <= f) s += step;
    }
    const int is = __shfl_sync(FULL, incl, s), ls = __shfl_sync(FULL, len, s);
    const int64_t qs = __shfl_sync(FULL, q0, s);
    as = __shfl_sync(FULL, a, s);
    return qs + (f - (is - ls));
}

// Marks the output columns of row i (A's row [a0, a1)) in bits (span from lo).
__device__ __forceinline__ void mark_row(const int32_t* __restrict__ aci, const int64_t* __restrict__ brp,
                                         const int32_t* __restrict__ bci, int64_t a0, int64_t a1, int lo, int lane,
                                         uint32_t* bits) {
    for (int64_t tb = a0; tb < a1; tb += 32) {
        int64_t q0;
        int len, incl, tot;
        double a;
        chunk_open(aci, nullptr, brp, bci, tb, a1, lane, -1, q0, len, incl, tot, a);
        for (int fb = 0; fb < tot; fb += 32 * kSpBatch) {
            int J[kSpBatch];
#pragma unroll
            for (int u = 0; u < kSpBatch; u++) {
                const int f = fb + 32 * u + lane;
                double as;
                const int64_t q = chunk_item(f, q0, len, incl, a, as);
                J[u] = f < tot ? bci[q] - lo : -1;
            }
#pragma unroll
            for (int u = 0; u < kSpBatch; u++)
                if (J[u] >= 0) atomicOr(&bits[J[u] >> 5], 1u << (J[u] & 31));
        }
    }
}

// Largest bitmap (words) any output row of A B needs.
__global__ void k_sp_span(int n, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                          const int64_t* __restrict__ brp, const int32_t* __restrict__ bci, int* maxw) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int best = 0;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        int lo, hi;
        row_span(arp, aci, brp, bci, i, lane, lo, hi);
        if (hi >= lo) best = max(best, ((hi - lo) >> 5) + 1);
    }
    if (lane == 0 && best > 0) atomicMax(maxw, best);
}

// One row-merge pass of C = A B (see the file header).  Shared memory per
// warp: bits[wmax], pre[wmax] (uint32 / int32) and, for the value modes,
// acc[cmax] (double).  SP_COUNT: rowcnt[i] = entries of row i (and the
// largest into *maxc); SP_COLS: sorted columns into cci; SP_VALUES: columns
// and values; SP_UPPER: columns, values of J >= i (0 below, for the mirror).
template <int MODE>
__global__ void k_sp_row(int n, const int64_t* __restrict__ arp, const int32_t* __restrict__ aci,
                         const double* __restrict__ av, const int64_t* __restrict__ brp,
                         const int32_t* __restrict__ bci, const double* __restrict__ bv, int wmax, int cmax,
                         int64_t* __restrict__ rowcnt, int* maxc, const int64_t* __restrict__ crp,
                         int32_t* __restrict__ cci, double* __restrict__ cv, int* flag) {
    extern __shared__ __align__(16) unsigned char sp_smem[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nwb = blockDim.x >> 5;
    const size_t per = (size_t)8 * wmax + (MODE >= SP_VALUES ? (size_t)8 * cmax : 0);
    unsigned char* base = sp_smem + per * wid;
    uint32_t* bits = reinterpret_cast<uint32_t*>(base);
    int32_t* pre = reinterpret_cast<int32_t*>(base + (size_t)4 * wmax);
    double* acc = reinterpret_cast<double*>(base + (size_t)8 * wmax);
    int best = 0;
    for (int i = blockIdx.x * nwb + wid; i < n; i += gridDim.x * nwb) {
        int lo, hi;
        row_span(arp, aci, brp, bci, i, lane, lo, hi);
        const int W = hi >= lo ? ((hi - lo) >> 5) + 1 : 0;
        if (W > wmax) {  // sized from k_sp_span; cannot happen
            if (lane == 0) atomicOr(flag, 1);
            continue;
        }
        for (int w = lane; w < W; w += 32) bits[w] = 0u;
        __syncwarp();
        const int64_t a0 = arp[i], a1 = arp[i + 1];
        mark_row(aci, brp, bci, a0, a1, lo, lane, bits);
        __syncwarp();
        // exclusive prefix of the words' popcounts (lane-contiguous chunks)
        const int chunk = (W + 31) >> 5;
        const int w0 = min(W, lane * chunk), w1 = min(W, w0 + chunk);
        int mine = 0;
        for (int w = w0; w < w1; w++) mine += __popc(bits[w]);
        int xs = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, xs, o);
            if (lane >= o) xs += y;
        }
        const int total = __shfl_sync(FULL, xs, 31);
        int run = xs - mine;
        for (int w = w0; w < w1; w++) {
            pre[w] = run;
            run += __popc(bits[w]);
        }
        __syncwarp();
        if (MODE == SP_COUNT) {
            if (lane == 0) rowcnt[i] = total;
            best = max(best, total);
            continue;
        }
        if (total > cmax && MODE >= SP_VALUES) {  // sized from the counting pass; cannot happen
            if (lane == 0) atomicOr(flag, 2);
            continue;
        }
        const int64_t cb = crp[i];
        for (int w = lane; w < W; w += 32) {
            uint32_t m = bits[w];
            int pos = pre[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                cci[cb + pos++] = lo + (w << 5) + bit;
            }
        }
        if constexpr (MODE != SP_COLS) {
            for (int u = lane; u < total; u += 32) acc[u] = 0.0;
            __syncwarp();
            const unsigned below = (1u << lane) - 1u;
            for (int64_t tb = a0; tb < a1; tb += 32) {
                int64_t q0;
                int len, incl, tot;
                double a;
                chunk_open(aci, av, brp, bci, tb, a1, lane, MODE == SP_UPPER ? i : -1, q0, len, incl, tot, a);
                for (int fb = 0; fb < tot; fb += 32 * kSpBatch) {
                    int J[kSpBatch];
                    double x[kSpBatch], y[kSpBatch];
    #pragma unroll
                    for (int u = 0; u < kSpBatch; u++) {
                        const int f = fb + 32 * u + lane;
                        const int64_t q = chunk_item(f, q0, len, incl, a, x[u]);
                        J[u] = -1;
                        y[u] = 0.0;
                        if (f < tot) {
                            J[u] = bci[q] - lo;
                            y[u] = bv[q];
                        }
                    }
    #pragma unroll
                    for (int u = 0; u < kSpBatch; u++) {
                        if (fb + 32 * u >= tot) break;  // warp-uniform
                        int r = -1 - lane;
                        if (J[u] >= 0) r = pre[J[u] >> 5] + __popc(bits[J[u] >> 5] & ((1u << (J[u] & 31)) - 1u));
                        const unsigned grp = __match_any_sync(FULL, r);
                        const int pos = __popc(grp & below);
                        const int npos = __reduce_max_sync(FULL, (unsigned)pos);
                        const double prod = __dmul_rn(x[u], y[u]);
                        for (int k = 0; k <= npos; k++) {
                            if (r >= 0 && pos == k) acc[r] = __dadd_rn(acc[r], prod);
                            __syncwarp();
                        }
                    }
                }
        }
        for (int u = lane; u < total; u += 32) cv[cb + u] = acc[u];
        }
        __syncwarp();
    }
    if (MODE == SP_COUNT) {
        best = __reduce_max_sync(FULL, best);
        if (lane == 0 && best > 0) atomicMax(maxc, best);
    }
}

// The same passes with one block of BT threads per output row (see the
// file header).  Shared memory: bits[wmax], pre[wmax], acc[cmax] (value
// modes), then the staged A entries of the numeric pass (B range start and
// length, value) and a reduction scratch.  With gbits (global, wmax words
// per row) the counting pass stores each row's bitmap and the later passes
// load it instead of marking the row again.
template <int MODE, int BT>
__global__ void __launch_bounds__(BT) k_sp_row_blk(int n, const int64_t* __restrict__ arp,
                                                   const int32_t* __restrict__ aci, const double* __restrict__ av,
                                                   const int64_t* __restrict__ brp, const int32_t* __restrict__ bci,
                                                   const double* __restrict__ bv, int wmax, int cmax,
                                                   int64_t* __restrict__ rowcnt, int* maxc,
                                                   const int64_t* __restrict__ crp, int32_t* __restrict__ cci,
                                                   double* __restrict__ cv, uint32_t* gbits, int* flag) {
    extern __shared__ __align__(16) unsigned char sp_smem[];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = BT / 32;
    uint32_t* bits = reinterpret_cast<uint32_t*>(sp_smem);
    int32_t* pre = reinterpret_cast<int32_t*>(sp_smem + (size_t)4 * wmax);
    double* acc = reinterpret_cast<double*>(sp_smem + (size_t)8 * wmax);
    unsigned char* tail = sp_smem + (size_t)8 * wmax + (MODE >= SP_VALUES ? (size_t)8 * cmax : 0);
    int64_t* sq0 = reinterpret_cast<int64_t*>(tail);
    double* sa = reinterpret_cast<double*>(tail + 8 * BT);
    int* slen = reinterpret_cast<int*>(tail + 16 * BT);
    int* red = reinterpret_cast<int*>(tail + 20 * BT);  // [0..NW) lo, [NW..2NW) hi, [2NW] total
    int best = 0;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t a0 = arp[i], a1 = arp[i + 1];
        // column span of the row
        int l = 0x7fffffff, hmax = -1;
        for (int64_t t = a0 + tid; t < a1; t += BT) {
            const int k = aci[t];
            const int64_t b0 = brp[k], b1 = brp[k + 1];
            if (b1 > b0) {
                l = min(l, bci[b0]);
                hmax = max(hmax, bci[b1 - 1]);
            }
        }
        l = __reduce_min_sync(FULL, l);
        hmax = __reduce_max_sync(FULL, hmax);
        if (lane == 0) {
            red[wid] = l;
            red[NW + wid] = hmax;
        }
        __syncthreads();
        int lo = red[0], hi = red[NW];
#pragma unroll
        for (int w = 1; w < NW; w++) {
            lo = min(lo, red[w]);
            hi = max(hi, red[NW + w]);
        }
        const int W = hi >= lo ? ((hi - lo) >> 5) + 1 : 0;
        if (W > wmax) {  // sized from k_sp_span; cannot happen
            if (tid == 0) atomicOr(flag, 1);
            __syncthreads();
            continue;
        }
        uint32_t* gb = gbits ? gbits + (size_t)i * wmax : nullptr;
        if (gb && MODE != SP_COUNT) {  // the counting pass's bitmap
            for (int w = tid; w < W; w += BT) bits[w] = gb[w];
        } else {
            for (int w = tid; w < W; w += BT) bits[w] = 0u;
            __syncthreads();
            // mark: warp wid takes A's entries a0 + wid, a0 + wid + NW, ...
            for (int64_t t = a0 + wid; t < a1; t += NW) {
                const int k = aci[t];
                const int64_t b0 = brp[k], b1 = brp[k + 1];
                for (int64_t qb = b0; qb < b1; qb += 32 * kSpUnroll) {  // warp-uniform trip count
                    int J[kSpUnroll];
#pragma unroll
                    for (int u = 0; u < kSpUnroll; u++) {
                        const int64_t q = qb + lane + 32 * u;
                        J[u] = q < b1 ? bci[q] - lo : -1;
                    }
#pragma unroll
                    for (int u = 0; u < kSpUnroll; u++)
                        if (J[u] >= 0) atomicOr(&bits[J[u] >> 5], 1u << (J[u] & 31));
                }
            }
        }
        __syncthreads();
        if (MODE == SP_COUNT && gb)
            for (int w = tid; w < W; w += BT) gb[w] = bits[w];
        // exclusive prefix of the words' popcounts (warp 0, lane-contiguous chunks)
        if (wid == 0) {
            const int chunk = (W + 31) >> 5;
            const int w0 = min(W, lane * chunk), w1 = min(W, w0 + chunk);
            int mine = 0;
            for (int w = w0; w < w1; w++) mine += __popc(bits[w]);
            int xs = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, xs, o);
                if (lane >= o) xs += y;
            }
            int run = xs - mine;
            for (int w = w0; w < w1; w++) {
                pre[w] = run;
                run += __popc(bits[w]);
            }
            if (lane == 31) red[2 * NW] = xs;
        }
        __syncthreads();
        const int total = red[2 * NW];
        if (MODE == SP_COUNT) {
            if (tid == 0) rowcnt[i] = total;
            best = max(best, total);
            __syncthreads();
            continue;
        }
        if (total > cmax && MODE >= SP_VALUES) {  // sized from the counting pass; cannot happen
            if (tid == 0) atomicOr(flag, 2);
            __syncthreads();
            continue;
        }
        const int64_t cb = crp[i];
        for (int w = tid; w < W; w += BT) {
            uint32_t m = bits[w];
            int pos = pre[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                cci[cb + pos++] = lo + (w << 5) + bit;
            }
        }
        if constexpr (MODE != SP_COLS) {
            for (int u = tid; u < total; u += BT) acc[u] = 0.0;
            for (int64_t tb = a0; tb < a1; tb += BT) {
                const int nt = (int)min((int64_t)BT, a1 - tb);
                __syncthreads();  // the previous stage's entries are consumed
                if (tid < nt) {
                    const int64_t t = tb + tid;
                    const int k = aci[t];
                    int64_t b0 = brp[k];
                    const int64_t b1 = brp[k + 1];
                    if (MODE == SP_UPPER) {  // first column >= i
                        int64_t hb = b1;
                        while (b0 < hb) {
                            const int64_t mid = (b0 + hb) >> 1;
                            if (bci[mid] < i) b0 = mid + 1;
                            else hb = mid;
                        }
                    }
                    sq0[tid] = b0;
                    slen[tid] = (int)(b1 - b0);
                    sa[tid] = av[t];
                }
                __syncthreads();
                for (int u = 0; u < nt; u++) {
                    const int64_t q0 = sq0[u];
                    const int len = slen[u];
                    const double a = sa[u];
                    for (int x = tid; x < len; x += BT * kSpUnroll) {
                        int J[kSpUnroll];
                        double y[kSpUnroll];
    #pragma unroll
                        for (int v = 0; v < kSpUnroll; v++) {
                            const int xv = x + BT * v;
                            J[v] = xv < len ? bci[q0 + xv] - lo : -1;
                            y[v] = xv < len ? bv[q0 + xv] : 0.0;
                        }
    #pragma unroll
                        for (int v = 0; v < kSpUnroll; v++)
                            if (J[v] >= 0) {
                                const int r = pre[J[v] >> 5] + __popc(bits[J[v] >> 5] & ((1u << (J[v] & 31)) - 1u));
                                acc[r] = __dadd_rn(acc[r], __dmul_rn(a, y[v]));
                            }
                    }
                    __syncthreads();  // successive t in ascending order
                }
        }
        for (int u = tid; u < total; u += BT) cv[cb + u] = acc[u];
        }
        __syncthreads();
    }
    if (MODE == SP_COUNT) {
        best = __reduce_max_sync(FULL, best);
        if (lane == 0 && best > 0) atomicMax(maxc, best);
    }
}

// P_bar values from the K P values (same pattern), in place:
// P_bar(i, J) = (J == agg(i) ? p_i : 0) - (theta_i / d_i) kp_iJ.
__global__ void k_sp_pbar(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, double* v,
                          const int32_t* __restrict__ agg, const double* __restrict__ pval,
                          const double* __restrict__ theta, double theta_c, const double* __restrict__ dl1) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const double t = __ddiv_rn(theta ? theta[i] : theta_c, dl1[i]);
        const int ai = agg[i];
        const double pi = pval[i];
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32)
            v[k] = __dsub_rn(ci[k] == ai ? pi : 0.0, __dmul_rn(t, v[k]));
    }
}

// Values of P_bar^T (pattern already listed): entry (J, a) = P_bar(a, J),
// found by binary search in P_bar's row a.
__global__ void k_sp_tvals(int nc, const int64_t* __restrict__ trp, const int32_t* __restrict__ tci, double* tv,
                           const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, int* flag) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int J = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; J < nc; J += nw) {
        for (int64_t k = trp[J] + lane; k < trp[J + 1]; k += 32) {
            const int a = tci[k];
            int64_t lo = rp[a], hi = rp[a + 1] - 1, pos = -1;
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int c = ci[mid];
                if (c == J) {
                    pos = mid;
                    break;
                }
                if (c < J) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0) atomicOr(flag, 4);
            tv[k] = pos < 0 ? 0.0 : v[pos];
        }
    }
}

// int64 row pointers [i] = i (the tentative P as CSR, one entry per row)
__global__ void k_sp_iota(int n, int64_t* rp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) rp[i] = i;
}

// int64 copy of int32 offsets
__global__ void k_sp_widen(int n, const int32_t* __restrict__ in, int64_t* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

// P^T of a matching pass (coarse row I: member mem0[I], and mem1[I] when
// >= 0; ascending) as CSR: counts, then columns and values
__global__ void k_sp_pairs_count(int nc, const int32_t* __restrict__ mem1, int64_t* cnt) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I < nc) cnt[I] = mem1[I] >= 0 ? 2 : 1;
}

__global__ void k_sp_pairs_fill(int nc, const int32_t* __restrict__ mem0, const int32_t* __restrict__ mem1,
                                const double* __restrict__ pval, const int64_t* __restrict__ rp, int32_t* ci,
                                double* v) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    const int64_t k = rp[I];
    const int a = mem0[I], b = mem1[I];
    const int lo = (b >= 0 && b < a) ? b : a, hi = (b >= 0 && b < a) ? a : b;
    ci[k] = lo;
    v[k] = pval[lo];
    if (b >= 0) {
        ci[k + 1] = hi;
        v[k + 1] = pval[hi];
    }
}

// ---------------------------------------------------------------- V-cycle
// f_c[I] = sum over P_bar^T row I of P_bar(a, I) r_a; x_c = f_c / d_c when
// x_c is given (pre-smoothing of the next level from zero).
template <typename A>
__global__ void __launch_bounds__(kBlock) k_sp_restrict(int nc, const int64_t* __restrict__ trp,
                                                         const int32_t* __restrict__ tci,
                                                         const double* __restrict__ tv, const A* __restrict__ r,
                                                         A* fc, A* xc, const A* __restrict__ invdc,
                                                         const SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; I < nc; I += nw) {
        A s = A(0);
        for (int64_t k = trp[I] + lane; k < trp[I + 1]; k += 32) s = fma((A)tv[k], r[tci[k]], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) {
            fc[I] = s;
            if (xc) xc[I] = s * invdc[I];
        }
    }
}

// x_f[i] += sum over P_bar row i of P_bar(i, J) y_J
template <typename A>
__global__ void __launch_bounds__(kBlock) k_sp_prolong(int n, const int64_t* __restrict__ rp,
                                                        const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                        const A* __restrict__ y, A* xf, const SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        A s = A(0);
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) s = fma((A)v[k], y[ci[k]], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) xf[i] += s;
    }
}

// coarsest level: e = A^-1 f (dense FP64 symmetric inverse, a warp per row)
template <typename A>
__global__ void __launch_bounds__(kBlock) k_sp_coarse(int n, const double* __restrict__ Ainv,
                                                       const A* __restrict__ f, A* e, const SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I >= n) return;
    const double* row = Ainv + (int64_t)I * n;
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s = fma(row[j], (double)f[j], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    if (lane == 0) e[I] = (A)s;
}

inline int sp_blocks(int64_t rows, int warps) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((rows + warps - 1) / warps, (int64_t)1 << 20));
}

}  // namespace

// ------------------------------------------------------------------ host
// C = A B (CSR, sorted columns) in the given mode.  C.rowptr, C.col (and
// C.val in the value modes) are allocated with dev_alloc on s and recorded
// in h->allocs (owned by the hierarchy).  Device words dflag[0] and
// dflag[1] are this call's span and count maxima; dflag[2] accumulates the
// rows' error bits (cleared by the caller).  b_avg is B's average row
// length: from kSpLongRow on, the block-per-row kernel runs, else the
// warp-per-row one.  Returns AMG_OK, AMG_ERR_ROW_TOO_LONG (an output row
// needs more shared memory than a block has), AMG_ERR_NOMEM or AMG_ERR_CUDA.
static int spgemm(amg_hierarchy* h, int nA, const int64_t* arp, const int32_t* aci, const double* av,
                  const int64_t* brp, const int32_t* bci, const double* bv, double b_avg, int mode, DevCSR& C,
                  int* dflag, int64_t* scratch64) {
    cudaStream_t s = h->s;
    int* hflag = h->flag_host;
    auto fail = [](cudaError_t e) { return e == cudaErrorMemoryAllocation ? AMG_ERR_NOMEM : AMG_ERR_CUDA; };
#define SP_CK(expr)                                 \
    do {                                            \
        cudaError_t e__ = (expr);                   \
        if (e__ != cudaSuccess) return fail(e__);   \
    } while (0)
    auto halloc = [&](void** p, size_t bytes) {
        cudaError_t e = dev_alloc(p, bytes, s);
        if (e == cudaSuccess) h->allocs.push_back(*p);
        return e;
    };
    int dev = 0, smem_optin = 0;
    SP_CK(cudaGetDevice(&dev));
    SP_CK(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    C = DevCSR{};
    C.n = nA;
    SP_CK(cudaMemsetAsync(dflag, 0, 2 * sizeof(int), s));
    k_sp_span<<<AMG_GRID(sp_blocks(nA, kWarpsPerBlock)), kBlock, 0, s>>>(nA, arp, aci, brp, bci, dflag);
    SP_CK(cudaGetLastError());
    SP_CK(cudaMemcpyAsync(hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    SP_CK(cudaStreamSynchronize(s));
    const int wmax = std::max(1, hflag[0]);
    SP_CK(halloc((void**)&C.rowptr, sizeof(int64_t) * ((size_t)nA + 1)));
    int64_t* rowcnt = nullptr;
    SP_CK(dev_alloc((void**)&rowcnt, sizeof(int64_t) * ((size_t)nA + 1), s));
    struct FreeCnt {
        int64_t* p;
        cudaStream_t s;
        ~FreeCnt() { cudaFreeAsync(p, s); }
    } free_cnt{rowcnt, s};
    // kernel by B's average row length: a warp per row (the tentative P), a
    // block of 64 threads (P_bar of the finest level), or of 256
    const int bt = b_avg >= kSpLongRow ? 256 : (b_avg >= kSpMidRow ? 64 : 0);
    const bool blk = bt > 0;
    // shared memory of the block-per-row kernel beyond bits/pre/acc: staged
    // A entries (8 + 8 + 4 bytes each) and the reduction scratch
    const size_t blk_tail = (size_t)20 * bt + 4 * (2 * (bt / 32) + 1) + 16;
    auto cfg = [&](auto kern, size_t bytes) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    auto blocks_blk = [&]() { return (int)std::max<int64_t>(1, std::min<int64_t>(nA, (int64_t)1 << 20)); };
    // the counting pass's row bitmaps, kept for the later pass when they fit the budget
    uint32_t* gbits = nullptr;
    if (blk && (size_t)nA * (size_t)wmax * 4 <= kSpBitsBudget &&
        dev_alloc((void**)&gbits, (size_t)nA * (size_t)wmax * 4 + 16, s) != cudaSuccess) {
        gbits = nullptr;  // no room: the later pass marks the rows again
        (void)cudaGetLastError();
    }
    struct FreeBits {
        uint32_t* p;
        cudaStream_t s;
        ~FreeBits() {
            if (p) cudaFreeAsync(p, s);
        }
    } free_bits{gbits, s};
    // launch of a block-per-row pass with BT threads
    auto run_blk = [&](auto mode_tag, auto bt_tag, size_t sm, int gb, int cm, int64_t* rc, int* mc) -> cudaError_t {
        constexpr int MODE = decltype(mode_tag)::value, BT = decltype(bt_tag)::value;
        cudaError_t e = cfg(k_sp_row_blk<MODE, BT>, sm);
        if (e != cudaSuccess) return e;
        k_sp_row_blk<MODE, BT><<<AMG_GRID(gb), BT, sm, s>>>(nA, arp, aci, av, brp, bci, bv, wmax, cm, rc, mc, C.rowptr,
                                                            C.col, C.val, gbits, dflag + 2);
        return cudaGetLastError();
    };
    auto blk_pass = [&](int m, size_t sm, int gb, int cm, int64_t* rc, int* mc) -> cudaError_t {
        using I64 = std::integral_constant<int, 64>;
        using I256 = std::integral_constant<int, 256>;
        switch (m) {
            case SP_COUNT:
                return bt == 64 ? run_blk(std::integral_constant<int, SP_COUNT>{}, I64{}, sm, gb, cm, rc, mc)
                                : run_blk(std::integral_constant<int, SP_COUNT>{}, I256{}, sm, gb, cm, rc, mc);
            case SP_COLS:
                return bt == 64 ? run_blk(std::integral_constant<int, SP_COLS>{}, I64{}, sm, gb, cm, rc, mc)
                                : run_blk(std::integral_constant<int, SP_COLS>{}, I256{}, sm, gb, cm, rc, mc);
            case SP_VALUES:
                return bt == 64 ? run_blk(std::integral_constant<int, SP_VALUES>{}, I64{}, sm, gb, cm, rc, mc)
                                : run_blk(std::integral_constant<int, SP_VALUES>{}, I256{}, sm, gb, cm, rc, mc);
            default:
                return bt == 64 ? run_blk(std::integral_constant<int, SP_UPPER>{}, I64{}, sm, gb, cm, rc, mc)
                                : run_blk(std::integral_constant<int, SP_UPPER>{}, I256{}, sm, gb, cm, rc, mc);
        }
    };
    size_t per = (size_t)8 * wmax;
    int warps = 0;
    if (blk) {
        if (per + blk_tail > (size_t)smem_optin) return AMG_ERR_ROW_TOO_LONG;
        SP_CK(blk_pass(SP_COUNT, per + blk_tail, blocks_blk(), 0, rowcnt, dflag + 1));
    } else {
        warps = (int)std::min<size_t>(kSpWarps, (size_t)smem_optin / per);
        if (warps < 1) return AMG_ERR_ROW_TOO_LONG;
        SP_CK(cfg(k_sp_row<SP_COUNT>, per * warps));
        k_sp_row<SP_COUNT><<<AMG_GRID(sp_blocks(nA, warps)), 32 * warps, per * warps, s>>>(
            nA, arp, aci, av, brp, bci, bv, wmax, 0, rowcnt, dflag + 1, nullptr, nullptr, nullptr, dflag + 2);
    }
    SP_CK(cudaGetLastError());
    SP_CK(launch_scan64(rowcnt, C.rowptr, nA, scratch64, s));
    SP_CK(cudaMemcpyAsync(hflag + 1, dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    SP_CK(cudaMemcpyAsync(reinterpret_cast<int64_t*>(hflag + 4), C.rowptr + nA, sizeof(int64_t),
                          cudaMemcpyDeviceToHost, s));
    SP_CK(cudaStreamSynchronize(s));
    const int cmax = std::max(1, hflag[1]);
    C.nnz = *reinterpret_cast<int64_t*>(hflag + 4);
    SP_CK(halloc((void**)&C.col, sizeof(int32_t) * ((size_t)C.nnz + 8)));
    if (mode >= SP_VALUES) SP_CK(halloc((void**)&C.val, sizeof(double) * ((size_t)C.nnz + 8)));
    per = (size_t)8 * wmax + (mode >= SP_VALUES ? (size_t)8 * cmax : 0);
    if (blk) {
        if (per + blk_tail > (size_t)smem_optin) return AMG_ERR_ROW_TOO_LONG;
        SP_CK(blk_pass(mode, per + blk_tail, blocks_blk(), cmax, nullptr, nullptr));
        return AMG_OK;
    }
    warps = (int)std::min<size_t>(kSpWarps, (size_t)smem_optin / per);
    if (warps < 1) return AMG_ERR_ROW_TOO_LONG;
    const int gb = sp_blocks(nA, warps);
    if (mode == SP_COLS) {
        SP_CK(cfg(k_sp_row<SP_COLS>, per * warps));
        k_sp_row<SP_COLS><<<AMG_GRID(gb), 32 * warps, per * warps, s>>>(nA, arp, aci, av, brp, bci, bv, wmax, cmax,
                                                                        nullptr, nullptr, C.rowptr, C.col, nullptr,
                                                                        dflag + 2);
    } else if (mode == SP_VALUES) {
        SP_CK(cfg(k_sp_row<SP_VALUES>, per * warps));
        k_sp_row<SP_VALUES><<<AMG_GRID(gb), 32 * warps, per * warps, s>>>(nA, arp, aci, av, brp, bci, bv, wmax,
                                                                          cmax, nullptr, nullptr, C.rowptr, C.col,
                                                                          C.val, dflag + 2);
    } else {
        SP_CK(cfg(k_sp_row<SP_UPPER>, per * warps));
        k_sp_row<SP_UPPER><<<AMG_GRID(gb), 32 * warps, per * warps, s>>>(nA, arp, aci, av, brp, bci, bv, wmax,
                                                                         cmax, nullptr, nullptr, C.rowptr, C.col,
                                                                         C.val, dflag + 2);
    }
    SP_CK(cudaGetLastError());
    return AMG_OK;
#undef SP_CK
}

// Release a matrix recorded in h->allocs (stream ordered).
static void drop(amg_hierarchy* h, void* p) {
    if (!p) return;
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) {
        cudaFreeAsync(p, h->s);
        h->allocs.erase(it);
    }
}

int smooth_level(amg_hierarchy* h, int l, DevCSR& Kc_out) {
    cudaStream_t s = h->s;
    Level& F = h->lev[l];
    const DevCSR& K = F.A;
    const int n = K.n, nc = F.nc;
    int* dflag = h->flag + 8;  // [8] span, [9] count, [10] error bits
    if (cudaMemsetAsync(h->flag + 10, 0, sizeof(int), s) != cudaSuccess) return AMG_ERR_CUDA;
    int64_t *scr = nullptr, *prp = nullptr, *mrp = nullptr;
    const size_t scr_n = scan64_scratch(std::max(n, nc)) + 1;
    struct Tmp3 {
        void* p[3] = {};
        cudaStream_t s;
        ~Tmp3() {
            for (void* q : p)
                if (q) cudaFreeAsync(q, s);
        }
    } tmp{{}, s};
    if (dev_alloc((void**)&scr, sizeof(int64_t) * scr_n, s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[0] = scr;
    if (dev_alloc((void**)&prp, sizeof(int64_t) * ((size_t)n + 1), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[1] = prp;
    if (dev_alloc((void**)&mrp, sizeof(int64_t) * ((size_t)nc + 1), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[2] = mrp;
    // the tentative P as CSR (one entry per row), P^T through the member lists
    k_sp_iota<<<AMG_GRID((n + 1 + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, prp);
    k_sp_widen<<<AMG_GRID((nc + 1 + kBlock - 1) / kBlock), kBlock, 0, s>>>(nc + 1, F.mem_ptr, mrp);
    // K P, then P_bar in place
    int rc = spgemm(h, n, K.rowptr, K.col, K.val, prp, F.agg, F.pval, 1.0, SP_VALUES, F.sp, dflag, scr);
    if (rc != AMG_OK) return rc;
    if (l == 0) {  // K P of level 0 is kept: theta rescales it (training of the smoothing weights)
        if (dev_alloc((void**)&F.kp, sizeof(double) * ((size_t)F.sp.nnz + 8), s) != cudaSuccess) return AMG_ERR_NOMEM;
        h->allocs.push_back(F.kp);
        if (cudaMemcpyAsync(F.kp, F.sp.val, sizeof(double) * F.sp.nnz, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return AMG_ERR_CUDA;
    }
    const double* theta = (l == 0) ? (h->theta0 ? h->theta0 : h->o.smooth_theta) : nullptr;
    k_sp_pbar<<<AMG_GRID(sp_blocks(n, kWarpsPerBlock)), kBlock, 0, s>>>(n, F.sp.rowptr, F.sp.col, F.sp.val, F.agg,
                                                                        F.pval, theta, h->o.smooth_omega, F.dl1);
    // P_bar^T: the pattern of P^T K (the members' rows of K), values by search
    rc = spgemm(h, nc, mrp, F.mem_idx, nullptr, K.rowptr, K.col, nullptr, (double)K.nnz / std::max(n, 1), SP_COLS,
                F.spT, dflag, scr);
    if (rc != AMG_OK) return rc;
    if (dev_alloc((void**)&F.spT.val, sizeof(double) * ((size_t)F.spT.nnz + 8), s) != cudaSuccess)
        return AMG_ERR_NOMEM;
    h->allocs.push_back(F.spT.val);
    k_sp_tvals<<<AMG_GRID(sp_blocks(nc, kWarpsPerBlock)), kBlock, 0, s>>>(nc, F.spT.rowptr, F.spT.col, F.spT.val,
                                                                         F.sp.rowptr, F.sp.col, F.sp.val, dflag + 2);
    // T = K P_bar, K_c = P_bar^T T (upper triangle), mirrored
    DevCSR T, Kc;
    rc = spgemm(h, n, K.rowptr, K.col, K.val, F.sp.rowptr, F.sp.col, F.sp.val, (double)F.sp.nnz / std::max(n, 1),
                    SP_VALUES, T, dflag, scr);
    if (rc == AMG_OK)
        rc = spgemm(h, nc, F.spT.rowptr, F.spT.col, F.spT.val, T.rowptr, T.col, T.val,
                    (double)T.nnz / std::max(n, 1), SP_UPPER, Kc, dflag, scr);
    drop(h, T.rowptr);
    drop(h, T.col);
    drop(h, T.val);
    if (rc != AMG_OK) return rc;
    // the mirror's error word is the hierarchy's deferred Galerkin check (flag[3])
    if (launch_galerkin_mirror(Kc, h->flag + 3, s) != cudaSuccess) return AMG_ERR_CUDA;
    if (cudaMemcpyAsync(h->flag_host, h->flag + 10, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMG_ERR_CUDA;
    if (h->flag_host[0]) return AMG_ERR_CUDA;  // a row outgrew its sizing, or a transpose entry was missing
    Kc_out = Kc;
    F.smoothed = 1;
    return AMG_OK;
}

int galerkin_pass_spgemm(amg_hierarchy* h, const DevCSR& A, const int32_t* agg, const double* pval,
                         const int32_t* mem0, const int32_t* mem1, int nc, DevCSR& C) {
    cudaStream_t s = h->s;
    const int n = A.n;
    int* dflag = h->flag + 8;
    if (cudaMemsetAsync(h->flag + 10, 0, sizeof(int), s) != cudaSuccess) return AMG_ERR_CUDA;
    struct Tmp {
        void* p[5] = {};
        cudaStream_t s;
        ~Tmp() {
            for (void* q : p)
                if (q) cudaFreeAsync(q, s);
        }
    } tmp{{}, s};
    int64_t *scr = nullptr, *prp = nullptr, *trp = nullptr, *cnt = nullptr;
    int32_t* tci = nullptr;
    double* tv = nullptr;
    const size_t scr_n = scan64_scratch(std::max(n, nc)) + 1;
    if (dev_alloc((void**)&scr, sizeof(int64_t) * scr_n, s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[0] = scr;
    if (dev_alloc((void**)&prp, sizeof(int64_t) * ((size_t)n + 1), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[1] = prp;
    if (dev_alloc((void**)&trp, sizeof(int64_t) * ((size_t)nc + 1), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[2] = trp;
    if (dev_alloc((void**)&cnt, sizeof(int64_t) * ((size_t)nc + 1), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[3] = cnt;
    if (dev_alloc((void**)&tci, sizeof(int32_t) * (2 * (size_t)nc + 8), s) != cudaSuccess) return AMG_ERR_NOMEM;
    tmp.p[4] = tci;
    if (dev_alloc((void**)&tv, sizeof(double) * (2 * (size_t)nc + 8), s) != cudaSuccess) return AMG_ERR_NOMEM;
    struct FreeV {
        double* p;
        cudaStream_t s;
        ~FreeV() { cudaFreeAsync(p, s); }
    } free_tv{tv, s};
    k_sp_iota<<<AMG_GRID((n + 1 + kBlock - 1) / kBlock), kBlock, 0, s>>>(n, prp);
    k_sp_pairs_count<<<AMG_GRID((nc + kBlock - 1) / kBlock), kBlock, 0, s>>>(nc, mem1, cnt);
    if (launch_scan64(cnt, trp, nc, scr, s) != cudaSuccess) return AMG_ERR_CUDA;
    k_sp_pairs_fill<<<AMG_GRID((nc + kBlock - 1) / kBlock), kBlock, 0, s>>>(nc, mem0, mem1, pval, trp, tci, tv);
    DevCSR T;
    int rc = spgemm(h, n, A.rowptr, A.col, A.val, prp, agg, pval, 1.0, SP_VALUES, T, dflag, scr);
    if (rc == AMG_OK) rc = spgemm(h, nc, trp, tci, tv, T.rowptr, T.col, T.val, (double)T.nnz / std::max(n, 1), SP_UPPER, C, dflag,
                    scr);
    drop(h, T.rowptr);
    drop(h, T.col);
    drop(h, T.val);
    if (rc != AMG_OK) return rc;
    if (launch_galerkin_mirror(C, h->flag + 3, s) != cudaSuccess) return AMG_ERR_CUDA;
    if (cudaMemcpyAsync(h->flag_host, h->flag + 10, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMG_ERR_CUDA;
    return h->flag_host[0] ? AMG_ERR_CUDA : AMG_OK;
}

int smooth_recompute(amg_hierarchy* h, const double* theta) {
    cudaStream_t s = h->s;
    Level& F = h->lev[0];
    Level& C = h->lev[1];
    if (!F.smoothed || !F.kp) return AMG_ERR_ARG;
    const DevCSR& K = F.A;
    const int n = K.n, nc = F.nc;
    int* dflag = h->flag + 8;
    if (cudaMemsetAsync(h->flag + 10, 0, sizeof(int), s) != cudaSuccess) return AMG_ERR_CUDA;
    // P_bar values from K P and theta, and its transpose's values
    if (cudaMemcpyAsync(F.sp.val, F.kp, sizeof(double) * F.sp.nnz, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return AMG_ERR_CUDA;
    k_sp_pbar<<<AMG_GRID(sp_blocks(n, kWarpsPerBlock)), kBlock, 0, s>>>(n, F.sp.rowptr, F.sp.col, F.sp.val, F.agg,
                                                                        F.pval, theta, h->o.smooth_omega, F.dl1);
    k_sp_tvals<<<AMG_GRID(sp_blocks(nc, kWarpsPerBlock)), kBlock, 0, s>>>(nc, F.spT.rowptr, F.spT.col, F.spT.val,
                                                                         F.sp.rowptr, F.sp.col, F.sp.val, dflag + 2);
    int64_t* scr = nullptr;
    if (dev_alloc((void**)&scr, sizeof(int64_t) * (scan64_scratch(std::max(n, nc)) + 1), s) != cudaSuccess)
        return AMG_ERR_NOMEM;
    DevCSR T, Kc;
    int rc = spgemm(h, n, K.rowptr, K.col, K.val, F.sp.rowptr, F.sp.col, F.sp.val, (double)F.sp.nnz / std::max(n, 1),
                    SP_VALUES, T, dflag, scr);
    if (rc == AMG_OK)
        rc = spgemm(h, nc, F.spT.rowptr, F.spT.col, F.spT.val, T.rowptr, T.col, T.val,
                    (double)T.nnz / std::max(n, 1), SP_UPPER, Kc, dflag, scr);
    cudaFreeAsync(scr, s);
    drop(h, T.rowptr);
    drop(h, T.col);
    drop(h, T.val);
    if (rc == AMG_OK && (Kc.nnz != C.A.nnz || Kc.n != C.A.n)) rc = AMG_ERR_CUDA;  // same structural pattern
    if (rc == AMG_OK && launch_galerkin_mirror(Kc, h->flag + 3, s) != cudaSuccess) rc = AMG_ERR_CUDA;
    if (rc == AMG_OK &&
        cudaMemcpyAsync(C.A.val, Kc.val, sizeof(double) * Kc.nnz, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        rc = AMG_ERR_CUDA;
    drop(h, Kc.rowptr);
    drop(h, Kc.col);
    drop(h, Kc.val);
    if (rc != AMG_OK) return rc;
    if (cudaMemcpyAsync(h->flag_host, h->flag + 10, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return AMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMG_ERR_CUDA;
    return h->flag_host[0] ? AMG_ERR_CUDA : AMG_OK;
}

template <typename A>
void sp_restrict(const Level& F, const Level& C, const A* r, A* fc, A* xc, const A* invdc, const SolveState* st,
                 cudaStream_t s) {
    launch_pdl(k_sp_restrict<A>, sp_blocks(C.A.n, kWarpsPerBlock), kBlock, 0, s, C.A.n, F.spT.rowptr, F.spT.col,
               F.spT.val, r, fc, xc, invdc, st);
}

template <typename A>
void sp_prolong(const Level& F, const A* y, A* xf, const SolveState* st, cudaStream_t s) {
    launch_pdl(k_sp_prolong<A>, sp_blocks(F.A.n, kWarpsPerBlock), kBlock, 0, s, F.A.n, F.sp.rowptr, F.sp.col,
               F.sp.val, y, xf, st);
}

template <typename A>
void sp_coarse(int n, const double* Ainv, const A* f, A* e, const SolveState* st, cudaStream_t s) {
    launch_pdl(k_sp_coarse<A>, (int)(((int64_t)n * 32 + kBlock - 1) / kBlock), kBlock, 0, s, n, Ainv, f, e, st);
}

template void sp_restrict<double>(const Level&, const Level&, const double*, double*, double*, const double*,
                                  const SolveState*, cudaStream_t);
template void sp_restrict<float>(const Level&, const Level&, const float*, float*, float*, const float*,
                                 const SolveState*, cudaStream_t);
template void sp_prolong<double>(const Level&, const double*, double*, const SolveState*, cudaStream_t);
template void sp_prolong<float>(const Level&, const float*, float*, const SolveState*, cudaStream_t);
template void sp_coarse<double>(int, const double*, const double*, double*, const SolveState*, cudaStream_t);
template void sp_coarse<float>(int, const double*, const float*, float*, const SolveState*, cudaStream_t);

}  // namespace amg
