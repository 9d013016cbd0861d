// Setup kernels of the matching-based aggregation AMG (arXiv 2511.21268,
// Sec. 3.1 and 3.2).  Every floating-point result that steers the matching
// (l1 diagonal, test vector, edge weights, prolongator values, Galerkin
// values) is computed with explicitly rounded operations (__dadd_rn,
// __dmul_rn, __ddiv_rn, __dsqrt_rn) in a fixed order:
//   - row sums run left to right over the row's entries in column order,
//     starting from +0.0;
//   - c_ij is evaluated in the canonical (lo = min(i,j), hi = max(i,j))
//     order: c = 1 - ((2 k) w_lo) w_hi / (k_lolo (w_lo w_lo) + k_hihi (w_hi w_hi));
//   - K_c(I,J), I <= J, sums (p_a k_ab) p_b over a in I ascending, then b in
//     J ascending; K_c(J,I) copies K_c(I,J).
// so the hierarchy is reproducible bit for bit.
//
// GB300 issues about two FP64 FMAs per SM per clock, so ordered row sums are
// never computed redundantly across lanes: a warp folds 32 rows at once, each
// lane owning one row, after staging 32x32 tiles through shared memory with
// coalesced loads.
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {

namespace cg = cooperative_groups;

namespace {

constexpr unsigned FULL = 0xffffffffu;

int blocks_for(int64_t units, int per_block, int cap = 1 << 20) {
    int64_t b = (units + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

// ------------------------------------------------------------------ CSR check
// flag bits: 1 malformed (rowptr order, column range or order), 2 non-finite
// value, 4 missing diagonal.
__global__ void k_validate(int n, int64_t nnz, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const double* __restrict__ v, int* flag) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nw) {
        int64_t b = rp[i], e = rp[i + 1];
        int bad = 0;
        if (b > e || b < 0 || e > nnz) {
            if (lane == 0) atomicOr(flag, 1);
            continue;
        }
        bool has_diag = false;
        for (int64_t k = b + lane; k < e; k += 32) {
            int j = ci[k];
            if (j < 0 || j >= n) bad |= 1;
            if (k > b && ci[k - 1] >= j) bad |= 1;
            if (((dbits(v[k]) >> 52) & 0x7ff) == 0x7ff) bad |= 2;  // inf or NaN, decided on the bits
            if (j == i) has_diag = true;
        }
        bad = __reduce_or_sync(FULL, bad);
        if (!__any_sync(FULL, has_diag)) bad |= 4;
        if (lane == 0 && bad) atomicOr(flag, bad);
    }
}

// ------------------------------------------------------------- ordered folds
// Warp-cooperative left-to-right row folds.  The warp owns rows
// row0 .. row0+31; in each chunk of CW columns, every load instruction stages
// CW consecutive entries of 32 / CW rows into tile[row][column] (coalesced
// per row), then every lane adds the staged terms of its own row in order.
// Padding terms are +0.0, which leaves a sum that started at +0.0 unchanged.
// The chunk width does not change the sums.  A narrow chunk (8) keeps the
// tile at 2.3 KB per warp, so that many warps share an SM when the matrix has
// the rows to fill them (the lanes' sums are dependent chains, and the loads
// of other warps fill their gaps); with few rows a wide chunk (32) does the
// same work in fewer synchronised steps.
// |x| by clearing the sign bit (an integer operation, not an FP64 one).
__device__ __forceinline__ double abs_bits(double x) {
    return __longlong_as_double(dbits(x) & 0x7fffffffffffffffLL);
}

template <int CW, typename Term>
__device__ __forceinline__ double fold_rows(int row0, int n, const int64_t* __restrict__ rp,
                                            const int32_t* __restrict__ ci, const double* __restrict__ v, Term term,
                                            double (*tile)[CW + 1]) {
    constexpr int kRowsPerLoad = 32 / CW;
    constexpr int kLoads = 32 / kRowsPerLoad;  // entries a lane loads per chunk
    const int lane = threadIdx.x & 31;
    const int sub = lane % CW, rsel = lane / CW;
    const int my = row0 + lane;
    const int64_t mb = my < n ? rp[my] : 0;
    const int mlen = my < n ? (int)(rp[my + 1] - mb) : 0;
    const int maxlen = __reduce_max_sync(FULL, mlen);
    // chunk c's entries (column and value; column -1 past a row's end),
    // loaded one chunk ahead of the sums so that the loads of the next chunk
    // are in flight while this one is folded
    auto load = [&](int c, int (&jj)[kLoads], double (&xx)[kLoads]) {
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            const int r = u * kRowsPerLoad + rsel;
            const int64_t rb = __shfl_sync(FULL, mb, r);
            const int rl = __shfl_sync(FULL, mlen, r);
            const int t = c + sub;
            jj[u] = t < rl ? ci[rb + t] : -1;
            xx[u] = t < rl ? v[rb + t] : 0.0;
        }
    };
    double acc = 0.0;
    if constexpr (kLoads > 8) {  // wide chunks: no register room for a second chunk
        for (int c = 0; c < maxlen; c += CW) {
#pragma unroll 16
            for (int u = 0; u < kLoads; u++) {
                const int r = u * kRowsPerLoad + rsel;
                const int64_t rb = __shfl_sync(FULL, mb, r);
                const int rl = __shfl_sync(FULL, mlen, r);
                const int t = c + sub;
                tile[r][sub] = t < rl ? term(ci[rb + t], v[rb + t], row0 + r) : 0.0;
            }
            __syncwarp();
#pragma unroll 8
            for (int s = 0; s < CW; s++) acc = __dadd_rn(acc, tile[lane][s]);
            __syncwarp();
        }
        return acc;
    }
    int j0[kLoads], j1[kLoads];
    double x0[kLoads], x1[kLoads];
    if (maxlen > 0) load(0, j0, x0);
    for (int c = 0; c < maxlen; c += CW) {
        if (c + CW < maxlen) load(c + CW, j1, x1);  // warp-uniform
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            const int r = u * kRowsPerLoad + rsel;
            tile[r][sub] = j0[u] >= 0 ? term(j0[u], x0[u], row0 + r) : 0.0;
        }
        __syncwarp();
#pragma unroll 8
        for (int s = 0; s < CW; s++) acc = __dadd_rn(acc, tile[lane][s]);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            j0[u] = j1[u];
            x0[u] = x1[u];
        }
    }
    return acc;
}

// The same fold for the terms x_k g[j_k] with a gathered factor g (the test
// vector sweep's K w): three chunks in flight -- the entries of chunk c+2
// load, the gathers of chunk c+1 (whose columns arrived) issue, and chunk c
// is multiplied and folded -- so that neither the stream nor the gathers
// wait on the FP64 sums.  kLoads = 4 keeps the three stages in registers at
// four blocks per SM.
template <int CW>
__device__ __forceinline__ double fold_rows_gather(int row0, int n, const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                   const double* __restrict__ g, double (*tile)[CW + 1]) {
    constexpr int kRowsPerLoad = 32 / CW;
    constexpr int kLoads = 32 / kRowsPerLoad;
    const int lane = threadIdx.x & 31;
    const int sub = lane % CW, rsel = lane / CW;
    const int my = row0 + lane;
    const int64_t mb = my < n ? rp[my] : 0;
    const int mlen = my < n ? (int)(rp[my + 1] - mb) : 0;
    const int maxlen = __reduce_max_sync(FULL, mlen);
    auto load = [&](int c, int (&jj)[kLoads], double (&xx)[kLoads]) {
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            const int r = u * kRowsPerLoad + rsel;
            const int64_t rb = __shfl_sync(FULL, mb, r);
            const int rl = __shfl_sync(FULL, mlen, r);
            const int t = c + sub;
            jj[u] = t < rl ? ci[rb + t] : -1;
            xx[u] = t < rl ? v[rb + t] : 0.0;
        }
    };
    auto gather = [&](const int (&jj)[kLoads], double (&gg)[kLoads]) {
#pragma unroll
        for (int u = 0; u < kLoads; u++) gg[u] = jj[u] >= 0 ? g[jj[u]] : 0.0;
    };
    int j1[kLoads], j2[kLoads];
    double x0[kLoads], g0[kLoads], x1[kLoads], g1[kLoads], x2[kLoads];
#pragma unroll
    for (int u = 0; u < kLoads; u++) {
        j1[u] = j2[u] = -1;
        x1[u] = x2[u] = g1[u] = 0.0;
    }
    double acc = 0.0;
    if (maxlen <= 0) return acc;
    {
        int j0[kLoads];
        load(0, j0, x0);
        if (CW < maxlen) load(CW, j1, x1);
        gather(j0, g0);
    }
    for (int c = 0; c < maxlen; c += CW) {
        if (c + 2 * CW < maxlen) load(c + 2 * CW, j2, x2);  // warp-uniform
        if (c + CW < maxlen) gather(j1, g1);
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            const int r = u * kRowsPerLoad + rsel;
            tile[r][sub] = __dmul_rn(x0[u], g0[u]);  // x = 0, g = 0 past a row's end: +0
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < CW; s++) acc = __dadd_rn(acc, tile[lane][s]);
        __syncwarp();
#pragma unroll
        for (int u = 0; u < kLoads; u++) {
            x0[u] = x1[u];
            g0[u] = g1[u];
            j1[u] = j2[u];
            x1[u] = x2[u];
        }
    }
    return acc;
}

// Chunk width of the folds: narrow when the rows give every SM at least 32
// warps.
inline bool fold_narrow(int n, int num_sms) { return (int64_t)(n + 31) / 32 >= 32LL * num_sms; }

// l1 diagonal (Sec. 3.2): d_i = k_ii + sum_{j != i} |k_ij|.
template <int CW>
__global__ void __launch_bounds__(kBlock, 3) k_l1diag(int n, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                    double* kii, double* dl1, double* invd, int* flag) {
    __shared__ double tiles[kWarpsPerBlock][32][CW + 1];
    __shared__ double diags[kWarpsPerBlock][32];  // the rows' diagonal entries (0 when a row has none)
    double(*tile)[CW + 1] = tiles[threadIdx.x >> 5];
    double* dg = diags[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; row0 < n; row0 += nwarps * 32) {
        dg[lane] = 0.0;
        __syncwarp();
        auto term = [&](int j, double x, int row) -> double {
            if (j == row) {
                dg[row - row0] = x;
                return 0.0;
            }
            return abs_bits(x);
        };
        const double s = fold_rows<CW>(row0, n, rp, ci, v, term, tile);
        __syncwarp();
        const int i = row0 + lane;
        if (i < n) {
            const double d = dg[lane];
            kii[i] = d;
            if (!(d > 0.0)) atomicOr(flag, 1);
            const double dl = __dadd_rn(d, s);
            dl1[i] = dl;
            if (invd) invd[i] = __ddiv_rn(1.0, dl);
        }
    }
}

__global__ void k_diag(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const double* __restrict__ v, double* kii) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = warp; i < n; i += nw)
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32)
            if (ci[k] == i) kii[i] = v[k];
}

// Test vector start: U[0,1) from draw i of SplitMix64(seed), or all ones.
__global__ void k_testvec_init(int n, int kind, uint64_t seed, double* w) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = kind == 1 ? 1.0 : (double)(splitmix64_at(seed, (uint64_t)i) >> 11) * 0x1.0p-53;
}

// One relaxation sweep on K w = 0 (Sec. 3.1): w_i <- w_i - (K w)_i / d_i.
template <int CW>
__global__ void __launch_bounds__(kBlock, 4) k_testvec_sweep(int n, const int64_t* __restrict__ rp,
                                                           const int32_t* __restrict__ ci,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ dl1,
                                                           const double* __restrict__ w, double* wout) {
    __shared__ double tiles[kWarpsPerBlock][32][CW + 1];
    double(*tile)[CW + 1] = tiles[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int row0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; row0 < n; row0 += nwarps * 32) {
        double s;
        if constexpr (CW <= 4) {
            s = fold_rows_gather<CW>(row0, n, rp, ci, v, w, tile);
        } else {
            auto term = [&](int j, double x, int) -> double { return __dmul_rn(x, w[j]); };
            s = fold_rows<CW>(row0, n, rp, ci, v, term, tile);
        }
        const int i = row0 + lane;
        if (i < n) wout[i] = __dsub_rn(w[i], __ddiv_rn(s, dl1[i]));
    }
}

// ------------------------------------------------------------------ matching
// Tests of an FP64 value decided on its bits, so that they take no FP64
// instruction (GB300 issues about two FP64 operations per SM per clock):
// x != 0.0 (NaN counts as nonzero, as in IEEE comparison), x > 0.0 (true on
// (0, +inf], false for zeros, negatives and NaN), and x is NaN.
__device__ __forceinline__ bool nonzero_bits(double x) {
    return ((unsigned long long)dbits(x) << 1) != 0ull;
}
__device__ __forceinline__ bool positive_bits(double x) {
    const long long b = dbits(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}
// 2 x on the bits, no FP64 instruction: one more in the exponent field for
// normal x below the top binade; a subnormal's significand doubles (a carry
// into the exponent field makes it normal); the top binade overflows to
// infinity; infinity stays.  (NaN does not reach it: the matrix is checked
// for non-finite values.)
__device__ __forceinline__ double twice(double x) {
    const unsigned long long u = (unsigned long long)dbits(x);
    const unsigned long long sign = u & 0x8000000000000000ULL, mag = u & 0x7fffffffffffffffULL;
    const int e = (int)(mag >> 52);
    unsigned long long r = u;
    if (e == 0) r = sign | (mag << 1);
    else if (e < 2046) r = u + (1ULL << 52);
    else if (e == 2046) r = sign | 0x7ff0000000000000ULL;
    return __longlong_as_double((long long)r);
}
__device__ __forceinline__ bool nan_bits(double x) {
    return (dbits(x) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}

// Edge key of every stored entry: order_key(c_ij) (Eq. cij) for eligible
// edges, 0 otherwise.  Eligible: j != i, k_ij != 0, denominator > 0 and
// w_lo^2 + w_hi^2 > 0.  Each edge is evaluated once, from its upper entry
// (row i, column j > i), and the key is written to that entry and to its
// mirror (row j, column i; found by binary search).  flag bit 64: a mirror
// entry is missing (structurally unsymmetric matrix); flag bit 128: a mirror
// entry's value differs from the upper entry's in its bits (symmetric only up
// to rounding), which the Galerkin kernels need to know.
__global__ void k_edge_keys(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const double* __restrict__ v, const double* __restrict__ kii,
                            const double* __restrict__ w, uint64_t* key, int* flag) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    bool asym = false;  // some K(j,i) differs from K(i,j) in its bits
    for (int i = warp; i < n; i += nw) {
        const double wi = w[i];
        const double wi2 = __dmul_rn(wi, wi), kwi2 = __dmul_rn(kii[i], wi2);
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) {
            const int j = ci[k];
            if (j < i) continue;  // written by the owner of the upper entry
            if (j == i) {
                key[k] = 0;
                continue;
            }
            const double a = v[k];
            uint64_t out = 0;
            if (nonzero_bits(a)) {
                const double wj = w[j];
                const double wj2 = __dmul_rn(wj, wj);
                const double num = __dmul_rn(__dmul_rn(twice(a), wi), wj);
                const double den = __dadd_rn(kwi2, __dmul_rn(kii[j], wj2));
                // w_i^2 + w_j^2 > 0: both squares are +0, positive, +inf or NaN
                const bool nrm2_pos = !nan_bits(wi2) && !nan_bits(wj2) && (positive_bits(wi2) || positive_bits(wj2));
                if (positive_bits(den) && nrm2_pos) out = order_key(__dsub_rn(1.0, div_rn(num, den)));
            }
            key[k] = out;
            int64_t lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int cm = ci[mid];
                if (cm == i) {
                    pos = mid;
                    break;
                }
                if (cm < i) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0) {
                atomicOr(flag, 64);
            } else {
                key[pos] = out;
                asym |= __double_as_longlong(v[pos]) != __double_as_longlong(a);
            }
        }
    }
    if (__any_sync(FULL, asym) && lane == 0) atomicOr(flag, 128);
}

// Matching state: -1 active (unmatched, may still match), -2 dead (no
// active eligible neighbour left: singleton), >= 0 partner.
__global__ void k_match_init(int n, int32_t* state) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) state[i] = -1;
}

// "a heavier than b" under the strict order (key desc, lo asc, hi asc).
__device__ __forceinline__ bool heavier(uint64_t ka, int loa, int hia, uint64_t kb, int lob, int hib) {
    if (ka != kb) return ka > kb;
    if (loa != lob) return loa < lob;
    return hia < hib;
}

// Loads of the matching state, which the rounds of one cooperative launch
// write from other SMs: COHERENT loads bypass L1 (ld.global.cg), plain
// loads are used between separate launches.
template <bool COHERENT>
__device__ __forceinline__ int ld_match(const int* p) {
    if (COHERENT) return __ldcg(p);
    return *p;
}

// Every active vertex proposes to its heaviest eligible active neighbour.
// Round 0 covers every vertex (list NULL); later rounds the vertices the
// previous round left active (list, *count).  Warps gw = 0 .. nw-1 of the
// grid take one vertex at a time.
template <bool COHERENT>
__device__ __forceinline__ void match_propose(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                              const uint64_t* __restrict__ key, const int32_t* state, int32_t* cand,
                                              const int32_t* list, const int* count, int gw, int nw) {
    const int m = list ? ld_match<COHERENT>(count) : n;
    const int lane = threadIdx.x & 31;
    for (int idx = gw; idx < m; idx += nw) {
        const int i = list ? ld_match<COHERENT>(list + idx) : idx;
        // Active neighbours only leave between rounds, so the heaviest one of
        // the previous round is still the heaviest while it stays active.
        if (list) {
            const int c = ld_match<COHERENT>(cand + i);
            if (c >= 0 && ld_match<COHERENT>(state + c) == -1) continue;
        }
        uint64_t bk = 0;
        int blo = 0x7fffffff, bhi = 0x7fffffff, bj = -1;
        // four 32-entry chunks per step: their keys and columns, then the
        // neighbours' states, are loaded together (the heaviest edge does not
        // depend on the order the entries are seen in)
        const int64_t b0 = rp[i], b1 = rp[i + 1];
        for (int64_t kb = b0; kb < b1; kb += 128) {
            uint64_t kk[4];
            int jj[4], sj[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const int64_t k = kb + lane + 32 * u;
                kk[u] = k < b1 ? key[k] : 0;
                jj[u] = k < b1 ? ci[k] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; u++) sj[u] = kk[u] != 0 ? ld_match<COHERENT>(state + jj[u]) : 0;
#pragma unroll
            for (int u = 0; u < 4; u++) {
                if (kk[u] == 0 || sj[u] != -1) continue;
                const int j = jj[u];
                const int lo = min(i, j), hi = max(i, j);
                if (bj < 0 || heavier(kk[u], lo, hi, bk, blo, bhi)) {
                    bk = kk[u];
                    blo = lo;
                    bhi = hi;
                    bj = j;
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t ok = __shfl_xor_sync(FULL, bk, o);
            const int olo = __shfl_xor_sync(FULL, blo, o);
            const int ohi = __shfl_xor_sync(FULL, bhi, o);
            const int oj = __shfl_xor_sync(FULL, bj, o);
            if (oj >= 0 && (bj < 0 || heavier(ok, olo, ohi, bk, blo, bhi))) {
                bk = ok;
                blo = olo;
                bhi = ohi;
                bj = oj;
            }
        }
        if (lane == 0) cand[i] = bj;
    }
}

// Commit of a round over its active vertices (list_in, *count_in; round 0:
// all): mutual proposals pair, vertices without a candidate become
// singletons, the others stay active and are appended to list_out, whose
// length *count_out (zero on entry) is the round's active count.  The list's
// order depends on the atomics; nothing computed from it does.  Blocks
// blk = 0 .. nblk-1 take blockDim.x vertices at a time.
template <bool COHERENT>
__device__ __forceinline__ void match_commit(int n, const int32_t* cand, int32_t* state, const int32_t* list_in,
                                             const int* count_in, int32_t* list_out, int* count_out, int blk,
                                             int nblk) {
    const int m = list_in ? ld_match<COHERENT>(count_in) : n;
    const int lane = threadIdx.x & 31;
    for (int base = blk * blockDim.x; base < m; base += nblk * blockDim.x) {  // warp-uniform
        const int idx = base + threadIdx.x;
        int i = -1;
        bool keep = false;
        if (idx < m) {
            i = list_in ? ld_match<COHERENT>(list_in + idx) : idx;
            const int c = ld_match<COHERENT>(cand + i);
            if (c < 0) state[i] = -2;
            else if (ld_match<COHERENT>(cand + c) == i) state[i] = c;
            else keep = true;
        }
        const unsigned b = __ballot_sync(FULL, keep);
        int off = 0;
        if (lane == 0 && b) off = atomicAdd(count_out, __popc(b));
        off = __shfl_sync(FULL, off, 0);
        if (keep) list_out[off + __popc(b & ((1u << lane) - 1u))] = i;
    }
}

__global__ void k_match_propose(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const uint64_t* __restrict__ key, const int32_t* __restrict__ state,
                                int32_t* cand, const int32_t* __restrict__ list, const int* __restrict__ count) {
    match_propose<false>(n, rp, ci, key, state, cand, list, count, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                         (gridDim.x * blockDim.x) >> 5);
}

__global__ void k_match_commit(int n, const int32_t* __restrict__ cand, int32_t* state,
                               const int32_t* __restrict__ list_in, const int* __restrict__ count_in,
                               int32_t* list_out, int* count_out) {
    match_commit<false>(n, cand, state, list_in, count_in, list_out, count_out, blockIdx.x, gridDim.x);
}

// Every round of one matching pass in one cooperative launch: propose, grid
// barrier, commit, grid barrier, until a round leaves no vertex active or
// max_rounds rounds have run.  *rounds_out = the number of rounds run, or
// max_rounds + 1 if the last one still left active vertices.  The launch
// fits the grid to the blocks that can be resident at once, so the
// barriers cannot wait on a block that never runs.
__global__ void __launch_bounds__(kBlock) k_match_rounds_coop(int n, const int64_t* __restrict__ rp,
                                                              const int32_t* __restrict__ ci,
                                                              const uint64_t* __restrict__ key, int32_t* state,
                                                              int32_t* cand, int* active, int32_t* lists,
                                                              int max_rounds, int* rounds_out) {
    cg::grid_group g = cg::this_grid();
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int r = 0; r < max_rounds; r++) {
        const int32_t* lin = r > 0 ? lists + (size_t)((r - 1) & 1) * n : nullptr;
        const int* cin = r > 0 ? active + r - 1 : nullptr;
        match_propose<true>(n, rp, ci, key, state, cand, lin, cin, gw, nw);
        g.sync();
        match_commit<true>(n, cand, state, lin, cin, lists + (size_t)(r & 1) * n, active + r, blockIdx.x, gridDim.x);
        g.sync();
        if (__ldcg(active + r) == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *rounds_out = r + 1;
            return;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *rounds_out = max_rounds + 1;
}

__global__ void k_match_finish(int n, const int32_t* __restrict__ state, int32_t* mate, int32_t* leader) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int s = state[i];
        const int m = s >= 0 ? s : -1;
        mate[i] = m;
        leader[i] = (m < 0 || m > i) ? 1 : 0;
    }
}

// Aggregates (Eq. prolongation): coarse index = rank of the aggregate's
// smallest fine index; pair (i<j): p = (w_i, w_j) / sqrt(w_i^2 + w_j^2);
// singleton: p = sign(w_i) (+1 for 0).  Also w_c = P^T w.
__global__ void k_aggregate(int n, const int32_t* __restrict__ mate, const int32_t* __restrict__ cidx,
                            const double* __restrict__ w, int32_t* agg, double* pval, int32_t* mem0, int32_t* mem1,
                            double* wc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int j = mate[i];
        if (j >= 0 && j < i) continue;  // handled by the pair's leader
        const int I = cidx[i];
        const double wi = w[i];
        if (j < 0) {
            agg[i] = I;
            const double p = wi < 0.0 ? -1.0 : 1.0;
            pval[i] = p;
            mem0[I] = i;
            mem1[I] = -1;
            wc[I] = __dadd_rn(0.0, __dmul_rn(p, wi));
        } else {
            const double wj = w[j];
            const double nrm = __dsqrt_rn(__dadd_rn(__dmul_rn(wi, wi), __dmul_rn(wj, wj)));
            const double pi = __ddiv_rn(wi, nrm), pj = __ddiv_rn(wj, nrm);
            agg[i] = I;
            agg[j] = I;
            pval[i] = pi;
            pval[j] = pj;
            mem0[I] = i;
            mem1[I] = j;
            wc[I] = __dadd_rn(__dadd_rn(0.0, __dmul_rn(pi, wi)), __dmul_rn(pj, wj));
        }
    }
}

// ------------------------------------------------------------------ scans
// Three-phase exclusive scan: per-block scan of 1024 items, sequential scan
// of the block totals (one block looping in chunks), add-back.
template <typename T>
__device__ T block_exclusive_scan(T v, T* sh, T* total) {
    // sh: 1024 / 32 entries
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T s = lane < (int)(blockDim.x >> 5) ? sh[lane] : (T)0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (int)(blockDim.x >> 5)) sh[lane] = s;
    }
    __syncthreads();
    T pre = (wid > 0 ? sh[wid - 1] : (T)0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return pre;
}

template <typename T>
__global__ void k_scan_blocks(const T* __restrict__ in, T* out, int n, T* bsum) {
    __shared__ T sh[32];
    __shared__ T tot;
    const int base = blockIdx.x * 1024;
    T loc[4];
    T s = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int idx = base + threadIdx.x * 4 + q;
        loc[q] = idx < n ? in[idx] : (T)0;
        s += loc[q];
    }
    T pre = block_exclusive_scan<T>(s, sh, &tot);
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int idx = base + threadIdx.x * 4 + q;
        if (idx < n) out[idx] = pre;
        pre += loc[q];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <typename T>
__global__ void k_scan_sums(T* bsum, int nb, T* total) {
    __shared__ T sh[32];
    __shared__ T tot;
    T carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int idx = base + threadIdx.x;
        T v = idx < nb ? bsum[idx] : (T)0;
        T pre = block_exclusive_scan<T>(v, sh, &tot);
        if (idx < nb) bsum[idx] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename T>
__global__ void k_scan_add(T* out, int n, const T* __restrict__ bsum) {
    const int base = blockIdx.x * 1024;
    const T add = bsum[blockIdx.x];
    for (int q = threadIdx.x; q < 1024; q += blockDim.x) {
        int idx = base + q;
        if (idx < n) out[idx] += add;
    }
}

template <typename T>
cudaError_t scan_impl(const T* in, T* out, int n, T* total, T* scratch, cudaStream_t s) {
    const int nb = (n + 1023) / 1024;
    if (n <= 0) {
        if (total) AMG_TRY(cudaMemsetAsync(total, 0, sizeof(T), s));
        return cudaSuccess;
    }
    k_scan_blocks<T><<<AMG_GRID(nb), 256, 0, s>>>(in, out, n, scratch);
    k_scan_sums<T><<<AMG_GRID(1), 1024, 0, s>>>(scratch, nb, total);
    k_scan_add<T><<<AMG_GRID(nb), 256, 0, s>>>(out, n, scratch);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Galerkin
// One block per coarse row I with fine members a0 < a1 (a1 = -1 for a
// singleton).  Candidate t enumerates the entries of row a0 then row a1 in
// column order; key = (agg[col] << 32) | t.  After a bitonic sort by key,
// equal coarse columns J form segments whose elements are in canonical
// (a ascending, b ascending) order.
__device__ __forceinline__ int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

__device__ void block_bitonic_sort(uint64_t* a, int P) {
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const uint64_t x = a[t], y = a[u];
                    const bool up = (t & k) == 0;
                    if ((x > y) == up) {
                        a[t] = y;
                        a[u] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__device__ int load_candidates(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               const int32_t* __restrict__ agg, int a0, int a1, uint64_t* keys, int cap,
                               int* len0_out) {
    const int64_t b0 = rp[a0];
    const int len0 = (int)(rp[a0 + 1] - b0);
    const int64_t b1 = a1 >= 0 ? rp[a1] : 0;
    const int len1 = a1 >= 0 ? (int)(rp[a1 + 1] - b1) : 0;
    const int c = len0 + len1;
    *len0_out = len0;
    if (c > cap) return -1;
    const int P = pow2ceil(c);
    for (int t = threadIdx.x; t < P; t += blockDim.x) {
        uint64_t kk = ~0ULL;
        if (t < c) {
            const int j = t < len0 ? ci[b0 + t] : ci[b1 + (t - len0)];
            kk = ((uint64_t)(uint32_t)agg[j] << 32) | (uint32_t)t;
        }
        keys[t] = kk;
    }
    __syncthreads();
    block_bitonic_sort(keys, P);
    return c;
}

__global__ void k_galerkin_count(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const int32_t* __restrict__ agg, const int32_t* __restrict__ mem0,
                                 const int32_t* __restrict__ mem1, int cap, int64_t* rowcnt) {
    extern __shared__ uint64_t keys[];
    __shared__ int cnt;
    for (int I = blockIdx.x; I < nc; I += gridDim.x) {
        if (threadIdx.x == 0) cnt = 0;
        int len0;
        const int c = load_candidates(rp, ci, agg, mem0[I], mem1[I], keys, cap, &len0);
        if (c < 0) {
            if (threadIdx.x == 0) rowcnt[I] = -1;
            __syncthreads();
            continue;
        }
        int local = 0;
        for (int t = threadIdx.x; t < c; t += blockDim.x)
            if (t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32)) local++;
        local = __reduce_add_sync(FULL, local);
        if ((threadIdx.x & 31) == 0 && local) atomicAdd(&cnt, local);
        __syncthreads();
        if (threadIdx.x == 0) rowcnt[I] = cnt;
        __syncthreads();
    }
}

__global__ void k_galerkin_fill(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const double* __restrict__ v, const int32_t* __restrict__ agg,
                                const double* __restrict__ pval, const int32_t* __restrict__ mem0,
                                const int32_t* __restrict__ mem1, int cap, const int64_t* __restrict__ crp,
                                int32_t* cci, double* cv) {
    extern __shared__ uint64_t keys[];
    __shared__ int wsum[32];
    for (int I = blockIdx.x; I < nc; I += gridDim.x) {
        const int a0 = mem0[I], a1 = mem1[I];
        int len0;
        const int c = load_candidates(rp, ci, agg, a0, a1, keys, cap, &len0);
        if (c < 0) continue;  // reported by the count kernel
        const int64_t b0 = rp[a0], b1 = a1 >= 0 ? rp[a1] : 0;
        const double p0 = pval[a0], p1 = a1 >= 0 ? pval[a1] : 0.0;
        // segment index of each segment start = exclusive count of starts before it;
        // thread-contiguous chunks keep the scan simple
        const int per = (c + blockDim.x - 1) / blockDim.x;
        const int t0 = min(c, threadIdx.x * per), t1 = min(c, t0 + per);
        int mine = 0;
        for (int t = t0; t < t1; t++)
            if (t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32)) mine++;
        // block exclusive scan of `mine`
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int x = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int sv = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(FULL, sv, o);
                if (lane >= o) sv += y;
            }
            if (lane < (int)(blockDim.x >> 5)) wsum[lane] = sv;
        }
        __syncthreads();
        int seg = (wid > 0 ? wsum[wid - 1] : 0) + x - mine;
        const int64_t base = crp[I];
        for (int t = t0; t < t1; t++) {
            const uint32_t J = (uint32_t)(keys[t] >> 32);
            if (!(t == 0 || (keys[t] >> 32) != (keys[t - 1] >> 32))) continue;
            const int64_t o = base + seg;
            seg++;
            cci[o] = (int32_t)J;
            double acc = 0.0;
            if ((int)J >= I) {
                for (int u = t; u < c && (uint32_t)(keys[u] >> 32) == J; u++) {
                    const int q = (int)(uint32_t)keys[u];
                    const bool first = q < len0;
                    const int64_t k = first ? b0 + q : b1 + (q - len0);
                    const double pa = first ? p0 : p1;
                    const double term = __dmul_rn(__dmul_rn(pa, v[k]), pval[ci[k]]);
                    acc = __dadd_rn(acc, term);
                }
            }
            cv[o] = acc;
        }
        __syncthreads();
    }
}

// K_c(I,J) for J < I := K_c(J,I) (binary search of I in row J).
__global__ void k_galerkin_mirror(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, double* v,
                                  int* flag) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int I = warp; I < n; I += nw) {
        for (int64_t k = rp[I] + lane; k < rp[I + 1]; k += 32) {
            const int J = ci[k];
            if (J >= I) break;
            int64_t lo = rp[J], hi = rp[J + 1] - 1;
            int64_t pos = -1;
            while (lo <= hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int cm = ci[mid];
                if (cm == I) {
                    pos = mid;
                    break;
                }
                if (cm < I) lo = mid + 1;
                else hi = mid - 1;
            }
            if (pos < 0) atomicOr(flag, 8);
            else v[k] = v[pos];
        }
    }
}

// Galerkin without sorting candidates.  One block per coarse row I: the
// coarse columns J = agg[b] of the member rows' entries set bits of a
// shared-memory bitmap over [Jmin, Jmax]; prefix popcounts of the bitmap
// words give every J its position in the sorted row.  A coarse entry
// K_c(I,J) has at most four terms; term (a, b) goes to slot
// 2 * rank(a in I) + rank(b in J), so summing the slots in order is the
// canonical (a ascending, b ascending) order -- no sort, bit-exact.
__device__ __forceinline__ void block_minmax(int v_min, int v_max, int* smin, int* smax) {
    v_min = __reduce_min_sync(FULL, v_min);
    v_max = __reduce_max_sync(FULL, v_max);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(smin, v_min);
        atomicMax(smax, v_max);
    }
}

template <bool FILL>
__global__ void k_galerkin_bitmap(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                  const double* __restrict__ v, const int32_t* __restrict__ agg,
                                  const double* __restrict__ pval, const int32_t* __restrict__ mem0,
                                  const int32_t* __restrict__ mem1, int cap, int words, int64_t* rowcnt,
                                  const int64_t* __restrict__ crp, int32_t* cci, double* cv, int* flag) {
    extern __shared__ __align__(16) unsigned char gsm[];
    uint32_t* bits = reinterpret_cast<uint32_t*>(gsm);
    int32_t* pre = reinterpret_cast<int32_t*>(gsm + 4 * (size_t)words);
    int32_t* slot = reinterpret_cast<int32_t*>(gsm + 8 * (size_t)words);  // FILL: [cap][4]
    __shared__ int jmin, jmax, wsum[33];
    for (int I = blockIdx.x; I < nc; I += gridDim.x) {
        const int a0 = mem0[I], a1 = mem1[I];
        const int64_t b0 = rp[a0];
        const int len0 = (int)(rp[a0 + 1] - b0);
        const int64_t b1 = a1 >= 0 ? rp[a1] : 0;
        const int len1 = a1 >= 0 ? (int)(rp[a1 + 1] - b1) : 0;
        const int c = len0 + len1;
        if (threadIdx.x == 0) {
            jmin = 0x7fffffff;
            jmax = -1;
        }
        __syncthreads();
        int lmin = 0x7fffffff, lmax = -1;
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            const int J = agg[t < len0 ? ci[b0 + t] : ci[b1 + (t - len0)]];
            lmin = min(lmin, J);
            lmax = max(lmax, J);
        }
        block_minmax(lmin, lmax, &jmin, &jmax);
        __syncthreads();
        const int J0 = jmin;
        const int W = ((jmax - J0) >> 5) + 1;
        if (W > words || (FILL && c > cap)) {  // sized from the row statistics; cannot happen
            if (threadIdx.x == 0) atomicOr(flag, 32);
            __syncthreads();
            continue;
        }
        for (int w = threadIdx.x; w < W; w += blockDim.x) bits[w] = 0u;
        __syncthreads();
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            const int J = agg[t < len0 ? ci[b0 + t] : ci[b1 + (t - len0)]] - J0;
            atomicOr(&bits[J >> 5], 1u << (J & 31));
        }
        __syncthreads();
        // exclusive prefix of popcounts over the W words (thread-contiguous chunks)
        const int per = (W + blockDim.x - 1) / blockDim.x;
        const int w0 = min(W, (int)threadIdx.x * per), w1 = min(W, w0 + per);
        int mine = 0;
        for (int w = w0; w < w1; w++) mine += __popc(bits[w]);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int xs = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, xs, o);
            if (lane >= o) xs += y;
        }
        if (lane == 31) wsum[wid] = xs;
        __syncthreads();
        if (wid == 0) {
            int sv = lane < (int)(blockDim.x >> 5) ? wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, sv, o);
                if (lane >= o) sv += y;
            }
            if (lane < (int)(blockDim.x >> 5)) wsum[lane] = sv;
            if (lane == 31) wsum[32] = sv;
        }
        __syncthreads();
        int run = (wid > 0 ? wsum[wid - 1] : 0) + xs - mine;
        for (int w = w0; w < w1; w++) {
            pre[w] = run;
            run += __popc(bits[w]);
        }
        const int u = wsum[32];
        if (!FILL) {
            if (threadIdx.x == 0) rowcnt[I] = u;
            __syncthreads();
            continue;
        }
        __syncthreads();
        const int64_t base = crp[I];
        // sorted coarse columns
        for (int w = threadIdx.x; w < W; w += blockDim.x) {
            uint32_t m = bits[w];
            int pos = pre[w];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                cci[base + pos++] = J0 + (w << 5) + bit;
            }
        }
        for (int t = threadIdx.x; t < 4 * u; t += blockDim.x) slot[t] = -1;
        __syncthreads();
        for (int t = threadIdx.x; t < c; t += blockDim.x) {
            const int b = t < len0 ? ci[b0 + t] : ci[b1 + (t - len0)];
            const int J = agg[b];
            const int jj = J - J0;
            const int pos = pre[jj >> 5] + __popc(bits[jj >> 5] & ((1u << (jj & 31)) - 1u));
            const int q = 2 * (t < len0 ? 0 : 1) + (b == mem0[J] ? 0 : 1);
            slot[4 * pos + q] = t;
        }
        __syncthreads();
        const double p0 = pval[a0], p1 = a1 >= 0 ? pval[a1] : 0.0;
        for (int pos = threadIdx.x; pos < u; pos += blockDim.x) {
            const int J = cci[base + pos];
            double acc = 0.0;
            if (J >= I) {
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const int t = slot[4 * pos + q];
                    if (t < 0) continue;
                    const bool first = t < len0;
                    const int64_t k = first ? b0 + t : b1 + (t - len0);
                    acc = __dadd_rn(acc, __dmul_rn(__dmul_rn(first ? p0 : p1, v[k]), pval[ci[k]]));
                }
            }
            cv[base + pos] = acc;
        }
        __syncthreads();
    }
}

// Galerkin product with one warp per coarse row I (Sec. 3, Eq. of the
// Galerkin projection).  The candidates of row I are the entries (a, b) of
// its member rows a (a0, then a1); each goes to coarse column J = agg[b].
// A warp-private bitmap over [Jmin, Jmax] with prefix popcounts ranks the
// distinct J (the sorted coarse row) without sorting.
//
// Counting kernel: the bitmap covers `words` words at a time (windows over
// the span), so any span fits; it records the widest span and the longest
// coarse row (stats[0], stats[1]) for the values kernel's sizing.
//
// Values kernel: a coarse entry K_c(I,J) has at most four terms, one per
// pair (a in I, b in J).  Each candidate records its index in the entry's
// slot 2 rank(a in I) + rank(b in J) for J >= I (the canonical order of
// K_c(I,J)); each entry then sums its slots' terms in slot order, a missing
// slot contributing a zero term (the running sum starts from +0.0 and is
// never -0.0, so adding a zero leaves it unchanged).  For J < I the entry is
// defined as K_c(J,I), whose canonical order runs over J's members first:
// with K(a,b) = K(b,a) in every bit its terms are (p_b K(a,b)) p_a in slot
// 2 rank(b in J) + rank(a in I), so the lower triangle is computed in place
// and needs no mirror pass.  When the level matrix is symmetric only up to
// rounding (sym == 0) the lower entries are left to the mirror kernel.
//
// GB300 runs FP64 at about two lanes per SM per clock: the values kernel
// computes each candidate's term once, in the pass that gathers its coarse
// column (2 multiplies, every lane busy), keeps it in shared memory, and
// spends 3 adds per entry on the slot sums.
constexpr int kGalWarps = 4;   // coarse rows per block
constexpr int kGalBatch = 8;   // candidates per lane in flight in the gathers
constexpr unsigned kNoSlot = 0xffffu;

__device__ __forceinline__ size_t gal_align(size_t x) { return (x + 15) & ~(size_t)15; }

// member rows of a coarse row and their ranges in the level matrix
struct GalRow {
    int a0, a1, len0, len1;
    int64_t b0, b1;
};

__device__ __forceinline__ GalRow gal_members(int a0, int a1, const int64_t* __restrict__ rp) {
    GalRow r{a0, a1, 0, 0, 0, 0};
    if (a0 >= 0) {
        r.b0 = rp[a0];
        r.len0 = (int)(rp[a0 + 1] - r.b0);
    }
    if (a1 >= 0) {
        r.b1 = rp[a1];
        r.len1 = (int)(rp[a1 + 1] - r.b1);
    }
    return r;
}

// Marks the candidates' columns d = jb[t] (>> shift) - wb in [0, 32 W) in
// the bitmap.  Each lane takes a contiguous run of candidates (an odd
// number, so the lanes' jb reads fall in distinct banks): neighbouring
// candidates mostly share a bitmap word, and contiguous runs keep the lanes
// of one atomic on different words.
__device__ __forceinline__ void gal_mark(const int32_t* jb, int c, int shift, int wb, int W, uint32_t* bits, int lane) {
    const int per = ((c + 31) >> 5) | 1;
    const int tb = min(c, lane * per), te = min(c, tb + per);
    for (int t = tb; t < te; t++) {
        const int d = (jb[t] >> shift) - wb;
        if (d >= 0 && d < 32 * W) atomicOr(&bits[d >> 5], 1u << (d & 31));
    }
}

template <bool FILL>
__global__ void __launch_bounds__(kGalWarps * 32)
    k_galerkin_warp(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                    const double* __restrict__ v, const int32_t* __restrict__ agg, const double* __restrict__ pval,
                    const int32_t* __restrict__ mate, const int32_t* __restrict__ mem0,
                    const int32_t* __restrict__ mem1, int cmax, int words, int umax, int sym, int64_t* rowcnt,
                    const int64_t* __restrict__ crp, int32_t* cci, double* cv, int* stats, int* flag) {
    extern __shared__ __align__(16) unsigned char gsm[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t o_tb = gal_align(4 * (size_t)cmax);
    const size_t o_bits = o_tb + (FILL ? gal_align(8 * (size_t)cmax) : 0);
    const size_t o_pre = o_bits + gal_align(4 * (size_t)words);
    const size_t o_sidx = o_pre + (FILL ? gal_align(2 * (size_t)words) : 0);
    const size_t per_warp = o_sidx + (FILL ? gal_align(8 * (size_t)umax) : 0);
    unsigned char* my = gsm + per_warp * wid;
    int32_t* jb = reinterpret_cast<int32_t*>(my);  // candidates' coarse columns (FILL: 2 J + rank(b in J))
    uint32_t* bits = reinterpret_cast<uint32_t*>(my + o_bits);
    uint16_t* pre = reinterpret_cast<uint16_t*>(my + o_pre);     // FILL: entries before each word
    uint2* sidx = reinterpret_cast<uint2*>(my + o_sidx);          // FILL: four 16-bit slots per entry
    double* tb = reinterpret_cast<double*>(my + o_tb);            // FILL: the candidates' terms
    const int stride = gridDim.x * kGalWarps;
    int I = blockIdx.x * kGalWarps + wid;
    GalRow cur = gal_members(I < nc ? mem0[I] : -1, I < nc ? mem1[I] : -1, rp);
    int span_max = 0, u_max = 0, err = 0;
    for (; I < nc; I += stride) {
        const int In = I + stride;  // the next row's members load during this row's gathers
        const int n0 = In < nc ? mem0[In] : -1, n1 = In < nc ? mem1[In] : -1;
        const int len0 = cur.len0, c = cur.len0 + cur.len1;
        const bool fits = c <= cmax;  // sized from the row statistics; cannot fail
        if (!fits) err = 1;
        int lo = 0x7fffffff, hi = -1;
        if (fits) {
            // FILL: the member rows' prolongator values, for the terms
            const double p0 = (FILL && c > 0) ? pval[cur.a0] : 0.0;
            const double p1 = (FILL && cur.a1 >= 0) ? pval[cur.a1] : 0.0;
            for (int t0 = 0; t0 < c; t0 += 32 * kGalBatch) {
                int bb[kGalBatch], jj[kGalBatch], mm[kGalBatch];
                double vk[kGalBatch], pb[kGalBatch];
#pragma unroll
                for (int r = 0; r < kGalBatch; r++) {
                    const int t = t0 + 32 * r + lane;
                    const int64_t k = t < len0 ? cur.b0 + t : cur.b1 + (t - len0);
                    bb[r] = t < c ? ci[k] : -1;
                    vk[r] = (FILL && t < c) ? v[k] : 0.0;
                }
#pragma unroll
                for (int r = 0; r < kGalBatch; r++) {
                    jj[r] = bb[r] >= 0 ? agg[bb[r]] : 0;
                    mm[r] = (FILL && bb[r] >= 0) ? mate[bb[r]] : -1;
                    pb[r] = (FILL && bb[r] >= 0) ? pval[bb[r]] : 0.0;
                }
#pragma unroll
                for (int r = 0; r < kGalBatch; r++) {
                    if (FILL && t0 + 32 * r >= c) break;  // warp-uniform: no FP64 issue for empty rounds
                    const int t = t0 + 32 * r + lane;
                    if (FILL) {
                        // (p_a K(a,b)) p_b for J >= I, (p_b K(a,b)) p_a for J < I
                        const bool upper = jj[r] >= I;
                        const double pa = t >= len0 ? p1 : p0;
                        const double term = __dmul_rn(__dmul_rn(upper ? pa : pb[r], vk[r]), upper ? pb[r] : pa);
                        if (t < c) tb[t] = term;
                    }
                    if (t < c) {
                        lo = min(lo, jj[r]);
                        hi = max(hi, jj[r]);
                        jb[t] = FILL ? 2 * jj[r] + ((mm[r] >= 0 && mm[r] < bb[r]) ? 1 : 0) : jj[r];
                    }
                }
            }
        }
        lo = __reduce_min_sync(FULL, lo);
        hi = __reduce_max_sync(FULL, hi);
        const GalRow nxt = gal_members(n0, n1, rp);
        __syncwarp();
        if (fits && c > 0 && !FILL) {
            int u = 0;
            for (int wb = lo; wb <= hi; wb += 32 * words) {
                const int W = min(words, ((hi - wb) >> 5) + 1);
                for (int w = lane; w < W; w += 32) bits[w] = 0u;
                __syncwarp();
                gal_mark(jb, c, 0, wb, W, bits, lane);
                __syncwarp();
                int cnt = 0;
                for (int w = lane; w < W; w += 32) cnt += __popc(bits[w]);
                u += __reduce_add_sync(FULL, cnt);
                __syncwarp();
            }
            if (lane == 0) rowcnt[I] = u;
            span_max = max(span_max, hi - lo + 1);
            u_max = max(u_max, u);
        } else if (!FILL && lane == 0) {
            rowcnt[I] = 0;
        }
        if (fits && c > 0 && FILL) {
            const int W = ((hi - lo) >> 5) + 1;
            if (W > words) err = 1;  // sized from the counting kernel; cannot happen
            int u = 0;
            if (W <= words) {
                for (int w = lane; w < W; w += 32) bits[w] = 0u;
                __syncwarp();
                gal_mark(jb, c, 1, lo, W, bits, lane);
                __syncwarp();
                // exclusive prefix of the words' popcounts (contiguous chunks per lane)
                const int per = (W + 31) >> 5;
                const int w0 = min(W, lane * per), w1 = min(W, w0 + per);
                int mine = 0;
                for (int w = w0; w < w1; w++) mine += __popc(bits[w]);
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(FULL, incl, o);
                    if (lane >= o) incl += y;
                }
                u = __shfl_sync(FULL, incl, 31);
                int run = incl - mine;
                for (int w = w0; w < w1; w++) {
                    pre[w] = (uint16_t)run;
                    run += __popc(bits[w]);
                }
                if (u > umax) err = 1;  // sized from the counting kernel; cannot happen
            }
            if (W <= words && u <= umax) {
                for (int pos = lane; pos < u; pos += 32) sidx[pos] = make_uint2(0xffffffffu, 0xffffffffu);
                __syncwarp();
                // every candidate's slot
                for (int t = lane; t < c; t += 32) {
                    const int e = jb[t];
                    const int J = e >> 1, rb = e & 1, ra = t >= len0 ? 1 : 0;
                    const int d = J - lo;
                    const int pos = pre[d >> 5] + __popc(bits[d >> 5] & ((1u << (d & 31)) - 1u));
                    const int q = J >= I ? 2 * ra + rb : 2 * rb + ra;
                    reinterpret_cast<uint16_t*>(sidx)[4 * pos + q] = (uint16_t)t;
                }
                __syncwarp();
                // entries: their slots' terms summed in slot order
                const int64_t base = crp[I];
                for (int pos = lane; pos < u; pos += 32) {
                    const uint2 raw = sidx[pos];
                    const unsigned tq[4] = {raw.x & 0xffffu, raw.x >> 16, raw.y & 0xffffu, raw.y >> 16};
                    const unsigned tv = tq[0] != kNoSlot ? tq[0] : tq[1] != kNoSlot ? tq[1] : tq[2] != kNoSlot ? tq[2] : tq[3];
                    const int J = jb[min((int)tv, c - 1)] >> 1;  // every entry holds a candidate
                    double term[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) term[q] = tq[q] != kNoSlot ? tb[tq[q]] : 0.0;
                    // +0.0 + term[0] without an FP64 add: only -0.0 changes (to +0.0)
                    double acc = dbits(term[0]) == (long long)0x8000000000000000ULL ? 0.0 : term[0];
                    acc = __dadd_rn(acc, term[1]);
                    acc = __dadd_rn(acc, term[2]);
                    acc = __dadd_rn(acc, term[3]);
                    cci[base + pos] = J;
                    cv[base + pos] = acc;
                }
            }
            __syncwarp();
        }
        cur = nxt;
    }
    if (!FILL) {
        span_max = __reduce_max_sync(FULL, span_max);
        u_max = __reduce_max_sync(FULL, u_max);
        if (lane == 0) {
            atomicMax(stats, span_max);
            atomicMax(stats + 1, u_max);
        }
    }
    if (__any_sync(FULL, err) && lane == 0) atomicOr(flag, 32);
}

// max over coarse rows of the coarse-column span Jmax - Jmin + 1
__global__ void k_row_span(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const int32_t* __restrict__ agg, const int32_t* __restrict__ mem0,
                           const int32_t* __restrict__ mem1, int* maxspan) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    int best = 0;
    for (int I = warp; I < nc; I += nw) {
        int lo = 0x7fffffff, hi = -1;
        for (int m = 0; m < 2; m++) {
            const int a = m == 0 ? mem0[I] : mem1[I];
            if (a < 0) continue;
            for (int64_t k = rp[a] + lane; k < rp[a + 1]; k += 32) {
                const int J = agg[ci[k]];
                lo = min(lo, J);
                hi = max(hi, J);
            }
        }
        lo = __reduce_min_sync(FULL, lo);
        hi = __reduce_max_sync(FULL, hi);
        best = max(best, hi - lo + 1);
    }
    if (lane == 0) atomicMax(maxspan, best);
}

// max over coarse rows of the candidate count len(a0) + len(a1)
__global__ void k_row_stats(int nc, const int64_t* __restrict__ rp, const int32_t* __restrict__ mem0,
                            const int32_t* __restrict__ mem1, int* maxcand, const int* __restrict__ nc_dev) {
    if (nc_dev) nc = *nc_dev;  // the coarse row count as the scan left it on the device
    int m = 0;
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        const int a0 = mem0[I], a1 = mem1[I];
        int c = (int)(rp[a0 + 1] - rp[a0]);
        if (a1 >= 0) c += (int)(rp[a1 + 1] - rp[a1]);
        m = max(m, c);
    }
    m = __reduce_max_sync(FULL, m);
    if ((threadIdx.x & 31) == 0) atomicMax(maxcand, m);
}

// Composite map P = P_1 ... P_m of one level.
struct PassPtrs {
    const int32_t* agg[kMaxPasses];
    const double* pval[kMaxPasses];
};

__global__ void k_compose(int n, int npass, PassPtrs pp, int32_t* agg, double* pval) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int a = pp.agg[0][i];
        double pv = pp.pval[0][i];
        for (int s = 1; s < npass; s++) {
            pv = __dmul_rn(pv, pp.pval[s][a]);
            a = pp.agg[s][a];
        }
        agg[i] = a;
        pval[i] = pv;
    }
}

__global__ void k_member_count(int n, const int32_t* __restrict__ agg, int32_t* cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) atomicAdd(&cnt[agg[i]], 1);
}

// Members in ascending fine order: rank of i among the members of agg[i]
// that precede it (members of one aggregate are at most 2^m apart in count,
// scanned through the aggregate's own list after an unordered fill).
__global__ void k_member_fill(int n, const int32_t* __restrict__ agg, const int32_t* __restrict__ mptr,
                              int32_t* midx, int* cursor) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int I = agg[i];
        const int slot = atomicAdd(&cursor[I], 1);
        midx[mptr[I] + slot] = i;
    }
}

__global__ void k_member_sort(int nc, const int32_t* __restrict__ mptr, int32_t* midx) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        const int b = mptr[I], e = mptr[I + 1];
        for (int u = b + 1; u < e; u++) {
            const int x = midx[u];
            int t = u - 1;
            while (t >= b && midx[t] > x) {
                midx[t + 1] = midx[t];
                t--;
            }
            midx[t + 1] = x;
        }
    }
}

// ------------------------------------------------------------------ coarsest
__global__ void k_dense_from_csr(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                 const double* __restrict__ v, double* D) {
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) D[(int64_t)i * n + j] = 0.0;
        __syncthreads();
        for (int64_t k = rp[i] + threadIdx.x; k < rp[i + 1]; k += blockDim.x) D[(int64_t)i * n + ci[k]] = v[k];
        __syncthreads();
    }
}

// Right-looking Cholesky D = L L^T in place (lower triangle, one block).
__global__ void k_cholesky(int n, double* D, int* flag) {
    __shared__ double piv;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int j = 0; j < n; j++) {
        if (threadIdx.x == 0) {
            const double djj = D[(int64_t)j * n + j];
            if (!(djj > 0.0)) {
                atomicOr(flag, 16);
                piv = 1.0;
            } else {
                piv = __dsqrt_rn(djj);
            }
            D[(int64_t)j * n + j] = piv;
        }
        __syncthreads();
        const double ljj = piv;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
            D[(int64_t)i * n + j] = div_rn(D[(int64_t)i * n + j], ljj);  // correctly rounded, short latency
        __syncthreads();
        // trailing update, a warp per row i > j, its lanes over the columns k in (j, i]
        for (int i = j + 1 + wid; i < n; i += nwarps) {
            const double lij = D[(int64_t)i * n + j];
            for (int k = j + 1 + lane; k <= i; k += 32)
                D[(int64_t)i * n + k] = __dsub_rn(D[(int64_t)i * n + k], __dmul_rn(lij, D[(int64_t)k * n + j]));
        }
        __syncthreads();
    }
}

// Column c of A^-1 = L^-T L^-1 e_c, a warp per column: forward substitution
// from row c (the rows above hold zeros), then backward substitution; each
// step scales by the diagonal's reciprocal and updates the remaining rows
// lane-parallel, so a step costs one multiply's latency rather than a
// division's and a block barrier.
__global__ void k_chol_inverse(int n, const double* __restrict__ L, double* Ainv, double* work) {
    extern __shared__ double rinv[];  // reciprocals of the factor's diagonal
    for (int i = threadIdx.x; i < n; i += blockDim.x) rinv[i] = __ddiv_rn(1.0, L[(int64_t)i * n + i]);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = gw; c < n; c += nw) {
        double* y = work + (int64_t)c * n;
        for (int i = lane; i < n; i += 32) y[i] = (i == c) ? 1.0 : 0.0;
        __syncwarp();
        for (int k = c; k < n; k++) {  // forward: L y = e_c
            const double yk = __dmul_rn(y[k], rinv[k]);
            __syncwarp();
            if (lane == 0) y[k] = yk;
            for (int i = k + 1 + lane; i < n; i += 32) y[i] = __dsub_rn(y[i], __dmul_rn(L[(int64_t)i * n + k], yk));
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; k--) {  // backward: L^T x = y
            const double xk = __dmul_rn(y[k], rinv[k]);
            __syncwarp();
            if (lane == 0) y[k] = xk;
            for (int i = lane; i < k; i += 32) y[i] = __dsub_rn(y[i], __dmul_rn(L[(int64_t)k * n + i], xk));
            __syncwarp();
        }
        for (int i = lane; i < n; i += 32) Ainv[(int64_t)i * n + c] = y[i];
        __syncwarp();
    }
}

// Precision copies for the mixed-precision solve (round to nearest even;
// BF16 through FP32).
__global__ void k_to_f32(const double* __restrict__ in, float* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}

__global__ void k_to_bf16(const double* __restrict__ in, __nv_bfloat16* out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __float2bfloat16_rn(__double2float_rn(in[i]));
}

// Block-diagonal assembly of a batch: instance rows are moved by row_off,
// its entries by nnz_off (flag bit 1: a column outside the instance).
__global__ void k_shift_block(int n, int64_t nnz, const int64_t* __restrict__ rp_in, int64_t row_off, int64_t nnz_off,
                              int64_t* rp_out, int32_t* col, int* flag) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g <= n) rp_out[g] = rp_in[g] + nnz_off;
    if (g < nnz) {
        const int c = col[nnz_off + g];
        if (c < 0 || c >= n) atomicOr(flag, 1);
        col[nnz_off + g] = c + (int32_t)row_off;
    }
}

__global__ void k_fill_sys_id(int nsys, const int64_t* __restrict__ off, int32_t* id) {
    const int s = blockIdx.x;
    if (s >= nsys) return;
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) id[i] = s;
}

// ------------------------------------------------ run-encoded column index
// A row qualifies when its columns split into runs of L consecutive
// columns, all of the same length L (2 <= L <= kMaxRunLen, rows shorter than
// 2^16 entries); the tensor-product
// IgA matrices have this form (L = the row's band width in the fastest
// direction).  k_run_rows (a warp per row) writes the run count and L of
// every row, or sets *flag when a row does not qualify.
__global__ void k_run_rows(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, int32_t* runcnt,
                           uint8_t* runlen, int* flag) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int64_t b = rp[i], e = rp[i + 1];
        // length of the first run: position of the first break after b
        int64_t first_break = e;
        for (int64_t k0 = b + 1; k0 < e && first_break == e; k0 += 32) {
            const int64_t k = k0 + lane;
            const bool brk = k < e && ci[k] != ci[k - 1] + 1;
            const unsigned m = __ballot_sync(0xffffffffu, brk);
            if (m) first_break = k0 + __ffs(m) - 1;
        }
        const int64_t L = first_break - b;
        bool ok = L >= 2 && L <= kMaxRunLen && (e - b) % L == 0 && (e - b) < 65536;
        if (ok) {
            // offset within the run of entry k = b + 1 + lane + 32 s, kept
            // incrementally (no division per entry)
            const int Li = (int)L, step = 32 % Li;
            int o = (1 + lane) % Li;
            for (int64_t k = b + 1 + lane; k < e; k += 32) {
                const bool brk = ci[k] != ci[k - 1] + 1;
                if (brk != (o == 0)) ok = false;
                o += step;
                if (o >= Li) o -= Li;
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0) {
            if (ok) {
                runcnt[i] = (int32_t)((e - b) / L);
                runlen[i] = (uint8_t)L;
            } else {
                runcnt[i] = 0;
                runlen[i] = 0;
                atomicOr(flag, 1);
            }
        }
    }
}

// run_start[run_ptr[i] + r] = first column of run r of row i
__global__ void k_run_fill(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const int32_t* __restrict__ run_ptr, const uint8_t* __restrict__ runlen,
                           int32_t* run_start) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int64_t b = rp[i];
        const int L = runlen[i];
        const int r0 = run_ptr[i], R = run_ptr[i + 1] - r0;
        for (int r = lane; r < R; r += 32) run_start[r0 + r] = ci[b + (int64_t)r * L];
    }
}

}  // namespace

// ============================================================== launch wrappers
cudaError_t launch_shift_block(int n, int64_t nnz, const int64_t* rp_in, int64_t row_off, int64_t nnz_off,
                               int64_t* rp_out, int32_t* col, int* flag, cudaStream_t s) {
    const int64_t m = (nnz > (int64_t)n + 1 ? nnz : (int64_t)n + 1);
    k_shift_block<<<AMG_GRID((int)((m + 255) / 256)), 256, 0, s>>>(n, nnz, rp_in, row_off, nnz_off, rp_out, col, flag);
    return cudaGetLastError();
}

cudaError_t launch_run_rows(const DevCSR& A, int32_t* runcnt, uint8_t* runlen, int* flag, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_run_rows<<<AMG_GRID(blocks_for(A.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, runcnt, runlen,
                                                                                    flag);
    return cudaGetLastError();
}

cudaError_t launch_run_fill(const DevCSR& A, const int32_t* run_ptr, const uint8_t* runlen, int32_t* run_start,
                            cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_run_fill<<<AMG_GRID(blocks_for(A.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, run_ptr,
                                                                                    runlen, run_start);
    return cudaGetLastError();
}

cudaError_t launch_fill_sys_id(int nsys, const int64_t* off, int32_t* id, cudaStream_t s) {
    k_fill_sys_id<<<AMG_GRID(nsys), 256, 0, s>>>(nsys, off, id);
    return cudaGetLastError();
}
cudaError_t launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
    k_to_f32<<<AMG_GRID(blocks_for(n, kBlock, 8192)), kBlock, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const double* in, __nv_bfloat16* out, int64_t n, cudaStream_t s) {
    k_to_bf16<<<AMG_GRID(blocks_for(n, kBlock, 8192)), kBlock, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_validate_csr(const DevCSR& A, int* flag, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    k_validate<<<AMG_GRID(blocks_for(A.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(A.n, A.nnz, A.rowptr, A.col, A.val, flag);
    return cudaGetLastError();
}

cudaError_t launch_l1diag(const DevCSR& A, double* kii, double* dl1, double* invd, int* flag, cudaStream_t s) {
    if (A.n == 0) return cudaSuccess;
    AMG_TRY(cudaMemsetAsync(kii, 0, sizeof(double) * A.n, s));
    int dev = 0, sms = 148;
    AMG_TRY(cudaGetDevice(&dev));
    AMG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (fold_narrow(A.n, sms))
        k_l1diag<8><<<AMG_GRID(blocks_for(A.n, kBlock, 4096)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, kii, dl1,
                                                                              invd, flag);
    else
        k_l1diag<32><<<AMG_GRID(blocks_for(A.n, kBlock, 4096)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, kii, dl1,
                                                                               invd, flag);
    return cudaGetLastError();
}

cudaError_t launch_diag(const DevCSR& A, double* kii, cudaStream_t s) {
    AMG_TRY(cudaMemsetAsync(kii, 0, sizeof(double) * A.n, s));
    k_diag<<<AMG_GRID(blocks_for(A.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, kii);
    return cudaGetLastError();
}

cudaError_t launch_testvec_init(int n, int kind, uint64_t seed, double* w, cudaStream_t s) {
    k_testvec_init<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, kind, seed, w);
    return cudaGetLastError();
}

cudaError_t launch_testvec_sweep(const DevCSR& A, const double* dl1, const double* w, double* wout, cudaStream_t s) {
    int dev = 0, sms = 148;
    AMG_TRY(cudaGetDevice(&dev));
    AMG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (fold_narrow(A.n, sms))
        k_testvec_sweep<4><<<AMG_GRID(blocks_for(A.n, kBlock, 4096)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val,
                                                                                     dl1, w, wout);
    else
        k_testvec_sweep<32><<<AMG_GRID(blocks_for(A.n, kBlock, 4096)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val,
                                                                                      dl1, w, wout);
    return cudaGetLastError();
}

cudaError_t launch_edge_keys(const DevCSR& A, const double* kii, const double* w, uint64_t* key, int* flag,
                             cudaStream_t s) {
    k_edge_keys<<<AMG_GRID(blocks_for(A.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, kii, w,
                                                                                key, flag);
    return cudaGetLastError();
}

cudaError_t launch_match_init(int n, int32_t* state, cudaStream_t s) {
    k_match_init<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, state);
    return cudaGetLastError();
}

// One batch of `count` rounds from round first_round: round r's active
// vertices are listed in lists[(r - 1) & 1] (n entries each) with their
// count in active[r - 1]; it writes the next list to lists[r & 1] and the
// count to active[r] (zeroed by the caller).  Grids are sized for the first
// round and loop over the (shrinking) lists.
cudaError_t launch_match_rounds(const DevCSR& A, const uint64_t* key, int32_t* state, int32_t* cand, int* active,
                                int32_t* lists, int first_round, int count, cudaStream_t s) {
    const int n = A.n;
    const int gp = blocks_for(n, kWarpsPerBlock, 2048), gc = blocks_for(n, kBlock, 1024);
    for (int r = 0; r < count; r++) {
        const int round = first_round + r;
        const int32_t* lin = round > 0 ? lists + (size_t)((round - 1) & 1) * n : nullptr;
        const int* cin = round > 0 ? active + round - 1 : nullptr;
        k_match_propose<<<AMG_GRID(gp), kBlock, 0, s>>>(n, A.rowptr, A.col, key, state, cand, lin, cin);
        k_match_commit<<<AMG_GRID(gc), kBlock, 0, s>>>(n, cand, state, lin, cin, lists + (size_t)(round & 1) * n,
                                                         active + round);
    }
    return cudaGetLastError();
}

// All rounds of a pass in one cooperative launch (see k_match_rounds_coop):
// up to four blocks per SM, never more than can be resident at once.
// active[0 .. max_rounds-1] must be zero on entry.
cudaError_t launch_match_rounds_coop(const DevCSR& A, const uint64_t* key, int32_t* state, int32_t* cand, int* active,
                                     int32_t* lists, int max_rounds, int* rounds_out, int num_sms, cudaStream_t s) {
    int per_sm = 0;
    AMG_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match_rounds_coop, kBlock, 0));
    if (per_sm < 1 || num_sms < 1) return cudaErrorNotSupported;
    // small levels: fewer blocks (about four vertices per warp in the first
    // round) make the grid barriers cheaper
    constexpr int kVertsPerBlock = 4 * (kBlock / 32);
    const int64_t want = ((int64_t)A.n + kVertsPerBlock - 1) / kVertsPerBlock;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * std::min(per_sm, 4), want));
    int n = A.n;
    const int64_t* rp = A.rowptr;
    const int32_t* ci = A.col;
    void* args[] = {&n, &rp, &ci, &key, &state, &cand, &active, &lists, &max_rounds, &rounds_out};
    return cudaLaunchCooperativeKernel(reinterpret_cast<void*>(k_match_rounds_coop), dim3(blocks), dim3(kBlock), args,
                                       0, s);
}

cudaError_t launch_match_finish(int n, const int32_t* state, int32_t* mate, int32_t* leader, cudaStream_t s) {
    k_match_finish<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, state, mate, leader);
    return cudaGetLastError();
}

cudaError_t launch_aggregate(int n, const int32_t* mate, const int32_t* cidx, const double* w, int32_t* agg,
                             double* pval, int32_t* mem0, int32_t* mem1, double* wc, cudaStream_t s) {
    k_aggregate<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, mate, cidx, w, agg, pval, mem0, mem1, wc);
    return cudaGetLastError();
}

size_t scan_scratch_ints(int n) { return (size_t)(n + 1023) / 1024 + 1; }
size_t scan64_scratch(int n) { return (size_t)(n + 1023) / 1024 + 1; }

cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int n, int32_t* total, int32_t* scratch,
                                  cudaStream_t s) {
    return scan_impl<int32_t>(in, out, n, total, scratch, s);
}

cudaError_t launch_scan64(const int64_t* in, int64_t* out, int n, int64_t* scratch, cudaStream_t s) {
    // out has n+1 entries: exclusive scan plus the total at out[n]
    return scan_impl<int64_t>(in, out, n, out + n, scratch, s);
}

static size_t galerkin_smem(int cap) { return sizeof(uint64_t) * (size_t)cap; }

cudaError_t launch_galerkin_count(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                  int nc, int cap, int64_t* rowcnt, cudaStream_t s) {
    const size_t sm = galerkin_smem(cap);
    if (sm > 48 * 1024) AMG_TRY(cudaFuncSetAttribute(k_galerkin_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_galerkin_count<<<AMG_GRID(blocks_for(nc, 1, 65536)), kBlock, sm, s>>>(nc, A.rowptr, A.col, agg, mem0, mem1, cap, rowcnt);
    return cudaGetLastError();
}

cudaError_t launch_galerkin_fill(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mem0,
                                 const int32_t* mem1, int cap, DevCSR& C, cudaStream_t s) {
    const size_t sm = galerkin_smem(cap);
    if (sm > 48 * 1024) AMG_TRY(cudaFuncSetAttribute(k_galerkin_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_galerkin_fill<<<AMG_GRID(blocks_for(C.n, 1, 65536)), kBlock, sm, s>>>(C.n, A.rowptr, A.col, A.val, agg, pval, mem0, mem1,
                                                                    cap, C.rowptr, C.col, C.val);
    return cudaGetLastError();
}

cudaError_t launch_galerkin_mirror(DevCSR& C, int* flag, cudaStream_t s) {
    k_galerkin_mirror<<<AMG_GRID(blocks_for(C.n, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(C.n, C.rowptr, C.col, C.val, flag);
    return cudaGetLastError();
}

// Threads per block of the bitmap Galerkin kernels: a coarse row of a 3-D
// p=3 level holds about 700 fine entries, so small blocks spend less of their
// time waiting at the row's block barriers and more rows are in flight per SM.
constexpr int kGalerkinBlock = 128;

static size_t bitmap_smem(int cap, int words, bool fill) {
    return 8 * (size_t)words + (fill ? 16 * (size_t)cap : 0);
}

cudaError_t launch_galerkin_count_bitmap(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                         int nc, int cap, int words, int64_t* rowcnt, int* flag, cudaStream_t s) {
    const size_t sm = bitmap_smem(cap, words, false);
    if (sm > 48 * 1024)
        AMG_TRY(cudaFuncSetAttribute(k_galerkin_bitmap<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_galerkin_bitmap<false><<<AMG_GRID(blocks_for(nc, 1, 65536)), kGalerkinBlock, sm, s>>>(
        nc, A.rowptr, A.col, A.val, agg, nullptr, mem0, mem1, cap, words, rowcnt, nullptr, nullptr, nullptr, flag);
    return cudaGetLastError();
}

cudaError_t launch_galerkin_fill_bitmap(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mem0,
                                        const int32_t* mem1, int cap, int words, DevCSR& C, int* flag, cudaStream_t s) {
    const size_t sm = bitmap_smem(cap, words, true);
    if (sm > 48 * 1024)
        AMG_TRY(cudaFuncSetAttribute(k_galerkin_bitmap<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_galerkin_bitmap<true><<<AMG_GRID(blocks_for(C.n, 1, 65536)), kGalerkinBlock, sm, s>>>(
        C.n, A.rowptr, A.col, A.val, agg, pval, mem0, mem1, cap, words, nullptr, C.rowptr, C.col, C.val, flag);
    return cudaGetLastError();
}

// Bitmap window of the warp counting kernel: 1024 words (32,768 coarse
// columns) per pass over a row's candidates.
constexpr int kGalCountWords = 1024;

static size_t galerkin_warp_bytes(int cmax, int words, int umax, bool fill) {
    auto al = [](size_t x) { return (x + 15) & ~(size_t)15; };
    const size_t w = al(4 * (size_t)cmax) + al(4 * (size_t)words) +
                     (fill ? al(8 * (size_t)cmax) + al(2 * (size_t)words) + al(8 * (size_t)umax) : 0);
    return w * kGalWarps;
}

size_t galerkin_warp_fill_smem(int cmax, int words, int umax) {
    return galerkin_warp_bytes(cmax, words, umax, true);
}

// Blocks of `kernel` that can be resident on the device at once (at least
// one): the warp-per-row kernels loop over their rows from that many blocks,
// so that each warp takes row after row (and loads the next row's members
// early) instead of one block being scheduled per few rows.
template <typename K>
static cudaError_t resident_blocks(K kernel, int threads, size_t smem, int* blocks) {
    int dev = 0, sms = 0, per_sm = 0;
    AMG_TRY(cudaGetDevice(&dev));
    AMG_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    AMG_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    *blocks = std::max(1, per_sm * sms);
    return cudaSuccess;
}

cudaError_t launch_galerkin_warp_count(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                       int nc, int cmax, int64_t* rowcnt, int* stats, int* flag, cudaStream_t s) {
    const size_t sm = galerkin_warp_bytes(cmax, kGalCountWords, 0, false);
    if (sm > 48 * 1024)
        AMG_TRY(cudaFuncSetAttribute(k_galerkin_warp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    // rows in flight are bounded by shared memory: ask for the largest carveout
    AMG_TRY(cudaFuncSetAttribute(k_galerkin_warp<false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    int res = 0;
    AMG_TRY(resident_blocks(k_galerkin_warp<false>, kGalWarps * 32, sm, &res));
    k_galerkin_warp<false><<<AMG_GRID(std::min(blocks_for(nc, kGalWarps, 1 << 20), res)), kGalWarps * 32, sm, s>>>(
        nc, A.rowptr, A.col, A.val, agg, nullptr, nullptr, mem0, mem1, cmax, kGalCountWords, 0, 0, rowcnt, nullptr,
        nullptr, nullptr, stats, flag);
    return cudaGetLastError();
}

cudaError_t launch_galerkin_warp_fill(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mate,
                                      const int32_t* mem0, const int32_t* mem1, int cmax, int words, int umax, int sym,
                                      DevCSR& C, int* flag, cudaStream_t s) {
    const size_t sm = galerkin_warp_bytes(cmax, words, umax, true);
    if (sm > 48 * 1024)
        AMG_TRY(cudaFuncSetAttribute(k_galerkin_warp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    AMG_TRY(cudaFuncSetAttribute(k_galerkin_warp<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared));
    int res = 0;
    AMG_TRY(resident_blocks(k_galerkin_warp<true>, kGalWarps * 32, sm, &res));
    k_galerkin_warp<true><<<AMG_GRID(std::min(blocks_for(C.n, kGalWarps, 1 << 20), res)), kGalWarps * 32, sm, s>>>(
        C.n, A.rowptr, A.col, A.val, agg, pval, mate, mem0, mem1, cmax, words, umax, sym, nullptr, C.rowptr, C.col,
        C.val, nullptr, flag);
    return cudaGetLastError();
}

cudaError_t launch_row_span(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1, int nc,
                            int* maxspan, cudaStream_t s) {
    k_row_span<<<AMG_GRID(blocks_for(nc, kWarpsPerBlock, 8192)), kBlock, 0, s>>>(nc, A.rowptr, A.col, agg, mem0, mem1,
                                                                               maxspan);
    return cudaGetLastError();
}

cudaError_t launch_row_stats(const DevCSR& A, const int32_t* mem0, const int32_t* mem1, int nc, int* maxcand,
                             cudaStream_t s, const int* nc_dev) {
    // nc_dev: read the row count there (nc then bounds it, for the grid)
    k_row_stats<<<AMG_GRID(blocks_for(nc, kBlock, 4096)), kBlock, 0, s>>>(nc, A.rowptr, mem0, mem1, maxcand, nc_dev);
    return cudaGetLastError();
}

cudaError_t launch_compose(int n, int npass, const Pass* passes, int32_t* agg, double* pval, cudaStream_t s) {
    PassPtrs pp{};
    for (int q = 0; q < npass; q++) {
        pp.agg[q] = passes[q].agg;
        pp.pval[q] = passes[q].pval;
    }
    k_compose<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, npass, pp, agg, pval);
    return cudaGetLastError();
}

cudaError_t launch_member_count(int n, const int32_t* agg, int nc, int32_t* cnt, cudaStream_t s) {
    AMG_TRY(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (nc + 1), s));
    k_member_count<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, agg, cnt);
    return cudaGetLastError();
}

cudaError_t launch_member_fill(int n, const int32_t* agg, const int32_t* mem_ptr, int nc, int32_t* mem_idx,
                               int* cursor, cudaStream_t s) {
    AMG_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * nc, s));
    k_member_fill<<<AMG_GRID(blocks_for(n, kBlock, 4096)), kBlock, 0, s>>>(n, agg, mem_ptr, mem_idx, cursor);
    k_member_sort<<<AMG_GRID(blocks_for(nc, kBlock, 4096)), kBlock, 0, s>>>(nc, mem_ptr, mem_idx);
    return cudaGetLastError();
}

cudaError_t launch_dense_from_csr(const DevCSR& A, double* D, cudaStream_t s) {
    k_dense_from_csr<<<AMG_GRID(blocks_for(A.n, 1, 4096)), kBlock, 0, s>>>(A.n, A.rowptr, A.col, A.val, D);
    return cudaGetLastError();
}

// Lower triangle of the factor, zeros above (row-major n x n).
__global__ void k_keep_factor(int n, const double* __restrict__ D, double* L) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
         t += (int64_t)gridDim.x * blockDim.x)
        L[t] = (t % n) <= (t / n) ? D[t] : 0.0;
}

// D (n x n, overwritten by its Cholesky factor); Ainv receives the inverse
// in its first n^2 doubles and the factor L (zeros above the diagonal) in
// the second n^2 (work space of the inverse before).
cudaError_t launch_dense_spd_inverse(int n, double* D, double* Ainv, int* flag, cudaStream_t s) {
    k_cholesky<<<AMG_GRID(1), 1024, 0, s>>>(n, D, flag);
    const size_t sm = sizeof(double) * (size_t)n;  // the diagonal's reciprocals (n <= 4096: 32 KB)
    if (sm > 48 * 1024) AMG_TRY(cudaFuncSetAttribute(k_chol_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_chol_inverse<<<AMG_GRID(blocks_for(n, kWarpsPerBlock, 4096)), kBlock, sm, s>>>(n, D, Ainv, Ainv + (int64_t)n * n);
    k_keep_factor<<<AMG_GRID(blocks_for((int64_t)n * n, kBlock, 1024)), kBlock, 0, s>>>(n, D, Ainv + (int64_t)n * n);
    return cudaGetLastError();
}

}  // namespace amg
