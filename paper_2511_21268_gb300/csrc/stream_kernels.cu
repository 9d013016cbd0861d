// Finest-level matrix passes of the mixed-precision solve, staged in shared
// memory by the bulk-copy (TMA) engine.
//
// The finest matrix is stored with run-encoded columns (every row a
// sequence of equal runs of consecutive columns, one start column per run).
// Its FP32 or BF16 values move 2-4 bytes per entry; loaded by lanes, that
// is 64-128 bytes per warp instruction, too little in flight to cover HBM
// latency (the row-group kernels reach about 60 % of the measured HBM
// bandwidth and stall on long scoreboard).  Here:
//   * each block owns a contiguous range of rows (persistent grid, one block
//     per SM) and first copies the window of the gathered vector that its
//     rows reference -- the band of an IgA matrix, the block's rows plus
//     about 2 p (n+p)^(d-1) entries -- into shared memory with one bulk copy,
//     so every gather is a shared-memory load;
//   * thread 0 streams the matrix in slabs of S consecutive rows (values and
//     run starts, tens of KB per slab) with cp.async.bulk into a ring of
//     NBUF buffers, each completing on its mbarrier, while the 8 warps
//     compute the previous slab from shared memory.
// Row sums are finished as in the row-group kernels (lane partials into a
// shared tile, 32/RPW lanes per row), so the epilogues (residual, smoothing
// with z and r.z, q = K p with p.q) are the same; dot products accumulate
// per thread over the block's rows and are written as one deterministic
// partial per block.
//
// Every wait on an mbarrier is bounded (clock and iteration limit); on
// expiry the kernel records AMG_ERR_TIMEOUT in the solve state, waits (again
// bounded) for its copies in flight and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "amg_internal.cuh"
#include "stream_common.cuh"

namespace amg {

namespace {

// Shared-memory layout: [vector window][NBUF x slab buffer][mbarriers
// (window + NBUF), copy bases, control words][row tiles].  A slab buffer
// holds the slab's values, run starts, row metadata (row offsets, run
// offsets, run lengths) and up to kMaxVec vector segments its epilogue reads,
// so the compute loop reads only shared memory.

struct StreamShape {
    uint32_t xbytes;  // vector window bytes
    uint32_t vbytes;  // value area bytes (per buffer)
    uint32_t rbytes;  // run-start area bytes (per buffer)
    int nbuf;         // buffers in the ring (2..kMaxBuf)
};

constexpr uint32_t kCtrlBytes = 128;  // barriers, bases and the control words

// per-buffer bytes of the row metadata and of the vector segments of a slab of S rows
template <int S>
__host__ __device__ constexpr uint32_t meta_bytes() {
    return align16((S + 1) * 8) + align16((S + 1) * 4) + align16(S) + kMaxVec * align16(S * 8);
}

template <int RPW>
__host__ __device__ inline uint32_t buffer_bytes(StreamShape sh) {
    return sh.vbytes + sh.rbytes + meta_bytes<kStreamWarps * RPW>();
}

template <int RPW>
__host__ __device__ constexpr uint32_t tile_bytes() {
    return (uint32_t)(kStreamWarps * RPW * 33 * sizeof(float));
}

template <int RPW>
__host__ __device__ inline uint32_t stream_smem_bytes(StreamShape sh) {
    return sh.xbytes + (uint32_t)sh.nbuf * buffer_bytes<RPW>(sh) + kCtrlBytes + tile_bytes<RPW>();
}

// Entries O .. LL-1 of one run: value at va + o vstride, vector entry at
// xa + 4 o; two accumulators halve the FMA dependency chain.
template <int O, int LL, typename V>
struct RunDot {
    static __device__ __forceinline__ void run(uint32_t va, uint32_t vstride, uint32_t xa, float& a0, float& a1) {
        const float v = lds_val(va, static_cast<const V*>(nullptr));
        const float x = lds_x<4 * O>(xa);
        if (O & 1) a1 = fmaf(v, x, a1);
        else a0 = fmaf(v, x, a0);
        RunDot<O + 1, LL, V>::run(va + vstride, vstride, xa, a0, a1);
    }
};
template <int LL, typename V>
struct RunDot<LL, LL, V> {
    static __device__ __forceinline__ void run(uint32_t, uint32_t, uint32_t, float&, float&) {}
};

// Lane partial of one row whose R runs have LL entries each, values
// run-interleaved (entry o of run r at value index o R + r from the row's
// first value, shared address va0); run starts at shared address ra; the
// window entry of column c at xbase + 4 c (32-bit wrap-around arithmetic).
// Lane t takes the runs t, t + 32, ...
template <int LL, typename V>
__device__ __forceinline__ float row_runs(uint32_t va0, uint32_t ra, uint32_t xbase, int R, int lane) {
    constexpr uint32_t es = sizeof(V);
    float a0 = 0.f, a1 = 0.f;
    const uint32_t vstride = (uint32_t)R * es;
    for (int r = lane; r < R; r += 32) {
        const uint32_t xa = xbase + 4u * (uint32_t)lds_s32(ra + 4u * (uint32_t)r);
        RunDot<0, LL, V>::run(va0 + es * (uint32_t)r, vstride, xa, a0, a1);
    }
    return a0 + a1;
}

// Slab k covers rows [k S, k S + S), S = 8 RPW; block b owns slabs
// [b nsl / G, (b + 1) nsl / G) and the vector window win[b] = (lo, hi),
// the smallest and largest column of those rows.  The row-offset, run and
// vector arrays read here are padded so that the 16-byte-widened copies of
// the last slab stay inside them.
//
// Warp specialisation: warp 8 (one lane) produces -- it issues the window
// copy and, for each slab, waits until the buffer is empty (all 8 compute
// warps arrived on empty[j]) and issues the slab's copies on full[j]; warps
// 0-7 wait on full[j], compute their RPW rows and arrive on empty[j].  The
// producer's reads of the slab bounds overlap the compute warps' work.
template <int RPW, typename V, typename Epi>
__global__ void __launch_bounds__(kStreamThreads, 1)
    k_stream(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ rptr, const uint8_t* __restrict__ rlen,
             const int32_t* __restrict__ rst, const V* __restrict__ val, const float* __restrict__ xg,
             const int2* __restrict__ win, StreamShape shape, Epi epi, double* part1, double* part2,
             SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    constexpr int S = kStreamWarps * RPW;
    constexpr int LPR = 32 / RPW;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nbuf = shape.nbuf;
    const float* xw = reinterpret_cast<const float*>(smem);
    unsigned char* ring = smem + shape.xbytes;
    const uint32_t bufstride = buffer_bytes<RPW>(shape);
    // offsets inside a buffer
    const uint32_t o_run = shape.vbytes, o_rp = o_run + shape.rbytes, o_rptr = o_rp + align16((S + 1) * 8),
                   o_rlen = o_rptr + align16((S + 1) * 4), o_vec = o_rlen + align16(S);
    unsigned char* ctl = ring + nbuf * bufstride;
    // [0] window, [1 + j] full[j], [1 + kMaxBuf + j] empty[j]
    uint64_t* bars = reinterpret_cast<uint64_t*>(ctl);
    int64_t* vbase = reinterpret_cast<int64_t*>(ctl + 56);        // first entry held by buffer j
    int* rbase = reinterpret_cast<int*>(ctl + 56 + 8 * kMaxBuf);  // first run held by buffer j
    volatile int* ctrl = reinterpret_cast<int*>(ctl + 56 + 12 * kMaxBuf);  // 0 = go on, 1 = give up
    int* xlo = reinterpret_cast<int*>(ctl + 56 + 12 * kMaxBuf + 4);        // first vector entry of the window
    float(*tiles)[RPW][33] = reinterpret_cast<float(*)[RPW][33]>(ctl + kCtrlBytes);
    __shared__ double red[kStreamWarps + 1];

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nsl = (n + S - 1) / S;
    const int s0 = (int)((int64_t)blockIdx.x * nsl / gridDim.x);
    const int s1 = (int)((int64_t)(blockIdx.x + 1) * nsl / gridDim.x);
    const uint32_t bar_win = smem_addr(&bars[0]);
    auto bar_full = [&](int j) { return smem_addr(&bars[1 + j]); };
    auto bar_empty = [&](int j) { return smem_addr(&bars[1 + kMaxBuf + j]); };

    if (threadIdx.x == 0) {
        mbar_init(bar_win, 1);
        for (int j = 0; j < kMaxBuf; j++) {
            mbar_init(bar_full(j), 1);
            mbar_init(bar_empty(j), kStreamWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *ctrl = 0;
        *xlo = 0;
        if (s0 < s1) *xlo = win[blockIdx.x].x & ~3;
    }
    __syncthreads();

    double acc1 = 0.0, acc2 = 0.0;
    if (wid == kStreamWarps) {
        // ------------------------------------------------------------ producer
        if (lane == 0 && s0 < s1) {
            const int2 w = win[blockIdx.x];
            const int lo = w.x & ~3;
            const uint32_t bytes = align16((uint32_t)(w.y + 1 - lo) * 4u);
            mbar_expect_tx(bar_win, bytes);
            bulk_g2s(smem_addr(smem), xg + lo, bytes, bar_win);
            int last_use[kMaxBuf] = {-1, -1, -1};  // last use issued into each buffer
            for (int k = s0; k < s1; k++) {
                if (*ctrl) break;
                const int u = (k - s0) / nbuf, j = (k - s0) % nbuf;
                if (u > 0 && !mbar_wait_bounded(bar_empty(j), (uint32_t)(u - 1) & 1u)) {
                    *ctrl = 1;
                    break;
                }
                // copy slab k into buffer j
                const int a = k * S, b = min(n, a + S);
                const int64_t e0 = rp[a], e1 = rp[b];
                const int64_t vb0 = (e0 * (int64_t)sizeof(V)) & ~(int64_t)15;
                const int64_t vb1 = (e1 * (int64_t)sizeof(V) + 15) & ~(int64_t)15;
                const int r0 = rptr[a], r1 = rptr[b];
                const int64_t rb0 = ((int64_t)r0 * 4) & ~(int64_t)15;
                const int64_t rb1 = ((int64_t)r1 * 4 + 15) & ~(int64_t)15;
                vbase[j] = vb0 / (int64_t)sizeof(V);
                rbase[j] = (int)(rb0 / 4);
                unsigned char* bv = ring + j * bufstride;
                const uint32_t cnt = (uint32_t)(b - a);
                // row metadata and epilogue vectors: a is a multiple of 16, so
                // every segment starts 16-byte aligned
                const uint32_t b_rp = align16((cnt + 1) * 8), b_rptr = align16((cnt + 1) * 4), b_rlen = align16(cnt);
                uint32_t tx = (uint32_t)(vb1 - vb0 + rb1 - rb0) + b_rp + b_rptr + b_rlen;
#pragma unroll
                for (int v = 0; v < kMaxVec; v++)
                    if (v < epi.nvec) tx += align16(cnt * (uint32_t)epi.es[v]);
                const uint32_t bar = bar_full(j);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(bar, tx);
                bulk_g2s(smem_addr(bv), reinterpret_cast<const unsigned char*>(val) + vb0, (uint32_t)(vb1 - vb0), bar);
                bulk_g2s(smem_addr(bv + o_run), reinterpret_cast<const unsigned char*>(rst) + rb0,
                         (uint32_t)(rb1 - rb0), bar);
                bulk_g2s(smem_addr(bv + o_rp), rp + a, b_rp, bar);
                bulk_g2s(smem_addr(bv + o_rptr), rptr + a, b_rptr, bar);
                bulk_g2s(smem_addr(bv + o_rlen), rlen + a, b_rlen, bar);
#pragma unroll
                for (int v = 0; v < kMaxVec; v++)
                    if (v < epi.nvec)
                        bulk_g2s(smem_addr(bv + o_vec + v * align16(S * 8)),
                                 reinterpret_cast<const unsigned char*>(epi.vec[v]) + (int64_t)a * epi.es[v],
                                 align16(cnt * (uint32_t)epi.es[v]), bar);
                if (j == 0) last_use[0] = u;
                else if (j == 1) last_use[1] = u;
                else last_use[2] = u;
            }
            if (*ctrl) {  // drain copies that may still be in flight (bounded), keeping smem alive
                mbar_wait_bounded(bar_win, 0u);
                if (last_use[0] >= 0) mbar_wait_bounded(bar_full(0), (uint32_t)last_use[0] & 1u);
                if (last_use[1] >= 0) mbar_wait_bounded(bar_full(1), (uint32_t)last_use[1] & 1u);
                if (last_use[2] >= 0) mbar_wait_bounded(bar_full(2), (uint32_t)last_use[2] & 1u);
            }
        }
    } else {
        // ------------------------------------------------------------ consumers
        bool ok = true;
        if (s0 < s1) ok = __all_sync(FULL, mbar_wait_bounded(bar_win, 0u));
        const float* xs = xw - *xlo;  // xs[c] = vector entry c (inside the window)
        // shared address of vector entry 0 (32-bit wrap-around: entry c at xbase + 4 c)
        const uint32_t xbase = smem_addr(xw) - 4u * (uint32_t)(*xlo);
        for (int k = s0; k < s1 && ok; k++) {
            const int u = (k - s0) / nbuf, j = (k - s0) % nbuf;
            ok = __all_sync(FULL, !*ctrl && mbar_wait_bounded(bar_full(j), (uint32_t)u & 1u));
            if (!ok) break;
            const unsigned char* bv = ring + j * bufstride;
            const V* sv = reinterpret_cast<const V*>(bv);
            const int32_t* sr = reinterpret_cast<const int32_t*>(bv + o_run);
            const int64_t* srp = reinterpret_cast<const int64_t*>(bv + o_rp);
            const int32_t* srptr = reinterpret_cast<const int32_t*>(bv + o_rptr);
            const uint8_t* srlen = bv + o_rlen;
            const unsigned char* seg = bv + o_vec;  // segment v at seg + v * align16(8 S)
            const int64_t vb = vbase[j];
            const int rbs = rbase[j];
            const int a = k * S;
#pragma unroll 1
            for (int t = 0; t < RPW; t++) {
                const int tl = wid * RPW + t;
                float acc = 0.f;
                if (a + tl < n) {
                    // row tl: R runs of L entries; values stored run-interleaved
                    // (entry o of run r at o R + r), so lane r reads run r
                    const int64_t b = srp[tl];
                    const int L = srlen[tl];
                    const int r0 = srptr[tl];
                    const int R = srptr[tl + 1] - r0;
                    const uint32_t va0 = smem_addr(sv) + (uint32_t)(b - vb) * (uint32_t)sizeof(V);
                    const uint32_t ra = smem_addr(sr) + 4u * (uint32_t)(r0 - rbs);
                    switch (L) {  // warp-uniform: the run length of the row
                        case 2: acc = row_runs<2, V>(va0, ra, xbase, R, lane); break;
                        case 3: acc = row_runs<3, V>(va0, ra, xbase, R, lane); break;
                        case 4: acc = row_runs<4, V>(va0, ra, xbase, R, lane); break;
                        case 5: acc = row_runs<5, V>(va0, ra, xbase, R, lane); break;
                        case 6: acc = row_runs<6, V>(va0, ra, xbase, R, lane); break;
                        case 7: acc = row_runs<7, V>(va0, ra, xbase, R, lane); break;
                        case 8: acc = row_runs<8, V>(va0, ra, xbase, R, lane); break;
                        default: acc = row_runs<9, V>(va0, ra, xbase, R, lane); break;
                    }
                }
                tiles[wid][t][lane] = acc;
            }
            __syncwarp();
            {
                const int r = lane / LPR, q = lane % LPR;
                float sum = 0.f;
#pragma unroll
                for (int t = 0; t < RPW; t++) sum += tiles[wid][r][q * RPW + t];
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
                const int tl = wid * RPW + r;
                if (q == 0 && a + tl < n) epi(a + tl, tl, sum, seg, align16(S * 8), xs, acc1, acc2);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_empty(j));  // this warp is done with buffer j
        }
        if (!ok && lane == 0) *ctrl = 1;
    }
    __syncthreads();
    if (*ctrl) {
        if (threadIdx.x == 0 && st) {
            st->status = AMG_ERR_TIMEOUT;
            st->done = 1;
        }
        return;
    }
    if (part1) block_sum_to(acc1, red, part1 + blockIdx.x);
    if (part2) block_sum_to(acc2, red, part2 + blockIdx.x);
}

// Run-interleaved copy of a run-encoded matrix's values: entry o of run r
// of row i (CSR position rp[i] + r L + o) goes to rp[i] + o R + r, so that
// consecutive lanes, one run each, read consecutive words.
template <typename T>
__global__ void k_interleave_runs(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ rptr,
                                  const uint8_t* __restrict__ rlen, const T* __restrict__ in, T* out) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const int64_t b = rp[i];
        const int L = rlen[i], R = rptr[i + 1] - rptr[i];
        for (int r = lane; r < R; r += 32)
            for (int o = 0; o < L; o++) out[b + (int64_t)o * R + r] = in[b + (int64_t)r * L + o];
    }
}

// Largest slab of S rows: entries and runs (atomic max over slabs).
__global__ void k_slab_max(int n, int S, const int64_t* __restrict__ rp, const int32_t* __restrict__ rptr, int* out) {
    pdl_entry();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int nsl = (n + S - 1) / S;
    if (k >= nsl) return;
    const int a = k * S, b = min(n, a + S);
    atomicMax(out, (int)(rp[b] - rp[a]));
    atomicMax(out + 1, rptr[b] - rptr[a]);
}

// Vector window of each block's rows: smallest first column and largest
// last column over the rows of its slabs (a thread block per grid block).
__global__ void k_block_window(int n, int S, int G, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                               int2* win) {
    pdl_entry();
    __shared__ int slo[256], shi[256];
    const int b = blockIdx.x;
    const int nsl = (n + S - 1) / S;
    const int a0 = (int)((int64_t)b * nsl / G) * S;
    const int a1 = min(n, (int)((int64_t)(b + 1) * nsl / G) * S);
    int lo = INT32_MAX, hi = -1;
    for (int i = a0 + threadIdx.x; i < a1; i += blockDim.x) {
        const int64_t e0 = rp[i], e1 = rp[i + 1];
        if (e1 > e0) {
            lo = min(lo, ci[e0]);
            hi = max(hi, ci[e1 - 1]);
        }
    }
    slo[threadIdx.x] = lo;
    shi[threadIdx.x] = hi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            slo[threadIdx.x] = min(slo[threadIdx.x], slo[threadIdx.x + o]);
            shi[threadIdx.x] = max(shi[threadIdx.x], shi[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) win[b] = a1 > a0 ? make_int2(slo[0], shi[0]) : make_int2(0, 0);
}

template <int RPW, typename V, typename Epi>
bool set_attrs(uint32_t smem) {
    auto fn = k_stream<RPW, V, Epi>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
    return cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100) == cudaSuccess;
}

template <int RPW, typename V, typename Epi>
cudaError_t launch(amg_hierarchy* h, const V* val, const float* x, StreamShape sh, const Epi& epi, double* p1,
                   double* p2, cudaStream_t s) {
    const Level& L0 = h->lev[0];
    const uint32_t smem = stream_smem_bytes<RPW>(sh);
    launch_pdl(k_stream<RPW, V, Epi>, h->stream_blocks, kStreamThreads, smem, s,
        L0.A.n, L0.A.rowptr, L0.run_ptr, L0.run_len, L0.run_start, val, x, reinterpret_cast<const int2*>(h->stream_win),
        sh, epi, p1, p2, h->st);
    return cudaGetLastError();
}

StreamShape shape_of(const amg_hierarchy* h, int q) {
    return StreamShape{(uint32_t)h->stream_xbytes, (uint32_t)h->stream_vbytes[q], (uint32_t)h->stream_rbytes[q],
                       h->stream_nbuf[q]};
}

template <typename Epi>
cudaError_t dispatch(amg_hierarchy* h, int q, const void* val, const float* x, const Epi& epi, double* p1, double* p2,
                     cudaStream_t s) {
    const StreamShape sh = shape_of(h, q);
    const int rpw = h->stream_rpw;
    if (q == 0) {
        const __nv_bfloat16* v = static_cast<const __nv_bfloat16*>(val);
        return rpw == 2 ? launch<2>(h, v, x, sh, epi, p1, p2, s) : launch<1>(h, v, x, sh, epi, p1, p2, s);
    }
    const float* v = static_cast<const float*>(val);
    return rpw == 2 ? launch<2>(h, v, x, sh, epi, p1, p2, s) : launch<1>(h, v, x, sh, epi, p1, p2, s);
}

}  // namespace

// Decide whether the staged passes apply (mixed precision, run-encoded
// finest level, vector window and buffers within the shared-memory budget)
// and size them.  Both value widths use the same slab height (and so the
// same per-block vector windows): 32-row slabs if both fit, else 16-row
// slabs; each width takes three buffers if they fit, else two.
int stream_prepare(amg_hierarchy* h, int* scratch2) {
    h->stream = 0;
    const Level& L0 = h->lev[0];
    if (!h->mixed || !L0.run_ptr || h->nlev < 2) return AMG_OK;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return AMG_ERR_CUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return AMG_ERR_CUDA;
    const int n = L0.A.n;
    const int G = h->num_sms;
    // every array the bulk copies read must start 16-byte aligned
    const void* arrays[] = {L0.A.rowptr, L0.run_ptr, L0.run_len, L0.run_start, L0.val32, L0.val16, L0.x32,
                            L0.t32,      L0.invd32,  h->p32,     h->r,         h->p,     h->q};
    for (const void* a : arrays)
        if (a && (reinterpret_cast<uintptr_t>(a) & 15)) return AMG_OK;
    {  // rows of many runs: the sliced lane-per-row slabs
        int used = 0;
        const int rc = sell_prepare(h, scratch2, optin, &used);
        if (rc != AMG_OK || used) return rc;
    }
    int2* win = nullptr;
    if (dev_alloc(reinterpret_cast<void**>(&win), sizeof(int2) * G, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
    h->allocs.push_back(win);
    for (int v = 0; v < 2; v++) {  // v = 0: RPW 2 (32-row slabs), v = 1: RPW 1 (16-row slabs)
        const int rpw = v == 0 ? 2 : 1;
        const int S = kStreamWarps * rpw;
        launch_pdl(k_block_window, G, 256, 0, h->s, n, S, G, L0.A.rowptr, L0.A.col, win);
        std::vector<int2> hw(G);
        int slab[2] = {0, 0};  // entries, runs of the largest slab
        if (cudaMemsetAsync(scratch2, 0, 2 * sizeof(int), h->s) != cudaSuccess) return AMG_ERR_CUDA;
        const int nsl = (n + S - 1) / S;
        launch_pdl(k_slab_max, (nsl + 255) / 256, 256, 0, h->s, n, S, L0.A.rowptr, L0.run_ptr, scratch2);
        if (cudaMemcpyAsync(hw.data(), win, sizeof(int2) * G, cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
            cudaMemcpyAsync(slab, scratch2, sizeof(slab), cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
            cudaStreamSynchronize(h->s) != cudaSuccess)
            return AMG_ERR_CUDA;
        int64_t xw = 16;
        for (int b = 0; b < G; b++)
            xw = std::max<int64_t>(xw, ((int64_t)(hw[b].y + 1 - (hw[b].x & ~3)) * 4 + 15) & ~(int64_t)15);
        bool fits = xw < (1 << 20);
        for (int q = 0; q < 2 && fits; q++) {  // q = 0: BF16 values, q = 1: FP32 values
            const int vsz = q == 0 ? 2 : 4;
            const uint32_t vb = (uint32_t)(((int64_t)slab[0] * vsz + 32 + 15) & ~(int64_t)15);
            const uint32_t rb = (uint32_t)(((int64_t)slab[1] * 4 + 32 + 15) & ~(int64_t)15);
            int chosen = 0;
            for (int nb = kMaxBuf; nb >= 2 && !chosen; nb--) {
                const StreamShape sh{(uint32_t)xw, vb, rb, nb};
                const uint32_t need = rpw == 2 ? stream_smem_bytes<2>(sh) : stream_smem_bytes<1>(sh);
                if (need + 256u <= (uint32_t)optin) chosen = nb;  // 256: static shared memory
            }
            if (!chosen) fits = false;
            h->stream_vbytes[q] = (int)vb;
            h->stream_rbytes[q] = (int)rb;
            h->stream_nbuf[q] = chosen;
        }
        if (!fits) continue;
        h->stream_xbytes = (int)xw;
        h->stream_rpw = rpw;
        h->stream_win = reinterpret_cast<int*>(win);
        const uint32_t m16 = rpw == 2 ? stream_smem_bytes<2>(shape_of(h, 0)) : stream_smem_bytes<1>(shape_of(h, 0));
        const uint32_t m32 = rpw == 2 ? stream_smem_bytes<2>(shape_of(h, 1)) : stream_smem_bytes<1>(shape_of(h, 1));
        bool attrs;
        if (rpw == 2)
            attrs = set_attrs<2, __nv_bfloat16, EpiResid>(m16) && set_attrs<2, __nv_bfloat16, EpiUp0>(m16) &&
                    set_attrs<2, float, EpiResid>(m32) && set_attrs<2, float, EpiUp0>(m32) &&
                    set_attrs<2, float, EpiPQ>(m32);
        else
            attrs = set_attrs<1, __nv_bfloat16, EpiResid>(m16) && set_attrs<1, __nv_bfloat16, EpiUp0>(m16) &&
                    set_attrs<1, float, EpiResid>(m32) && set_attrs<1, float, EpiUp0>(m32) &&
                    set_attrs<1, float, EpiPQ>(m32);
        if (!attrs) return AMG_ERR_CUDA;
        // run-interleaved copies of the finest values read by these kernels
        Level& F0 = h->lev[0];
        const int64_t nnz = F0.A.nnz;
        const int gw = (int)std::min<int64_t>((n + 7) / 8, 8192);
        if (F0.val16) {
            if (dev_alloc(reinterpret_cast<void**>(&F0.val16t), sizeof(__nv_bfloat16) * (nnz + 16), h->s) != cudaSuccess)
                return AMG_ERR_NOMEM;
            h->allocs.push_back(F0.val16t);
            launch_pdl(k_interleave_runs<__nv_bfloat16>, gw, 256, 0, h->s, n, F0.A.rowptr, F0.run_ptr, F0.run_len,
                       F0.val16, F0.val16t);
        }
        if (dev_alloc(reinterpret_cast<void**>(&F0.val32t), sizeof(float) * (nnz + 16), h->s) != cudaSuccess) return AMG_ERR_NOMEM;
        h->allocs.push_back(F0.val32t);
        launch_pdl(k_interleave_runs<float>, gw, 256, 0, h->s, n, F0.A.rowptr, F0.run_ptr, F0.run_len, F0.val32,
                   F0.val32t);
        if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
        if ((reinterpret_cast<uintptr_t>(F0.val32t) & 15) || (reinterpret_cast<uintptr_t>(F0.val16t) & 15))
            return AMG_OK;
        h->stream_blocks = G;
        h->stream = 1;
        return AMG_OK;
    }
    return AMG_OK;  // does not fit: the row-group kernels run the finest level
}

cudaError_t launch_stream_resid(amg_hierarchy* h, const double* f, const float* x, float* rbuf, cudaStream_t s) {
    if (h->stream == 2) return sell_resid(h, f, x, rbuf, s);
    const Level& L0 = h->lev[0];
    const EpiResid epi{{f, nullptr, nullptr}, {8, 0, 0}, 1, rbuf};
    if (L0.val16) return dispatch(h, 0, L0.val16t, x, epi, nullptr, nullptr, s);
    return dispatch(h, 1, L0.val32t, x, epi, nullptr, nullptr, s);
}

cudaError_t launch_stream_up0(amg_hierarchy* h, const double* r, const float* x, const float* invd, double* z,
                              const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s) {
    if (h->stream == 2) return sell_up0(h, r, x, invd, z, q, part_rz, part_zq, flexible, s);
    const Level& L0 = h->lev[0];
    const EpiUp0 epi{{r, invd, q}, {8, 4, 8}, flexible ? 3 : 2, z, flexible};
    double* p2 = flexible ? part_zq : nullptr;
    if (L0.val16) return dispatch(h, 0, L0.val16t, x, epi, part_rz, p2, s);
    return dispatch(h, 1, L0.val32t, x, epi, part_rz, p2, s);
}

cudaError_t launch_stream_spmv_pq(amg_hierarchy* h, const float* p32, const double* p, const double* r, double* q,
                                  double* part_pq, double* part_pr, int flexible, cudaStream_t s) {
    if (h->stream == 2) return sell_spmv_pq(h, p32, p, r, q, part_pq, part_pr, flexible, s);
    const Level& L0 = h->lev[0];
    const EpiPQ epi{{p, r, nullptr}, {8, 8, 0}, flexible ? 2 : 1, q, flexible};
    return dispatch(h, 1, L0.val32t, p32, epi, part_pq, flexible ? part_pr : nullptr, s);
}

// Self-test of the bounded mbarrier wait of the staged passes: one thread
// waits, with a limit of `limit` cycles, on a barrier that nothing ever
// completes (it must give up) and on one whose phase it completes itself
// (it must return at once).
__global__ void k_wait_probe(long long limit, int* out) {
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x != 0) return;
    const uint32_t b0 = smem_addr(&bars[0]), b1 = smem_addr(&bars[1]);
    mbar_init(b0, 1);
    mbar_init(b1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    out[0] = mbar_wait_bounded(b0, 0u, limit) ? 0 : 1;  // never completed: expires
    mbar_arrive(b1);
    out[1] = mbar_wait_bounded(b1, 0u, limit) ? 1 : 0;  // completed phase 0
}

}  // namespace amg

int amg_staged_wait_selftest(double limit_ms, int32_t* timed_out, int32_t* completed) {
    if (!timed_out || !completed || !(limit_ms > 0.0) || limit_ms > 1000.0) return AMG_ERR_ARG;
    int dev = 0, khz = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess)
        return AMG_ERR_CUDA;
    int* d = nullptr;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return AMG_ERR_NOMEM;
    int hbuf[2] = {-1, -1};
    const long long limit = (long long)(limit_ms * (double)khz);  // kHz x ms = cycles
    amg::k_wait_probe<<<1, 32>>>(limit, d);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(hbuf, d, sizeof(hbuf), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return AMG_ERR_CUDA;
    *timed_out = hbuf[0];
    *completed = hbuf[1];
    return AMG_OK;
}
