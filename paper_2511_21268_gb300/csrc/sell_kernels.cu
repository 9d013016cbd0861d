// Finest-level passes of the mixed-precision solve on a sliced copy of the
// run-encoded matrix: 32-row slabs, one lane per row.
//
// The lane-per-run slab kernels (stream_kernels.cu) spend most of their
// issue slots on per-row work: row metadata, the run-length dispatch, the
// lane-partial tile and its shuffle reduction, and lanes left idle when a
// row's run count is not a multiple of 32 (49 runs of a 3-D cubic row fill
// 64 lane slots).  Here the finest matrix is re-laid out once, at setup, in
// slabs of 32 consecutive rows:
//   * slab k has Rs[k] = the largest run count of its rows run slots; slot r
//     of lane t (row 32 k + t) holds the start of that row's run r and LM
//     value slots (LM = the largest run length, rounded up to odd), stored
//     slot-major and lane-minor: value o of slot r of lane t at
//     ((soff[k] + r) LM + o) 32 + t, start at (soff[k] + r) 32 + t; the start
//     is kept as a 16-bit offset into the vector window of the grid block
//     that owns the slab (the window always fits in 64 K entries);
//   * rows with fewer runs, shorter runs, or no row at all (the last slab)
//     are padded with zero values whose columns stay inside the matrix; a run
//     that would reach past the last column is shifted left, its values
//     placed at the shifted offsets.
// Each block (one per SM) owns a contiguous range of slabs and first copies
// the window of the gathered vector its slabs reference into shared memory.
// A producer warp streams the slabs (values, start columns, epilogue vector
// segments) with cp.async.bulk into a ring of buffers completing on
// mbarriers.  The 16 compute warps split a slab's run slots (warp w takes
// slots w', w' + 16, ...; the assignment rotates from slab to slab), each
// lane accumulating its own row, so a slot costs one start-column load, and
// per value one value load, one vector load and one FMA, every load from
// shared memory at a compile-time offset.  Every compute warp writes its 32
// partial row sums to the buffer and moves on; a dedicated epilogue warp
// waits for all 16, adds them in a fixed pairwise tree (deterministic), and
// runs the epilogue (residual, smoothing with z and r.z, q = K p with p.q)
// with one lane per row, so no compute warp waits for an epilogue.  Dot
// products accumulate in the epilogue lanes in slab order and are written
// as one deterministic partial per block.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records
// AMG_ERR_TIMEOUT in the solve state, waits (again bounded) for its copies
// in flight and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "amg_internal.cuh"
#include "stream_common.cuh"

namespace amg {

namespace {

constexpr int kSlab = 32;                                   // rows per slab (one per lane)
constexpr uint32_t kSegBytes = kSlab * 8;                   // one staged epilogue segment
constexpr int kSellVec = 4;                                 // staged epilogue vectors, at most
constexpr int kMaxWinIntervals = 64;                        // window copies per block, at most
constexpr uint32_t kPartBytes = kStreamWarps * kSlab * 4;   // partial row sums of the 16 warps
constexpr int kSellBuf = 6;                                 // largest ring
constexpr int kProdWarp = kStreamWarps;                     // warp 16: producer
constexpr int kEpiWarp = kStreamWarps + 1;                  // warp 17: epilogues
constexpr int kSellThreads = (kStreamWarps + 2) * 32;
constexpr uint32_t kSellCtl = 256;                          // barriers and control words

struct SellShape {
    uint32_t xbytes;  // vector window bytes
    uint32_t vbytes;  // value area bytes per buffer (largest slab)
    uint32_t rbytes;  // start-column area bytes per buffer
    int nbuf;         // buffers in the ring (2..kSellBuf)
};

__host__ __device__ inline uint32_t sell_buffer_bytes(SellShape sh) {
    return sh.vbytes + sh.rbytes + kSellVec * kSegBytes + kPartBytes;
}

__host__ __device__ inline uint32_t sell_smem_bytes(SellShape sh) {
    return sh.xbytes + (uint32_t)sh.nbuf * sell_buffer_bytes(sh) + kSellCtl;
}

// Up sweep of level 0 for the sliced slabs: z = x + (r - K x) / d, r.z and
// z.q; x_i comes from a staged segment (the compacted window holds only
// the columns the slabs read, in their own order).
struct EpiUp0S {
    const void* vec[kSellVec];  // r (FP64), 1/d (FP32), x (FP32), q (FP64, flexible)
    int es[kSellVec];
    int nvec;
    double* z;
    int flexible;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t ss,
                                               const float*, double& rz, double& zq) const {
        const double ra = reinterpret_cast<const double*>(seg)[t];
        const float di = reinterpret_cast<const float*>(seg + ss)[t];
        const float xi = reinterpret_cast<const float*>(seg + 2 * ss)[t];
        const double za = (double)fmaf(di, (float)ra - s, xi);
        z[i] = za;
        rz += ra * za;
        if (flexible) zq += za * reinterpret_cast<const double*>(seg + 3 * ss)[t];
    }
};

// Level 1 (FP32 vectors): down-sweep residual rbuf = f - K x, and the up
// sweep's smoothed value y = x + (f - K x) / d (the prolongation into the
// finer level follows as a separate gather).
struct EpiResidF {
    const void* vec[1];  // f (FP32)
    int es[1];
    int nvec;
    float* rbuf;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t,
                                               const float*, double&, double&) const {
        rbuf[i] = reinterpret_cast<const float*>(seg)[t] - s;
    }
};

struct EpiUpY {
    const void* vec[3];  // f, 1/d, x (FP32)
    int es[3];
    int nvec;
    float* y;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t ss,
                                               const float*, double&, double&) const {
        const float f = reinterpret_cast<const float*>(seg)[t];
        const float di = reinterpret_cast<const float*>(seg + ss)[t];
        const float xi = reinterpret_cast<const float*>(seg + 2 * ss)[t];
        y[i] = fmaf(di, f - s, xi);
    }
};

// number of staged vectors an epilogue type can name
template <typename Epi>
constexpr int epi_vecs() {
    return (int)(sizeof(Epi::vec) / sizeof(Epi::vec[0]));
}

template <int OFF>
__device__ __forceinline__ float lds_val_at(uint32_t a, const float*) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
    return v;
}
template <int OFF>
__device__ __forceinline__ float lds_val_at(uint32_t a, const __nv_bfloat16*) {
    unsigned short u;
    asm volatile("ld.shared.u16 %0, [%1+%2];" : "=h"(u) : "r"(a), "n"(OFF));
    return __uint_as_float((uint32_t)u << 16);
}

__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    unsigned short u;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(u) : "r"(a));
    return (uint32_t)u;
}

// Value slots O .. LM-1 of one run slot: value o at va + o 32 sizeof(V),
// vector entry at xa + 4 o; two accumulators halve the FMA chain.
template <int O, int LM, typename V>
struct SlotDot {
    static __device__ __forceinline__ void run(uint32_t va, uint32_t xa, float& a0, float& a1) {
        const float v = lds_val_at<O * kSlab * (int)sizeof(V)>(va, static_cast<const V*>(nullptr));
        const float x = lds_x<4 * O>(xa);
        if (O & 1) a1 = fmaf(v, x, a1);
        else a0 = fmaf(v, x, a0);
        SlotDot<O + 1, LM, V>::run(va, xa, a0, a1);
    }
};
template <int LM, typename V>
struct SlotDot<LM, LM, V> {
    static __device__ __forceinline__ void run(uint32_t, uint32_t, float&, float&) {}
};

// BF16 run slots hold their values in pairs: value pair p (values 2p, 2p+1)
// of lane t at 4 (p 32 + t) bytes, then (odd LM) the last value at 2 (2P 32
// + t) bytes past the P = LM / 2 pairs.  One 4-byte load brings two values,
// so a slot of 7 costs 4 shared-memory loads instead of 7 (the BF16 passes
// are bound by the SM's shared-memory wavefronts, not by the FMAs).  The
// FMAs and their accumulators are the same as value by value.
template <int LM>
__device__ __forceinline__ void slot_dot_bf16(uint32_t sbase, int lane, uint32_t xa, float& a0, float& a1) {
    constexpr int P = LM / 2;
    const uint32_t pa = sbase + 4u * (uint32_t)lane;
#pragma unroll
    for (int p = 0; p < P; p++) {
        uint32_t u;
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(u) : "r"(pa + 4u * kSlab * (uint32_t)p));
        const float v0 = __uint_as_float(u << 16), v1 = __uint_as_float(u & 0xffff0000u);
        float x0, x1;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x0) : "r"(xa + 8u * (uint32_t)p));
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x1) : "r"(xa + 8u * (uint32_t)p + 4u));
        a0 = fmaf(v0, x0, a0);
        a1 = fmaf(v1, x1, a1);
    }
    if constexpr (LM & 1) {
        unsigned short h;
        asm volatile("ld.shared.u16 %0, [%1];" : "=h"(h) : "r"(sbase + 4u * kSlab * P + 2u * (uint32_t)lane));
        float x2;
        asm volatile("ld.shared.f32 %0, [%1];" : "=f"(x2) : "r"(xa + 8u * P));
        a0 = fmaf(__uint_as_float((uint32_t)h << 16), x2, a0);
    }
}

// Position of value o of lane t in a BF16 run slot of LM values (above).
__device__ __forceinline__ int bf16_slot_pos(int o, int t, int LM) {
    const int P = LM / 2;
    return o < 2 * P ? ((o >> 1) * kSlab + t) * 2 + (o & 1) : 2 * P * kSlab + t;
}

// Block b owns slabs [b nsl / G, (b + 1) nsl / G) and the vector window
// win[b] = (lo, hi), the smallest and largest column its slabs read.  The
// epilogue vectors are read in 16-byte-widened segments of the slab's rows
// (the vectors are padded for the last slab).
template <int LM, typename V, typename Epi>
__global__ void __launch_bounds__(kSellThreads, 1)
    k_sell(int n, int nsl, const int32_t* __restrict__ soff, const V* __restrict__ val, const uint16_t* __restrict__ rs,
           const float* __restrict__ xg, const int4* __restrict__ wint, const int* __restrict__ wcnt,
           const int* __restrict__ wbytes, SellShape shape, Epi epi, double* part1, double* part2, SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    const int nbuf = shape.nbuf;
    const float* xw = reinterpret_cast<const float*>(smem);
    unsigned char* ring = smem + shape.xbytes;
    const uint32_t bufstride = sell_buffer_bytes(shape);
    const uint32_t o_rs = shape.vbytes, o_seg = o_rs + shape.rbytes, o_part = o_seg + kSellVec * kSegBytes;
    unsigned char* ctl = ring + nbuf * bufstride;
    // [0] window, [1 + j] full[j], [1 + kSellBuf + j] empty[j], [1 + 2 kSellBuf + j] partials[j]
    uint64_t* bars = reinterpret_cast<uint64_t*>(ctl);
    constexpr int kBarBytes = 8 * (1 + 3 * kSellBuf);
    static_assert(kBarBytes + 4 * kSellBuf + 8 <= (int)kSellCtl, "control area");
    int* rsl = reinterpret_cast<int*>(ctl + kBarBytes);                                 // run slots of buffer j
    volatile int* ctrl = reinterpret_cast<int*>(ctl + kBarBytes + 4 * kSellBuf);       // 0 = go on, 1 = give up
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int s0 = (int)((int64_t)blockIdx.x * nsl / gridDim.x);
    const int s1 = (int)((int64_t)(blockIdx.x + 1) * nsl / gridDim.x);
    const uint32_t bar_win = smem_addr(&bars[0]);
    auto bar_full = [&](int j) { return smem_addr(&bars[1 + j]); };
    auto bar_empty = [&](int j) { return smem_addr(&bars[1 + kSellBuf + j]); };
    auto bar_part = [&](int j) { return smem_addr(&bars[1 + 2 * kSellBuf + j]); };

    if (threadIdx.x == 0) {
        mbar_init(bar_win, 1);
        for (int j = 0; j < kSellBuf; j++) {
            mbar_init(bar_full(j), 1);
            mbar_init(bar_empty(j), kStreamWarps + 1);  // compute warps + the epilogue warp
            mbar_init(bar_part(j), kStreamWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *ctrl = 0;
    }
    __syncthreads();

    double acc1 = 0.0, acc2 = 0.0;
    if (wid == kProdWarp) {
        // ------------------------------------------------------------ producer
        // The whole warp loads the slot offsets of the next 32 slabs at once
        // (one coalesced load instead of a dependent load per slab); lane 0
        // waits for buffers and issues the copies.
        if (s0 < s1) {
            int last_use = -1;  // last slab issued (lane 0)
            // the compacted window: interval q copies entries [x, x + y) of the
            // vector to window offset z (all multiples of 4)
            if (lane == 0) mbar_expect_tx(bar_win, (uint32_t)wbytes[blockIdx.x]);
            __syncwarp();
            for (int q = lane; q < wcnt[blockIdx.x]; q += 32) {
                const int4 iv = wint[blockIdx.x * kMaxWinIntervals + q];
                bulk_g2s(smem_addr(smem) + 4u * (uint32_t)iv.z, xg + iv.x, 4u * (uint32_t)iv.y, bar_win);
            }
            bool go = true;
            for (int kb = s0; kb < s1 && go; kb += 32) {
                const int ofs = soff[min(kb + lane, s1)];
                const int ofs_end = soff[min(kb + 32, s1)];
                const int cnt_k = min(32, s1 - kb);
                for (int t = 0; t < cnt_k; t++) {
                    const int o0 = __shfl_sync(FULL, ofs, t);
                    const int o1n = __shfl_sync(FULL, ofs, (t + 1) & 31);
                    const int o1 = t == 31 ? ofs_end : o1n;
                    if (lane == 0) {
                        const int k = kb + t;
                        const int u = (k - s0) / nbuf, j = (k - s0) % nbuf;
                        if (*ctrl || (u > 0 && !mbar_wait_bounded(bar_empty(j), (uint32_t)(u - 1) & 1u))) {
                            *ctrl = 1;
                            go = false;
                        } else {
                            const int R = o1 - o0;
                            rsl[j] = R;
                            const int a = k * kSlab;
                            const uint32_t cnt = (uint32_t)min(kSlab, n - a);
                            const uint32_t vb = (uint32_t)R * (uint32_t)(LM * kSlab * sizeof(V));
                            const uint32_t rb = (uint32_t)R * (uint32_t)(kSlab * 2);
                            uint32_t tx = vb + rb;
#pragma unroll
                            for (int v = 0; v < epi_vecs<Epi>(); v++)
                                if (v < epi.nvec) tx += align16(cnt * (uint32_t)epi.es[v]);
                            unsigned char* bv = ring + j * bufstride;
                            const uint32_t bar = bar_full(j);
                            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                            mbar_expect_tx(bar, tx);
                            if (R > 0) {
                                bulk_g2s(smem_addr(bv), val + (int64_t)o0 * (LM * kSlab), vb, bar);
                                bulk_g2s(smem_addr(bv + o_rs), rs + (int64_t)o0 * kSlab, rb, bar);
                            }
#pragma unroll
                            for (int v = 0; v < epi_vecs<Epi>(); v++)
                                if (v < epi.nvec)
                                    bulk_g2s(smem_addr(bv + o_seg + v * kSegBytes),
                                             reinterpret_cast<const unsigned char*>(epi.vec[v]) +
                                                 (int64_t)a * epi.es[v],
                                             align16(cnt * (uint32_t)epi.es[v]), bar);
                            last_use = k;
                        }
                    }
                    go = __shfl_sync(FULL, go, 0);
                    if (!go) break;
                }
            }
            if (lane == 0 && *ctrl) {  // drain copies that may still be in flight (bounded), keeping smem alive
                mbar_wait_bounded(bar_win, 0u);
                for (int k = max(s0, last_use - nbuf + 1); k <= last_use; k++)
                    mbar_wait_bounded(bar_full((k - s0) % nbuf), (uint32_t)((k - s0) / nbuf) & 1u);
            }
        }
    } else if (wid == kEpiWarp) {
        // ------------------------------------------------------------ epilogues
        // slab by slab: wait for the 16 partial row sums, add them in a fixed
        // pairwise tree, run the epilogue (a lane per row), release the buffer
        bool ok = true;
        for (int k = s0; k < s1 && ok; k++) {
            const int u = (k - s0) / nbuf, j = (k - s0) % nbuf;
            ok = __all_sync(FULL, !*ctrl && mbar_wait_bounded(bar_part(j), (uint32_t)u & 1u));
            if (!ok) break;
            const unsigned char* bv = ring + j * bufstride;
            const float* part = reinterpret_cast<const float*>(bv + o_part);
            float t[kStreamWarps];
#pragma unroll
            for (int w = 0; w < kStreamWarps; w++) t[w] = part[w * kSlab + lane];
#pragma unroll
            for (int h = kStreamWarps / 2; h > 0; h >>= 1)
#pragma unroll
                for (int w = 0; w < h; w++) t[w] += t[w + h];
            const int i = k * kSlab + lane;
            if (i < n) epi(i, lane, t[0], bv + o_seg, kSegBytes, nullptr, acc1, acc2);
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_empty(j));
        }
        if (!ok && lane == 0) *ctrl = 1;
    } else {
        // ------------------------------------------------------------ compute warps
        bool ok = true;
        if (s0 < s1) ok = __all_sync(FULL, mbar_wait_bounded(bar_win, 0u));
        const uint32_t xbase = smem_addr(xw);  // window offset q at xbase + 4 q
        for (int k = s0; k < s1 && ok; k++) {
            const int u = (k - s0) / nbuf, j = (k - s0) % nbuf;
            ok = __all_sync(FULL, !*ctrl && mbar_wait_bounded(bar_full(j), (uint32_t)u & 1u));
            if (!ok) break;
            unsigned char* bv = ring + j * bufstride;
            const int R = rsl[j];
            const int r0 = (wid + k - s0) & (kStreamWarps - 1);  // rotating slot offset
            const uint32_t va0 = smem_addr(bv) + (uint32_t)sizeof(V) * (uint32_t)lane;
            const uint32_t ra0 = smem_addr(bv + o_rs) + 2u * (uint32_t)lane;
            float a0 = 0.f, a1 = 0.f;
            int r = r0;
            if constexpr (LM == 1) {  // one entry per slot: four slots in flight
                float a2 = 0.f, a3 = 0.f;
#pragma unroll 1
                for (; r + 3 * kStreamWarps < R; r += 4 * kStreamWarps) {
                    uint32_t xa[4];
                    float v[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const uint32_t ru = (uint32_t)(r + u * kStreamWarps);
                        xa[u] = xbase + 4u * lds_u16(ra0 + ru * (uint32_t)(kSlab * 2));
                        v[u] = lds_val_at<0>(va0 + ru * (uint32_t)(kSlab * sizeof(V)), static_cast<const V*>(nullptr));
                    }
                    a0 = fmaf(v[0], lds_x<0>(xa[0]), a0);
                    a1 = fmaf(v[1], lds_x<0>(xa[1]), a1);
                    a2 = fmaf(v[2], lds_x<0>(xa[2]), a2);
                    a3 = fmaf(v[3], lds_x<0>(xa[3]), a3);
                }
                a0 += a2;
                a1 += a3;
            }
#pragma unroll 1
            for (; r < R; r += kStreamWarps) {
                const uint32_t xa = xbase + 4u * lds_u16(ra0 + (uint32_t)r * (uint32_t)(kSlab * 2));
                if constexpr (LM > 1 && sizeof(V) == 2)
                    slot_dot_bf16<LM>(smem_addr(bv) + (uint32_t)r * (uint32_t)(LM * kSlab * 2), lane, xa, a0, a1);
                else
                    SlotDot<0, LM, V>::run(va0 + (uint32_t)r * (uint32_t)(LM * kSlab * sizeof(V)), xa, a0, a1);
            }
            float* part = reinterpret_cast<float*>(bv + o_part);
            part[wid * kSlab + lane] = a0 + a1;
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(bar_part(j));
                mbar_arrive(bar_empty(j));  // done with buffer j
            }
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
    if (wid == kEpiWarp) {  // the block's dot-product partials (fixed order)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            acc1 += __shfl_xor_sync(FULL, acc1, o);
            acc2 += __shfl_xor_sync(FULL, acc2, o);
        }
        if (lane == 0) {
            if (part1) part1[blockIdx.x] = acc1;
            if (part2) part2[blockIdx.x] = acc2;
        }
    }
}

// ------------------------------------------------------------------ FP64
// The plain FP64 solve's finest-level passes on the same sliced slabs, with
// FP64 values.  GB300 issues about two FP64 FMAs per clock per SM, so these
// passes are bound by the FP64 pipe, not by HBM (about 87 M FMAs against
// 0.7 GB per pass on the 3-D p=3 n=64 system), and what counts is that nearly
// every FP64 instruction is a useful FMA.  A warp takes a whole slab and a
// lane its row; each lane runs its row's FMA chain over the run slots (two
// accumulators), with 8-16 values per lane in flight whatever the run
// length.  There are no partial sums to reduce across lanes and no lanes
// idle past a row's end, only the padded slots.
// Values come straight from global memory (one coalesced 256-byte load per
// value slot and warp); the block's compacted window of the gathered vector
// is first copied into shared memory in FP64 (the same window offsets as
// the FP32 copy).  Dot products: each lane adds its rows' terms in slab
// order, then the lanes and the warps are summed in a fixed order (one
// deterministic partial per block).
constexpr int kS64MinWarps = 12, kS64MaxWarps = 20;  // warps per block: chosen at setup (load balance)
constexpr int kS64Static = 1024;                      // static shared memory and slack

struct Epi64PQ {  // q = K p, p.q and (flexible) p.r
    const double* p;
    const double* r;
    double* q;
    int flexible;
    __device__ __forceinline__ void operator()(int i, double s, double& a1, double& a2) const {
        q[i] = s;
        const double pi = p[i];
        a1 += pi * s;
        if (flexible) a2 += pi * r[i];
    }
};

struct Epi64Resid {  // rbuf = f - K x
    const double* f;
    double* rbuf;
    __device__ __forceinline__ void operator()(int i, double s, double&, double&) const { rbuf[i] = f[i] - s; }
};

struct Epi64Up0 {  // z = x + (r - K x) / d, r.z and (flexible) z.q
    const double* r;
    const double* x;
    const double* invd;
    double* z;
    const double* q;
    int flexible;
    __device__ __forceinline__ void operator()(int i, double s, double& a1, double& a2) const {
        const double ra = r[i];
        const double za = fma(invd[i], ra - s, x[i]);
        z[i] = za;
        a1 += ra * za;
        if (flexible) a2 += za * q[i];
    }
};

// Chebyshev steps of the finest level (the paper's smoother, see
// vcycle_cheb): the matrix pass reads d (or x), the rest is row-local.
struct Epi64ChebStep {  // r = rprev - K dprev; dnew = a dprev + b D^-1 r; x += dprev (r may be rprev)
    const double* dprev;
    const double* rprev;
    double* r;
    const double* invd;
    double a, b;
    double* dnew;
    double* x;
    __device__ __forceinline__ void operator()(int i, double s, double&, double&) const {
        const double ri = rprev[i] - s;
        const double dp = dprev[i];
        r[i] = ri;
        dnew[i] = fma(b, invd[i] * ri, a * dp);
        x[i] += dp;
    }
};

struct Epi64ChebResid {  // r = rprev - K dprev; x += dprev (end of pre-smoothing)
    const double* dprev;
    const double* rprev;
    double* r;
    double* x;
    __device__ __forceinline__ void operator()(int i, double s, double&, double&) const {
        r[i] = rprev[i] - s;
        x[i] += dprev[i];
    }
};

struct Epi64ChebPost0 {  // r = f - K x; d = c0 D^-1 r (start of post-smoothing)
    const double* f;
    const double* invd;
    double c0;
    double* r;
    double* d;
    __device__ __forceinline__ void operator()(int i, double s, double&, double&) const {
        const double ri = f[i] - s;
        r[i] = ri;
        d[i] = c0 * invd[i] * ri;
    }
};

template <int LM, typename Epi>
__global__ void __launch_bounds__(kS64MaxWarps * 32, 1)
    k_sell64(int n, int nsl, const int32_t* __restrict__ soff, const double* __restrict__ val,
             const uint16_t* __restrict__ rs, const double* __restrict__ xg, const int4* __restrict__ wint,
             const int* __restrict__ wcnt, Epi epi, double* part1, double* part2, const SolveState* st) {
    pdl_entry();
    if (st && st->done) return;
    extern __shared__ __align__(128) unsigned char smem[];
    double* xw = reinterpret_cast<double*>(smem);
    __shared__ double red[2][kS64MaxWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int s0 = (int)((int64_t)blockIdx.x * nsl / gridDim.x);
    const int s1 = (int)((int64_t)(blockIdx.x + 1) * nsl / gridDim.x);
    // the compacted window: interval q holds entries [x, x + y) of the
    // vector at window offset z (all multiples of 4 entries)
    const int nq = s0 < s1 ? wcnt[blockIdx.x] : 0;
    for (int q = wid; q < nq; q += nw) {
        const int4 iv = wint[blockIdx.x * kMaxWinIntervals + q];
        const double2* src = reinterpret_cast<const double2*>(xg + iv.x);
        double2* dst = reinterpret_cast<double2*>(xw + iv.z);
        for (int e = lane; e < (iv.y >> 1); e += 32) dst[e] = src[e];
    }
    __syncthreads();
    double acc1 = 0.0, acc2 = 0.0;
    for (int k = s0 + wid; k < s1; k += nw) {
        const int o0 = __ldg(soff + k), R = __ldg(soff + k + 1) - o0;
        const double* __restrict__ vk = val + (int64_t)o0 * (LM * kSlab) + lane;
        const uint16_t* __restrict__ rk = rs + (int64_t)o0 * kSlab + lane;
        // SP slots per step (8-16 values per lane), the next step's values
        // loaded while this step's FMAs run; slot j of a step feeds
        // accumulator j & 1
        constexpr int SP = LM == 1 ? 8 : LM == 3 ? 4 : 2;
        double a0 = 0.0, a1 = 0.0;
        auto step = [&](const double (&v)[SP][LM], const int (&c)[SP], int live) {
#pragma unroll
            for (int j = 0; j < SP; j++)
                if (j < live)
#pragma unroll
                    for (int o = 0; o < LM; o++) {
                        if (j & 1) a1 = fma(v[j][o], xw[c[j] + o], a1);
                        else a0 = fma(v[j][o], xw[c[j] + o], a0);
                    }
        };
        int r = 0;
        if (R >= SP) {
            double v[SP][LM];
            int c[SP];
#pragma unroll
            for (int j = 0; j < SP; j++) {
                c[j] = __ldg(rk + j * kSlab);
#pragma unroll
                for (int o = 0; o < LM; o++) v[j][o] = __ldg(vk + (j * LM + o) * kSlab);
            }
#pragma unroll 1
            for (; r + 2 * SP <= R; r += SP) {
                double w[SP][LM];
                int d[SP];
#pragma unroll
                for (int j = 0; j < SP; j++) {
                    d[j] = __ldg(rk + (r + SP + j) * kSlab);
#pragma unroll
                    for (int o = 0; o < LM; o++) w[j][o] = __ldg(vk + ((r + SP + j) * LM + o) * kSlab);
                }
                step(v, c, SP);
#pragma unroll
                for (int j = 0; j < SP; j++) {
                    c[j] = d[j];
#pragma unroll
                    for (int o = 0; o < LM; o++) v[j][o] = w[j][o];
                }
            }
            step(v, c, SP);
            r += SP;
        }
        if (r < R) {  // fewer than SP slots left: one predicated step
            double v[SP][LM];
            int c[SP];
#pragma unroll
            for (int j = 0; j < SP; j++) {
                const bool in = r + j < R;
                c[j] = in ? __ldg(rk + (r + j) * kSlab) : 0;
#pragma unroll
                for (int o = 0; o < LM; o++) v[j][o] = in ? __ldg(vk + ((r + j) * LM + o) * kSlab) : 0.0;
            }
            step(v, c, R - r);
        }
        const int i = k * kSlab + lane;
        if (i < n) epi(i, a0 + a1, acc1, acc2);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc1 += __shfl_xor_sync(FULL, acc1, o);
        acc2 += __shfl_xor_sync(FULL, acc2, o);
    }
    if (lane == 0) {
        red[0][wid] = acc1;
        red[1][wid] = acc2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < nw; w++) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        if (part1) part1[blockIdx.x] = t1;
        if (part2) part2[blockIdx.x] = t2;
    }
}

// Run slots of each slab (the largest run count of its rows) and the
// largest run length of the matrix (atomic max); a warp per slab.
__global__ void k_sell_slots(int n, int nsl, const int32_t* __restrict__ rptr, const uint8_t* __restrict__ rlen,
                             int32_t* slots, int* lmax) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nsl; k += nw) {
        const int i = k * kSlab + lane;
        int R = 0, L = 0;
        if (i < n) {
            R = rptr[i + 1] - rptr[i];
            L = rlen[i];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            R = max(R, __shfl_xor_sync(FULL, R, o));
            L = max(L, __shfl_xor_sync(FULL, L, o));
        }
        if (lane == 0) {
            slots[k] = R;
            atomicMax(lmax, L);
        }
    }
}

// Start column of slot r of row i in the sliced layout: the run's start c
// shifted left to min(c, n - LM) (its values move right by the shift), or
// the slab's padding column for an empty slot.
__device__ __forceinline__ int slot_start(int c0, int n, int LM) { return min(c0, n - LM); }

// Smallest and largest column each slab reads (a warp per slab, a lane per
// row): swin[k].
__global__ void k_sell_span(int n, int nsl, int LM, const int32_t* __restrict__ rptr,
                            const int32_t* __restrict__ rst, const int32_t* __restrict__ soff, int2* swin) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nsl; k += nw) {
        const int i = k * kSlab + lane;
        const int f0 = rptr[k * kSlab];
        const int cpad = rptr[k * kSlab + 1] > f0 ? max(0, slot_start(rst[f0], n, LM)) : 0;
        int lo = cpad, hi = cpad + LM - 1;
        if (i < n) {
            const int r0 = rptr[i], Ri = rptr[i + 1] - r0;
            for (int r = 0; r < Ri; r++) {
                const int c = slot_start(rst[r0 + r], n, LM);
                lo = min(lo, c);
                hi = max(hi, c + LM - 1);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = min(lo, __shfl_xor_sync(FULL, lo, o));
            hi = max(hi, __shfl_xor_sync(FULL, hi, o));
        }
        if (lane == 0) swin[k] = make_int2(lo, hi);
    }
}

// The vector window of grid block b (owner of slab k when
// b = ((k + 1) G - 1) / nsl) is compacted: column c lies in 4-entry group
// g = (c - lo4) / 4, lo4 = win[b].x & ~3; only groups some slot reads are
// copied, in order, and group g lands at window offset 4 rank[goff[b] + g].
// k_sell_mark sets bit g of the block's group bitmap (from word
// wordoff[b]) for every group a slot reads; lanes of a warp whose groups
// fall in the same word OR their masks first (one atomic per word).
__device__ __forceinline__ int slot_pad(const int32_t* __restrict__ rptr, const int32_t* __restrict__ rst, int k,
                                        int n, int LM) {
    const int f0 = rptr[k * kSlab];
    return rptr[k * kSlab + 1] > f0 ? max(0, slot_start(rst[f0], n, LM)) : 0;
}

__global__ void k_sell_mark(int n, int nsl, int G, int LM, const int32_t* __restrict__ rptr,
                            const int32_t* __restrict__ rst, const int32_t* __restrict__ soff,
                            const int2* __restrict__ win, const int* __restrict__ wordoff, uint32_t* bits) {
    pdl_entry();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; k < nsl; k += nw) {
        const int i = k * kSlab + lane;
        const int Rs = soff[k + 1] - soff[k];
        const int b = (int)(((int64_t)(k + 1) * G - 1) / nsl);
        const int lo4 = win[b].x & ~3;
        uint32_t* bb = bits + wordoff[b];
        int r0 = 0, Ri = 0;
        if (i < n) {
            r0 = rptr[i];
            Ri = rptr[i + 1] - r0;
        }
        const int cpad = slot_pad(rptr, rst, k, n, LM);
        for (int r = 0; r < Rs; r++) {
            const int c = r < Ri ? slot_start(rst[r0 + r], n, LM) : cpad;
            const int g0 = (c - lo4) >> 2, g1 = (c + LM - 1 - lo4) >> 2;  // at most 3 groups, 2 words
            const int wa = g0 >> 5, wb = g1 >> 5;
            uint32_t ma = 0, mb = 0;
            for (int g = g0; g <= g1; g++) {
                if ((g >> 5) == wa) ma |= 1u << (g & 31);
                else mb |= 1u << (g & 31);
            }
            // lanes sharing a word OR their masks; the lowest of them writes
            const unsigned pa = __match_any_sync(FULL, wa);
            ma = __reduce_or_sync(pa, ma);
            if (lane == __ffs(pa) - 1) atomicOr(bb + wa, ma);
            const bool two = wb != wa;
            const unsigned pb = __match_any_sync(FULL, two ? wb : -1);
            mb = __reduce_or_sync(pb, mb);
            if (two && lane == __ffs(pb) - 1) atomicOr(bb + wb, mb);
        }
    }
}

// Intervals of the compacted window of grid block b (one warp per grid
// block): maximal runs of marked groups, found 32 groups at a time (a lane
// per group; run boundaries by ballot, written in order), at most
// kMaxWinIntervals of them: the smallest gaps are filled, the threshold T
// being the least gap length that leaves few enough runs when every gap
// <= T is copied too.  Writes the runs as (first column, entries, window
// offset) to wint[b kMaxWinIntervals + q], their count, the window bytes
// and the group ranks.  More run boundaries than the scan buffer holds:
// one interval over the whole range (no compaction).
__global__ void k_sell_intervals(int G, const int2* __restrict__ win, const int* __restrict__ wordoff,
                                 const int* __restrict__ goff, const uint32_t* __restrict__ bits, int4* wint,
                                 int* wcnt, int* wbytes, uint16_t* rank) {
    pdl_entry();
    constexpr int kBounds = 4096;  // run boundaries (2 per run)
    __shared__ int bpos[kBounds];
    __shared__ int ia[kMaxWinIntervals], ie[kMaxWinIntervals], id[kMaxWinIntervals];
    __shared__ int nint_s;
    const int b = blockIdx.x, lane = threadIdx.x;
    if (b >= G) return;
    const int lo4 = win[b].x & ~3;
    const int ng = goff[b + 1] - goff[b];
    const uint32_t* bb = bits + wordoff[b];
    // boundaries: g where marked(g) != marked(g - 1) (marked(-1) = marked(ng) = 0)
    int nb = 0;
    bool prev_last = false, over = false;
    for (int base = 0; base <= ng; base += 32) {
        const int g = base + lane;
        const bool m = g < ng && ((bb[g >> 5] >> (g & 31)) & 1u);
        const bool mp = __shfl_up_sync(FULL, m, 1);
        const bool prev = lane == 0 ? prev_last : mp;
        const unsigned bm = __ballot_sync(FULL, g <= ng && m != prev);
        const int at = nb + __popc(bm & ((1u << lane) - 1u));
        if (((bm >> lane) & 1u) && at < kBounds) bpos[at] = g;
        nb += __popc(bm);
        prev_last = __shfl_sync(FULL, m, 31);
    }
    if (nb > kBounds) over = true;
    __syncwarp();
    int nr = nb / 2;  // runs [bpos[2q], bpos[2q + 1])
    if (over || nr == 0) {
        if (lane == 0) {
            bpos[0] = 0;
            bpos[1] = ng;
        }
        nr = 1;
        __syncwarp();
    }
    int T = -1;  // fill gaps <= T
    if (nr > kMaxWinIntervals) {
        int lo = 0, hi = ng;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            int cnt = 0;
            for (int q = lane; q + 1 < nr; q += 32) cnt += (bpos[2 * q + 2] - bpos[2 * q + 1] > mid);
            cnt = 1 + __reduce_add_sync(FULL, cnt);
            if (cnt <= kMaxWinIntervals) hi = mid;
            else lo = mid + 1;
        }
        T = lo;
    }
    if (lane == 0) {  // merge runs separated by gaps <= T, assign window offsets
        int m = 0, d = 0;
        for (int q = 0; q < nr; q++) {
            const int a = bpos[2 * q];
            int e = bpos[2 * q + 1];
            while (q + 1 < nr && bpos[2 * q + 2] - e <= T) e = bpos[2 * (++q) + 1];
            ia[m] = a;
            ie[m] = e;
            id[m] = d;
            wint[b * kMaxWinIntervals + m] = make_int4(lo4 + 4 * a, 4 * (e - a), 4 * d, 0);
            d += e - a;
            m++;
        }
        nint_s = m;
        wcnt[b] = m;
        wbytes[b] = 16 * d;
    }
    __syncwarp();
    const int m = nint_s;
    for (int q = 0; q < m; q++)
        for (int g = ia[q] + lane; g < ie[q]; g += 32) rank[goff[b] + g] = (uint16_t)(id[q] + g - ia[q]);
}

// Fill the sliced copy, a thread block per slab: FP32 values, BF16 values
// (if o16: rounded from the FP32 value, as the BF16 copy of the level is;
// stored in value pairs within each run slot, see slot_dot_bf16)
// and the compacted-window offsets of the slot starts.  The slab's rows are
// consecutive, so their CSR values and run starts are two contiguous ranges:
// the block stages them in shared memory (sized for the largest slab: cap
// values, then capr run starts) with coalesced loads and writes the outputs
// in their own order, coalesced.  A run of row i (start c, L entries) goes to
// slot r at start c' = min(c, n - LM), its value q at offset q + c - c';
// empty slots (r >= the row's runs, or no row) read LM zeros from the
// slab's padding column (its first row's first start).
// T: the value type of the copy (FP32, with an optional BF16 copy, for the
// mixed-precision passes; FP64 for the plain FP64 passes).
template <typename T>
__global__ void __launch_bounds__(256) k_sell_fill(int n, int nsl, int G, int LM, int cap, int capr,
                                                   const int64_t* __restrict__ rp,
                                                   const int32_t* __restrict__ rptr, const uint8_t* __restrict__ rlen,
                                                   const int32_t* __restrict__ rst, const int32_t* __restrict__ soff,
                                                   const int2* __restrict__ win, const int* __restrict__ goff,
                                                   const uint16_t* __restrict__ rank, const T* __restrict__ v32,
                                                   T* o32, __nv_bfloat16* o16, uint16_t* ors) {
    pdl_entry();
    extern __shared__ __align__(16) unsigned char fill_smem[];
    T* sv = reinterpret_cast<T*>(fill_smem);
    int* srs = reinterpret_cast<int*>(fill_smem + sizeof(T) * (size_t)cap);
    __shared__ int mr0[kSlab], mri[kSlab], mli[kSlab];
    __shared__ int64_t me0[kSlab];
    for (int k = blockIdx.x; k < nsl; k += gridDim.x) {
        const int a = k * kSlab, e = min(n, a + kSlab);
        const int64_t ebase = rp[a], eend = rp[e];
        const int rbase = rptr[a], rend = rptr[e];
        const bool staged = eend - ebase <= cap && rend - rbase <= capr;
        __syncthreads();  // the previous slab's readers are done
        if (staged) {  // U loads in flight per thread before the stores (a slab of FP64 values
                       // fills most of the shared memory, so few blocks share an SM)
            constexpr int U = sizeof(T) == 8 ? 24 : 8;
            for (int64_t q0 = ebase + threadIdx.x; q0 < eend; q0 += U * blockDim.x) {
                T t[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t q = q0 + (int64_t)u * blockDim.x;
                    t[u] = q < eend ? v32[q] : T(0);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int64_t q = q0 + (int64_t)u * blockDim.x;
                    if (q < eend) sv[q - ebase] = t[u];
                }
            }
            for (int q0 = rbase + threadIdx.x; q0 < rend; q0 += U * blockDim.x) {
                int t[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int q = q0 + u * blockDim.x;
                    t[u] = q < rend ? rst[q] : 0;
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int q = q0 + u * blockDim.x;
                    if (q < rend) srs[q - rbase] = t[u];
                }
            }
        }
        if (threadIdx.x < kSlab) {
            const int i = a + threadIdx.x;
            int r0 = 0, ri = 0, li = 0;
            int64_t e0 = 0;
            if (i < n) {
                r0 = rptr[i];
                ri = rptr[i + 1] - r0;
                li = rlen[i];
                e0 = rp[i];
            }
            mr0[threadIdx.x] = staged ? r0 - rbase : r0;
            mri[threadIdx.x] = ri;
            mli[threadIdx.x] = li;
            me0[threadIdx.x] = staged ? e0 - ebase : e0;
        }
        __syncthreads();
        const int o0 = soff[k], Rs = soff[k + 1] - o0;
        const int b = (int)(((int64_t)(k + 1) * G - 1) / nsl);
        const int lo4 = win[b].x & ~3;
        const uint16_t* rk = rank + goff[b];
        const int cpad = slot_pad(rptr, rst, k, n, LM);
        const int* runs = staged ? srs : rst;
#pragma unroll 4
        for (int q = threadIdx.x; q < Rs * kSlab; q += blockDim.x) {  // slot starts
            const int t = q & (kSlab - 1), r = q / kSlab;
            const int c = r < mri[t] ? slot_start(runs[mr0[t] + r], n, LM) : cpad;
            ors[((int64_t)o0 + r) * kSlab + t] = (uint16_t)(4 * rk[(c - lo4) >> 2] + ((c - lo4) & 3));
        }
        for (int q = threadIdx.x; q < Rs * LM * kSlab; q += blockDim.x) {  // values
            const int t = q & (kSlab - 1), ro = q / kSlab;
            const int r = ro / LM, o = ro - r * LM;
            T val = T(0);
            if (r < mri[t]) {
                const int c0 = runs[mr0[t] + r];
                const int qv = o - (c0 - slot_start(c0, n, LM));
                if (qv >= 0 && qv < mli[t]) {
                    const int64_t src = me0[t] + (int64_t)r * mli[t] + qv;
                    val = staged ? sv[src] : v32[src];
                }
            }
            const int64_t dst = (((int64_t)o0 + r) * LM + o) * kSlab + t;
            o32[dst] = val;
            if constexpr (sizeof(T) == 4)  // BF16 slots in value pairs (slot_dot_bf16)
                if (o16)
                    o16[((int64_t)o0 + r) * LM * kSlab + (LM > 1 ? bf16_slot_pos(o, t, LM) : t)] =
                        __float2bfloat16_rn(val);
        }
    }
}

// int32 copy of row offsets (a plain CSR level's run pointers: every entry
// a run of one column).
__global__ void k_rowptr32(int n, const int64_t* __restrict__ rp, int32_t* out) {
    pdl_entry();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) out[i] = (int32_t)rp[i];
}

// Window of each grid block: smallest and largest column over its slabs.
__global__ void k_sell_window(int nsl, int G, const int2* __restrict__ swin, int2* win) {
    pdl_entry();
    __shared__ int slo[256], shi[256];
    const int b = blockIdx.x;
    const int k0 = (int)((int64_t)b * nsl / G), k1 = (int)((int64_t)(b + 1) * nsl / G);
    int lo = INT32_MAX, hi = -1;
    for (int k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        lo = min(lo, swin[k].x);
        hi = max(hi, swin[k].y);
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
    if (threadIdx.x == 0) win[b] = k1 > k0 ? make_int2(slo[0], shi[0]) : make_int2(0, 0);
}

SellShape sell_shape(const SellLevel& S, int q) {
    return SellShape{(uint32_t)S.xbytes, (uint32_t)S.vbytes[q], (uint32_t)S.rbytes, S.nbuf[q]};
}

template <int LM, typename V, typename Epi>
bool sell_attr(uint32_t smem) {
    return cudaFuncSetAttribute(k_sell<LM, V, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
           cudaSuccess;
}

template <int LM>
bool sell_attrs_lm(uint32_t m16, uint32_t m32) {
    return sell_attr<LM, __nv_bfloat16, EpiResid>(m16) && sell_attr<LM, __nv_bfloat16, EpiUp0S>(m16) &&
           sell_attr<LM, float, EpiResid>(m32) && sell_attr<LM, float, EpiUp0S>(m32) &&
           sell_attr<LM, float, EpiPQ>(m32);
}

template <int LM, typename V, typename Epi>
cudaError_t sell_launch_lm(amg_hierarchy* h, const SellLevel& S, int n, int q, const V* val, const float* x,
                           const Epi& epi, double* p1, double* p2, cudaStream_t s) {
    const SellShape sh = sell_shape(S, q);
    launch_pdl(k_sell<LM, V, Epi>, S.G, kSellThreads, sell_smem_bytes(sh), s, n, S.nsl, S.soff, val, S.rs, x,
               static_cast<const int4*>(S.wint), S.wcnt, S.wbytes, sh, epi, p1, p2, h->st);
    return cudaGetLastError();
}

template <typename V, typename Epi>
cudaError_t sell_launch(amg_hierarchy* h, int q, const V* val, const float* x, const Epi& epi, double* p1,
                        double* p2, cudaStream_t s) {
    const SellLevel& S = h->sell[0];
    const int n = h->lev[0].A.n;
    switch (S.lm) {
        case 3: return sell_launch_lm<3>(h, S, n, q, val, x, epi, p1, p2, s);
        case 5: return sell_launch_lm<5>(h, S, n, q, val, x, epi, p1, p2, s);
        case 7: return sell_launch_lm<7>(h, S, n, q, val, x, epi, p1, p2, s);
        default: return sell_launch_lm<9>(h, S, n, q, val, x, epi, p1, p2, s);
    }
}

// Build the sliced copy of one level (rows with runs: rp row offsets, rptr
// run pointers, rlen run lengths, rst run starts; a plain CSR level passes
// int32 row offsets as rptr, ones as rlen and its columns as rst) and size
// its ring.  Leaves S.on = 0 when the slabs average fewer than kMinSlots run
// slots (too few to occupy the 16 compute warps) or the window and two
// buffers do not fit the shared-memory budget.
int prepare_level(amg_hierarchy* h, SellLevel& S, int n, const int64_t* rp, const int32_t* rptr, const uint8_t* rlen,
                  const int32_t* rst, const float* v32, bool with16, int* scratch, int optin,
                  const double* v64 = nullptr) {
    const bool fp64 = v64 != nullptr;  // FP64 copy for k_sell64 (no copy ring), else FP32 (+ BF16) for k_sell
    constexpr int kMinSlots = 16;
    if (n < 16) return AMG_OK;
    const int nsl = (n + kSlab - 1) / kSlab;
    int32_t* slots = nullptr;
    if (dev_alloc(reinterpret_cast<void**>(&slots), sizeof(int32_t) * (nsl + 1), h->s) != cudaSuccess)
        return AMG_ERR_NOMEM;
    h->allocs.push_back(slots);
    const int gw = std::min((nsl + 7) / 8, 8192);
    if (cudaMemsetAsync(scratch, 0, sizeof(int), h->s) != cudaSuccess) return AMG_ERR_CUDA;
    launch_pdl(k_sell_slots, gw, 256, 0, h->s, n, nsl, rptr, rlen, slots, scratch);
    std::vector<int32_t> hs(nsl + 1);
    int lmax = 0;
    if (cudaMemcpyAsync(hs.data(), slots, sizeof(int32_t) * nsl, cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
        cudaMemcpyAsync(&lmax, scratch, sizeof(int), cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
        cudaStreamSynchronize(h->s) != cudaSuccess)
        return AMG_ERR_CUDA;
    if (lmax < 1 || lmax > kMaxRunLen) return AMG_OK;
    const int LM = lmax | 1;
    if (n < LM) return AMG_OK;
    int64_t total = 0;
    int rmax = 0;
    for (int k = 0; k < nsl; k++) {
        const int32_t r = hs[k];
        hs[k] = (int32_t)total;
        total += r;
        rmax = std::max(rmax, r);
    }
    hs[nsl] = (int32_t)total;
    if (total < (int64_t)kMinSlots * nsl || total * LM * kSlab >= ((int64_t)1 << 40) || total >= INT32_MAX)
        return AMG_OK;
    // shared-memory shape
    const int64_t vb16 = (int64_t)rmax * LM * kSlab * 2, vb32 = (int64_t)rmax * LM * kSlab * 4;
    const int64_t rb = (int64_t)rmax * kSlab * 2;
    if (!fp64 && vb32 + rb > (1 << 20)) return AMG_OK;
    if (cudaMemcpyAsync(slots, hs.data(), sizeof(int32_t) * (nsl + 1), cudaMemcpyHostToDevice, h->s) != cudaSuccess)
        return AMG_ERR_CUDA;
    // the sliced copy
    float* o32 = nullptr;
    double* o64 = nullptr;
    __nv_bfloat16* o16 = nullptr;
    uint16_t* ors = nullptr;
    int2* swin = nullptr;
    int2* win = nullptr;
    const size_t nv = (size_t)total * LM * kSlab;
    if (fp64) {
        if (dev_alloc(reinterpret_cast<void**>(&o64), sizeof(double) * nv, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
        h->allocs.push_back(o64);
    } else {
        if (dev_alloc(reinterpret_cast<void**>(&o32), sizeof(float) * nv, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
        h->allocs.push_back(o32);
    }
    if (with16 && !fp64) {
        if (dev_alloc(reinterpret_cast<void**>(&o16), sizeof(__nv_bfloat16) * nv, h->s) != cudaSuccess)
            return AMG_ERR_NOMEM;
        h->allocs.push_back(o16);
    }
    if (dev_alloc(reinterpret_cast<void**>(&ors), sizeof(uint16_t) * (size_t)total * kSlab, h->s) != cudaSuccess)
        return AMG_ERR_NOMEM;
    h->allocs.push_back(ors);
    if (dev_alloc(reinterpret_cast<void**>(&swin), sizeof(int2) * nsl, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
    h->allocs.push_back(swin);
    // blocks of the launch: one per SM unless a block's vector window
    // outgrows the 16-bit offsets or the shared memory; then 2, 4 or 8 per SM
    // (smaller blocks, smaller windows)
    const int Gmax = 8 * h->num_sms;
    if (dev_alloc(reinterpret_cast<void**>(&win), sizeof(int2) * Gmax, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
    h->allocs.push_back(win);
    const void* arrays[] = {o32, o64, o16, ors};
    for (const void* a : arrays)
        if (a && (reinterpret_cast<uintptr_t>(a) & 15)) return AMG_OK;
    launch_pdl(k_sell_span, gw, 256, 0, h->s, n, nsl, LM, rptr, rst, slots, swin);
    int *wordoff = nullptr, *goff = nullptr, *wcnt = nullptr, *wbytes = nullptr;
    int4* wint = nullptr;
    auto alloc = [&](void** p, size_t bytes) {
        if (dev_alloc(p, bytes, h->s) != cudaSuccess) return false;
        h->allocs.push_back(*p);
        return true;
    };
    if (!alloc(reinterpret_cast<void**>(&wordoff), sizeof(int) * (Gmax + 1)) ||
        !alloc(reinterpret_cast<void**>(&goff), sizeof(int) * (Gmax + 1)) ||
        !alloc(reinterpret_cast<void**>(&wcnt), sizeof(int) * Gmax) ||
        !alloc(reinterpret_cast<void**>(&wbytes), sizeof(int) * Gmax) ||
        !alloc(reinterpret_cast<void**>(&wint), sizeof(int4) * (size_t)Gmax * kMaxWinIntervals))
        return AMG_ERR_NOMEM;
    int G = 0;
    int64_t xw = 16;
    int nb[2] = {0, 0};
    uint16_t* rank_sel = nullptr;  // group ranks of the chosen block count
    for (int g = h->num_sms; g <= Gmax && !G; g *= 2) {
        if (g > h->num_sms && g > nsl) break;  // more blocks than slabs: nothing gained
        launch_pdl(k_sell_window, g, 256, 0, h->s, nsl, g, swin, win);
        std::vector<int2> hw(g);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hw.data(), win, sizeof(int2) * g, cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
            cudaStreamSynchronize(h->s) != cudaSuccess)
            return AMG_ERR_CUDA;
        // compacted windows: group bitmaps, intervals and group ranks
        std::vector<int> hword(g + 1, 0), hgoff(g + 1, 0);
        bool fits = true;
        for (int b = 0; b < g && fits; b++) {
            const int lo4 = hw[b].x & ~3;
            const int ng = hw[b].y >= lo4 ? ((hw[b].y - lo4) >> 2) + 1 : 0;
            if ((int64_t)ng * 16 > 4 * 65536) fits = false;  // offsets into the window are 16-bit
            hgoff[b + 1] = hgoff[b] + ng;
            hword[b + 1] = hword[b] + (ng + 31) / 32;
        }
        if (!fits) continue;
        uint32_t* bits = nullptr;
        uint16_t* rank = nullptr;
        if (!alloc(reinterpret_cast<void**>(&bits), sizeof(uint32_t) * std::max(hword[g], 1)) ||
            !alloc(reinterpret_cast<void**>(&rank), sizeof(uint16_t) * std::max(hgoff[g], 1)))
            return AMG_ERR_NOMEM;
        std::vector<int> hwb(g);
        if (cudaMemcpyAsync(wordoff, hword.data(), sizeof(int) * (g + 1), cudaMemcpyHostToDevice, h->s) !=
                cudaSuccess ||
            cudaMemcpyAsync(goff, hgoff.data(), sizeof(int) * (g + 1), cudaMemcpyHostToDevice, h->s) != cudaSuccess ||
            cudaMemsetAsync(bits, 0, sizeof(uint32_t) * std::max(hword[g], 1), h->s) != cudaSuccess)
            return AMG_ERR_CUDA;
        launch_pdl(k_sell_mark, gw, 256, 0, h->s, n, nsl, g, LM, rptr, rst, slots, win, wordoff, bits);
        launch_pdl(k_sell_intervals, g, 32, 0, h->s, g, win, wordoff, goff, bits, wint, wcnt, wbytes, rank);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(hwb.data(), wbytes, sizeof(int) * g, cudaMemcpyDeviceToHost, h->s) != cudaSuccess ||
            cudaStreamSynchronize(h->s) != cudaSuccess)
            return AMG_ERR_CUDA;
        xw = 16;
        for (int b = 0; b < g; b++) xw = std::max<int64_t>(xw, hwb[b]);
        if (fp64) {  // the window in FP64 and the block's dot-product scratch
            if (2 * xw + kS64Static > optin) continue;
        } else {
            nb[0] = nb[1] = 0;
            for (int q = 0; q < 2; q++) {
                const uint32_t vb = (uint32_t)(q == 0 ? vb16 : vb32);
                for (int k = kSellBuf; k >= 2 && !nb[q]; k--) {
                    const SellShape sh{(uint32_t)xw, vb, (uint32_t)rb, k};
                    if (sell_smem_bytes(sh) + 256u <= (uint32_t)optin) nb[q] = k;  // 256: static shared memory
                }
            }
            if (!nb[1] || (with16 && !nb[0])) continue;
        }
        G = g;
        rank_sel = rank;
    }
    if (!G) return AMG_OK;
    // stage: the largest slab's values and run starts (within the opt-in budget)
    const int64_t es = fp64 ? 8 : 4;
    const int capr = (int)std::min<int64_t>((int64_t)rmax * kSlab, (optin - 1024) / (4 + es));
    const int cap = (int)std::min<int64_t>((int64_t)capr * LM, (optin - 1024 - 4 * (int64_t)capr) / es);
    const size_t fsm = (size_t)es * cap + 4 * (size_t)capr;
    if (fp64) {
        if (cudaFuncSetAttribute(k_sell_fill<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) !=
            cudaSuccess)
            return AMG_ERR_CUDA;
        launch_pdl(k_sell_fill<double>, std::min(nsl, 65535), 256, fsm, h->s, n, nsl, G, LM, cap, capr, rp, rptr,
                   rlen, rst, slots, win, goff, rank_sel, v64, o64, nullptr, ors);
    } else {
        if (cudaFuncSetAttribute(k_sell_fill<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm) !=
            cudaSuccess)
            return AMG_ERR_CUDA;
        launch_pdl(k_sell_fill<float>, std::min(nsl, 65535), 256, fsm, h->s, n, nsl, G, LM, cap, capr, rp, rptr,
                   rlen, rst, slots, win, goff, rank_sel, v32, o32, o16, ors);
    }
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    S.lm = LM;
    S.nsl = nsl;
    S.soff = slots;
    S.v32 = o32;
    S.v64 = o64;
    S.v16 = o16;
    S.rs = ors;
    S.vbytes[0] = (int)vb16;
    S.vbytes[1] = (int)vb32;
    S.rbytes = (int)rb;
    S.slots = total;
    S.xbytes = (int)xw;
    S.nbuf[0] = nb[0];
    S.nbuf[1] = nb[1];
    S.wint = wint;
    S.wcnt = wcnt;
    S.wbytes = wbytes;
    S.G = G;
    S.on = 1;
    return AMG_OK;
}

}  // namespace

// Level 0: the sliced copy of the run-encoded finest level; sets h->stream =
// 2 and *used = 1 when it applies, else leaves the hierarchy unchanged.
int sell_prepare(amg_hierarchy* h, int* scratch, int optin, int* used) {
    *used = 0;
    Level& F0 = h->lev[0];
    SellLevel& S = h->sell[0];
    const int rc = prepare_level(h, S, F0.A.n, F0.A.rowptr, F0.run_ptr, F0.run_len, F0.run_start, F0.val32,
                                 F0.val16 != nullptr, scratch, optin);
    if (rc != AMG_OK || !S.on) return rc;
    const uint32_t m16 = S.nbuf[0] ? sell_smem_bytes(sell_shape(S, 0)) : 0u;
    const uint32_t m32 = sell_smem_bytes(sell_shape(S, 1));
    bool attrs;
    switch (S.lm) {
        case 3: attrs = sell_attrs_lm<3>(m16 ? m16 : m32, m32); break;
        case 5: attrs = sell_attrs_lm<5>(m16 ? m16 : m32, m32); break;
        case 7: attrs = sell_attrs_lm<7>(m16 ? m16 : m32, m32); break;
        default: attrs = sell_attrs_lm<9>(m16 ? m16 : m32, m32); break;
    }
    if (!attrs) return AMG_ERR_CUDA;
    if ((size_t)S.G + 2 > (size_t)h->npart) return AMG_OK;  // one dot-product partial per block
    h->stream_blocks = S.G;
    h->stream = 2;
    *used = 1;
    return AMG_OK;
}

cudaError_t sell_resid(amg_hierarchy* h, const double* f, const float* x, float* rbuf, cudaStream_t s) {
    const EpiResid epi{{f, nullptr, nullptr}, {8, 0, 0}, 1, rbuf};
    if (h->sell[0].v16) return sell_launch(h, 0, h->sell[0].v16, x, epi, nullptr, nullptr, s);
    return sell_launch(h, 1, h->sell[0].v32, x, epi, nullptr, nullptr, s);
}

cudaError_t sell_up0(amg_hierarchy* h, const double* r, const float* x, const float* invd, double* z,
                     const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s) {
    const EpiUp0S epi{{r, invd, x, q}, {8, 4, 4, 8}, flexible ? 4 : 3, z, flexible};
    double* p2 = flexible ? part_zq : nullptr;
    if (h->sell[0].v16) return sell_launch(h, 0, h->sell[0].v16, x, epi, part_rz, p2, s);
    return sell_launch(h, 1, h->sell[0].v32, x, epi, part_rz, p2, s);
}

cudaError_t sell_spmv_pq(amg_hierarchy* h, const float* p32, const double* p, const double* r, double* q,
                         double* part_pq, double* part_pr, int flexible, cudaStream_t s) {
    const EpiPQ epi{{p, r, nullptr}, {8, 8, 0}, flexible ? 2 : 1, q, flexible};
    return sell_launch(h, 1, h->sell[0].v32, p32, epi, part_pq, flexible ? part_pr : nullptr, s);
}

// Level 1 (plain CSR, FP32 values): the sliced copy with every entry a run
// of one column, when the hierarchy is mixed precision, has a level below
// level 1, fits int32 entry offsets, and the layout applies.
int sell_prepare_level1(amg_hierarchy* h, int* scratch) {
    SellLevel& S = h->sell[1];
    S.on = 0;
    if (!h->mixed || h->nlev < 3 || h->stream != 2) return AMG_OK;
    Level& L1 = h->lev[1];
    const int n = L1.A.n;
    if (n < 16 * kSlab || L1.A.nnz >= INT32_MAX || !L1.val32) return AMG_OK;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return AMG_ERR_CUDA;
    int32_t* rp32 = nullptr;
    uint8_t* ones = nullptr;
    if (dev_alloc(reinterpret_cast<void**>(&rp32), sizeof(int32_t) * (n + 1), h->s) != cudaSuccess)
        return AMG_ERR_NOMEM;
    h->allocs.push_back(rp32);
    if (dev_alloc(reinterpret_cast<void**>(&ones), (size_t)n + 16, h->s) != cudaSuccess) return AMG_ERR_NOMEM;
    h->allocs.push_back(ones);
    if (cudaMemsetAsync(ones, 1, (size_t)n + 16, h->s) != cudaSuccess) return AMG_ERR_CUDA;
    launch_pdl(k_rowptr32, std::min((n + 256) / 256, 4096), 256, 0, h->s, n, L1.A.rowptr, rp32);
    const int rc = prepare_level(h, S, n, L1.A.rowptr, rp32, ones, L1.A.col, L1.val32, false, scratch, optin);
    if (rc != AMG_OK || !S.on) return rc;
    if (S.lm != 1) {  // every run has one entry here
        S.on = 0;
        return AMG_OK;
    }
    const uint32_t m32 = sell_smem_bytes(sell_shape(S, 1));
    if (!sell_attr<1, float, EpiResidF>(m32) || !sell_attr<1, float, EpiUpY>(m32)) return AMG_ERR_CUDA;
    return AMG_OK;
}

cudaError_t sell_resid1(amg_hierarchy* h, const float* f, const float* x, float* rbuf, cudaStream_t s) {
    const EpiResidF epi{{f}, {4}, 1, rbuf};
    return sell_launch_lm<1>(h, h->sell[1], h->lev[1].A.n, 1, h->sell[1].v32, x, epi, nullptr, nullptr, s);
}

cudaError_t sell_upy1(amg_hierarchy* h, const float* f, const float* x, const float* invd, float* y, cudaStream_t s) {
    const EpiUpY epi{{f, invd, x}, {4, 4, 4}, 3, y};
    return sell_launch_lm<1>(h, h->sell[1], h->lev[1].A.n, 1, h->sell[1].v32, x, epi, nullptr, nullptr, s);
}

// ------------------------------------------------------------------ FP64
namespace {

template <int LM, typename Epi>
cudaError_t sell64_launch_lm(amg_hierarchy* h, const double* x, const Epi& epi, double* p1, double* p2,
                             cudaStream_t s) {
    const SellLevel& S = h->sell[0];
    launch_pdl(k_sell64<LM, Epi>, S.G, h->sell64_warps * 32, 2 * (size_t)S.xbytes, s, h->lev[0].A.n, S.nsl,
               S.soff, static_cast<const double*>(S.v64), S.rs, x, static_cast<const int4*>(S.wint), S.wcnt, epi,
               p1, p2, h->st);
    return cudaGetLastError();
}

template <typename Epi>
cudaError_t sell64_launch(amg_hierarchy* h, const double* x, const Epi& epi, double* p1, double* p2, cudaStream_t s) {
    switch (h->sell[0].lm) {
        case 3: return sell64_launch_lm<3>(h, x, epi, p1, p2, s);
        case 5: return sell64_launch_lm<5>(h, x, epi, p1, p2, s);
        case 7: return sell64_launch_lm<7>(h, x, epi, p1, p2, s);
        default: return sell64_launch_lm<9>(h, x, epi, p1, p2, s);
    }
}

// A warp takes whole slabs, so a block's time goes as ceil(slabs / W) W for
// the block with the most slabs (the FP64 pipe is shared by its W warps).
int sell64_pick_warps(const SellLevel& S, int G) {
    const int cmax = (S.nsl + G - 1) / G;
    int best = kS64MaxWarps;
    for (int w = kS64MaxWarps; w >= kS64MinWarps; w--)
        if (((cmax + w - 1) / w) * w < ((cmax + best - 1) / best) * best) best = w;
    return best;
}

template <int LM>
bool sell64_attrs_lm(int smem) {
    return cudaFuncSetAttribute(k_sell64<LM, Epi64PQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_sell64<LM, Epi64Resid>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_sell64<LM, Epi64Up0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_sell64<LM, Epi64ChebStep>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_sell64<LM, Epi64ChebResid>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_sell64<LM, Epi64ChebPost0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
               cudaSuccess;
}

}  // namespace

// Plain FP64 solve: the sliced copy of the run-encoded finest level with FP64
// values; sets h->sell64 when it applies, else leaves the hierarchy unchanged.
int sell64_prepare(amg_hierarchy* h, int* scratch) {
    h->sell64 = 0;
    Level& F0 = h->lev[0];
    SellLevel& S = h->sell[0];
    if (h->mixed || !F0.run_ptr || h->nlev < 2) return AMG_OK;
    const void* arrays[] = {F0.A.rowptr, F0.A.val, F0.x, F0.t, F0.invd, h->p, h->r, h->q, h->z};
    for (const void* a : arrays)
        if (a && (reinterpret_cast<uintptr_t>(a) & 15)) return AMG_OK;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return AMG_ERR_CUDA;
    const int rc = prepare_level(h, S, F0.A.n, F0.A.rowptr, F0.run_ptr, F0.run_len, F0.run_start, nullptr, false,
                                 scratch, optin, F0.A.val);
    if (rc != AMG_OK || !S.on) return rc;
    const int smem = 2 * S.xbytes;
    bool attrs;
    switch (S.lm) {
        case 3: attrs = sell64_attrs_lm<3>(smem); break;
        case 5: attrs = sell64_attrs_lm<5>(smem); break;
        case 7: attrs = sell64_attrs_lm<7>(smem); break;
        default: attrs = sell64_attrs_lm<9>(smem); break;
    }
    if (!attrs) return AMG_ERR_CUDA;
    if ((size_t)S.G + 2 > (size_t)h->npart) return AMG_OK;  // one dot-product partial per block
    h->sell64_warps = sell64_pick_warps(S, S.G);
    h->stream_blocks = S.G;
    h->sell64 = 1;
    return AMG_OK;
}

void sell64_warp_range(int* lo, int* hi) {
    *lo = kS64MinWarps;
    *hi = kS64MaxWarps;
}

cudaError_t sell64_spmv_pq(amg_hierarchy* h, const double* p, const double* r, double* q, double* part_pq,
                           double* part_pr, int flexible, cudaStream_t s) {
    return sell64_launch(h, p, Epi64PQ{p, r, q, flexible}, part_pq, flexible ? part_pr : nullptr, s);
}

cudaError_t sell64_resid(amg_hierarchy* h, const double* f, const double* x, double* rbuf, cudaStream_t s) {
    return sell64_launch(h, x, Epi64Resid{f, rbuf}, nullptr, nullptr, s);
}

cudaError_t sell64_up0(amg_hierarchy* h, const double* r, const double* x, const double* invd, double* z,
                       const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s) {
    return sell64_launch(h, x, Epi64Up0{r, x, invd, z, q, flexible}, part_rz, flexible ? part_zq : nullptr, s);
}

cudaError_t sell64_cheb_step(amg_hierarchy* h, const double* dprev, const double* rprev, double* r,
                             const double* invd, double a, double b, double* dnew, double* x, cudaStream_t s) {
    return sell64_launch(h, dprev, Epi64ChebStep{dprev, rprev, r, invd, a, b, dnew, x}, nullptr, nullptr, s);
}

cudaError_t sell64_cheb_resid(amg_hierarchy* h, const double* dprev, const double* rprev, double* r, double* x,
                              cudaStream_t s) {
    return sell64_launch(h, dprev, Epi64ChebResid{dprev, rprev, r, x}, nullptr, nullptr, s);
}

cudaError_t sell64_cheb_post0(amg_hierarchy* h, const double* x, const double* f, const double* invd, double c0,
                              double* r, double* d, cudaStream_t s) {
    return sell64_launch(h, x, Epi64ChebPost0{f, invd, c0, r, d}, nullptr, nullptr, s);
}

}  // namespace amg
