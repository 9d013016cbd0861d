// Shared pieces of the bulk-copy staged finest-level passes (the
// lane-per-run slab kernels and the sliced run-encoded kernels): mbarrier
// and bulk-copy wrappers with bounded waits, the epilogues, and
// shared-memory loads with 32-bit shared addresses.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace amg {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kStreamWarps = 16;                    // compute warps
constexpr int kStreamThreads = (kStreamWarps + 1) * 32;  // + one producer warp
constexpr int kMaxBuf = 3;
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
constexpr int kWaitIters = 1 << 28;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// global -> shared bulk copy completing on the mbarrier (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// try_wait that may suspend the thread for up to `ns` nanoseconds; the
// hardware resumes it when the phase completes.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint32_t bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of the mbarrier, suspending in the
// barrier between polls (the hardware resumes the waiter as soon as the
// phase completes; a sleep between polls instead cost microseconds per
// wait); every lane of a warp may call it together.  `limit`: clock cycles
// before giving up (about 2 s by default).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, long long limit = kWaitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (int it = 0; it < kWaitIters; it++) {
        if (mbar_try_wait_suspend(bar, parity, 20000u)) return true;
        if (clock64() - t0 > limit) break;
    }
    return false;
}

__device__ __forceinline__ float ldsv(const float* p, uint32_t k) { return p[k]; }
__device__ __forceinline__ float ldsv(const __nv_bfloat16* p, uint32_t k) { return __bfloat162float(p[k]); }

// epilogue input vectors staged per slab
constexpr int kMaxVec = 3;

__host__ __device__ constexpr uint32_t align16(uint32_t b) { return (b + 15u) & ~15u; }

// Epilogues: the owner lane of row i (t = i - first row of the slab) gets
// its total s; seg + v ss holds the slab's staged segment of the epilogue's
// input vector vec[v] (element t = entry i), xs the vector window (entry c
// at xs[c]); a1/a2 are the thread's running dot-product terms.
struct EpiResid {  // rbuf = f - K x
    const void* vec[kMaxVec];
    int es[kMaxVec];
    int nvec;
    float* rbuf;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t,
                                               const float*, double&, double&) const {
        const double fi = reinterpret_cast<const double*>(seg)[t];
        rbuf[i] = (float)fi - s;
    }
};

struct EpiUp0 {  // z = x + (r - K x) / d, r.z, z.q
    const void* vec[kMaxVec];  // r (FP64), 1/d (FP32), q (FP64, flexible)
    int es[kMaxVec];
    int nvec;
    double* z;
    int flexible;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t ss,
                                               const float* xs, double& rz, double& zq) const {
        const double ra = reinterpret_cast<const double*>(seg)[t];
        const float di = reinterpret_cast<const float*>(seg + ss)[t];
        const double za = (double)fmaf(di, (float)ra - s, xs[i]);
        z[i] = za;
        rz += ra * za;
        if (flexible) zq += za * reinterpret_cast<const double*>(seg + 2 * ss)[t];
    }
};

struct EpiPQ {  // q = K p, p.q, p.r
    const void* vec[kMaxVec];  // p (FP64), r (FP64, flexible)
    int es[kMaxVec];
    int nvec;
    double* q;
    int flexible;
    __device__ __forceinline__ void operator()(int i, int t, float s, const unsigned char* seg, uint32_t ss,
                                               const float*, double& pq, double& pr) const {
        const double qs = (double)s;
        q[i] = qs;
        const double pi = reinterpret_cast<const double*>(seg)[t];
        pq += pi * qs;
        if (flexible) pr += pi * reinterpret_cast<const double*>(seg + ss)[t];
    }
};

// Deterministic per-block sum of one double per thread -> out (thread 0).
__device__ __forceinline__ void block_sum_to(double v, double* sh, double* out) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w <= kStreamWarps; w++) t += sh[w];
        *out = t;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Shared-memory loads with 32-bit shared addresses (the vector entry at a
// compile-time offset from the run's first column).
__device__ __forceinline__ float lds_val(uint32_t a, const float*) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float lds_val(uint32_t a, const __nv_bfloat16*) {
    unsigned short u;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(u) : "r"(a));
    return __uint_as_float((uint32_t)u << 16);
}
__device__ __forceinline__ int lds_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
template <int OFF>
__device__ __forceinline__ float lds_x(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
    return v;
}

}  // namespace
}  // namespace amg
