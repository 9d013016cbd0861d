// FP64 FMA throughput probe (measurement support; the paper has no
// counterpart).  The plain FP64 finest-level passes issue one FP64 FMA per
// stored matrix entry, and on GB300 their limit is the FP64 pipe rather than
// HBM; this kernel measures that pipe's rate on the GPU at hand so that the
// passes' roofline fraction is taken against a measured, not a nominal,
// FP64 peak.
//
// Each thread runs C independent FMA chains x <- x * a + b (a just below 1,
// b small: the values stay bounded and normal), kUnroll steps per loop
// trip, so every warp has C FMAs in flight per step and the grid keeps
// every SM's FP64 units busy.  The final values are summed per thread and
// written out, so no FMA can be removed.  The rate a variant reaches
// depends on more than the FMA count: with the multiplier and addend shared
// by all chains most shapes level off at 0.84 of the unit-count rate, while
// four chains with their own operands at 128 threads reach it; the caller
// times every variant and keeps the fastest.
#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace {

constexpr int kUnroll = 16;

template <int C, bool OWN>
__global__ void k_dfma_probe(int64_t trips, double a0, double b0, double* out) {
    double x[C], a[C], b[C];
#pragma unroll
    for (int c = 0; c < C; c++) {
        x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
        a[c] = a0 + 1e-12 * c;
        b[c] = b0 * (1 + c);
    }
    for (int64_t t = 0; t < trips; t++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int c = 0; c < C; c++) x[c] = OWN ? fma(x[c], a[c], b[c]) : fma(x[c], a0, b0);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < C; c++) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

struct Variant {
    void (*kern)(int64_t, double, double, double*);
    int chains, threads;
};

const Variant kVariants[] = {
    {k_dfma_probe<8, false>, 8, 256},
    {k_dfma_probe<4, true>, 4, 128},
    {k_dfma_probe<2, true>, 2, 128},
    {k_dfma_probe<8, true>, 8, 128},
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

}  // namespace

extern "C" int amg_dfma_probe(int32_t variant, int32_t blocks, int64_t trips, double* out_dev, void* cuda_stream,
                              int32_t* threads, double* flops) {
    if (variant == -1 && threads) {  // query: number of variants
        *threads = kNumVariants;
        return AMG_OK;
    }
    if (variant < 0 || variant >= kNumVariants) return AMG_ERR_ARG;
    const Variant& v = kVariants[variant];
    if (threads) *threads = v.threads;
    if (blocks == 0) return AMG_OK;  // query of the block size only
    if (blocks < 1 || trips < 1 || !out_dev) return AMG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    v.kern<<<AMG_GRID(blocks), v.threads, 0, s>>>(trips, 0.999999999, 1e-9, out_dev);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    if (flops) *flops = 2.0 * v.chains * kUnroll * (double)trips * (double)blocks * v.threads;
    return AMG_OK;
}

// Check of the library's correctly rounded division (div_rn, used by the
// edge weights of the matching): q[i] = div_rn(a[i], b[i]) and the number of
// quotients its fast path accepted.
namespace {
__global__ void k_div_check(int64_t n, const double* __restrict__ a, const double* __restrict__ b, double* q,
                            unsigned long long* fast) {
    unsigned long long local = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double f;
        const bool ok = amg::div_rn_fast(a[i], b[i], &f);
        q[i] = amg::div_rn(a[i], b[i]);
        local += ok ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
    if ((threadIdx.x & 31) == 0 && local) atomicAdd(fast, local);
}
}  // namespace

extern "C" int amg_div_check(int64_t n, const double* a_dev, const double* b_dev, double* q_dev,
                             uint64_t* fast_count_dev, void* cuda_stream) {
    if (n < 0 || (n > 0 && (!a_dev || !b_dev || !q_dev || !fast_count_dev))) return AMG_ERR_ARG;
    if (n == 0) return AMG_OK;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    k_div_check<<<AMG_GRID((int)blocks), 256, 0, s>>>(n, a_dev, b_dev, q_dev,
                                                     reinterpret_cast<unsigned long long*>(fast_count_dev));
    return cudaGetLastError() == cudaSuccess ? AMG_OK : AMG_ERR_CUDA;
}
