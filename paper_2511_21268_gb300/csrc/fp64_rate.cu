// FP64 FMA throughput probe (measurement support; the paper has no
// counterpart).  The plain FP64 finest-level passes issue one FP64 FMA per
// stored matrix entry, and on GB300 their limit is the FP64 pipe rather than
// HBM; this kernel measures that pipe's rate on the GPU at hand so that the
// passes' roofline fraction is taken against a measured, not a nominal,
// FP64 peak.
//
// Each thread runs kChains independent FMA chains x <- x * a + b (a just
// below 1, b small: the values stay bounded and normal), kUnroll steps per
// loop trip, so every warp has kChains FMAs in flight per step and the grid
// (several blocks per SM) keeps every SM's FP64 units busy.  The final
// values are summed per thread and written out, so no FMA can be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "amg_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_dfma_probe(int64_t trips, double a, double b, double* out) {
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) x[c] = 1.0 + 1e-3 * (double)(threadIdx.x + c);
    for (int64_t t = 0; t < trips; t++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int c = 0; c < kChains; c++) x[c] = fma(x[c], a, b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += x[c];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int amg_dfma_probe(int32_t blocks, int64_t trips, double* out_dev, void* cuda_stream, double* flops) {
    if (blocks < 1 || trips < 1 || !out_dev) return AMG_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    k_dfma_probe<<<AMG_GRID(blocks), kProbeThreads, 0, s>>>(trips, 0.999999999, 1e-9, out_dev);
    if (cudaGetLastError() != cudaSuccess) return AMG_ERR_CUDA;
    if (flops) *flops = 2.0 * kChains * kUnroll * (double)trips * (double)blocks * kProbeThreads;
    return AMG_OK;
}
