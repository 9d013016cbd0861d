// amg_relres_noalloc: the relative residual ||F - K u||_2 / ||F||_2 of a
// device-resident CSR system, computed without allocating any memory.
//
// Who needs this: callers that cannot call cudaMalloc -- for example an
// application whose own pool allocator reserved the GPU's memory up front
// and forbids allocations outside it, or a time-critical loop where an
// allocation (and the device synchronisation it can trigger) is not
// acceptable.  amg_pcg_solve reports the same quantity but keeps its
// reduction scratch inside an amg_hierarchy, which must be allocated first.
//
// The reduction scratch here is a file-scope static device array of fixed
// size (about 1 MB per GPU, held by every GPU that loads the library until
// the process exits).  Limit: n <= AMG_NOALLOC_MAX_ROWS rows.
//
// Host code must not use the array's name as a device address (on the host
// it only names a host-side stand-in).  The first call on each device looks
// up the real address with cudaGetSymbolAddress while that device is
// current, caches it per device and passes it to the kernels.  The device is
// the one that owns the caller's stream (the current device for the NULL
// stream); the call makes it current for its duration and restores the
// caller's current device before returning.
//
// Launch failures are read from the launch calls themselves, so an earlier
// unrelated error pending in the caller's context is neither reported as
// this call's failure nor cleared.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "amg_gb300.h"

namespace {

constexpr int kNoallocWarps = 8;  // one row per warp, 8 warps per block
constexpr int kNoallocMaxBlocks = AMG_NOALLOC_MAX_ROWS / kNoallocWarps;
constexpr int kNoallocMaxDevices = 64;

// [0, B): ||r||^2 block partials, [B, 2B): ||F||^2 block partials,
// [2B]: the result.  Every slot a call reads is written earlier in the same
// call, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoallocMaxBlocks + 2];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kNoallocMaxDevices] = {};

__global__ void k_noalloc_partials(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                   const double* __restrict__ v, const double* __restrict__ u,
                                   const double* __restrict__ F, double* scratch, int nblocks) {
    __shared__ double srr[kNoallocWarps], sff[kNoallocWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * kNoallocWarps + wid;
    double rr = 0.0, ff = 0.0;
    if (i < n) {
        double s = 0.0;
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) s = fma(v[k], u[ci[k]], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const double fi = F[i], ri = fi - s;
        rr = ri * ri;
        ff = fi * fi;
    }
    if (lane == 0) {
        srr[wid] = rr;
        sff[wid] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kNoallocWarps; w++) {
            a += srr[w];
            b += sff[w];
        }
        scratch[blockIdx.x] = a;
        scratch[nblocks + blockIdx.x] = b;
    }
}

__global__ void k_noalloc_finish(double* scratch, int nblocks) {
    __shared__ double sa[32], sb[32];
    double a = 0.0, b = 0.0;
    for (int t = threadIdx.x; t < nblocks; t += blockDim.x) {
        a += scratch[t];
        b += scratch[nblocks + t];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            ta += sa[w];
            tb += sb[w];
        }
        scratch[2 * kNoallocMaxBlocks] = tb > 0.0 ? sqrt(ta) / sqrt(tb) : 0.0;
    }
}

// Device address of the scratch array on device `dev`, which must be the
// current device (looked up once per device).
int noalloc_scratch(int dev, double** out) {
    if (dev < 0 || dev >= kNoallocMaxDevices) return AMG_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return AMG_ERR_CUDA;
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AMG_OK;
}

// The work of amg_relres_noalloc on the current device, which owns s.
int relres_on_device(int dev, const amg_csr* K, const double* F, const double* u, double* relres, cudaStream_t s) {
    double* scratch = nullptr;
    int rc = noalloc_scratch(dev, &scratch);
    if (rc != AMG_OK) return rc;
    int n = K->n;
    int nblocks = (n + kNoallocWarps - 1) / kNoallocWarps;
    const int64_t* rp = K->rowptr;
    const int32_t* ci = K->col;
    const double* v = K->val;
    void* a1[] = {&n, &rp, &ci, &v, &u, &F, &scratch, &nblocks};
    cudaError_t e = cudaLaunchKernel((const void*)k_noalloc_partials, dim3(nblocks), dim3(kNoallocWarps * 32), a1, 0, s);
    void* a2[] = {&scratch, &nblocks};
    if (e == cudaSuccess) e = cudaLaunchKernel((const void*)k_noalloc_finish, dim3(1), dim3(256), a2, 0, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();  // this call's own launch error; leave no trace of it
        return AMG_ERR_CUDA;
    }
    if (cudaMemcpyAsync(relres, scratch + 2 * kNoallocMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return AMG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return AMG_ERR_CUDA;
    return AMG_OK;
}

}  // namespace

extern "C" int amg_relres_noalloc(const amg_csr* K, const double* F, const double* u, double* relres,
                                  void* cuda_stream) {
    if (!K || !F || !u || !relres || !K->rowptr || !K->col || !K->val) return AMG_ERR_ARG;
    if (K->mem != AMG_MEM_DEVICE || K->n < 1) return AMG_ERR_ARG;
    if (K->n > AMG_NOALLOC_MAX_ROWS) return AMG_ERR_ARG;  // beyond the static scratch
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int cur = 0, dev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess) return AMG_ERR_CUDA;
    if (cudaStreamGetDevice(s, &dev) != cudaSuccess) return AMG_ERR_CUDA;
    if (dev == cur) return relres_on_device(dev, K, F, u, relres, s);
    if (cudaSetDevice(dev) != cudaSuccess) return AMG_ERR_CUDA;
    const int rc = relres_on_device(dev, K, F, u, relres, s);
    if (cudaSetDevice(cur) != cudaSuccess) return AMG_ERR_CUDA;
    return rc;
}
