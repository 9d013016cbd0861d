// Learned per-row smoother damping (the paper has no learned component).
//
// The l1-Jacobi smoother of Sec. 3.2 is scaled per row,
//   x <- x + diag(omega_i / d_i) (f - K x),   0 < omega_i < omega_max,
// which stays convergent in the K-norm while 2 diag(d / omega) - K is
// positive definite, i.e. for every omega_i < 2 / lambda_max(D^-1 K).  The l1
// diagonal bounds lambda_max by 1; IgA levels have 0.7-0.9, where the
// best damping lies above 2.  So each level gets omega_max = 2 / lam_hat with
// lam_hat = min(1, a Lanczos upper estimate of lambda_max(D^-1 K)) (15 steps
// from a SplitMix64 start; the largest Ritz value plus its residual bound).
// omega comes from a two-layer message-passing network over each level's
// matrix graph (the same weights on every level); applying it only rescales
// each level's 1/d_i, so the FP64 and mixed-precision V-cycle kernels run
// the learned smoother unchanged.
//
// Network (hidden width 32):
//   node features  x_i = [rho_i, sig_i, log2(nnz_i) / 8, 1],
//                  rho_i = sum_{j!=i} |k_ij| / k_ii, sig_i = sum_{j!=i} k_ij / k_ii
//   edge weights   a_ij = k_ij / sqrt(k_ii k_jj)  (j != i; a_ii = 0)
//   h0 = relu(W0 x + b0); m_l = sum_j a_ij h_{l-1,j};
//   h_l = relu(U_l m_l + V_l h_{l-1} + b_l) (l = 1, 2);
//   omega = omega_max sigmoid(q.h2 + c)
// Training loss over probe vectors x_k (SplitMix64 uniform in (-1, 1)):
//   L = (1/m) sum_k log(y_k^T K y_k / x_k^T K x_k),  y_k = x_k - B_omega K x_k,
// B_omega the V-cycle (one pre- and one post-sweep, exact coarsest solve).
// The gradient runs the V-cycle steps backwards (FP64; the coarsest solve's
// adjoint is a second solve with the same symmetric inverse), then the
// network backwards (FP32 per node, per-block FP32 partial sums of the
// weight gradients added over blocks in FP64 in block order: deterministic).
//
// Layout: node-major [n][32] FP32 activations, a warp per node with
// lane = hidden unit; the aggregation is a 32-column SpMM over the level's
// CSR (one coalesced 128-byte row of h per stored entry); layer weights
// staged in shared memory, transposed so that a warp reads 32 consecutive
// words.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "amg_internal.cuh"

namespace amg {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int H = AMG_MPNN_HIDDEN;
static_assert(H == kWarp, "a warp per node, lane = hidden unit");
// flat parameter layout: W0[32][4], b0, U1[32][32], V1, b1, U2, V2, b2, q, c, qt, ct
constexpr int O_W0 = 0, O_B0 = O_W0 + H * 4, O_U1 = O_B0 + H, O_V1 = O_U1 + H * H, O_B1 = O_V1 + H * H,
              O_U2 = O_B1 + H, O_V2 = O_U2 + H * H, O_B2 = O_V2 + H * H, O_Q = O_B2 + H, O_C = O_Q + H,
              O_QT = O_C + 1, O_CT = O_QT + H, O_END = O_CT + 1;
static_assert(O_END == AMG_MPNN_NPARAM, "parameter layout");
constexpr int kGradBlocks = 256;           // blocks of the weight-gradient kernels
constexpr int kGradSlots = 2 * H * H + H;  // partial sums one block writes (largest kernel)
constexpr int kLzMax = 16;                 // Lanczos steps of the damping cap (at most)
constexpr int kLzSteps = 15;               // Lanczos steps taken (fewer on levels with fewer rows)
constexpr int kLzParts = 592;              // block partials of the Lanczos dot products (at most)
constexpr uint64_t kLzSeed = 0x4C414E43ULL;  // start vector of level l: SplitMix64(kLzSeed + l)

__device__ __forceinline__ float round_bf16(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// ---------------------------------------------------------------- features
// s_i = 1 / sqrt(k_ii) (FP32 copy of the FP64 value)
__global__ void k_nn_rsqrt_diag(int n, const double* __restrict__ kii, float* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) s[i] = (float)(1.0 / sqrt(kii[i]));
}

// Node features and edge weights in FP32: a_ij = s_i k_ij s_j (j != i),
// rho_i = sum |k_ij| / k_ii, sig_i = sum k_ij / k_ii over j != i.
__global__ void k_nn_features(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const double* __restrict__ v, const double* __restrict__ kii,
                              const float* __restrict__ sd, float* __restrict__ x, float* __restrict__ ap) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float si = sd[i];
        float ab = 0.f, sg = 0.f;
        const int64_t e = rp[i + 1];
        int64_t k = rp[i] + lane;
        // four entries per lane in flight
        for (; k + 96 < e; k += 128) {
            int j[4];
            float a[4], s[4];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                j[u] = ci[k + 32 * u];
                a[u] = (float)v[k + 32 * u];
            }
#pragma unroll
            for (int u = 0; u < 4; u++) s[u] = sd[j[u]];
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const bool off = j[u] != i;
                ab += off ? fabsf(a[u]) : 0.f;
                sg += off ? a[u] : 0.f;
                ap[k + 32 * u] = off ? si * a[u] * s[u] : 0.f;
            }
        }
        for (; k < e; k += 32) {
            const int j = ci[k];
            const float a = (float)v[k];
            float out = 0.f;
            if (j != i) {
                ab += fabsf(a);
                sg += a;
                out = si * a * sd[j];
            }
            ap[k] = out;
        }
        ab = warp_sumf(ab);
        sg = warp_sumf(sg);
        if (lane == 0) {
            const float ki = (float)kii[i];
            x[4 * (int64_t)i + 0] = ab / ki;
            x[4 * (int64_t)i + 1] = sg / ki;
            x[4 * (int64_t)i + 2] = (float)(log2((double)(rp[i + 1] - rp[i])) / 8.0);
            x[4 * (int64_t)i + 3] = 1.f;
        }
    }
}

// ------------------------------------------------------------------ forward
// One layer's weights in shared memory; Ut[k][j] = U[j][k] so that lane j
// reads consecutive words.
struct NetSmem {
    float W0t[4 * H], b0[H], Ut[H * H], Vt[H * H], b[H], q[H], qt[H], c, ct;
};

__device__ void load_net(const float* __restrict__ w, NetSmem& s, int layer, int bf16) {
    auto rd = [&](int o) { return bf16 ? round_bf16(w[o]) : w[o]; };
    const int oU = layer == 1 ? O_U1 : O_U2, oV = layer == 1 ? O_V1 : O_V2, oB = layer == 1 ? O_B1 : O_B2;
    for (int t = threadIdx.x; t < H * 4; t += blockDim.x) s.W0t[(t & 3) * H + (t >> 2)] = rd(O_W0 + t);
    for (int t = threadIdx.x; t < H; t += blockDim.x) {
        s.b0[t] = rd(O_B0 + t);
        s.b[t] = rd(oB + t);
        s.q[t] = rd(O_Q + t);
        s.qt[t] = rd(O_QT + t);
    }
    for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
        const int j = t / H, k = t % H;  // source U[j][k]
        s.Ut[k * H + j] = rd(oU + t);
        s.Vt[k * H + j] = rd(oV + t);
    }
    if (threadIdx.x == 0) {
        s.c = rd(O_C);
        s.ct = rd(O_CT);
    }
    __syncthreads();
}

// h0 = relu(u0), u0 = W0 x + b0
__global__ void __launch_bounds__(kBlock) k_nn_in(int n, const float* __restrict__ w, int bf16,
                                                   const float* __restrict__ x, float* __restrict__ u0,
                                                   float* __restrict__ h0) {
    __shared__ NetSmem s;
    load_net(w, s, 1, bf16);
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float4 xi = *reinterpret_cast<const float4*>(x + 4 * (int64_t)i);
        float u = s.b0[lane];
        u = fmaf(s.W0t[0 * H + lane], xi.x, u);
        u = fmaf(s.W0t[1 * H + lane], xi.y, u);
        u = fmaf(s.W0t[2 * H + lane], xi.z, u);
        u = fmaf(s.W0t[3 * H + lane], xi.w, u);
        u0[(int64_t)i * H + lane] = u;
        h0[(int64_t)i * H + lane] = fmaxf(u, 0.f);
    }
}

// out = base + A' h: a warp per row, lane = hidden unit; 32 entries' (a, j)
// are loaded at once (coalesced) and broadcast by shuffles.  A' is
// symmetric, so this also applies A'^T in the backward pass.
__global__ void __launch_bounds__(kBlock) k_nn_spmm(int n, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ ci, const float* __restrict__ ap,
                                                     const float* __restrict__ h, const float* __restrict__ base,
                                                     float* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        float acc0 = base ? base[(int64_t)i * H + lane] : 0.f, acc1 = 0.f;
        const int64_t k0 = rp[i], k1 = rp[i + 1];
        for (int64_t kb = k0; kb < k1; kb += 32) {
            const int cnt = k1 - kb < 32 ? (int)(k1 - kb) : 32;
            float a = 0.f;
            int j = 0;
            if (lane < cnt) {
                a = ap[kb + lane];
                j = ci[kb + lane];
            }
            // 8 rows of h in flight per lane
            int t = 0;
            for (; t + 7 < cnt; t += 8) {
                float hv[8], av[8];
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    av[u] = __shfl_sync(FULL, a, t + u);
                    hv[u] = h[(int64_t)__shfl_sync(FULL, j, t + u) * H + lane];
                }
#pragma unroll
                for (int u = 0; u < 8; u += 2) {
                    acc0 = fmaf(av[u], hv[u], acc0);
                    acc1 = fmaf(av[u + 1], hv[u + 1], acc1);
                }
            }
            for (; t < cnt; t++) {
                const float a0 = __shfl_sync(FULL, a, t);
                const int j0 = __shfl_sync(FULL, j, t);
                acc0 = fmaf(a0, h[(int64_t)j0 * H + lane], acc0);
            }
        }
        out[(int64_t)i * H + lane] = acc0 + acc1;
    }
}

// u = U m + V hp + b, h = relu(u); layer 2 also forms sigmoid(z) and omega,
// and (sgt non-NULL) the second head's sigmoid(zt) and theta (cap omega_max).
__global__ void __launch_bounds__(kBlock) k_nn_dense(int n, const float* __restrict__ w, int bf16, int layer,
                                                      const float* __restrict__ m, const float* __restrict__ hp,
                                                      float* __restrict__ u, float* __restrict__ h,
                                                      float* __restrict__ sg, float* __restrict__ omega,
                                                      const double* __restrict__ cap, float* __restrict__ sgt,
                                                      float* __restrict__ theta) {
    __shared__ NetSmem s;
    load_net(w, s, layer, bf16);
    const float omax = layer == 2 ? (float)cap[1] : 0.f;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float mi = m[(int64_t)i * H + lane], hi = hp[(int64_t)i * H + lane];
        float a0 = s.b[lane], a1 = 0.f;
#pragma unroll
        for (int k = 0; k < H; k++) {
            a0 = fmaf(s.Ut[k * H + lane], __shfl_sync(FULL, mi, k), a0);
            a1 = fmaf(s.Vt[k * H + lane], __shfl_sync(FULL, hi, k), a1);
        }
        const float acc = a0 + a1;
        u[(int64_t)i * H + lane] = acc;
        const float hh = fmaxf(acc, 0.f);
        h[(int64_t)i * H + lane] = hh;
        if (layer == 2) {
            const float t = warp_sumf(s.q[lane] * hh);
            if (lane == 0) {
                const float sgm = 1.f / (1.f + expf(-(t + s.c)));
                sg[i] = sgm;
                omega[i] = omax * sgm;
            }
            if (sgt) {
                const float tt = warp_sumf(s.qt[lane] * hh);
                if (lane == 0) {
                    const float st = 1.f / (1.f + expf(-(tt + s.ct)));
                    sgt[i] = st;
                    theta[i] = omax * st;
                }
            }
        }
    }
}

// ----------------------------------------------------------------- backward
// Fixed-order sum of one value per lane over the block's warps; warp 0
// writes the 32 sums to dst.
__device__ __forceinline__ void block_lane_sum(float (&red)[kWarpsPerBlock][H], float v, float* dst) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    red[wid][lane] = v;
    __syncthreads();
    if (wid == 0) {
        float t = 0.f;
        for (int k = 0; k < kWarpsPerBlock; k++) t += red[k][lane];
        dst[lane] = t;
    }
    __syncthreads();
}

// dz = domega omega_max sg (1 - sg) and (dtheta non-NULL) dzt = dtheta
// omega_max sgt (1 - sgt); partials dq[j] = sum dz h2[j] (slots [0, H)),
// dc = sum dz (slot H), dqt[j] (slots [H + 1, 2 H + 1)), dct (slot 2 H + 1);
// du2 = (dz q + dzt qt) [u2 > 0]
__global__ void __launch_bounds__(kBlock) k_nn_out_bwd(int n, const float* __restrict__ w,
                                                        const double* __restrict__ domega,
                                                        const float* __restrict__ sg, const float* __restrict__ h2,
                                                        const float* __restrict__ u2, float* __restrict__ du2,
                                                        float* __restrict__ part, const double* __restrict__ cap,
                                                        const double* __restrict__ dtheta,
                                                        const float* __restrict__ sgt) {
    __shared__ float red[kWarpsPerBlock][H];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const float q = w[O_Q + lane], qt = w[O_QT + lane];
    const float omax = (float)cap[1];
    float aq = 0.f, ac = 0.f, aqt = 0.f, act = 0.f;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float s = sg[i];
        const float dz = (float)domega[i] * omax * s * (1.f - s);
        float dzt = 0.f;
        if (dtheta) {
            const float st = sgt[i];
            dzt = (float)dtheta[i] * omax * st * (1.f - st);
        }
        const float hv = h2[(int64_t)i * H + lane];
        aq = fmaf(dz, hv, aq);
        ac += dz;
        aqt = fmaf(dzt, hv, aqt);
        act += dzt;
        du2[(int64_t)i * H + lane] = u2[(int64_t)i * H + lane] > 0.f ? fmaf(dz, q, dzt * qt) : 0.f;
    }
    float* out = part + (int64_t)blockIdx.x * kGradSlots;
    block_lane_sum(red, aq, out);
    block_lane_sum(red, lane == 0 ? ac : 0.f, out + H);  // slot H holds dc (H+1.. overwritten next)
    block_lane_sum(red, aqt, out + H + 1);
    block_lane_sum(red, lane == 0 ? act : 0.f, out + 2 * H + 1);
}

// Dense layer backward: dm = U^T du, dhp = V^T du; partials dU = du m^T
// (slot k H + j for U[j][k]), dV = du hp^T (slot H H + k H + j), db = du
// (slot 2 H H + j).
__global__ void __launch_bounds__(kBlock) k_nn_dense_bwd(int n, const float* __restrict__ w, int layer,
                                                          const float* __restrict__ du, const float* __restrict__ m,
                                                          const float* __restrict__ hp, float* __restrict__ dm,
                                                          float* __restrict__ dhp, float* __restrict__ part) {
    __shared__ float Us[H * H], Vs[H * H];
    __shared__ float red[kWarpsPerBlock][H];
    const int oU = layer == 1 ? O_U1 : O_U2, oV = layer == 1 ? O_V1 : O_V2;
    for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
        Us[t] = w[oU + t];
        Vs[t] = w[oV + t];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    float gU[H], gV[H], gb = 0.f;
#pragma unroll
    for (int k = 0; k < H; k++) gU[k] = gV[k] = 0.f;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float dj = du[(int64_t)i * H + lane];  // lane as output unit j
        const float mk = m[(int64_t)i * H + lane];   // lane as input unit k
        const float hk = hp[(int64_t)i * H + lane];
        float am = 0.f, ah = 0.f;
#pragma unroll
        for (int j = 0; j < H; j++) {
            const float dd = __shfl_sync(FULL, dj, j);
            am = fmaf(Us[j * H + lane], dd, am);
            ah = fmaf(Vs[j * H + lane], dd, ah);
        }
        dm[(int64_t)i * H + lane] = am;
        dhp[(int64_t)i * H + lane] = ah;
#pragma unroll
        for (int k = 0; k < H; k++) {
            gU[k] = fmaf(dj, __shfl_sync(FULL, mk, k), gU[k]);
            gV[k] = fmaf(dj, __shfl_sync(FULL, hk, k), gV[k]);
        }
        gb += dj;
    }
    float* out = part + (int64_t)blockIdx.x * kGradSlots;
#pragma unroll
    for (int k = 0; k < H; k++) {
        block_lane_sum(red, gU[k], out + k * H);
        block_lane_sum(red, gV[k], out + H * H + k * H);
    }
    block_lane_sum(red, gb, out + 2 * H * H);
}

// dh *= [u > 0] (in place), over cnt entries
__global__ void k_nn_relu_mask(int64_t cnt, const float* __restrict__ u, float* __restrict__ dh) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < cnt && !(u[g] > 0.f)) dh[g] = 0.f;
}

// partials dW0[j][f] = sum du0[j] x[f] (slot f H + j), db0 (slot 4 H + j)
__global__ void __launch_bounds__(kBlock) k_nn_in_bwd(int n, const float* __restrict__ du0,
                                                       const float* __restrict__ x, float* __restrict__ part) {
    __shared__ float red[kWarpsPerBlock][H];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        const float dj = du0[(int64_t)i * H + lane];
        const float4 xi = *reinterpret_cast<const float4*>(x + 4 * (int64_t)i);
        g[0] = fmaf(dj, xi.x, g[0]);
        g[1] = fmaf(dj, xi.y, g[1]);
        g[2] = fmaf(dj, xi.z, g[2]);
        g[3] = fmaf(dj, xi.w, g[3]);
        g[4] += dj;
    }
    float* out = part + (int64_t)blockIdx.x * kGradSlots;
#pragma unroll
    for (int f = 0; f < 5; f++) block_lane_sum(red, g[f], out + f * H);
}

// gacc[dst[t]] += sum over blocks (in block order, FP64) of slot t
__global__ void k_nn_grad_sum(int nblocks, const float* __restrict__ part, int count, const int* __restrict__ dst,
                              double* __restrict__ gacc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; b++) s += (double)part[(int64_t)b * kGradSlots + t];
    gacc[dst[t]] += s;
}

// ------------------------------------------------ damped V-cycle (FP64)
// out = y + s K x  (y may be NULL), a warp per row
__global__ void __launch_bounds__(kBlock) k_v_spmv(int n, const int64_t* __restrict__ rp,
                                                    const int32_t* __restrict__ ci, const double* __restrict__ v,
                                                    const double* __restrict__ x, const double* __restrict__ y,
                                                    double s, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
        double acc = 0.0;
        for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) acc = fma(v[k], x[ci[k]], acc);
        acc = warp_sum(acc);
        if (lane == 0) out[i] = (y ? y[i] : 0.0) + s * acc;
    }
}

// out = a + (omega / d) b   (a may be NULL)
__global__ void k_v_damp(int n, const double* __restrict__ a, const float* __restrict__ om,
                         const double* __restrict__ d, const double* __restrict__ b, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (a ? a[i] : 0.0) + ((double)om[i] / d[i]) * b[i];
}

// dom += g r / d
__global__ void k_v_domega(int n, const double* __restrict__ g, const double* __restrict__ r,
                           const double* __restrict__ d, double* __restrict__ dom) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dom[i] += g[i] * r[i] / d[i];
}

// fc = P^T r over each coarse row's members (ascending)
__global__ void k_v_restrict(int nc, const int32_t* __restrict__ mptr, const int32_t* __restrict__ midx,
                             const double* __restrict__ pval, const double* __restrict__ r, double* __restrict__ fc) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nc) return;
    double acc = 0.0;
    for (int m = mptr[I]; m < mptr[I + 1]; m++) acc = fma(pval[midx[m]], r[midx[m]], acc);
    fc[I] = acc;
}

// out = a + P e  (a may be NULL)
__global__ void k_v_prolong(int n, const int32_t* __restrict__ agg, const double* __restrict__ pval,
                            const double* __restrict__ e, const double* __restrict__ a, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (a ? a[i] : 0.0) + pval[i] * e[agg[i]];
}

// out = A^-1 f with the dense symmetric inverse of the coarsest matrix
__global__ void k_v_dense(int nd, const double* __restrict__ Ainv, const double* __restrict__ f,
                          double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int I = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (I >= nd) return;
    double s = 0.0;
    for (int j = lane; j < nd; j += 32) s = fma(Ainv[(int64_t)I * nd + j], f[j], s);
    s = warp_sum(s);
    if (lane == 0) out[I] = s;
}

// out = dr2 + dr1 + (omega / d) dx1  (the three contributions to d loss / d f)
__global__ void k_v_df(int n, const double* __restrict__ dr2, const double* __restrict__ dr1,
                       const float* __restrict__ om, const double* __restrict__ d, const double* __restrict__ dx1,
                       double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (dr2[i] + dr1[i]) + ((double)om[i] / d[i]) * dx1[i];
}

// probe x_i = 2 U - 1, U = top 53 bits of draw (k n + i) of SplitMix64(seed) / 2^53
__global__ void k_v_probe(int n, uint64_t seed, int k, double* __restrict__ x) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const uint64_t z = splitmix64_at(seed, (uint64_t)k * (uint64_t)n + (uint64_t)i);
        x[i] = 2.0 * ((double)(z >> 11) * 0x1.0p-53) - 1.0;
    }
}

__global__ void k_v_sub(int n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - b[i];
}

// dots[0] = a.b, dots[1] = c.d (one block, fixed order)
__global__ void __launch_bounds__(1024) k_v_dot2(int n, const double* __restrict__ a, const double* __restrict__ b,
                                                 const double* __restrict__ c, const double* __restrict__ d,
                                                 double* __restrict__ dots) {
    __shared__ double s1[32], s2[32];
    double t1 = 0.0, t2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        t1 = fma(a[i], b[i], t1);
        t2 = fma(c[i], d[i], t2);
    }
    t1 = warp_sum(t1);
    t2 = warp_sum(t2);
    if ((threadIdx.x & 31) == 0) {
        s1[threadIdx.x >> 5] = t1;
        s2[threadIdx.x >> 5] = t2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double u1 = 0.0, u2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            u1 += s1[w];
            u2 += s2[w];
        }
        dots[0] = u1;
        dots[1] = u2;
    }
}

// loss += (log(y.Ky) - log(x.Kx)) / m; gbar = -2 Ky / (y.Ky) / m
// (d/dz of log(y^T K y) with y = x - z); flags a non-positive quotient
__global__ void k_v_lossgrad(int n, const double* __restrict__ Ky, const double* __restrict__ dots, double inv_m,
                             double* __restrict__ gbar, double* __restrict__ loss, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double yKy = dots[0], xKx = dots[1];
    const bool ok = yKy > 0.0 && xKx > 0.0;
    if (i < n) gbar[i] = ok ? -2.0 * Ky[i] / yKy * inv_m : 0.0;
    if (i == 0) {
        if (ok)
            *loss += (log(yKy) - log(xKx)) * inv_m;
        else
            *bad = 1;
    }
}

// ------------------------------ two-grid loss of the smoothing weights (FP64)
// out = x - (omega / d) kx
__global__ void k_tg_damp_sub(int n, const double* __restrict__ x, const float* __restrict__ om,
                              const double* __restrict__ d, const double* __restrict__ kx, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = x[i] - ((double)om[i] / d[i]) * kx[i];
}

// out = (omega / d) a
__global__ void k_tg_mul(int n, const float* __restrict__ om, const double* __restrict__ d,
                         const double* __restrict__ a, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ((double)om[i] / d[i]) * a[i];
}

// loss += (log(y.Ky) - log(x.Kx)) / m; ybar = 2 Ky / (y.Ky) / m; flags a
// non-positive quotient
__global__ void k_tg_lossgrad(int n, const double* __restrict__ Ky, const double* __restrict__ dots, double inv_m,
                              double* __restrict__ ybar, double* __restrict__ loss, int* __restrict__ bad) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double yKy = dots[0], xKx = dots[1];
    const bool ok = yKy > 0.0 && xKx > 0.0;
    if (i < n) ybar[i] = ok ? 2.0 * Ky[i] / yKy * inv_m : 0.0;
    if (i == 0) {
        if (ok)
            *loss += (log(yKy) - log(xKx)) * inv_m;
        else
            *bad = 1;
    }
}

// dth += (a KPe - b KPg) / d
__global__ void k_tg_dtheta(int n, const double* __restrict__ a, const double* __restrict__ kpe,
                            const double* __restrict__ b, const double* __restrict__ kpg, const double* __restrict__ d,
                            double* __restrict__ dth) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dth[i] += (a[i] * kpe[i] - b[i] * kpg[i]) / d[i];
}

// FP64 copy of an FP32 vector
__global__ void k_tg_to64(int n, const float* __restrict__ in, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (double)in[i];
}

// out = (first ? 0 : out) + s a
__global__ void k_scale_add(int n, const double* __restrict__ a, double s, int first, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (first ? 0.0 : out[i]) + s * a[i];
}

// Adam (Kingma and Ba, 2015) on the flat weights; t counts from 1
__global__ void k_adam(int n, float* __restrict__ w, const double* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = (float)g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mh = mi / (1.f - powf(b1, (float)t)), vh = vi / (1.f - powf(b2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + eps);
}

// smoother diagonal: invd = omega / dl1 (omega NULL: the constant omc / dl1,
// which for omc = 1 is the plain 1 / dl1 rounded as in setup) and its FP32
// copy
__global__ void k_set_damping(int n, const float* __restrict__ om, double omc, const double* __restrict__ dl1,
                              double* __restrict__ invd, float* __restrict__ invd32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = om ? (double)om[i] / dl1[i] : __ddiv_rn(omc, dl1[i]);
    invd[i] = v;
    if (invd32) invd32[i] = __double2float_rn(v);
}

// ------------------------------------------- damping cap (Lanczos estimate)
// isd = 1 / sqrt(d)
__global__ void k_lz_isd(int n, const double* __restrict__ d, double* __restrict__ isd) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) isd[i] = 1.0 / sqrt(d[i]);
}

// xs = isd q (the vector K multiplies in S q = isd K (isd q))
__global__ void k_lz_scale(int n, const double* __restrict__ isd, const double* __restrict__ q,
                           double* __restrict__ xs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) xs[i] = isd[i] * q[i];
}

// Fixed-order sum of one value per thread over the block -> part[blockIdx.x].
__device__ __forceinline__ void lz_block_sum(double t, double* part) {
    __shared__ double sh[kBlock / 32];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < kBlock / 32; k++) u += sh[k];
        part[blockIdx.x] = u;
    }
}

// w = isd y - beta_prev qp (beta_prev NULL: none); block partials of q . w
__global__ void __launch_bounds__(kBlock) k_lz_w(int n, const double* __restrict__ isd, const double* __restrict__ y,
                                                  const double* __restrict__ qp, const double* __restrict__ bprev,
                                                  const double* __restrict__ q, double* __restrict__ w,
                                                  double* __restrict__ part) {
    const double b = bprev ? *bprev : 0.0;
    double t = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double wi = isd[i] * y[i] - b * qp[i];
        w[i] = wi;
        t = fma(q[i], wi, t);
    }
    lz_block_sum(t, part);
}

// w -= alpha q; block partials of w . w
__global__ void __launch_bounds__(kBlock) k_lz_orth(int n, const double* __restrict__ alpha,
                                                     const double* __restrict__ q, double* __restrict__ w,
                                                     double* __restrict__ part) {
    const double a = *alpha;
    double t = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double wi = w[i] - a * q[i];
        w[i] = wi;
        t = fma(wi, wi, t);
    }
    lz_block_sum(t, part);
}

// block partials of x . x
__global__ void __launch_bounds__(kBlock) k_lz_norm2(int n, const double* __restrict__ x, double* __restrict__ part) {
    double t = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) t = fma(x[i], x[i], t);
    lz_block_sum(t, part);
}

// *out = sum of nb block partials (one block, fixed order)
__global__ void __launch_bounds__(kBlock) k_lz_fin(int nb, const double* __restrict__ part, double* __restrict__ out) {
    double t = 0.0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) t += part[k];
    __shared__ double sh[kBlock / 32];
    t = warp_sum(t);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < kBlock / 32; k++) u += sh[k];
        *out = u;
    }
}

// beta = sqrt(*nrm2) (written by block 0, thread 0 to *beta); qp = q;
// q = w / beta (zero once beta = 0: the Krylov space is invariant)
__global__ void k_lz_next(int n, const double* __restrict__ nrm2, double* __restrict__ beta, double* __restrict__ q,
                          double* __restrict__ qp, const double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double b = sqrt(*nrm2);
    if (i == 0) *beta = b;
    if (i < n) {
        qp[i] = q[i];
        q[i] = b > 0.0 ? w[i] / b : 0.0;
    }
}

// q = x / ||x|| (x already holds the start vector; nrm2 = x . x)
__global__ void k_lz_start(int n, const double* __restrict__ nrm2, double* __restrict__ q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = q[i] / sqrt(*nrm2);
}

// Largest eigenvalue theta of the symmetric tridiagonal T (diagonal
// alpha[0..k), off-diagonal beta[0..k-1)), the steps used being those before
// the first zero beta, by Sturm-sequence bisection; its eigenvector s from
// the three-term recurrence (all components share a sign for the largest
// eigenvalue: no cancellation); cap[0] = lam_hat = min(1, theta + beta_k
// |s_k| / ||s||), cap[1] = 2 / lam_hat.  One thread.
__global__ void k_lz_finish(int steps, const double* __restrict__ ab, double* __restrict__ cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double* al = ab;
    const double* be = ab + kLzMax;
    int k = 0;
    while (k < steps) {
        k++;
        if (!(be[k - 1] > 0.0)) break;
    }
    // Gershgorin interval
    double lo = al[0], hi = al[0];
    for (int j = 0; j < k; j++) {
        const double r = (j > 0 ? fabs(be[j - 1]) : 0.0) + (j + 1 < k ? fabs(be[j]) : 0.0);
        lo = fmin(lo, al[j] - r);
        hi = fmax(hi, al[j] + r);
    }
    // eigenvalues below x: sign changes of the LDL^T pivots of T - x I
    auto below = [&](double x) {
        int c = 0;
        double dd = al[0] - x;
        if (dd < 0.0) c++;
        for (int j = 1; j < k; j++) {
            if (dd == 0.0) dd = 1e-300;
            dd = (al[j] - x) - be[j - 1] * be[j - 1] / dd;
            if (dd < 0.0) c++;
        }
        return c;
    };
    for (int it = 0; it < 200; it++) {  // the largest eigenvalue lies in [lo, hi]
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (below(mid) == k) hi = mid;
        else lo = mid;
    }
    const double th = hi;
    double sp = 0.0, sc = 1.0, nrm = 1.0;
    for (int j = 0; j + 1 < k; j++) {
        const double sn = ((th - al[j]) * sc - (j > 0 ? be[j - 1] * sp : 0.0)) / be[j];
        sp = sc;
        sc = sn;
        nrm += sc * sc;
    }
    const double resid = be[k - 1] > 0.0 ? be[k - 1] * fabs(sc) / sqrt(nrm) : 0.0;
    const double lam = fmin(1.0, th + resid);
    cap[0] = lam;
    cap[1] = 2.0 / lam;
}

inline int eblk(int64_t n) { return (int)std::max<int64_t>(1, (n + kBlock - 1) / kBlock); }

}  // namespace

// ------------------------------------------------------------------ host side
// Per-level buffers of the network and of the differentiated V-cycle.
struct MpnnLevel {
    static constexpr int kTape = 8;  // u0 h0 m1 u1 h1 m2 u2 h2, [n][32] each
    static constexpr int kVec = 7;   // FP64 V-cycle vectors
    float* x = nullptr;              // features [n][4]
    float* ap = nullptr;             // normalised off-diagonal values [nnz]
    float* t[kTape] = {};
    float* sg = nullptr;  // sigmoid(z)
    float* omega = nullptr;
    float* sgt = nullptr;    // second head: sigmoid(zt)
    float* theta = nullptr;  // second head: prolongator-smoothing weight
    double* domega = nullptr;
    double* v[kVec] = {};
    double* ab = nullptr;   // Lanczos coefficients: alpha [0, kLzMax), beta [kLzMax, 2 kLzMax), then
                            // kLzParts block partials of the dot products
    double* cap = nullptr;  // [0] lam_hat, [1] omega_max = 2 / lam_hat
    int alloc = 0;     // buffers allocated
    int features = 0;  // features (and the damping cap) enqueued
};

struct MpnnWork {
    MpnnLevel lev[AMG_MAX_LEVELS];
    float* bw[3] = {};       // backward scratch, [n0][32] each
    float* part = nullptr;   // per-block gradient partials
    double* gacc = nullptr;  // FP64 gradient accumulator
    double* gsum = nullptr;  // mean gradient over the hierarchies of a training step
    double *px = nullptr, *py = nullptr, *pky = nullptr;  // probe, y, K y
    double* dots = nullptr;
    double* loss = nullptr;
    int* bad = nullptr;
    int* dst = nullptr;  // [4][kGradSlots] slot -> weight index maps
    float *adam_m = nullptr, *adam_v = nullptr;
    // two-grid loss of the smoothing weights: level-0 and coarse vectors
    static constexpr int kTgFine = 17, kTgCoarse = 4;
    double* tgf[kTgFine] = {};
    double* tgc[kTgCoarse] = {};
    double* tgd = nullptr;  // dense coarse matrix for its inverse
    int tg_alloc = 0;
    double* theta64 = nullptr;  // level-0 theta in FP64 (setup with network weights)
    int have_omega = 0;  // omega of a network evaluation present
    int shared = 0;      // training buffers allocated
    // setup with weights: the finest level's network runs on `side` from the
    // moment its diagonal is known, concurrently with the rest of the setup
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
    int forked = 0;
    std::vector<void*> allocs;
};

namespace {

// Vector slots of a level in the differentiated V-cycle.
enum { V_F = 0, V_X1, V_R, V_X2, V_OUT, V_G, V_T };

int grid_rows(const amg_hierarchy* h, int64_t n) {
    const int64_t cap = (int64_t)std::max(1, h->num_sms) * 8;
    return (int)std::min<int64_t>(std::max<int64_t>(1, (n + kWarpsPerBlock - 1) / kWarpsPerBlock), cap);
}
int grid_grad(int64_t n) {
    return (int)std::min<int64_t>(std::max<int64_t>(1, (n + kWarpsPerBlock - 1) / kWarpsPerBlock), kGradBlocks);
}

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return AMG_OK;
    return e == cudaErrorMemoryAllocation ? AMG_ERR_NOMEM : AMG_ERR_CUDA;
}

int mp_alloc(amg_hierarchy* h, void** p, size_t bytes) {
    cudaError_t e = dev_alloc(p, bytes ? bytes : 16, h->s);
    if (e != cudaSuccess) return status_of(e);
    h->mp->allocs.push_back(*p);
    return AMG_OK;
}

#define MP_ALLOC(ptr, bytes)                                               \
    do {                                                                   \
        int r__ = mp_alloc(h, reinterpret_cast<void**>(&(ptr)), (bytes));  \
        if (r__ != AMG_OK) return r__;                                     \
    } while (0)

#define MP_CK(expr)                           \
    do {                                      \
        int r__ = status_of(expr);            \
        if (r__ != AMG_OK) return r__;        \
    } while (0)

#define MP_TRY(expr)                   \
    do {                               \
        int r__ = (expr);              \
        if (r__ != AMG_OK) return r__; \
    } while (0)

int ensure_work(amg_hierarchy* h) {
    if (h->mp) return AMG_OK;
    h->mp = new (std::nothrow) MpnnWork();
    return h->mp ? AMG_OK : AMG_ERR_NOMEM;
}

// Network buffers of level l, allocated on the library stream (stream-ordered).
int alloc_level(amg_hierarchy* h, int l) {
    MpnnLevel& m = h->mp->lev[l];
    if (m.alloc) return AMG_OK;
    const Level& L = h->lev[l];
    const int64_t n = L.A.n;
    MP_ALLOC(m.x, sizeof(float) * 4 * n);
    MP_ALLOC(m.ap, sizeof(float) * L.A.nnz);
    for (int t = 0; t < MpnnLevel::kTape; t++) MP_ALLOC(m.t[t], sizeof(float) * H * n);
    MP_ALLOC(m.sg, sizeof(float) * n);
    MP_ALLOC(m.omega, sizeof(float) * n);
    MP_ALLOC(m.sgt, sizeof(float) * n);
    MP_ALLOC(m.theta, sizeof(float) * n);
    MP_ALLOC(m.domega, sizeof(double) * n);
    for (int t = 0; t < MpnnLevel::kVec; t++) MP_ALLOC(m.v[t], sizeof(double) * n);
    MP_ALLOC(m.ab, sizeof(double) * (2 * kLzMax + kLzParts));
    MP_ALLOC(m.cap, sizeof(double) * 2);
    m.alloc = 1;
    return AMG_OK;
}

// Damping cap of level l on stream s: Lanczos on D^-1/2 K D^-1/2 from the
// SplitMix64(kLzSeed + l) start vector, min(kLzSteps, n) steps, then
// lam_hat and omega_max into m.cap (see k_lz_finish).  Uses the level's
// V-cycle vectors as workspace.
void cap_level(amg_hierarchy* h, int l, cudaStream_t s) {
    MpnnLevel& m = h->mp->lev[l];
    const Level& L = h->lev[l];
    const int n = L.A.n;
    const int steps = std::min(kLzSteps, n);
    double *q = m.v[V_F], *qp = m.v[V_X1], *wv = m.v[V_R], *isd = m.v[V_X2], *sc = m.v[V_T];
    double *xs = m.v[V_OUT], *y = m.v[V_G];
    double* part = m.ab + 2 * kLzMax;  // block partials
    const int ge = eblk(n), gp = std::min(ge, kLzParts);
    k_lz_isd<<<AMG_GRID(ge), kBlock, 0, s>>>(n, L.dl1, isd);
    k_v_probe<<<AMG_GRID(ge), kBlock, 0, s>>>(n, kLzSeed + (uint64_t)l, 0, q);
    k_lz_norm2<<<AMG_GRID(gp), kBlock, 0, s>>>(n, q, part);
    k_lz_fin<<<AMG_GRID(1), kBlock, 0, s>>>(gp, part, sc);
    k_lz_start<<<AMG_GRID(ge), kBlock, 0, s>>>(n, sc, q);
    cudaMemsetAsync(qp, 0, sizeof(double) * n, s);
    for (int j = 0; j < steps; j++) {
        k_lz_scale<<<AMG_GRID(ge), kBlock, 0, s>>>(n, isd, q, xs);
        launch_spmv(L.A, xs, y, s);
        k_lz_w<<<AMG_GRID(gp), kBlock, 0, s>>>(n, isd, y, qp, j > 0 ? m.ab + kLzMax + j - 1 : nullptr, q, wv,
                                               part);
        k_lz_fin<<<AMG_GRID(1), kBlock, 0, s>>>(gp, part, m.ab + j);
        k_lz_orth<<<AMG_GRID(gp), kBlock, 0, s>>>(n, m.ab + j, q, wv, part);
        k_lz_fin<<<AMG_GRID(1), kBlock, 0, s>>>(gp, part, sc);
        k_lz_next<<<AMG_GRID(ge), kBlock, 0, s>>>(n, sc, m.ab + kLzMax + j, q, qp, wv);
    }
    k_lz_finish<<<AMG_GRID(1), 32, 0, s>>>(steps, m.ab, m.cap);
}

// Node features and edge weights of level l (see the file header), and its
// damping cap, on stream s; the buffers must be allocated and ordered
// before s.
void features_level(amg_hierarchy* h, int l, cudaStream_t s) {
    MpnnLevel& m = h->mp->lev[l];
    if (m.features) return;
    const Level& L = h->lev[l];
    const int64_t n = L.A.n;
    // m.sg holds 1 / sqrt(k_ii) until the first network evaluation
    k_nn_rsqrt_diag<<<AMG_GRID(eblk(n)), kBlock, 0, s>>>((int)n, L.kii, m.sg);
    k_nn_features<<<AMG_GRID(grid_rows(h, n)), kBlock, 0, s>>>((int)n, L.A.rowptr, L.A.col, L.A.val, L.kii, m.sg,
                                                                 m.x, m.ap);
    cap_level(h, l, s);
    m.features = 1;
}

// Allocate the network buffers and compute the features of every level (once
// per hierarchy), and the training buffers.
int prepare(amg_hierarchy* h) {
    MP_TRY(ensure_work(h));
    MpnnWork& w = *h->mp;
    for (int l = 0; l < h->nlev; l++) {
        MP_TRY(alloc_level(h, l));
        features_level(h, l, h->s);
    }
    if (w.shared) return AMG_OK;
    cudaStream_t s = h->s;
    const int64_t n0 = h->lev[0].A.n;
    for (int t = 0; t < 3; t++) MP_ALLOC(w.bw[t], sizeof(float) * H * n0);
    MP_ALLOC(w.part, sizeof(float) * kGradBlocks * kGradSlots);
    MP_ALLOC(w.gacc, sizeof(double) * AMG_MPNN_NPARAM);
    MP_ALLOC(w.gsum, sizeof(double) * AMG_MPNN_NPARAM);
    MP_ALLOC(w.px, sizeof(double) * n0);
    MP_ALLOC(w.py, sizeof(double) * n0);
    MP_ALLOC(w.pky, sizeof(double) * n0);
    MP_ALLOC(w.dots, sizeof(double) * 2);
    MP_ALLOC(w.loss, sizeof(double));
    MP_ALLOC(w.bad, sizeof(int));
    MP_ALLOC(w.dst, sizeof(int) * 4 * kGradSlots);
    MP_ALLOC(w.adam_m, sizeof(float) * AMG_MPNN_NPARAM);
    MP_ALLOC(w.adam_v, sizeof(float) * AMG_MPNN_NPARAM);
    // slot -> flat weight index for the four backward kernels
    std::vector<int> dst(4 * kGradSlots, 0);
    int* d_out = dst.data();
    int* d_l2 = d_out + kGradSlots;
    int* d_l1 = d_l2 + kGradSlots;
    int* d_in = d_l1 + kGradSlots;
    for (int j = 0; j < H; j++) {
        d_out[j] = O_Q + j;
        d_out[H + 1 + j] = O_QT + j;
    }
    d_out[H] = O_C;
    d_out[2 * H + 1] = O_CT;
    for (int k = 0; k < H; k++)
        for (int j = 0; j < H; j++) {
            d_l2[k * H + j] = O_U2 + j * H + k;
            d_l2[H * H + k * H + j] = O_V2 + j * H + k;
            d_l1[k * H + j] = O_U1 + j * H + k;
            d_l1[H * H + k * H + j] = O_V1 + j * H + k;
        }
    for (int j = 0; j < H; j++) {
        d_l2[2 * H * H + j] = O_B2 + j;
        d_l1[2 * H * H + j] = O_B1 + j;
    }
    for (int f = 0; f < 4; f++)
        for (int j = 0; j < H; j++) d_in[f * H + j] = O_W0 + j * 4 + f;
    for (int j = 0; j < H; j++) d_in[4 * H + j] = O_B0 + j;
    MP_CK(cudaMemcpyAsync(w.dst, dst.data(), sizeof(int) * dst.size(), cudaMemcpyHostToDevice, s));
    MP_CK(cudaStreamSynchronize(s));  // dst is a host stack vector
    MP_CK(cudaGetLastError());
    w.shared = 1;
    return AMG_OK;
}

// omega of level l from the network (input layer, two message-passing
// layers, output; FP32 arithmetic, weights rounded to BF16 first when
// bf16 != 0), on stream s.
void forward_level(amg_hierarchy* h, int l, const float* wd, int bf16, cudaStream_t s) {
    const Level& L = h->lev[l];
    MpnnLevel& m = h->mp->lev[l];
    const int n = L.A.n;
    const int g = grid_rows(h, n);
    float *u0 = m.t[0], *h0 = m.t[1], *m1 = m.t[2], *u1 = m.t[3], *h1 = m.t[4], *m2 = m.t[5], *u2 = m.t[6],
          *h2 = m.t[7];
    k_nn_in<<<AMG_GRID(g), kBlock, 0, s>>>(n, wd, bf16, m.x, u0, h0);
    k_nn_spmm<<<AMG_GRID(g), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, m.ap, h0, nullptr, m1);
    k_nn_dense<<<AMG_GRID(g), kBlock, 0, s>>>(n, wd, bf16, 1, m1, h0, u1, h1, nullptr, nullptr, nullptr, nullptr,
                                               nullptr);
    k_nn_spmm<<<AMG_GRID(g), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, m.ap, h1, nullptr, m2);
    k_nn_dense<<<AMG_GRID(g), kBlock, 0, s>>>(n, wd, bf16, 2, m2, h1, u2, h2, m.sg, m.omega, m.cap,
                                               l == 0 ? m.sgt : nullptr, m.theta);
}

// omega of levels [0, nlev - 1); the coarsest level has no smoother.
cudaError_t net_forward(amg_hierarchy* h, const float* wd, int bf16) {
    for (int l = 0; l + 1 < h->nlev; l++) forward_level(h, l, wd, bf16, h->s);
    h->mp->have_omega = 1;
    return cudaGetLastError();
}

// Network backward of level l given its domega (and, on level 0, dtheta of
// the second head when non-NULL); gradients added to gacc.
cudaError_t net_backward(amg_hierarchy* h, const float* wd, int l, const double* dtheta = nullptr) {
    MpnnWork& w = *h->mp;
    cudaStream_t s = h->s;
    Level& L = h->lev[l];
    MpnnLevel& m = w.lev[l];
    const int n = L.A.n;
    const int g = grid_rows(h, n), gg = grid_grad(n);
    const int64_t cnt = (int64_t)n * H;
    float *u0 = m.t[0], *h0 = m.t[1], *m1 = m.t[2], *u1 = m.t[3], *h1 = m.t[4], *m2 = m.t[5], *u2 = m.t[6],
          *h2 = m.t[7];
    float *b0 = w.bw[0], *b1 = w.bw[1], *b2 = w.bw[2];
    const int gs = eblk(kGradSlots);
    k_nn_out_bwd<<<AMG_GRID(gg), kBlock, 0, s>>>(n, wd, m.domega, m.sg, h2, u2, b0, w.part, m.cap, dtheta, m.sgt);
    k_nn_grad_sum<<<AMG_GRID(gs), kBlock, 0, s>>>(gg, w.part, 2 * H + 2, w.dst, w.gacc);
    // layer 2: du2 (b0) -> dm2 (b1), V2^T du2 (b2); dh1 = A' dm2 + V2^T du2 (b0)
    k_nn_dense_bwd<<<AMG_GRID(gg), kBlock, 0, s>>>(n, wd, 2, b0, m2, h1, b1, b2, w.part);
    k_nn_grad_sum<<<AMG_GRID(gs), kBlock, 0, s>>>(gg, w.part, 2 * H * H + H, w.dst + kGradSlots, w.gacc);
    k_nn_spmm<<<AMG_GRID(g), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, m.ap, b1, b2, b0);
    k_nn_relu_mask<<<AMG_GRID(eblk(cnt)), kBlock, 0, s>>>(cnt, u1, b0);
    // layer 1
    k_nn_dense_bwd<<<AMG_GRID(gg), kBlock, 0, s>>>(n, wd, 1, b0, m1, h0, b1, b2, w.part);
    k_nn_grad_sum<<<AMG_GRID(gs), kBlock, 0, s>>>(gg, w.part, 2 * H * H + H, w.dst + 2 * kGradSlots, w.gacc);
    k_nn_spmm<<<AMG_GRID(g), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, m.ap, b1, b2, b0);
    k_nn_relu_mask<<<AMG_GRID(eblk(cnt)), kBlock, 0, s>>>(cnt, u0, b0);
    // input layer
    k_nn_in_bwd<<<AMG_GRID(gg), kBlock, 0, s>>>(n, b0, m.x, w.part);
    k_nn_grad_sum<<<AMG_GRID(gs), kBlock, 0, s>>>(gg, w.part, 5 * H, w.dst + 3 * kGradSlots, w.gacc);
    return cudaGetLastError();
}


// Damped V-cycle from level l on f = v[V_F] into v[V_OUT], keeping the tape
// (f in V_F, r2 in V_R):
//   x1 = Dw f; r1 = f - K x1; e = V_{l+1}(P^T r1); x2 = x1 + P e;
//   r2 = f - K x2; out = x2 + Dw r2,   Dw = diag(omega / d)
void vcycle_fwd(amg_hierarchy* h, int l) {
    MpnnWork& w = *h->mp;
    cudaStream_t s = h->s;
    Level& L = h->lev[l];
    MpnnLevel& m = w.lev[l];
    const int n = L.A.n;
    if (l == h->nlev - 1) {
        k_v_dense<<<AMG_GRID(eblk((int64_t)n * 32)), kBlock, 0, s>>>(n, h->Ainv, m.v[V_F], m.v[V_OUT]);
        return;
    }
    Level& C = h->lev[l + 1];
    MpnnLevel& mc = w.lev[l + 1];
    const int gr = grid_rows(h, n), ge = eblk(n);
    k_v_damp<<<AMG_GRID(ge), kBlock, 0, s>>>(n, nullptr, m.omega, L.dl1, m.v[V_F], m.v[V_X1]);
    k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, L.A.val, m.v[V_X1], m.v[V_F], -1.0, m.v[V_R]);
    k_v_restrict<<<AMG_GRID(eblk(C.A.n)), kBlock, 0, s>>>(C.A.n, L.mem_ptr, L.mem_idx, L.pval, m.v[V_R],
                                                           mc.v[V_F]);
    vcycle_fwd(h, l + 1);
    k_v_prolong<<<AMG_GRID(ge), kBlock, 0, s>>>(n, L.agg, L.pval, mc.v[V_OUT], m.v[V_X1], m.v[V_X2]);
    k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, L.A.val, m.v[V_X2], m.v[V_F], -1.0, m.v[V_R]);
    k_v_damp<<<AMG_GRID(ge), kBlock, 0, s>>>(n, m.v[V_X2], m.omega, L.dl1, m.v[V_R], m.v[V_OUT]);
}

// Reverse of vcycle_fwd: g = d loss / d out in v[V_G]; d loss / d f into
// v[V_OUT]; d loss / d omega added to domega.
void vcycle_bwd(amg_hierarchy* h, int l) {
    MpnnWork& w = *h->mp;
    cudaStream_t s = h->s;
    Level& L = h->lev[l];
    MpnnLevel& m = w.lev[l];
    const int n = L.A.n;
    if (l == h->nlev - 1) {  // A^-1 is symmetric: the adjoint is the same solve
        k_v_dense<<<AMG_GRID(eblk((int64_t)n * 32)), kBlock, 0, s>>>(n, h->Ainv, m.v[V_G], m.v[V_OUT]);
        return;
    }
    Level& C = h->lev[l + 1];
    MpnnLevel& mc = w.lev[l + 1];
    const int gr = grid_rows(h, n), ge = eblk(n);
    double* g = m.v[V_G];
    double* dr2 = m.v[V_T];
    double* dx2 = m.v[V_X2];
    double* dr1 = m.v[V_X1];
    // out = x2 + Dw r2: d omega += g r2 / d; dr2 = Dw g; dx2 = g
    k_v_domega<<<AMG_GRID(ge), kBlock, 0, s>>>(n, g, m.v[V_R], L.dl1, m.domega);
    k_v_damp<<<AMG_GRID(ge), kBlock, 0, s>>>(n, nullptr, m.omega, L.dl1, g, dr2);
    // r2 = f - K x2: df = dr2; dx2 = g - K dr2
    k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, L.A.val, dr2, g, -1.0, dx2);
    // x2 = x1 + P e: dx1 = dx2 (so far); de = P^T dx2
    k_v_restrict<<<AMG_GRID(eblk(C.A.n)), kBlock, 0, s>>>(C.A.n, L.mem_ptr, L.mem_idx, L.pval, dx2, mc.v[V_G]);
    vcycle_bwd(h, l + 1);  // d loss / d fc in mc.v[V_OUT]
    // fc = P^T r1: dr1 = P dfc; r1 = f - K x1: df += dr1, dx1 = dx2 - K dr1
    k_v_prolong<<<AMG_GRID(ge), kBlock, 0, s>>>(n, L.agg, L.pval, mc.v[V_OUT], nullptr, dr1);
    double* dx1 = g;  // g is no longer needed
    k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L.A.rowptr, L.A.col, L.A.val, dr1, dx2, -1.0, dx1);
    // x1 = Dw f: df += Dw dx1; d omega += dx1 f / d
    k_v_domega<<<AMG_GRID(ge), kBlock, 0, s>>>(n, dx1, m.v[V_F], L.dl1, m.domega);
    k_v_df<<<AMG_GRID(ge), kBlock, 0, s>>>(n, dr2, dr1, m.omega, L.dl1, dx1, m.v[V_OUT]);
}

// Loss and gradient for the weights wd: gradient left in gacc, loss in
// loss (device).
int loss_grad_enqueue(amg_hierarchy* h, const float* wd, int nprobe, uint64_t seed) {
    MpnnWork& w = *h->mp;
    cudaStream_t s = h->s;
    Level& L0 = h->lev[0];
    MpnnLevel& m0 = w.lev[0];
    const int n = L0.A.n;
    const int gr = grid_rows(h, n), ge = eblk(n);
    MP_CK(cudaMemsetAsync(w.loss, 0, sizeof(double), s));
    MP_CK(cudaMemsetAsync(w.bad, 0, sizeof(int), s));
    MP_CK(cudaMemsetAsync(w.gacc, 0, sizeof(double) * AMG_MPNN_NPARAM, s));
    for (int l = 0; l < h->nlev; l++)
        MP_CK(cudaMemsetAsync(w.lev[l].domega, 0, sizeof(double) * h->lev[l].A.n, s));
    MP_CK(net_forward(h, wd, 0));
    const double inv_m = 1.0 / nprobe;
    for (int k = 0; k < nprobe; k++) {
        k_v_probe<<<AMG_GRID(ge), kBlock, 0, s>>>(n, seed, k, w.px);
        // f = K x; z = B f; y = x - z
        k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, w.px, nullptr, 1.0,
                                                 m0.v[V_F]);
        vcycle_fwd(h, 0);
        k_v_sub<<<AMG_GRID(ge), kBlock, 0, s>>>(n, w.px, m0.v[V_OUT], w.py);
        k_v_spmv<<<AMG_GRID(gr), kBlock, 0, s>>>(n, L0.A.rowptr, L0.A.col, L0.A.val, w.py, nullptr, 1.0, w.pky);
        k_v_dot2<<<AMG_GRID(1), 1024, 0, s>>>(n, w.py, w.pky, w.px, m0.v[V_F], w.dots);
        k_v_lossgrad<<<AMG_GRID(ge), kBlock, 0, s>>>(n, w.pky, w.dots, inv_m, m0.v[V_G], w.loss, w.bad);
        vcycle_bwd(h, 0);
    }
    for (int l = 0; l + 1 < h->nlev; l++) MP_CK(net_backward(h, wd, l));
    MP_CK(cudaGetLastError());
    return AMG_OK;
}

template <typename T>
int read_host(amg_hierarchy* h, const T* dptr, T* out);

// Loss of the smoothing weights (two-grid, see the file header of the
// oracle's counterpart) for the network's second head on a two-level
// hierarchy whose level-0 prolongator is smoothed; the network's theta is
// installed into the hierarchy (P_bar, the coarse matrix and its inverse
// are rewritten).  Gradient left in gacc (omega held fixed), loss in loss.
int theta_loss_grad_enqueue(amg_hierarchy* h, const float* wd, int nprobe, uint64_t seed) {
    MpnnWork& w = *h->mp;
    cudaStream_t s = h->s;
    Level& L0 = h->lev[0];
    Level& L1 = h->lev[1];
    MpnnLevel& m0 = w.lev[0];
    const int n = L0.A.n, nc = L1.A.n;
    const int gr = grid_rows(h, n), ge = eblk(n), gc = eblk(nc);
    if (!w.tg_alloc) {
        for (int k = 0; k < MpnnWork::kTgFine; k++) MP_ALLOC(w.tgf[k], sizeof(double) * n);
        for (int k = 0; k < MpnnWork::kTgCoarse; k++) MP_ALLOC(w.tgc[k], sizeof(double) * nc);
        MP_ALLOC(w.tgd, sizeof(double) * (size_t)nc * nc);
        w.tg_alloc = 1;
    }
    double *Kx = w.tgf[0], *x1 = w.tgf[1], *Kx1 = w.tgf[2], *x2 = w.tgf[3], *Kx2 = w.tgf[4], *y = w.tgf[5],
           *Ky = w.tgf[6], *ybar = w.tgf[7], *t = w.tgf[8], *x2bar = w.tgf[9], *pbg = w.tgf[10], *a = w.tgf[11],
           *kpe = w.tgf[12], *kpg = w.tgf[13], *dth = w.tgf[14], *th64 = w.tgf[15];
    double *g = w.tgc[0], *e = w.tgc[1], *ebar = w.tgc[2], *gbar = w.tgc[3];
    MP_CK(cudaMemsetAsync(w.loss, 0, sizeof(double), s));
    MP_CK(cudaMemsetAsync(w.bad, 0, sizeof(int), s));
    MP_CK(cudaMemsetAsync(w.gacc, 0, sizeof(double) * AMG_MPNN_NPARAM, s));
    MP_CK(cudaMemsetAsync(m0.domega, 0, sizeof(double) * n, s));
    MP_CK(cudaMemsetAsync(dth, 0, sizeof(double) * n, s));
    forward_level(h, 0, wd, 0, s);
    k_tg_to64<<<AMG_GRID(ge), kBlock, 0, s>>>(n, m0.theta, th64);
    MP_CK(cudaGetLastError());
    MP_TRY(smooth_recompute(h, th64));
    MP_CK(launch_dense_from_csr(L1.A, w.tgd, s));
    MP_CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    MP_CK(launch_dense_spd_inverse(nc, w.tgd, h->Ainv, h->flag, s));
    int notspd = 0;
    MP_TRY(read_host(h, h->flag, &notspd));
    if (notspd) return AMG_ERR_BREAKDOWN;
    const DevCSR& K = L0.A;
    const DevCSR& P = L0.sp;
    const DevCSR& PT = L0.spT;
    const float* om = m0.omega;
    const double inv_m = 1.0 / nprobe;
    auto spmv = [&](const DevCSR& M, const double* xin, const double* base, double sc, double* out) {
        k_v_spmv<<<AMG_GRID(grid_rows(h, M.n)), kBlock, 0, s>>>(M.n, M.rowptr, M.col, M.val, xin, base, sc, out);
    };
    for (int k = 0; k < nprobe; k++) {
        k_v_probe<<<AMG_GRID(ge), kBlock, 0, s>>>(n, seed, k, w.px);
        spmv(K, w.px, nullptr, 1.0, Kx);
        k_tg_damp_sub<<<AMG_GRID(ge), kBlock, 0, s>>>(n, w.px, om, L0.dl1, Kx, x1);
        spmv(K, x1, nullptr, 1.0, Kx1);
        spmv(PT, Kx1, nullptr, 1.0, g);
        k_v_dense<<<AMG_GRID(eblk((int64_t)nc * 32)), kBlock, 0, s>>>(nc, h->Ainv, g, e);
        spmv(P, e, x1, -1.0, x2);
        spmv(K, x2, nullptr, 1.0, Kx2);
        k_tg_damp_sub<<<AMG_GRID(ge), kBlock, 0, s>>>(n, x2, om, L0.dl1, Kx2, y);
        spmv(K, y, nullptr, 1.0, Ky);
        k_v_dot2<<<AMG_GRID(1), 1024, 0, s>>>(n, y, Ky, w.px, Kx, w.dots);
        k_tg_lossgrad<<<AMG_GRID(ge), kBlock, 0, s>>>(n, Ky, w.dots, inv_m, ybar, w.loss, w.bad);
        k_tg_mul<<<AMG_GRID(ge), kBlock, 0, s>>>(n, om, L0.dl1, ybar, t);
        spmv(K, t, ybar, -1.0, x2bar);
        spmv(PT, x2bar, nullptr, -1.0, ebar);
        k_v_dense<<<AMG_GRID(eblk((int64_t)nc * 32)), kBlock, 0, s>>>(nc, h->Ainv, ebar, gbar);
        spmv(P, gbar, nullptr, 1.0, pbg);
        spmv(K, pbg, x2bar, 1.0, a);
        // K P e and K P gbar with the unsmoothed product (pattern of P_bar)
        k_v_spmv<<<AMG_GRID(grid_rows(h, n)), kBlock, 0, s>>>(n, P.rowptr, P.col, L0.kp, e, nullptr, 1.0, kpe);
        k_v_spmv<<<AMG_GRID(grid_rows(h, n)), kBlock, 0, s>>>(n, P.rowptr, P.col, L0.kp, gbar, nullptr, 1.0, kpg);
        k_tg_dtheta<<<AMG_GRID(ge), kBlock, 0, s>>>(n, a, kpe, Kx2, kpg, L0.dl1, dth);
    }
    (void)gc;
    MP_CK(net_backward(h, wd, 0, dth));
    MP_CK(cudaGetLastError());
    return AMG_OK;
}

// Install the damping of the last network evaluation (learned) or the
// constant damping omc (omc = 1: the plain l1-Jacobi diagonal) on every
// level that has a smoother.
cudaError_t set_damping(amg_hierarchy* h, bool learned, double omc = 1.0) {
    cudaStream_t s = h->s;
    for (int l = 0; l + 1 < h->nlev; l++) {
        Level& L = h->lev[l];
        k_set_damping<<<AMG_GRID(eblk(L.A.n)), kBlock, 0, s>>>(L.A.n, learned ? h->mp->lev[l].omega : nullptr, omc,
                                                                L.dl1, L.invd, L.invd32);
    }
    return cudaGetLastError();
}

int sync_status(amg_hierarchy* h) { return status_of(cudaStreamSynchronize(h->s)); }

template <typename T>
int read_host(amg_hierarchy* h, const T* dptr, T* out) {
    MP_CK(cudaMemcpyAsync(h->flag_host, dptr, sizeof(T), cudaMemcpyDeviceToHost, h->s));
    MP_CK(cudaStreamSynchronize(h->s));
    memcpy(out, h->flag_host, sizeof(T));
    return AMG_OK;
}

}  // namespace

// Setup with network weights, first half: once the finest level's diagonal
// is known, its features and network run on a second stream while the setup
// goes on building the coarse levels on the library stream.
int mpnn_setup_fork(amg_hierarchy* h) {
    MP_TRY(ensure_work(h));
    MpnnWork& w = *h->mp;
    MP_TRY(alloc_level(h, 0));
    MP_CK(cudaStreamCreateWithFlags(&w.side, cudaStreamNonBlocking));
    MP_CK(cudaEventCreateWithFlags(&w.ev_fork, cudaEventDisableTiming));
    MP_CK(cudaEventCreateWithFlags(&w.ev_done, cudaEventDisableTiming));
    MP_CK(cudaEventRecord(w.ev_fork, h->s));
    MP_CK(cudaStreamWaitEvent(w.side, w.ev_fork, 0));
    features_level(h, 0, w.side);
    forward_level(h, 0, h->o.mpnn_weights, h->o.mpnn_bf16, w.side);
    MP_CK(cudaEventRecord(w.ev_done, w.side));
    w.forked = 1;
    MP_CK(cudaGetLastError());
    return AMG_OK;
}

// Setup with network weights and a smoothed level 0: the finest level's
// second head gives the smoothing weights; wait for its evaluation on the
// second stream and hand them to the smoothing step in FP64.
int mpnn_setup_theta(amg_hierarchy* h) {
    if (!h->mp || !h->mp->forked) return AMG_OK;
    MpnnWork& w = *h->mp;
    const int n = h->lev[0].A.n;
    MP_CK(cudaStreamWaitEvent(h->s, w.ev_done, 0));
    if (!w.theta64) MP_ALLOC(w.theta64, sizeof(double) * n);
    k_tg_to64<<<AMG_GRID(eblk(n)), kBlock, 0, h->s>>>(n, w.lev[0].theta, w.theta64);
    MP_CK(cudaGetLastError());
    h->theta0 = w.theta64;
    return AMG_OK;
}

// Second half, at the end of the setup: the network on the other levels with
// a smoother, the join with the finest level's evaluation, and the damping
// omega / d installed on every smoothed level (as amg_mpnn_apply does).
int mpnn_setup_join(amg_hierarchy* h) {
    MP_TRY(ensure_work(h));
    MpnnWork& w = *h->mp;
    for (int l = w.forked ? 1 : 0; l + 1 < h->nlev; l++) {
        MP_TRY(alloc_level(h, l));
        features_level(h, l, h->s);
        forward_level(h, l, h->o.mpnn_weights, h->o.mpnn_bf16, h->s);
    }
    if (w.forked) MP_CK(cudaStreamWaitEvent(h->s, w.ev_done, 0));
    w.have_omega = 1;
    MP_CK(set_damping(h, true));
    h->damping_learned = 1;
    return AMG_OK;
}

void mpnn_free(amg_hierarchy* h) {
    if (!h->mp) return;
    MpnnWork& w = *h->mp;
    // a setup that failed between fork and join leaves work on the second
    // stream that reads buffers freed below
    if (w.side) cudaStreamSynchronize(w.side);
    for (void* p : w.allocs) cudaFreeAsync(p, h->s);
    if (w.ev_fork) cudaEventDestroy(w.ev_fork);
    if (w.ev_done) cudaEventDestroy(w.ev_done);
    if (w.side) cudaStreamDestroy(w.side);
    delete h->mp;
    h->mp = nullptr;
}

}  // namespace amg

using namespace amg;

#define MP_RC(expr)                    \
    do {                               \
        int r__ = (expr);              \
        if (r__ != AMG_OK) return r__; \
    } while (0)

extern "C" {

int amg_mpnn_apply(amg_hierarchy* h, const float* w, int32_t bf16_weights) {
    if (!h || bf16_weights < 0 || bf16_weights > 1 || h->o.cheb_degree > 0) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    if (w) {
        MP_RC(prepare(h));
        MP_RC(status_of(net_forward(h, w, bf16_weights)));
    }
    MP_RC(status_of(set_damping(h, w != nullptr)));
    MP_RC(sync_status(h));
    h->damping_learned = w != nullptr;
    return AMG_OK;
}

int amg_mpnn_omega(amg_hierarchy* h, int32_t level, float* omega) {
    if (!h || !omega || level < 0 || level + 1 >= h->nlev) return AMG_ERR_ARG;
    if (!h->mp || !h->mp->have_omega) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    MP_RC(status_of(cudaMemcpyAsync(omega, h->mp->lev[level].omega, sizeof(float) * h->lev[level].A.n,
                                    cudaMemcpyDeviceToDevice, h->s)));
    return sync_status(h);
}

static bool any_smoothed(const amg_hierarchy* h) {
    if (h->o.cheb_degree > 0) return true;  // the network's V-cycle smooths with l1-Jacobi sweeps
    for (int l = 0; l < h->nlev; l++)
        if (h->lev[l].smoothed) return true;
    return false;
}

// A hierarchy for the smoothing weights' two-grid loss: two levels, level 0
// smoothed (with its K P kept).
static bool twogrid_theta(const amg_hierarchy* h) {
    return h->nlev == 2 && h->lev[0].smoothed && h->lev[0].kp && h->nsys == 0 && h->o.cheb_degree == 0;
}

int amg_mpnn_loss_grad(amg_hierarchy* h, const float* w, int32_t nprobe, uint64_t seed, double* loss,
                       double* grad) {
    if (!h || !w || !loss || !grad || nprobe < 1 || h->nlev < 2 || any_smoothed(h)) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    MP_RC(prepare(h));
    MP_RC(loss_grad_enqueue(h, w, nprobe, seed));
    MpnnWork& mw = *h->mp;
    MP_RC(status_of(
        cudaMemcpyAsync(grad, mw.gacc, sizeof(double) * AMG_MPNN_NPARAM, cudaMemcpyDeviceToDevice, h->s)));
    double lh = 0.0;
    int bad = 0;
    MP_RC(read_host(h, mw.loss, &lh));
    MP_RC(read_host(h, mw.bad, &bad));
    *loss = lh;
    if (bad) return AMG_ERR_BREAKDOWN;
    return isfinite(lh) ? AMG_OK : AMG_ERR_NAN;
}

int amg_mpnn_theta_loss_grad(amg_hierarchy* h, const float* w, int32_t nprobe, uint64_t seed, double* loss,
                             double* grad) {
    if (!h || !w || !loss || !grad || nprobe < 1 || !twogrid_theta(h)) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    MP_RC(prepare(h));
    MP_RC(theta_loss_grad_enqueue(h, w, nprobe, seed));
    MpnnWork& mw = *h->mp;
    mw.have_omega = 1;
    MP_RC(status_of(
        cudaMemcpyAsync(grad, mw.gacc, sizeof(double) * AMG_MPNN_NPARAM, cudaMemcpyDeviceToDevice, h->s)));
    double lh = 0.0;
    int bad = 0;
    MP_RC(read_host(h, mw.loss, &lh));
    MP_RC(read_host(h, mw.bad, &bad));
    *loss = lh;
    if (bad) return AMG_ERR_BREAKDOWN;
    return isfinite(lh) ? AMG_OK : AMG_ERR_NAN;
}

int amg_mpnn_theta(amg_hierarchy* h, float* theta) {
    if (!h || !theta || h->nlev < 2) return AMG_ERR_ARG;
    if (!h->mp || !h->mp->have_omega) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    if (h->mp->forked) MP_RC(status_of(cudaStreamWaitEvent(h->s, h->mp->ev_done, 0)));
    MP_RC(status_of(cudaMemcpyAsync(theta, h->mp->lev[0].theta, sizeof(float) * h->lev[0].A.n,
                                    cudaMemcpyDeviceToDevice, h->s)));
    return sync_status(h);
}

int amg_mpnn_adam(amg_hierarchy* h, float* w, const double* grad, float* m, float* v, int32_t t, float lr,
                  float beta1, float beta2, float eps) {
    if (!h || !w || !grad || !m || !v || t < 1 || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) ||
        !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    k_adam<<<AMG_GRID(eblk(AMG_MPNN_NPARAM)), kBlock, 0, h->s>>>(AMG_MPNN_NPARAM, w, grad, m, v, t, lr, beta1, beta2,
                                                                  eps);
    MP_RC(status_of(cudaGetLastError()));
    return sync_status(h);
}

int amg_mpnn_train(amg_hierarchy* const* hs, int32_t count, float* w, int32_t steps, int32_t nprobe, uint64_t seed,
                   float lr, double* loss_hist) {
    if (!hs || count < 1 || count > 64 || !w || steps < 0 || nprobe < 1 || !(lr > 0.f)) return AMG_ERR_ARG;
    for (int k = 0; k < count; k++)
        if (!hs[k] || hs[k]->nlev < 2 || (any_smoothed(hs[k]) && !twogrid_theta(hs[k]))) return AMG_ERR_ARG;
    for (int k = 0; k < count; k++) {
        MP_RC(join_caller_stream(hs[k]));
        MP_RC(prepare(hs[k]));
        MP_RC(sync_status(hs[k]));
    }
    amg_hierarchy* h0 = hs[0];
    MpnnWork& w0 = *h0->mp;
    MP_RC(status_of(cudaMemsetAsync(w0.adam_m, 0, sizeof(float) * AMG_MPNN_NPARAM, h0->s)));
    MP_RC(status_of(cudaMemsetAsync(w0.adam_v, 0, sizeof(float) * AMG_MPNN_NPARAM, h0->s)));
    MP_RC(sync_status(h0));
    for (int t = 0; t < steps; t++) {
        double lsum = 0.0;
        // every hierarchy's loss and gradient with the same weights (its own
        // stream, waited for on the host before the weights change)
        for (int k = 0; k < count; k++) {
            if (twogrid_theta(hs[k]))
                MP_RC(theta_loss_grad_enqueue(hs[k], w, nprobe, seed + (uint64_t)t));
            else
                MP_RC(loss_grad_enqueue(hs[k], w, nprobe, seed + (uint64_t)t));
            int bad = 0;
            double lk = 0.0;
            MP_RC(read_host(hs[k], hs[k]->mp->bad, &bad));
            if (bad) return AMG_ERR_BREAKDOWN;
            MP_RC(read_host(hs[k], hs[k]->mp->loss, &lk));
            if (!isfinite(lk)) return AMG_ERR_NAN;
            lsum += lk;
        }
        // mean gradient (fixed hierarchy order), then one Adam step
        for (int k = 0; k < count; k++)
            k_scale_add<<<AMG_GRID(eblk(AMG_MPNN_NPARAM)), kBlock, 0, h0->s>>>(
                AMG_MPNN_NPARAM, hs[k]->mp->gacc, 1.0 / count, k == 0, w0.gsum);
        k_adam<<<AMG_GRID(eblk(AMG_MPNN_NPARAM)), kBlock, 0, h0->s>>>(AMG_MPNN_NPARAM, w, w0.gsum, w0.adam_m,
                                                                       w0.adam_v, t + 1, lr, 0.9f, 0.999f, 1e-8f);
        MP_RC(status_of(cudaGetLastError()));
        MP_RC(sync_status(h0));
        if (loss_hist) loss_hist[t] = lsum / count;
    }
    return AMG_OK;
}

int amg_set_damping(amg_hierarchy* h, double omega) {
    if (!h || !(omega > 0.0) || !isfinite(omega)) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    MP_RC(status_of(set_damping(h, false, omega)));
    MP_RC(sync_status(h));
    h->damping_learned = 0;
    return AMG_OK;
}

int amg_smoother_bound(amg_hierarchy* h, int32_t level, double* lambda_hat) {
    if (!h || !lambda_hat || level < 0 || level >= h->nlev) return AMG_ERR_ARG;
    MP_RC(join_caller_stream(h));
    MP_RC(ensure_work(h));
    if (h->mp->forked) MP_RC(status_of(cudaStreamWaitEvent(h->s, h->mp->ev_done, 0)));
    MP_RC(alloc_level(h, level));
    features_level(h, level, h->s);
    MP_RC(status_of(cudaGetLastError()));
    MP_RC(read_host(h, h->mp->lev[level].cap, lambda_hat));
    return AMG_OK;
}

int amg_mpnn_select(amg_hierarchy* h, const float* w, double omega_ref, const double* F, double rtol, int32_t itmax,
                    int32_t* used, int32_t* iters_ref, int32_t* iters_learned) {
    if (!h || !w || !F || !(rtol > 0.0) || itmax < 1 || h->nsys > 0 || !(omega_ref > 0.0) || !isfinite(omega_ref))
        return AMG_ERR_ARG;
    const int n = h->lev[0].A.n;
    double* u = nullptr;
    MP_RC(status_of(dev_alloc(reinterpret_cast<void**>(&u), sizeof(double) * n, h->s)));
    struct Release {
        double* p;
        cudaStream_t s;
        ~Release() { cudaFreeAsync(p, s); }
    } release{u, h->s};
    int32_t ir = 0, il = 0;
    MP_RC(amg_set_damping(h, omega_ref));
    MP_RC(status_of(cudaMemsetAsync(u, 0, sizeof(double) * n, h->s)));
    const int rr = amg_pcg_solve(h, F, u, AMG_MEM_DEVICE, rtol, itmax, &ir, nullptr);
    if (rr == AMG_ERR_CUDA || rr == AMG_ERR_NOMEM) return rr;
    // from here on every early return puts the reference damping back
    struct Restore {
        amg_hierarchy* h;
        double om;
        bool keep = false;
        ~Restore() {
            if (!keep) amg_set_damping(h, om);
        }
    } restore{h, omega_ref};
    MP_RC(amg_mpnn_apply(h, w, 1));
    MP_RC(status_of(cudaMemsetAsync(u, 0, sizeof(double) * n, h->s)));
    const int rl = amg_pcg_solve(h, F, u, AMG_MEM_DEVICE, rtol, itmax, &il, nullptr);
    if (rl == AMG_ERR_CUDA || rl == AMG_ERR_NOMEM) return rl;
    // keep the learned damping only if it converged in no more iterations
    restore.keep = rl == AMG_OK && (rr != AMG_OK || il <= ir);
    if (used) *used = restore.keep ? 1 : 0;
    if (iters_ref) *iters_ref = ir;
    if (iters_learned) *iters_learned = il;
    return AMG_OK;
}

}  // extern "C"
