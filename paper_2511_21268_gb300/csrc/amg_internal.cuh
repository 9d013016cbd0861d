// Internal declarations shared by the CUDA translation units of the AMG
// library: hierarchy layout, launch wrappers and small device helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <utility>
#include <stdint.h>

#include <vector>

#include "amg_gb300.h"

namespace amg {

constexpr int kWarp = 32;
constexpr int kBlock = 256;  // threads per block of the row kernels
constexpr int kWarpsPerBlock = kBlock / kWarp;
constexpr int kMaxPasses = 4;
constexpr int kMaxMembers = 1 << kMaxPasses;
constexpr int kMaxPartials = 2048;  // block partial sums of one reduction
constexpr int kMaxRunLen = 9;       // longest run of the run-encoded column format (2p+1, p <= 4)

// Device-side state words of a solve.
struct SolveState {
    int done;      // 1 once converged / failed / itmax
    int iters;     // completed CG iterations
    int status;    // AMG_OK or an error
    int pad;
    double nF;     // ||F||
    double tol;    // rtol * ||F||
    double rho;    // r^T z (PCG) of the current direction
    double alpha;
    double beta;
    double pq;     // p^T K p
    double nr;     // ||r|| of the last iteration
    int itmax;
    int replace_now;  // mixed precision: recompute r = F - K x in FP64 this iteration
    int repl_every;   // mixed precision: replacement period (0 = only at convergence)
    int pad3;
};

// Per-system CG state of a multi-system solve (several right-hand sides or
// a batch of block-diagonal systems).
struct MultiState {
    int done, iters, status, replace_now;
    double nF, tol, rho, alpha, beta, pq, nr;
};

// Workspace of a multi-system solve.  Vectors are interleaved [N][R].
struct MultiWork {
    int R = 0, Rp = 0, S = 0;
    const int32_t* seg = nullptr;     // batch: system of each row (R = 1)
    const int64_t* segoff = nullptr;  // batch: [S + 1] row offsets of the systems
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *F = nullptr;
    float* p32 = nullptr;
    double *pa = nullptr, *pb = nullptr;  // per-element products for the dots
    double* dots = nullptr;               // [S][7]
    double* stage = nullptr;              // column-major staging for copies
    MultiState* st = nullptr;
    MultiState* st_host = nullptr;
    int* active = nullptr;     // systems still iterating
    int* active_host = nullptr;
    int* params = nullptr;     // itmax, replacement period
    void* lf[AMG_MAX_LEVELS] = {};
    void* lx[AMG_MAX_LEVELS] = {};
    void* lt[AMG_MAX_LEVELS] = {};
    cudaGraphExec_t graph = nullptr;
    long long graph_kernels = 0;
    std::vector<void*> allocs;
};

// One matching pass on a matrix with n rows -> nc coarse rows.
struct Pass {
    int n = 0, nc = 0;
    int32_t* mate = nullptr;   // partner, -1 singleton (exported convention)
    int32_t* agg = nullptr;    // fine -> coarse
    double* pval = nullptr;    // prolongator value
    int rounds = 0;
};

struct MpnnWork;  // learned-damping buffers (mpnn.cu)

struct DevCSR {
    int n = 0;
    int64_t nnz = 0;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
};

struct Level {
    DevCSR A;
    double* kii = nullptr;   // diagonal
    double* dl1 = nullptr;   // l1 diagonal
    double* invd = nullptr;  // 1 / dl1
    double* w = nullptr;     // test vector (setup only)
    // map to the next level (absent on the coarsest)
    int npass = 0;
    Pass pass[kMaxPasses];
    int nc = 0;
    int32_t* agg = nullptr;      // composite fine -> coarse
    double* pval = nullptr;      // composite prolongator value
    int32_t* mem_ptr = nullptr;  // [nc+1] members of each next-level row
    int32_t* mem_idx = nullptr;  // [n] fine rows, ascending within a row
    // smoothed prolongator P_bar = (I - diag(theta) D^-1 K) P (when smoothed):
    // sp = P_bar (n x nc, CSR), spT = P_bar^T (nc x n, CSR, rows ascending)
    int smoothed = 0;
    DevCSR sp, spT;
    double* kp = nullptr;  // level 0: values of K P (pattern of sp), which theta rescales into P_bar
    void* cd[2] = {};      // Chebyshev smoother directions (V-cycle precision), when cheb_degree > 0
    // V-cycle vectors (FP64 mode)
    double* f = nullptr;
    double* x = nullptr;
    double* t = nullptr;  // residual / ping-pong buffer
    // mixed precision: FP32 values (BF16 values of the finest level in the
    // V-cycle when requested), FP32 1/dl1 and FP32 V-cycle vectors
    float* val32 = nullptr;
    __nv_bfloat16* val16 = nullptr;
    float* invd32 = nullptr;
    float* f32 = nullptr;
    float* x32 = nullptr;
    float* t32 = nullptr;
    // finest level, staged mixed-precision passes: values with each row's
    // runs interleaved (entry o of run r at rowptr[i] + o R + r)
    __nv_bfloat16* val16t = nullptr;
    float* val32t = nullptr;
    int maxrow = 0;
    // run-encoded columns (level 0, when every row is a sequence of equal
    // runs of consecutive columns): row i has run_ptr[i+1] - run_ptr[i] runs
    // of run_len[i] entries; run r starts at column run_start[r] and at entry
    // rowptr[i] + (r - run_ptr[i]) * run_len[i]
    int32_t* run_ptr = nullptr;
    uint8_t* run_len = nullptr;
    int32_t* run_start = nullptr;
    int64_t nruns = 0;
};

// Sliced copy of one level for the staged passes: slab k (32 consecutive
// rows, a lane per row) has soff[k + 1] - soff[k] run slots; slot r of lane
// t holds lm value slots and the 16-bit offset of its first column in the
// owning block's compacted vector window.
struct SellLevel {
    int on = 0;
    int lm = 0;                    // value slots per run slot (1, 3, 5, 7, 9)
    int nsl = 0;                   // slabs
    int64_t slots = 0;             // run slots in all
    int32_t* soff = nullptr;       // nsl + 1
    uint16_t* rs = nullptr;        // window offset of each (slot, lane)
    float* v32 = nullptr;          // FP32 values, slot-major, lane-minor
    double* v64 = nullptr;         // FP64 values (plain FP64 solve; then v32 = v16 = nullptr)
    __nv_bfloat16* v16 = nullptr;  // BF16 values (BF16 finest values only)
    int vbytes[2] = {};            // value area per buffer: [0] BF16, [1] FP32
    int rbytes = 0;                // offset area per buffer
    int xbytes = 0;                // largest compacted window
    int nbuf[2] = {};              // ring buffers: [0] BF16, [1] FP32 values
    void* wint = nullptr;          // int4 per window interval (kMaxWinIntervals per block)
    int* wcnt = nullptr;           // window intervals of each block
    int* wbytes = nullptr;         // compacted window bytes of each block
    int G = 0;                     // blocks of the launch (1, 2, 4 or 8 per SM: the windows must fit)
};

}  // namespace amg

struct amg_hierarchy {
    amg_opts o;
    cudaStream_t s = nullptr;
    int nlev = 0;
    amg::Level lev[AMG_MAX_LEVELS];
    int ndense = 0;
    double* Ainv = nullptr;  // dense inverse of the coarsest matrix (row-major)
    double* ccg = nullptr;   // coarse CG work vectors (5 x coarsest rows), coarse_solver = 1
    // CG workspace (level 0)
    double *x = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *F = nullptr;
    float* p32 = nullptr;  // FP32 copy of p for the mixed-precision outer SpMV
    int mixed = 0;         // precision != AMG_FP64
    double* partials = nullptr;  // 7 slots of npart doubles
    int npart = 0;
    double rtol = 0.0;
    int itmax = 0;
    cudaStream_t us = nullptr;   // caller's stream
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evs = nullptr;
    std::vector<void*> allocs;   // device allocations owned by the hierarchy
    amg::SolveState* st = nullptr;
    amg::SolveState* st_host = nullptr;  // pinned mirror
    int* flag = nullptr;                 // device scratch flag / counter
    int* flag_host = nullptr;            // pinned mirror
    double* hist = nullptr;              // residual history (device)
    int hist_cap = 0;
    amg_info info;
    int num_sms = 0;
    int coop = 0;  // the device runs cooperative launches (all matching rounds of a pass in one)
    bool own_stream = false;
    // captured iteration graph
    cudaGraphExec_t graph = nullptr;
    int graph_iters = 0;
    long long graph_kernels = 0;  // kernels per graph launch
    // opt-in timing of the three fine-level matrix-pass kernels of each CG
    // iteration (q = K p, down-sweep residual, up-sweep) with event-record
    // nodes in the iteration graph
    int prof = 0;
    cudaEvent_t prof_ev[16][3][2] = {};
    double prof_ms[3] = {0, 0, 0};
    long long prof_cnt[3] = {0, 0, 0};
    int prof_slot = -1;  // iteration slot being captured, -1 = not capturing
    // setup phase timing: an event at every phase change
    cudaEvent_t ph_ev[512] = {};
    int ph_id[512] = {};
    int ph_n = 0;
    int* round_active = nullptr;  // active count after each matching round (device)
    // bulk-copy streamed finest-level passes of the mixed-precision solve
    int stream = 0;             // in use: 1 = lane-per-run slabs, 2 = sliced (lane-per-row) slabs
    int stream_blocks = 0;      // persistent grid (one block per SM)
    int stream_rpw = 0;         // rows per warp of a slab (slab = 8 warps x rpw rows)
    int stream_xbytes = 0;      // shared-memory bytes of the vector window
    int stream_vbytes[2] = {};  // value buffer bytes: [0] BF16 values, [1] FP32 values
    int stream_rbytes[2] = {};  // run-start buffer bytes
    int stream_nbuf[2] = {};    // buffers in the copy ring
    int* stream_win = nullptr;  // int2 per block: first and last column of its rows
    // sliced copies (32-row slabs, lane per row): [0] the finest level (when
    // stream == 2, FP32 and BF16 values; or when sell64, FP64 values), [1]
    // level 1 in mixed precision (plain CSR, each entry a run of length 1)
    amg::SellLevel sell[2];
    int sell64 = 0;        // plain FP64 solve: the finest-level passes run on sell[0] (FP64 values)
    double tune_ms = 0.0;  // host time of the setup's autotuning (0 when skipped or cached)
    int galerkin_spgemm_passes = 0;  // pass Galerkin products done by the SpGEMM path (too-wide rows)
    int sell64_warps = 0;  // warps per block of those passes
    // multi-system solves
    amg::MultiWork* mw = nullptr;
    // learned smoother damping: network buffers, and whether the smoother
    // diagonals currently hold omega / d instead of 1 / d
    amg::MpnnWork* mp = nullptr;
    int damping_learned = 0;
    // level-0 smoothing weights from the network of a setup given weights
    // (device FP64, owned by the network buffers), NULL otherwise
    const double* theta0 = nullptr;
    // block-diagonal batch (amg_setup_batch): systems and their row offsets
    int nsys = 0;
    std::vector<int64_t> sys_off;    // host copy [nsys + 1]
    int32_t* sys_id = nullptr;       // device [N]
    int64_t* sys_off_dev = nullptr;  // device [nsys + 1]
};

namespace amg {

// ----------------------------------------------------------------- launch wrappers
// setup_kernels.cu
cudaError_t launch_validate_csr(const DevCSR& A, int* flag, cudaStream_t s);
cudaError_t launch_l1diag(const DevCSR& A, double* kii, double* dl1, double* invd, int* flag, cudaStream_t s);
cudaError_t launch_diag(const DevCSR& A, double* kii, cudaStream_t s);
cudaError_t launch_testvec_init(int n, int kind, uint64_t seed, double* w, cudaStream_t s);
cudaError_t launch_testvec_sweep(const DevCSR& A, const double* dl1, const double* w, double* wout, cudaStream_t s);
cudaError_t launch_edge_keys(const DevCSR& A, const double* kii, const double* w, uint64_t* key, int* flag,
                             cudaStream_t s);
cudaError_t launch_match_init(int n, int32_t* state, cudaStream_t s);
cudaError_t launch_match_rounds(const DevCSR& A, const uint64_t* key, int32_t* state, int32_t* cand, int* active,
                                int32_t* lists, int first_round, int count, cudaStream_t s);
cudaError_t launch_match_rounds_coop(const DevCSR& A, const uint64_t* key, int32_t* state, int32_t* cand, int* active,
                                     int32_t* lists, int max_rounds, int* rounds_out, int num_sms, cudaStream_t s);
cudaError_t launch_match_finish(int n, const int32_t* state, int32_t* mate, int32_t* leader, cudaStream_t s);
cudaError_t launch_aggregate(int n, const int32_t* mate, const int32_t* cidx, const double* w, int32_t* agg,
                             double* pval, int32_t* mem0, int32_t* mem1, double* wc, cudaStream_t s);
cudaError_t launch_exclusive_scan(const int32_t* in, int32_t* out, int n, int32_t* total, int32_t* scratch,
                                  cudaStream_t s);
size_t scan_scratch_ints(int n);
cudaError_t launch_galerkin_count(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                  int nc, int cap, int64_t* rowcnt, cudaStream_t s);
cudaError_t launch_galerkin_fill(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mem0,
                                 const int32_t* mem1, int cap, DevCSR& C, cudaStream_t s);
cudaError_t launch_galerkin_mirror(DevCSR& C, int* flag, cudaStream_t s);
cudaError_t launch_galerkin_count_bitmap(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                         int nc, int cap, int words, int64_t* rowcnt, int* flag, cudaStream_t s);
cudaError_t launch_galerkin_fill_bitmap(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mem0,
                                        const int32_t* mem1, int cap, int words, DevCSR& C, int* flag, cudaStream_t s);
// Warp-per-row Galerkin kernels (candidate counts up to kGalWarpCand):
// counting (row lengths, and stats[0] = widest coarse-column span, stats[1] =
// longest coarse row) and values (sym: the level matrix is symmetric in every
// bit, so the lower triangle is computed in place; else the mirror fills it).
constexpr int kGalWarpCand = 4096;
size_t galerkin_warp_fill_smem(int cmax, int words, int umax);  // bytes per block
cudaError_t launch_galerkin_warp_count(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1,
                                       int nc, int cmax, int64_t* rowcnt, int* stats, int* flag, cudaStream_t s);
cudaError_t launch_galerkin_warp_fill(const DevCSR& A, const int32_t* agg, const double* pval, const int32_t* mate,
                                      const int32_t* mem0, const int32_t* mem1, int cmax, int words, int umax, int sym,
                                      DevCSR& C, int* flag, cudaStream_t s);
cudaError_t launch_row_span(const DevCSR& A, const int32_t* agg, const int32_t* mem0, const int32_t* mem1, int nc,
                            int* maxspan, cudaStream_t s);
cudaError_t launch_scan64(const int64_t* in, int64_t* out, int n, int64_t* scratch, cudaStream_t s);
size_t scan64_scratch(int n);
cudaError_t launch_row_stats(const DevCSR& A, const int32_t* mem0, const int32_t* mem1, int nc, int* maxcand,
                             cudaStream_t s, const int* nc_dev = nullptr);
cudaError_t launch_compose(int n, int npass, const Pass* passes, int32_t* agg, double* pval, cudaStream_t s);
cudaError_t launch_member_count(int n, const int32_t* agg, int nc, int32_t* cnt, cudaStream_t s);
cudaError_t launch_member_fill(int n, const int32_t* agg, const int32_t* mem_ptr, int nc, int32_t* mem_idx,
                               int* cursor, cudaStream_t s);
cudaError_t launch_dense_from_csr(const DevCSR& A, double* D, cudaStream_t s);
cudaError_t launch_dense_spd_inverse(int n, double* D, double* Ainv, int* flag, cudaStream_t s);
cudaError_t launch_to_f32(const double* in, float* out, int64_t n, cudaStream_t s);
cudaError_t launch_to_bf16(const double* in, __nv_bfloat16* out, int64_t n, cudaStream_t s);

// solve_kernels.cu
cudaError_t launch_spmv(const DevCSR& A, const double* x, double* y, cudaStream_t s);
cudaError_t enqueue_vcycle(amg_hierarchy* h, cudaStream_t s);
cudaError_t enqueue_vcycle_standalone(amg_hierarchy* h, cudaStream_t s);
cudaError_t enqueue_pcg_start(amg_hierarchy* h, cudaStream_t s);
cudaError_t enqueue_pcg_iteration(amg_hierarchy* h, cudaStream_t s);
cudaError_t launch_final_residual(amg_hierarchy* h, cudaStream_t s);
cudaError_t launch_rowgroup_pq(amg_hierarchy* h, cudaStream_t s);
double* final_residual_slot(amg_hierarchy* h);
// multi_solve.cu
cudaError_t enqueue_multi_start(amg_hierarchy* h, cudaStream_t s);
cudaError_t enqueue_multi_iteration(amg_hierarchy* h, cudaStream_t s);
cudaError_t enqueue_multi_final(amg_hierarchy* h, cudaStream_t s);
int multi_dot_stride();
// mpnn.cu
void mpnn_free(amg_hierarchy* h);
int mpnn_setup_fork(amg_hierarchy* h);
int mpnn_setup_join(amg_hierarchy* h);
int mpnn_setup_theta(amg_hierarchy* h);
// stream_kernels.cu
int stream_prepare(amg_hierarchy* h, int* scratch2);
cudaError_t launch_stream_resid(amg_hierarchy* h, const double* f, const float* x, float* rbuf, cudaStream_t s);
cudaError_t launch_stream_up0(amg_hierarchy* h, const double* r, const float* x, const float* invd, double* z,
                              const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s);
cudaError_t launch_stream_spmv_pq(amg_hierarchy* h, const float* p32, const double* p, const double* r, double* q,
                                  double* part_pq, double* part_pr, int flexible, cudaStream_t s);
// sell_kernels.cu
int sell_prepare(amg_hierarchy* h, int* scratch, int optin, int* used);
int sell_prepare_level1(amg_hierarchy* h, int* scratch);
cudaError_t sell_resid1(amg_hierarchy* h, const float* f, const float* x, float* rbuf, cudaStream_t s);
cudaError_t sell_upy1(amg_hierarchy* h, const float* f, const float* x, const float* invd, float* y, cudaStream_t s);
int sell64_prepare(amg_hierarchy* h, int* scratch);
void sell64_warp_range(int* lo, int* hi);
cudaError_t sell64_spmv_pq(amg_hierarchy* h, const double* p, const double* r, double* q, double* part_pq,
                           double* part_pr, int flexible, cudaStream_t s);
cudaError_t sell64_resid(amg_hierarchy* h, const double* f, const double* x, double* rbuf, cudaStream_t s);
cudaError_t sell64_up0(amg_hierarchy* h, const double* r, const double* x, const double* invd, double* z,
                       const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s);
// Chebyshev steps of the finest level on the sliced FP64 copy (see
// vcycle_cheb in solve_kernels.cu).
cudaError_t sell64_cheb_step(amg_hierarchy* h, const double* dprev, const double* rprev, double* r,
                             const double* invd, double a, double b, double* dnew, double* x, cudaStream_t s);
cudaError_t sell64_cheb_resid(amg_hierarchy* h, const double* dprev, const double* rprev, double* r, double* x,
                              cudaStream_t s);
cudaError_t sell64_cheb_post0(amg_hierarchy* h, const double* x, const double* f, const double* invd, double c0,
                              double* r, double* d, cudaStream_t s);
cudaError_t sell_resid(amg_hierarchy* h, const double* f, const float* x, float* rbuf, cudaStream_t s);
cudaError_t sell_up0(amg_hierarchy* h, const double* r, const float* x, const float* invd, double* z,
                     const double* q, double* part_rz, double* part_zq, int flexible, cudaStream_t s);
cudaError_t sell_spmv_pq(amg_hierarchy* h, const float* p32, const double* p, const double* r, double* q,
                         double* part_pq, double* part_pr, int flexible, cudaStream_t s);
// smooth_kernels.cu: smoothed prolongator and its Galerkin product for level
// l (member lists and l1 diagonal present); the coarse matrix goes to Kc
int smooth_level(amg_hierarchy* h, int l, DevCSR& Kc);
// smooth_kernels.cu: level 0's P_bar for new per-row weights theta (device,
// FP64) and the coarse matrix P_bar^T K P_bar rewritten in place (same pattern)
int smooth_recompute(amg_hierarchy* h, const double* theta);
// smooth_kernels.cu: a matching pass's Galerkin product P^T A P by the
// row-merge SpGEMMs (rows too wide for the bitmap and sorting kernels); C's
// arrays are recorded in h->allocs
int galerkin_pass_spgemm(amg_hierarchy* h, const DevCSR& A, const int32_t* agg, const double* pval,
                         const int32_t* mem0, const int32_t* mem1, int nc, DevCSR& C);
template <typename A>
void sp_restrict(const Level& F, const Level& C, const A* r, A* fc, A* xc, const A* invdc, const SolveState* st,
                 cudaStream_t s);
template <typename A>
void sp_prolong(const Level& F, const A* y, A* xf, const SolveState* st, cudaStream_t s);
template <typename A>
void sp_coarse(int n, const double* Ainv, const A* f, A* e, const SolveState* st, cudaStream_t s);
// amg_api.cu: order the library stream after the caller's stream
int join_caller_stream(amg_hierarchy* h);
// amg_api.cu: stream-ordered device allocation from the library's memory pool
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s);
// Records a CUDA error for amg_last_cuda_error; AMG_ERR_NOMEM for an
// allocation failure, else AMG_ERR_CUDA.
int report_cuda(cudaError_t e, const char* what);
cudaError_t launch_interleave(int n, int R, int64_t ld, const double* src, double* dst, cudaStream_t s);
cudaError_t launch_deinterleave(int n, int R, int64_t ld, const double* src, double* dst, cudaStream_t s);
// batch assembly (setup_kernels.cu)
cudaError_t launch_shift_block(int n, int64_t nnz, const int64_t* rp_in, int64_t row_off, int64_t nnz_off,
                               int64_t* rp_out, int32_t* col, int* flag, cudaStream_t s);
cudaError_t launch_fill_sys_id(int nsys, const int64_t* off, int32_t* id, cudaStream_t s);
cudaError_t launch_run_rows(const DevCSR& A, int32_t* runcnt, uint8_t* runlen, int* flag, cudaStream_t s);
cudaError_t launch_run_fill(const DevCSR& A, const int32_t* run_ptr, const uint8_t* runlen, int32_t* run_start,
                            cudaStream_t s);
int rows_per_warp(int n, int num_sms);
int row_blocks(int n, int rpw);
int vec_blocks(int n, int num_sms);
size_t partial_slot_size(int n0, int num_sms);  // >= num_sms + 2
size_t partial_slot_count();

// ----------------------------------------------------------------- device helpers
#ifdef __CUDACC__
// The bits of an FP64 value through an opaque move, so that the compiler
// keeps integer operations on them integer: masking the sign bit of a
// reinterpreted double would otherwise become an FP64 absolute value, and
// some tests of the bits FP64 comparisons, on GB300's narrow FP64 pipe.
__device__ __forceinline__ long long dbits(double x) {
    long long r;
    asm("mov.b64 %0, %1;" : "=l"(r) : "d"(x));
    return r;
}

// Monotone map of a finite double to an unsigned key (larger value ->
// larger key); -0 is folded onto +0.  Key 0 is reserved for "no edge".
__device__ __forceinline__ uint64_t order_key(double c) {
    uint64_t b = (uint64_t)dbits(c);
    if ((b << 1) == 0) b = 0;  // -0 -> +0, decided on the bits
    return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

// Correctly rounded a / b (IEEE binary64, round to nearest even): the same
// bits as __ddiv_rn(a, b), in fewer FP64 operations for operands of
// moderate magnitude (both normal, binary exponents in [-500, 500]); other
// operands go to __ddiv_rn.
//   1. y0 ~ 1/b: the FP32 reciprocal (SFU approximation) of b's leading 23
//      mantissa bits, scaled by integer exponent arithmetic (relative error
//      about 2^-22).
//   2. One Newton-Raphson step, y1 = y0 + y0 (1 - b y0) (error below 2^-44).
//   3. q0 = a y1 and Markstein's correction q = q0 + (a - b q0) y1, whose
//      value before rounding lies within about 2^-89 (relative) of a / b.
//   4. Acceptance: the FMA residual r = a - b q is exact whenever q is a
//      faithful quotient (Boldo and Daumas, "Representable correcting terms
//      for possibly underflowing floating point operations", 2003), and then
//      |r| < |b| h(q), h(q) the half-gap from q to its nearer neighbour
//      (half an ulp; a quarter at a power of two), says a / b is closer to q
//      than to either neighbour, i.e. q = RN(a / b).  When q is not faithful
//      |r| is at least |b| times a full gap, so the test fails; it also fails
//      on exact ties.  A failed test falls back to __ddiv_rn.
// Six FP64 operations on the fast path; the tests run on integer bits.
// div_rn_fast returns false (and leaves *q unset) where the fast path
// declines.
__device__ __forceinline__ bool div_rn_fast(double a, double b, double* q_out) {
    const long long ab = dbits(a), bb = dbits(b);
    const int ea = (int)((ab >> 52) & 0x7ff) - 1023, eb = (int)((bb >> 52) & 0x7ff) - 1023;
    if (ea < -500 || ea > 500 || eb < -500 || eb > 500) return false;
    // 1. reciprocal estimate: f = 1.m (FP32, top 23 mantissa bits), 1/f in (1/2, 1]
    const float f = __int_as_float(0x3f800000 | (int)((bb >> 29) & 0x7fffff));
    float rcp;  // PTX rcp.approx.ftz.f32: the SFU reciprocal, about 1 ulp of FP32
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rcp) : "f"(f));
    const int rf = __float_as_int(rcp);
    const int erf = ((rf >> 23) & 0xff) - 127;  // -1 or 0
    const long long y0b = (bb & (long long)0x8000000000000000ULL) | ((long long)(erf - eb + 1023) << 52) |
                          ((long long)(rf & 0x7fffff) << 29);
    const double y0 = __longlong_as_double(y0b);
    // -b by its sign bit (an integer operation)
    const double nb = __longlong_as_double(bb ^ (long long)0x8000000000000000ULL);
    // 2. Newton-Raphson step
    const double y1 = __fma_rn(y0, __fma_rn(nb, y0, 1.0), y0);
    // 3. quotient and correction
    const double q0 = __dmul_rn(a, y1);
    const double q = __fma_rn(__fma_rn(nb, q0, a), y1, q0);
    // 4. exact residual and acceptance test on the bits
    const double r = __fma_rn(nb, q, a);
    const long long qb = dbits(q) & 0x7fffffffffffffffLL;
    const int eq = (int)(qb >> 52) - 1023;
    const int k = ((qb & 0xfffffffffffffLL) == 0 ? eq - 54 : eq - 53);  // log2 of h(q)
    const long long tb = (bb & 0x7fffffffffffffffLL) + ((long long)k << 52);  // |b| h(q), exact
    const long long rb = dbits(r) & 0x7fffffffffffffffLL;
    if (eq < -1010 || eq > 1010 || rb >= tb) return false;
    *q_out = q;
    return true;
}

// The fallback is a call, so that none of the compiler's division is
// scheduled speculatively ahead of the fast path's test.
static __device__ __noinline__ double div_rn_slow(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ double div_rn(double a, double b) {
    double q;
    return div_rn_fast(a, b, &q) ? q : div_rn_slow(a, b);
}

// SplitMix64 (Steele, Lea, Flood 2014): draw k of the stream seeded `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
#endif

}  // namespace amg

// Every kernel launch goes through AMG_GRID(grid) so the library can report
// how many kernels it launched (amg_kernel_launches).
namespace amg {
long long note_launch();
}
#define AMG_GRID(g) (amg::note_launch(), (g))

namespace amg {
// Programmatic dependent launch.  A kernel launched with launch_pdl starts
// with pdl_entry(), which waits until the previous kernel of the stream has
// completed and its memory is visible, before any other instruction touches
// memory; the launch itself (block scheduling) overlaps the predecessor's
// completion.  Kernels do not trigger their dependents early: blocks of
// later kernels parked on the SMs slowed the solve (the staged passes need
// a whole SM's shared memory).  Launched without the attribute the wait
// does nothing.
__device__ __forceinline__ void pdl_entry() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch `kernel` (whose first statement is pdl_entry()) allowing
// programmatic stream serialization with the previous kernel.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    note_launch();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
}  // namespace amg

#define AMG_TRY(expr)                          \
    do {                                       \
        cudaError_t e__ = (expr);              \
        if (e__ != cudaSuccess) return e__;    \
    } while (0)
