// C ABI of the AMG-PCG library: hierarchy construction (setup driver),
// solve loop and data export.  See include/amg_gb300.h for the contract.
//
// Setup (arXiv 2511.21268 Sec. 3.1, 3.2), per level l:
//   l1 diagonal -> (level 0) test vector -> m matching passes, each:
//   edge keys -> locally dominant matching rounds -> aggregates and
//   prolongator values -> Galerkin product of the pass -> restricted test
//   vector; then the composite map P = P_1 ... P_m and its member lists.
// Coarsening stops at coarse_max rows, on stagnation or at max_levels; the
// coarsest matrix is inverted densely.
//
// Solve: the CG start phase is launched directly, the iterations run as a
// captured CUDA graph of kGraphIters iterations whose kernels turn into
// no-ops once the device-side state says "done"; the host reads the state
// once per graph launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "amg_internal.cuh"

using namespace amg;

namespace amg {
static std::atomic<long long> g_launches{0};
long long note_launch() { return ++g_launches; }
}  // namespace amg

namespace {

constexpr int kGraphIters = 8;
constexpr int kMaxGalerkinCap = 16384;  // candidate entries per Galerkin row (shared memory)
constexpr double kBitmapSmem = 200.0 * 1024;  // shared memory budget of the bitmap Galerkin kernels
constexpr double kWarpGalerkinSmem = 160.0 * 1024;  // and of the warp-per-row values kernel (per block)
constexpr int kHistCap = 1 << 16;
// Matrix column/value arrays get kPad trailing entries: the FP32/BF16 matrix
// passes load groups of four entries from 4-aligned positions.
constexpr size_t kPad = 8;

thread_local char g_cuda_err[512] = "";

}  // namespace

namespace amg {
// Device memory of the library comes from its own stream-ordered memory pool
// (one per device) that keeps freed memory reserved, so that building and
// freeing hierarchies in a loop reuses it instead of returning it to the
// driver at every synchronisation.  The caller's default pool is untouched.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, s);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> g(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pools[dev], &props);
            if (e != cudaSuccess) {
                pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}
}  // namespace amg

namespace {

// Process-wide pool of the small per-hierarchy resources whose creation is
// slow (page-locked host blocks, CUDA events), so that building and freeing
// hierarchies in a loop does not pay for them every time.  Keyed by device.
struct ResourcePool {
    std::mutex mu;
    std::vector<std::pair<int, void*>> pinned;              // (device, 512-byte block)
    std::vector<std::pair<int, cudaEvent_t>> timed, plain;  // (device, event)
};
ResourcePool& pool() {
    static ResourcePool* p = new ResourcePool();  // never destroyed: outlives static destructors
    return *p;
}
constexpr size_t kPinnedBlock = 512;

cudaError_t pinned_get(void** out) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> g(pool().mu);
        auto& v = pool().pinned;
        for (size_t i = 0; i < v.size(); i++)
            if (v[i].first == dev) {
                *out = v[i].second;
                v.erase(v.begin() + i);
                return cudaSuccess;
            }
    }
    return cudaMallocHost(out, kPinnedBlock);
}
void pinned_put(void* p) {
    if (!p) return;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(pool().mu);
    pool().pinned.emplace_back(dev, p);
}
cudaError_t event_get(cudaEvent_t* e, bool timing) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> g(pool().mu);
        auto& v = timing ? pool().timed : pool().plain;
        for (size_t i = v.size(); i-- > 0;)
            if (v[i].first == dev) {
                *e = v[i].second;
                v.erase(v.begin() + i);
                return cudaSuccess;
            }
    }
    return timing ? cudaEventCreate(e) : cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}
void event_put(cudaEvent_t e, bool timing) {
    if (!e) return;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(pool().mu);
    (timing ? pool().timed : pool().plain).emplace_back(dev, e);
}

int cuda_fail(cudaError_t e, const char* what) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? AMG_ERR_NOMEM : AMG_ERR_CUDA;
}

#define CK(expr)                                          \
    do {                                                  \
        cudaError_t e__ = (expr);                         \
        if (e__ != cudaSuccess) return cuda_fail(e__, #expr); \
    } while (0)

#define RC(expr)                     \
    do {                             \
        int r__ = (expr);            \
        if (r__ != AMG_OK) return r__; \
    } while (0)

constexpr int kRoundBatch = 16;  // matching rounds between host reads (later rounds are no-ops)
constexpr int kMaxSystems = 1024;  // systems of one batch (one scalar thread each)

// Mark the start of setup phase `id` (see amg_info.setup_phase_ms).
void phase(amg_hierarchy* h, int id) {
    if (h->ph_n >= 512) return;
    if (!h->ph_ev[h->ph_n] && event_get(&h->ph_ev[h->ph_n], true) != cudaSuccess) return;
    cudaEventRecord(h->ph_ev[h->ph_n], h->s);
    h->ph_id[h->ph_n++] = id;
}

template <typename T>
int dalloc(amg_hierarchy* h, T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = dev_alloc(&q, sizeof(T) * count, h->s);
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    h->allocs.push_back(q);
    *p = (T*)q;
    return AMG_OK;
}

// temporary device buffer freed at scope exit (stream ordered)
struct Tmp {
    cudaStream_t s;
    void* p = nullptr;
    explicit Tmp(cudaStream_t st) : s(st) {}
    ~Tmp() {
        if (p) cudaFreeAsync(p, s);
    }
    template <typename T>
    int get(T** out, size_t count) {
        if (count == 0) count = 1;
        cudaError_t e = dev_alloc(&p, sizeof(T) * count, s);
        if (e != cudaSuccess) return cuda_fail(e, "device allocation");
        *out = (T*)p;
        return AMG_OK;
    }
};

void forget(amg_hierarchy* h, void* p) {
    auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
    if (it != h->allocs.end()) {
        cudaFreeAsync(p, h->s);
        h->allocs.erase(it);
    }
}

int read_flag(amg_hierarchy* h, int* value) {
    CK(cudaMemcpyAsync(h->flag_host, h->flag, sizeof(int), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    *value = *h->flag_host;
    return AMG_OK;
}

template <typename T>
int read_scalar(amg_hierarchy* h, const T* dptr, T* value) {
    CK(cudaMemcpyAsync(h->flag_host, dptr, sizeof(T), cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    memcpy(value, h->flag_host, sizeof(T));
    return AMG_OK;
}

int pow2ceil(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Galerkin product of one matching pass with the warp-per-row kernels: the
// counting kernel gives the row lengths and the widest span and row, which
// size the values kernel (the block kernels take rows too wide for it).
int galerkin_warp(amg_hierarchy* h, const DevCSR& A, const Pass& P, const int32_t* mem0, const int32_t* mem1, int nc,
                  int maxcand, int bit_symmetric, DevCSR& C) {
    cudaStream_t s = h->s;
    C.n = nc;
    RC(dalloc(h, &C.rowptr, (size_t)nc + 1));
    int64_t *rowcnt, *scr64;
    Tmp trc(s), ts64(s);
    RC(trc.get(&rowcnt, nc));
    RC(ts64.get(&scr64, scan64_scratch(nc) + 1));
    // Galerkin errors accumulate in flag[3], read once after the last level;
    // flag[1], flag[2]: widest span, longest coarse row (zeroed by the caller)
    CK(launch_galerkin_warp_count(A, P.agg, mem0, mem1, nc, maxcand, rowcnt, h->flag + 1, h->flag + 3, s));
    CK(launch_scan64(rowcnt, C.rowptr, nc, scr64, s));
    CK(cudaMemcpyAsync(h->flag_host, C.rowptr + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->flag_host + 2, h->flag + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int64_t nnzc = 0;
    memcpy(&nnzc, h->flag_host, sizeof(int64_t));
    const int maxspan = h->flag_host[2], maxu = h->flag_host[3];
    C.nnz = nnzc;
    RC(dalloc(h, &C.col, (size_t)nnzc + kPad));
    RC(dalloc(h, &C.val, (size_t)nnzc + kPad));
    const int words = (maxspan + 31) / 32 + 1;
    const bool mirror = !bit_symmetric;
    if ((double)galerkin_warp_fill_smem(maxcand, words, maxu) <= kWarpGalerkinSmem) {
        CK(launch_galerkin_warp_fill(A, P.agg, P.pval, P.mate, mem0, mem1, maxcand, words, maxu, bit_symmetric, C,
                                     h->flag + 3, s));
        if (mirror) CK(launch_galerkin_mirror(C, h->flag + 3, s));
    } else if (8.0 * words + 16.0 * maxcand <= kBitmapSmem) {
        CK(launch_galerkin_fill_bitmap(A, P.agg, P.pval, mem0, mem1, maxcand, words, C, h->flag + 3, s));
        CK(launch_galerkin_mirror(C, h->flag + 3, s));
    } else {
        const int cap = pow2ceil(std::max(maxcand, 1));  // <= kGalWarpCand < kMaxGalerkinCap
        CK(launch_galerkin_fill(A, P.agg, P.pval, mem0, mem1, cap, C, s));
        CK(launch_galerkin_mirror(C, h->flag + 3, s));
    }
    return AMG_OK;
}

// One matching pass on A with test vector w: fills P and the coarse matrix C
// (allocated in the hierarchy) and the coarse test vector *wc.  kii_known:
// A's diagonal when the caller has it (a level's first pass), else NULL.
int match_pass(amg_hierarchy* h, const DevCSR& A, const double* w, Pass& P, DevCSR& C, double** wc,
               const double* kii_known) {
    const int n = A.n;
    cudaStream_t s = h->s;
    const double* kii = kii_known;
    Tmp tk(s), tkey(s), tstate(s), tcand(s), tlead(s), tcidx(s), tscan(s), tlists(s);
    if (!kii) {
        double* kd = nullptr;
        RC(tk.get(&kd, n));
        CK(launch_diag(A, kd, s));
        kii = kd;
    }
    uint64_t* key;
    int32_t *state, *cand, *leader, *cidx, *scr;
    RC(tkey.get(&key, A.nnz));
    RC(tstate.get(&state, n));
    RC(tcand.get(&cand, n));
    RC(tlead.get(&leader, n));
    RC(tcidx.get(&cidx, n));
    RC(tscan.get(&scr, scan_scratch_ints(n) + 1));
    int32_t* lists;  // the rounds' active-vertex lists (two, alternating)
    RC(tlists.get(&lists, 2 * (size_t)n));
    phase(h, 2);
    CK(cudaMemsetAsync(h->flag + 1, 0, sizeof(int), s));
    CK(launch_edge_keys(A, kii, w, key, h->flag + 1, s));
    phase(h, 3);
    CK(launch_match_init(n, state, s));
    // rounds in batches of kRoundBatch between host checks; rounds after
    // the last active vertex are no-ops.  round_active[r] = active count
    // after round r gives the exact round count.
    const int maxr = h->o.max_match_rounds;
    CK(cudaMemsetAsync(h->round_active, 0, sizeof(int) * (maxr + kRoundBatch), s));
    int rounds = 0, done = 0;
    if (h->coop) {  // every round in one launch; its round count is read with the aggregation's counts
        CK(launch_match_rounds_coop(A, key, state, cand, h->round_active, lists, maxr, h->flag + 6, h->num_sms, s));
        CK(cudaMemcpyAsync(h->flag_host + 40, h->flag + 6, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h->flag_host + 32, h->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        done = 1;
    }
    while (!done) {
        if (rounds >= maxr) return AMG_ERR_TIMEOUT;
        const int cnt = std::min(kRoundBatch, maxr - rounds);
        CK(launch_match_rounds(A, key, state, cand, h->round_active, lists, rounds, cnt, s));
        CK(cudaMemcpyAsync(h->flag_host, h->round_active + rounds, sizeof(int) * cnt, cudaMemcpyDeviceToHost, s));
        // the edge-key kernel's unsymmetric-pattern flag rides on the same read
        CK(cudaMemcpyAsync(h->flag_host + 32, h->flag + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int r = 0; r < cnt; r++) {
            if (h->flag_host[r] == 0) {
                rounds += r + 1;
                done = 1;
                break;
            }
        }
        if (!done) rounds += cnt;
    }
    phase(h, 4);
    // Aggregates and the coarse rows' widest candidate list are computed
    // before the host learns the coarse size: the buffers sized by it take
    // the fine size n (an upper bound), and one read brings back the coarse
    // size, the widest list, and (cooperative matching) the round count and
    // the edge-key flags.
    P.n = n;
    RC(dalloc(h, &P.mate, n));
    CK(launch_match_finish(n, state, P.mate, leader, s));
    int32_t* total = scr + scan_scratch_ints(n);
    CK(launch_exclusive_scan(leader, cidx, n, total, scr, s));
    RC(dalloc(h, &P.agg, n));
    RC(dalloc(h, &P.pval, n));
    int32_t *mem0, *mem1;
    Tmp tm0(s), tm1(s);
    RC(tm0.get(&mem0, n));
    RC(tm1.get(&mem1, n));
    RC(dalloc(h, wc, n));
    CK(launch_aggregate(n, P.mate, cidx, w, P.agg, P.pval, mem0, mem1, *wc, s));
    phase(h, 5);
    CK(cudaMemsetAsync(h->flag, 0, 3 * sizeof(int), s));
    CK(launch_row_stats(A, mem0, mem1, n, h->flag, s, total));
    CK(cudaMemcpyAsync(h->flag_host, total, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(h->flag_host + 1, h->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->coop) {
        rounds = h->flag_host[40];
        if (rounds > maxr) return AMG_ERR_TIMEOUT;
    }
    P.rounds = rounds;
    if (h->flag_host[32] & 64) return AMG_ERR_ARG;  // structurally unsymmetric matrix
    // values symmetric in every bit: the Galerkin kernels may compute the
    // lower triangle in place
    const int bit_symmetric = (h->flag_host[32] & 128) ? 0 : 1;
    const int nc = h->flag_host[0];
    const int maxcand_all = h->flag_host[1];
    P.nc = nc;
    // Galerkin product of this pass
    if (nc < (1 << 30) && maxcand_all <= kGalWarpCand) {
        RC(galerkin_warp(h, A, P, mem0, mem1, nc, maxcand_all, bit_symmetric, C));
        phase(h, 1);
        return AMG_OK;
    }
    // widest coarse-column span as well (one read)
    CK(launch_row_span(A, P.agg, mem0, mem1, nc, h->flag + 2, s));
    CK(cudaMemcpyAsync(h->flag_host, h->flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const int maxcand = h->flag_host[0], maxspan = h->flag_host[2];
    const int cap = pow2ceil(std::max(maxcand, 1));
    // bitmap kernels when the widest coarse-column span fits shared memory,
    // else the candidate-sorting kernels
    const int words = (maxspan + 31) / 32 + 1;
    const bool bitmap = 8.0 * words + 16.0 * maxcand <= kBitmapSmem;
    if (!bitmap && cap > kMaxGalerkinCap) {
        // rows too wide for both kernels (dense coarse levels of smoothed
        // hierarchies): the row-merge SpGEMMs, same product up to rounding
        RC(galerkin_pass_spgemm(h, A, P.agg, P.pval, mem0, mem1, nc, C));
        h->galerkin_spgemm_passes++;
        phase(h, 1);
        return AMG_OK;
    }
    C.n = nc;
    RC(dalloc(h, &C.rowptr, (size_t)nc + 1));
    int64_t *rowcnt, *scr64;
    Tmp trc(s), ts64(s);
    RC(trc.get(&rowcnt, nc));
    RC(ts64.get(&scr64, scan64_scratch(nc) + 1));
    // Galerkin errors accumulate in flag[3], read once after the last level
    if (bitmap) CK(launch_galerkin_count_bitmap(A, P.agg, mem0, mem1, nc, maxcand, words, rowcnt, h->flag + 3, s));
    else CK(launch_galerkin_count(A, P.agg, mem0, mem1, nc, cap, rowcnt, s));
    CK(launch_scan64(rowcnt, C.rowptr, nc, scr64, s));
    int64_t nnzc = 0;
    RC(read_scalar(h, C.rowptr + nc, &nnzc));
    C.nnz = nnzc;
    RC(dalloc(h, &C.col, (size_t)nnzc + kPad));
    RC(dalloc(h, &C.val, (size_t)nnzc + kPad));
    if (bitmap) CK(launch_galerkin_fill_bitmap(A, P.agg, P.pval, mem0, mem1, maxcand, words, C, h->flag + 3, s));
    else CK(launch_galerkin_fill(A, P.agg, P.pval, mem0, mem1, cap, C, s));
    CK(launch_galerkin_mirror(C, h->flag + 3, s));
    phase(h, 1);
    return AMG_OK;
}

void free_level_matrix(amg_hierarchy* h, DevCSR& A) {
    forget(h, A.rowptr);
    forget(h, A.col);
    forget(h, A.val);
    A = DevCSR{};
}

// Run-encoded columns of level L (left as plain CSR when a row does not
// split into equal runs of consecutive columns).
int build_runs(amg_hierarchy* h, Level& L) {
    cudaStream_t s = h->s;
    const int n = L.A.n;
    if (n < 1) return AMG_OK;
    int32_t* cnt;
    Tmp tc(s);
    RC(tc.get(&cnt, (size_t)n + 1));
    uint8_t* len;
    RC(dalloc(h, &len, (size_t)n + 16));  // padded for 16-byte copies
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    CK(cudaMemsetAsync(cnt + n, 0, sizeof(int32_t), s));
    CK(launch_run_rows(L.A, cnt, len, h->flag, s));
    int bad = 0;
    RC(read_flag(h, &bad));
    if (bad) {
        forget(h, len);
        return AMG_OK;
    }
    RC(dalloc(h, &L.run_ptr, (size_t)n + 5));  // padded for 16-byte copies
    int32_t* scr;
    Tmp tsc(s);
    RC(tsc.get(&scr, scan_scratch_ints(n + 1)));
    CK(launch_exclusive_scan(cnt, L.run_ptr, n + 1, nullptr, scr, s));
    int32_t total = 0;
    RC(read_scalar(h, L.run_ptr + n, &total));
    RC(dalloc(h, &L.run_start, (size_t)total + kPad));
    CK(launch_run_fill(L.A, L.run_ptr, len, L.run_start, s));
    L.run_len = len;
    L.nruns = total;
    return AMG_OK;
}

// ------------------------------------------------------------ autotuning
// The finest level's matrix passes have several layouts (sliced slabs with
// a chosen number of warps per block in FP64; staged slabs in mixed
// precision; CSR row groups).  With opts.autotune the setup times the
// q = K p pass of each candidate on the hierarchy's own matrix and vectors
// (CUDA events on its stream: one warm-up and five timed launches each)
// and keeps the fastest; the three passes of an iteration share the layout.
// The choice is cached for the process by the matrix shape, so later setups
// of the same shape apply it without timing.
struct TuneKey {
    int n;
    int64_t nnz;
    int mixed, stream, sell64, lm;
    bool operator==(const TuneKey& o) const {
        return n == o.n && nnz == o.nnz && mixed == o.mixed && stream == o.stream && sell64 == o.sell64 && lm == o.lm;
    }
};
struct TuneChoice {
    int rowgroups;  // 1: CSR row groups
    int warps;      // FP64 sliced passes: warps per block
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneChoice>> g_tune_cache;

int autotune(amg_hierarchy* h) {
    if (!h->sell64 && !h->stream) return AMG_OK;  // one layout only
    const auto t0 = std::chrono::steady_clock::now();
    const TuneKey key{h->lev[0].A.n, h->lev[0].A.nnz, h->mixed, h->stream, h->sell64, h->sell[0].lm};
    TuneChoice choice{0, h->sell64_warps};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto& kv : g_tune_cache)
            if (kv.first == key) {
                choice = kv.second;
                cached = true;
            }
    }
    if (!cached) {
        cudaStream_t s = h->s;
        const int n = h->lev[0].A.n;
        CK(cudaMemsetAsync(h->p, 0, sizeof(double) * n, s));
        CK(cudaMemsetAsync(h->r, 0, sizeof(double) * n, s));
        if (h->p32) CK(cudaMemsetAsync(h->p32, 0, sizeof(float) * n, s));
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        struct Ev {
            cudaEvent_t a, b;
            ~Ev() {
                cudaEventDestroy(a);
                cudaEventDestroy(b);
            }
        } ev{e0, e1};
        auto timed = [&](auto&& launch, float* ms) -> int {
            CK(launch());
            CK(cudaEventRecord(e0, s));
            for (int k = 0; k < 5; k++) CK(launch());
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(ms, e0, e1));
            return AMG_OK;
        };
        const int save_sell64 = h->sell64, save_stream = h->stream, save_warps = h->sell64_warps;
        float best = 1e30f, ms = 0.f;
        if (save_sell64) {
            int lo, hi;
            sell64_warp_range(&lo, &hi);
            for (int w = lo; w <= hi; w++) {
                h->sell64_warps = w;
                RC(timed([&] { return sell64_spmv_pq(h, h->p, h->r, h->q, h->partials, h->partials, 0, s); }, &ms));
                if (ms < best) {
                    best = ms;
                    choice = TuneChoice{0, w};
                }
            }
        } else {
            RC(timed([&] {
                return h->stream == 2 ? sell_spmv_pq(h, h->p32, h->p, h->r, h->q, h->partials, h->partials, 0, s)
                                      : launch_stream_spmv_pq(h, h->p32, h->p, h->r, h->q, h->partials, h->partials,
                                                              0, s);
            }, &ms));
            best = ms;
            choice = TuneChoice{0, save_warps};
        }
        h->sell64 = 0;
        h->stream = 0;
        RC(timed([&] { return launch_rowgroup_pq(h, s); }, &ms));
        h->sell64 = save_sell64;
        h->stream = save_stream;
        h->sell64_warps = save_warps;
        if (ms < best) choice = TuneChoice{1, save_warps};
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache.push_back({key, choice});
    }
    if (choice.rowgroups) {
        h->sell64 = 0;
        h->stream = 0;
        h->sell[1].on = 0;  // level 1's sliced passes follow the finest level's staged layout
    } else {
        h->sell64_warps = choice.warps;
    }
    h->tune_ms = cached ? 0.0 : std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return AMG_OK;
}

int build(amg_hierarchy* h, const amg_csr* K) {
    cudaStream_t s = h->s;
    const int n0 = K->n;
    phase(h, 0);
    Level& L0 = h->lev[0];
    L0.A.n = n0;
    L0.A.nnz = K->nnz;
    // + 2: the staged finest-level passes copy row offsets in 16-byte units
    RC(dalloc(h, &L0.A.rowptr, (size_t)n0 + 3));
    RC(dalloc(h, &L0.A.col, (size_t)K->nnz + kPad));
    RC(dalloc(h, &L0.A.val, (size_t)K->nnz + kPad));
    const cudaMemcpyKind kind = K->mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(L0.A.rowptr, K->rowptr, sizeof(int64_t) * (n0 + 1), kind, s));
    CK(cudaMemcpyAsync(L0.A.col, K->col, sizeof(int32_t) * K->nnz, kind, s));
    CK(cudaMemcpyAsync(L0.A.val, K->val, sizeof(double) * K->nnz, kind, s));
    // structural checks
    int64_t ends[2];
    CK(cudaMemcpyAsync(h->flag_host, L0.A.rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ends[0] = *(int64_t*)h->flag_host;
    CK(cudaMemcpyAsync(h->flag_host, L0.A.rowptr + n0, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    ends[1] = *(int64_t*)h->flag_host;
    if (ends[0] != 0 || ends[1] != K->nnz) return AMG_ERR_ARG;
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    CK(launch_validate_csr(L0.A, h->flag, s));
    int bad = 0;
    RC(read_flag(h, &bad));
    if (bad & 1) return AMG_ERR_ARG;
    if (bad & 2) return AMG_ERR_NAN;
    if (bad & 4) return AMG_ERR_NOT_SPD;

    RC(dalloc(h, &h->round_active, (size_t)h->o.max_match_rounds + kRoundBatch));
    for (int l = 0;; l++) {
        phase(h, 1);
        Level& F = h->lev[l];
        const int n = F.A.n;
        RC(dalloc(h, &F.kii, n));
        RC(dalloc(h, &F.dl1, n));
        RC(dalloc(h, &F.invd, n));
        if (l == 0) {
            CK(cudaMemsetAsync(h->flag, 0, 16 * sizeof(int), s));  // also clears the deferred error words
            CK(launch_l1diag(F.A, F.kii, F.dl1, F.invd, h->flag, s));
            RC(read_flag(h, &bad));
            if (bad) return AMG_ERR_NOT_SPD;
            // the finest level will have a smoother: start its network now
            if (h->o.mpnn_weights && n > h->o.coarse_max && h->o.max_levels > 1) RC(mpnn_setup_fork(h));
        } else {  // coarse levels: checked once after the loop (flag[4])
            CK(launch_l1diag(F.A, F.kii, F.dl1, F.invd, h->flag + 4, s));
        }
        h->nlev = l + 1;
        if (n <= h->o.coarse_max || l + 1 >= h->o.max_levels) break;
        if (l == 0) {
            RC(dalloc(h, &F.w, n));
            double* wt;
            Tmp tw(s);
            RC(tw.get(&wt, n));
            CK(launch_testvec_init(n, h->o.testvec_kind, h->o.seed, F.w, s));
            for (int sw = 0; sw < h->o.testvec_sweeps; sw++) {
                CK(launch_testvec_sweep(F.A, F.dl1, F.w, wt, s));
                CK(cudaMemcpyAsync(F.w, wt, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
            }
        }
        // m matching passes
        DevCSR cur = F.A;
        double* cw = F.w;
        DevCSR next;
        double* nw = nullptr;
        F.npass = h->o.match_passes;
        for (int q = 0; q < F.npass; q++) {
            next = DevCSR{};
            RC(match_pass(h, cur, cw, F.pass[q], next, &nw, q == 0 ? F.kii : nullptr));
            if (q > 0) {  // intermediate pass matrix no longer needed
                free_level_matrix(h, cur);
                forget(h, cw);
            }
            cur = next;
            cw = nw;
        }
        const int nc = cur.n;
        if ((double)nc > h->o.stag * (double)n) {  // stagnation: discard and stop
            free_level_matrix(h, cur);
            forget(h, cw);
            for (int q = 0; q < F.npass; q++) {
                forget(h, F.pass[q].mate);
                forget(h, F.pass[q].agg);
                forget(h, F.pass[q].pval);
                F.pass[q] = Pass{};
            }
            F.npass = 0;
            break;
        }
        if (l + 1 >= AMG_MAX_LEVELS) return AMG_ERR_ARG;
        // composite map and member lists
        phase(h, 6);
        F.nc = nc;
        RC(dalloc(h, &F.agg, n));
        RC(dalloc(h, &F.pval, n));
        CK(launch_compose(n, F.npass, F.pass, F.agg, F.pval, s));
        int32_t* cnt;
        Tmp tc(s), tsc(s), tcur(s);
        RC(tc.get(&cnt, (size_t)nc + 1));
        RC(dalloc(h, &F.mem_ptr, (size_t)nc + 1));
        RC(dalloc(h, &F.mem_idx, n));
        CK(launch_member_count(n, F.agg, nc, cnt, s));
        int32_t* scr;
        RC(tsc.get(&scr, scan_scratch_ints(nc + 1)));
        CK(launch_exclusive_scan(cnt, F.mem_ptr, nc + 1, nullptr, scr, s));
        int* cursor;
        RC(tcur.get(&cursor, nc));
        CK(launch_member_fill(n, F.agg, F.mem_ptr, nc, F.mem_idx, cursor, s));
        if (h->o.smooth_levels < 0 || l < h->o.smooth_levels) {
            // smoothed prolongator: its Galerkin product replaces the tentative one
            phase(h, 10);
            // a setup given network weights smooths level 0 with the network's theta
            if (l == 0 && h->o.mpnn_weights) RC(mpnn_setup_theta(h));
            DevCSR Kc;
            RC(smooth_level(h, l, Kc));
            free_level_matrix(h, cur);
            cur = Kc;
        }
        Level& C = h->lev[l + 1];
        C.A = cur;
        C.w = cw;
    }
    // deferred checks of the coarse levels: Galerkin structure, positive diagonals
    CK(cudaMemcpyAsync(h->flag_host, h->flag, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h->flag_host[3]) return AMG_ERR_ARG;  // structurally unsymmetric input
    if (h->flag_host[4]) return AMG_ERR_NOT_SPD;
    // coarsest level: dense inverse
    phase(h, 7);
    Level& Lc = h->lev[h->nlev - 1];
    const int nd = Lc.A.n;
    if (nd > h->o.dense_max) return AMG_ERR_COARSE_TOO_LARGE;
    h->ndense = nd;
    double* D;
    Tmp td(s);
    RC(td.get(&D, (size_t)nd * nd));
    RC(dalloc(h, &h->Ainv, (size_t)2 * nd * nd));
    CK(launch_dense_from_csr(Lc.A, D, s));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    CK(launch_dense_spd_inverse(nd, D, h->Ainv, h->flag, s));
    RC(read_flag(h, &bad));
    if (bad) return AMG_ERR_NOT_SPD;
    if (h->o.coarse_solver == 1) RC(dalloc(h, &h->ccg, (size_t)5 * nd));
    // solve workspace
    phase(h, 8);
    for (int l = 0; l < h->nlev; l++) {
        Level& F = h->lev[l];
        const int n = F.A.n;
        if (h->mixed) {  // FP32 copies of the level (BF16 finest values in the V-cycle if asked)
            RC(dalloc(h, &F.val32, (size_t)F.A.nnz + kPad));
            CK(launch_to_f32(F.A.val, F.val32, F.A.nnz, s));
            if (l == 0 && h->o.precision == AMG_FP32_BF16FINE && h->nlev > 1) {
                RC(dalloc(h, &F.val16, (size_t)F.A.nnz + kPad));
                CK(launch_to_bf16(F.A.val, F.val16, F.A.nnz, s));
            }
            RC(dalloc(h, &F.invd32, (size_t)n + 4));
            CK(launch_to_f32(F.invd, F.invd32, n, s));
            if (l > 0) RC(dalloc(h, &F.f32, (size_t)n + 4));  // padded: staged segment copies
            // + 4: the staged finest-level passes copy vector windows widened
            // to 16-byte boundaries
            RC(dalloc(h, &F.x32, (size_t)n + 4));
            RC(dalloc(h, &F.t32, (size_t)n + 4));
            if (h->o.cheb_degree > 0)
                for (int c = 0; c < 2; c++) RC(dalloc(h, reinterpret_cast<float**>(&F.cd[c]), (size_t)n + 4));
        } else {
            if (l > 0) RC(dalloc(h, &F.f, n));
            // + 4: the FP64 sliced passes copy vector windows in 4-entry groups
            RC(dalloc(h, &F.x, (size_t)n + 4));
            RC(dalloc(h, &F.t, (size_t)n + 4));
            if (h->o.cheb_degree > 0)
                for (int c = 0; c < 2; c++) RC(dalloc(h, reinterpret_cast<double**>(&F.cd[c]), (size_t)n + 4));
        }
    }
    if (h->mixed) RC(dalloc(h, &h->p32, (size_t)n0 + 4));
    // run-encoded columns of the finest matrix when every row qualifies
    if (h->o.matrix_format >= 1 && h->nlev > 0 && L0.A.nnz < INT32_MAX) RC(build_runs(h, L0));
    // the vectorised loads need 16-byte aligned column and value arrays
    for (int l = 0; l < h->nlev; l++) {
        const Level& F = h->lev[l];
        const void* ptrs[4] = {F.A.col, F.A.val, F.val32, F.val16};
        for (const void* p : ptrs)
            if (p && (reinterpret_cast<uintptr_t>(p) & 15)) return AMG_ERR_CUDA;
    }
    // CG vectors, padded by 4 entries for the 16-byte copies of the staged passes
    RC(dalloc(h, &h->x, (size_t)n0 + 4));
    RC(dalloc(h, &h->r, (size_t)n0 + 4));
    RC(dalloc(h, &h->p, (size_t)n0 + 4));
    RC(dalloc(h, &h->q, (size_t)n0 + 4));
    RC(dalloc(h, &h->z, (size_t)n0 + 4));
    RC(dalloc(h, &h->F, (size_t)n0 + 4));
    h->npart = (int)partial_slot_size(n0, h->num_sms);
    RC(dalloc(h, &h->partials, partial_slot_count() * h->npart));
    RC(dalloc(h, &h->st, 1));
    h->hist_cap = kHistCap;
    RC(dalloc(h, &h->hist, kHistCap));
    CK(cudaMemsetAsync(h->st, 0, sizeof(SolveState), s));
    if (h->o.matrix_format == 2) {
        RC(stream_prepare(h, h->flag));
        RC(sell_prepare_level1(h, h->flag));
        RC(sell64_prepare(h, h->flag));
    }
    if (h->o.autotune && h->o.cheb_degree == 0) RC(autotune(h));
    if (h->o.mpnn_weights) {
        phase(h, 9);
        RC(mpnn_setup_join(h));
    }
    return AMG_OK;
}

// Bytes of a level's column information per matrix pass: 4 per entry in
// CSR; with run-encoded columns 4 per run + 4 per row (run_ptr) + 1 per
// row (run length).
double index_bytes(const Level& L) {
    if (L.run_ptr) return (double)L.nruns * 4.0 + (L.A.n + 1.0) * 4.0 + (double)L.A.n;
    return (double)L.A.nnz * 4.0;
}

// Index and row-structure bytes of one finest-level pass of the precision
// in use (padding excluded): the sliced slabs read a 16-bit window offset
// per run and one slot offset per slab; the other formats read the row
// offsets (8 B per row) and the column index (index_bytes).
static double fine_structure_bytes(const amg_hierarchy* h) {
    const Level& L0 = h->lev[0];
    if (h->stream == 2 || h->sell64) return (double)L0.nruns * 2.0 + (h->sell[0].nsl + 1.0) * 4.0;
    return index_bytes(L0) + (L0.A.n + 1.0) * 8.0;
}

void fill_info(amg_hierarchy* h) {
    amg_info& I = h->info;
    I.levels = h->nlev;
    double tot = 0.0, vbytes = 0.0;
    for (int l = 0; l < h->nlev; l++) {
        I.n[l] = h->lev[l].A.n;
        I.nnz[l] = h->lev[l].A.nnz;
        tot += (double)h->lev[l].A.nnz;
        int rounds = 0;
        for (int q = 0; q < h->lev[l].npass; q++) rounds += h->lev[l].pass[q].rounds;
        I.match_rounds[l] = rounds;
        I.level_format[l] = h->lev[l].run_ptr ? 1 : 0;
        I.smoothed[l] = h->lev[l].smoothed;
        I.p_nnz[l] = l + 1 < h->nlev ? (h->lev[l].smoothed ? h->lev[l].sp.nnz : h->lev[l].A.n) : 0;
    }
    I.staged_passes = h->sell64 ? 3 : h->stream;
    const bool sl = h->stream == 2 || h->sell64;
    I.staged_slots = sl ? h->sell[0].slots * h->sell[0].lm * 32 : 0;
    I.staged_buffers[0] = h->stream == 2 ? h->sell[0].nbuf[0] : h->stream ? h->stream_nbuf[0] : 0;
    I.staged_buffers[1] = h->stream == 2 ? h->sell[0].nbuf[1] : h->stream ? h->stream_nbuf[1] : 0;
    // the FP64 passes hold the same window entries in FP64
    I.staged_window_bytes = h->sell64 ? 2 * h->sell[0].xbytes
                            : sl      ? h->sell[0].xbytes
                            : h->stream ? h->stream_xbytes
                                        : 0;
    I.staged_level1 = h->sell[1].on;
    I.sell64_warps = h->sell64 ? h->sell64_warps : 0;
    I.tune_ms = h->tune_ms;
    I.opc = tot / (double)h->lev[0].A.nnz;
    // algorithmic bytes: one matrix pass = nnz (value + 4) + (n + 1) 8 + x read + y write
    // (value and vector sizes of the V-cycle precision: 8 / 8 in FP64, 4 / 4 in
    // mixed precision with 2-byte values on the finest level when BF16)
    const double vb = h->mixed ? 4.0 : 8.0;
    auto pass_bytes = [&](const Level& L, double valb) {
        const DevCSR& A = L.A;
        const double sb = (&L == &h->lev[0]) ? fine_structure_bytes(h) : index_bytes(L) + (A.n + 1.0) * 8.0;
        return (double)A.nnz * valb + sb + 2.0 * A.n * vb;
    };
    if (h->nlev == 1) {
        vbytes = (double)h->ndense * h->ndense * 8.0 + 2.0 * h->ndense * 8.0;
    } else {
        for (int l = 0; l < h->nlev - 1; l++) {
            const DevCSR& A = h->lev[l].A;
            const double valb = (l == 0 && h->lev[0].val16) ? 2.0 : vb;
            vbytes += 2.0 * pass_bytes(h->lev[l], valb) + 6.0 * A.n * vb;
            // a smoothed prolongator is read twice (P_bar^T r and P_bar y): 12 B per entry
            if (h->lev[l].smoothed) vbytes += 2.0 * 12.0 * (double)h->lev[l].sp.nnz;
        }
        vbytes += (double)h->ndense * h->ndense * 8.0 + 2.0 * h->ndense * 8.0;
    }
    I.vcycle_bytes = vbytes;
    const DevCSR& A0 = h->lev[0].A;
    // outer q = K p (FP32 values in mixed mode) + CG vectors; mixed mode adds an
    // FP64 residual replacement every resid_replace_every iterations
    const double ib0 = index_bytes(h->lev[0]);
    double outer = (double)A0.nnz * vb + fine_structure_bytes(h) + 2.0 * A0.n * 8.0;
    if (h->mixed && h->o.resid_replace_every > 0)
        outer += ((double)A0.nnz * 8.0 + ib0 + (A0.n + 1.0) * 8.0 + 3.0 * A0.n * 8.0) / h->o.resid_replace_every;
    I.iter_bytes = vbytes + outer + 10.0 * A0.n * 8.0;
}

void free_multi(amg_hierarchy* h) {
    MultiWork* w = h->mw;
    if (!w) return;
    if (w->graph) cudaGraphExecDestroy(w->graph);
    for (void* p : w->allocs) cudaFreeAsync(p, h->s);
    if (w->st_host) cudaFreeHost(w->st_host);
    if (w->active_host) cudaFreeHost(w->active_host);
    delete w;
    h->mw = nullptr;
}

template <typename T>
int walloc(amg_hierarchy* h, MultiWork& w, T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = dev_alloc(&q, sizeof(T) * (count ? count : 1), h->s);
    if (e != cudaSuccess) return cuda_fail(e, "device allocation");
    w.allocs.push_back(q);
    *p = static_cast<T*>(q);
    return AMG_OK;
}

void destroy(amg_hierarchy* h) {
    if (!h) return;
    free_multi(h);
    mpnn_free(h);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (void* p : h->allocs) cudaFreeAsync(p, h->s);
    h->allocs.clear();
    if (h->s) cudaStreamSynchronize(h->s);
    pinned_put(h->flag_host);  // st_host lives in the same block
    event_put(h->ev0, true);
    event_put(h->ev1, true);
    event_put(h->evs, false);
    for (auto& a : h->prof_ev)
        for (auto& b : a)
            for (auto& e : b) event_put(e, true);
    for (auto& e : h->ph_ev) event_put(e, true);
    if (h->s && h->own_stream) cudaStreamDestroy(h->s);
    delete h;
}

// order the internal stream after the caller's stream (no-op when the
// library runs on the caller's stream itself)
int join_caller(amg_hierarchy* h) {
    if (!h->own_stream) return AMG_OK;
    CK(cudaEventRecord(h->evs, h->us));
    CK(cudaStreamWaitEvent(h->s, h->evs, 0));
    return AMG_OK;
}

}  // namespace

namespace amg {
int join_caller_stream(amg_hierarchy* h) { return join_caller(h); }
int report_cuda(cudaError_t e, const char* what) { return cuda_fail(e, what); }
}  // namespace amg

namespace {

int check_opts(const amg_opts& o) {
    if (o.nu_pre < 1 || o.nu_post < 1 || o.nu_pre > 64 || o.nu_post > 64) return AMG_ERR_ARG;
    if (o.match_passes < 1 || o.match_passes > kMaxPasses) return AMG_ERR_ARG;
    if (o.coarse_max < 1 || o.max_levels < 1 || o.max_levels > AMG_MAX_LEVELS) return AMG_ERR_ARG;
    if (o.dense_max < 1 || o.dense_max > 8192) return AMG_ERR_ARG;
    if (o.testvec_sweeps < 0 || o.testvec_kind < 0 || o.testvec_kind > 1) return AMG_ERR_ARG;
    if (!(o.stag > 0.0) || o.max_match_rounds < 1) return AMG_ERR_ARG;
    if (o.precision < AMG_FP64 || o.precision > AMG_FP32_BF16FINE) return AMG_ERR_ARG;
    if (o.flexible < 0 || o.flexible > 1 || o.resid_replace_every < 0) return AMG_ERR_ARG;
    if (o.matrix_format < 0 || o.matrix_format > 2) return AMG_ERR_ARG;
    if (o.mpnn_bf16 < 0 || o.mpnn_bf16 > 1) return AMG_ERR_ARG;
    if (o.smooth_levels < -1 || !(o.smooth_omega >= 0.0) || !std::isfinite(o.smooth_omega)) return AMG_ERR_ARG;
    if (o.cheb_degree < 0 || o.cheb_degree > 64) return AMG_ERR_ARG;
    if (o.cheb_degree > 0 && o.mpnn_weights) return AMG_ERR_ARG;  // the network damps l1-Jacobi sweeps
    if (o.coarse_solver < 0 || o.coarse_solver > 1 || !(o.coarse_tol >= 0.0) || o.coarse_maxit < 1)
        return AMG_ERR_ARG;
    if (o.autotune < 0 || o.autotune > 1) return AMG_ERR_ARG;
    return AMG_OK;
}

}  // namespace

extern "C" {

int amg_opts_default(amg_opts* o) {
    if (!o) return AMG_ERR_ARG;
    memset(o, 0, sizeof(*o));
    o->nu_pre = 1;
    o->nu_post = 1;
    o->match_passes = 2;
    o->coarse_max = 200;
    o->max_levels = 30;
    o->dense_max = 4096;
    o->testvec_sweeps = 4;
    o->testvec_kind = 0;
    o->seed = 20251126ULL;
    o->stag = 0.9;
    o->max_match_rounds = 1000;
    o->precision = AMG_FP64;
    o->flexible = 0;
    o->resid_replace_every = 20;
    o->matrix_format = 2;
    o->mpnn_weights = nullptr;
    o->mpnn_bf16 = 1;
    o->smooth_levels = 0;
    o->smooth_omega = 4.0 / 3.0;
    o->smooth_theta = nullptr;
    o->cheb_degree = 0;
    o->coarse_solver = 0;
    o->coarse_tol = 1e-4;
    o->coarse_maxit = 30;
    o->autotune = 0;
    return AMG_OK;
}

static bool csr_args_ok(const amg_csr* K) {
    if (!K || K->n < 1 || K->nnz < K->n || !K->rowptr || !K->col || !K->val) return false;
    if (K->mem != AMG_MEM_HOST && K->mem != AMG_MEM_DEVICE) return false;
    return K->nnz <= (int64_t)INT32_MAX * 4;
}

// Hierarchy shell: options, stream, events, pinned mirrors.
static int create_hierarchy(const amg_opts* opts, void* cuda_stream, amg_hierarchy** out) {
    amg_hierarchy* h = new (std::nothrow) amg_hierarchy();
    if (!h) return AMG_ERR_NOMEM;
    if (opts) h->o = *opts;
    else amg_opts_default(&h->o);
    int rc = check_opts(h->o);
    if (rc != AMG_OK) {
        delete h;
        return rc;
    }
    memset(&h->info, 0, sizeof(h->info));
    // the FP32/BF16 V-cycle is symmetric only up to rounding: mixed precision
    // always runs the flexible CG variant
    h->mixed = h->o.precision != AMG_FP64;
    if (h->mixed) h->o.flexible = 1;
    h->us = (cudaStream_t)cuda_stream;
    // A caller-provided stream is used directly (so caller events bracket the
    // kernels); the legacy default stream cannot be captured into a graph,
    // so a NULL stream gets a private stream ordered after it.
    cudaError_t e = cudaSuccess;
    if (h->us) {
        h->s = h->us;
        h->own_stream = false;
    } else {
        e = cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking);
        h->own_stream = true;
    }
    if (e == cudaSuccess) e = event_get(&h->ev0, true);
    if (e == cudaSuccess) e = event_get(&h->ev1, true);
    if (e == cudaSuccess) e = event_get(&h->evs, false);
    void* pin = nullptr;  // flag words (256 B) and the solve-state mirror in one pooled block
    if (e == cudaSuccess) e = pinned_get(&pin);
    if (e == cudaSuccess) {
        static_assert(256 + sizeof(SolveState) <= kPinnedBlock, "pinned block layout");
        h->flag_host = static_cast<int*>(pin);
        h->st_host = reinterpret_cast<SolveState*>(static_cast<char*>(pin) + 256);
    }
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->coop, cudaDevAttrCooperativeLaunch, dev);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "amg_setup init");
        destroy(h);
        return rc;
    }
    rc = join_caller(h);
    if (rc == AMG_OK) rc = dalloc(h, &h->flag, 16);
    if (rc != AMG_OK) {
        destroy(h);
        return rc;
    }
    *out = h;
    return AMG_OK;
}

// Build the hierarchy of K (device or host CSR), time it, fill the info.
static int finish_setup(amg_hierarchy* h, const amg_csr* K) {
    cudaEventRecord(h->ev0, h->s);
    int rc = build(h, K);
    cudaEventRecord(h->ev1, h->s);
    if (rc == AMG_OK) {
        cudaError_t e = cudaStreamSynchronize(h->s);
        if (e != cudaSuccess) rc = cuda_fail(e, "amg_setup");
    }
    if (rc != AMG_OK) {
        cudaStreamSynchronize(h->s);
        return rc;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->info.setup_ms = ms;
    for (int k = 0; k < h->ph_n; k++) {
        float dt = 0.f;
        cudaEvent_t end = (k + 1 < h->ph_n) ? h->ph_ev[k + 1] : h->ev1;
        if (cudaEventElapsedTime(&dt, h->ph_ev[k], end) == cudaSuccess && h->ph_id[k] < 12)
            h->info.setup_phase_ms[h->ph_id[k]] += dt;
    }
    fill_info(h);
    return AMG_OK;
}

int amg_setup(const amg_csr* K, const amg_opts* opts, void* cuda_stream, amg_hierarchy** out) {
    if (!out) return AMG_ERR_ARG;
    *out = nullptr;
    if (!csr_args_ok(K)) return AMG_ERR_ARG;
    amg_hierarchy* h = nullptr;
    int rc = create_hierarchy(opts, cuda_stream, &h);
    if (rc != AMG_OK) return rc;
    rc = finish_setup(h, K);
    if (rc != AMG_OK) {
        destroy(h);
        return rc;
    }
    *out = h;
    return AMG_OK;
}

// Block-diagonal assembly of `count` systems into one device CSR, then the
// usual setup.  Row offsets of the systems are kept for the solves.
static int batch_build(amg_hierarchy* h, int count, const amg_csr* Ks, const std::vector<int64_t>& roff,
                       const std::vector<int64_t>& zoff) {
    cudaStream_t s = h->s;
    const int64_t N = roff[count], Z = zoff[count];
    int64_t maxn = 0;
    for (int k = 0; k < count; k++) maxn = std::max<int64_t>(maxn, Ks[k].n);
    int64_t *rp_all, *rp_tmp;
    int32_t* col_all;
    double* val_all;
    Tmp t1(s), t2(s), t3(s), t4(s);
    RC(t1.get(&rp_all, (size_t)N + 1));
    RC(t2.get(&col_all, (size_t)Z));
    RC(t3.get(&val_all, (size_t)Z));
    RC(t4.get(&rp_tmp, (size_t)maxn + 1));
    CK(cudaMemsetAsync(h->flag, 0, sizeof(int), s));
    for (int k = 0; k < count; k++) {
        const amg_csr& K = Ks[k];
        const cudaMemcpyKind kind = K.mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        CK(cudaMemcpyAsync(col_all + zoff[k], K.col, sizeof(int32_t) * K.nnz, kind, s));
        CK(cudaMemcpyAsync(val_all + zoff[k], K.val, sizeof(double) * K.nnz, kind, s));
        CK(cudaMemcpyAsync(rp_tmp, K.rowptr, sizeof(int64_t) * (K.n + 1), kind, s));
        int64_t first = 0, last = 0;
        RC(read_scalar(h, rp_tmp, &first));
        RC(read_scalar(h, rp_tmp + K.n, &last));
        if (first != 0 || last != K.nnz) return AMG_ERR_ARG;
        CK(launch_shift_block(K.n, K.nnz, rp_tmp, roff[k], zoff[k], rp_all + roff[k], col_all, h->flag, s));
        CK(cudaStreamSynchronize(s));  // rp_tmp is reused by the next system
    }
    int bad = 0;
    RC(read_flag(h, &bad));
    if (bad) return AMG_ERR_ARG;
    h->nsys = count;
    h->sys_off = roff;
    RC(dalloc(h, &h->sys_off_dev, (size_t)count + 1));
    RC(dalloc(h, &h->sys_id, (size_t)N));
    CK(cudaMemcpyAsync(h->sys_off_dev, roff.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, s));
    CK(launch_fill_sys_id(count, h->sys_off_dev, h->sys_id, s));
    const amg_csr all = {(int32_t)N, Z, rp_all, col_all, val_all, AMG_MEM_DEVICE};
    return finish_setup(h, &all);
}

int amg_setup_batch(int32_t count, const amg_csr* Ks, const amg_opts* opts, void* cuda_stream, amg_hierarchy** out) {
    if (!out) return AMG_ERR_ARG;
    *out = nullptr;
    if (count < 1 || count > kMaxSystems || !Ks) return AMG_ERR_ARG;
    std::vector<int64_t> roff(count + 1, 0), zoff(count + 1, 0);
    for (int k = 0; k < count; k++) {
        if (!csr_args_ok(&Ks[k])) return AMG_ERR_ARG;
        roff[k + 1] = roff[k] + Ks[k].n;
        zoff[k + 1] = zoff[k] + Ks[k].nnz;
    }
    if (roff[count] > INT32_MAX || zoff[count] > (int64_t)INT32_MAX * 4) return AMG_ERR_ARG;
    amg_hierarchy* h = nullptr;
    int rc = create_hierarchy(opts, cuda_stream, &h);
    if (rc != AMG_OK) return rc;
    rc = batch_build(h, count, Ks, roff, zoff);
    if (rc != AMG_OK) {
        cudaStreamSynchronize(h->s);
        destroy(h);
        return rc;
    }
    *out = h;
    return AMG_OK;
}

static int run_solve(amg_hierarchy* h, int32_t* iters) {
    cudaStream_t s = h->s;
    CK(cudaEventRecord(h->ev0, s));
    CK(enqueue_pcg_start(h, s));
    h->info.graph_build_ms = 0.0;
    if (!h->graph) {
        const auto tb0 = std::chrono::steady_clock::now();
        cudaGraph_t g;
        const long long before = amg::g_launches.load();
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kGraphIters && e == cudaSuccess; k++) {
            h->prof_slot = h->prof ? k : -1;
            e = enqueue_pcg_iteration(h, s);
        }
        h->prof_slot = -1;
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        h->graph_kernels = amg::g_launches.load() - before;
        amg::g_launches -= h->graph_kernels;  // captured, not launched
        if (e != cudaSuccess) return cuda_fail(e, "capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        h->graph_iters = kGraphIters;
        h->info.graph_build_ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - tb0).count();
    }
    const int max_launches = h->itmax / kGraphIters + 2;
    int it_before = 0;
    for (int k = 0; k <= max_launches + 1; k++) {
        CK(cudaMemcpyAsync(h->st_host, h->st, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (h->prof && k > 0) {  // accumulate the kernels of the launch that just finished
            const int ndone = h->st_host->iters - it_before;
            for (int j = 0; j < kGraphIters; j++)
                for (int q = 0; q < 3; q++) {
                    const int full = q == 0 ? ndone : ndone - (h->st_host->done ? 1 : 0);
                    if (j >= full) continue;
                    float ms = 0.f;
                    if (cudaEventElapsedTime(&ms, h->prof_ev[j][q][0], h->prof_ev[j][q][1]) == cudaSuccess) {
                        h->prof_ms[q] += ms;
                        h->prof_cnt[q]++;
                    }
                }
        }
        it_before = h->st_host->iters;
        if (h->st_host->done || k > max_launches) break;
        CK(cudaGraphLaunch(h->graph, s));
        amg::g_launches += h->graph_kernels;
    }
    CK(cudaEventRecord(h->ev1, s));
    CK(launch_final_residual(h, s));
    CK(cudaStreamSynchronize(s));
    *iters = h->st_host->iters;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->info.solve_ms = ms;
    return h->st_host->done ? h->st_host->status : AMG_ERR_NOT_CONVERGED;
}

int amg_pcg_solve(amg_hierarchy* h, const double* F, double* u, int32_t mem, double rtol, int32_t itmax,
                  int32_t* iters, double* relres) {
    if (!h || !F || !u || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE) || !(rtol >= 0.0) || itmax < 0)
        return AMG_ERR_ARG;
    const int n = h->lev[0].A.n;
    cudaStream_t s = h->s;
    RC(join_caller(h));
    const cudaMemcpyKind in = mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind outk = mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(h->F, F, sizeof(double) * n, in, s));
    CK(cudaMemcpyAsync(h->x, u, sizeof(double) * n, in, s));
    h->rtol = rtol;
    h->itmax = itmax;
    int32_t it = 0;
    int rc = run_solve(h, &it);
    if (rc == AMG_ERR_CUDA || rc == AMG_ERR_NOMEM) return rc;
    double res[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(h->flag_host, final_residual_slot(h), 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    memcpy(res, h->flag_host, sizeof(res));
    if (!(h->st_host->nF > 0.0) && rc == AMG_OK) {  // F = 0: u = 0
        CK(cudaMemsetAsync(h->x, 0, sizeof(double) * n, s));
        res[0] = 0.0;
    }
    const double rel = res[1] > 0.0 ? res[0] / res[1] : 0.0;
    CK(cudaMemcpyAsync(u, h->x, sizeof(double) * n, outk, s));
    CK(cudaStreamSynchronize(s));
    h->info.iters = it;
    h->info.status = rc;
    h->info.final_relres = rel;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return rc;
}

// ------------------------------------------------------ multi-system solves
// Workspace for S systems over R interleaved vectors (reused when unchanged).
static int ensure_multi(amg_hierarchy* h, int R, int S, const int32_t* seg, const int64_t* segoff) {
    if (h->mw && h->mw->R == R && h->mw->S == S && h->mw->seg == seg) return AMG_OK;
    CK(cudaStreamSynchronize(h->s));
    free_multi(h);
    MultiWork* w = new (std::nothrow) MultiWork();
    if (!w) return AMG_ERR_NOMEM;
    h->mw = w;
    w->R = R;
    w->Rp = pow2ceil(R);
    w->S = S;
    w->seg = seg;
    w->segoff = segoff;
    const size_t E = (size_t)h->lev[0].A.n * R;
    RC(walloc(h, *w, &w->x, E));
    RC(walloc(h, *w, &w->r, E));
    RC(walloc(h, *w, &w->p, E));
    RC(walloc(h, *w, &w->q, E));
    RC(walloc(h, *w, &w->z, E));
    RC(walloc(h, *w, &w->F, E));
    RC(walloc(h, *w, &w->pa, E));
    RC(walloc(h, *w, &w->pb, E));
    RC(walloc(h, *w, &w->stage, E));
    if (h->mixed) RC(walloc(h, *w, &w->p32, E));
    RC(walloc(h, *w, &w->dots, (size_t)S * multi_dot_stride()));
    RC(walloc(h, *w, &w->st, (size_t)S));
    RC(walloc(h, *w, &w->active, 1));
    RC(walloc(h, *w, &w->params, 2));
    CK(cudaMemsetAsync(w->pb, 0, sizeof(double) * E, h->s));
    for (int l = 0; l < h->nlev; l++) {
        const size_t El = (size_t)h->lev[l].A.n * R;
        const size_t b = h->mixed ? 4 : 8;
        char *f = nullptr, *x = nullptr, *t = nullptr;
        if (l > 0) RC(walloc(h, *w, &f, El * b));
        RC(walloc(h, *w, &x, El * b));
        RC(walloc(h, *w, &t, El * b));
        w->lf[l] = f;
        w->lx[l] = x;
        w->lt[l] = t;
    }
    CK(cudaMallocHost(&w->st_host, sizeof(MultiState) * S));
    CK(cudaMallocHost(&w->active_host, sizeof(int)));
    return AMG_OK;
}

// Runs the multi-system CG on the workspace (F and x already filled).
// iters/relres/status per system (host arrays, may be NULL).
static int run_multi(amg_hierarchy* h, int32_t* iters, double* relres, int32_t* zero_rhs) {
    MultiWork& w = *h->mw;
    cudaStream_t s = h->s;
    CK(cudaEventRecord(h->ev0, s));
    CK(enqueue_multi_start(h, s));
    if (!w.graph) {
        cudaGraph_t g;
        const long long before = amg::g_launches.load();
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < kGraphIters && e == cudaSuccess; k++) e = enqueue_multi_iteration(h, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        w.graph_kernels = amg::g_launches.load() - before;
        amg::g_launches -= w.graph_kernels;
        if (e != cudaSuccess) return cuda_fail(e, "capture");
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&w.graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            w.graph = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
    }
    const int max_launches = h->itmax / kGraphIters + 2;
    for (int k = 0; k <= max_launches + 1; k++) {
        CK(cudaMemcpyAsync(w.active_host, w.active, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (*w.active_host == 0 || k > max_launches) break;
        CK(cudaGraphLaunch(w.graph, s));
        amg::g_launches += w.graph_kernels;
    }
    CK(cudaEventRecord(h->ev1, s));
    CK(enqueue_multi_final(h, s));
    std::vector<double> dots((size_t)w.S * multi_dot_stride());
    CK(cudaMemcpyAsync(dots.data(), w.dots, sizeof(double) * dots.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(w.st_host, w.st, sizeof(MultiState) * w.S, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, h->ev0, h->ev1);
    h->info.solve_ms = ms;
    int worst = AMG_OK, maxit = 0;
    for (int k = 0; k < w.S; k++) {
        const MultiState& m = w.st_host[k];
        const double rr = std::sqrt(dots[(size_t)k * multi_dot_stride() + 0]);
        const double ff = std::sqrt(dots[(size_t)k * multi_dot_stride() + 1]);
        int st = m.done ? m.status : AMG_ERR_NOT_CONVERGED;
        if (iters) iters[k] = m.iters;
        if (relres) relres[k] = (ff > 0.0 && m.nF > 0.0) ? rr / ff : 0.0;
        if (zero_rhs) zero_rhs[k] = !(m.nF > 0.0) && st == AMG_OK;
        if (st != AMG_OK && (worst == AMG_OK || st == AMG_ERR_NAN)) worst = st;
        maxit = std::max(maxit, m.iters);
    }
    h->info.iters = maxit;
    h->info.status = worst;
    return worst;
}

static int check_multi_opts(const amg_hierarchy* h) {
    if (h->o.coarse_solver != 0) return AMG_ERR_ARG;  // the multi-system solves use the dense coarse inverse
    // the multi-system V-cycle prolongates with the tentative P's member lists
    // and smooths with one l1-Jacobi sweep
    for (int l = 0; l < h->nlev; l++)
        if (h->lev[l].smoothed) return AMG_ERR_ARG;
    if (h->o.cheb_degree > 0) return AMG_ERR_ARG;
    return (h->o.nu_pre == 1 && h->o.nu_post == 1) ? AMG_OK : AMG_ERR_ARG;
}

int amg_pcg_solve_multi(amg_hierarchy* h, int32_t nrhs, const double* F, double* U, int64_t ld, int32_t mem,
                        double rtol, int32_t itmax, int32_t* iters, double* relres) {
    if (!h || !F || !U || nrhs < 1 || nrhs > 32 || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE) ||
        !(rtol >= 0.0) || itmax < 0 || h->nsys > 0)
        return AMG_ERR_ARG;
    const int n = h->lev[0].A.n;
    if (ld < n) return AMG_ERR_ARG;
    RC(check_multi_opts(h));
    RC(join_caller(h));
    RC(ensure_multi(h, nrhs, nrhs, nullptr, nullptr));
    MultiWork& w = *h->mw;
    cudaStream_t s = h->s;
    const size_t colb = sizeof(double) * n, ldb = sizeof(double) * ld;
    if (mem == AMG_MEM_HOST) {
        CK(cudaMemcpy2DAsync(w.stage, colb, F, ldb, colb, nrhs, cudaMemcpyHostToDevice, s));
        CK(launch_interleave(n, nrhs, n, w.stage, w.F, s));
        CK(cudaMemcpy2DAsync(w.stage, colb, U, ldb, colb, nrhs, cudaMemcpyHostToDevice, s));
        CK(launch_interleave(n, nrhs, n, w.stage, w.x, s));
    } else {
        CK(launch_interleave(n, nrhs, ld, F, w.F, s));
        CK(launch_interleave(n, nrhs, ld, U, w.x, s));
    }
    h->rtol = rtol;
    h->itmax = itmax;
    std::vector<int32_t> zero(nrhs, 0);
    const int rc = run_multi(h, iters, relres, zero.data());
    if (rc == AMG_ERR_CUDA || rc == AMG_ERR_NOMEM) return rc;
    if (mem == AMG_MEM_HOST) {
        CK(launch_deinterleave(n, nrhs, n, w.x, w.stage, s));
        CK(cudaMemcpy2DAsync(U, ldb, w.stage, colb, colb, nrhs, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        for (int k = 0; k < nrhs; k++)
            if (zero[k]) memset(U + (size_t)k * ld, 0, colb);
    } else {
        CK(launch_deinterleave(n, nrhs, ld, w.x, U, s));
        for (int k = 0; k < nrhs; k++)
            if (zero[k]) CK(cudaMemsetAsync(U + (size_t)k * ld, 0, colb, s));
        CK(cudaStreamSynchronize(s));
    }
    return rc;
}

int amg_pcg_solve_batch(amg_hierarchy* h, const double* const* F, double* const* U, int32_t mem, double rtol,
                        int32_t itmax, int32_t* iters, double* relres) {
    if (!h || !F || !U || h->nsys < 1 || (mem != AMG_MEM_HOST && mem != AMG_MEM_DEVICE) || !(rtol >= 0.0) ||
        itmax < 0)
        return AMG_ERR_ARG;
    for (int k = 0; k < h->nsys; k++)
        if (!F[k] || !U[k]) return AMG_ERR_ARG;
    RC(check_multi_opts(h));
    RC(join_caller(h));
    RC(ensure_multi(h, 1, h->nsys, h->sys_id, h->sys_off_dev));
    MultiWork& w = *h->mw;
    cudaStream_t s = h->s;
    const cudaMemcpyKind in = mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind outk = mem == AMG_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int k = 0; k < h->nsys; k++) {
        const int64_t o = h->sys_off[k], nk = h->sys_off[k + 1] - o;
        CK(cudaMemcpyAsync(w.F + o, F[k], sizeof(double) * nk, in, s));
        CK(cudaMemcpyAsync(w.x + o, U[k], sizeof(double) * nk, in, s));
    }
    h->rtol = rtol;
    h->itmax = itmax;
    std::vector<int32_t> zero(h->nsys, 0);
    const int rc = run_multi(h, iters, relres, zero.data());
    if (rc == AMG_ERR_CUDA || rc == AMG_ERR_NOMEM) return rc;
    for (int k = 0; k < h->nsys; k++) {
        const int64_t o = h->sys_off[k], nk = h->sys_off[k + 1] - o;
        if (zero[k]) {
            if (mem == AMG_MEM_DEVICE) CK(cudaMemsetAsync(U[k], 0, sizeof(double) * nk, s));
            else {
                CK(cudaStreamSynchronize(s));
                memset(U[k], 0, sizeof(double) * nk);
            }
        } else {
            CK(cudaMemcpyAsync(U[k], w.x + o, sizeof(double) * nk, outk, s));
        }
    }
    CK(cudaStreamSynchronize(s));
    return rc;
}

int amg_vcycle_apply(amg_hierarchy* h, const double* r_dev, double* z_dev) {
    if (!h || !r_dev || !z_dev) return AMG_ERR_ARG;
    const int n = h->lev[0].A.n;
    cudaStream_t s = h->s;
    RC(join_caller(h));
    CK(cudaMemsetAsync(h->st, 0, sizeof(SolveState), s));
    CK(cudaMemcpyAsync(h->r, r_dev, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(enqueue_vcycle_standalone(h, s));
    CK(cudaMemcpyAsync(z_dev, h->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

int amg_level_spmv(amg_hierarchy* h, int32_t level, const double* x_dev, double* y_dev) {
    if (!h || level < 0 || level >= h->nlev || !x_dev || !y_dev) return AMG_ERR_ARG;
    RC(join_caller(h));
    CK(launch_spmv(h->lev[level].A, x_dev, y_dev, h->s));
    CK(cudaStreamSynchronize(h->s));
    return AMG_OK;
}

int amg_get_info(const amg_hierarchy* h, amg_info* info) {
    if (!h || !info) return AMG_ERR_ARG;
    *info = h->info;
    return AMG_OK;
}

int amg_export_level(const amg_hierarchy* hc, int32_t level, int64_t* rowptr, int32_t* col, double* val, double* dl1,
                     double* w, int32_t* agg, double* pval) {
    amg_hierarchy* h = const_cast<amg_hierarchy*>(hc);
    if (!h || level < 0 || level >= h->nlev) return AMG_ERR_ARG;
    const Level& L = h->lev[level];
    cudaStream_t s = h->s;
    const int n = L.A.n;
    if (rowptr) CK(cudaMemcpyAsync(rowptr, L.A.rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, s));
    if (col) CK(cudaMemcpyAsync(col, L.A.col, sizeof(int32_t) * L.A.nnz, cudaMemcpyDeviceToHost, s));
    if (val) CK(cudaMemcpyAsync(val, L.A.val, sizeof(double) * L.A.nnz, cudaMemcpyDeviceToHost, s));
    if (dl1) CK(cudaMemcpyAsync(dl1, L.dl1, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    if (w) {
        if (!L.w) return AMG_ERR_ARG;
        CK(cudaMemcpyAsync(w, L.w, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    if (agg || pval) {
        if (level == h->nlev - 1) return AMG_ERR_ARG;
        if (agg) CK(cudaMemcpyAsync(agg, L.agg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        if (pval) CK(cudaMemcpyAsync(pval, L.pval, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

int amg_export_prolongator(const amg_hierarchy* hc, int32_t level, int64_t* nnz, int64_t* rowptr, int32_t* col,
                           double* val) {
    amg_hierarchy* h = const_cast<amg_hierarchy*>(hc);
    if (!h || !nnz || level < 0 || level + 1 >= h->nlev) return AMG_ERR_ARG;
    RC(join_caller(h));
    const Level& L = h->lev[level];
    const int n = L.A.n;
    if (L.smoothed) {
        *nnz = L.sp.nnz;
        if (rowptr) CK(cudaMemcpyAsync(rowptr, L.sp.rowptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToHost, h->s));
        if (col) CK(cudaMemcpyAsync(col, L.sp.col, sizeof(int32_t) * L.sp.nnz, cudaMemcpyDeviceToHost, h->s));
        if (val) CK(cudaMemcpyAsync(val, L.sp.val, sizeof(double) * L.sp.nnz, cudaMemcpyDeviceToHost, h->s));
    } else {
        *nnz = n;
        if (col) CK(cudaMemcpyAsync(col, L.agg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->s));
        if (val) CK(cudaMemcpyAsync(val, L.pval, sizeof(double) * n, cudaMemcpyDeviceToHost, h->s));
        if (rowptr)
            for (int i = 0; i <= n; i++) rowptr[i] = i;
    }
    CK(cudaStreamSynchronize(h->s));
    return AMG_OK;
}

int amg_export_coarse(const amg_hierarchy* hc, int32_t* n, double* L, double* Ainv) {
    amg_hierarchy* h = const_cast<amg_hierarchy*>(hc);
    if (!h || !n || !h->Ainv) return AMG_ERR_ARG;
    RC(join_caller(h));
    const int nd = h->ndense;
    *n = nd;
    const size_t bytes = sizeof(double) * (size_t)nd * nd;
    if (Ainv) CK(cudaMemcpyAsync(Ainv, h->Ainv, bytes, cudaMemcpyDeviceToHost, h->s));
    if (L) CK(cudaMemcpyAsync(L, h->Ainv + (size_t)nd * nd, bytes, cudaMemcpyDeviceToHost, h->s));
    CK(cudaStreamSynchronize(h->s));
    return AMG_OK;
}

int amg_export_pass(const amg_hierarchy* hc, int32_t level, int32_t pass, int64_t* n_s, int32_t* mate, int32_t* agg,
                    double* pval) {
    amg_hierarchy* h = const_cast<amg_hierarchy*>(hc);
    if (!h || level < 0 || level >= h->nlev || pass < 0 || pass >= h->lev[level].npass) return AMG_ERR_ARG;
    const Pass& P = h->lev[level].pass[pass];
    cudaStream_t s = h->s;
    if (n_s) *n_s = P.n;
    if (mate) CK(cudaMemcpyAsync(mate, P.mate, sizeof(int32_t) * P.n, cudaMemcpyDeviceToHost, s));
    if (agg) CK(cudaMemcpyAsync(agg, P.agg, sizeof(int32_t) * P.n, cudaMemcpyDeviceToHost, s));
    if (pval) CK(cudaMemcpyAsync(pval, P.pval, sizeof(double) * P.n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return AMG_OK;
}

int64_t amg_kernel_launches(void) { return (int64_t)amg::g_launches.load(); }

int amg_profile_kernels(amg_hierarchy* h, int32_t enable) {
    if (!h || enable < 0 || enable > 1) return AMG_ERR_ARG;
    if (enable && !h->prof_ev[0][0][0]) {
        for (auto& a : h->prof_ev)
            for (auto& b : a)
                for (auto& e : b)
                    if (!e) CK(event_get(&e, true));
    }
    if (h->prof != enable && h->graph) {  // the iteration graph changes shape
        CK(cudaStreamSynchronize(h->s));
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    h->prof = enable;
    for (int q = 0; q < 3; q++) {
        h->prof_ms[q] = 0.0;
        h->prof_cnt[q] = 0;
    }
    return AMG_OK;
}

int amg_kernel_times(const amg_hierarchy* h, double* ms, int64_t* count, double* bytes) {
    if (!h) return AMG_ERR_ARG;
    const double n = h->lev[0].A.n, nnz = (double)h->lev[0].A.nnz;
    const double flex = h->o.flexible ? 8.0 * n : 0.0;
    double b[3];
    if (h->mixed) {  // FP32 outer values, FP32 (or BF16) V-cycle values, FP32 V-cycle vectors
        const double vcv = h->lev[0].val16 ? 2.0 : 4.0;
        const double rows = fine_structure_bytes(h);
        b[0] = nnz * 4.0 + rows + 4.0 * n + 8.0 * n + 8.0 * n + flex;  // p32 gather, q, p
        b[1] = nnz * vcv + rows + 8.0 * n + 4.0 * n + 4.0 * n;  // r, x, rbuf
        b[2] = nnz * vcv + rows + 8.0 * n + 4.0 * n + 4.0 * n + 8.0 * n + flex;  // r, x, invd, z
    } else {
        const double base = nnz * 8.0 + fine_structure_bytes(h);
        b[0] = base + 16.0 * n + flex;
        b[1] = base + 24.0 * n;
        b[2] = base + 32.0 * n + flex;
    }
    for (int q = 0; q < 3; q++) {
        if (ms) ms[q] = h->prof_ms[q];
        if (count) count[q] = h->prof_cnt[q];
        if (bytes) bytes[q] = b[q];
    }
    return AMG_OK;
}

int amg_free(amg_hierarchy* h) {
    if (!h) return AMG_ERR_ARG;
    destroy(h);
    return AMG_OK;
}

const char* amg_strerror(int code) {
    switch (code) {
        case AMG_OK: return "ok";
        case AMG_ERR_ARG: return "invalid argument or malformed matrix";
        case AMG_ERR_NOT_SPD: return "matrix not symmetric positive definite (diagonal or coarse Cholesky)";
        case AMG_ERR_BREAKDOWN: return "CG breakdown (p^T K p <= 0)";
        case AMG_ERR_NOT_CONVERGED: return "not converged within itmax";
        case AMG_ERR_TIMEOUT: return "matching did not finish within max_match_rounds";
        case AMG_ERR_CUDA: return "CUDA runtime error";
        case AMG_ERR_NAN: return "NaN or Inf encountered";
        case AMG_ERR_COARSE_TOO_LARGE: return "coarsest level larger than dense_max";
        case AMG_ERR_NOMEM: return "device memory allocation failed";
        case AMG_ERR_ROW_TOO_LONG: return "Galerkin row exceeds kernel capacity";
        default: return "unknown status";
    }
}

const char* amg_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"
