/*
 * amg_gb300.h -- C ABI of the GB300 (sm_103a) matching-based aggregation
 * AMG preconditioned conjugate gradient solver for symmetric positive
 * definite systems K u = F, such as the stiffness systems of isogeometric
 * (B-spline / NURBS) discretisations of the Poisson problem.
 *
 * Method: arXiv 2511.21268 ("Parallel matching-based AMG preconditioners for
 * elliptic equations discretized by IgA").
 *   - Sec. 3: Galerkin hierarchy K^(l+1) = P^T K^(l) P (Eq. galerkin_matrix_
 *     projection), two-level correction applied recursively as a V-cycle,
 *     used as the preconditioner of CG.
 *   - Sec. 3.1: aggregation by compatible weighted matching -- test vector w
 *     from relaxation on K w = 0, edge weights c_ij (Eq. cij), maximum
 *     product matching (Eq. maxprod) approximated greedily, pair/singleton
 *     prolongator (Eq. prolongation), m-step aggregation P = P_1 ... P_m,
 *     operator complexity (Eq. OPC).
 *   - Sec. 3.2: l1-Jacobi smoother, d_i = k_ii + sum_{j!=i} |k_ij|.
 *   - Sec. 4 ("Solver invocation"): u is the initial guess on input and the
 *     solution on output; iteration count and final residual are returned.
 *
 * Conventions for every entry point:
 *   - Return value 0 (AMG_OK) on success, a negative AMG_ERR_* code
 *     otherwise; amg_strerror() names it.  No C++ exception crosses the ABI.
 *   - Pointers are plain host or device addresses as stated per argument;
 *     the caller keeps ownership of everything it passes in and the library
 *     copies what it keeps.  The opaque amg_hierarchy is owned by the
 *     library (device memory) until amg_free().
 *   - All GPU work is enqueued on the CUDA stream given to amg_setup (NULL =
 *     the legacy default stream); calls return after that work finished.
 *   - Arithmetic: setup in FP64 with explicitly rounded operations in a
 *     fixed order (results reproducible bit for bit); the solve in FP64
 *     (AMG_FP64) or with an FP32/BF16 V-cycle (see amg_opts.precision).
 */
#ifndef AMG_GB300_H
#define AMG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define AMG_OK 0
#define AMG_ERR_ARG (-1)            /* invalid argument or malformed CSR */
#define AMG_ERR_NOT_SPD (-2)        /* nonpositive diagonal or failed coarse Cholesky */
#define AMG_ERR_BREAKDOWN (-3)      /* p^T K p <= 0 in CG */
#define AMG_ERR_NOT_CONVERGED (-4)  /* itmax reached before rtol */
#define AMG_ERR_TIMEOUT (-5)        /* matching did not finish within max_match_rounds */
#define AMG_ERR_CUDA (-6)           /* CUDA runtime error (see amg_last_cuda_error) */
#define AMG_ERR_NAN (-7)            /* NaN/Inf met in the data or the iteration */
#define AMG_ERR_COARSE_TOO_LARGE (-8) /* coarsest level above dense_max rows */
#define AMG_ERR_NOMEM (-9)          /* device allocation failed */
#define AMG_ERR_ROW_TOO_LONG (-10)  /* a Galerkin row exceeds the kernel's capacity */

/* ---- precision of the V-cycle (amg_opts.precision) ---- */
#define AMG_FP64 0          /* everything FP64 */
#define AMG_FP32 1          /* FP32 level matrices and V-cycle vectors, FP64 outer CG */
#define AMG_FP32_BF16FINE 2 /* as AMG_FP32 with BF16 values of the finest matrix in the V-cycle */

/* ---- where a pointer lives ---- */
#define AMG_MEM_HOST 0
#define AMG_MEM_DEVICE 1

/* Square sparse matrix in CSR: rowptr[n+1] (int64, rowptr[0] = 0,
 * nondecreasing), col[nnz] (int32, strictly increasing within each row,
 * diagonal stored), val[nnz] (FP64).  `mem` says whether the three arrays
 * are host or device pointers.  Read only; the library copies it. */
typedef struct {
    int32_t n;
    int64_t nnz;
    const int64_t* rowptr;
    const int32_t* col;
    const double* val;
    int32_t mem;
} amg_csr;

/* Options; fill with amg_opts_default() and override fields. */
typedef struct {
    int32_t nu_pre;              /* l1-Jacobi pre-smoothing sweeps (1) */
    int32_t nu_post;             /* l1-Jacobi post-smoothing sweeps (1) */
    int32_t match_passes;        /* m: matching passes per level, aggregates <= 2^m (2) */
    int32_t coarse_max;          /* stop coarsening at <= this many rows (200) */
    int32_t max_levels;          /* hierarchy depth limit (30) */
    int32_t dense_max;           /* largest coarsest level solved densely (4096) */
    int32_t testvec_sweeps;      /* relaxation sweeps for the test vector (4) */
    int32_t testvec_kind;        /* 0 = SplitMix64 random start, 1 = all ones (0) */
    uint64_t seed;               /* SplitMix64 seed of the random start (20251126) */
    double stag;                 /* discard a level keeping > stag * rows (0.9) */
    int32_t max_match_rounds;    /* bound on matching rounds per pass (1000) */
    int32_t precision;           /* AMG_FP64 / AMG_FP32 / AMG_FP32_BF16FINE (AMG_FP64) */
    int32_t flexible;            /* 0 = PCG, 1 = flexible CG with one direction (0) */
    int32_t resid_replace_every; /* FP64 true-residual replacement period, 0 = off (20) */
    int32_t matrix_format;       /* finest-level matrix passes: 0 = plain CSR; 1 = run-encoded
                                    columns when every row is a sequence of equal runs (2..9
                                    entries, rows < 65536 entries) of consecutive columns, as in
                                    tensor-product IgA matrices; 2 = as 1, and the finest-level
                                    passes run on a sliced copy (32-row slabs, a lane per row):
                                    streamed into shared memory by bulk copies in mixed precision,
                                    FP64 values with a warp per slab in FP64 (2) */
    const float* mpnn_weights;   /* NULL, or the weights of the damping network (AMG_MPNN_NPARAM
                                    floats in the layout of amg_mpnn_apply; DEVICE pointer, read
                                    during amg_setup only).  Setup then installs the learned damping
                                    exactly as amg_mpnn_apply(h, mpnn_weights, mpnn_bf16) right after
                                    it would; the finest level's features and network run on a
                                    second stream alongside the coarse-level setup (NULL) */
    int32_t mpnn_bf16;           /* 1: weights rounded to BF16, 0: FP32, for mpnn_weights (1) */
    int32_t smooth_levels;       /* smoothed prolongator (Sec. 3.1, "Variants") on the first
                                    smooth_levels levels (-1 = every level, 0 = none):
                                    P_bar = (I - diag(theta) D^-1 K) P, D the l1 diagonal, and the
                                    coarse matrix P_bar^T K P_bar; needs amg_pcg_solve /
                                    amg_vcycle_apply (not the multi-system solves or the damping
                                    network's training) (0) */
    double smooth_omega;         /* theta of the smoothed levels; 4/3 is the classical 4 / (3 rho(D^-1 K))
                                    with rho <= 1 from the l1 diagonal (1.3333333333333333) */
    const double* smooth_theta;  /* NULL, or a per-row theta for level 0 (DEVICE pointer, n doubles,
                                    read during amg_setup only) (NULL) */
    int32_t cheb_degree;         /* 0: nu_pre / nu_post l1-Jacobi sweeps; k >= 1: the 4th-kind Chebyshev
                                    acceleration of l1-Jacobi of degree k before and after the coarse
                                    correction on every level (Sec. 3.2 / Sec. 5; rho(D^-1 K) <= 1 from
                                    the l1 diagonal, no spectral estimate; d[0] = (4/3) D^-1 r[0],
                                    d[i] = (2i-1)/(2i+3) d[i-1] + (8i+4)/(2i+3) D^-1 r[i]); matrix passes
                                    on CSR row groups; needs amg_pcg_solve / amg_vcycle_apply and no
                                    damping network (0) */
    int32_t coarse_solver;       /* coarsest level: 0 = exact solve with the dense inverse; 1 = CG
                                    preconditioned by Jacobi (z = r / k_ii) from zero, to coarse_tol or
                                    coarse_maxit iterations (Sec. 5), a variable preconditioner: use it
                                    with flexible = 1 (0) */
    double coarse_tol;           /* coarse CG: stop once ||r|| <= coarse_tol ||f|| (0.0001) */
    int32_t coarse_maxit;        /* coarse CG: at most this many iterations (30) */
    int32_t autotune;            /* 1: at setup, time the finest level's q = K p pass in each available
                                    layout (sliced slabs with every supported warps-per-block count in
                                    FP64, the staged slabs in mixed precision, CSR row groups) and keep
                                    the fastest for all three passes; cached per process by the
                                    matrix shape, so later setups of that shape do not time (0) */
} amg_opts;

#define AMG_MAX_LEVELS 32

typedef struct {
    int32_t levels;
    int64_t n[AMG_MAX_LEVELS];
    int64_t nnz[AMG_MAX_LEVELS];
    double opc;          /* sum_l nnz_l / nnz_0, Eq. (OPC) */
    double setup_ms;     /* device time of the last amg_setup */
    double solve_ms;     /* device time of the last solve */
    int32_t iters;       /* iterations of the last solve */
    int32_t status;      /* status of the last solve */
    double final_relres; /* ||F - K u|| / ||F|| of the last solve, recomputed in FP64 */
    double vcycle_bytes; /* algorithmic bytes of one V-cycle */
    double iter_bytes;   /* algorithmic bytes of one CG iteration (incl. V-cycle) */
    int32_t match_rounds[AMG_MAX_LEVELS]; /* total matching rounds per level */
    /* setup time by phase (ms, stream-ordered events): [0] input copy and
     * checks, [1] l1 diagonals and test vector, [2] edge weights,
     * [3] matching rounds, [4] aggregation, [5] Galerkin products,
     * [6] composite maps and member lists, [7] coarsest inverse,
     * [8] precision copies and solve workspace, [9] learned damping at the
     * end of a setup with mpnn_weights (network on the coarse levels, wait for
     * the finest level's evaluation, install), [10] smoothed prolongators
     * and their Galerkin products (smooth_levels) */
    double setup_phase_ms[12];
    int32_t level_format[AMG_MAX_LEVELS]; /* 1 = run-encoded columns, 0 = plain CSR */
    int32_t staged_passes; /* finest-level passes: 0 = row-group kernels; mixed precision:
                              1 = staged slabs with a lane per run, 2 = staged sliced slabs with
                              a lane per row; FP64: 3 = sliced slabs with FP64 values, a warp per
                              slab and a lane per row (2 and 3 need matrix_format 2) */
    int64_t staged_slots;  /* value slots of the sliced slabs (padding included), 0 if unused */
    int32_t staged_buffers[2]; /* copy-ring buffers of the staged passes: [0] BF16 values, [1] FP32
                                  (0 for the FP64 sliced passes, which read values directly) */
    int32_t staged_window_bytes; /* largest per-block vector window of the staged passes */
    int32_t staged_level1; /* 1: level 1 also runs sliced staged passes (plain CSR, FP32 values) */
    double graph_build_ms; /* host time capturing and instantiating the iteration graph in the last
                              solve (0 when the hierarchy's graph was reused) */
    int32_t smoothed[AMG_MAX_LEVELS]; /* 1 where the level's prolongator is smoothed */
    int64_t p_nnz[AMG_MAX_LEVELS];    /* stored entries of each level's prolongator */
    int32_t sell64_warps;  /* warps per block of the FP64 sliced passes (0 when not in use) */
    double tune_ms;        /* host time the setup spent autotuning (0: not asked, or a cached choice) */
} amg_info;

typedef struct amg_hierarchy amg_hierarchy;

/* Fill *o with the defaults listed above.  Returns AMG_OK or AMG_ERR_ARG (o NULL). */
int amg_opts_default(amg_opts* o);

/* Build the AMG hierarchy of K on the GPU (Sec. 3, 3.1, 3.2):
 * l1 diagonal, test vector, edge weights, greedy-equivalent matching,
 * aggregation, Galerkin products, coarsest dense factorisation.
 * K: CSR as described at amg_csr (host or device).  opts: NULL = defaults.
 * cuda_stream: a cudaStream_t (NULL = default stream) used for all later
 * work on this hierarchy.  *out receives the library-owned hierarchy.
 * Errors: AMG_ERR_ARG (malformed CSR/options), AMG_ERR_NOT_SPD,
 * AMG_ERR_TIMEOUT, AMG_ERR_COARSE_TOO_LARGE, AMG_ERR_ROW_TOO_LONG,
 * AMG_ERR_NOMEM, AMG_ERR_CUDA; *out is NULL on error. */
int amg_setup(const amg_csr* K, const amg_opts* opts, void* cuda_stream, amg_hierarchy** out);

/* Solve K u = F by preconditioned CG (flexible CG if opts.flexible) with one
 * V-cycle as preconditioner, stopping when ||F - K u_k||_2 <= rtol ||F||_2
 * on the recursive residual or after itmax iterations.
 * F[n]: right-hand side; u[n]: initial guess in, solution out; both FP64,
 * host pointers if mem == AMG_MEM_HOST, device pointers if AMG_MEM_DEVICE.
 * iters, relres (may be NULL): iterations done, final ||F - K u|| / ||F||.
 * Errors: AMG_ERR_ARG, AMG_ERR_NOT_CONVERGED (u holds the last iterate),
 * AMG_ERR_BREAKDOWN, AMG_ERR_NAN, AMG_ERR_CUDA. */
int amg_pcg_solve(amg_hierarchy* h, const double* F, double* u, int32_t mem, double rtol, int32_t itmax,
                  int32_t* iters, double* relres);

/* Several right-hand sides of one matrix: nrhs (1..32) independent
 * (flexible) CG solves sharing the hierarchy, each with its own scalars and
 * convergence test; every matrix pass of an iteration reads the matrix once
 * for all right-hand sides (SpMM).  F and U are column-major n x nrhs with
 * leading dimension ld >= n (U: initial guesses in, solutions out), host or
 * device per `mem`.  iters[nrhs], relres[nrhs] (may be NULL) receive each
 * system's iteration count and final ||F - K u|| / ||F||.  Requires
 * nu_pre = nu_post = 1 and a hierarchy from amg_setup.  Returns AMG_OK when
 * every system converged, otherwise the first failure status (NaN first).
 * Errors as amg_pcg_solve. */
int amg_pcg_solve_multi(amg_hierarchy* h, int32_t nrhs, const double* F, double* U, int64_t ld, int32_t mem,
                        double rtol, int32_t itmax, int32_t* iters, double* relres);

/* A batch of independent systems K_k u_k = F_k (count <= 1024): the
 * matrices are assembled block-diagonally into one hierarchy (no entry
 * couples two systems, so every aggregate and coarse operator stays inside
 * one block and the V-cycle acts on each system separately).  Ks[count] as
 * in amg_setup (each CSR in its own 0-based numbering, host or device).
 * Errors as amg_setup. */
int amg_setup_batch(int32_t count, const amg_csr* Ks, const amg_opts* opts, void* cuda_stream,
                    amg_hierarchy** out);

/* Solve every system of a batch hierarchy with its own CG iteration in one
 * graph-captured loop; converged systems are frozen while others continue.
 * F[count], U[count]: per-system pointers (host or device per `mem`; U holds
 * initial guesses in, solutions out).  iters[count], relres[count] as in
 * amg_pcg_solve_multi.  Requires nu_pre = nu_post = 1. */
int amg_pcg_solve_batch(amg_hierarchy* h, const double* const* F, double* const* U, int32_t mem, double rtol,
                        int32_t itmax, int32_t* iters, double* relres);

/* Apply one V-cycle z = B r (device pointers, n = rows of level 0).  Used by
 * the parity tests and by callers with their own Krylov method. */
int amg_vcycle_apply(amg_hierarchy* h, const double* r_dev, double* z_dev);

/* y = K_l x on level l (device pointers). */
int amg_level_spmv(amg_hierarchy* h, int32_t level, const double* x_dev, double* y_dev);

/* Statistics of the hierarchy and of the last solve. */
int amg_get_info(const amg_hierarchy* h, amg_info* info);

/* Copy level data to host buffers (any pointer may be NULL):
 * K_l as CSR (rowptr[n+1], col[nnz], val[nnz]); dl1[n], w[n] (test vector);
 * agg[n], pval[n]: composite map to level l+1 (not for the coarsest). */
int amg_export_level(const amg_hierarchy* h, int32_t level, int64_t* rowptr, int32_t* col, double* val,
                     double* dl1, double* w, int32_t* agg, double* pval);

/* Level l's prolongator to level l+1 on the host: the smoothed P_bar where
 * the level is smoothed (amg_opts.smooth_levels), else the tentative P (one
 * entry per row).  *nnz (required) receives its stored entries; rowptr[n_l +
 * 1], col[nnz], val[nnz] (any may be NULL) its CSR, columns ascending.
 * AMG_ERR_ARG for a bad level (the coarsest has none). */
int amg_export_prolongator(const amg_hierarchy* h, int32_t level, int64_t* nnz, int64_t* rowptr, int32_t* col,
                           double* val);

/* The coarsest level's dense factorisation on the host: *n (required)
 * receives its size n_L; L[n_L^2] (may be NULL) the Cholesky factor,
 * row-major with zeros above the diagonal (l_jj = sqrt(a_jj - sum_k<j
 * l_jk^2), l_ij = (a_ij - sum_k<j l_ik l_jk) / l_jj, k ascending, each product
 * and difference rounded once); Ainv[n_L^2] (may be NULL) the inverse the
 * V-cycle applies, row-major (column c = L^-T L^-1 e_c by forward and
 * backward substitution).  AMG_ERR_ARG without a hierarchy. */
int amg_export_coarse(const amg_hierarchy* h, int32_t* n, double* L, double* Ainv);

/* Copy matching pass s of level l to host buffers: mate[n_s] (partner or
 * -1 for a singleton), agg[n_s], pval[n_s]; *n_s = rows the pass matched. */
int amg_export_pass(const amg_hierarchy* h, int32_t level, int32_t pass, int64_t* n_s, int32_t* mate, int32_t* agg,
                    double* pval);

/* Number of CUDA kernels this library has launched in this process (graph
 * launches count every kernel node).  Never fails. */
int64_t amg_kernel_launches(void);

/* Opt-in kernel timing (enable = 1 / 0).  While enabled, amg_pcg_solve
 * records CUDA events, on the stream the kernels run on, around the three
 * finest-level matrix passes of every CG iteration: [0] q = K p,
 * [1] down-sweep residual r = f - K x, [2] up-sweep smoothing.  Resets the
 * accumulated times. */
int amg_profile_kernels(amg_hierarchy* h, int32_t enable);

/* Accumulated timing of those kernels: ms[3] total milliseconds, count[3]
 * launches that did full work, bytes[3] algorithmic bytes of one launch
 * (values and column indices once, row pointers once, each vector read or
 * written once).  Any pointer may be NULL. */
int amg_kernel_times(const amg_hierarchy* h, double* ms, int64_t* count, double* bytes);

/* FP64 FMA throughput probe (measurement support; no paper counterpart):
 * enqueues on cuda_stream (NULL = default stream) one kernel of `blocks`
 * blocks, each thread running independent FMA chains x <- x a + b for
 * trips x 16 steps, and returns at once (time it with events on the same
 * stream).  `variant` picks the chain count, whether the chains share their
 * operands and the block size (*threads, host, receives it): the rate
 * depends on these beyond the FMA count, so a caller times every variant
 * and keeps the fastest.  variant = -1 writes the number of variants to
 * *threads; blocks = 0 only writes the variant's block size.  out_dev:
 * DEVICE array of blocks x *threads doubles that receives the chains' sums
 * (keeps the work observable).  *flops (host, may be NULL): the kernel's
 * floating-point operations, 2 per FMA.  Used to measure the FP64 rate that
 * bounds the FP64 matrix passes.  Errors: AMG_ERR_ARG (bad variant, blocks <
 * 0, trips < 1, out_dev NULL), AMG_ERR_CUDA. */
int amg_dfma_probe(int32_t variant, int32_t blocks, int64_t trips, double* out_dev, void* cuda_stream,
                   int32_t* threads, double* flops);

/* Check of the correctly rounded FP64 division the setup uses for the edge
 * weights c_ij (Sec. 3.1, Eq. of the edge weights): q_dev[i] = a_dev[i] /
 * b_dev[i] rounded to nearest even, for i < n, and *fast_count_dev (DEVICE,
 * added to, not cleared) += the number of quotients the division's fast path
 * accepted (a reciprocal estimate, one Newton-Raphson step, a residual
 * correction and an exact residual test; the rest go to the compiler's
 * division).  All arrays are DEVICE memory of n doubles; the work is
 * enqueued on cuda_stream (NULL = default stream) and the call returns at
 * once.  Used by the tests to hold the division to IEEE results.  Errors:
 * AMG_ERR_ARG (n < 0, a NULL array with n > 0), AMG_ERR_CUDA. */
int amg_div_check(int64_t n, const double* a_dev, const double* b_dev, double* q_dev, uint64_t* fast_count_dev,
                  void* cuda_stream);

/* Largest system amg_relres_noalloc accepts (rows). */
#define AMG_NOALLOC_MAX_ROWS (1 << 19)

/* ||F - K u||_2 / ||F||_2 for a device-resident CSR matrix K (K->mem must be
 * AMG_MEM_DEVICE) and device vectors F[n], u[n]; the result is written to
 * the host double *relres (0 when F = 0).  The work is enqueued on
 * cuda_stream (NULL = default stream) and the call returns after it.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory -- e.g. an application whose own pool
 * allocator reserved the GPU's memory up front and forbids allocations
 * outside it, or a time-critical loop where a cudaMalloc (and the device
 * synchronisation it may cause) is not acceptable.  It allocates nothing:
 * its reduction scratch is a fixed static device array of about 1 MB that
 * every GPU which loads the library keeps until the process exits.
 * The work runs on the device that owns cuda_stream (the current device
 * for NULL); the call makes that device current while it works and restores
 * the caller's current device.  The first call on a device looks up that
 * array's device address (with the device current) and caches it; make that
 * first call before any stream capture.  All calls share the array, so calls
 * that overlap on the GPU (e.g. on different streams) race; serialise them.
 * Launch failures are taken from this call's own launches: an unrelated
 * error the caller left pending is neither reported nor cleared.
 * Errors: AMG_ERR_ARG for NULL pointers, host-resident K, n < 1 or
 * n > AMG_NOALLOC_MAX_ROWS; AMG_ERR_CUDA on a CUDA failure. */
int amg_relres_noalloc(const amg_csr* K, const double* F, const double* u, double* relres, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Learned per-row smoother damping.  The paper has no learned component;
 * this extends its l1-Jacobi smoother (Sec. 3.2, x <- x + D^-1 (f - K x))
 * to x <- x + diag(omega_i / d_i) (f - K x) with 0 < omega_i < omega_max.
 * The smoother is a K-norm contraction (and the V-cycle SPD) while
 * 2 diag(d / omega) - K is positive definite, i.e. for every omega_i below
 * 2 / lambda_max(D^-1 K); the l1 diagonal gives lambda_max <= 1, so (0, 2)
 * is always admissible.  Per level, omega_max = 2 / lam_hat with lam_hat =
 * min(1, the Lanczos upper estimate of amg_smoother_bound).  omega comes
 * from a two-layer message-passing network (hidden width AMG_MPNN_HIDDEN)
 * evaluated on every level's matrix graph:
 *   x_i  = [sum_{j!=i}|k_ij|/k_ii, sum_{j!=i} k_ij/k_ii, log2(nnz_i)/8, 1]
 *   a_ij = k_ij / sqrt(k_ii k_jj) (j != i)
 *   h0 = relu(W0 x + b0); h_l = relu(U_l (A' h_{l-1}) + V_l h_{l-1} + b_l),
 *   l = 1, 2; omega = omega_max sigmoid(q . h2 + c).
 * A second head gives the per-row weight of the smoothed prolongator of
 * level 0 (Sec. 3.1, "Variants", with a per-row weight):
 *   theta = omega_max sigmoid(qt . h2 + ct),
 *   P_bar = (I - diag(theta) D^-1 K) P,
 * used by a setup given the weights with amg_opts.smooth_levels != 0.
 * Weights: AMG_MPNN_NPARAM floats, row-major blocks in the order
 * W0[32][4], b0[32], U1[32][32], V1[32][32], b1[32], U2, V2, b2, q[32], c[1],
 * qt[32], ct[1].
 * All weight, gradient and moment pointers are DEVICE pointers owned by the
 * caller.  The network buffers (about 10 floats x 32 per row of every level
 * plus one float per stored entry) are allocated on first use and kept
 * with the hierarchy.  The calls order themselves after the caller's
 * stream and return when their work is done.
 * ------------------------------------------------------------------------ */
#define AMG_MPNN_HIDDEN 32
#define AMG_MPNN_NPARAM 4386

/* Evaluate the network with weights w (weights rounded to BF16 when
 * bf16_weights = 1, FP32 when 0; FP32 arithmetic) on every level that has a
 * smoother and install omega / d as its smoother diagonal (FP64 and, in
 * the mixed-precision modes, FP32).  w = NULL restores the plain 1 / d
 * bit for bit.  Later solves, V-cycles and multi-system solves use the
 * installed diagonal.  Errors: AMG_ERR_ARG (h NULL, bf16_weights not 0/1),
 * AMG_ERR_NOMEM, AMG_ERR_CUDA. */
int amg_mpnn_apply(amg_hierarchy* h, const float* w, int32_t bf16_weights);

/* Copy the omega of the last network evaluation (amg_mpnn_apply or
 * amg_mpnn_loss_grad) on `level` to the device array omega[n_level].
 * AMG_ERR_ARG if there was none or the level has no smoother. */
int amg_mpnn_omega(amg_hierarchy* h, int32_t level, float* omega);

/* Training objective and its gradient for weights w (FP32 network):
 *   loss = (1/m) sum_k log(y_k^T K y_k / x_k^T K x_k), y_k = x_k - B K x_k,
 * B the V-cycle with the network's damping (one pre- and one post-sweep,
 * exact coarsest solve), probe k entry i = 2 U - 1 with U the (k n + i)-th
 * SplitMix64(seed) draw scaled to [0, 1) on 53 bits, m = nprobe.
 * *loss (host) receives the loss, grad[AMG_MPNN_NPARAM] (device, FP64) the
 * gradient (reverse mode through the V-cycle in FP64 and through the
 * network in FP32; deterministic).  Does not change the installed damping.
 * Errors: AMG_ERR_ARG (NULL pointers, nprobe < 1, a single-level
 * hierarchy), AMG_ERR_BREAKDOWN (a non-positive energy, e.g. from a
 * diverging network), AMG_ERR_NAN, AMG_ERR_NOMEM, AMG_ERR_CUDA. */
int amg_mpnn_loss_grad(amg_hierarchy* h, const float* w, int32_t nprobe, uint64_t seed, double* loss,
                       double* grad);

/* Training objective of the smoothing weights theta (the network's second
 * head) and its gradient, on a two-level hierarchy whose level-0
 * prolongator is smoothed (amg_setup with smooth_levels = 1 and
 * max_levels = 2):
 *   loss = (1/m) sum_k log(y_k^T K y_k / x_k^T K x_k),
 *   y_k = (I - M K)(I - P_bar K_c^-1 P_bar^T K)(I - M K) x_k,
 * the two-grid error propagator with the exact coarse solve, K_c =
 * P_bar^T K P_bar, M = diag(omega / d) with the network's omega held fixed
 * (its gradient flows through theta only), probes as in amg_mpnn_loss_grad.
 * The network's theta is installed into h (P_bar, the coarse matrix and its
 * dense inverse are rewritten).  grad[AMG_MPNN_NPARAM] (device, FP64) and
 * *loss (host) as in amg_mpnn_loss_grad.  amg_mpnn_train uses this loss for
 * every such hierarchy it is given.  Errors: AMG_ERR_ARG (NULL pointers,
 * nprobe < 1, another hierarchy shape), AMG_ERR_BREAKDOWN (a non-positive
 * energy or coarse matrix), AMG_ERR_NAN, AMG_ERR_NOMEM, AMG_ERR_CUDA. */
int amg_mpnn_theta_loss_grad(amg_hierarchy* h, const float* w, int32_t nprobe, uint64_t seed, double* loss,
                             double* grad);

/* Copy the level-0 theta of the last network evaluation (second head) to
 * the device array theta[n_0].  AMG_ERR_ARG if there was none. */
int amg_mpnn_theta(amg_hierarchy* h, float* theta);

/* One Adam step (Kingma and Ba 2015) on w with gradient grad (FP64) and
 * moments m, v (FP32, zero before the first step); t counts steps from 1.
 * AMG_ERR_ARG on NULL pointers or parameters out of range. */
int amg_mpnn_adam(amg_hierarchy* h, float* w, const double* grad, float* m, float* v, int32_t t, float lr,
                  float beta1, float beta2, float eps);

/* `steps` Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the
 * mean over the `count` hierarchies hs[0..count) (1 <= count <= 64, all on
 * the current device) of the loss of amg_mpnn_loss_grad (of
 * amg_mpnn_theta_loss_grad for a two-level hierarchy with a smoothed level
 * 0; other smoothed hierarchies: AMG_ERR_ARG), with probe seed
 * seed + step; w (device) is updated in place; loss_hist (host, optional)
 * receives each step's mean loss before its update.  The Adam moments live
 * with hs[0].  Errors as amg_mpnn_loss_grad. */
int amg_mpnn_train(amg_hierarchy* const* hs, int32_t count, float* w, int32_t steps, int32_t nprobe, uint64_t seed,
                   float lr, double* loss_hist);

/* Fallback rule: solve K u = F (F device, u0 = 0) with the reference
 * damping -- the constant omega_ref on every smoothed level (omega_ref = 1:
 * the plain l1-Jacobi smoother) -- and with the network's damping (BF16
 * weights); keep the learned damping installed only if it converged in no
 * more iterations than the reference, else install the reference damping
 * (also on every error return after the reference solve).  *used = 1 if the
 * learned damping stays; the two iteration counts are returned.  Not for
 * batch hierarchies.  Errors: AMG_ERR_ARG (NULL pointers, omega_ref <= 0,
 * rtol <= 0, itmax < 1, a batch hierarchy), AMG_ERR_NOMEM, AMG_ERR_CUDA. */
int amg_mpnn_select(amg_hierarchy* h, const float* w, double omega_ref, const double* F, double rtol, int32_t itmax,
                    int32_t* used, int32_t* iters_ref, int32_t* iters_learned);

/* Install the constant damping x <- x + (omega / d_i) (f - K x) on every
 * level that has a smoother (FP64 and, in the mixed-precision modes, FP32
 * diagonals); omega = 1 restores the plain l1-Jacobi smoother of Sec. 3.2
 * bit for bit.  omega must be positive; the smoother converges for omega <
 * 2 / lambda_max(D^-1 K) (at least 2, see amg_smoother_bound).  The paper
 * has no damping parameter; this is the constant baseline of the learned
 * damping.  Errors: AMG_ERR_ARG (h NULL, omega not > 0 or not finite),
 * AMG_ERR_CUDA. */
int amg_set_damping(amg_hierarchy* h, double omega);

/* lam_hat of `level` on the host: min(1, theta + beta_k |s_k|), theta the
 * largest Ritz value of 15 Lanczos steps (fewer on levels with fewer rows)
 * on D^-1/2 K D^-1/2 (spectrum of D^-1 K, D the l1 diagonal of Sec. 3.2)
 * from a SplitMix64(0x4C414E43 + level) start vector, beta_k |s_k| its
 * residual bound.  An upper estimate of lambda_max(D^-1 K) that caps the
 * learned damping at omega_max = 2 / lam_hat.  Computed once per level and
 * kept with the hierarchy.  Errors: AMG_ERR_ARG (h or lambda_hat NULL, level
 * out of range), AMG_ERR_NOMEM, AMG_ERR_CUDA. */
int amg_smoother_bound(amg_hierarchy* h, int32_t level, double* lambda_hat);

/* Release the hierarchy and its device memory. */
int amg_free(amg_hierarchy* h);

/* Static description of a status code. */
const char* amg_strerror(int code);

/* ------------------------------------------------------------ IgA assembly
 * Stiffness matrix K and load vector F of -div(kappa grad u) = f on one
 * tensor-product B-spline patch (Sec. 2.2, single-patch discretization):
 *   k_ij = int kappa(F(xi)) (grad_xi N_j)^T J^-1 J^-T (grad_xi N_i) |det J| dxi,
 *   f_i  = int f(F(xi)) N_i |det J| dxi
 * over the parametric cube [0,1]^3, J = dF/dxi, N_i the tensor products of
 * the degree-p B-splines on the open uniform knot vector with n elements per
 * direction (Sec. 2.1), nq Gauss points per element and direction.  The
 * discrete space is the B-spline space on the parametric cube for both
 * geometries (non-isoparametric for the annulus, Sec. 2.4).  Computed on
 * the GPU by sum factorization: the 3-D quadrature sums are contracted one
 * direction at a time with 1-D tables of products of B-spline values and
 * derivatives, the tensor-product alternative to the element loop that
 * Sec. 2.2 points to.  FP64; agrees with an element loop to rounding. */
#define AMG_GEOM_CUBE 0     /* F(xi) = xi */
#define AMG_GEOM_ANNULUS 1  /* quarter annulus of radii 1 and 2 extruded over z in [0,1]: (1 + xi1) c(xi2) + xi3 e_z, c the quadratic NURBS arc through (1,0), (1,1), (0,1) with weights 1, sqrt(2)/2, 1 */
#define AMG_SRC_ONE 0       /* f = 1 */
#define AMG_SRC_SINE 1      /* f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) */

typedef struct {
    int32_t n;                 /* elements per direction, >= 1 */
    int32_t p;                 /* B-spline degree, 1..8 */
    int32_t nq;                /* Gauss points per element and direction, 1..16; 0 = p + 1; n nq <= 768 */
    int32_t geometry;          /* AMG_GEOM_CUBE or AMG_GEOM_ANNULUS */
    int32_t with_boundary;     /* 0: the functions nonzero on the boundary are eliminated (homogeneous Dirichlet data), m = n + p - 2 unknowns per direction; 1: all, m = n + p */
    int32_t source;            /* AMG_SRC_ONE or AMG_SRC_SINE */
    int32_t kappa_m;           /* random Fourier features of kappa; 0: kappa = 1 */
    double kappa_sigma;        /* kappa = exp(sigma sqrt(2/M) sum_m cos(omega_m . x + phi_m)) */
    const double* kappa_omega; /* device, kappa_m x 3 frequencies, row-major */
    const double* kappa_phi;   /* device, kappa_m phases */
} amg_iga_patch;

/* Size of the system of patch P: *n = m^3 unknowns (numbered i1 + m (i2 +
 * m i3)), *nnz = stored entries of K (row I couples to every J with
 * |i_k - j_k| <= p per direction).  Host only.  AMG_OK or AMG_ERR_ARG. */
int amg_iga_size(const amg_iga_patch* P, int64_t* n, int64_t* nnz);

/* Assembles K (CSR: rowptr[n+1] int64, col[nnz] int32 ascending per row,
 * val[nnz]) and, when F is not NULL, F[n] -- all device arrays of the sizes
 * amg_iga_size gives, owned by the caller -- on cuda_stream (NULL = legacy
 * default stream) of the current device; returns after the work finished.
 * Device workspace is taken from the library's stream-ordered pool and
 * released before the return: at its peak 8 (4 R Q^2 + 4 R^2 Q) bytes with
 * Q = n nq and R = (2p+1) m (2.7 GB for n = 64, p = 3; 8.9 GB for n = 96),
 * plus 8 Q^2 (2M rounded up to 16) for kappa.  *flops (may be NULL) receives the
 * floating-point operations of the quadrature sums (2 per multiply-add).
 * Returns AMG_OK, AMG_ERR_ARG, AMG_ERR_NOMEM or AMG_ERR_CUDA. */
int amg_iga_assemble(const amg_iga_patch* P, int64_t* rowptr, int32_t* col, double* val, double* F,
                     void* cuda_stream, double* flops);

/* Self-test of the bounded waits of the staged passes (the mbarrier waits of
 * the bulk-copy pipelines, which on expiry end the kernel with
 * AMG_ERR_TIMEOUT instead of hanging).  Runs one thread on the current
 * device that waits, with a limit of limit_ms (0 < limit_ms <= 1000), on an
 * mbarrier that nothing completes and then on one whose phase it completed
 * itself.  *timed_out = 1 when the first wait gave up; *completed = 1 when
 * the second returned.  Synchronous; returns AMG_OK, AMG_ERR_ARG,
 * AMG_ERR_NOMEM or AMG_ERR_CUDA.  No GPU fault or hang is involved: the
 * waits are bounded. */
int amg_staged_wait_selftest(double limit_ms, int32_t* timed_out, int32_t* completed);

/* Text of the last CUDA runtime error seen by this thread ("" if none). */
const char* amg_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMG_GB300_H */
