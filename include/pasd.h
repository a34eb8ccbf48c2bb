/*
 * pasd.h - C ABI of the GB300 (sm_103a) PASD solver for tensor robust PCA.
 *
 * The method is Parallel Active Subspace Decomposition (Jiang & Ng, arXiv
 * 1712.09999): split an observed N-way tensor T into a low-rank part X and a
 * sparse part E (Eq. 1), by running the ADMM of Algorithm 1 on the
 * reformulation of Eq. 3, in which every mode-n unfolding of the low-rank part
 * is U_n V_n with U_n an I_n x R_n column-orthonormal "active subspace" and V_n
 * a small R_n x prod_{m!=n} I_m factor.
 *
 * Conventions shared by every entry point
 *  - Tensors are dense float32 in C order (the last index is contiguous),
 *    D = prod_n I_n elements, addressed by plain device pointers that the
 *    caller owns. Unless an entry point says otherwise, pointers are DEVICE
 *    pointers on the device the context was created for.
 *  - Streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 *    default stream). Work is enqueued on that stream; entry points that say
 *    "synchronous" also wait for it.
 *  - Every entry point returns a pasd_status; nothing throws across the ABI.
 *    On failure a human-readable reason is available from pasd_last_error()
 *    (thread-local, valid until the next call on the same thread).
 *  - The library owns all solver state (U_n, V_n in factored form, E, the
 *    multipliers, workspaces); the caller owns T, L and E.
 */
#ifndef PASD_H
#define PASD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PASD_OK = 0,               /* converged (stop rule met)                          */
    PASD_PENDING = 1,          /* served solve still running (pasd_poll only)        */
    PASD_NOT_CONVERGED = 2,    /* max_iter loop bodies ran without meeting the rule  */
    PASD_ERR_INVALID_ARG = -1, /* bad parameters, shapes or pointers                 */
    PASD_ERR_OOM = -2,         /* device allocation failed or HBM budget exceeded    */
    PASD_ERR_CUDA = -3,        /* a CUDA runtime call failed                         */
    PASD_ERR_NONFINITE = -4,   /* a NaN/Inf appeared in the iterate                  */
    PASD_ERR_TIMEOUT = -5,     /* a bounded wait ran out                             */
    PASD_ERR_BUSY = -6,        /* the submit queue is full                           */
    PASD_ERR_UNKNOWN_TICKET = -7,
    PASD_ERR_UNSUPPORTED = -8  /* shape/rank outside the built kernels' limits       */
} pasd_status;

typedef enum {
    PASD_PREC_FP32 = 0,   /* FP32 storage and arithmetic on the hot path            */
    PASD_PREC_MIXED = 1   /* the V-step product U_n^T G_n (Eq. 13) on the tensor
                             cores (tcgen05, TF32 operands split hi + lo, FP32
                             accumulation); everything else as PASD_PREC_FP32.
                             Contract: L and E within 1e-3 of the FP64 result
                             (measured: about 2x the FP32 path's deviation)     */
} pasd_precision;

typedef enum {
    PASD_STOP_INF_ABS = 0,     /* Algorithm 1: max_n ||T - Z_n - E||_inf < tol        */
    PASD_STOP_FRO_REL = 1,     /* max_n ||T - Z_n - E||_F / ||T||_F < tol             */
    PASD_STOP_FIXED_ITERS = 2  /* run exactly max_iter loop bodies                    */
} pasd_stop;

#define PASD_MAX_ORDER 8
#define PASD_MAX_RANK 64

/* Problem statement (Eq. 1 / Eq. 3 and the inputs of Algorithm 1).
 * A zero in an optional field selects the paper's default. */
typedef struct {
    int32_t order;                        /* N >= 2                                    */
    int64_t dims[PASD_MAX_ORDER];         /* I_1..I_N (C order)                        */
    int32_t rank_bound[PASD_MAX_ORDER];   /* R_n, 1 <= R_n <= min(I_n, PASD_MAX_RANK)   */
    double alpha[PASD_MAX_ORDER];         /* output weights alpha_n: all finite and > 0,
                                             or all 0 for the default 1/N (a mix of
                                             zero and nonzero entries is INVALID_ARG)  */
    double lambda;                        /* > 0: lambda_n = alpha_n / lambda          */
    double lambda_n[PASD_MAX_ORDER];      /* used when lambda <= 0: per-mode nuclear
                                             weights, finite and >= 0;
                                             0 -> sqrt(max(I_n, D/I_n)) / N            */
    double mu0;                           /* 0 -> 1e-4                                  */
    double mu_max;                        /* 0 -> 1e10                                  */
    double rho;                           /* 0 -> 1.1 (must be > 1)                     */
    double tol;                           /* 0 -> 1e-5                                  */
    int32_t stop_rule;                    /* pasd_stop                                  */
    int32_t max_iter;                     /* 0 -> 1000                                  */
    int32_t precision;                    /* pasd_precision                             */
    int32_t check_every;                  /* loop bodies between host reads of the
                                             device stop flag; 0 -> 8                  */
    uint32_t flags;                       /* PASD_F_* bits                              */
} pasd_params;

/* Skip the idle start. While V_n = 0 and E = 0 a loop body of Algorithm 1 only
 * rescales the multipliers (G_n = T - E + Y_n/mu becomes g T), and it stays so
 * while g sigma_max(U_n^T T_(n)) <= lambda_n/mu for every n and g max|T| <=
 * 1/(N mu). After the first body the solver evaluates these conditions from
 * that body's singular values and residual and replaces the idle bodies that
 * follow (all but the last) by their closed form: the same iterate, the same
 * trace records (kept 0), counted in `iters` and reported in `skipped`. */
#define PASD_F_SKIP_IDLE 1u

/* FP64 eigen-solves. The R_n x R_n symmetric eigen-problems of each loop body
 * (the Gram matrix A_n A_n^T of the SVT after Eq. 13, and M^T M of the U-step's
 * polar factor, Eq. 10) are solved in double: cyclic Jacobi with correctly
 * rounded rotations to a relative threshold of 1e-13, and the inverse square
 * roots of the U-step formed in double, each rounded to float once. The Gram
 * matrices themselves and every I_n x R_n product stay FP32. Rank bounds up to
 * 56 (UNSUPPORTED above: the double workspace must fit shared memory). The
 * default keeps these solves in FP32 (relative Jacobi threshold 1e-6). */
#define PASD_F_FP64_EIG 2u

typedef struct {
    int32_t status;                       /* pasd_status of the solve                  */
    int32_t iters;                        /* completed loop bodies                     */
    double res_inf;                       /* max_n ||T - Z_n - E||_inf at exit         */
    double res_fro_rel;                   /* max_n ||T - Z_n - E||_F / ||T||_F         */
    double objective;                     /* sum_n lambda_n ||V_n||_* + ||E||_1 (Eq. 3)*/
    double nuclear[PASD_MAX_ORDER];       /* ||V_n||_*                                 */
    double l1_E;                          /* ||E||_1                                    */
    double mu_final;                      /* mu after the last loop body               */
    int32_t kept[PASD_MAX_ORDER];         /* singular values kept by the last SVT      */
    double latency_s;                     /* served solves: submit -> retire, seconds  */
    int32_t skipped;                      /* loop bodies replaced by the idle-start
                                             closed form (PASD_F_SKIP_IDLE), included
                                             in iters                                  */
    int32_t batched;                      /* served solves: 1 if it advanced in the
                                             batched executor, 0 on a stream of its own */
} pasd_result;

typedef struct pasd_ctx pasd_ctx;
typedef struct pasd_plan pasd_plan_t;

/* Context on one CUDA device. `hbm_budget_bytes` bounds the summed footprint
 * of the solver state the served path keeps resident (0 -> 90% of free HBM).
 * Creates the served-path scheduler thread lazily on the first pasd_submit.
 * The submit queue holds at most 4096 solves that wait for admission; the
 * environment variable PASD_MAX_QUEUE (an integer >= 1, read here) sets
 * another bound. */
pasd_status pasd_ctx_create(int device, size_t hbm_budget_bytes, pasd_ctx** out);
/* Waits for the served solves still queued or in flight, then frees the
 * context. Plans made with a context must be destroyed before it (or never):
 * pasd_plan_destroy reads the plan's context. */
pasd_status pasd_ctx_destroy(pasd_ctx* ctx);

/* Fills `p` with the paper's defaults (Algorithm 1 initialisation and the
 * Sec. 5.1 settings: mu0 = 1e-4, mu_max = 1e10, rho = 1.1, tol = 1e-5,
 * max_iter = 1000, lambda_n = sqrt(max(I_n, prod_{m!=n} I_m)) / N, alpha_n = 1/N)
 * for a tensor of `order` modes with sizes `dims` and rank bounds `ranks`. */
pasd_status pasd_params_default(pasd_params* p, int32_t order, const int64_t* dims,
                                const int32_t* ranks);

/* Validates the problem and lays out the solver state for it. Allocates no
 * device memory (that happens on first use); `footprint_bytes` (may be NULL)
 * receives the device bytes the state will take. Errors: INVALID_ARG when
 * N < 2, any R_n > I_n (the Stiefel set St(I_n, R_n) is empty) or R_n < 1,
 * a weight that is negative, not finite or (for alpha) zero beside nonzero
 * ones, rho <= 1 or mu_max < mu0; UNSUPPORTED when R_n > PASD_MAX_RANK
 * or when I_n x (R_n rounded up to its rank bucket, plus 4) reaches 2^31.
 * Environment, read here (for comparisons and debugging; the same arithmetic up
 * to the grouping of partial sums): PASD_NO_TMA=1 plans the kernels fed by per-thread asynchronous
 * copies instead of bulk tensor copies; PASD_NO_GRAPH=1 launches each loop
 * body's kernels directly instead of replaying a captured CUDA graph;
 * PASD_NO_FEWROW=1 runs modes of at most 8 rows on the general streaming
 * products instead of their few-row kernels.
 * Test hook: PASD_TEST_WAIT_TIMEOUT=1 makes the plan's bulk-copy-fed
 * elementwise pass issue no copy at all and give up its wait after a few
 * thousand polls, so the first loop body ends the solve with PASD_ERR_TIMEOUT
 * (nothing is in flight when the kernels return; the context stays usable). */
pasd_status pasd_plan(pasd_ctx* ctx, const pasd_params* p, pasd_plan_t** out,
                      size_t* footprint_bytes);
pasd_status pasd_plan_destroy(pasd_plan_t* plan);

/* Algorithm 1 end to end, synchronous on `stream`: initialise, iterate until
 * the stop rule or max_iter, then write the output X = sum_n alpha_n Z_n /
 * sum_n alpha_n into L and the sparse part into E (both D floats, device).
 * L and E are written only when the result is PASD_OK or PASD_NOT_CONVERGED.
 * T must stay valid and unchanged until the call returns. */
pasd_status pasd_solve(pasd_plan_t* plan, const float* T, float* L, float* E,
                       pasd_result* result, void* stream);

/* Same as pasd_solve, but T, L and E are HOST buffers (D floats each); the
 * host<->device copies are part of the call. */
pasd_status pasd_solve_host(pasd_plan_t* plan, const float* T_host, float* L_host,
                            float* E_host, pasd_result* result, void* stream);

/* Served path (continuous batching). Queues one solve of `plan` on device
 * tensors T, L, E; the caller keeps them alive and untouched until pasd_poll
 * returns something other than PASD_PENDING. A solve is admitted when its
 * plan's footprint fits the context's HBM budget; admitted solves advance
 * together and retire as they converge. Solves on the bulk-copy kernels (orders
 * 2-4, last mode a multiple of 4 or padded to one) join a batch: each loop body
 * is one launch per kernel for all members (grouped by the kernels' template
 * parameters: rank bucket, tile threads, tensor order), replayed as one
 * captured CUDA graph per body that is rebuilt when solves join or leave at
 * chunk boundaries; kernels without a batched form (few-row modes, the
 * tensor-core A-pass of mixed precision) are launched per member inside that
 * body. Solves on the fallback kernels run each on a stream of its own.
 * Results are the same bit for bit either way. Knobs (read by pasd_ctx_create):
 * PASD_NO_BATCH=1 puts every served solve on its own stream; PASD_BATCHES
 * (1-16, default 4) batches run on streams of their own and a new solve joins
 * the smallest; PASD_BATCH_CHUNK (1-64, default 8) bodies per chunk. The solve's
 * stream is not ordered after any stream of the caller: T must be fully
 * written (its producing stream synchronised) before pasd_submit is called.
 * One plan serves one solve at a time (further submits of it wait in the
 * queue). While a served solve of a plan is queued or running, the plan belongs
 * to the served path: pasd_plan_destroy, pasd_solve, pasd_solve_host,
 * pasd_begin/iterate/finish, pasd_state_get and pasd_profile_iterations return
 * BUSY for it (and do nothing). It is the caller's again once the solve has
 * retired, at the latest when pasd_poll returns its final status. Errors: BUSY
 * when the queue is full. */
pasd_status pasd_submit(pasd_ctx* ctx, pasd_plan_t* plan, const float* T, float* L,
                        float* E, uint64_t* ticket);
/* PASD_PENDING while the solve is queued or running; otherwise its final
 * status, with `out` filled (out may be NULL). A ticket can be polled to
 * completion once; afterwards it is UNKNOWN_TICKET. */
pasd_status pasd_poll(pasd_ctx* ctx, uint64_t ticket, pasd_result* out);

/* Stepwise form of pasd_solve (asynchronous on `stream`):
 *   pasd_begin   - Algorithm 1 initialisation for observation T (device);
 *   pasd_iterate - enqueue `iters` loop bodies; bodies after the stop rule
 *                  holds are skipped on the device;
 *   pasd_finish  - write L and E (device) and fill `result` (synchronous).
 * The first pasd_begin on a plan (also inside pasd_solve and the served path)
 * allocates the plan's device memory and clears it; the clear is complete
 * before anything is enqueued on `stream`, whatever that stream is. */
pasd_status pasd_begin(pasd_plan_t* plan, const float* T, void* stream);
pasd_status pasd_iterate(pasd_plan_t* plan, int32_t iters, void* stream);
pasd_status pasd_finish(pasd_plan_t* plan, float* L, float* E, pasd_result* result,
                        void* stream);

/* Read-only export of solver state to HOST memory (synchronous on `stream`),
 * for inspection and testing. `mode` selects n for per-mode items.
 *   PASD_STATE_U      U_n                      I_n x R_n       float32 (row-major)
 *   PASD_STATE_A      U_n^T G_n (SVT argument)  R_n x P_n       float32, column order of
 *                     the unfolding = C order over the other modes
 *   PASD_STATE_W      eigenvectors of A_n A_n^T, columns by descending eigenvalue,
 *                                              R_n x R_n       float32
 *   PASD_STATE_SIGMA  singular values of A_n    R_n            float32, descending
 *   PASD_STATE_F      SVT factors max(1 - tau/sigma, 0)  R_n   float32
 *   PASD_STATE_E      E                        D              float32
 *   PASD_STATE_Y      multiplier Y_n           D              float32
 *   PASD_STATE_MU     mu (current)             1              float64
 *   PASD_STATE_KEPT   kept count per mode      N              int32
 *   PASD_STATE_TRACE  per-iteration records    iters x PASD_TRACE_STRIDE float64:
 *                     [k, res_inf, res_fro_rel, objective, mu_used, kept_1..kept_8]
 * V_n = W diag(F) W^T A_n and Z_n = fold_n(U_n V_n). `bytes` must equal the
 * item's size (TRACE: a multiple of the record size, at most iters records). */
enum {
    PASD_STATE_U = 0, PASD_STATE_A = 1, PASD_STATE_W = 2, PASD_STATE_SIGMA = 3,
    PASD_STATE_F = 4, PASD_STATE_E = 5, PASD_STATE_Y = 6, PASD_STATE_MU = 7,
    PASD_STATE_KEPT = 8, PASD_STATE_TRACE = 9
};
#define PASD_TRACE_STRIDE 13
pasd_status pasd_state_get(pasd_plan_t* plan, int32_t item, int32_t mode, void* dst_host,
                           size_t bytes, void* stream);

/* Number of kernel launches pasd_iterate enqueues per loop body. */
int32_t pasd_launches_per_iter(const pasd_plan_t* plan);

/* The plan's kernel configuration as a one-line JSON object written to `buf`
 * (`len` bytes, NUL-terminated; INVALID_ARG if it does not fit): the fused
 * pass's tile box per mode, regions, threads and resident CTAs per SM, the
 * M-pass's CTAs and waves, the modes on the few-row kernels, launches per body,
 * and the autotuner's state ("pending" before the first pasd_begin, then
 * "timed", "cached" or "off"). The paper has no counterpart (a
 * measurement aid). Tile autotuning: at the first pasd_begin of a plan the
 * library times the fused pass with 1, 2 and 3 resident CTAs per SM (each with
 * the largest tile that fits that share of shared memory, in an idle and an
 * active body), the M-pass with one and two waves of CTAs and the FP32 A-pass
 * with its default and half its default columns per thread, on the plan's own
 * buffers, and keeps a candidate only if it beats the planner's default by more
 * than 3%; the choice is cached per device and problem shape for the life of the
 * process, so plans of one shape share it (and their results agree bit for
 * bit). The choice changes only how partial sums are grouped, i.e. results in
 * their last bits. PASD_NO_TUNE=1 (read at that first pasd_begin) keeps the
 * planner's default. */
pasd_status pasd_plan_info(const pasd_plan_t* plan, char* buf, size_t len);

/* The mode-n product of the V-step (Eq. 13) as a standalone operation: for a
 * C-order float32 tensor X viewed as [pre][I][post] (the mode-n unfolding X_(n)
 * has I rows and pre*post columns, Sec. 2.1), computes
 *   A    = U^T X_(n)   stored as [pre][R][post]  (device, pre*R*post floats)
 *   gram = A A^T       R x R row-major           (device; may be NULL)
 * with U an I x R row-major device matrix. The unfolding is read in place.
 * R must be one of 4, 8, ..., 32, 40, 48, 56, 64 (pad U with zero columns for
 * other ranks); otherwise UNSUPPORTED. Scratch for the per-CTA Gram partial
 * sums (ceil(pre*post/256) * R * R floats) is allocated and freed inside the
 * call; the call is synchronous on `stream`. */
pasd_status pasd_mode_product(const float* X, int64_t pre, int64_t I, int64_t post, const float* U,
                              int32_t R, float* A, float* gram, void* stream);

/* Allocation-free variant of pasd_mode_product, for callers that cannot
 * allocate device memory where they need the product (a framework allocator
 * that must own every device byte, or a latency-critical loop in which
 * cudaMalloc/cudaFree would synchronise the device). The paper has no
 * counterpart; this is an interface convenience.
 * Same arguments, results and rank rule as pasd_mode_product, but the Gram
 * partial sums go to a fixed 4 MiB scratch array compiled into the library
 * (held on every device that loads the library until the process exits), so
 * the call allocates nothing and is asynchronous on `stream`. Limit:
 * ceil(pre*post/256) * R * R <= 1048576, else UNSUPPORTED (outputs untouched).
 * Every call looks up the scratch's device address on the current device (a
 * host-side lookup, no device work). The first call on a device, and the first
 * after a cudaDeviceReset of it, also clears the scratch's flags on `stream`,
 * waiting for that clear (so that call returns after it); make it before any
 * stream capture. All calls share the
 * scratch and it keeps the last call's contents: calls whose work overlaps on
 * the GPU race on it and must be serialised by the caller. */
pasd_status pasd_mode_product_noalloc(const float* X, int64_t pre, int64_t I, int64_t post,
                                      const float* U, int32_t R, float* A, float* gram,
                                      void* stream);

/* Kernel timing for measurement: runs `iters` loop bodies on `stream` as plain
 * launches (not the captured graph), brackets each kernel group with CUDA
 * events on that stream, synchronizes, and writes the summed milliseconds per
 * group into kernel_ms[0 .. PASD_PROFILE_SLOTS-1] in this order:
 *   0 polar (U-step), 1 A-pass (all modes), 2 SVT, 3 Vrot (small factor in the
 *   SVT eigenbasis), 4 fused elementwise pass, 5 M-pass (the next U-step's
 *   product G_n V_n^T), 6 finalize.
 * The solver state advances exactly as with pasd_iterate. */
#define PASD_PROFILE_SLOTS 7
pasd_status pasd_profile_iterations(pasd_plan_t* plan, int32_t iters, double* kernel_ms,
                                    void* stream);

const char* pasd_status_string(pasd_status s);
const char* pasd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PASD_H */
