// Host runtime behind include/pasd.h: contexts, plans (layout + lazy device
// arena), the per-iteration CUDA graph, the synchronous solve loop, the
// served path (continuous batching over per-solve streams) and state export.
#include "../../include/pasd.h"
#include "pasd_impl.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace pasd;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static pasd_status fail(pasd_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}
void pasd_set_error(const std::string& msg) { g_last_error = msg; }

namespace pasd {
// (kernel, device) -> the largest dynamic shared-memory size set so far
void set_smem_attr(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    int& cur = done[std::make_pair(kernel, dev)];
    if (bytes > cur && cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) == cudaSuccess)
        cur = bytes;
}
}  // namespace pasd
#define CUDA_TRY(call)                                                                   \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(e_ == cudaErrorMemoryAllocation ? PASD_ERR_OOM : PASD_ERR_CUDA,  \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

// ---------------------------------------------------------------------------
// structures
// ---------------------------------------------------------------------------
struct Job {
    uint64_t ticket;
    pasd_plan_t* plan;
    const float* T;
    float* L;
    float* E;
    std::chrono::steady_clock::time_point t_submit;
};

struct pasd_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    size_t smem_per_sm = 0;
    size_t hbm_budget = 0;
    // served path
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job> queue;
    std::map<uint64_t, pasd_result> done;
    std::map<uint64_t, int> state;   // 0 queued, 1 running
    std::thread worker;
    bool worker_started = false;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t max_queue = 4096;
    bool no_batch = false;    // PASD_NO_BATCH=1 at creation: every served solve on its own stream
    int n_batches = 4;        // batches of the served path (PASD_BATCHES, 1..16)
    int batch_chunk = 8;      // loop bodies between a batch's flag reads (PASD_BATCH_CHUNK, 1..64)
};

struct pasd_plan {
    pasd_ctx* ctx = nullptr;
    pasd_params p{};
    int N = 0;
    int64_t D = 0;
    ModeGeom m[PASD_MAXN];
    double lam[PASD_MAXN];
    double alpha[PASD_MAXN];
    FusedGeom fg{};          // geometry in use
    FusedGeom fg_plain{};    // single-buffer geometry (fallback when TMA is unavailable)
    bool want_tma = false;
    FusedTmaPlan* tma = nullptr;
    float* Tc = nullptr;     // plan-owned copy of the observation
    // The last mode is padded to a multiple of 4 (zeros) when that lets the TMA
    // kernels run (N <= 4): the padded entries stay exactly zero through every
    // step (T = 0 there gives E' = 0, Y' = 0, and U's padded rows stay zero), so the
    // result on the real entries is the unpadded one. D and the mode geometry are
    // the padded ones; D_real, I_real are the caller's.
    bool pad = false;
    int64_t D_real = 0;
    int64_t I_last_real = 0;
    float* Lpad = nullptr;   // output-pass target when padded
    int ncta_ap[PASD_MAXN];
    int n_mp[PASD_MAXN];
    size_t footprint = 0;
    // device arena
    char* arena = nullptr;
    DevScalars* sc = nullptr;
    DevScalars* tune_sc = nullptr;       // scalars the autotuner's timing launches read
    float *E = nullptr, *G[PASD_MAXN], *A[PASD_MAXN], *U[PASD_MAXN], *Urot[PASD_MAXN], *Vr[PASD_MAXN];
    float *W[PASD_MAXN], *F[PASD_MAXN], *sigma[PASD_MAXN];
    float *gram[PASD_MAXN], *mp[PASD_MAXN], *scratch[PASD_MAXN], *Mred[PASD_MAXN];
    float *part = nullptr, *sq_part = nullptr;
    int32_t* kept = nullptr;
    double* trace = nullptr;
    float* dev_io = nullptr;     // staging for pasd_solve_host: T, L, E
    float* y_tmp = nullptr;
    // launch descriptors
    SmallArgs small{};
    ApassArgs ap[PASD_MAXN];
    FusedArgs fu{};
    FinalizeArgs fin{};
    VrotArgs vr{};
    MpassArgs mpa{};
    size_t mp_smem = 0;
    bool mp_use_tma = false;
    MpassSmallArgs mp_small[PASD_MAXN];  // few-row modes' M-pass (fewrow.cu)
    int n_mp_big = 0;                    // modes on the shared M-pass launch
    MpassTmaArgs mpt{};
    size_t mpt_smem = 0;
    int mpt_slots = 0;                   // TMA M-pass CTAs resident at once
    int64_t mpt_tot = 0, mpt_work[PASD_MAXN];
    // autotuner candidates of the fused pass (k CTAs per SM) and its choices
    FusedGeom fcand[3];
    int fcand_k[3];
    int n_fcand = 0;
    int default_fused_k = 0;             // CTAs per SM of the planner's default geometry
    int tuned_fused_k = 0;               // CTAs per SM of the geometry in use
    int tuned_mp_waves = 1;
    int ap_tma_default_nc[PASD_MAXN];
    bool tuned = false;
    const char* tune_mode = "pending";   // pending (no pasd_begin yet), timed, cached, off
    MpassTmaPlan* mp_tma = nullptr;
    // A-pass: TMA plans (one per padded rank) and the modes on the cp.async kernel
    bool ap_small[PASD_MAXN];            // modes on the few-row kernel (apass_small.cu)
    int ap_small_grid[PASD_MAXN];
    bool ap_use_tma[PASD_MAXN];
    int ap_kind = APASS_FFMA;            // arithmetic of the TMA-fed A-pass (ApassKind)
    ApassTmaPlan* ap_tma[PASD_MAXN];
    int n_ap_tma = 0;
    ApassArgs ap_plain[PASD_MAXN];
    int n_ap_plain = 0;
    // graph
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = true;
    DevScalars* host_sc = nullptr;   // pinned mirror
    cudaStream_t own_stream = nullptr;   // served path
    cudaEvent_t ev = nullptr;
    bool busy = false;
    int served = 0;          // served solves queued or running (guarded by ctx->mu)
    int nparts_max = 0;                  // residual partials: room for every fused geometry
    int ap_launches = 1;
    int mp_launches = 1;
    int vr_launches = 1;
    // idle-start skip (PASD_F_SKIP_IDLE): armed by pasd_begin, run after the first body
    float* idle_g = nullptr;
    IdleSkipArgs idle{};
    bool skip_pending = false;
    // test hook (PASD_TEST_WAIT_TIMEOUT=1 at plan time): the fused pass issues no
    // bulk copy and waits a few thousand polls, so its bounded wait runs out
    bool test_wait_timeout = false;
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" pasd_status pasd_ctx_create(int device, size_t hbm_budget_bytes, pasd_ctx** out) {
    if (!out) return fail(PASD_ERR_INVALID_ARG, "out is NULL");
    int count = 0;
    CUDA_TRY(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count) return fail(PASD_ERR_INVALID_ARG, "no such device");
    CUDA_TRY(cudaSetDevice(device));
    pasd_ctx* c = new pasd_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete c; return fail(PASD_ERR_CUDA, cudaGetErrorString(e)); }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    c->smem_per_sm = prop.sharedMemPerMultiprocessor;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->hbm_budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
    if (const char* nb = std::getenv("PASD_NO_BATCH")) c->no_batch = nb[0] == '1';
    if (const char* q = std::getenv("PASD_BATCHES")) {
        const long v = std::strtol(q, nullptr, 10);
        if (v >= 1 && v <= 16) c->n_batches = (int)v;
    }
    if (const char* q = std::getenv("PASD_BATCH_CHUNK")) {
        const long v = std::strtol(q, nullptr, 10);
        if (v >= 1 && v <= 64) c->batch_chunk = (int)v;
    }
    if (const char* q = std::getenv("PASD_MAX_QUEUE")) {
        const long v = std::strtol(q, nullptr, 10);
        if (v >= 1) c->max_queue = (size_t)v;
    }
    *out = c;
    return PASD_OK;
}

static void worker_main(pasd_ctx* c);

extern "C" pasd_status pasd_ctx_destroy(pasd_ctx* c) {
    if (!c) return fail(PASD_ERR_INVALID_ARG, "ctx is NULL");
    {
        std::unique_lock<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv.notify_all();
    if (c->worker.joinable()) c->worker.join();
    delete c;
    return PASD_OK;
}

// ---------------------------------------------------------------------------
// params and plan
// ---------------------------------------------------------------------------
extern "C" pasd_status pasd_params_default(pasd_params* p, int32_t order, const int64_t* dims,
                                           const int32_t* ranks) {
    if (!p || !dims || !ranks) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    if (order < 2 || order > PASD_MAX_ORDER) return fail(PASD_ERR_INVALID_ARG, "order out of range");
    std::memset(p, 0, sizeof(*p));
    p->order = order;
    for (int n = 0; n < order; ++n) { p->dims[n] = dims[n]; p->rank_bound[n] = ranks[n]; }
    p->mu0 = 1e-4; p->mu_max = 1e10; p->rho = 1.1; p->tol = 1e-5; p->max_iter = 1000;
    p->stop_rule = PASD_STOP_INF_ABS; p->precision = PASD_PREC_FP32; p->check_every = 8;
    return PASD_OK;
}

static int rank_bucket(int R) {
    static const int b[] = {4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64};
    for (int v : b) if (R <= v) return v;
    return -1;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static MpassTmaArgs mpass_tma_layout(const pasd_plan_t* pl, int waves);

extern "C" pasd_status pasd_plan(pasd_ctx* c, const pasd_params* pin, pasd_plan_t** out,
                                 size_t* footprint_bytes) {
    if (!c || !pin || !out) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_params p = *pin;
    const int N = p.order;
    if (N < 2 || N > PASD_MAX_ORDER) return fail(PASD_ERR_INVALID_ARG, "order must be in [2, 8]");
    int64_t D = 1;
    for (int n = 0; n < N; ++n) {
        if (p.dims[n] < 1) return fail(PASD_ERR_INVALID_ARG, "dims must be >= 1");
        if (p.rank_bound[n] < 1) return fail(PASD_ERR_INVALID_ARG, "rank bound must be >= 1");
        if (p.rank_bound[n] > p.dims[n])
            return fail(PASD_ERR_INVALID_ARG, "rank bound R_n > I_n: St(I_n, R_n) is empty");
        if (p.rank_bound[n] > PASD_MAX_RANK)
            return fail(PASD_ERR_UNSUPPORTED, "rank bound above PASD_MAX_RANK");
        D *= p.dims[n];
    }
    if (p.mu0 == 0) p.mu0 = 1e-4;
    if (p.mu_max == 0) p.mu_max = 1e10;
    if (p.rho == 0) p.rho = 1.1;
    if (p.tol == 0) p.tol = 1e-5;
    if (p.max_iter == 0) p.max_iter = 1000;
    if (p.check_every <= 0) p.check_every = 8;
    if (!(p.mu0 > 0) || !(p.rho > 1) || !(p.mu_max >= p.mu0) || !(p.tol > 0) || p.max_iter < 1)
        return fail(PASD_ERR_INVALID_ARG, "need mu0 > 0, rho > 1, mu_max >= mu0, tol > 0, max_iter >= 1");
    if (p.stop_rule < 0 || p.stop_rule > 2) return fail(PASD_ERR_INVALID_ARG, "bad stop rule");
    if (p.precision != PASD_PREC_FP32 && p.precision != PASD_PREC_MIXED)
        return fail(PASD_ERR_INVALID_ARG, "bad precision");
    if (p.flags & ~(uint32_t)(PASD_F_SKIP_IDLE | PASD_F_FP64_EIG)) return fail(PASD_ERR_INVALID_ARG, "unknown flag bits");
    if (p.flags & PASD_F_FP64_EIG)
        for (int n = 0; n < N; ++n)
            if (p.rank_bound[n] > 56)
                return fail(PASD_ERR_UNSUPPORTED, "PASD_F_FP64_EIG: rank bounds above 56 do not fit shared memory");

    pasd_plan_t* pl = new pasd_plan_t();
    pl->ctx = c;
    pl->N = N;
    pl->D = D;
    // weights: all alpha_n zero selects the default 1/N; otherwise every one must be
    // finite and > 0 (a partly filled weight vector is an error, not a mix)
    {
        int zeros = 0;
        for (int n = 0; n < N; ++n) {
            const double a = p.alpha[n];
            if (!std::isfinite(a) || a < 0) { delete pl; return fail(PASD_ERR_INVALID_ARG, "alpha_n must be finite and > 0"); }
            zeros += a == 0;
        }
        if (zeros != 0 && zeros != N) {
            delete pl;
            return fail(PASD_ERR_INVALID_ARG, "alpha_n must all be > 0, or all 0 for the default 1/N");
        }
        for (int n = 0; n < N; ++n) pl->alpha[n] = zeros ? 1.0 / N : p.alpha[n];
    }
    if (std::isnan(p.lambda) || std::isinf(p.lambda)) { delete pl; return fail(PASD_ERR_INVALID_ARG, "lambda must be finite"); }
    for (int n = 0; n < N; ++n)
        if (p.lambda <= 0 && !(p.lambda_n[n] >= 0 && std::isfinite(p.lambda_n[n]))) {
            delete pl;
            return fail(PASD_ERR_INVALID_ARG, "lambda_n must be finite and > 0 (0 selects the default)");
        }
    int64_t dint[PASD_MAXN];
    for (int n = 0; n < N; ++n) dint[n] = p.dims[n];
    pl->D_real = D;
    pl->I_last_real = p.dims[N - 1];
    if (N <= 4 && p.dims[N - 1] % 4 != 0) {
        const char* nt0 = std::getenv("PASD_NO_TMA");
        if (!(nt0 && nt0[0] == '1')) {
            pl->pad = true;
            dint[N - 1] = (p.dims[N - 1] + 3) / 4 * 4;
            pl->D = D / p.dims[N - 1] * dint[N - 1];
        }
    }
    for (int n = 0; n < N; ++n) {
        ModeGeom& g = pl->m[n];
        // default lambda_n from the caller's sizes
        int64_t preR = 1, postR = 1;
        for (int m = 0; m < n; ++m) preR *= p.dims[m];
        for (int m = n + 1; m < N; ++m) postR *= p.dims[m];
        g.I = dint[n];
        g.pre = 1;
        for (int m = 0; m < n; ++m) g.pre *= dint[m];
        g.post = 1;
        for (int m = n + 1; m < N; ++m) g.post *= dint[m];
        g.P = g.pre * g.post;
        g.R = p.rank_bound[n];
        g.Rp = rank_bucket(g.R);
        // the per-mode kernels index I_n x (Rp_n + 4) matrices with 32-bit offsets
        if (g.I * (int64_t)(g.Rp + 4) >= ((int64_t)1 << 31)) {
            delete pl;
            return fail(PASD_ERR_UNSUPPORTED, "mode length times rank bucket reaches 2^31");
        }
        double lam;
        if (p.lambda > 0) lam = pl->alpha[n] / p.lambda;
        else if (p.lambda_n[n] > 0) lam = p.lambda_n[n];
        else lam = std::sqrt((double)std::max<int64_t>(p.dims[n], preR * postR)) / N;
        pl->lam[n] = lam;
    }
    pl->p = p;
    int64_t Is[PASD_MAXN];
    int Rps[PASD_MAXN];
    for (int n = 0; n < N; ++n) { Is[n] = pl->m[n].I; Rps[n] = pl->m[n].Rp; }
    size_t smem_limit = std::min<size_t>(c->smem_optin, 200 * 1024);
    if (!plan_fused_geom(pl->fg_plain, N, Is, Rps, c->num_sms, smem_limit)) {
        delete pl;
        return fail(PASD_ERR_UNSUPPORTED, "no tile shape fits shared memory for these ranks");
    }
    const char* nt = std::getenv("PASD_NO_TMA");
    // one CTA per SM with the largest tile that fits, or two resident CTAs per SM
    // (more copies in flight) with tiles that fit half the SM's shared memory:
    // whichever keeps more threads resident, two CTAs on a tie
    if (!(nt && nt[0] == '1')) {
        FusedGeom one{}, two{};
        const size_t half = c->smem_per_sm / 2 > 2048 ? c->smem_per_sm / 2 - 1024 : 0;
        const bool ok1 = plan_fused_tma(one, N, Is, Rps, c->num_sms, c->smem_optin);
        const bool ok2 = plan_fused_tma(two, N, Is, Rps, 2 * c->num_sms, std::min(half, c->smem_optin));
        if (ok2 && (!ok1 || 2 * two.nthreads >= one.nthreads)) { pl->fg = two; pl->want_tma = true; pl->default_fused_k = 2; }
        else if (ok1) { pl->fg = one; pl->want_tma = true; pl->default_fused_k = 1; }
        // the autotuner's candidates: k = 1, 2, 3 resident CTAs per SM, each with
        // the largest tile that fits 1/k of the SM's shared memory
        for (int k = 1; k <= 3; ++k) {
            FusedGeom gk{};
            const size_t share = c->smem_per_sm / k > 2048 ? c->smem_per_sm / k - 1024 : 0;
            const size_t lim = k == 1 ? c->smem_optin : std::min(share, c->smem_optin);
            if (plan_fused_tma(gk, N, Is, Rps, k * c->num_sms, lim)) {
                pl->fcand[pl->n_fcand] = gk;
                pl->fcand_k[pl->n_fcand] = k;
                ++pl->n_fcand;
            }
        }
    }
    if (!pl->want_tma) pl->fg = pl->fg_plain;
    const bool tma_ok = !(nt && nt[0] == '1');
    // A-pass products: FP32 multiply-adds (FP32 precision), or the tensor cores
    // with the TF32 hi/lo split (mixed precision). The split products land about
    // 2x further from FP64 than the FMAs, and at these skinny shapes (N = Rp)
    // converting each stage into split operands costs more than the FMAs, so the
    // FP32 path keeps the FMA kernel.
    pl->ap_kind = p.precision == PASD_PREC_MIXED ? APASS_TC : APASS_FFMA;
    const char* nf = std::getenv("PASD_NO_FEWROW");
    const bool no_fewrow = nf && nf[0] == '1';
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        pl->ap_small[n] = !no_fewrow && apass_small_supported(g.I, g.Rp);
        pl->ap_small_grid[n] = apass_small_grid(c->num_sms, g.P);
        pl->ap_use_tma[n] = !pl->ap_small[n] && tma_ok && apass_tma_supported(g.I, g.post);
        // Gram partials: room for the CTA count of the kernel in use (the TMA plan
        // may be refused later, leaving the cp.async kernel)
        pl->ncta_ap[n] = pl->ap_small[n] ? pl->ap_small_grid[n]
                                         : std::max(apass_ncta(g.P), apass_tma_tasks(g.I, g.pre, g.post, pl->ap_kind));
    }
    // M-pass: row strips x column ranges, as many CTAs as fit on the device at
    // once (one wave), split over the modes in proportion to their columns
    {
        int64_t work[PASD_MAXN], tot = 0;
        size_t smem = 0;
        for (int n = 0; n < N; ++n) {
            const ModeGeom& g = pl->m[n];
            MpassMode& mm = pl->mpa.m[n];
            mm.I = g.I; mm.post = g.post; mm.P = g.P; mm.Rp = g.Rp;
            mm.variant = mpass_variant(g.I, g.post);
            mm.IS = mpass_strip_rows(g.I, g.Rp);
            mm.nstrips = (int)((g.I + mm.IS - 1) / mm.IS);
            // few-row modes run their own kernel (no CTAs here)
            work[n] = pl->ap_small[n] ? 0 : (int64_t)mm.nstrips * ((g.P + MP_CB - 1) / MP_CB);
            tot += work[n];
            smem = std::max(smem, mpass_smem_bytes(mm.IS, g.Rp, mm.variant));
        }
        const int slots = c->num_sms * mpass_ctas_per_sm(smem);
        int start = 0;
        for (int n = 0; n < N; ++n) {
            MpassMode& mm = pl->mpa.m[n];
            pl->mpa.cta_start[n] = start;
            if (pl->ap_small[n]) {
                mm.ncg = 0;
                mm.cols_per_cg = MP_CB;
                pl->n_mp[n] = pl->ap_small_grid[n];
                continue;
            }
            int64_t target = (int64_t)((double)slots * (double)work[n] / (double)std::max<int64_t>(tot, 1));
            int64_t ncg = std::max<int64_t>(1, target / mm.nstrips);
            int64_t cols = (mm.P + ncg - 1) / ncg;
            cols = (cols + MP_CB - 1) / MP_CB * MP_CB;
            mm.cols_per_cg = cols;
            mm.ncg = (int)((mm.P + cols - 1) / cols);
            pl->n_mp[n] = mm.ncg;
            start += mm.nstrips * mm.ncg;
        }
        pl->mpa.cta_start[N] = start;
        pl->mpa.N = N;
        pl->mp_smem = smem;
    }
    // TMA-fed M-pass when every mode's layout allows it: CTAs = row strips x
    // ranges of whole chunks, one wave, split over the modes by work
    pl->mp_use_tma = tma_ok;
    for (int n = 0; n < N; ++n)
        pl->mp_use_tma = pl->mp_use_tma && (pl->ap_small[n] || mpass_tma_supported(pl->m[n].I, pl->m[n].post));
    if (pl->mp_use_tma) {
        int64_t work[PASD_MAXN], tot = 0;
        size_t smem = 0;
        for (int n = 0; n < N; ++n) {
            const ModeGeom& g = pl->m[n];
            MpassTmaMode& mm = pl->mpt.m[n];
            mm.I = g.I; mm.pre = g.pre; mm.post = g.post; mm.P = g.P; mm.Rp = g.Rp;
            mm.rowmajor = g.post == 1;
            mm.IS = mpass_strip_rows(g.I, g.Rp);
            mm.nstrips = (int)((g.I + mm.IS - 1) / mm.IS);
            mm.nch = mpass_tma_chunks(g.pre, g.post);
            mm.nbb = mm.rowmajor ? 1 : (int)((g.post + MP_CB - 1) / MP_CB);
            work[n] = pl->ap_small[n] ? 0 : (int64_t)mm.nstrips * mm.nch;
            tot += work[n];
            if (!pl->ap_small[n]) smem = std::max(smem, mpass_tma_smem_bytes(mm.IS, g.Rp));
        }
        pl->mpt.N = N;
        pl->mpt_smem = smem;
        pl->mpt_slots = c->num_sms * mpass_tma_ctas_per_sm(smem);
        pl->mpt_tot = tot;
        for (int n = 0; n < N; ++n) pl->mpt_work[n] = work[n];
        // the autotuner's candidates: one or two waves of CTAs (column ranges)
        for (int waves = 2; waves >= 1; --waves) {
            MpassTmaArgs a = mpass_tma_layout(pl, waves);
            for (int n = 0; n < N; ++n) pl->n_mp[n] = std::max(pl->n_mp[n], a.m[n].ncg);
        }
        pl->mpt = mpass_tma_layout(pl, 1);
    }
    int nparts = std::max(pl->fg.nregions, pl->fg_plain.nregions);
    for (int q = 0; q < pl->n_fcand; ++q) nparts = std::max(nparts, pl->fcand[q].nregions);
    pl->nparts_max = nparts;
    // footprint (padded sizes)
    const int64_t Dp = pl->D;
    size_t f = align256(sizeof(DevScalars));
    f += align256(Dp * 4);                                  // T copy
    f += align256(Dp * 4);                                  // E
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        f += align256(Dp * 4);                              // G_n
        f += 2 * align256((size_t)g.P * g.Rp * 4);          // A_n, Vrot_n
        f += 2 * align256((size_t)g.I * g.Rp * 4);          // U_n, Urot_n
        f += align256((size_t)g.Rp * g.Rp * 4) + 2 * align256(g.Rp * 4);
        f += align256((size_t)pl->ncta_ap[n] * g.Rp * g.Rp * 4);
        f += align256((size_t)pl->n_mp[n] * g.I * g.Rp * 4);
        f += align256((size_t)4 * g.I * g.Rp * 4);
        f += align256((size_t)g.I * g.Rp * 4);              // Mred_n
    }
    f += align256((size_t)nparts * (3 + N) * 4);
    f += align256(1024 * 4) + align256(PASD_MAXN * 4) + align256(4);   // + idle-skip factor
    f += align256(sizeof(DevScalars));                     // autotuner scalars
    f += align256((size_t)p.max_iter * PASD_TRACE_STRIDE * 8);
    if (pl->pad) f += align256(Dp * 4);                    // output-pass target
    pl->footprint = f;
    if (footprint_bytes) *footprint_bytes = f;
    const char* ng = std::getenv("PASD_NO_GRAPH");
    pl->use_graph = !(ng && ng[0] == '1');
    const char* tw = std::getenv("PASD_TEST_WAIT_TIMEOUT");
    pl->test_wait_timeout = tw && tw[0] == '1';
    *out = pl;
    return PASD_OK;
}

// TMA M-pass CTAs: row strips x column ranges, `waves` times as many as fit on
// the device at once, split over the (non few-row) modes in proportion to their work
static MpassTmaArgs mpass_tma_layout(const pasd_plan_t* pl, int waves) {
    MpassTmaArgs a = pl->mpt;
    const int slots = waves * pl->mpt_slots;
    int start = 0;
    for (int n = 0; n < pl->N; ++n) {
        MpassTmaMode& mm = a.m[n];
        a.cta_start[n] = start;
        if (pl->ap_small[n]) { mm.ncg = 0; mm.cpr = 1; continue; }
        int64_t target = (int64_t)((double)slots * (double)pl->mpt_work[n] / (double)std::max<int64_t>(pl->mpt_tot, 1));
        int64_t ncg = std::max<int64_t>(1, target / mm.nstrips);
        mm.cpr = (int)((mm.nch + ncg - 1) / ncg);
        mm.ncg = (mm.nch + mm.cpr - 1) / mm.cpr;
        start += mm.nstrips * mm.ncg;
    }
    a.cta_start[pl->N] = start;
    return a;
}

static void launch_fused_pass(pasd_plan_t* pl, int output, float* L, cudaStream_t s) {
    if (pl->tma) {
        launch_fused_tma(pl->tma, output, L, s);
    } else {
        FusedArgs fo = pl->fu;
        fo.output = output;
        fo.L = L;
        launch_fused(fo, s);
    }
}

static int launch_apass_all(pasd_plan_t* pl, cudaStream_t s) {
    int launches = 0;
    for (int n = 0; n < pl->N; ++n)
        if (pl->ap_small[n]) { launch_apass_small(pl->ap[n], pl->ap_small_grid[n], s); ++launches; }
    for (int q = 0; q < pl->n_ap_tma; ++q) { launch_apass_tma(pl->ap_tma[q], s); ++launches; }
    if (pl->n_ap_plain > 0) launches += launch_apass_modes(pl->ap_plain, pl->n_ap_plain, s);
    return launches;
}

static int launch_mpass_any(pasd_plan_t* pl, cudaStream_t s) {
    int launches = 0;
    for (int n = 0; n < pl->N; ++n)
        if (pl->ap_small[n]) { launch_mpass_small(pl->mp_small[n], pl->ap_small_grid[n], s); ++launches; }
    if (pl->n_mp_big == 0) return launches;
    if (pl->mp_use_tma) launch_mpass_tma(pl->mp_tma, s);
    else launch_mpass(pl->mpa, pl->mp_smem, s);
    return launches + 1;
}

static void enqueue_iteration(pasd_plan_t* pl, cudaStream_t s) {
    launch_polar(pl->small, s);
    pl->ap_launches = launch_apass_all(pl, s);
    launch_svt(pl->small, s);
    pl->vr_launches = launch_vrot(pl->vr, s);
    launch_fused_pass(pl, 0, nullptr, s);
    pl->mp_launches = launch_mpass_any(pl, s);
    launch_finalize(pl->fin, s);
}

// ---------------------------------------------------------------------------
// autotuner: tile shapes per problem shape, timed on the plan's own buffers at
// its first use and cached for the process
// ---------------------------------------------------------------------------
struct TuneChoice {
    int fused_k;     // resident CTAs per SM of the fused pass's geometry
    int mp_waves;    // waves of M-pass CTAs
    // A-pass FMA kernel, per launch group (modes of one padded rank): 0 default,
    // 1 half the columns per thread, 2 rows split in two thread groups
    int ap_var[PASD_MAXN];
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;

static std::string tune_key(const pasd_plan_t* pl) {
    std::string k = std::to_string(pl->ctx->device) + "|" + std::to_string(pl->want_tma) + "|" +
                    std::to_string(pl->ap_kind);
    for (int n = 0; n < pl->N; ++n)
        k += "|" + std::to_string(pl->m[n].I) + "x" + std::to_string(pl->m[n].Rp) + (pl->ap_small[n] ? "s" : "");
    return k;
}

// mean milliseconds of `reps` launches after one untimed launch (nan on error)
template <class F>
static float time_launches(cudaStream_t s, F f, int reps) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return NAN;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return NAN; }
    f();
    cudaEventRecord(a, s);
    for (int i = 0; i < reps; ++i) f();
    cudaEventRecord(b, s);
    float ms = NAN;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaGetLastError() == cudaSuccess) {
        cudaEventElapsedTime(&ms, a, b);
        ms /= reps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms;
}

// Tuning state: the launches read only these scalars (nothing has been solved:
// the arena is zero, so every value the timed kernels read or write stays zero).
static void set_tune_scalars(pasd_plan_t* pl, bool active) {
    DevScalars h{};
    h.mu = 1.0;
    h.t_norm_fro = 1.0;
    for (int n = 0; n < pl->N; ++n) h.kept[n] = active ? std::max(1, pl->m[n].R / 2) : 0;
    cudaMemcpyAsync(pl->tune_sc, &h, sizeof(h), cudaMemcpyHostToDevice, pl->cap_stream);
}

static MpassTmaArgs mpass_candidate(const pasd_plan_t* pl, int waves, DevScalars* sc) {
    MpassTmaArgs a = mpass_tma_layout(pl, waves);
    a.sc = sc;
    for (int n = 0; n < pl->N; ++n) a.m[n].part = pl->mp[n];
    return a;
}

static MpassTmaPlan* make_mpass_candidate(const pasd_plan_t* pl, const MpassTmaArgs& a) {
    const float* gp[PASD_MAXN];
    const float* vp[PASD_MAXN];
    for (int n = 0; n < pl->N; ++n) { gp[n] = pl->G[n]; vp[n] = pl->Vr[n]; }
    char err[256];
    return make_mpass_tma(a, gp, vp, pl->mpt_smem, err, sizeof(err));
}

// Switches the plan's kernels to the choice `c` (fused geometry, M-pass layout,
// A-pass columns per thread); a shape whose maps the driver refuses stays as it was.
static void apply_tune(pasd_plan_t* pl, const TuneChoice& c) {
    char err[256];
    if (pl->tma && c.fused_k != pl->tuned_fused_k) {
        for (int q = 0; q < pl->n_fcand; ++q) {
            if (pl->fcand_k[q] != c.fused_k) continue;
            FusedArgs fu2 = pl->fu;
            fu2.g = pl->fcand[q];
            FusedTmaPlan* tp = make_fused_tma(fu2, pl->Tc, err, sizeof(err));
            if (!tp) break;
            destroy_fused_tma(pl->tma);
            pl->tma = tp;
            pl->fg = pl->fcand[q];
            pl->fu.g = pl->fg;
            pl->fin.nparts = pl->fg.nregions;
            pl->tuned_fused_k = c.fused_k;
            break;
        }
    }
    if (pl->mp_tma && c.mp_waves != pl->tuned_mp_waves) {
        MpassTmaArgs a = mpass_candidate(pl, c.mp_waves, pl->sc);
        MpassTmaPlan* mp = make_mpass_candidate(pl, a);
        if (mp) {
            destroy_mpass_tma(pl->mp_tma);
            pl->mp_tma = mp;
            pl->mpt = a;
            for (int n = 0; n < pl->N; ++n)
                if (!pl->ap_small[n]) pl->fin.n_mp[n] = a.m[n].ncg;
            pl->tuned_mp_waves = c.mp_waves;
        }
    }
    for (int q = 0; q < pl->n_ap_tma; ++q) {
        const int cur = apass_tma_cols(pl->ap_tma[q]);
        if (cur == 0) continue;
        const int def = pl->ap_tma_default_nc[q];
        apass_tma_set_cols(pl->ap_tma[q], c.ap_var[q] == 1 ? def / 2 : def, c.ap_var[q] == 2 ? 2 : 1);
    }
}

// Times the candidates on the plan's own buffers (before its first pasd_begin
// fills them) and keeps one only if it beats the planner's default by more than
// 3%, so timing noise between near-equal shapes does not flip the choice; the
// choice is cached per device and problem shape.
// PASD_TUNE_APASS=0|1|2 forces the FP32 A-pass variant of every plan (default
// columns, half the columns, rows split in two groups) over the timed or cached
// choice, for comparisons; it does not enter the cache.
static void force_apass_variant(pasd_plan_t* pl) {
    const char* f = std::getenv("PASD_TUNE_APASS");
    if (!f || f[0] < '0' || f[0] > '2' || f[1] != 0) return;
    const int var = f[0] - '0';
    for (int q = 0; q < pl->n_ap_tma; ++q) {
        const int def = pl->ap_tma_default_nc[q];
        if (def == 0) continue;
        apass_tma_set_cols(pl->ap_tma[q], var == 1 ? def / 2 : def, var == 2 ? 2 : 1);
    }
}

static void autotune_impl(pasd_plan_t* pl);
static void autotune(pasd_plan_t* pl) {
    autotune_impl(pl);
    force_apass_variant(pl);
}

static void autotune_impl(pasd_plan_t* pl) {
    pl->tuned = true;
    pl->tuned_fused_k = pl->default_fused_k;
    pl->tuned_mp_waves = 1;
    for (int q = 0; q < pl->n_ap_tma; ++q) pl->ap_tma_default_nc[q] = apass_tma_cols(pl->ap_tma[q]);
    const char* nt = std::getenv("PASD_NO_TUNE");
    if (nt && nt[0] == '1') { pl->tune_mode = "off"; return; }
    const std::string key = tune_key(pl);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { apply_tune(pl, it->second); pl->tune_mode = "cached"; return; }
    }
    pl->tune_mode = "timed";
    cudaStream_t s = pl->cap_stream;
    TuneChoice choice{pl->default_fused_k, 1, {0}};
    char err[256];
    if (pl->tma && pl->n_fcand > 1) {
        float t_def = NAN, best = INFINITY;
        int best_k = pl->default_fused_k;
        for (int q = 0; q < pl->n_fcand; ++q) {
            FusedArgs fc = pl->fu;
            fc.g = pl->fcand[q];
            fc.sc = pl->tune_sc;
            FusedTmaPlan* tp = make_fused_tma(fc, pl->Tc, err, sizeof(err));
            if (!tp) continue;
            float t = 0.f;
            for (int active = 0; active < 2; ++active) {
                set_tune_scalars(pl, active != 0);
                t += time_launches(s, [&] { launch_fused_tma(tp, 0, nullptr, s); }, 3);
            }
            destroy_fused_tma(tp);
            if (!(t == t)) continue;
            if (pl->fcand_k[q] == pl->default_fused_k) t_def = t;
            if (t < best) { best = t; best_k = pl->fcand_k[q]; }
        }
        if (t_def == t_def && best < 0.97f * t_def) choice.fused_k = best_k;
    }
    // The M-pass and the A-pass read G_n (D floats per mode), which can fit in L2
    // when they are launched back to back; in a loop body each runs after the
    // fused pass has streamed (2N + 3) 4D bytes through it. So each of their
    // candidates is timed behind an idle fused pass, whose own time is subtracted.
    FusedTmaPlan* evict = nullptr;
    if (pl->tma) {
        FusedArgs fe = pl->fu;
        fe.sc = pl->tune_sc;
        evict = make_fused_tma(fe, pl->Tc, err, sizeof(err));
    }
    // mean time of f() behind the eviction pass, under the tuning scalars as set
    auto behind_evict = [&](auto f) {
        if (!evict) return time_launches(s, f, 5);
        const float te = time_launches(s, [&] { launch_fused_tma(evict, 0, nullptr, s); }, 5);
        return time_launches(s, [&] {
            launch_fused_tma(evict, 0, nullptr, s);
            f();
        }, 5) - te;
    };
    if (pl->mp_tma) {
        set_tune_scalars(pl, true);   // the M-pass as in an active body
        float tw[3] = {NAN, NAN, NAN};
        for (int waves = 1; waves <= 2; ++waves) {
            MpassTmaPlan* mp = make_mpass_candidate(pl, mpass_candidate(pl, waves, pl->tune_sc));
            if (!mp) continue;
            tw[waves] = behind_evict([&] { launch_mpass_tma(mp, s); });
            destroy_mpass_tma(mp);
        }
        if (tw[1] == tw[1] && tw[2] == tw[2] && tw[2] < 0.97f * tw[1]) choice.mp_waves = 2;
    }
    set_tune_scalars(pl, false);
    if (pl->n_ap_tma > 0 && pl->ap_kind == APASS_FFMA) {
        // the A-pass reads only the done flag, which is clear before the first pasd_begin
        // each launch group (modes of one padded rank) takes its own variant
        for (int q = 0; q < pl->n_ap_tma; ++q) {
            const int def = pl->ap_tma_default_nc[q];
            if (def == 0) continue;
            float th[3] = {NAN, NAN, NAN};
            for (int var = 0; var < 3; ++var) {
                apass_tma_set_cols(pl->ap_tma[q], var == 1 ? def / 2 : def, var == 2 ? 2 : 1);
                th[var] = behind_evict([&] { launch_apass_tma(pl->ap_tma[q], s); });
            }
            apass_tma_set_cols(pl->ap_tma[q], def, 1);
            float best = th[0];
            for (int var = 1; var < 3; ++var)
                if (th[0] == th[0] && th[var] == th[var] && th[var] < 0.97f * th[0] && th[var] < best) {
                    best = th[var];
                    choice.ap_var[q] = var;
                }
        }
    }
    cudaStreamSynchronize(s);
    cudaGetLastError();
    if (evict) destroy_fused_tma(evict);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache.emplace(key, choice);
    }
    apply_tune(pl, choice);
}

static pasd_status ensure_allocated(pasd_plan_t* pl) {
    if (pl->arena) return PASD_OK;
    CUDA_TRY(cudaSetDevice(pl->ctx->device));
    char* base = nullptr;
    CUDA_TRY(cudaMalloc(&base, pl->footprint));
    pl->arena = base;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base + off; off += align256(bytes); return p; };
    const int N = pl->N;
    const int64_t D = pl->D;
    pl->sc = reinterpret_cast<DevScalars*>(take(sizeof(DevScalars)));
    pl->Tc = reinterpret_cast<float*>(take(D * 4));
    pl->E = reinterpret_cast<float*>(take(D * 4));
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        pl->G[n] = reinterpret_cast<float*>(take(D * 4));
        pl->A[n] = reinterpret_cast<float*>(take((size_t)g.P * g.Rp * 4));
        pl->Vr[n] = reinterpret_cast<float*>(take((size_t)g.P * g.Rp * 4));
        pl->U[n] = reinterpret_cast<float*>(take((size_t)g.I * g.Rp * 4));
        pl->Urot[n] = reinterpret_cast<float*>(take((size_t)g.I * g.Rp * 4));
        pl->W[n] = reinterpret_cast<float*>(take((size_t)g.Rp * g.Rp * 4));
        pl->F[n] = reinterpret_cast<float*>(take(g.Rp * 4));
        pl->sigma[n] = reinterpret_cast<float*>(take(g.Rp * 4));
        pl->gram[n] = reinterpret_cast<float*>(take((size_t)pl->ncta_ap[n] * g.Rp * g.Rp * 4));
        pl->mp[n] = reinterpret_cast<float*>(take((size_t)pl->n_mp[n] * g.I * g.Rp * 4));
        pl->scratch[n] = reinterpret_cast<float*>(take((size_t)4 * g.I * g.Rp * 4));
        pl->Mred[n] = reinterpret_cast<float*>(take((size_t)g.I * g.Rp * 4));
    }
    pl->part = reinterpret_cast<float*>(take((size_t)pl->nparts_max * (3 + N) * 4));
    pl->tune_sc = reinterpret_cast<DevScalars*>(take(sizeof(DevScalars)));
    pl->sq_part = reinterpret_cast<float*>(take(1024 * 4));
    pl->kept = reinterpret_cast<int32_t*>(take(PASD_MAXN * 4));
    pl->idle_g = reinterpret_cast<float*>(take(4));
    pl->trace = reinterpret_cast<double*>(take((size_t)pl->p.max_iter * PASD_TRACE_STRIDE * 8));
    if (pl->pad) pl->Lpad = reinterpret_cast<float*>(take(D * 4));
    // zeros everywhere once: the padded entries of T, E, G_n are never written.
    // The clear runs on the plan's own non-blocking stream and is complete before
    // this returns: a plain cudaMemset would be queued on the legacy default stream,
    // which work on non-blocking streams (the served path's, or a caller's) does not
    // wait for, so behind other work there it could land in the middle of a solve.
    CUDA_TRY(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
    CUDA_TRY(cudaMemsetAsync(pl->arena, 0, pl->footprint, pl->cap_stream));
    CUDA_TRY(cudaStreamSynchronize(pl->cap_stream));
    CUDA_TRY(cudaMallocHost(&pl->host_sc, sizeof(DevScalars)));
    CUDA_TRY(cudaEventCreateWithFlags(&pl->ev, cudaEventDisableTiming));

    // launch descriptors
    SmallArgs& sa = pl->small;
    sa.N = N;
    sa.sc = pl->sc;
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        SmallModeArgs& m = sa.m[n];
        m.I = g.I; m.R = g.R; m.Rp = g.Rp; m.lambda = pl->lam[n];
        m.U = pl->U[n]; m.Urot = pl->Urot[n]; m.W = pl->W[n]; m.F = pl->F[n]; m.sigma = pl->sigma[n];
        m.gram_part = pl->gram[n]; m.n_gram = pl->ncta_ap[n];
        m.Mred = pl->Mred[n];
        m.scratch = pl->scratch[n];
        m.kept = pl->kept + n;
        ApassArgs& a = pl->ap[n];
        a.G = pl->G[n]; a.U = pl->U[n]; a.A = pl->A[n]; a.gram_part = pl->gram[n]; a.sc = pl->sc;
        a.I = g.I; a.pre = g.pre; a.post = g.post; a.P = g.P; a.R = g.R; a.Rp = g.Rp;
        a.ncta = apass_ncta(g.P);      // CTAs of the cp.async kernel
    }
    FusedArgs& fu = pl->fu;
    fu.g = pl->fg;
    fu.sc = pl->sc;
    fu.E = pl->E;
    double asum = 0;
    for (int n = 0; n < N; ++n) asum += pl->alpha[n];
    for (int n = 0; n < N; ++n) {
        fu.G[n] = pl->G[n]; fu.A[n] = pl->Vr[n]; fu.Wz[n] = pl->Urot[n];
        fu.alpha_w[n] = (float)(pl->alpha[n] / asum);
    }
    fu.part = pl->part;
    fu.part_stride = 3 + N;
    fu.rho = pl->p.rho;
    fu.mu_max = pl->p.mu_max;
    fu.output = 0;
    fu.L = nullptr;
    fu.test_no_copy = pl->test_wait_timeout ? 1 : 0;
    fu.wait_polls = pl->test_wait_timeout ? 4096u : 0u;   // 0: the kernels' default bound
    VrotArgs& va = pl->vr;
    va.N = N;
    va.sc = pl->sc;
    va.cta_start[0] = 0;
    int vr_maxRp = 4;
    for (int n = 0; n < N; ++n) vr_maxRp = std::max(vr_maxRp, pl->m[n].Rp);
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        VrotMode& vm = va.m[n];
        vm.A = pl->A[n]; vm.V = pl->Vr[n]; vm.W = pl->W[n]; vm.F = pl->F[n];
        vm.P = g.P; vm.post = g.post; vm.R = g.R; vm.Rp = g.Rp; vm.mode = n;
        va.cta_start[n + 1] = va.cta_start[n] + vrot_ctas(g.P, g.post, vr_maxRp);
    }
    pl->mpa.sc = pl->sc;
    for (int n = 0; n < N; ++n) {
        MpassMode& mm = pl->mpa.m[n];
        mm.G = pl->G[n]; mm.V = pl->Vr[n]; mm.part = pl->mp[n];
    }
    FinalizeArgs& fi = pl->fin;
    fi.N = N; fi.sc = pl->sc; fi.part = pl->part; fi.nparts = pl->fg.nregions; fi.stride = 3 + N;
    for (int n = 0; n < N; ++n) fi.lambda[n] = pl->lam[n];
    fi.rho = pl->p.rho; fi.mu_max = pl->p.mu_max; fi.tol = pl->p.tol;
    fi.stop_rule = pl->p.stop_rule; fi.max_iter = pl->p.max_iter; fi.trace = pl->trace;
    {
        IdleSkipArgs& ia = pl->idle;
        ia.sc = pl->sc;
        ia.N = N;
        for (int n = 0; n < N; ++n) { ia.sigma[n] = pl->sigma[n]; ia.lambda[n] = pl->lam[n]; ia.G[n] = pl->G[n]; }
        ia.rho = pl->p.rho;
        ia.mu_max = pl->p.mu_max;
        ia.max_iter = pl->p.max_iter;
        ia.trace = pl->trace;
        ia.T = pl->Tc;
        ia.D = pl->D;
        ia.g = pl->idle_g;
    }
    {
        int maxRp = 4;
        for (int n = 0; n < N; ++n) maxRp = std::max(maxRp, pl->m[n].Rp);
        for (int n = 0; n < N; ++n) {
            const ModeGeom& g = pl->m[n];
            fi.mp_part[n] = pl->mp[n]; fi.I[n] = g.I; fi.R[n] = g.R; fi.Rp[n] = g.Rp; fi.Mred[n] = pl->Mred[n];
            sa.m[n].fp64_eig = (pl->p.flags & PASD_F_FP64_EIG) ? 1 : 0;
            sa.m[n].polar_in_smem = polar_smem_bytes(maxRp, g.I, sa.m[n].fp64_eig != 0) <=
                                    std::min<size_t>(pl->ctx->smem_optin, 200 * 1024);
        }
    }
    if (pl->want_tma) {
        char err[256] = {0};
        pl->tma = make_fused_tma(fu, pl->Tc, err, sizeof(err));
        if (!pl->tma) {
            // tensor maps refused: use the single-buffer pass
            pl->fg = pl->fg_plain;
            fu.g = pl->fg;
            fi.nparts = pl->fg.nregions;
        }
    }
    // M-pass: the TMA kernel when every mode allows it and its maps are accepted;
    // the finalize sums exactly the partials the kernel in use writes
    if (pl->mp_use_tma) {
        pl->mpt.sc = pl->sc;
        const float* gp[PASD_MAXN];
        const float* vp[PASD_MAXN];
        for (int n = 0; n < N; ++n) {
            pl->mpt.m[n].part = pl->mp[n];
            gp[n] = pl->G[n];
            vp[n] = pl->Vr[n];
        }
        char err[256] = {0};
        pl->mp_tma = make_mpass_tma(pl->mpt, gp, vp, pl->mpt_smem, err, sizeof(err));
        if (!pl->mp_tma) pl->mp_use_tma = false;
    }
    pl->n_mp_big = 0;
    for (int n = 0; n < N; ++n) {
        const ModeGeom& g = pl->m[n];
        if (pl->ap_small[n]) {
            MpassSmallArgs& ms = pl->mp_small[n];
            ms.G = pl->G[n]; ms.V = pl->Vr[n]; ms.part = pl->mp[n]; ms.sc = pl->sc;
            ms.I = g.I; ms.pre = g.pre; ms.post = g.post; ms.P = g.P; ms.Rp = g.Rp; ms.mode = n;
            fi.n_mp[n] = pl->ap_small_grid[n];
        } else {
            ++pl->n_mp_big;
            fi.n_mp[n] = pl->mp_use_tma ? pl->mpt.m[n].ncg : pl->mpa.m[n].ncg;
        }
    }

    // A-pass: TMA plans for the modes whose layout allows them (grouped by padded
    // rank), the cp.async kernel for the rest or when a tensor map is refused
    {
        pl->n_ap_tma = 0;
        pl->n_ap_plain = 0;
        bool grouped[PASD_MAXN] = {false};
        for (int n = 0; n < N; ++n) {
            if (!pl->ap_use_tma[n] || grouped[n]) continue;
            int modes[PASD_MAXN], cnt = 0;
            for (int k = n; k < N; ++k)
                if (pl->ap_use_tma[k] && !grouped[k] && pl->m[k].Rp == pl->m[n].Rp) { modes[cnt++] = k; grouped[k] = true; }
            char err[256] = {0};
            ApassTmaPlan* tp = make_apass_tma(pl->ap, modes, cnt, pl->ap_kind, pl->ctx->num_sms, err, sizeof(err));
            if (tp) pl->ap_tma[pl->n_ap_tma++] = tp;
            else for (int q = 0; q < cnt; ++q) pl->ap_use_tma[modes[q]] = false;
        }
        for (int n = 0; n < N; ++n) {
            const ModeGeom& g = pl->m[n];
            if (pl->ap_small[n]) { sa.m[n].n_gram = pl->ap_small_grid[n]; continue; }
            if (!pl->ap_use_tma[n]) pl->ap_plain[pl->n_ap_plain++] = pl->ap[n];
            sa.m[n].n_gram = pl->ap_use_tma[n] ? apass_tma_tasks(g.I, g.pre, g.post, pl->ap_kind) : apass_ncta(g.P);
        }
    }

    autotune(pl);

    if (pl->use_graph) {
        CUDA_TRY(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeRelaxed));
        enqueue_iteration(pl, pl->cap_stream);
        CUDA_TRY(cudaStreamEndCapture(pl->cap_stream, &pl->graph));
        CUDA_TRY(cudaGraphInstantiate(&pl->exec, pl->graph, 0));
    }
    return PASD_OK;
}

// A plan with served solves queued or running belongs to the served path: the
// entry points that touch its state refuse it until they have retired.
static pasd_status check_not_served(pasd_plan_t* pl) {
    std::unique_lock<std::mutex> lk(pl->ctx->mu);
    if (pl->served > 0) return fail(PASD_ERR_BUSY, "plan has served solves queued or running");
    return PASD_OK;
}

extern "C" pasd_status pasd_plan_destroy(pasd_plan_t* pl) {
    if (!pl) return fail(PASD_ERR_INVALID_ARG, "plan is NULL");
    pasd_status chk = check_not_served(pl);
    if (chk != PASD_OK) return chk;
    if (pl->tma) destroy_fused_tma(pl->tma);
    for (int q = 0; q < pl->n_ap_tma; ++q) destroy_apass_tma(pl->ap_tma[q]);
    if (pl->mp_tma) destroy_mpass_tma(pl->mp_tma);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    if (pl->own_stream) cudaStreamDestroy(pl->own_stream);
    if (pl->ev) cudaEventDestroy(pl->ev);
    if (pl->host_sc) cudaFreeHost(pl->host_sc);
    if (pl->arena) cudaFree(pl->arena);
    if (pl->dev_io) cudaFree(pl->dev_io);
    if (pl->y_tmp) cudaFree(pl->y_tmp);
    delete pl;
    return PASD_OK;
}

extern "C" pasd_status pasd_profile_iterations(pasd_plan_t* pl, int32_t iters, double* ms,
                                               void* stream) {
    if (!pl || !ms || iters < 0) return fail(PASD_ERR_INVALID_ARG, "bad argument");
    pasd_status chk = check_not_served(pl);
    if (chk != PASD_OK) return chk;
    if (!pl->arena) return fail(PASD_ERR_INVALID_ARG, "pasd_begin has not run");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[PASD_PROFILE_SLOTS + 1];
    for (auto& e : ev) CUDA_TRY(cudaEventCreate(&e));
    for (int k = 0; k < PASD_PROFILE_SLOTS; ++k) ms[k] = 0.0;
    for (int it = 0; it < iters; ++it) {
        CUDA_TRY(cudaEventRecord(ev[0], s));
        launch_polar(pl->small, s);
        CUDA_TRY(cudaEventRecord(ev[1], s));
        launch_apass_all(pl, s);
        CUDA_TRY(cudaEventRecord(ev[2], s));
        launch_svt(pl->small, s);
        CUDA_TRY(cudaEventRecord(ev[3], s));
        launch_vrot(pl->vr, s);
        CUDA_TRY(cudaEventRecord(ev[4], s));
        launch_fused_pass(pl, 0, nullptr, s);
        CUDA_TRY(cudaEventRecord(ev[5], s));
        launch_mpass_any(pl, s);
        CUDA_TRY(cudaEventRecord(ev[6], s));
        launch_finalize(pl->fin, s);
        CUDA_TRY(cudaEventRecord(ev[7], s));
        CUDA_TRY(cudaEventSynchronize(ev[7]));
        for (int k = 0; k < PASD_PROFILE_SLOTS; ++k) {
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, ev[k], ev[k + 1]));
            ms[k] += t;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    CUDA_TRY(cudaGetLastError());
    return PASD_OK;
}

extern "C" pasd_status pasd_plan_info(const pasd_plan_t* pl, char* buf, size_t len) {
    if (!pl || !buf || len == 0) return fail(PASD_ERR_INVALID_ARG, "bad argument");
    const FusedGeom& g = pl->fg;
    std::string box, few;
    for (int n = 0; n < pl->N; ++n) {
        box += (n ? "," : "") + std::to_string(g.b[n]);
        if (pl->ap_small[n]) few += (few.empty() ? "" : ",") + std::to_string(n);
    }
    int mp_ctas = pl->mp_use_tma ? pl->mpt.cta_start[pl->N] : pl->mpa.cta_start[pl->N];
    std::string apc, aps;
    for (int q = 0; q < pl->n_ap_tma; ++q) {
        apc += (q ? "," : "") + std::to_string(apass_tma_cols(pl->ap_tma[q]));
        aps += (q ? "," : "") + std::to_string(apass_tma_split(pl->ap_tma[q]));
    }
    char tmp[1024];
    snprintf(tmp, sizeof(tmp),
             "{\"autotune\": \"%s\", \"fused\": {\"tma\": %d, \"ctas_per_sm\": %d, \"box\": [%s], \"regions\": %d, "
             "\"threads\": %d, \"candidates\": %d}, \"mpass\": {\"tma\": %d, \"waves\": %d, \"ctas\": %d}, "
             "\"apass_cols_per_thread\": [%s], \"apass_row_groups\": [%s], \"fewrow_modes\": [%s], "
             "\"launches_per_iter\": %d}",
             pl->tune_mode, pl->tma != nullptr || (!pl->arena && pl->want_tma) ? 1 : 0,
             pl->tuned ? pl->tuned_fused_k : pl->default_fused_k, box.c_str(), g.nregions,
             g.tma ? g.nthreads : FU_THREADS, pl->n_fcand, pl->mp_use_tma ? 1 : 0, pl->tuned_mp_waves, mp_ctas,
             apc.c_str(), aps.c_str(), few.c_str(), pl->ap_launches + pl->mp_launches + pl->vr_launches + 4);
    if (std::strlen(tmp) + 1 > len) return fail(PASD_ERR_INVALID_ARG, "buffer too small");
    std::memcpy(buf, tmp, std::strlen(tmp) + 1);
    return PASD_OK;
}

extern "C" int32_t pasd_launches_per_iter(const pasd_plan_t* pl) {
    return pl ? pl->ap_launches + pl->mp_launches + pl->vr_launches + 4 : 0;
}

// ---------------------------------------------------------------------------
// stepwise solve
// ---------------------------------------------------------------------------
static pasd_status begin_impl(pasd_plan_t* pl, const float* T, void* stream) {
    pasd_status st = ensure_allocated(pl);
    if (st != PASD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = pl->N;
    if (pl->pad) {
        // caller's rows of I_real floats into rows of the padded length (padding stays zero)
        const int64_t Ip = pl->m[N - 1].I, Ir = pl->I_last_real;
        CUDA_TRY(cudaMemcpy2DAsync(pl->Tc, Ip * 4, T, Ir * 4, Ir * 4, pl->D_real / Ir, cudaMemcpyDeviceToDevice, s));
    } else {
        CUDA_TRY(cudaMemcpyAsync(pl->Tc, T, pl->D * 4, cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaMemsetAsync(pl->E, 0, pl->D * 4, s));
    for (int n = 0; n < N; ++n) CUDA_TRY(cudaMemcpyAsync(pl->G[n], pl->Tc, pl->D * 4, cudaMemcpyDeviceToDevice, s));
    int64_t Is[PASD_MAXN];
    int Rs[PASD_MAXN], Rps[PASD_MAXN];
    for (int n = 0; n < N; ++n) { Is[n] = pl->m[n].I; Rs[n] = pl->m[n].R; Rps[n] = pl->m[n].Rp; }
    launch_init_state(pl->sc, pl->Tc, pl->p.mu0, N, pl->U, Is, Rs, Rps, pl->W, pl->F, pl->Urot, pl->kept, s);
    launch_norm_fro(pl->Tc, pl->D, pl->sq_part, 1024, pl->sc, s);
    pl->skip_pending = (pl->p.flags & PASD_F_SKIP_IDLE) != 0;
    CUDA_TRY(cudaGetLastError());
    return PASD_OK;
}

static pasd_status iterate_impl(pasd_plan_t* pl, int32_t iters, void* stream) {
    if (!pl->arena) return fail(PASD_ERR_INVALID_ARG, "pasd_begin has not run");
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < iters; ++i) {
        if (pl->use_graph) CUDA_TRY(cudaGraphLaunch(pl->exec, s));
        else enqueue_iteration(pl, s);
        if (pl->skip_pending) {
            // first body after pasd_begin: replace the provably idle bodies that follow
            launch_idle_skip(pl->idle, pl->ctx->num_sms, s);
            pl->skip_pending = false;
        }
    }
    CUDA_TRY(cudaGetLastError());
    return PASD_OK;
}

static pasd_status read_scalars(pasd_plan_t* pl, cudaStream_t s) {
    CUDA_TRY(cudaMemcpyAsync(pl->host_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return PASD_OK;
}

static void fill_result(pasd_plan_t* pl, pasd_result* r) {
    const DevScalars& h = *pl->host_sc;
    std::memset(r, 0, sizeof(*r));
    r->status = h.done ? h.status : PASD_NOT_CONVERGED;
    r->iters = h.k;
    r->res_inf = h.res_inf;
    r->res_fro_rel = h.res_fro_rel;
    r->objective = h.objective;
    r->l1_E = h.l1_E;
    r->mu_final = h.mu;
    for (int n = 0; n < pl->N; ++n) { r->kept[n] = h.kept[n]; r->nuclear[n] = h.nuclear[n]; }
    r->skipped = h.skipped;
}

static pasd_status finish_impl(pasd_plan_t* pl, float* L, float* E, pasd_result* res, void* stream) {
    if (!pl->arena) return fail(PASD_ERR_INVALID_ARG, "pasd_begin has not run");
    cudaStream_t s = (cudaStream_t)stream;
    pasd_status st = read_scalars(pl, s);
    if (st != PASD_OK) return st;
    pasd_result r;
    fill_result(pl, &r);
    if (res) *res = r;
    if (r.status != PASD_OK && r.status != PASD_NOT_CONVERGED) {
        return fail((pasd_status)r.status, r.status == PASD_ERR_TIMEOUT
                                               ? "solve failed: a bounded wait for a bulk copy ran out on the device"
                                               : "solve failed: non-finite values in the iterate");
    }
    // output: L = sum_n alpha_n Z_n / sum alpha_n, E (Algorithm 1, Output)
    if (pl->pad) {
        const int64_t Ip = pl->m[pl->N - 1].I, Ir = pl->I_last_real, rows = pl->D_real / Ir;
        launch_fused_pass(pl, 1, pl->Lpad, s);   // the output pass ignores the stop flag
        CUDA_TRY(cudaMemcpy2DAsync(L, Ir * 4, pl->Lpad, Ip * 4, Ir * 4, rows, cudaMemcpyDeviceToDevice, s));
        CUDA_TRY(cudaMemcpy2DAsync(E, Ir * 4, pl->E, Ip * 4, Ir * 4, rows, cudaMemcpyDeviceToDevice, s));
    } else {
        launch_fused_pass(pl, 1, L, s);   // the output pass ignores the stop flag
        CUDA_TRY(cudaMemcpyAsync(E, pl->E, pl->D * 4, cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    CUDA_TRY(cudaGetLastError());
    return (pasd_status)r.status;
}

static pasd_status run_loop(pasd_plan_t* pl, cudaStream_t s) {
    const int chunk = pl->p.check_every;
    const int max_iter = pl->p.max_iter;
    int launched = 0;
    // keep one chunk in flight while the previous chunk's flag is checked
    pasd_status st = iterate_impl(pl, std::min(chunk, max_iter), s);
    if (st != PASD_OK) return st;
    launched += std::min(chunk, max_iter);
    for (;;) {
        CUDA_TRY(cudaMemcpyAsync(pl->host_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaEventRecord(pl->ev, s));
        if (launched < max_iter) {
            int n = std::min(chunk, max_iter - launched);
            st = iterate_impl(pl, n, s);
            if (st != PASD_OK) return st;
            launched += n;
        }
        CUDA_TRY(cudaEventSynchronize(pl->ev));
        if (pl->host_sc->done) break;
        if (launched >= max_iter) {
            CUDA_TRY(cudaStreamSynchronize(s));
            break;
        }
    }
    return PASD_OK;
}

extern "C" pasd_status pasd_begin(pasd_plan_t* pl, const float* T, void* stream) {
    if (!pl || !T) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_status st = check_not_served(pl);
    if (st != PASD_OK) return st;
    return begin_impl(pl, T, stream);
}

extern "C" pasd_status pasd_iterate(pasd_plan_t* pl, int32_t iters, void* stream) {
    if (!pl || iters < 0) return fail(PASD_ERR_INVALID_ARG, "bad argument");
    pasd_status st = check_not_served(pl);
    if (st != PASD_OK) return st;
    return iterate_impl(pl, iters, stream);
}

extern "C" pasd_status pasd_finish(pasd_plan_t* pl, float* L, float* E, pasd_result* res,
                                   void* stream) {
    if (!pl || !L || !E) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_status st = check_not_served(pl);
    if (st != PASD_OK) return st;
    return finish_impl(pl, L, E, res, stream);
}

extern "C" pasd_status pasd_solve(pasd_plan_t* pl, const float* T, float* L, float* E,
                                  pasd_result* res, void* stream) {
    if (!pl || !T || !L || !E) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_status st = check_not_served(pl);
    if (st != PASD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = begin_impl(pl, T, stream);
    if (st != PASD_OK) return st;
    st = run_loop(pl, s);
    if (st != PASD_OK) return st;
    return finish_impl(pl, L, E, res, stream);
}

extern "C" pasd_status pasd_solve_host(pasd_plan_t* pl, const float* Th, float* Lh, float* Eh,
                                       pasd_result* res, void* stream) {
    if (!pl || !Th || !Lh || !Eh) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_status chk = check_not_served(pl);
    if (chk != PASD_OK) return chk;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t Dr = pl->D_real;
    if (!pl->dev_io) CUDA_TRY(cudaMalloc(&pl->dev_io, (size_t)3 * Dr * 4));
    float* Td = pl->dev_io;
    float* Ld = Td + Dr;
    float* Ed = Ld + Dr;
    CUDA_TRY(cudaMemcpyAsync(Td, Th, Dr * 4, cudaMemcpyHostToDevice, s));
    pasd_status st = pasd_solve(pl, Td, Ld, Ed, res, stream);
    if (st != PASD_OK && st != PASD_NOT_CONVERGED) return st;
    CUDA_TRY(cudaMemcpyAsync(Lh, Ld, Dr * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(Eh, Ed, Dr * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}

// ---------------------------------------------------------------------------
// state export
// ---------------------------------------------------------------------------
extern "C" pasd_status pasd_state_get(pasd_plan_t* pl, int32_t item, int32_t mode, void* dst,
                                      size_t bytes, void* stream) {
    if (!pl || !dst) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    pasd_status chk = check_not_served(pl);
    if (chk != PASD_OK) return chk;
    if (!pl->arena) return fail(PASD_ERR_INVALID_ARG, "no state yet");
    cudaStream_t s = (cudaStream_t)stream;
    const int N = pl->N;
    bool per_mode = item == PASD_STATE_U || item == PASD_STATE_A || item == PASD_STATE_W ||
                    item == PASD_STATE_SIGMA || item == PASD_STATE_F || item == PASD_STATE_Y;
    if (per_mode && (mode < 0 || mode >= N)) return fail(PASD_ERR_INVALID_ARG, "mode out of range");
    auto copy2d = [&](const float* src, int64_t rows, int cols, int ld) -> pasd_status {
        if (bytes != (size_t)rows * cols * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
        CUDA_TRY(cudaMemcpy2DAsync(dst, cols * 4, src, ld * 4, cols * 4, rows, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        return PASD_OK;
    };
    switch (item) {
        case PASD_STATE_U: {
            const int64_t rows = (pl->pad && mode == N - 1) ? pl->I_last_real : pl->m[mode].I;
            return copy2d(pl->U[mode], rows, pl->m[mode].R, pl->m[mode].Rp);
        }
        case PASD_STATE_W: return copy2d(pl->W[mode], pl->m[mode].R, pl->m[mode].R, pl->m[mode].Rp);
        case PASD_STATE_SIGMA: return copy2d(pl->sigma[mode], 1, pl->m[mode].R, pl->m[mode].Rp);
        case PASD_STATE_F: return copy2d(pl->F[mode], 1, pl->m[mode].R, pl->m[mode].Rp);
        case PASD_STATE_A: {
            // device layout [pre][Rp][post] -> host [R][pre*post] (unfolding column order)
            const ModeGeom& g = pl->m[mode];
            if (pl->pad && mode < N - 1) {
                // columns with a padded last-mode index are dropped
                const int64_t Ip = pl->m[N - 1].I, Ir = pl->I_last_real;
                const int64_t post_r = g.post / Ip * Ir, P_r = g.pre * post_r;
                if (bytes != (size_t)g.R * P_r * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
                std::vector<float> tmp((size_t)g.pre * g.Rp * g.post);
                CUDA_TRY(cudaMemcpyAsync(tmp.data(), pl->A[mode], tmp.size() * 4, cudaMemcpyDeviceToHost, s));
                CUDA_TRY(cudaStreamSynchronize(s));
                float* h = (float*)dst;
                const int64_t rest = g.post / Ip;
                for (int r = 0; r < g.R; ++r)
                    for (int64_t a = 0; a < g.pre; ++a)
                        for (int64_t b = 0; b < rest; ++b)
                            std::memcpy(h + (size_t)r * P_r + a * post_r + b * Ir,
                                        tmp.data() + ((size_t)a * g.Rp + r) * g.post + b * Ip, Ir * 4);
                return PASD_OK;
            }
            if (bytes != (size_t)g.R * g.P * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            float* h = (float*)dst;
            for (int r = 0; r < g.R; ++r) {
                // rows r of every a-block: pre blocks of `post` contiguous floats
                CUDA_TRY(cudaMemcpy2DAsync(h + (size_t)r * g.P, g.post * 4, pl->A[mode] + (size_t)r * g.post,
                                           (size_t)g.Rp * g.post * 4, g.post * 4, g.pre,
                                           cudaMemcpyDeviceToHost, s));
            }
            CUDA_TRY(cudaStreamSynchronize(s));
            return PASD_OK;
        }
        case PASD_STATE_E:
            if (pl->pad) return copy2d(pl->E, pl->D_real / pl->I_last_real, (int)pl->I_last_real, (int)pl->m[N - 1].I);
            if (bytes != (size_t)pl->D * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            CUDA_TRY(cudaMemcpyAsync(dst, pl->E, bytes, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            return PASD_OK;
        case PASD_STATE_Y: {
            if (bytes != (size_t)pl->D_real * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            if (!pl->y_tmp) CUDA_TRY(cudaMalloc(&pl->y_tmp, pl->D * 4));
            pasd_status st = read_scalars(pl, s);
            if (st != PASD_OK) return st;
            launch_export_y(pl->G[mode], pl->host_sc->T, pl->E, pl->sc, pl->y_tmp, pl->D, s);
            if (pl->pad) return copy2d(pl->y_tmp, pl->D_real / pl->I_last_real, (int)pl->I_last_real, (int)pl->m[N - 1].I);
            CUDA_TRY(cudaMemcpyAsync(dst, pl->y_tmp, bytes, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            return PASD_OK;
        }
        case PASD_STATE_MU: {
            if (bytes != 8) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            pasd_status st = read_scalars(pl, s);
            if (st != PASD_OK) return st;
            std::memcpy(dst, &pl->host_sc->mu, 8);
            return PASD_OK;
        }
        case PASD_STATE_KEPT: {
            if (bytes != (size_t)N * 4) return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            pasd_status st = read_scalars(pl, s);
            if (st != PASD_OK) return st;
            std::memcpy(dst, pl->host_sc->kept, bytes);
            return PASD_OK;
        }
        case PASD_STATE_TRACE: {
            pasd_status st = read_scalars(pl, s);
            if (st != PASD_OK) return st;
            size_t rec = PASD_TRACE_STRIDE * 8;
            if (bytes % rec != 0 || bytes / rec > (size_t)pl->host_sc->k)
                return fail(PASD_ERR_INVALID_ARG, "size mismatch");
            CUDA_TRY(cudaMemcpyAsync(dst, pl->trace, bytes, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            return PASD_OK;
        }
        default: return fail(PASD_ERR_INVALID_ARG, "unknown state item");
    }
}

// ---------------------------------------------------------------------------
// served path: continuous batching over per-solve streams
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// batched executor: the served path advances its batchable solves together, one
// launch per kernel of a loop body (grouped by the kernels' template
// parameters) for all of them, replayed as one captured graph per body
// ---------------------------------------------------------------------------
// A plan can join a batch when all its streaming kernels are the bulk-copy FP32
// ones that have batched forms (few-row modes run as their own launches).
// A-pass launches without a batched form (the tensor-core A-pass of mixed
// precision) run inside the batched body as launches of their own; the batched
// polar and SVT kernels are the FP32 ones, so FP64 eigen-solve plans run alone.
static bool batchable(const pasd_plan_t* pl) {
    return pl->arena && pl->tma && pl->n_ap_plain == 0 && !(pl->p.flags & PASD_F_FP64_EIG);
}

struct BatchLaunch {
    int k1 = 0, k2 = 0;          // A-pass: Rp, columns per thread; Vrot: RB, four-column path; fused: N, threads
    size_t ent = 0, map = 0;     // byte offsets of the entries and of the CTA -> entry map
    int grid = 0;
    size_t smem = 0;
};

struct BatchExec {
    std::vector<pasd_plan_t*> members;
    std::vector<char> host;      // staging of the device tables
    char* dev = nullptr;
    size_t dev_bytes = 0;
    size_t small_ent = 0;
    int n_small = 0;
    size_t polar_smem = 0, svt_smem = 0;
    std::vector<BatchLaunch> apass, vrot, fused, mpass, mplain, fin;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int num_sms = 0;
};

static size_t stage_bytes(std::vector<char>& h, size_t bytes, size_t align = 256) {
    size_t off = (h.size() + align - 1) / align * align;
    h.resize(off + bytes);
    return off;
}

// Groups entries by key; for each group lays out [entries][CTA -> entry map].
template <class Key, class Item>
static void layout_groups(BatchExec& b, std::vector<BatchLaunch>& out, const std::map<Key, std::vector<Item>>& groups,
                          size_t entry_bytes, int (*ctas)(const Item&), void (*fill)(void*, const Item&, int),
                          size_t (*smem)(const Item&), void (*keys)(const Key&, BatchLaunch&)) {
    out.clear();
    for (const auto& kv : groups) {
        BatchLaunch L;
        keys(kv.first, L);
        const size_t ent = stage_bytes(b.host, entry_bytes * kv.second.size(), 256);
        int start = 0;
        std::vector<int> owner;
        for (size_t e = 0; e < kv.second.size(); ++e) {
            const Item& it = kv.second[e];
            const int c = ctas(it);
            fill(b.host.data() + ent + e * entry_bytes, it, start);
            for (int q = 0; q < c; ++q) owner.push_back((int)e);
            start += c;
            L.smem = std::max(L.smem, smem(it));
        }
        if (start == 0) continue;
        const size_t map = stage_bytes(b.host, owner.size() * sizeof(int), 256);
        std::memcpy(b.host.data() + map, owner.data(), owner.size() * sizeof(int));
        L.ent = ent;
        L.map = map;
        L.grid = start;
        out.push_back(L);
    }
}

struct ApItem { const ApassTmaPlan* p; };
struct VrItem { VrotArgs a; };   // one rank bucket of a plan's modes
struct FuItem { const FusedTmaPlan* p; };
struct MpItem { const MpassTmaPlan* p; };
struct MqItem { const pasd_plan_t* pl; };
struct FiItem { const pasd_plan_t* pl; };

static void launch_batch_body(BatchExec& b, cudaStream_t s) {
    const char* d = b.dev;
    auto ent = [&](size_t off) { return static_cast<const void*>(d + off); };
    auto map = [&](size_t off) { return reinterpret_cast<const int*>(d + off); };
    launch_polar_batched(reinterpret_cast<const SmallBatchEntry*>(d + b.small_ent), b.n_small, b.polar_smem, s);
    for (const BatchLaunch& L : b.apass) launch_apass_batched(L.k1, L.k2, ent(L.ent), map(L.map), L.grid, L.smem, s);
    for (pasd_plan_t* pl : b.members) {
        for (int q = 0; q < pl->n_ap_tma; ++q)
            if (apass_batch_ctas(pl->ap_tma[q]) < 0) launch_apass_tma(pl->ap_tma[q], s);
        for (int n = 0; n < pl->N; ++n)
            if (pl->ap_small[n]) launch_apass_small(pl->ap[n], pl->ap_small_grid[n], s);
    }
    launch_svt_batched(reinterpret_cast<const SmallBatchEntry*>(d + b.small_ent), b.n_small, b.svt_smem, s);
    for (const BatchLaunch& L : b.vrot)
        launch_vrot_batched(L.k1, L.k2 != 0, reinterpret_cast<const VrotBatchEntry*>(d + L.ent), map(L.map), L.grid, s);
    for (const BatchLaunch& L : b.fused) launch_fused_batched(L.k1, ent(L.ent), map(L.map), L.grid, L.k2, L.smem, s);
    for (pasd_plan_t* pl : b.members)
        for (int n = 0; n < pl->N; ++n)
            if (pl->ap_small[n]) launch_mpass_small(pl->mp_small[n], pl->ap_small_grid[n], s);
    for (const BatchLaunch& L : b.mpass) launch_mpass_batched(ent(L.ent), map(L.map), L.grid, L.smem, s);
    for (const BatchLaunch& L : b.mplain)
        launch_mpass_plain_batched(reinterpret_cast<const MpassPlainBatchEntry*>(d + L.ent), map(L.map), L.grid, L.smem,
                                   s);
    for (const BatchLaunch& L : b.fin)
        launch_finalize_batched(reinterpret_cast<const FinBatchEntry*>(d + L.ent), map(L.map), L.grid, s);
}

static void batch_release(BatchExec& b) {
    if (b.exec) cudaGraphExecDestroy(b.exec);
    if (b.graph) cudaGraphDestroy(b.graph);
    b.exec = nullptr;
    b.graph = nullptr;
}

// Rebuilds the device tables and the body graph for the current members.
static bool batch_build(BatchExec& b, cudaStream_t s) {
    b.host.clear();
    if (b.members.empty()) { batch_release(b); return true; }
    // polar / SVT: one CTA per (solve, mode)
    {
        std::vector<SmallBatchEntry> e;
        b.polar_smem = b.svt_smem = 0;
        for (pasd_plan_t* pl : b.members) {
            for (int n = 0; n < pl->N; ++n) e.push_back(SmallBatchEntry{pl->small.m[n], pl->sc, n});
            b.polar_smem = std::max(b.polar_smem, polar_launch_smem(pl->small));
            b.svt_smem = std::max(b.svt_smem, svt_launch_smem(pl->small));
        }
        b.n_small = (int)e.size();
        b.small_ent = stage_bytes(b.host, e.size() * sizeof(SmallBatchEntry));
        std::memcpy(b.host.data() + b.small_ent, e.data(), e.size() * sizeof(SmallBatchEntry));
    }
    std::map<std::pair<int, int>, std::vector<ApItem>> ap;
    std::map<std::pair<int, int>, std::vector<VrItem>> vr;
    std::map<std::pair<int, int>, std::vector<FuItem>> fu;
    std::map<int, std::vector<MpItem>> mp;
    std::map<int, std::vector<MqItem>> mq;
    std::map<int, std::vector<FiItem>> fi;
    for (pasd_plan_t* pl : b.members) {
        for (int q = 0; q < pl->n_ap_tma; ++q)
            if (apass_batch_ctas(pl->ap_tma[q]) >= 0)
                ap[{apass_batch_rp(pl->ap_tma[q]), apass_tma_variant(pl->ap_tma[q])}].push_back(ApItem{pl->ap_tma[q]});
        {
            VrotArgs sub[PASD_MAXN];
            int rbs[PASD_MAXN];
            bool v4s[PASD_MAXN];
            const int ns = vrot_split(pl->vr, sub, rbs, v4s);
            for (int k = 0; k < ns; ++k) vr[{rbs[k], v4s[k] ? 1 : 0}].push_back(VrItem{sub[k]});
        }
        fu[{fused_batch_order(pl->tma), fused_batch_threads(pl->tma)}].push_back(FuItem{pl->tma});
        if (pl->n_mp_big > 0) {
            if (pl->mp_tma) mp[0].push_back(MpItem{pl->mp_tma});
            else mq[0].push_back(MqItem{pl});
        }
        fi[0].push_back(FiItem{pl});
    }
    auto pair_keys = [](const std::pair<int, int>& k, BatchLaunch& L) { L.k1 = k.first; L.k2 = k.second; };
    layout_groups<std::pair<int, int>, ApItem>(
        b, b.apass, ap, apass_batch_entry_bytes(), [](const ApItem& i) { return apass_batch_ctas(i.p); },
        [](void* e, const ApItem& i, int st) { apass_batch_fill(e, i.p, st); },
        [](const ApItem& i) { return apass_batch_smem(i.p); }, pair_keys);
    layout_groups<std::pair<int, int>, VrItem>(
        b, b.vrot, vr, sizeof(VrotBatchEntry), [](const VrItem& i) { return i.a.cta_start[i.a.N]; },
        [](void* e, const VrItem& i, int st) {
            VrotBatchEntry v{i.a, st};
            std::memcpy(e, &v, sizeof(v));
        },
        [](const VrItem&) { return (size_t)0; }, pair_keys);
    layout_groups<std::pair<int, int>, FuItem>(
        b, b.fused, fu, fused_batch_entry_bytes(), [](const FuItem& i) { return fused_batch_ctas(i.p); },
        [](void* e, const FuItem& i, int st) { fused_batch_fill(e, i.p, st); },
        [](const FuItem& i) { return fused_batch_smem(i.p); }, pair_keys);
    layout_groups<int, MpItem>(
        b, b.mpass, mp, mpass_batch_entry_bytes(), [](const MpItem& i) { return mpass_batch_ctas(i.p); },
        [](void* e, const MpItem& i, int st) { mpass_batch_fill(e, i.p, st); },
        [](const MpItem& i) { return mpass_batch_smem(i.p); }, [](const int&, BatchLaunch&) {});
    layout_groups<int, MqItem>(
        b, b.mplain, mq, sizeof(MpassPlainBatchEntry), [](const MqItem& i) { return i.pl->mpa.cta_start[i.pl->N]; },
        [](void* e, const MqItem& i, int st) {
            MpassPlainBatchEntry m{i.pl->mpa, st};
            std::memcpy(e, &m, sizeof(m));
        },
        [](const MqItem& i) { return i.pl->mp_smem; }, [](const int&, BatchLaunch&) {});
    layout_groups<int, FiItem>(
        b, b.fin, fi, sizeof(FinBatchEntry), [](const FiItem& i) { return finalize_ctas(i.pl->fin); },
        [](void* e, const FiItem& i, int st) {
            FinBatchEntry f{i.pl->fin, st};
            std::memcpy(e, &f, sizeof(f));
        },
        [](const FiItem&) { return (size_t)0; }, [](const int&, BatchLaunch&) {});
    if (b.host.size() > b.dev_bytes) {
        // grows by doubling: cudaFree waits for the whole device, other batches included
        const size_t want = std::max(b.host.size(), 2 * b.dev_bytes);
        if (b.dev) cudaFree(b.dev);
        b.dev = nullptr;
        b.dev_bytes = 0;
        if (cudaMalloc(&b.dev, want) != cudaSuccess) return false;
        b.dev_bytes = want;
        batch_release(b);   // the old graph's launches point into the freed table
    }
    if (cudaMemcpyAsync(b.dev, b.host.data(), b.host.size(), cudaMemcpyHostToDevice, s) != cudaSuccess) return false;
    if (cudaStreamSynchronize(s) != cudaSuccess) return false;
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return false;
    launch_batch_body(b, s);
    if (cudaStreamEndCapture(s, &g) != cudaSuccess) return false;
    // same launches as the graph in use (kernels and order), new grids and entries:
    // update the executable graph in place instead of instantiating a new one
    if (b.exec) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(b.exec, g, &info) == cudaSuccess) {
            cudaGraphDestroy(b.graph);
            b.graph = g;
            return true;
        }
        cudaGetLastError();
        batch_release(b);
    }
    b.graph = g;
    return cudaGraphInstantiate(&b.exec, b.graph, 0) == cudaSuccess;
}

// ---------------------------------------------------------------------------
// served path: continuous batching (one batch of the batchable solves on one
// stream, the others on a stream each)
// ---------------------------------------------------------------------------
struct Active {
    Job job;
    size_t footprint = 0;    // the plan's, taken at admission: once a result is
                             // published the caller may destroy the plan
    int launched = 0;
    bool flag_pending = false;
    bool started = false;
    bool batched = false;
    int batch = 0;           // which batch, when batched
    bool in_chunk = false;   // part of its batch's chunk in flight
};

static void publish(pasd_ctx* c, Active& a, pasd_result r) {
    r.latency_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - a.job.t_submit).count();
    r.batched = a.batched ? 1 : 0;
    pasd_plan_t* pl = a.job.plan;
    std::unique_lock<std::mutex> lk(c->mu);
    c->done[a.job.ticket] = r;
    c->state.erase(a.job.ticket);
    pl->busy = false;
    --pl->served;
    a.launched = -1;
}

// One batch of the served path: its members advance together on its stream, a
// chunk of loop bodies at a time; the tables are rebuilt (between chunks, with the
// stream idle) when members join or leave.
struct SubBatch {
    BatchExec b;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    bool pending = false;        // a chunk is in flight
    bool rebuild = false;
    int size() const { return (int)b.members.size(); }
};

static void worker_main(pasd_ctx* c) {
    cudaSetDevice(c->device);
    std::vector<Active> active;
    size_t in_use = 0;
    const bool use_batch = !c->no_batch;
    // A few batches on streams of their own: one batch would serialise the loop
    // body's phases, leaving the GPU to the one-CTA-per-mode kernels of all solves
    // at once; batches on separate streams overlap one's small kernels with
    // another's streaming passes, and the host waits on none of them.
    constexpr int kMaxBatches = 16;
    const int kBatches = c->n_batches;
    const int kBatchChunk = c->batch_chunk;
    SubBatch subs[kMaxBatches];
    for (;;) {
        // admission
        {
            std::unique_lock<std::mutex> lk(c->mu);
            bool idle = active.empty();
            if (idle && c->queue.empty()) {
                if (c->stop) break;
                c->cv.wait_for(lk, std::chrono::milliseconds(2));
                if (c->stop && c->queue.empty()) break;
            }
            for (auto it = c->queue.begin(); it != c->queue.end();) {
                pasd_plan_t* pl = it->plan;
                size_t need = pl->footprint;
                if (!pl->busy && in_use + need <= c->hbm_budget) {
                    Active a;
                    a.job = *it;
                    a.footprint = need;
                    pl->busy = true;
                    in_use += need;
                    c->state[it->ticket] = 1;
                    active.push_back(a);
                    it = c->queue.erase(it);
                } else {
                    ++it;
                }
            }
        }
        // start newly admitted solves: into the smallest batch when their kernels allow it
        for (auto& a : active) {
            if (a.started || a.launched < 0) continue;
            a.started = true;
            pasd_plan_t* pl = a.job.plan;
            pasd_status st = ensure_allocated(pl);
            cudaStream_t s = nullptr;
            if (st == PASD_OK) {
                a.batched = use_batch && batchable(pl);
                if (a.batched) {
                    int j = 0;
                    for (int q = 1; q < kBatches; ++q)
                        if (subs[q].size() < subs[j].size()) j = q;
                    SubBatch& sb = subs[j];
                    if (!sb.s) {
                        cudaStreamCreateWithFlags(&sb.s, cudaStreamNonBlocking);
                        cudaEventCreateWithFlags(&sb.ev, cudaEventDisableTiming);
                    }
                    a.batch = j;
                    s = sb.s;
                } else {
                    if (!pl->own_stream) cudaStreamCreateWithFlags(&pl->own_stream, cudaStreamNonBlocking);
                    s = pl->own_stream;
                }
                st = begin_impl(pl, a.job.T, s);   // after the batch's chunk in flight, if any
            }
            if (st != PASD_OK) {
                pasd_result r{};
                r.status = st;
                publish(c, a, r);
                continue;
            }
            if (a.batched) {
                subs[a.batch].b.members.push_back(pl);
                subs[a.batch].rebuild = true;
            }
        }
        bool progressed = false;
        // batches whose stream is idle: rebuild if needed, then the next chunk
        for (int j = 0; j < kBatches; ++j) {
            SubBatch& sb = subs[j];
            if (sb.pending || sb.b.members.empty()) continue;
            if (sb.rebuild) {
                sb.rebuild = false;
                if (!batch_build(sb.b, sb.s)) {
                    // no tables: the members continue on streams of their own
                    cudaStreamSynchronize(sb.s);
                    for (auto& a : active)
                        if (a.batched && a.batch == j && a.launched >= 0) {
                            a.batched = false;
                            pasd_plan_t* pl = a.job.plan;
                            if (!pl->own_stream) cudaStreamCreateWithFlags(&pl->own_stream, cudaStreamNonBlocking);
                        }
                    sb.b.members.clear();
                    batch_release(sb.b);
                    continue;
                }
            }
            for (int i = 0; i < kBatchChunk; ++i) {
                cudaGraphLaunch(sb.b.exec, sb.s);
                if (i == 0)
                    for (pasd_plan_t* pl : sb.b.members)
                        if (pl->skip_pending) {
                            // first body after pasd_begin: replace the provably idle bodies that follow
                            launch_idle_skip(pl->idle, pl->ctx->num_sms, sb.s);
                            pl->skip_pending = false;
                        }
            }
            for (pasd_plan_t* pl : sb.b.members)
                cudaMemcpyAsync(pl->host_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, sb.s);
            cudaEventRecord(sb.ev, sb.s);
            sb.pending = true;
            for (auto& a : active)
                if (a.batched && a.batch == j && a.launched >= 0) {
                    a.launched += kBatchChunk;
                    a.in_chunk = true;
                }
        }
        // the others: one chunk each, on their own streams
        for (auto& a : active) {
            if (a.launched < 0 || a.batched || a.flag_pending) continue;
            pasd_plan_t* pl = a.job.plan;
            int n = std::min(pl->p.check_every, pl->p.max_iter - a.launched);
            if (n > 0) {
                iterate_impl(pl, n, pl->own_stream);
                a.launched += n;
            }
            cudaMemcpyAsync(pl->host_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, pl->own_stream);
            cudaEventRecord(pl->ev, pl->own_stream);
            a.flag_pending = true;
        }
        // retire finished batch members once their batch's chunk has completed
        for (int j = 0; j < kBatches; ++j) {
            SubBatch& sb = subs[j];
            if (!sb.pending || cudaEventQuery(sb.ev) != cudaSuccess) continue;
            sb.pending = false;
            progressed = true;
            for (auto& a : active) {
                // only the members of the completed chunk have fresh flags (a solve
                // that joined meanwhile has not run a body yet)
                if (!a.batched || a.batch != j || a.launched < 0 || !a.in_chunk) continue;
                a.in_chunk = false;
                pasd_plan_t* pl = a.job.plan;
                if (pl->host_sc->done || a.launched >= pl->p.max_iter) {
                    pasd_result r{};
                    r.status = finish_impl(pl, a.job.L, a.job.E, &r, sb.s);
                    auto it = std::find(sb.b.members.begin(), sb.b.members.end(), pl);
                    if (it != sb.b.members.end()) sb.b.members.erase(it);
                    sb.rebuild = true;
                    publish(c, a, r);
                }
            }
        }
        // retire finished solo solves
        for (auto& a : active) {
            if (a.launched < 0 || a.batched) continue;
            pasd_plan_t* pl = a.job.plan;
            if (!a.flag_pending) continue;
            if (cudaEventQuery(pl->ev) != cudaSuccess) continue;
            a.flag_pending = false;
            progressed = true;
            if (pl->host_sc->done || a.launched >= pl->p.max_iter) {
                pasd_result r{};
                r.status = finish_impl(pl, a.job.L, a.job.E, &r, pl->own_stream);
                publish(c, a, r);
            }
        }
        for (auto it = active.begin(); it != active.end();) {
            if (it->launched < 0) {
                in_use -= it->footprint;
                it = active.erase(it);
            } else {
                ++it;
            }
        }
        if (!progressed && !active.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
    for (SubBatch& sb : subs) {
        if (sb.s) cudaStreamSynchronize(sb.s);
        batch_release(sb.b);
        if (sb.b.dev) cudaFree(sb.b.dev);
        if (sb.ev) cudaEventDestroy(sb.ev);
        if (sb.s) cudaStreamDestroy(sb.s);
    }
}

extern "C" pasd_status pasd_submit(pasd_ctx* c, pasd_plan_t* pl, const float* T, float* L,
                                   float* E, uint64_t* ticket) {
    if (!c || !pl || !T || !L || !E || !ticket) return fail(PASD_ERR_INVALID_ARG, "NULL argument");
    if (pl->ctx != c) return fail(PASD_ERR_INVALID_ARG, "plan belongs to another context");
    if (pl->footprint > c->hbm_budget) return fail(PASD_ERR_OOM, "plan footprint exceeds the HBM budget");
    std::unique_lock<std::mutex> lk(c->mu);
    if (c->queue.size() >= c->max_queue) return fail(PASD_ERR_BUSY, "submit queue is full");
    Job j;
    j.ticket = c->next_ticket++;
    j.plan = pl;
    j.T = T;
    j.L = L;
    j.E = E;
    j.t_submit = std::chrono::steady_clock::now();
    c->queue.push_back(j);
    c->state[j.ticket] = 0;
    ++pl->served;
    *ticket = j.ticket;
    if (!c->worker_started) {
        c->worker_started = true;
        c->worker = std::thread(worker_main, c);
    }
    lk.unlock();
    c->cv.notify_all();
    return PASD_OK;
}

extern "C" pasd_status pasd_poll(pasd_ctx* c, uint64_t ticket, pasd_result* out) {
    if (!c) return fail(PASD_ERR_INVALID_ARG, "ctx is NULL");
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->done.find(ticket);
    if (it != c->done.end()) {
        pasd_result r = it->second;
        c->done.erase(it);
        if (out) *out = r;
        return (pasd_status)r.status;
    }
    if (c->state.count(ticket)) return PASD_PENDING;
    return fail(PASD_ERR_UNKNOWN_TICKET, "unknown ticket");
}

extern "C" const char* pasd_status_string(pasd_status s) {
    switch (s) {
        case PASD_OK: return "PASD_OK";
        case PASD_PENDING: return "PASD_PENDING";
        case PASD_NOT_CONVERGED: return "PASD_NOT_CONVERGED";
        case PASD_ERR_INVALID_ARG: return "PASD_ERR_INVALID_ARG";
        case PASD_ERR_OOM: return "PASD_ERR_OOM";
        case PASD_ERR_CUDA: return "PASD_ERR_CUDA";
        case PASD_ERR_NONFINITE: return "PASD_ERR_NONFINITE";
        case PASD_ERR_TIMEOUT: return "PASD_ERR_TIMEOUT";
        case PASD_ERR_BUSY: return "PASD_ERR_BUSY";
        case PASD_ERR_UNKNOWN_TICKET: return "PASD_ERR_UNKNOWN_TICKET";
        case PASD_ERR_UNSUPPORTED: return "PASD_ERR_UNSUPPORTED";
    }
    return "unknown status";
}

extern "C" const char* pasd_last_error(void) { return g_last_error.c_str(); }
