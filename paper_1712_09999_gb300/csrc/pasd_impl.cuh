// Internal definitions shared by the PASD kernels and the host runtime.
//
// Notation follows the paper (Jiang & Ng, arXiv 1712.09999): mode n of an
// N-way C-order tensor has size I_n; pre_n = prod_{m<n} I_m, post_n =
// prod_{m>n} I_m, P_n = pre_n * post_n. The mode-n unfolding X_(n) (Sec. 2.1)
// is read in place as the 3-D view [pre_n, I_n, post_n]; its column index is
// j = a * post_n + b (C order over the other modes).
//
// Device-resident solver state of one plan (all float32 unless noted):
//   E                 D         sparse part
//   G_n               D each    G_n = T - E + Y_n / mu (the argument of Eq. 9 - Eq. 13);
//                               the multipliers are kept in this scaled, shifted form
//   U_n               I_n x Rp  active subspace (row-major, columns >= R_n are zero)
//   A_n               [pre_n][Rp][post_n]   A_n = U_n^T G_n, the SVT argument of Eq. 13
//   W_n, F_n, S_n     eigen-system of A_n A_n^T (R x R), SVT factors, kept count
//   Wz_n              I_n x Rp  U_n W diag(F) W^T, so that Z_n = fold_n(Wz_n A_n)
//   partial buffers   per-CTA Gram and G_n A_n^T sums, reduced in a fixed order
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define PASD_MAXN 8
#define PASD_MAXR 64

namespace pasd {

// Raises a kernel's dynamic shared-memory limit to at least `bytes` on the
// current device. The attribute is set once per (kernel, device, size) and
// remembered, so launches on the hot path make no driver call for it.
void set_smem_attr(const void* kernel, int bytes);


// Scalars that live on the device so that a captured iteration graph can be
// replayed without host involvement.
struct DevScalars {
    const float* T;        // observation (caller's device buffer)
    double mu;             // mu^k (used by every sub-step of iteration k)
    double t_norm_fro;     // ||T||_F
    int32_t k;             // completed loop bodies
    int32_t done;          // 1 -> every kernel returns immediately
    int32_t status;        // pasd_status once done
    int32_t kept[PASD_MAXN];
    double nuclear[PASD_MAXN];
    double res_inf, res_fro_rel, objective, l1_E, mu_used;
    int32_t nonfinite;
    int32_t skipped;       // idle loop bodies replaced by their closed form
    int32_t w_ident[PASD_MAXN];   // 1: the last SVT's eigenbasis W_n is exactly I (Urot = U)
};

struct ModeGeom {
    int64_t I, pre, post, P;
    int R, Rp;       // rank bound and its round-up to a multiple of 4
};

// ----------------------------------------------------------------------------
// A-pass: A_n = U_n^T G_n (+ per-CTA Gram partials of A_n A_n^T)
// ----------------------------------------------------------------------------
constexpr int AP_THREADS = 128;
constexpr int AP_BN = 256;       // columns of the unfolding per CTA
constexpr int AP_BK = 16;        // rows of the contraction per pipeline stage
constexpr int AP_STAGES = 4;

struct ApassArgs {
    const float* G;      // G_n (D floats)
    const float* U;      // I x Rp
    float* A;            // [pre][Rp][post]
    float* gram_part;    // [ncta][Rp][Rp]
    const DevScalars* sc;
    int64_t I, pre, post, P;
    int R, Rp;
    int ncta;
};

void launch_apass(const ApassArgs& a, cudaStream_t s);

// TMA-fed A-pass (post % 4 == 0, or post == 1 with I % 4 == 0): one launch per
// group of modes with the same padded rank; one CTA per task (column block).
constexpr int AT_STAGES = 2;
struct ApassTmaMode {
    int64_t I, pre, post, P;
    int BN;                // columns per task
    int nbb;               // tasks per a-row (post > 1)
    int rowmajor;          // post == 1
    float* A;              // [pre][Rp][post]
    float* gram_part;      // [tasks][Rp][Rp]
};
struct ApassTmaArgs {
    int count, Rp;
    DevScalars* sc;
    ApassTmaMode m[PASD_MAXN];
    int cta_start[PASD_MAXN + 1];
};
struct ApassTmaPlan;
// Arithmetic of a TMA-fed A-pass launch: FP32 FMAs, or the tensor cores
// (tcgen05, TF32 with the hi/lo split that keeps FP32 accuracy).
enum ApassKind { APASS_FFMA = 0, APASS_TC = 1 };
bool apass_tma_supported(int64_t I, int64_t post);
int apass_tma_tasks(int64_t I, int64_t pre, int64_t post, int kind);
// modes[0..count) index `a`; all share a[modes[0]].Rp. nullptr (with err) if a map is refused.
ApassTmaPlan* make_apass_tma(const ApassArgs* a, const int* modes, int count, int kind, int num_sms, char* err,
                             size_t errlen);
void launch_apass_tma(const ApassTmaPlan* p, cudaStream_t s);
// FMA kernel's columns per thread (0 for the tensor-core kernel); the setter
// accepts the default or half of it (an autotuner candidate)
int apass_tma_cols(const ApassTmaPlan* p);
int apass_tma_split(const ApassTmaPlan* p);
int apass_tma_variant(const ApassTmaPlan* p);   // columns per thread + 100 x row groups (batch key)
void apass_tma_set_cols(ApassTmaPlan* p, int nc, int ks = 1);
void destroy_apass_tma(ApassTmaPlan* p);
// All modes in as few launches as possible (one per distinct padded rank);
// returns the number of launches.
int launch_apass_modes(const ApassArgs* a, int N, cudaStream_t s);
size_t apass_smem_bytes(int Rp, bool rowmajor);
int apass_ncta(int64_t P);
// Modes with I_n <= 8 and Rp <= 8 (fewrow.cu): one thread per four columns, a
// fixed grid, one Gram partial (A-pass) or one G_n Vrot_n^T partial (M-pass)
// per CTA.
bool apass_small_supported(int64_t I, int Rp);
int apass_small_grid(int num_sms, int64_t P);
void launch_apass_small(const ApassArgs& a, int grid, cudaStream_t s);
struct MpassSmallArgs {
    const float* G;        // G_n (D floats)
    const float* V;        // Vrot_n, [pre][Rp][post]
    float* part;           // [grid][I][Rp]
    const DevScalars* sc;
    int64_t I, pre, post, P;
    int Rp, mode;
};
void launch_mpass_small(const MpassSmallArgs& m, int grid, cudaStream_t s);

// ----------------------------------------------------------------------------
// Small per-mode kernels (one CTA per mode): polar (U-step), SVT, finalize
// ----------------------------------------------------------------------------
struct SmallModeArgs {
    int64_t I;
    int R, Rp;
    double lambda;         // lambda_n
    float* U;              // I x Rp
    float* Urot;           // I x Rp: U W, the subspace in the SVT eigenbasis
    float* W;              // Rp x Rp (columns = eigenvectors, by descending eigenvalue)
    float* F;              // Rp
    float* sigma;          // Rp
    const float* gram_part; int n_gram;     // [n_gram][Rp][Rp]
    const float* Mred;     // I x Rp: G Vrot^T summed over regions (by finalize)
    float* scratch;        // 4 * I * Rp floats (U-step matrices when not in smem)
    int32_t* kept;         // device int (per mode)
    int polar_in_smem;     // 1: the U-step keeps its I x R matrices in shared memory
    int fp64_eig;          // 1: the R x R eigen-solves in double (PASD_F_FP64_EIG)
};

struct SmallArgs {
    int N;
    SmallModeArgs m[PASD_MAXN];
    DevScalars* sc;
};

void launch_polar(const SmallArgs& a, cudaStream_t s);
void launch_svt(const SmallArgs& a, cudaStream_t s);

struct FinalizeArgs {
    int N;
    DevScalars* sc;
    const float* part;     // [nparts][stride]: resmax, l1, nonfinite, res2[N]
    int nparts, stride;
    double lambda[PASD_MAXN];
    double rho, mu_max, tol;
    int stop_rule, max_iter;
    double* trace;         // [max_iter][13]
    // column-range partials of G_n Vrot_n^T from the M-pass, summed into Mred
    const float* mp_part[PASD_MAXN];   // [n_mp][I][Rp]
    int n_mp[PASD_MAXN];
    int64_t I[PASD_MAXN];
    int R[PASD_MAXN], Rp[PASD_MAXN];
    float* Mred[PASD_MAXN];            // [I][Rp]
};
size_t polar_smem_bytes(int maxRp, int64_t maxI, bool fp64);
void launch_finalize(const FinalizeArgs& a, cudaStream_t s);
void launch_init_state(DevScalars* sc, const float* T, double mu0, int N, float** U,
                       const int64_t* I, const int* R, const int* Rp, float** W, float** F,
                       float** Urot, int32_t* kept, cudaStream_t s);

// Idle-start skip (idle.cu): after the first loop body, replaces the bodies
// that provably keep V = E = 0 by their closed form.
struct IdleSkipArgs {
    DevScalars* sc;
    int N;
    const float* sigma[PASD_MAXN];   // singular values of U_n^T G_n, descending
    double lambda[PASD_MAXN];
    double rho, mu_max;
    int max_iter;
    double* trace;                   // [max_iter][13] or null
    const float* T;                  // plan copy of T
    float* G[PASD_MAXN];
    int64_t D;
    float* g;                        // device scalar: the factor g (0: no skip)
};
void launch_idle_skip(const IdleSkipArgs& a, int num_sms, cudaStream_t s);

struct VrotMode {
    const float* A;        // [pre][Rp][post]
    float* V;              // [pre][Rp][post]
    const float* W;        // Rp x Rp
    const float* F;        // Rp
    int64_t P, post;
    int R, Rp;
    int mode;              // index of the mode in the plan (its kept count)
};
struct VrotArgs {
    int N;
    const DevScalars* sc;
    VrotMode m[PASD_MAXN];
    int cta_start[PASD_MAXN + 1];
};
// One launch per rank bucket of the modes (a mode's loops are sized by its own
// bucket); returns the number of launches.
int launch_vrot(const VrotArgs& a, cudaStream_t s);
// The modes of `a` split by rank bucket: sub-arguments, bucket and whether the
// four-column path is needed, at most one per bucket; returns their number.
int vrot_split(const VrotArgs& a, VrotArgs* out, int* rb_out, bool* v4_out);
// CTAs the Vrot launch gives a mode of P columns (maxRp: the largest Rp of the plan)
int vrot_ctas(int64_t P, int64_t post, int maxRp);
void launch_norm_fro(const float* T, int64_t D, float* part, int nparts, DevScalars* sc,
                     cudaStream_t s);
void launch_export_y(const float* G, const float* T, const float* E, const DevScalars* sc,
                     float* Y, int64_t D, cudaStream_t s);

// ----------------------------------------------------------------------------
// M-pass: M_n = G_(n) Vrot_n^T over the kept rows (the next U-step's product),
// per column range partial sums part[range][I][Rp], summed by the finalize kernel.
// ----------------------------------------------------------------------------
constexpr int MP_THREADS = 256;
constexpr int MP_CB = 32;        // unfolding columns per pipeline stage
constexpr int MP_STAGES = 3;

struct MpassMode {
    const float* G;        // G_n (D floats)
    const float* V;        // Vrot_n, [pre][Rp][post]
    float* part;           // [ncg][I][Rp]
    int64_t I, post, P;
    int64_t cols_per_cg;   // unfolding columns per range (a multiple of MP_CB)
    int Rp, IS, nstrips, ncg, variant;
};
struct MpassArgs {
    int N;
    const DevScalars* sc;
    MpassMode m[PASD_MAXN];
    int cta_start[PASD_MAXN + 1];   // CTA b works on mode k with cta_start[k] <= b < cta_start[k+1]
};
size_t mpass_smem_bytes(int IS, int Rp, int variant);
int mpass_variant(int64_t I, int64_t post);
int mpass_strip_rows(int64_t I, int Rp);
int mpass_ctas_per_sm(size_t smem);

// TMA-fed M-pass (post == 1 with I % 4 == 0, or post % 4 == 0 and post >= MP_CB):
// one launch for all modes; CTA = (row strip, range of cpr chunks of MP_CB columns).
constexpr int MT_STAGES = 3;
struct MpassTmaMode {
    int64_t I, pre, post, P;
    int Rp, IS, nstrips;
    int nch;               // chunks (post > 1: pre * nbb; post == 1: ceil(pre / MP_CB))
    int nbb;               // chunks per a-row (post > 1)
    int cpr;               // chunks per column range
    int ncg;               // column ranges
    int rowmajor;          // post == 1
    float* part;           // [ncg][I][Rp]
};
struct MpassTmaArgs {
    int N;
    DevScalars* sc;
    MpassTmaMode m[PASD_MAXN];
    int cta_start[PASD_MAXN + 1];
};
struct MpassTmaPlan;
bool mpass_tma_supported(int64_t I, int64_t post);
int mpass_tma_chunks(int64_t pre, int64_t post);
size_t mpass_tma_smem_bytes(int IS, int Rp);
int mpass_tma_ctas_per_sm(size_t smem);
MpassTmaPlan* make_mpass_tma(const MpassTmaArgs& a, const float* const* G, const float* const* V, size_t smem,
                             char* err, size_t errlen);
void launch_mpass_tma(const MpassTmaPlan* p, cudaStream_t s);
void destroy_mpass_tma(MpassTmaPlan* p);
void launch_mpass(const MpassArgs& a, size_t smem, cudaStream_t s);

// ----------------------------------------------------------------------------
// Fused elementwise pass: Z_n, E-step (Eq. 15), multipliers and residuals, over
// power-of-two tiles ("boxes").
// ----------------------------------------------------------------------------
constexpr int FU_THREADS = 256;

struct FusedGeom {
    int N;
    int64_t I[PASD_MAXN];
    int64_t stride[PASD_MAXN];     // element stride of mode n (= post_n)
    int64_t astr[PASD_MAXN][PASD_MAXN];  // for mode n, stride of mode m<n inside pre_n
    int Rp[PASD_MAXN];
    int b[PASD_MAXN], sh[PASD_MAXN];     // box extents (powers of two) and log2
    int esh[PASD_MAXN];                  // bit offset of l_m inside the element index e
    int csh[PASD_MAXN][PASD_MAXN];       // for mode n: bit offset of l_m (m != n) inside c
    int C[PASD_MAXN];                    // B / b_n
    int B;                               // elements per tile
    int mb[PASD_MAXN];                   // micro-box extent per mode (1 or 2), prod = B / FU_THREADS
    int mbsh[PASD_MAXN];                 // bit offset of the micro-box coordinate in the thread id
    int64_t nt[PASD_MAXN];               // tiles per mode
    int Q[PASD_MAXN];                    // region grid
    int nregions;
    int as_off[PASD_MAXN], ws_off[PASD_MAXN];   // smem layout (floats)
    int smem_floats;
    // TMA-pipelined variant (two stages of [Xs | As_n | Ws_n], see fused_tma.cu)
    int tma;                             // 1 when the TMA kernel is used
    int nthreads;                        // B / 8
    int split0;                          // 1: a thread's two element groups lie B / 2 apart
                                         // (mode 0), not b_{N-2} / 2 apart along mode N-2
    int stage_floats;                    // floats per stage
    int xs_off;                          // element tiles (T, E, G_0..G_{N-1}) inside a stage
    uint32_t stage_tx_bytes;             // bytes one stage's TMA loads deliver
    uint32_t out_tx_bytes;               // bytes of the Vrot / Urot loads only (output pass)
};

struct FusedArgs {
    FusedGeom g;
    DevScalars* sc;
    float* E;
    float* G[PASD_MAXN];
    const float* A[PASD_MAXN];      // Vrot_n = diag(F) W^T A_n  (rows >= kept are zero)
    const float* Wz[PASD_MAXN];     // Urot_n = U_n W           (Z_n = Urot Vrot)
    float* part;           // [nregions][stride] reduction partials
    int part_stride;
    double rho, mu_max;
    // output mode (writes L = sum alpha_n Z_n / sum alpha_n, no state update)
    int output;
    float* L;
    float alpha_w[PASD_MAXN];
    // test hook of the TMA pass: issue no bulk copy (nothing is ever in flight),
    // and give up a wait after wait_polls polls (0: kWaitPolls)
    int test_no_copy;
    uint32_t wait_polls;
};

bool plan_fused_geom(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                     size_t smem_limit);
void launch_fused(const FusedArgs& a, cudaStream_t s);

// TMA-fed, double-buffered version of the fused pass (N <= 4, I_N % 4 == 0).
// The element tiles come from plan-owned buffers (T is copied at begin), so the
// tensor maps are fixed for the life of the plan.
struct FusedTmaPlan;
bool plan_fused_tma(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                    size_t smem_limit);
// Encodes the tensor maps; returns false if the driver refuses one.
FusedTmaPlan* make_fused_tma(const FusedArgs& a, const float* T_copy, char* err, size_t errlen);
void destroy_fused_tma(FusedTmaPlan* p);
void launch_fused_tma(FusedTmaPlan* p, int output, float* L, cudaStream_t s);

// ----------------------------------------------------------------------------
// Batched launches: one launch runs one kernel of a loop body for many solves.
// Each entry holds one solve's arguments for that kernel (and, for the bulk-copy
// kernels, its tensor maps, read from global memory); `block_entry` maps each
// CTA of the batched grid to its entry, whose CTAs begin at `start`. An entry's
// CTAs do exactly the work of that solve's own launch, so the results are the
// same bit for bit.
// ----------------------------------------------------------------------------
struct SmallBatchEntry {        // polar and SVT: one CTA per (solve, mode)
    SmallModeArgs m;
    DevScalars* sc;
    int mode;
};
struct FinBatchEntry {
    FinalizeArgs a;
    int start;
};
struct VrotBatchEntry {
    VrotArgs a;
    int start;
};
size_t polar_launch_smem(const SmallArgs& a);
size_t svt_launch_smem(const SmallArgs& a);
int finalize_ctas(const FinalizeArgs& a);
void launch_polar_batched(const SmallBatchEntry* e, int n, size_t smem, cudaStream_t s);
void launch_svt_batched(const SmallBatchEntry* e, int n, size_t smem, cudaStream_t s);
void launch_finalize_batched(const FinBatchEntry* e, const int* block_entry, int grid, cudaStream_t s);
void launch_vrot_batched(int rb, bool v4, const VrotBatchEntry* e, const int* block_entry, int grid, cudaStream_t s);
// bulk-copy kernels: entries are opaque here (filled by their files)
size_t fused_batch_entry_bytes();
int fused_batch_order(const FusedTmaPlan* p);   // N + 8 split0: one kernel per value
int fused_batch_ctas(const FusedTmaPlan* p);
int fused_batch_threads(const FusedTmaPlan* p);
size_t fused_batch_smem(const FusedTmaPlan* p);
void fused_batch_fill(void* entry, const FusedTmaPlan* p, int start);
void launch_fused_batched(int order, const void* entries, const int* block_entry, int grid, int threads, size_t smem,
                          cudaStream_t s);
size_t apass_batch_entry_bytes();
int apass_batch_rp(const ApassTmaPlan* p);
int apass_batch_ctas(const ApassTmaPlan* p);     // -1: not an FMA plan (not batched)
size_t apass_batch_smem(const ApassTmaPlan* p);
void apass_batch_fill(void* entry, const ApassTmaPlan* p, int start);
// every entry of one launch has padded rank Rp and variant `var` (apass_tma_variant)
void launch_apass_batched(int Rp, int var, const void* entries, const int* block_entry, int grid, size_t smem,
                          cudaStream_t s);
struct MpassPlainBatchEntry {   // the M-pass without bulk copies
    MpassArgs a;
    int start;
};
void launch_mpass_plain_batched(const MpassPlainBatchEntry* e, const int* block_entry, int grid, size_t smem,
                                cudaStream_t s);
size_t mpass_batch_entry_bytes();
int mpass_batch_ctas(const MpassTmaPlan* p);
size_t mpass_batch_smem(const MpassTmaPlan* p);
void mpass_batch_fill(void* entry, const MpassTmaPlan* p, int start);
void launch_mpass_batched(const void* entries, const int* block_entry, int grid, size_t smem, cudaStream_t s);

}  // namespace pasd
