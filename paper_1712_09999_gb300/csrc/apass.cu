// A-pass: the mode-n product A_n = U_n^T G_n of the V-step (Eq. 13), read in
// place from the mode-n unfolding of G_n (Sec. 2.1) with no materialised
// permutation, plus per-CTA partial sums of the Gram matrix A_n A_n^T used by
// the SVT (definition after Eq. 13).
//
// G_(n) is viewed as [pre][I][post]. A CTA owns AP_BN consecutive unfolding
// columns j (crossing a-boundaries is allowed) and streams the whole
// contraction dimension I through a cp.async pipeline in chunks of AP_BK rows:
//   post > 1 : a chunk is AP_BK rows of contiguous columns  -> smem [k][col]
//   post == 1: a chunk is AP_BK contiguous floats per column -> smem [col][k]
// Each thread accumulates 2 columns x Rp outputs in FP32 registers (FFMA); U
// is broadcast from shared memory. Columns past P and rows past I are zero-filled
// by the copy, so they contribute nothing to A or to the Gram sums.
#include "pasd_impl.cuh"
#include "tc.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cstring>

namespace pasd {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int n>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(n)); }

// Layout variants: 0 = strided columns, 16-byte copies (post % 4 == 0)
//                  1 = strided columns, 4-byte copies
//                  2 = contiguous rows (post == 1), 16-byte copies (I % 4 == 0)
//                  3 = contiguous rows (post == 1), 4-byte copies
template <int V>
struct ApLayout {
    static constexpr bool rowmajor = (V >= 2);
    static constexpr int gs_ld = rowmajor ? (AP_BK + 4) : (AP_BN + 4);
    static constexpr int gs_stage = rowmajor ? AP_BN * gs_ld : AP_BK * gs_ld;
};

// Shared memory of the Gram partial reduction with NT threads (after the A tile
// [AP_BN][RP + 4]).
static constexpr inline __host__ __device__ int gram_red_floats(int RP, int NT) {
    const int nb = RP / 4, nbt = nb * (nb + 1) / 2;
    const int nsl = nbt >= NT ? 1 : NT / nbt;
    return nsl * nbt * 16;
}

// Per-CTA Gram partial: the sum over this CTA's BN columns of A[:, j] A[:, j]^T;
// thread t holds columns t + NT q (q < CPT) in acc[q] (zero for absent columns).
// 4 x 4 blocks on and above the diagonal, each summed over NSL column slices
// and then over the slices in order (deterministic); written with its mirror.
// `smem` must be free (no copy in flight) and hold BN (RP + 4) +
// gram_red_floats(RP, NT) floats.
// BAR = 0 synchronises the whole CTA; BAR > 0 only the NT threads that run the
// epilogue (named barrier BAR), whose index among them is t.
template <int BAR, int NT>
__device__ __forceinline__ void epi_sync() {
    if (BAR == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;\n" ::"n"(BAR), "n"(NT) : "memory");
}
template <int RP, int NT, int CPT, int BN = AP_BN, int BAR = 0>
__device__ __forceinline__ void gram_epilogue(const float (&acc)[CPT][RP], float* smem, float* gp,
                                              int t = threadIdx.x) {
    constexpr int ALD = RP + 4;
    float* As = smem;   // [BN][ALD]
#pragma unroll
    for (int q = 0; q < CPT; ++q)
#pragma unroll
        for (int r4 = 0; r4 < RP / 4; ++r4)
            *reinterpret_cast<float4*>(As + (t + NT * q) * ALD + 4 * r4) =
                make_float4(acc[q][4 * r4], acc[q][4 * r4 + 1], acc[q][4 * r4 + 2], acc[q][4 * r4 + 3]);
    constexpr int NB = RP / 4;
    constexpr int NBT = NB * (NB + 1) / 2;
    constexpr int NSL = NBT >= NT ? 1 : NT / NBT;
    float* red = smem + BN * ALD;
    epi_sync<BAR, NT>();
    for (int w = t; w < NBT * NSL; w += NT) {
        int blk = w % NBT, sl = w / NBT;
        int bi = 0, rem = blk;
        while (rem >= NB - bi) { rem -= NB - bi; ++bi; }
        int bj = bi + rem;
        float g[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = 0.f;
        for (int c = sl; c < BN; c += NSL) {
            float4 x = *reinterpret_cast<const float4*>(As + c * ALD + 4 * bi);
            float4 y = *reinterpret_cast<const float4*>(As + c * ALD + 4 * bj);
            float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) g[p * 4 + q] = fmaf(xs[p], ys[q], g[p * 4 + q]);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) red[(sl * NBT + blk) * 16 + q] = g[q];
    }
    epi_sync<BAR, NT>();
    for (int o = t; o < NBT * 16; o += NT) {
        int blk = o / 16, q = o % 16;
        float sum = 0.f;
        for (int sl = 0; sl < NSL; ++sl) sum += red[(sl * NBT + blk) * 16 + q];
        int bi = 0, rem = blk;
        while (rem >= NB - bi) { rem -= NB - bi; ++bi; }
        int bj = bi + rem;
        int r = 4 * bi + q / 4, c = 4 * bj + q % 4;
        gp[r * RP + c] = sum;
        gp[c * RP + r] = sum;
    }
}

size_t apass_smem_bytes(int Rp, bool rowmajor) {
    size_t gs = (size_t)AP_STAGES * (rowmajor ? AP_BN * (AP_BK + 4) : AP_BK * (AP_BN + 4));
    size_t us = (size_t)AP_STAGES * AP_BK * Rp;
    size_t pipe = gs + us;
    size_t epi = (size_t)AP_BN * (Rp + 4) + gram_red_floats(Rp, AP_THREADS);
    return 4 * (pipe > epi ? pipe : epi);
}

int apass_ncta(int64_t P) { return (int)((P + AP_BN - 1) / AP_BN); }

template <int RP, int V>
__device__ __forceinline__ void apass_body(const ApassArgs& a, int cta, float* smem) {
    using L = ApLayout<V>;
    float* Gs = smem;
    float* Us = smem + AP_STAGES * L::gs_stage;

    const int t = threadIdx.x;
    const int64_t j0 = (int64_t)cta * AP_BN;
    const int64_t I = a.I, post = a.post, P = a.P;
    const float* __restrict__ G = a.G;
    const int nk = (int)((I + AP_BK - 1) / AP_BK);

    // per-thread source column bases for the copies
    int64_t cbase[2];
    bool cval[2];
    if (V == 0) {
        int64_t j = j0 + 4 * (t & 63);
        cval[0] = j < P;
        int64_t aa = cval[0] ? j / post : 0, bb = cval[0] ? j % post : 0;
        cbase[0] = aa * I * post + bb;
        cval[1] = false; cbase[1] = 0;
    } else if (V == 1) {
        for (int h = 0; h < 2; ++h) {
            int64_t j = j0 + t + 128 * h;
            cval[h] = j < P;
            int64_t aa = cval[h] ? j / post : 0, bb = cval[h] ? j % post : 0;
            cbase[h] = aa * I * post + bb;
        }
    } else {
        cbase[0] = cbase[1] = 0; cval[0] = cval[1] = true;
    }

    auto issue = [&](int kc, int st) {
        float* gs = Gs + st * L::gs_stage;
        const int64_t i0 = (int64_t)kc * AP_BK;
        if (V == 0) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                int row = (t >> 6) + 2 * s;
                int64_t i = i0 + row;
                bool ok = cval[0] && i < I;
                const float* src = ok ? G + cbase[0] + i * post : G;
                cp_async16(gs + row * L::gs_ld + 4 * (t & 63), src, ok ? 16 : 0);
            }
        } else if (V == 1) {
#pragma unroll 8
            for (int s = 0; s < 32; ++s) {
                int row = s >> 1, h = s & 1;
                int64_t i = i0 + row;
                bool ok = cval[h] && i < I;
                const float* src = ok ? G + cbase[h] + i * post : G;
                cp_async4(gs + row * L::gs_ld + t + 128 * h, src, ok ? 4 : 0);
            }
        } else if (V == 2) {
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                int n = (t >> 2) + 32 * s;
                int ch = t & 3;
                int64_t j = j0 + n, i = i0 + 4 * ch;
                bool ok = j < P && i < I;
                const float* src = ok ? G + j * I + i : G;
                cp_async16(gs + n * L::gs_ld + 4 * ch, src, ok ? 16 : 0);
            }
        } else {
#pragma unroll 8
            for (int s = 0; s < 32; ++s) {
                int n = (t >> 4) + 8 * s;
                int kk = t & 15;
                int64_t j = j0 + n, i = i0 + kk;
                bool ok = j < P && i < I;
                const float* src = ok ? G + j * I + i : G;
                cp_async4(gs + n * L::gs_ld + kk, src, ok ? 4 : 0);
            }
        }
        // U rows i0 .. i0 + AP_BK (Rp floats each, 16-byte aligned)
        float* us = Us + st * AP_BK * RP;
        for (int q = t; q < AP_BK * RP / 4; q += AP_THREADS) {
            int k = q / (RP / 4), c4 = q % (RP / 4);
            int64_t i = i0 + k;
            bool ok = i < I;
            const float* src = ok ? a.U + i * RP + 4 * c4 : a.U;
            cp_async16(us + k * RP + 4 * c4, src, ok ? 16 : 0);
        }
    };

    float acc[2][RP];
    float* acc0 = acc[0];
    float* acc1 = acc[1];
#pragma unroll
    for (int r = 0; r < RP; ++r) { acc0[r] = 0.f; acc1[r] = 0.f; }

#pragma unroll
    for (int s = 0; s < AP_STAGES - 1; ++s) {
        if (s < nk) issue(s, s);
        cp_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        cp_wait<AP_STAGES - 2>();
        __syncthreads();
        {
            int nxt = kc + AP_STAGES - 1;
            if (nxt < nk) issue(nxt, nxt % AP_STAGES);
            cp_commit();
        }
        const int st = kc % AP_STAGES;
        const float* gs = Gs + st * L::gs_stage;
        const float* us = Us + st * AP_BK * RP;
        if (!L::rowmajor) {
#pragma unroll 4
            for (int k = 0; k < AP_BK; ++k) {
                float g0 = gs[k * L::gs_ld + t];
                float g1 = gs[k * L::gs_ld + t + 128];
                const float4* u4 = reinterpret_cast<const float4*>(us + k * RP);
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4) {
                    float4 u = u4[r4];
                    acc0[4 * r4 + 0] = fmaf(g0, u.x, acc0[4 * r4 + 0]);
                    acc0[4 * r4 + 1] = fmaf(g0, u.y, acc0[4 * r4 + 1]);
                    acc0[4 * r4 + 2] = fmaf(g0, u.z, acc0[4 * r4 + 2]);
                    acc0[4 * r4 + 3] = fmaf(g0, u.w, acc0[4 * r4 + 3]);
                    acc1[4 * r4 + 0] = fmaf(g1, u.x, acc1[4 * r4 + 0]);
                    acc1[4 * r4 + 1] = fmaf(g1, u.y, acc1[4 * r4 + 1]);
                    acc1[4 * r4 + 2] = fmaf(g1, u.z, acc1[4 * r4 + 2]);
                    acc1[4 * r4 + 3] = fmaf(g1, u.w, acc1[4 * r4 + 3]);
                }
            }
        } else {
#pragma unroll 1
            for (int k4 = 0; k4 < AP_BK / 4; ++k4) {
                float4 g0v = *reinterpret_cast<const float4*>(gs + t * L::gs_ld + 4 * k4);
                float4 g1v = *reinterpret_cast<const float4*>(gs + (t + 128) * L::gs_ld + 4 * k4);
                float g0s[4] = {g0v.x, g0v.y, g0v.z, g0v.w};
                float g1s[4] = {g1v.x, g1v.y, g1v.z, g1v.w};
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4* u4 = reinterpret_cast<const float4*>(us + (4 * k4 + kk) * RP);
                    float g0 = g0s[kk], g1 = g1s[kk];
#pragma unroll
                    for (int r4 = 0; r4 < RP / 4; ++r4) {
                        float4 u = u4[r4];
                        acc0[4 * r4 + 0] = fmaf(g0, u.x, acc0[4 * r4 + 0]);
                        acc0[4 * r4 + 1] = fmaf(g0, u.y, acc0[4 * r4 + 1]);
                        acc0[4 * r4 + 2] = fmaf(g0, u.z, acc0[4 * r4 + 2]);
                        acc0[4 * r4 + 3] = fmaf(g0, u.w, acc0[4 * r4 + 3]);
                        acc1[4 * r4 + 0] = fmaf(g1, u.x, acc1[4 * r4 + 0]);
                        acc1[4 * r4 + 1] = fmaf(g1, u.y, acc1[4 * r4 + 1]);
                        acc1[4 * r4 + 2] = fmaf(g1, u.z, acc1[4 * r4 + 2]);
                        acc1[4 * r4 + 3] = fmaf(g1, u.w, acc1[4 * r4 + 3]);
                    }
                }
            }
        }
    }
    cp_wait<0>();
    __syncthreads();

    // ---- store A (layout [pre][Rp][post]) ----
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float* acc = h ? acc1 : acc0;
        int64_t j = j0 + t + 128 * h;
        if (j < P) {
            if (L::rowmajor) {
                float4* dst = reinterpret_cast<float4*>(a.A + j * RP);
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4)
                    dst[r4] = make_float4(acc[4 * r4], acc[4 * r4 + 1], acc[4 * r4 + 2], acc[4 * r4 + 3]);
            } else {
                int64_t aa = j / post, bb = j % post;
                float* dst = a.A + aa * RP * post + bb;
#pragma unroll
                for (int r = 0; r < RP; ++r) dst[(int64_t)r * post] = acc[r];
            }
        }
    }

    gram_epilogue<RP, AP_THREADS, 2>(acc, smem, a.gram_part + (size_t)cta * RP * RP);
}

static int apass_variant(const ApassArgs& a) {
    if (a.post == 1) return (a.I % 4 == 0) ? 2 : 3;
    return (a.post % 4 == 0) ? 0 : 1;
}

// One launch covers every mode with the same padded rank: CTAs
// [cta_start[k], cta_start[k+1]) work on mode group member k, so the modes'
// products run concurrently.
struct ApassMulti {
    int count;
    ApassArgs m[PASD_MAXN];
    int variant[PASD_MAXN];
    int cta_start[PASD_MAXN + 1];
};

template <int RP>
__global__ void __launch_bounds__(AP_THREADS) apass_kernel(const ApassMulti mm) {
    extern __shared__ __align__(16) float smem[];
    int k = 0;
    while (k + 1 < mm.count && (int)blockIdx.x >= mm.cta_start[k + 1]) ++k;
    const ApassArgs& a = mm.m[k];
    if (a.sc->done) return;
    const int cta = blockIdx.x - mm.cta_start[k];
    switch (mm.variant[k]) {
        case 0: apass_body<RP, 0>(a, cta, smem); break;
        case 1: apass_body<RP, 1>(a, cta, smem); break;
        case 2: apass_body<RP, 2>(a, cta, smem); break;
        default: apass_body<RP, 3>(a, cta, smem); break;
    }
}

template <int RP>
static void launch_rp(const ApassMulti& mm, cudaStream_t s) {
    size_t smem = std::max(apass_smem_bytes(RP, false), apass_smem_bytes(RP, true));
    set_smem_attr((const void*)apass_kernel<RP>, (int)smem);
    apass_kernel<RP><<<mm.cta_start[mm.count], AP_THREADS, smem, s>>>(mm);
}

static void launch_multi(const ApassMulti& mm, int Rp, cudaStream_t s) {
    switch (Rp) {
        case 4: launch_rp<4>(mm, s); break;
        case 8: launch_rp<8>(mm, s); break;
        case 12: launch_rp<12>(mm, s); break;
        case 16: launch_rp<16>(mm, s); break;
        case 20: launch_rp<20>(mm, s); break;
        case 24: launch_rp<24>(mm, s); break;
        case 28: launch_rp<28>(mm, s); break;
        case 32: launch_rp<32>(mm, s); break;
        case 40: launch_rp<40>(mm, s); break;
        case 48: launch_rp<48>(mm, s); break;
        case 56: launch_rp<56>(mm, s); break;
        case 64: launch_rp<64>(mm, s); break;
        default: break;
    }
}

int launch_apass_modes(const ApassArgs* a, int N, cudaStream_t s) {
    bool done[PASD_MAXN] = {false};
    int launches = 0;
    for (int n = 0; n < N; ++n) {
        if (done[n]) continue;
        ApassMulti mm{};
        mm.cta_start[0] = 0;
        for (int k = n; k < N; ++k) {
            if (done[k] || a[k].Rp != a[n].Rp) continue;
            done[k] = true;
            mm.m[mm.count] = a[k];
            mm.variant[mm.count] = apass_variant(a[k]);
            mm.cta_start[mm.count + 1] = mm.cta_start[mm.count] + a[k].ncta;
            ++mm.count;
        }
        launch_multi(mm, a[n].Rp, s);
        ++launches;
    }
    return launches;
}

void launch_apass(const ApassArgs& a, cudaStream_t s) { launch_apass_modes(&a, 1, s); }

// ---------------------------------------------------------------------------
// TMA-fed A-pass. The G tile of each pipeline stage arrives by one bulk tensor
// copy (and the U rows by another), so a stage costs one issuing thread instead
// of a copy instruction per 16 bytes per thread, and the copies stay out of the
// load/store pipe the FMA loop reads shared memory through.
//   post > 1 : a task is BN consecutive columns inside one a-row of the
//              unfolding (BN = min(256, post)); the tile is [k][col], dense.
//   post == 1: a task is 256 consecutive columns (rows of G); the tile is
//              [col][k] with the 64-byte swizzle (16-byte group g of row c sits
//              at g ^ ((c >> 1) & 3)), so the float4 reads below are conflict-free.
// Each column of A accumulates over k in the same order as in the cp.async
// kernel, so A is identical; the Gram partials group the columns differently.
// ---------------------------------------------------------------------------
struct ApassTmaMaps {
    CUtensorMap g[PASD_MAXN];
    CUtensorMap u[PASD_MAXN];
};

struct ApassTmaPlan {
    ApassTmaMaps maps;
    ApassTmaArgs args;
    size_t smem;
    int kind;      // ApassKind
    int grid;      // persistent grid of the tensor-core kernel (one CTA per SM)
    int nc;        // FMA kernel: columns per thread
    int ks;        // FMA kernel: thread groups splitting each stage's rows (1 or 2)
    size_t pipe_floats, epi_base_floats;   // shared-memory parts independent of nc
};

// Stage stride in floats: 512-byte multiples, the period of the 64-byte swizzle,
// so every stage's G tile starts on a swizzle boundary.
static inline __host__ __device__ int at_stage_floats(int BN, int RP) {
    return (AP_BK * BN + AP_BK * RP + 127) / 128 * 128;
}

// Columns per thread: by default four while the 4 x RP accumulators fit in
// registers, two beyond; the autotuner may halve it (twice the warps per CTA,
// half the accumulators per thread: more latency hiding, less reuse of each
// broadcast U row).
template <int RP> struct AtShape {
    static constexpr int COLS = RP <= 40 ? 4 : 2;
    static constexpr int THREADS = AP_BN / COLS;
};

// KS = 2 splits every stage's AP_BK rows between two groups of NT threads that
// hold the same columns (twice the warps for the same tiles and registers per
// thread); group 1 hands its sums to group 0 through shared memory at the end,
// and A = (group 0's rows) + (group 1's rows) in that order.
// Resident CTAs the register budget is sized for: as many as hold the
// accumulators and about 48 more registers a thread, at most 4.
static constexpr inline __host__ __device__ int at_min_blocks(int RP, int NC, int KS) {
    return KS == 1 ? 0 : (65536 / ((AP_BN / NC) * KS * (NC * RP + 48)) < 1 ? 1
                          : 65536 / ((AP_BN / NC) * KS * (NC * RP + 48)) > 4 ? 4
                          : 65536 / ((AP_BN / NC) * KS * (NC * RP + 48)));
}

// The row-group split is offered up to this padded rank: beyond it the
// accumulators of the default columns do not fit the register budget of
// four resident CTAs.
constexpr int kSplitMaxRp = 24;

template <int RP, int NC, int KS>
__device__ __forceinline__ void apass_tma_body(const ApassTmaMaps& maps, const ApassTmaArgs& aa, const int block) {
    extern __shared__ __align__(16) float sm_raw[];
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sm_raw) + 511) & ~uintptr_t(511));
    __shared__ __align__(8) uint64_t full[AT_STAGES];
    int k = 0;
    while (k + 1 < aa.count && (int)block >= aa.cta_start[k + 1]) ++k;
    const ApassTmaMode& m = aa.m[k];
    DevScalars* sc = aa.sc;
    constexpr int NT = AP_BN / NC;
    if (sc->done) return;
    const int task = block - aa.cta_start[k];
    const int t = threadIdx.x;
    const int grp = KS == 1 ? 0 : t / NT;        // row group
    const int lt = KS == 1 ? t : t - grp * NT;   // column slot within the group
    const int64_t I = m.I, post = m.post;
    const int BN = m.BN;
    int64_t a0, b0;
    int ncol;
    if (!m.rowmajor) {
        a0 = task / m.nbb;
        b0 = (int64_t)(task % m.nbb) * BN;
        ncol = (int)((post - b0) < BN ? (post - b0) : BN);
    } else {
        a0 = (int64_t)task * BN;
        b0 = 0;
        ncol = (int)((m.pre - a0) < BN ? (m.pre - a0) : BN);
    }
    const int nk = (int)((I + AP_BK - 1) / AP_BK);
    const int sst = at_stage_floats(BN, RP);
    const int gfl = AP_BK * BN;
    const uint32_t tx = (uint32_t)(4 * (AP_BK * BN + AP_BK * RP));

    if (t == 0) {
        for (int s2 = 0; s2 < AT_STAGES; ++s2) mbar_init(&full[s2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int kc) {
        const int st = kc % AT_STAGES;
        float* gs = smem + st * sst;
        mbar_expect_tx(&full[st], tx);
        if (!m.rowmajor) {
            const int c[3] = {(int)b0, kc * AP_BK, (int)a0};
            tma_load<3>(gs, &maps.g[k], &full[st], c);
        } else {
            const int c[2] = {kc * AP_BK, (int)a0};
            tma_load<2>(gs, &maps.g[k], &full[st], c);
        }
        const int cu[2] = {0, kc * AP_BK};
        tma_load<2>(gs + gfl, &maps.u[k], &full[st], cu);
    };
    if (t == 0)
        for (int s2 = 0; s2 < AT_STAGES - 1 && s2 < nk; ++s2) issue(s2);

    // thread lt of its group: columns lt + NT q of the task (q < NC); several columns
    // per thread amortise each broadcast read of a U row over NC x RP multiply-adds
    // accumulators in pairs (r, r + 1): each paired FMA (__ffma2_rn) does two of
    // the multiply-adds, each rounded as fmaf would, in one instruction
    float2 acc2[NC][RP / 2];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int r = 0; r < RP / 2; ++r) acc2[q][r] = make_float2(0.f, 0.f);
    bool failed = false;
    int fail_kc = 0;
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % AT_STAGES;
        const uint32_t par = (uint32_t)((kc / AT_STAGES) & 1);
        const bool ok = mbar_wait_bounded(&full[st], par, kWaitPolls);
        // also orders every thread's reads of the stage refilled below
        if (__syncthreads_or(!ok)) { failed = true; fail_kc = kc; break; }
        if (t == 0 && kc + AT_STAGES - 1 < nk) issue(kc + AT_STAGES - 1);
        const float* gs = smem + st * sst;
        const float* us = gs + gfl;
        if (!m.rowmajor) {
            int col[NC];     // a column past the task reads a valid one and is never stored
#pragma unroll
            for (int q = 0; q < NC; ++q) col[q] = lt + NT * q < BN ? lt + NT * q : lt;
            constexpr int KR = AP_BK / KS;
#pragma unroll 2
            for (int kk = grp * KR; kk < grp * KR + KR; ++kk) {
                float2 g[NC];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const float v = gs[kk * BN + col[q]];
                    g[q] = make_float2(v, v);
                }
                const float4* u4 = reinterpret_cast<const float4*>(us + kk * RP);
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4) {
                    const float4 u = u4[r4];
                    const float2 uxy = make_float2(u.x, u.y), uzw = make_float2(u.z, u.w);
#pragma unroll
                    for (int q = 0; q < NC; ++q) {
                        acc2[q][2 * r4 + 0] = __ffma2_rn(g[q], uxy, acc2[q][2 * r4 + 0]);
                        acc2[q][2 * r4 + 1] = __ffma2_rn(g[q], uzw, acc2[q][2 * r4 + 1]);
                    }
                }
            }
        } else {
            const int sw = (lt >> 1) & 3;   // the same for every column lt + NT q (NT even)
            constexpr int K4 = AP_BK / 4 / KS;
#pragma unroll
            for (int k4 = grp * K4; k4 < grp * K4 + K4; ++k4) {
                float gq[NC][4];
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    const float4 v = *reinterpret_cast<const float4*>(gs + (lt + NT * q) * AP_BK + 4 * (k4 ^ sw));
                    gq[q][0] = v.x; gq[q][1] = v.y; gq[q][2] = v.z; gq[q][3] = v.w;
                }
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const float4* u4 = reinterpret_cast<const float4*>(us + (4 * k4 + kk) * RP);
#pragma unroll
                    for (int r4 = 0; r4 < RP / 4; ++r4) {
                        const float4 u = u4[r4];
                        const float2 uxy = make_float2(u.x, u.y), uzw = make_float2(u.z, u.w);
#pragma unroll
                        for (int q = 0; q < NC; ++q) {
                            const float2 gg = make_float2(gq[q][kk], gq[q][kk]);
                            acc2[q][2 * r4 + 0] = __ffma2_rn(gg, uxy, acc2[q][2 * r4 + 0]);
                            acc2[q][2 * r4 + 1] = __ffma2_rn(gg, uzw, acc2[q][2 * r4 + 1]);
                        }
                    }
                }
            }
        }
    }
    if (failed) {
        // a copy never landed: record it and leave once the copies in flight are
        // accounted for (bounded), so no copy writes into a reassigned CTA's memory
        if (t == 0) {
            // chunks fail_kc .. fail_kc + AT_STAGES - 2 were issued, each in its own phase
            for (int c = fail_kc; c < fail_kc + AT_STAGES - 1 && c < nk; ++c)
                mbar_wait_bounded(&full[c % AT_STAGES], (uint32_t)((c / AT_STAGES) & 1), kWaitPolls);
            sc->status = -5;   // PASD_ERR_TIMEOUT
            sc->done = 1;
            __threadfence();
        }
        return;
    }
    __syncthreads();   // every stage consumed and no copy in flight: smem is free for the epilogue
    float acc[NC][RP];
#pragma unroll
    for (int q = 0; q < NC; ++q)
#pragma unroll
        for (int r = 0; r < RP / 2; ++r) {
            acc[q][2 * r] = acc2[q][r].x;
            acc[q][2 * r + 1] = acc2[q][r].y;
        }
    if (KS == 2) {
        // group 1's sums to group 0 ([q][lt][RP]), added after group 0's own
        float* hand = smem;
        if (grp == 1)
#pragma unroll
            for (int q = 0; q < NC; ++q)
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4)
                    *reinterpret_cast<float4*>(hand + (q * NT + lt) * RP + 4 * r4) =
                        make_float4(acc[q][4 * r4], acc[q][4 * r4 + 1], acc[q][4 * r4 + 2], acc[q][4 * r4 + 3]);
        __syncthreads();
        if (grp == 1) return;   // group 0 alone from here (named barrier 1 below)
#pragma unroll
        for (int q = 0; q < NC; ++q)
#pragma unroll
            for (int r4 = 0; r4 < RP / 4; ++r4) {
                const float4 h = *reinterpret_cast<const float4*>(hand + (q * NT + lt) * RP + 4 * r4);
                acc[q][4 * r4 + 0] += h.x;
                acc[q][4 * r4 + 1] += h.y;
                acc[q][4 * r4 + 2] += h.z;
                acc[q][4 * r4 + 3] += h.w;
            }
        asm volatile("bar.sync 1, %0;\n" ::"n"(NT) : "memory");   // read before the epilogue overwrites it
    }

    // columns past the task carry no data: zero them for the Gram sums
#pragma unroll
    for (int q = 0; q < NC; ++q)
        if (lt + NT * q >= ncol)
#pragma unroll
            for (int r = 0; r < RP; ++r) acc[q][r] = 0.f;
    // ---- store A (layout [pre][Rp][post]) ----
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const int c = lt + NT * q;
        if (c < ncol) {
            if (m.rowmajor) {
                float4* dst = reinterpret_cast<float4*>(m.A + (a0 + c) * RP);
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4)
                    dst[r4] = make_float4(acc[q][4 * r4], acc[q][4 * r4 + 1], acc[q][4 * r4 + 2], acc[q][4 * r4 + 3]);
            } else {
                float* dst = m.A + a0 * RP * post + b0 + c;
#pragma unroll
                for (int r = 0; r < RP; ++r) dst[(int64_t)r * post] = acc[q][r];
            }
        }
    }
    gram_epilogue<RP, NT, NC, AP_BN, (KS == 2 ? 1 : 0)>(acc, smem, m.gram_part + (size_t)task * RP * RP, lt);
}

template <int RP, int NC, int KS>
__global__ void __launch_bounds__(AP_BN / NC * KS, at_min_blocks(RP, NC, KS))
    apass_tma_kernel(const __grid_constant__ ApassTmaMaps maps, const ApassTmaArgs aa) {
    apass_tma_body<RP, NC, KS>(maps, aa, blockIdx.x);
}

// Batched: CTAs [start, start + tasks) of an entry run one solve's A-pass group
// (modes with one padded rank); maps from global memory, arguments from shared.
struct ApassBatchEntry {
    ApassTmaMaps maps;
    ApassTmaArgs args;
    int start;
};
template <int RP, int NC, int KS>
__global__ void __launch_bounds__(AP_BN / NC * KS, at_min_blocks(RP, NC, KS))
    apass_tma_kernel_batched(const ApassBatchEntry* e, const int* block_entry) {
    const ApassBatchEntry& x = e[block_entry[blockIdx.x]];
    __shared__ __align__(16) ApassTmaArgs s_aa;
    load_args_to_smem(&s_aa, &x.args);
    const int block = blockIdx.x - x.start;
    if (threadIdx.x == 0) {
        int k = 0;
        while (k + 1 < s_aa.count && block >= s_aa.cta_start[k + 1]) ++k;
        tensormap_acquire(&x.maps.g[k]);
        tensormap_acquire(&x.maps.u[k]);
    }
    apass_tma_body<RP, NC, KS>(x.maps, s_aa, block);
}

// ---------------------------------------------------------------------------
// Tensor-core A-pass (tcgen05, kind::tf32, accumulators in tensor memory),
// persistent and warp-specialised.
// A task is TC_BN = 128 consecutive unfolding columns; the MMA forms the
// transposed product A^T[col][r] = sum_i G[i][col] U[i][r] with M = 128
// (columns, one tensor-memory lane each), N = Rp rounded up to 16, and K = I
// streamed in stages of 16 rows. Both operands must be K-major (i contiguous),
// so every stage is rewritten into that layout in shared memory:
//   post > 1 : the copy lands [k][col]; each converter thread transposes a column
//   post == 1: the copy lands [col][k] with the 64-byte swizzle (operand layout)
// and U's [k][r] rows likewise become [r][k].
// TF32 keeps the top 19 bits of each FP32 operand (the MMA ignores the rest),
// so x = hi + lo with hi and lo rounded to TF32 (x = hi + lo up to 2^-24 |x|),
// and all four products are formed as two MMAs per step: G_hi and then G_lo
// against [U_hi; U_lo] stacked along N, so the first half of the accumulator
// collects g_hi u_hi + g_lo u_hi and the second half g_hi u_lo + g_lo u_lo;
// the halves are added in the epilogue. Each product is then good to about
// 2^-23 relative, the accuracy of FP32 multiply-adds. (A single TF32 product
// per term leaves the Gram eigenvalues of the discarded directions too noisy
// for the SVT threshold, so no cheaper form is offered.)
// Roles (one CTA per SM, looping over tasks):
//   warp 0      : bulk tensor copies of G and U into TP_RAW raw stages
//   warp 1      : tensor-memory owner and MMA issuer (one thread)
//   warps 2..9  : converters, raw stage -> one of NOPS operand buffers (a
//                 thread takes 8 rows of one column; the conversion is latency-
//                 bound, so it gets most of the warps)
//   warps 10..13: epilogue, accumulator -> A and the Gram partial, while the
//                 MMAs of the next task fill the other accumulator
// Hand-offs are mbarriers; every wait is bounded and a timeout stops all roles.
// ---------------------------------------------------------------------------
constexpr int TC_BN = 128;
constexpr int TC_BK = 16;
constexpr int TP_RAW = 6;
constexpr int TP_MAX_OPS = 6;
constexpr int TP_THREADS = 448;
constexpr int TP_CONV_WARPS = 8;

template <int RP>
struct TcShape {
    static constexpr int NP = (RP + 15) / 16 * 16;            // N of the U_hi block
    static constexpr int NB = 2 * NP;                          // rows of [U_hi; U_lo]
    static constexpr int TMEM_COLS = 2 * NB <= 64 ? 64 : 2 * NB <= 128 ? 128 : 256;   // two accumulators
    static constexpr int RAWG = TC_BN * TC_BK * 4;             // bytes of a raw G box
    static constexpr int RAWU = (TC_BK * RP * 4 + 1023) / 1024 * 1024;
    static constexpr int RAW_STRIDE = RAWG + RAWU;
    static constexpr int GHI = 0;
    static constexpr int GLO = RAWG;
    static constexpr int UB = 2 * RAWG;
    static constexpr int OP_STRIDE = UB + (NB * 64 + 1023) / 1024 * 1024;
    static constexpr int EPI_BYTES = 4 * (TC_BN * (RP + 4) + gram_red_floats(RP, 128));
    static constexpr int OPS = TP_RAW * RAW_STRIDE;
    // operand buffers: as many as fit (up to TP_MAX_OPS); more buffers hide the
    // completion latency of each stage's MMAs from the converters
    static constexpr int NOPS_FIT = (226 * 1024 - 1024 - OPS - EPI_BYTES) / OP_STRIDE;
    static constexpr int NOPS = NOPS_FIT < TP_MAX_OPS ? NOPS_FIT : TP_MAX_OPS;
    static constexpr int EPI = OPS + NOPS * OP_STRIDE;
    static constexpr int SMEM = EPI + EPI_BYTES;
    static_assert(NOPS >= 2, "A-pass tensor-core stages do not fit shared memory");
};

// Column range, a-row and contraction length of global task `gt`.
struct TcTask {
    int k;            // mode slot
    int64_t a0, b0;
    int ncol, nk;
};
__device__ __forceinline__ TcTask tc_task(const ApassTmaArgs& aa, int gt) {
    TcTask r;
    int k = 0;
    while (k + 1 < aa.count && gt >= aa.cta_start[k + 1]) ++k;
    const ApassTmaMode& m = aa.m[k];
    const int task = gt - aa.cta_start[k];
    r.k = k;
    if (!m.rowmajor) {
        r.a0 = task / m.nbb;
        r.b0 = (int64_t)(task % m.nbb) * TC_BN;
        r.ncol = (int)((m.post - r.b0) < TC_BN ? (m.post - r.b0) : TC_BN);
    } else {
        r.a0 = (int64_t)task * TC_BN;
        r.b0 = 0;
        r.ncol = (int)((m.pre - r.a0) < TC_BN ? (m.pre - r.a0) : TC_BN);
    }
    r.nk = (int)((m.I + TC_BK - 1) / TC_BK);
    return r;
}

template <int RP>
__global__ void __launch_bounds__(TP_THREADS, 1) apass_tc_kernel(const __grid_constant__ ApassTmaMaps maps,
                                                                const ApassTmaArgs aa) {
    using S = TcShape<RP>;
    extern __shared__ __align__(1024) unsigned char tc_sm_raw[];
    unsigned char* sm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_sm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t raw_full[TP_RAW], raw_empty[TP_RAW];
    __shared__ __align__(8) uint64_t op_full[TP_MAX_OPS], op_empty[TP_MAX_OPS];
    __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    DevScalars* sc = aa.sc;
    if (sc->done) return;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ntask = aa.cta_start[aa.count];

    if (warp == 1) tmem_alloc(&tmem_base, S::TMEM_COLS);
    if (t == 0) {
        for (int i = 0; i < TP_RAW; ++i) { mbar_init(&raw_full[i], 1); mbar_init(&raw_empty[i], TP_CONV_WARPS); }
        for (int i = 0; i < S::NOPS; ++i) { mbar_init(&op_full[i], TP_CONV_WARPS); mbar_init(&op_empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 128); }
        abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = tmem_base;
    auto give_up = [&]() {
        abort_flag = 1;
        sc->status = -5;   // PASD_ERR_TIMEOUT
        sc->done = 1;
        __threadfence();
    };
    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        for (uint32_t i = 0; i < kWaitPolls; ++i) {
            if (mbar_try_wait(bar, parity)) return true;
            if ((i & 255) == 255 && abort_flag) return false;
        }
        give_up();
        return false;
    };

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            const uint32_t tx = (uint32_t)(S::RAWG + TC_BK * RP * 4);
            int n = 0;
            for (int gt = blockIdx.x; gt < ntask && !abort_flag; gt += gridDim.x) {
                const TcTask tk = tc_task(aa, gt);
                for (int kc = 0; kc < tk.nk; ++kc, ++n) {
                    const int s = n % TP_RAW;
                    if (!wait(&raw_empty[s], (uint32_t)(((n / TP_RAW) & 1) ^ 1))) break;
                    unsigned char* raw = sm + s * S::RAW_STRIDE;
                    mbar_expect_tx(&raw_full[s], tx);
                    if (!aa.m[tk.k].rowmajor) {
                        const int c[3] = {(int)tk.b0, kc * TC_BK, (int)tk.a0};
                        tma_load<3>(raw, &maps.g[tk.k], &raw_full[s], c);
                    } else {
                        const int c[2] = {kc * TC_BK, (int)tk.a0};
                        tma_load<2>(raw, &maps.g[tk.k], &raw_full[s], c);
                    }
                    const int cu[2] = {0, kc * TC_BK};
                    tma_load<2>(raw + S::RAWG, &maps.u[tk.k], &raw_full[s], cu);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int n = 0, j = 0;
            for (int gt = blockIdx.x; gt < ntask && !abort_flag; gt += gridDim.x, ++j) {
                const TcTask tk = tc_task(aa, gt);
                const int a = j & 1;
                if (!wait(&acc_empty[a], (uint32_t)(((j >> 1) & 1) ^ 1))) break;
                const uint32_t dt = tm + (uint32_t)(a * S::NB);
                bool ok = true;
                for (int kc = 0; kc < tk.nk; ++kc, ++n) {
                    const int o = n % S::NOPS;
                    if (!wait(&op_full[o], (uint32_t)((n / S::NOPS) & 1))) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t ob = smem_u32(sm + S::OPS + o * S::OP_STRIDE);
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const uint64_t bd = tc_desc_sw64(ob + S::UB + 32 * jj);
                        tc_mma_tf32(dt, tc_desc_sw64(ob + S::GHI + 32 * jj), bd, tc_idesc_tf32(128, S::NB),
                                    (kc > 0 || jj > 0) ? 1u : 0u);
                        tc_mma_tf32(dt, tc_desc_sw64(ob + S::GLO + 32 * jj), bd, tc_idesc_tf32(128, S::NB), 1u);
                    }
                    tc_commit(&op_empty[o]);    // operand buffer o may be refilled once these MMAs are done
                }
                if (!ok) break;
                tc_commit(&acc_full[a]);        // accumulator a complete
            }
        }
    } else if (warp < 2 + TP_CONV_WARPS) {
        // ---------------- converters ----------------
        const int ct = t - 64;                  // 0 .. 255
        const int c = ct & (TC_BN - 1);         // column of the task
        const int kh = ct >> 7;                 // rows 8 kh .. 8 kh + 7 of the stage
        const int sw = (c >> 1) & 3;
        int n = 0;
        for (int gt = blockIdx.x; gt < ntask && !abort_flag; gt += gridDim.x) {
            const TcTask tk = tc_task(aa, gt);
            const bool rowmajor = aa.m[tk.k].rowmajor;
            bool ok = true;
            for (int kc = 0; kc < tk.nk; ++kc, ++n) {
                const int s = n % TP_RAW, o = n % S::NOPS;
                if (!wait(&raw_full[s], (uint32_t)((n / TP_RAW) & 1))) { ok = false; break; }
                if (!wait(&op_empty[o], (uint32_t)(((n / S::NOPS) & 1) ^ 1))) { ok = false; break; }
                const unsigned char* raw = sm + s * S::RAW_STRIDE;
                unsigned char* op = sm + S::OPS + o * S::OP_STRIDE;
                const float* rg = reinterpret_cast<const float*>(raw);
                float* ghi = reinterpret_cast<float*>(op + S::GHI);
                float* glo = reinterpret_cast<float*>(op + S::GLO);
#pragma unroll
                for (int kq = 0; kq < 2; ++kq) {
                    const int k4 = 2 * kh + kq;
                    const int off = c * 16 + ((k4 ^ sw) << 2);
                    float4 v;
                    if (!rowmajor) {
                        v.x = rg[(4 * k4 + 0) * TC_BN + c];
                        v.y = rg[(4 * k4 + 1) * TC_BN + c];
                        v.z = rg[(4 * k4 + 2) * TC_BN + c];
                        v.w = rg[(4 * k4 + 3) * TC_BN + c];
                    } else {
                        v = *reinterpret_cast<const float4*>(rg + off);
                    }
                    float4 h, l;
                    tf32_split(v.x, h.x, l.x);
                    tf32_split(v.y, h.y, l.y);
                    tf32_split(v.z, h.z, l.z);
                    tf32_split(v.w, h.w, l.w);
                    *reinterpret_cast<float4*>(ghi + off) = h;
                    *reinterpret_cast<float4*>(glo + off) = l;
                }
                const float* ru = reinterpret_cast<const float*>(raw + S::RAWG);
                float* ub = reinterpret_cast<float*>(op + S::UB);
                for (int u = ct; u < S::NP * 4; u += 32 * TP_CONV_WARPS) {
                    const int r = u % S::NP, k4 = u / S::NP;
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (r < RP) {
                        v.x = ru[(4 * k4 + 0) * RP + r];
                        v.y = ru[(4 * k4 + 1) * RP + r];
                        v.z = ru[(4 * k4 + 2) * RP + r];
                        v.w = ru[(4 * k4 + 3) * RP + r];
                    }
                    float4 h, l;
                    tf32_split(v.x, h.x, l.x);
                    tf32_split(v.y, h.y, l.y);
                    tf32_split(v.z, h.z, l.z);
                    tf32_split(v.w, h.w, l.w);
                    const int rl = S::NP + r;
                    *reinterpret_cast<float4*>(ub + r * 16 + ((k4 ^ ((r >> 1) & 3)) << 2)) = h;
                    *reinterpret_cast<float4*>(ub + rl * 16 + ((k4 ^ ((rl >> 1) & 3)) << 2)) = l;
                }
                fence_proxy_async_smem();      // operand writes visible to the tensor cores
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&raw_empty[s]);    // raw stage s read (this warp's part)
                    mbar_arrive(&op_full[o]);      // operand buffer o written (this warp's part)
                }
            }
            if (!ok) break;
        }
    } else {
        // ---------------- epilogue ----------------
        const int q = warp & 3;                 // tensor-memory lane quarter of this warp
        const int c = 32 * q + lane;            // column of the task
        float* epi = reinterpret_cast<float*>(sm + S::EPI);
        int j = 0;
        for (int gt = blockIdx.x; gt < ntask && !abort_flag; gt += gridDim.x, ++j) {
            const TcTask tk = tc_task(aa, gt);
            const ApassTmaMode& m = aa.m[tk.k];
            const int a = j & 1;
            if (!wait(&acc_full[a], (uint32_t)((j >> 1) & 1))) break;
            tc_fence_after();
            float acc[1][RP];
            {
                const uint32_t la = tm + ((uint32_t)(32 * q) << 16) + (uint32_t)(a * S::NB);
                float v[16];
#pragma unroll
                for (int c16 = 0; c16 < S::NP / 16; ++c16) {
                    tmem_ld16(la + 16 * c16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (16 * c16 + i < RP) acc[0][16 * c16 + i] = v[i];
                }
#pragma unroll
                for (int c16 = 0; c16 < S::NP / 16; ++c16) {
                    tmem_ld16(la + S::NP + 16 * c16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (16 * c16 + i < RP) acc[0][16 * c16 + i] += v[i];
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[a]);         // accumulator a may be overwritten
            if (c >= tk.ncol)
#pragma unroll
                for (int r = 0; r < RP; ++r) acc[0][r] = 0.f;
            else if (m.rowmajor) {
                float4* dst = reinterpret_cast<float4*>(m.A + (tk.a0 + c) * RP);
#pragma unroll
                for (int r4 = 0; r4 < RP / 4; ++r4)
                    dst[r4] = make_float4(acc[0][4 * r4], acc[0][4 * r4 + 1], acc[0][4 * r4 + 2], acc[0][4 * r4 + 3]);
            } else {
                float* dst = m.A + tk.a0 * RP * m.post + tk.b0 + c;
#pragma unroll
                for (int r = 0; r < RP; ++r) dst[(int64_t)r * m.post] = acc[0][r];
            }
            const int task = gt - aa.cta_start[tk.k];
            gram_epilogue<RP, 128, 1, TC_BN, 1>(acc, epi, m.gram_part + (size_t)task * RP * RP, c);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tm, S::TMEM_COLS);
}

template <int RP, int NC, int KS>
static void launch_tma_rp_nc(const ApassTmaPlan& p, cudaStream_t s) {
    set_smem_attr((const void*)apass_tma_kernel<RP, NC, KS>, (int)p.smem);
    apass_tma_kernel<RP, NC, KS><<<p.args.cta_start[p.args.count], AP_BN / NC * KS, p.smem, s>>>(p.maps, p.args);
}
// variants: default columns per thread, half of them, or the default with the
// rows of each stage split between two thread groups
template <int RP>
static void launch_tma_rp(const ApassTmaPlan& p, cudaStream_t s) {
    constexpr int C = AtShape<RP>::COLS;
    if constexpr (RP <= kSplitMaxRp) {
        if (p.ks == 2) { launch_tma_rp_nc<RP, C, 2>(p, s); return; }
    }
    if (p.nc == C) launch_tma_rp_nc<RP, C, 1>(p, s);
    else launch_tma_rp_nc<RP, C / 2, 1>(p, s);
}

template <int RP>
static void launch_tc_rp(const ApassTmaPlan& p, cudaStream_t s) {
    set_smem_attr((const void*)apass_tc_kernel<RP>, (int)p.smem);
    const int ntask = p.args.cta_start[p.args.count];
    const int grid = ntask < p.grid ? ntask : p.grid;
    apass_tc_kernel<RP><<<grid, TP_THREADS, p.smem, s>>>(p.maps, p.args);
}

static void launch_tc(const ApassTmaPlan& p, cudaStream_t s) {
    switch (p.args.Rp) {
        case 4: launch_tc_rp<4>(p, s); break;
        case 8: launch_tc_rp<8>(p, s); break;
        case 12: launch_tc_rp<12>(p, s); break;
        case 16: launch_tc_rp<16>(p, s); break;
        case 20: launch_tc_rp<20>(p, s); break;
        case 24: launch_tc_rp<24>(p, s); break;
        case 28: launch_tc_rp<28>(p, s); break;
        case 32: launch_tc_rp<32>(p, s); break;
        case 40: launch_tc_rp<40>(p, s); break;
        case 48: launch_tc_rp<48>(p, s); break;
        case 56: launch_tc_rp<56>(p, s); break;
        case 64: launch_tc_rp<64>(p, s); break;
        default: break;
    }
}

static size_t tc_smem(int Rp) {
    switch (Rp) {
        case 4: return TcShape<4>::SMEM;
        case 8: return TcShape<8>::SMEM;
        case 12: return TcShape<12>::SMEM;
        case 16: return TcShape<16>::SMEM;
        case 20: return TcShape<20>::SMEM;
        case 24: return TcShape<24>::SMEM;
        case 28: return TcShape<28>::SMEM;
        case 32: return TcShape<32>::SMEM;
        case 40: return TcShape<40>::SMEM;
        case 48: return TcShape<48>::SMEM;
        case 56: return TcShape<56>::SMEM;
        default: return TcShape<64>::SMEM;
    }
}

void launch_apass_tma(const ApassTmaPlan* p, cudaStream_t s) {
    if (p->kind == APASS_TC) { launch_tc(*p, s); return; }
    switch (p->args.Rp) {
        case 4: launch_tma_rp<4>(*p, s); break;
        case 8: launch_tma_rp<8>(*p, s); break;
        case 12: launch_tma_rp<12>(*p, s); break;
        case 16: launch_tma_rp<16>(*p, s); break;
        case 20: launch_tma_rp<20>(*p, s); break;
        case 24: launch_tma_rp<24>(*p, s); break;
        case 28: launch_tma_rp<28>(*p, s); break;
        case 32: launch_tma_rp<32>(*p, s); break;
        case 40: launch_tma_rp<40>(*p, s); break;
        case 48: launch_tma_rp<48>(*p, s); break;
        case 56: launch_tma_rp<56>(*p, s); break;
        case 64: launch_tma_rp<64>(*p, s); break;
        default: break;
    }
}

bool apass_tma_supported(int64_t I, int64_t post) {
    if (post == 1) return I % 4 == 0;
    return post % 4 == 0;
}

// Columns per task of each A-pass kind (post > 1: within one a-row).
static int64_t task_cols(int64_t post, int kind) {
    if (kind != APASS_FFMA) return TC_BN;
    return post == 1 ? 256 : (post < 256 ? post : 256);
}

int apass_tma_tasks(int64_t I, int64_t pre, int64_t post, int kind) {
    (void)I;
    const int64_t BN = task_cols(post, kind);
    if (post == 1) return (int)((pre + BN - 1) / BN);
    return (int)(pre * ((post + BN - 1) / BN));
}

ApassTmaPlan* make_apass_tma(const ApassArgs* a, const int* modes, int count, int kind, int num_sms, char* err,
                             size_t errlen) {
    ApassTmaPlan* p = new ApassTmaPlan();
    std::memset(&p->maps, 0, sizeof(p->maps));
    p->kind = kind;
    p->grid = num_sms;
    p->args = ApassTmaArgs{};
    p->args.count = count;
    p->args.sc = const_cast<DevScalars*>(a[modes[0]].sc);
    p->args.Rp = a[modes[0]].Rp;
    int start = 0;
    size_t smem = 0;
    for (int q = 0; q < count; ++q) {
        const ApassArgs& x = a[modes[q]];
        ApassTmaMode& mm = p->args.m[q];
        mm.I = x.I; mm.pre = x.pre; mm.post = x.post; mm.P = x.P;
        mm.rowmajor = x.post == 1;
        mm.BN = (int)task_cols(x.post, kind);
        mm.nbb = mm.rowmajor ? 1 : (int)((x.post + mm.BN - 1) / mm.BN);
        mm.A = x.A;
        mm.gram_part = x.gram_part;
        const int ntask = apass_tma_tasks(x.I, x.pre, x.post, kind);
        p->args.cta_start[q] = start;
        start += ntask;
        const int Rp = x.Rp;
        bool ok;
        if (!mm.rowmajor) {
            uint64_t d[3] = {(uint64_t)x.post, (uint64_t)x.I, (uint64_t)x.pre};
            uint32_t b[3] = {(uint32_t)mm.BN, (uint32_t)AP_BK, 1u};
            ok = encode_tiled_f32(&p->maps.g[q], x.G, 3, d, b, CU_TENSOR_MAP_SWIZZLE_NONE, err, errlen, "A-pass G");
        } else {
            uint64_t d[2] = {(uint64_t)x.I, (uint64_t)x.pre};
            uint32_t b[2] = {(uint32_t)AP_BK, (uint32_t)mm.BN};
            ok = encode_tiled_f32(&p->maps.g[q], x.G, 2, d, b, CU_TENSOR_MAP_SWIZZLE_64B, err, errlen, "A-pass G");
        }
        if (ok) {
            uint64_t d[2] = {(uint64_t)Rp, (uint64_t)x.I};
            uint32_t b[2] = {(uint32_t)Rp, (uint32_t)AP_BK};
            ok = encode_tiled_f32(&p->maps.u[q], x.U, 2, d, b, CU_TENSOR_MAP_SWIZZLE_NONE, err, errlen, "A-pass U");
        }
        if (!ok) { delete p; return nullptr; }
        if (kind == APASS_FFMA) {
            const size_t pipe = (size_t)AT_STAGES * at_stage_floats(mm.BN, Rp);
            p->pipe_floats = std::max(p->pipe_floats, pipe);
            p->epi_base_floats = std::max(p->epi_base_floats, (size_t)AP_BN * (Rp + 4));
            const size_t epi = (size_t)AP_BN * (Rp + 4) + gram_red_floats(Rp, Rp <= 40 ? AP_BN / 4 : AP_BN / 2);
            smem = std::max(smem, 4 * std::max(pipe, epi) + 512);
        } else {
            smem = std::max(smem, tc_smem(Rp) + 1024);
        }
    }
    p->args.cta_start[count] = start;
    p->smem = smem;
    p->nc = p->args.Rp <= 40 ? 4 : 2;
    p->ks = 1;
    return p;
}

size_t apass_batch_entry_bytes() { return sizeof(ApassBatchEntry); }
int apass_batch_rp(const ApassTmaPlan* p) { return p->args.Rp; }
int apass_batch_ctas(const ApassTmaPlan* p) { return p->kind == APASS_FFMA ? p->args.cta_start[p->args.count] : -1; }
size_t apass_batch_smem(const ApassTmaPlan* p) { return p->smem; }
void apass_batch_fill(void* entry, const ApassTmaPlan* p, int start) {
    // built in an aligned local and copied: `entry` points into a byte staging
    // buffer that need not meet the tensor maps' 64-byte alignment
    ApassBatchEntry e;
    std::memset(&e, 0, sizeof(e));
    e.maps = p->maps;
    e.args = p->args;
    e.start = start;
    std::memcpy(entry, &e, sizeof(e));
}
template <int RP, int NC, int KS>
static void launch_batched_rp_nc(const void* entries, const int* block_entry, int grid, size_t smem, cudaStream_t s) {
    set_smem_attr((const void*)apass_tma_kernel_batched<RP, NC, KS>, (int)smem);
    apass_tma_kernel_batched<RP, NC, KS><<<grid, AP_BN / NC * KS, smem, s>>>(static_cast<const ApassBatchEntry*>(entries), block_entry);
}
template <int RP>
static void launch_batched_rp(int var, const void* entries, const int* block_entry, int grid, size_t smem,
                              cudaStream_t s) {
    constexpr int C = AtShape<RP>::COLS;
    const int nc = var % 100, ks = var / 100;
    if constexpr (RP <= kSplitMaxRp) {
        if (ks == 2) { launch_batched_rp_nc<RP, C, 2>(entries, block_entry, grid, smem, s); return; }
    }
    if (nc == C) launch_batched_rp_nc<RP, C, 1>(entries, block_entry, grid, smem, s);
    else launch_batched_rp_nc<RP, C / 2, 1>(entries, block_entry, grid, smem, s);
}
void launch_apass_batched(int Rp, int var, const void* entries, const int* block_entry, int grid, size_t smem,
                          cudaStream_t s) {
    switch (Rp) {
        case 4: launch_batched_rp<4>(var, entries, block_entry, grid, smem, s); break;
        case 8: launch_batched_rp<8>(var, entries, block_entry, grid, smem, s); break;
        case 12: launch_batched_rp<12>(var, entries, block_entry, grid, smem, s); break;
        case 16: launch_batched_rp<16>(var, entries, block_entry, grid, smem, s); break;
        case 20: launch_batched_rp<20>(var, entries, block_entry, grid, smem, s); break;
        case 24: launch_batched_rp<24>(var, entries, block_entry, grid, smem, s); break;
        case 28: launch_batched_rp<28>(var, entries, block_entry, grid, smem, s); break;
        case 32: launch_batched_rp<32>(var, entries, block_entry, grid, smem, s); break;
        case 40: launch_batched_rp<40>(var, entries, block_entry, grid, smem, s); break;
        case 48: launch_batched_rp<48>(var, entries, block_entry, grid, smem, s); break;
        case 56: launch_batched_rp<56>(var, entries, block_entry, grid, smem, s); break;
        case 64: launch_batched_rp<64>(var, entries, block_entry, grid, smem, s); break;
        default: break;
    }
}

int apass_tma_cols(const ApassTmaPlan* p) { return p->kind == APASS_FFMA ? p->nc : 0; }
int apass_tma_split(const ApassTmaPlan* p) { return p->kind == APASS_FFMA ? p->ks : 0; }
int apass_tma_variant(const ApassTmaPlan* p) { return p->kind == APASS_FFMA ? p->nc + 100 * p->ks : 0; }

// Columns per thread of the FMA kernel (its default or half of it) and row
// groups (1, or 2 with the default columns).
void apass_tma_set_cols(ApassTmaPlan* p, int nc, int ks) {
    if (p->kind != APASS_FFMA) return;
    const int def = p->args.Rp <= 40 ? 4 : 2;
    if (nc != def && nc != def / 2) return;
    if (ks != 1 && (ks != 2 || nc != def || p->args.Rp > kSplitMaxRp)) return;
    p->nc = nc;
    p->ks = ks;
    // the row groups' hand-off ([nc][AP_BN / nc][Rp]) fits in the epilogue's A tile
    const size_t epi = p->epi_base_floats + gram_red_floats(p->args.Rp, AP_BN / nc);
    p->smem = 4 * std::max(p->pipe_floats, epi) + 512;
}

void destroy_apass_tma(ApassTmaPlan* p) { delete p; }


}  // namespace pasd
