// M-pass: the product M_n = G_n V_n^T of the next U-step (Eq. 9), in the
// eigenbasis W of the last SVT: with Vrot_n = diag(F) W^T A_n (rows at and past
// the kept count s_n are zero), M_n W diag(F)^{-1} restricted to the kept columns
// is G_(n) Vrot_n[:s]^T, an I_n x s_n contraction over the P_n unfolding columns.
// It runs right after the fused pass, so it reads the freshly written G_n.
//
// G_(n) is viewed as [pre][I][post] (Sec. 2.1), read in place. A CTA owns a strip
// of at most `IS` rows and a range of unfolding columns, which it streams in
// chunks of MP_CB columns through a cp.async pipeline:
//   post > 1 : a chunk is IS rows of MP_CB columns   -> smem [i][col], 16-byte
//              column groups XOR-swizzled by 8-row block, so the row loads of
//              a thread at one column hit distinct banks across the warp
//   post == 1: a chunk is MP_CB columns of IS rows   -> smem [col][i]
// and the matching Vrot_n columns -> smem [col][r]. Each thread accumulates an
// 8-row x 4-rank FP32 register tile over all of its columns (FFMA); when few
// ranks are kept, idle threads take alternate columns and the tiles are added
// in a fixed order at the end. One partial M per column range is written to
// part[range][I][Rp]; the finalize kernel sums them in a fixed order, so the
// result does not depend on timing.
#include "pasd_impl.cuh"
#include "tma.cuh"

#include <algorithm>
#include <cstring>

namespace pasd {

namespace {

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

}  // namespace

// Stage sizes (floats) for a mode, rows rounded up to whole 8-row blocks (the
// register tiles read them); [col][i] stages use the row stride mp_ldi.
static inline __host__ __device__ int mp_ldi(int IS) { return (IS + 7) / 8 * 8; }
static inline __host__ __device__ int mp_g_stage(int IS, int variant) {
    (void)variant;
    return MP_CB * mp_ldi(IS);
}
static inline __host__ __device__ int mp_v_stage(int Rp) { return MP_CB * Rp; }

size_t mpass_smem_bytes(int IS, int Rp, int variant) {
    size_t stage = (size_t)mp_g_stage(IS, variant) + mp_v_stage(Rp);
    size_t red = (size_t)MP_THREADS * 32;
    size_t pipe = (size_t)MP_STAGES * stage;
    return 4 * (pipe > red ? pipe : red);
}

int mpass_variant(int64_t I, int64_t post) {
    if (post == 1) return (I % 4 == 0) ? 2 : 3;
    return (post % 4 == 0) ? 0 : 1;
}

int mpass_strip_rows(int64_t I, int Rp) {
    int cap = 8 * (MP_THREADS / (Rp / 4));
    cap = std::min(cap, 256);
    return (int)std::min<int64_t>(I, cap);
}

// Column position (a, b) of unfolding column j = a * post + b, advanced by `d`
// columns at a time without a division after the first.
struct ColPos {
    int64_t a, b;
    __device__ __forceinline__ void init(int64_t j, int64_t post) { a = j / post; b = j - a * post; }
    __device__ __forceinline__ void advance(int64_t d, int64_t post) {
        b += d;
        while (b >= post) { b -= post; ++a; }
    }
};

template <int V>
__device__ __forceinline__ void mpass_body(const MpassMode& m, int s, int cta, float* smem) {
    constexpr bool colmajor = (V >= 2);      // smem [col][i]
    const int t = threadIdx.x;
    const int strip = cta % m.nstrips, cg = cta / m.nstrips;
    const int64_t I = m.I, post = m.post, P = m.P;
    const int64_t i_lo = (int64_t)strip * m.IS;
    const int IS = (int)((I - i_lo) < m.IS ? (I - i_lo) : m.IS);
    const int LDI = mp_ldi(m.IS);
    const int64_t c_lo = (int64_t)cg * m.cols_per_cg;
    const int64_t c_hi = (c_lo + m.cols_per_cg) < P ? (c_lo + m.cols_per_cg) : P;
    const int nk = c_hi > c_lo ? (int)((c_hi - c_lo + MP_CB - 1) / MP_CB) : 0;
    const int Rp = m.Rp;
    const int gst = mp_g_stage(m.IS, V), vst = mp_v_stage(Rp);
    float* Gs = smem;
    float* Vs = smem + MP_STAGES * gst;
    const float* __restrict__ G = m.G;
    const float* __restrict__ Vr = m.V;

    // thread -> (task, column group inside the CTA); task -> (8-row block q, rank block rq)
    const int nrq = s / 4;
    const int nq = (IS + 7) / 8;
    const int ntask = nq * nrq;
    const int KG = (ntask > 0 && MP_THREADS / ntask > 1) ? MP_THREADS / ntask : 1;
    const int task = ntask > 0 ? t % ntask : 0;
    const int kg = ntask > 0 ? t / ntask : KG;
    const bool active = kg < KG;
    const int q = task / (nrq > 0 ? nrq : 1), rq = task % (nrq > 0 ? nrq : 1);

    // copy positions, advanced chunk by chunk (chunks are issued in order)
    // G (post > 1): the thread's column (group) is fixed: t % 8 (16-byte) or t % MP_CB
    constexpr int CG4 = MP_CB / 4;           // 16-byte column groups per chunk row
    const int gc = (V == 0) ? 4 * (t % CG4) : (t & (MP_CB - 1));
    ColPos gpos;
    if (!colmajor) gpos.init(c_lo + gc, post);
    // Vrot: column t % MP_CB, rows t / MP_CB + 8 k
    const int vc = t & (MP_CB - 1);
    ColPos vpos;
    vpos.init(c_lo + vc, post);

    auto issue = [&](int kc, int st) {
        const int64_t j0 = c_lo + (int64_t)kc * MP_CB;
        float* gs = Gs + st * gst;
        if (V == 0) {
            const int cs = t % CG4;
            const bool jok = j0 + gc < c_hi;
            const float* base = G + (gpos.a * I + i_lo) * post + gpos.b;
            for (int row = t / CG4; row < IS; row += MP_THREADS / CG4) {
                const int phys = cs ^ ((row >> 3) & 7);
                cp_async16(gs + row * MP_CB + 4 * phys, jok ? base + (int64_t)row * post : G, jok ? 16 : 0);
            }
            gpos.advance(MP_CB, post);
        } else if (V == 1) {
            const bool jok = j0 + gc < c_hi;
            const float* base = G + (gpos.a * I + i_lo) * post + gpos.b;
            for (int row = t / MP_CB; row < IS; row += MP_THREADS / MP_CB) {
                const int pc = (((gc >> 2) ^ ((row >> 3) & 7)) << 2) | (gc & 3);
                cp_async4(gs + row * MP_CB + pc, jok ? base + (int64_t)row * post : G, jok ? 4 : 0);
            }
            gpos.advance(MP_CB, post);
        } else if (V == 2) {
            const int IS4 = (IS + 3) / 4;
            for (int idx = t; idx < MP_CB * IS4; idx += MP_THREADS) {
                const int iseg = idx % IS4, c = idx / IS4;
                const int64_t j = j0 + c;
                const bool ok = j < c_hi;
                cp_async16(gs + c * LDI + 4 * iseg, ok ? G + j * I + i_lo + 4 * iseg : G, ok ? 16 : 0);
            }
        } else {
            for (int idx = t; idx < MP_CB * IS; idx += MP_THREADS) {
                const int i = idx % IS, c = idx / IS;
                const int64_t j = j0 + c;
                const bool ok = j < c_hi;
                cp_async4(gs + c * LDI + i, ok ? G + j * I + i_lo + i : G, ok ? 4 : 0);
            }
        }
        // Vrot columns j0 .. j0 + MP_CB, kept rows, into [col][r]
        float* vs = Vs + st * vst;
        const bool vok = j0 + vc < c_hi;
        const float* vbase = Vr + vpos.a * Rp * post + vpos.b;
        for (int r = t / MP_CB; r < s; r += MP_THREADS / MP_CB)
            cp_async4(vs + vc * Rp + r, vok ? vbase + (int64_t)r * post : Vr, vok ? 4 : 0);
        vpos.advance(MP_CB, post);
    };

    float acc[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[k][r] = 0.f;

#pragma unroll
    for (int st = 0; st < MP_STAGES - 1; ++st) {
        if (st < nk) issue(st, st);
        cp_commit();
    }
    for (int kc = 0; kc < nk; ++kc) {
        cp_wait<MP_STAGES - 2>();
        __syncthreads();
        {
            const int nxt = kc + MP_STAGES - 1;
            if (nxt < nk) issue(nxt, nxt % MP_STAGES);
            cp_commit();
        }
        const int st = kc % MP_STAGES;
        const float* gs = Gs + st * gst;
        const float* vs = Vs + st * vst + 4 * rq;
        if (active) {
            if (colmajor) {
                const float* gq = gs + 8 * q;
#pragma unroll 4
                for (int c = kg; c < MP_CB; c += KG) {
                    const float4 g0 = *reinterpret_cast<const float4*>(gq + c * LDI);
                    const float4 g1 = *reinterpret_cast<const float4*>(gq + c * LDI + 4);
                    const float4 v = *reinterpret_cast<const float4*>(vs + c * Rp);
                    const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[k][r] = fmaf(gg[k], vv[r], acc[k][r]);
                }
            } else {
                const int sw = q & 7;
                const float* gq = gs + (8 * q) * MP_CB;
#pragma unroll 4
                for (int c = kg; c < MP_CB; c += KG) {
                    const int pc = (((c >> 2) ^ sw) << 2) | (c & 3);
                    float gg[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) gg[k] = gq[k * MP_CB + pc];
                    const float4 v = *reinterpret_cast<const float4*>(vs + c * Rp);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int k = 0; k < 8; ++k)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[k][r] = fmaf(gg[k], vv[r], acc[k][r]);
                }
            }
        }
    }
    cp_wait<0>();
    __syncthreads();

    // ---- the column groups of the CTA, added in order; partial rows of this strip ----
    float* dst = m.part + ((int64_t)cg * I + i_lo) * Rp;
    if (KG > 1) {
        float* red = smem;      // [KG][ntask][32], reuses the pipeline buffers
        if (active) {
            float4* o = reinterpret_cast<float4*>(red + ((size_t)kg * ntask + task) * 32);
#pragma unroll
            for (int k = 0; k < 8; ++k) o[k] = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
        }
        __syncthreads();
        for (int w = t; w < ntask * 8; w += MP_THREADS) {
            const int tk = w >> 3, k = w & 7;
            const int qq = tk / nrq, rr = tk % nrq;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int g = 0; g < KG; ++g) {
                const float4 v = *reinterpret_cast<const float4*>(red + ((size_t)g * ntask + tk) * 32 + 4 * k);
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            const int row = 8 * qq + k;
            if (row < IS) *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rr) = sum;
        }
    } else if (active) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int row = 8 * q + k;
            if (row < IS)
                *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rq) =
                    make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
        }
    }
}

__device__ __forceinline__ void mpass_body(const MpassArgs& ma, const int block) {
    extern __shared__ __align__(16) float smem[];
    const DevScalars* sc = ma.sc;
    if (sc->done) return;
    int k = 0;
    while (k + 1 < ma.N && (int)block >= ma.cta_start[k + 1]) ++k;
    const MpassMode& m = ma.m[k];
    const int s = (sc->kept[k] + 3) & ~3;      // kept rows rounded up (Vrot rows past s_n are zero)
    if (s == 0) return;                        // no kept direction: the U-step does not read M_n
    const int cta = block - ma.cta_start[k];
    switch (m.variant) {
        case 0: mpass_body<0>(m, s, cta, smem); break;
        case 1: mpass_body<1>(m, s, cta, smem); break;
        case 2: mpass_body<2>(m, s, cta, smem); break;
        default: mpass_body<3>(m, s, cta, smem); break;
    }
}

__global__ void __launch_bounds__(MP_THREADS) mpass_kernel(const MpassArgs ma) { mpass_body(ma, blockIdx.x); }

// Batched: CTAs [start, start + ctas) of an entry run one solve's M-pass.
__global__ void __launch_bounds__(MP_THREADS) mpass_kernel_batched(const MpassPlainBatchEntry* e,
                                                                   const int* block_entry) {
    const MpassPlainBatchEntry& x = e[block_entry[blockIdx.x]];
    __shared__ __align__(16) MpassArgs s_ma;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(&x.a);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_ma);
    for (int w = threadIdx.x; w < (int)(sizeof(MpassArgs) / 4); w += blockDim.x) dst[w] = src[w];
    __syncthreads();
    mpass_body(s_ma, blockIdx.x - x.start);
}

int mpass_ctas_per_sm(size_t smem) {
    set_smem_attr((const void*)mpass_kernel, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mpass_kernel, MP_THREADS, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

void launch_mpass_plain_batched(const MpassPlainBatchEntry* e, const int* block_entry, int grid, size_t smem,
                                cudaStream_t s) {
    set_smem_attr((const void*)mpass_kernel_batched, (int)smem);
    mpass_kernel_batched<<<grid, MP_THREADS, smem, s>>>(e, block_entry);
}

void launch_mpass(const MpassArgs& a, size_t smem, cudaStream_t s) {
    set_smem_attr((const void*)mpass_kernel, (int)smem);
    mpass_kernel<<<a.cta_start[a.N], MP_THREADS, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// TMA-fed M-pass. Each chunk is one bulk tensor copy of G and one of Vrot:
//   post > 1 : a chunk is MP_CB columns inside one a-row of the unfolding; the
//              G box is [IS][32] and the Vrot box [Rp][32], both with the
//              128-byte swizzle (16-byte group g of row r at g ^ (r & 7)).
//              A thread's 8 rows are strided (q, q + nq8, ...), so the rows it
//              reads at one column group fall in distinct swizzle phases across
//              the warp; it reads whole 16-byte groups (4 columns) at a time.
//   post == 1: a chunk is MP_CB rows of G ([32][IS]) and of Vrot ([32][Rp]).
// Register tiles are 8 rows x 4 ranks; idle threads take alternate column
// groups and the tiles are added in a fixed order, as in the cp.async kernel.
// ---------------------------------------------------------------------------
struct MpassTmaMaps {
    CUtensorMap g[PASD_MAXN];
    CUtensorMap v[PASD_MAXN];
};
struct MpassTmaPlan {
    MpassTmaMaps maps;
    MpassTmaArgs args;
    size_t smem;
};

// G tile then Vrot tile, each starting on a 1 KB boundary (the 128-byte swizzle's
// period); +8 floats past the Vrot tile for the last column's 8-row overreach.
static inline __host__ __device__ int mt_g_floats(int IS) { return (MP_CB * IS + 255) / 256 * 256; }
static inline __host__ __device__ int mt_stage_floats(int IS, int Rp) {
    return mt_g_floats(IS) + (MP_CB * Rp + 8 + 255) / 256 * 256;
}

__device__ __forceinline__ void mpass_tma_body(const MpassTmaMaps& maps, const MpassTmaArgs& ma, const int block) {
    extern __shared__ __align__(16) float sm_raw[];
    float* smem = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[MT_STAGES];
    DevScalars* sc = ma.sc;
    if (sc->done) return;
    int k = 0;
    while (k + 1 < ma.N && (int)block >= ma.cta_start[k + 1]) ++k;
    const MpassTmaMode& m = ma.m[k];
    const int s = (sc->kept[k] + 3) & ~3;      // kept rows rounded up (Vrot rows past s_n are zero)
    if (s == 0) return;                        // no kept direction: the U-step does not read M_n
    const int cta = block - ma.cta_start[k];
    const int t = threadIdx.x;
    const int strip = cta % m.nstrips, rg = cta / m.nstrips;
    const int64_t I = m.I;
    const int64_t i_lo = (int64_t)strip * m.IS;
    const int IS = (int)((I - i_lo) < m.IS ? (I - i_lo) : m.IS);
    const int ch_lo = rg * m.cpr;
    const int ch_hi = (ch_lo + m.cpr) < m.nch ? (ch_lo + m.cpr) : m.nch;
    const int nk = ch_hi > ch_lo ? ch_hi - ch_lo : 0;
    const int Rp = m.Rp;
    const int sst = mt_stage_floats(m.IS, Rp);
    const int gfl = mt_g_floats(m.IS);
    const uint32_t tx = (uint32_t)(4 * (MP_CB * m.IS + MP_CB * Rp));

    // thread -> (task, column group); task -> (8-row block q, rank block rq)
    const int nrq = s / 4;
    const int nq = (IS + 7) / 8;
    const int ntask = nq * nrq;
    const int ngroups = m.rowmajor ? MP_CB : MP_CB / 4;      // columns / 16-byte column groups
    int KG = MP_THREADS / ntask;
    if (KG > ngroups) KG = ngroups;
    if (KG < 1) KG = 1;
    const int task = t % ntask, kg = t / ntask;
    const bool active = kg < KG;
    const int q = task / nrq, rq = task % nrq;

    if (t == 0) {
        for (int s2 = 0; s2 < MT_STAGES; ++s2) mbar_init(&full[s2], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int kc) {
        const int st = kc % MT_STAGES;
        float* gs = smem + st * sst;
        const int ch = ch_lo + kc;
        mbar_expect_tx(&full[st], tx);
        if (!m.rowmajor) {
            const int a = ch / m.nbb, b0 = (ch % m.nbb) * MP_CB;
            const int cg3[3] = {b0, (int)i_lo, a};
            tma_load<3>(gs, &maps.g[k], &full[st], cg3);
            const int cv3[3] = {b0, 0, a};
            tma_load<3>(gs + gfl, &maps.v[k], &full[st], cv3);
        } else {
            const int a0 = ch * MP_CB;
            const int cg2[2] = {(int)i_lo, a0};
            tma_load<2>(gs, &maps.g[k], &full[st], cg2);
            const int cv2[2] = {0, a0};
            tma_load<2>(gs + gfl, &maps.v[k], &full[st], cv2);
        }
    };
    if (t == 0)
        for (int s2 = 0; s2 < MT_STAGES - 1 && s2 < nk; ++s2) issue(s2);

    float acc[8][4];
#pragma unroll
    for (int kk = 0; kk < 8; ++kk)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[kk][r] = 0.f;
    const int nq8 = nq;
    bool failed = false;
    int fail_kc = 0;
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc % MT_STAGES;
        const uint32_t par = (uint32_t)((kc / MT_STAGES) & 1);
        const bool ok = mbar_wait_bounded(&full[st], par, kWaitPolls);
        if (__syncthreads_or(!ok)) { failed = true; fail_kc = kc; break; }
        if (t == 0 && kc + MT_STAGES - 1 < nk) issue(kc + MT_STAGES - 1);
        const float* gs = smem + st * sst;
        const float* vs = gs + gfl;
        if (!active) continue;
        if (!m.rowmajor) {
            for (int c4 = kg; c4 < MP_CB / 4; c4 += KG) {
                float4 v[4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int r = 4 * rq + rr;
                    v[rr] = *reinterpret_cast<const float4*>(vs + r * MP_CB + 4 * (c4 ^ (r & 7)));
                }
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int row = q + kk * nq8;
                    const float4 g = *reinterpret_cast<const float4*>(gs + row * MP_CB + 4 * (c4 ^ (row & 7)));
#pragma unroll
                    for (int rr = 0; rr < 4; ++rr) {
                        float a2 = acc[kk][rr];
                        a2 = fmaf(g.x, v[rr].x, a2);
                        a2 = fmaf(g.y, v[rr].y, a2);
                        a2 = fmaf(g.z, v[rr].z, a2);
                        acc[kk][rr] = fmaf(g.w, v[rr].w, a2);
                    }
                }
            }
        } else {
            const float* gq = gs + 8 * q;
            const float* vq = vs + 4 * rq;
#pragma unroll 4
            for (int c = kg; c < MP_CB; c += KG) {
                const float4 g0 = *reinterpret_cast<const float4*>(gq + c * m.IS);
                const float4 g1 = *reinterpret_cast<const float4*>(gq + c * m.IS + 4);
                const float4 v = *reinterpret_cast<const float4*>(vq + c * Rp);
                const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int kk = 0; kk < 8; ++kk)
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[kk][r] = fmaf(gg[kk], vv[r], acc[kk][r]);
            }
        }
    }
    if (failed) {
        if (t == 0) {
            // chunks fail_kc .. fail_kc + MT_STAGES - 2 were issued, each in its own phase
            for (int c = fail_kc; c < fail_kc + MT_STAGES - 1 && c < nk; ++c)
                mbar_wait_bounded(&full[c % MT_STAGES], (uint32_t)((c / MT_STAGES) & 1), kWaitPolls);
            sc->status = -5;   // PASD_ERR_TIMEOUT
            sc->done = 1;
            __threadfence();
        }
        return;
    }
    __syncthreads();   // all stages consumed, no copy in flight

    // ---- column groups added in order; rows of this strip (row of slot kk: see the reads) ----
    float* dst = m.part + ((int64_t)rg * I + i_lo) * Rp;
    auto row_of = [&](int qq, int kk) { return m.rowmajor ? 8 * qq + kk : qq + kk * nq8; };
    if (KG > 1) {
        float* red = smem;      // [KG][ntask][32]
        if (active) {
            float4* o = reinterpret_cast<float4*>(red + ((size_t)kg * ntask + task) * 32);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) o[kk] = make_float4(acc[kk][0], acc[kk][1], acc[kk][2], acc[kk][3]);
        }
        __syncthreads();
        for (int w = t; w < ntask * 8; w += MP_THREADS) {
            const int tk = w >> 3, kk = w & 7;
            const int qq = tk / nrq, rr = tk % nrq;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int g = 0; g < KG; ++g) {
                const float4 v = *reinterpret_cast<const float4*>(red + ((size_t)g * ntask + tk) * 32 + 4 * kk);
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            const int row = row_of(qq, kk);
            if (row < IS) *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rr) = sum;
        }
    } else if (active) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
            const int row = row_of(q, kk);
            if (row < IS)
                *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rq) =
                    make_float4(acc[kk][0], acc[kk][1], acc[kk][2], acc[kk][3]);
        }
    }
}

__global__ void __launch_bounds__(MP_THREADS) mpass_tma_kernel(const __grid_constant__ MpassTmaMaps maps,
                                                               const MpassTmaArgs ma) {
    mpass_tma_body(maps, ma, blockIdx.x);
}

// Batched: CTAs [start, start + ctas) of an entry run one solve's M-pass.
struct MpassBatchEntry {
    MpassTmaMaps maps;
    MpassTmaArgs args;
    int start;
};
__global__ void __launch_bounds__(MP_THREADS) mpass_tma_kernel_batched(const MpassBatchEntry* e, const int* block_entry) {
    const MpassBatchEntry& x = e[block_entry[blockIdx.x]];
    __shared__ __align__(16) MpassTmaArgs s_ma;
    load_args_to_smem(&s_ma, &x.args);
    const int block = blockIdx.x - x.start;
    if (threadIdx.x == 0) {
        int k = 0;
        while (k + 1 < s_ma.N && block >= s_ma.cta_start[k + 1]) ++k;
        tensormap_acquire(&x.maps.g[k]);
        tensormap_acquire(&x.maps.v[k]);
    }
    mpass_tma_body(x.maps, s_ma, block);
}

bool mpass_tma_supported(int64_t I, int64_t post) {
    if (post == 1) return I % 4 == 0;
    return post % 4 == 0 && post >= MP_CB;
}

int mpass_tma_chunks(int64_t pre, int64_t post) {
    if (post == 1) return (int)((pre + MP_CB - 1) / MP_CB);
    return (int)(pre * ((post + MP_CB - 1) / MP_CB));
}

size_t mpass_tma_smem_bytes(int IS, int Rp) {
    size_t pipe = (size_t)MT_STAGES * mt_stage_floats(IS, Rp);
    size_t red = (size_t)MP_THREADS * 32;
    return 4 * (pipe > red ? pipe : red) + 1024;
}

int mpass_tma_ctas_per_sm(size_t smem) {
    set_smem_attr((const void*)mpass_tma_kernel, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mpass_tma_kernel, MP_THREADS, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

MpassTmaPlan* make_mpass_tma(const MpassTmaArgs& a, const float* const* G, const float* const* V, size_t smem,
                             char* err, size_t errlen) {
    MpassTmaPlan* p = new MpassTmaPlan();
    std::memset(&p->maps, 0, sizeof(p->maps));
    p->args = a;
    p->smem = smem;
    for (int n = 0; n < a.N; ++n) {
        const MpassTmaMode& mm = a.m[n];
        bool ok;
        if (!mm.rowmajor) {
            uint64_t d[3] = {(uint64_t)mm.post, (uint64_t)mm.I, (uint64_t)mm.pre};
            uint32_t b[3] = {(uint32_t)MP_CB, (uint32_t)mm.IS, 1u};
            ok = encode_tiled_f32(&p->maps.g[n], G[n], 3, d, b, CU_TENSOR_MAP_SWIZZLE_128B, err, errlen, "M-pass G");
            uint64_t dv[3] = {(uint64_t)mm.post, (uint64_t)mm.Rp, (uint64_t)mm.pre};
            uint32_t bv[3] = {(uint32_t)MP_CB, (uint32_t)mm.Rp, 1u};
            ok = ok && encode_tiled_f32(&p->maps.v[n], V[n], 3, dv, bv, CU_TENSOR_MAP_SWIZZLE_128B, err, errlen, "M-pass Vrot");
        } else {
            uint64_t d[2] = {(uint64_t)mm.I, (uint64_t)mm.pre};
            uint32_t b[2] = {(uint32_t)mm.IS, (uint32_t)MP_CB};
            ok = encode_tiled_f32(&p->maps.g[n], G[n], 2, d, b, CU_TENSOR_MAP_SWIZZLE_NONE, err, errlen, "M-pass G");
            uint64_t dv[2] = {(uint64_t)mm.Rp, (uint64_t)mm.pre};
            uint32_t bv[2] = {(uint32_t)mm.Rp, (uint32_t)MP_CB};
            ok = ok && encode_tiled_f32(&p->maps.v[n], V[n], 2, dv, bv, CU_TENSOR_MAP_SWIZZLE_NONE, err, errlen, "M-pass Vrot");
        }
        if (!ok) { delete p; return nullptr; }
    }
    return p;
}

size_t mpass_batch_entry_bytes() { return sizeof(MpassBatchEntry); }
int mpass_batch_ctas(const MpassTmaPlan* p) { return p->args.cta_start[p->args.N]; }
size_t mpass_batch_smem(const MpassTmaPlan* p) { return p->smem; }
void mpass_batch_fill(void* entry, const MpassTmaPlan* p, int start) {
    // built in an aligned local and copied: `entry` points into a byte staging
    // buffer that need not meet the tensor maps' 64-byte alignment
    MpassBatchEntry e;
    std::memset(&e, 0, sizeof(e));
    e.maps = p->maps;
    e.args = p->args;
    e.start = start;
    std::memcpy(entry, &e, sizeof(e));
}
void launch_mpass_batched(const void* entries, const int* block_entry, int grid, size_t smem, cudaStream_t s) {
    set_smem_attr((const void*)mpass_tma_kernel_batched, (int)smem);
    mpass_tma_kernel_batched<<<grid, MP_THREADS, smem, s>>>(static_cast<const MpassBatchEntry*>(entries), block_entry);
}

void launch_mpass_tma(const MpassTmaPlan* p, cudaStream_t s) {
    set_smem_attr((const void*)mpass_tma_kernel, (int)p->smem);
    mpass_tma_kernel<<<p->args.cta_start[p->args.N], MP_THREADS, p->smem, s>>>(p->maps, p->args);
}

void destroy_mpass_tma(MpassTmaPlan* p) { delete p; }

}  // namespace pasd
