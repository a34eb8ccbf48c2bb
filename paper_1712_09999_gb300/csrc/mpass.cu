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
//              column groups XOR-swizzled by row block, so the four row loads of
//              a thread at one column hit distinct banks across the warp
//   post == 1: a chunk is MP_CB columns of IS rows   -> smem [col][i]
// and the matching Vrot_n columns -> smem [col][r]. Each thread accumulates a
// 4-row x 4-rank FP32 register tile over all of its columns (FFMA); when few
// ranks are kept, idle threads take alternate columns and the tiles are added
// in a fixed order at the end. One partial M per column range is written to
// part[range][I][Rp]; the finalize kernel sums them in a fixed order, so the
// result does not depend on timing.
#include "pasd_impl.cuh"

#include <algorithm>

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

// Stage sizes (floats) for a mode.
// (rows rounded up to whole 4-row blocks, which the register tiles read)
static inline __host__ __device__ int mp_g_stage(int IS, int variant) {
    (void)variant;
    return MP_CB * ((IS + 3) / 4 * 4);
}
static inline __host__ __device__ int mp_v_stage(int Rp) { return MP_CB * Rp; }

size_t mpass_smem_bytes(int IS, int Rp, int variant) {
    size_t stage = (size_t)mp_g_stage(IS, variant) + mp_v_stage(Rp);
    size_t red = (size_t)MP_THREADS * 16;
    size_t pipe = (size_t)MP_STAGES * stage;
    return 4 * (pipe > red ? pipe : red);
}

int mpass_variant(int64_t I, int64_t post) {
    if (post == 1) return (I % 4 == 0) ? 2 : 3;
    return (post % 4 == 0) ? 0 : 1;
}

int mpass_strip_rows(int64_t I, int Rp) {
    int cap = 4 * (MP_THREADS / (Rp / 4));
    cap = std::min(cap, 256);
    return (int)std::min<int64_t>(I, cap);
}

template <int V>
__device__ __forceinline__ void mpass_body(const MpassMode& m, int s, int cta, float* smem) {
    constexpr bool colmajor = (V >= 2);      // smem [col][i]
    const int t = threadIdx.x;
    const int strip = cta % m.nstrips, cg = cta / m.nstrips;
    const int64_t I = m.I, post = m.post, P = m.P;
    const int64_t i_lo = (int64_t)strip * m.IS;
    const int IS = (int)((I - i_lo) < m.IS ? (I - i_lo) : m.IS);
    const int LDI = (m.IS + 3) / 4 * 4;
    const int64_t c_lo = (int64_t)cg * m.cols_per_cg;
    const int64_t c_hi = (c_lo + m.cols_per_cg) < P ? (c_lo + m.cols_per_cg) : P;
    const int nk = c_hi > c_lo ? (int)((c_hi - c_lo + MP_CB - 1) / MP_CB) : 0;
    const int Rp = m.Rp;
    const int gst = mp_g_stage(m.IS, V), vst = mp_v_stage(Rp);
    float* Gs = smem;
    float* Vs = smem + MP_STAGES * gst;
    const float* __restrict__ G = m.G;
    const float* __restrict__ Vr = m.V;

    // thread -> (task, column group inside the CTA); task -> (row block q, rank block rq)
    const int nrq = s / 4;
    const int nq = (IS + 3) / 4;
    const int ntask = nq * nrq;
    const int KG = (ntask > 0 && MP_THREADS / ntask > 1) ? MP_THREADS / ntask : 1;
    const int task = ntask > 0 ? t % ntask : 0;
    const int kg = ntask > 0 ? t / ntask : KG;
    const bool active = kg < KG;
    const int q = task / (nrq > 0 ? nrq : 1), rq = task % (nrq > 0 ? nrq : 1);

    auto issue = [&](int kc, int st) {
        const int64_t j0 = c_lo + (int64_t)kc * MP_CB;
        float* gs = Gs + st * gst;
        if (V == 0) {
            // 16-byte column groups; the group index of a thread is fixed (t % 8)
            const int cs = t & 7;
            const int64_t j = j0 + 4 * cs;
            const bool jok = j < c_hi;
            const int64_t aa = jok ? j / post : 0, bb = jok ? j % post : 0;
            const float* base = G + (aa * I + i_lo) * post + bb;
            for (int row = t >> 3; row < IS; row += MP_THREADS / 8) {
                const float* src = jok ? base + (int64_t)row * post : G;
                const int phys = cs ^ ((row >> 2) & 7);
                cp_async16(gs + row * MP_CB + 4 * phys, src, jok ? 16 : 0);
            }
        } else if (V == 1) {
            const int c = t & (MP_CB - 1);
            const int64_t j = j0 + c;
            const bool jok = j < c_hi;
            const int64_t aa = jok ? j / post : 0, bb = jok ? j % post : 0;
            const float* base = G + (aa * I + i_lo) * post + bb;
            for (int row = t / MP_CB; row < IS; row += MP_THREADS / MP_CB) {
                const int pc = (((c >> 2) ^ ((row >> 2) & 7)) << 2) | (c & 3);
                const float* src = jok ? base + (int64_t)row * post : G;
                cp_async4(gs + row * MP_CB + pc, src, jok ? 4 : 0);
            }
        } else if (V == 2) {
            const int IS4 = (IS + 3) / 4;
            for (int idx = t; idx < MP_CB * IS4; idx += MP_THREADS) {
                const int iseg = idx % IS4, c = idx / IS4;
                const int64_t j = j0 + c;
                const bool ok = j < c_hi;
                const float* src = ok ? G + j * I + i_lo + 4 * iseg : G;
                cp_async16(gs + c * LDI + 4 * iseg, src, ok ? 16 : 0);
            }
        } else {
            for (int idx = t; idx < MP_CB * IS; idx += MP_THREADS) {
                const int i = idx % IS, c = idx / IS;
                const int64_t j = j0 + c;
                const bool ok = j < c_hi;
                const float* src = ok ? G + j * I + i_lo + i : G;
                cp_async4(gs + c * LDI + i, src, ok ? 4 : 0);
            }
        }
        // Vrot columns j0 .. j0 + MP_CB, kept rows, into [col][r]
        float* vs = Vs + st * vst;
        for (int idx = t; idx < MP_CB * s; idx += MP_THREADS) {
            const int c = idx % MP_CB, r = idx / MP_CB;
            const int64_t j = j0 + c;
            const bool ok = j < c_hi;
            const int64_t aa = ok ? j / post : 0, bb = ok ? j % post : 0;
            const float* src = ok ? Vr + (aa * Rp + r) * post + bb : Vr;
            cp_async4(vs + c * Rp + r, src, ok ? 4 : 0);
        }
    };

    float acc[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
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
                const float* gq = gs + 4 * q;
#pragma unroll 4
                for (int c = kg; c < MP_CB; c += KG) {
                    const float4 g = *reinterpret_cast<const float4*>(gq + c * LDI);
                    const float4 v = *reinterpret_cast<const float4*>(vs + c * Rp);
                    const float gg[4] = {g.x, g.y, g.z, g.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[k][r] = fmaf(gg[k], vv[r], acc[k][r]);
                }
            } else {
                const int sw = q & 7;
                const float* gq = gs + (4 * q) * MP_CB;
#pragma unroll 4
                for (int c = kg; c < MP_CB; c += KG) {
                    const int pc = (((c >> 2) ^ sw) << 2) | (c & 3);
                    const float gg[4] = {gq[pc], gq[MP_CB + pc], gq[2 * MP_CB + pc], gq[3 * MP_CB + pc]};
                    const float4 v = *reinterpret_cast<const float4*>(vs + c * Rp);
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int k = 0; k < 4; ++k)
#pragma unroll
                        for (int r = 0; r < 4; ++r) acc[k][r] = fmaf(gg[k], vv[r], acc[k][r]);
                }
            }
        }
    }
    cp_wait<0>();
    __syncthreads();
    if (ntask == 0) return;

    // ---- the column groups of the CTA, added in order; partial rows of this strip ----
    float* dst = m.part + ((int64_t)cg * I + i_lo) * Rp;
    if (KG > 1) {
        float* red = smem;      // [KG][ntask][16], reuses the pipeline buffers
        if (active) {
            float4* o = reinterpret_cast<float4*>(red + ((size_t)kg * ntask + task) * 16);
#pragma unroll
            for (int k = 0; k < 4; ++k) o[k] = make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
        }
        __syncthreads();
        for (int w = t; w < ntask * 4; w += MP_THREADS) {
            const int tk = w >> 2, k = w & 3;
            const int qq = tk / nrq, rr = tk % nrq;
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int g = 0; g < KG; ++g) {
                const float4 v = *reinterpret_cast<const float4*>(red + ((size_t)g * ntask + tk) * 16 + 4 * k);
                sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            }
            const int row = 4 * qq + k;
            if (row < IS) *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rr) = sum;
        }
    } else if (active) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int row = 4 * q + k;
            if (row < IS)
                *reinterpret_cast<float4*>(dst + (int64_t)row * Rp + 4 * rq) =
                    make_float4(acc[k][0], acc[k][1], acc[k][2], acc[k][3]);
        }
    }
}

__global__ void __launch_bounds__(MP_THREADS) mpass_kernel(const MpassArgs ma) {
    extern __shared__ __align__(16) float smem[];
    const DevScalars* sc = ma.sc;
    if (sc->done) return;
    int k = 0;
    while (k + 1 < ma.N && (int)blockIdx.x >= ma.cta_start[k + 1]) ++k;
    const MpassMode& m = ma.m[k];
    const int s = (sc->kept[k] + 3) & ~3;      // kept rows rounded up (Vrot rows past s_n are zero)
    if (s == 0) return;                        // no kept direction: the U-step does not read M_n
    const int cta = blockIdx.x - ma.cta_start[k];
    switch (m.variant) {
        case 0: mpass_body<0>(m, s, cta, smem); break;
        case 1: mpass_body<1>(m, s, cta, smem); break;
        case 2: mpass_body<2>(m, s, cta, smem); break;
        default: mpass_body<3>(m, s, cta, smem); break;
    }
}

int mpass_ctas_per_sm(size_t smem) {
    cudaFuncSetAttribute(mpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mpass_kernel, MP_THREADS, smem) != cudaSuccess || n < 1)
        n = 1;
    return n;
}

void launch_mpass(const MpassArgs& a, size_t smem, cudaStream_t s) {
    cudaFuncSetAttribute(mpass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mpass_kernel<<<a.cta_start[a.N], MP_THREADS, smem, s>>>(a);
}

}  // namespace pasd
