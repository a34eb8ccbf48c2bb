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

#include <algorithm>

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

size_t apass_smem_bytes(int Rp, bool rowmajor) {
    size_t gs = (size_t)AP_STAGES * (rowmajor ? AP_BN * (AP_BK + 4) : AP_BK * (AP_BN + 4));
    size_t us = (size_t)AP_STAGES * AP_BK * Rp;
    size_t pipe = gs + us;
    size_t epi = (size_t)AP_BN * (Rp + 4);
    int nb = Rp / 4, nbt = nb * (nb + 1) / 2;
    int nsl = nbt >= AP_THREADS ? 1 : AP_THREADS / nbt;
    size_t red = (size_t)nsl * nbt * 16;
    return 4 * ((pipe > epi ? pipe : epi) + red);
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

    float acc0[RP], acc1[RP];
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

    // ---- Gram partial: sum over this CTA's columns of A[:, j] A[:, j]^T ----
    constexpr int ALD = RP + 4;
    float* As = smem;   // [AP_BN][ALD] (reuses the pipeline buffers)
#pragma unroll
    for (int r4 = 0; r4 < RP / 4; ++r4) {
        *reinterpret_cast<float4*>(As + t * ALD + 4 * r4) =
            make_float4(acc0[4 * r4], acc0[4 * r4 + 1], acc0[4 * r4 + 2], acc0[4 * r4 + 3]);
        *reinterpret_cast<float4*>(As + (t + 128) * ALD + 4 * r4) =
            make_float4(acc1[4 * r4], acc1[4 * r4 + 1], acc1[4 * r4 + 2], acc1[4 * r4 + 3]);
    }
    constexpr int NB = RP / 4;
    constexpr int NBT = NB * (NB + 1) / 2;
    constexpr int NSL = NBT >= AP_THREADS ? 1 : AP_THREADS / NBT;
    size_t pipe = (size_t)AP_STAGES * (L::gs_stage + AP_BK * RP);
    size_t epi = (size_t)AP_BN * ALD;
    float* red = smem + (pipe > epi ? pipe : epi);
    __syncthreads();
    for (int w = t; w < NBT * NSL; w += AP_THREADS) {
        int blk = w % NBT, sl = w / NBT;
        int bi = 0, rem = blk;
        while (rem >= NB - bi) { rem -= NB - bi; ++bi; }
        int bj = bi + rem;
        float g[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) g[q] = 0.f;
        for (int c = sl; c < AP_BN; c += NSL) {
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
    __syncthreads();
    float* gp = a.gram_part + (size_t)cta * RP * RP;
    for (int o = t; o < NBT * 16; o += AP_THREADS) {
        int blk = o / 16, q = o % 16;
        float s = 0.f;
        for (int sl = 0; sl < NSL; ++sl) s += red[(sl * NBT + blk) * 16 + q];
        int bi = 0, rem = blk;
        while (rem >= NB - bi) { rem -= NB - bi; ++bi; }
        int bj = bi + rem;
        int r = 4 * bi + q / 4, c = 4 * bj + q % 4;
        gp[r * RP + c] = s;
        gp[c * RP + r] = s;
    }
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
    cudaFuncSetAttribute(apass_kernel<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

}  // namespace pasd
