// TMA-fed fused elementwise pass (same arithmetic as fused.cu, which stays as
// the path for N > 4 or a contiguous mode whose length is not a multiple of 4).
//
// Per tile (a box of extents b_n), one lane of a producer warp issues bulk
// tensor copies (cp.async.bulk.tensor) into a ring of stages while the
// consumer warps compute earlier tiles; full / empty mbarriers pass each stage
// between them:
//   Xs   : T, E, G_0..G_{N-1} boxes, C order of the box (element index e)
//   As_n : the Vrot_n columns the tile needs (kept rows), a box of the N-D
//          tensor Vrot_n ([pre][Rp][post] viewed with I_n replaced by Rp),
//          i.e. smem layout [c_hi][r][c_lo] (c_lo = the post-mode part of the
//          column index) for n < N-1 and [c][r] for the contiguous mode
//   Ws_n : rows o_n .. o_n + b_n of Urot_n ([l][r])
// Out-of-range parts of a box are zero-filled by the copy engine, so the
// arithmetic below needs no masks: a zero element stays zero through the
// update and adds nothing to the residual sums.
// Results (E', G_n') go from registers straight to HBM as 16-byte stores (four
// consecutive elements of the contiguous mode, whose length is a multiple of 4
// here), so a stage is free for the next copy as soon as every warp has read
// it: no shared-memory write-back and no store to wait for before a refill.
#include "pasd_impl.cuh"
#include "tma.cuh"

#include <cuda.h>
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstring>

namespace pasd {

bool plan_geom_impl(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                    size_t smem_limit, bool tma);

// Tensor maps only: passed as a __grid_constant__ parameter because the bulk
// copies take their address. Everything else goes in a plain by-value
// parameter (constant-bank operands, no memory loads).
constexpr int kTmaMaxN = 4;            // the TMA pass handles N <= 4
constexpr int kMaxStages = 4;          // element-tile stages while nothing is kept
constexpr int kHeights = PASD_MAXR / 4;  // one map per row count 4, 8, ..., 64
struct FusedTmaMaps {
    CUtensorMap tm_x[kTmaMaxN + 2];          // T copy, E, G_0..G_{N-1}
    CUtensorMap tm_a[kTmaMaxN][kHeights];    // Vrot_n, first 4(h+1) rows
    CUtensorMap tm_w[kTmaMaxN][kHeights];    // Urot_n, first 4(h+1) columns
};

struct FusedTmaPlan {
    FusedTmaMaps maps;
    FusedArgs base;
};

// CTA size: the consumer warps over the g.nthreads micro-boxes, then the producer warp
static int fused_block_threads(const FusedGeom& g) { return ((g.nthreads + 31) / 32 + 1) * 32; }


// ---------------------------------------------------------------------------
// kernel
// ---------------------------------------------------------------------------
// Only the kept directions carry Z_n: with s_n kept singular values,
// Z_n = Urot[:, :s] Vrot[:s], so per element and mode the pass does
// sp_n = round_up(s_n, 4) multiply-adds and loads only sp_n rows of Vrot and
// columns of Urot (one tensor map per height). The next U-step's product
// G_n' Vrot^T is formed by the M-pass that follows.
template <int N, int SM>
__device__ __forceinline__ void fused_tma_body(const FusedTmaMaps& tm, const FusedArgs& fa, const int output,
                                               float* const Lout, const int block) {
    DevScalars* sc = fa.sc;
    if (!output && sc->done) return;
    const FusedGeom& g = fa.g;
    extern __shared__ __align__(1024) float sm_raw[];
    // stage buffers aligned to 1024 bytes (the launch adds 1 KB of slack)
    float* sm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(sm_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full_bar[kMaxStages];    // stage filled (copies landed)
    __shared__ __align__(8) uint64_t empty_bar[kMaxStages];   // stage read by every consumer warp
    __shared__ int tile_o[kMaxStages][N];   // origins of the tiles in the stages
    __shared__ int s_fail;
    __shared__ long long s_fail_it;
    const int t = threadIdx.x;
    // warp roles: ncw consumer warps own the micro-boxes (threads t < nthr), the
    // last warp issues every copy, so no consumer waits on a copy's issue
    const int nthr = g.nthreads;
    const int ncw = (nthr + 31) >> 5;
    const bool producer = t >= ncw * 32;
    const bool comp = t < nthr;
    const int B = g.B;

    int sp[N];                         // kept count rounded up to 4 (0: mode has no low-rank part)
    uint32_t tx = output ? 0u : (uint32_t)(4 * (N + 2) * B);
#pragma unroll
    for (int n = 0; n < N; ++n) {
        sp[n] = (sc->kept[n] + 3) & ~3;
        tx += (uint32_t)(4 * (g.C[n] + g.b[n]) * sp[n]);
    }

    int q[N];
    {
        int r = block;
        for (int n = N - 1; n >= 0; --n) { q[n] = r % g.Q[n]; r /= g.Q[n]; }
    }
    int64_t ts[N], te[N];
    int64_t ntile = 1;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        ts[n] = (int64_t)q[n] * g.nt[n] / g.Q[n];
        te[n] = (int64_t)(q[n] + 1) * g.nt[n] / g.Q[n];
        ntile *= te[n] - ts[n];
    }
    // odometer over the region's tiles (C order), advanced by the producer lane
    int tc[N];
#pragma unroll
    for (int n = 0; n < N; ++n) tc[n] = (int)ts[n];

    // micro-box of this thread: two groups of 4 consecutive elements along mode
    // N-1, half = b_SM / 2 apart along the split mode SM. With SM = N-2 the 8
    // lanes of a quarter-warp read 8 consecutive 16-byte groups (no bank
    // conflicts) in the element tiles and in the Vrot slices of the modes before
    // N-2 when (b_{N-1} / 4) (b_{N-2} / 2) >= 8; otherwise (SM = 0) thread t takes
    // elements 4 t .. 4 t + 3 of the tile's first half and the same of its second
    const int half = g.b[SM] / 2;
    int u0[N];
    if (SM == N - 2) {
#pragma unroll
        for (int n = 0; n < N; ++n)
            u0[n] = ((t >> g.mbsh[n]) & (g.b[n] / g.mb[n] - 1)) * (n == N - 2 ? 1 : g.mb[n]);
    } else {
#pragma unroll
        for (int n = 0; n < N; ++n) u0[n] = ((4 * t) >> g.esh[n]) & (g.b[n] - 1);
    }
    int e0 = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) e0 += u0[n] << g.esh[n];
    int cb[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
        int c = 0;
#pragma unroll
        for (int m = 0; m < N; ++m)
            if (m != n) c += u0[m] << g.csh[n][m];
        cb[n] = c;
    }

    const double mu = sc->mu;
    double mun = fa.rho * mu;
    if (mun > fa.mu_max) mun = fa.mu_max;
    const float cfac = (float)(mu / mun);
    const float thr = (float)(1.0 / (mu * N));
    const float invN = 1.0f / N;
    float resmax = 0.f, l1 = 0.f, chk = 0.f, res2[N];
#pragma unroll
    for (int n = 0; n < N; ++n) res2[n] = 0.f;

    // Stages. With nothing kept (pure streaming) a stage holds only the element
    // tiles, so the same shared memory holds up to kMaxStages of them; with a
    // refold to compute, two full stages alternate. The producer lane fills a
    // stage as soon as every consumer warp has released it (empty barrier), so
    // copies run up to nst tiles ahead of the arithmetic.
    bool early = !output;
#pragma unroll
    for (int n = 0; n < N; ++n) early = early && sp[n] == 0;
    const int xs_stride = (((N + 2) * B + 255) / 256) * 256;   // 1 KB multiples
    int nst = 2, sstride = g.stage_floats;
    if (early) {
        nst = g.smem_floats / xs_stride;
        nst = nst < kMaxStages ? nst : kMaxStages;
        if (nst >= 2 && g.xs_off == 0) sstride = xs_stride; else nst = 2;
    }
    if (t == 0) {
        for (int i = 0; i < nst; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], ncw);
        }
        s_fail = 0;
        s_fail_it = LLONG_MAX;
        fence_mbar_init();
    }
    __syncthreads();

    const uint32_t polls = fa.wait_polls ? fa.wait_polls : kWaitPolls;
    // producer lane: origins, odometer, barrier arming and the copies of one tile
    auto issue = [&](int st) {
        int o[N];
#pragma unroll
        for (int n = 0; n < N; ++n) { o[n] = tc[n] * g.b[n]; tile_o[st][n] = o[n]; }
#pragma unroll
        for (int n = N - 1; n >= 0; --n) {
            if (++tc[n] < te[n]) break;
            tc[n] = (int)ts[n];
        }
        float* stg = sm + st * sstride;
        uint64_t* bar = &full_bar[st];
        mbar_expect_tx(bar, tx);
        int cx[N];
#pragma unroll
        for (int k = 0; k < N; ++k) cx[k] = o[N - 1 - k];
        if (!output)
#pragma unroll
            for (int a = 0; a < N + 2; ++a) tma_load<N>(stg + g.xs_off + a * B, &tm.tm_x[a], bar, cx);
#pragma unroll
        for (int n = 0; n < N; ++n) {
            if (sp[n] == 0) continue;
            const int h = sp[n] / 4 - 1;
            int ca[N];
#pragma unroll
            for (int k = 0; k < N; ++k) ca[k] = (N - 1 - k == n) ? 0 : o[N - 1 - k];
            tma_load<N>(stg + g.as_off[n], &tm.tm_a[n][h], bar, ca);
            int cw[2] = {0, o[n]};
            tma_load<2>(stg + g.ws_off[n], &tm.tm_w[n][h], bar, cw);
        }
    };

    int64_t issued = 0;      // producer lane: tiles whose copies went out
    if (producer) {
        if ((t & 31) == 0 && !fa.test_no_copy) {   // test hook: no arrival, no copy in flight
            for (int64_t i = 0; i < ntile; ++i) {
                const int st = (int)(i % nst);
                // stage st last held tile i - nst: wait until every consumer warp read it
                if (i >= nst && !mbar_wait_bounded(&empty_bar[st], (uint32_t)((i / nst - 1) & 1), polls)) break;
                issue(st);
                issued = i + 1;
            }
        }
    }
    // consumer warps advance independently, at most nst tiles apart (the ring)
    for (int64_t it = 0; !producer && it < ntile; ++it) {
        const int st = (int)(it % nst);
        const uint32_t par = (uint32_t)((it / nst) & 1);
        const bool ok = mbar_wait_bounded(&full_bar[st], par, polls);
        if (!__all_sync(0xffffffffu, ok)) {
            // this warp gives up at tile it; the earliest such tile is recorded
            if ((t & 31) == 0) {
                s_fail = 1;
                atomicMin(&s_fail_it, (long long)it);
            }
            break;
        }
        float* stg = sm + st * sstride;
        float* Xs = stg + g.xs_off;
        int o[N];
#pragma unroll
        for (int n = 0; n < N; ++n) o[n] = tile_o[st][n];

        if (comp) {
        // ---- Z_n for the thread's 8 elements (j = d2 * 4 + d1), rank sp_n ----
        // Z_n in pairs (z2) for the modes before the last, whose products pair up
        // along the contiguous mode; the last mode's chains stay scalar (z)
        float z[N][8];
        float2 z2[N][4];
#pragma unroll
        for (int n = 0; n < N; ++n)
#pragma unroll
            for (int j = 0; j < 8; ++j) z[n][j] = 0.f;
#pragma unroll
        for (int n = 0; n < N; ++n)
#pragma unroll
            for (int j = 0; j < 4; ++j) z2[n][j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const int h = sp[n];
            if (h == 0) continue;
            const float* As = stg + g.as_off[n];     // Vrot slice, row stride per block = h
            const float* Ws = stg + g.ws_off[n];     // Urot rows [l][h]
            if (n == N - 1) {
                const float* Wt = Ws + u0[n] * h;
                const float* At = As + cb[n] * h;
                const int a2 = (half << g.csh[n][SM]) * h;    // column of the second group
                for (int r = 0; r < h; r += 4) {
                    float4 w[4];
#pragma unroll
                    for (int d1 = 0; d1 < 4; ++d1) w[d1] = *reinterpret_cast<const float4*>(Wt + d1 * h + r);
#pragma unroll
                    for (int d2 = 0; d2 < 2; ++d2) {
                        const float4 a = *reinterpret_cast<const float4*>(At + d2 * a2 + r);
#pragma unroll
                        for (int d1 = 0; d1 < 4; ++d1) {
                            float acc = z[n][d2 * 4 + d1];
                            acc = fmaf(w[d1].x, a.x, acc);
                            acc = fmaf(w[d1].y, a.y, acc);
                            acc = fmaf(w[d1].z, a.z, acc);
                            z[n][d2 * 4 + d1] = fmaf(w[d1].w, a.w, acc);
                        }
                    }
                }
            } else {
                const int H = g.esh[n];
                const int chi = cb[n] >> H, clo = cb[n] & ((1 << H) - 1);
                const int rs = 1 << H;
                const float* Ab = As + ((chi * h) << H) + clo;
                const float* Wt = Ws + u0[n] * h;
                if (n == SM) {
                    for (int r = 0; r < h; r += 4) {
                        const float4 w0 = *reinterpret_cast<const float4*>(Wt + r);
                        const float4 w1 = *reinterpret_cast<const float4*>(Wt + half * h + r);
                        const float w0s[4] = {w0.x, w0.y, w0.z, w0.w}, w1s[4] = {w1.x, w1.y, w1.z, w1.w};
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            // paired FMAs: each lane rounds as fmaf, in the same order
                            const float4 a = *reinterpret_cast<const float4*>(Ab + (r + kk) * rs);
                            const float2 axy = make_float2(a.x, a.y), azw = make_float2(a.z, a.w);
                            const float2 w0 = make_float2(w0s[kk], w0s[kk]), w1 = make_float2(w1s[kk], w1s[kk]);
                            z2[n][0] = __ffma2_rn(w0, axy, z2[n][0]);
                            z2[n][1] = __ffma2_rn(w0, azw, z2[n][1]);
                            z2[n][2] = __ffma2_rn(w1, axy, z2[n][2]);
                            z2[n][3] = __ffma2_rn(w1, azw, z2[n][3]);
                        }
                    }
                } else {
                    // the second group's column: a post mode of n moves c_lo, a pre
                    // mode (SM = 0 < n) moves c_hi, whose stride is h rows of 2^H
                    const int s2 = SM > n ? (half << g.csh[n][SM]) : (half << g.csh[n][SM]) * h;
                    for (int r = 0; r < h; r += 4) {
                        const float4 w = *reinterpret_cast<const float4*>(Wt + r);
                        const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const float2 w2 = make_float2(ws[kk], ws[kk]);
#pragma unroll
                            for (int d2 = 0; d2 < 2; ++d2) {
                                const float4 a = *reinterpret_cast<const float4*>(Ab + (r + kk) * rs + d2 * s2);
                                z2[n][2 * d2] = __ffma2_rn(w2, make_float2(a.x, a.y), z2[n][2 * d2]);
                                z2[n][2 * d2 + 1] = __ffma2_rn(w2, make_float2(a.z, a.w), z2[n][2 * d2 + 1]);
                            }
                        }
                    }
                }
            }
        }

#pragma unroll
        for (int n = 0; n < N - 1; ++n)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                z[n][2 * j] = z2[n][j].x;
                z[n][2 * j + 1] = z2[n][j].y;
            }

        if (output) {
            // L = sum_n alpha_n Z_n / sum alpha_n, stored directly (once per solve)
            int64_t tbase = 0;
            bool vbase = true;
#pragma unroll
            for (int n = 0; n < N; ++n) tbase += (int64_t)(o[n] + u0[n]) * g.stride[n];
#pragma unroll
            for (int n = 0; n < N - 1; ++n)
                if (n != SM) vbase = vbase && (o[n] + u0[n] < g.I[n]);
#pragma unroll
            for (int d2 = 0; d2 < 2; ++d2) {
                const bool v2 = vbase && (o[SM] + u0[SM] + d2 * half < g.I[SM]);
                const int64_t rowoff = tbase + (int64_t)(d2 * half) * g.stride[SM];
#pragma unroll
                for (int d1 = 0; d1 < 4; ++d1) {
                    if (v2 && (o[N - 1] + u0[N - 1] + d1 < g.I[N - 1])) {
                        float s = 0.f;
#pragma unroll
                        for (int n = 0; n < N; ++n) s = fmaf(fa.alpha_w[n], z[n][d2 * 4 + d1], s);
                        Lout[rowoff + d1] = s;
                    }
                }
            }
        } else {

        // ---- elementwise update; results to HBM from registers ----
        //   gz_n = G_n - Z_n,  Ebar = mean_n(G_n + E - Z_n) = E + mean(gz),
        //   E' = prox(Ebar),  d = T - E',  r_n = d - Z_n,
        //   G_n' = d + (mu/mu') (gz_n + E - E')
        int64_t gbase = 0;
        bool valid = o[N - 1] + u0[N - 1] < g.I[N - 1];
#pragma unroll
        for (int n = 0; n < N; ++n) gbase += (int64_t)(o[n] + u0[n]) * g.stride[n];
#pragma unroll
        for (int n = 0; n < N - 1; ++n)
            if (n != SM) valid = valid && (o[n] + u0[n] < g.I[n]);
#pragma unroll
        for (int d2 = 0; d2 < 2; ++d2) {
            const int eb = e0 + ((d2 * half) << g.esh[SM]);
            float4 x = *reinterpret_cast<const float4*>(Xs + eb);
            const float tv[4] = {x.x, x.y, x.z, x.w};
            x = *reinterpret_cast<const float4*>(Xs + B + eb);
            const float ev[4] = {x.x, x.y, x.z, x.w};
            float gv[N][4];
#pragma unroll
            for (int n = 0; n < N; ++n) {
                x = *reinterpret_cast<const float4*>(Xs + (2 + n) * B + eb);
                gv[n][0] = x.x; gv[n][1] = x.y; gv[n][2] = x.z; gv[n][3] = x.w;
            }
            float en[4];
#pragma unroll
            for (int d1 = 0; d1 < 4; ++d1) {
                float sgz = 0.f;
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    gv[n][d1] -= z[n][d2 * 4 + d1];
                    sgz += gv[n][d1];
                }
                const float ebar = fmaf(sgz, invN, ev[d1]);
                const float mag = fabsf(ebar) - thr;
                const float e = mag > 0.f ? copysignf(mag, ebar) : 0.f;
                en[d1] = e;
                const float d = tv[d1] - e;
                const float qd = ev[d1] - e;
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    const float r = d - z[n][d2 * 4 + d1];
                    resmax = fmaxf(resmax, fabsf(r));
                    res2[n] = fmaf(r, r, res2[n]);
                    const float gnew = fmaf(cfac, gv[n][d1] + qd, d);
                    gv[n][d1] = gnew;
                    chk += gnew;
                }
                l1 += fabsf(e);
                chk += e;
            }
            if (valid && o[SM] + u0[SM] + d2 * half < g.I[SM]) {
                const int64_t e = gbase + (int64_t)(d2 * half) * g.stride[SM];
                *reinterpret_cast<float4*>(fa.E + e) = make_float4(en[0], en[1], en[2], en[3]);
#pragma unroll
                for (int n = 0; n < N; ++n)
                    *reinterpret_cast<float4*>(fa.G[n] + e) = make_float4(gv[n][0], gv[n][1], gv[n][2], gv[n][3]);
            }
        }
        }   // update
        }   // comp
        // stage st fully read by this warp
        __syncwarp();
        if ((t & 31) == 0) mbar_arrive(&empty_bar[st]);
    }
    __syncthreads();
    if (s_fail) {
        // a copy never arrived: leave once every tile issued from the earliest one a
        // warp gave up on (at most nst, one per stage: the tiles before it were read
        // by every warp) has been waited for in its own phase, bounded, so no copy
        // lands after the CTA has exited
        if (producer && (t & 31) == 0) {
            for (int64_t c = s_fail_it; c < issued; ++c)
                mbar_wait_bounded(&full_bar[c % nst], (uint32_t)((c / nst) & 1), polls);
            sc->status = -5;   // PASD_ERR_TIMEOUT
            sc->done = 1;
            __threadfence();
        }
        return;
    }
    if (output) return;

    // ---- block reductions of the residual statistics ----
    __shared__ float wred[FU_THREADS / 32][PASD_MAXN + 3];   // consumer warps
    const int nonfin = !isfinite(chk);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        resmax = fmaxf(resmax, __shfl_down_sync(0xffffffffu, resmax, off));
        l1 += __shfl_down_sync(0xffffffffu, l1, off);
#pragma unroll
        for (int n = 0; n < N; ++n) res2[n] += __shfl_down_sync(0xffffffffu, res2[n], off);
    }
    int nf = nonfin;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nf |= __shfl_down_sync(0xffffffffu, nf, off);
    const int wid = t >> 5, lane = t & 31;
    if (lane == 0 && !producer) {
        wred[wid][0] = resmax;
        wred[wid][1] = l1;
        wred[wid][2] = (float)nf;
#pragma unroll
        for (int n = 0; n < N; ++n) wred[wid][3 + n] = res2[n];
    }
    __syncthreads();
    if (t == 0) {
        float mx = 0.f, s1 = 0.f, nfs = 0.f, s2[N];
#pragma unroll
        for (int n = 0; n < N; ++n) s2[n] = 0.f;
        for (int w = 0; w < ncw; ++w) {
            mx = fmaxf(mx, wred[w][0]);
            s1 += wred[w][1];
            nfs = fmaxf(nfs, wred[w][2]);
#pragma unroll
            for (int n = 0; n < N; ++n) s2[n] += wred[w][3 + n];
        }
        float* p = fa.part + (size_t)block * fa.part_stride;
        p[0] = mx;
        p[1] = s1;
        p[2] = nfs;
#pragma unroll
        for (int n = 0; n < N; ++n) p[3 + n] = s2[n];
    }
}

template <int N, int SM>
__global__ void __launch_bounds__(FU_THREADS + 32, 1)
    fused_tma_kernel(const __grid_constant__ FusedTmaMaps tm, const FusedArgs fa, const int output,
                     float* const Lout) {
    fused_tma_body<N, SM>(tm, fa, output, Lout, blockIdx.x);
}

// Batched: the CTAs [start, start + nregions) of an entry run that solve's
// regions; its maps are read from global memory, its arguments from shared.
struct FusedBatchEntry {
    FusedTmaMaps maps;
    FusedArgs args;
    int start;
};
template <int N, int SM>
__global__ void __launch_bounds__(FU_THREADS + 32, 1)
    fused_tma_kernel_batched(const FusedBatchEntry* e, const int* block_entry) {
    const FusedBatchEntry& x = e[block_entry[blockIdx.x]];
    __shared__ __align__(16) FusedArgs s_fa;
    load_args_to_smem(&s_fa, &x.args);
    if (s_fa.sc->done) return;
    if (threadIdx.x == blockDim.x - 32) {   // the producer lane, which issues the copies
        for (int a = 0; a < N + 2; ++a) tensormap_acquire(&x.maps.tm_x[a]);
        for (int n = 0; n < N; ++n) {
            const int sp = (s_fa.sc->kept[n] + 3) & ~3;
            if (sp) { tensormap_acquire(&x.maps.tm_a[n][sp / 4 - 1]); tensormap_acquire(&x.maps.tm_w[n][sp / 4 - 1]); }
        }
    }
    fused_tma_body<N, SM>(x.maps, s_fa, 0, nullptr, blockIdx.x - x.start);
}

// ---------------------------------------------------------------------------
// host: planning, tensor maps, launch
// ---------------------------------------------------------------------------
bool plan_fused_tma(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                    size_t smem_limit) {
    if (N < 2 || N > kTmaMaxN) return false;
    if (I[N - 1] % 4 != 0) return false;
    for (int n = 0; n < N; ++n)
        if (I[n] >= (int64_t)1 << 31) return false;
    return plan_geom_impl(g, N, I, Rp, num_sms, smem_limit, true);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// dims / box innermost first (dense C-order array)
bool encode_tiled_f32(CUtensorMap* m, const float* base, int rank, const uint64_t* dims, const uint32_t* box,
                      CUtensorMapSwizzle swizzle, char* err, size_t errlen, const char* what) {
    EncodeTiledFn fn = get_encode();
    if (!fn) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled unavailable");
        return false;
    }
    cuuint64_t gd[5], gs[4];
    cuuint32_t bd[5], es[5];
    uint64_t stride = 4;
    for (int k = 0; k < rank; ++k) {
        gd[k] = dims[k];
        bd[k] = box[k];
        es[k] = 1;
        if (k > 0) gs[k - 1] = stride;
        stride *= dims[k];
    }
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(base), gd, gs, bd, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        snprintf(err, errlen, "cuTensorMapEncodeTiled(%s) failed with %d", what, (int)r);
        return false;
    }
    return true;
}

static bool encode(CUtensorMap* m, const float* base, int rank, const uint64_t* dims, const uint32_t* box,
                   char* err, size_t errlen, const char* what) {
    return encode_tiled_f32(m, base, rank, dims, box, CU_TENSOR_MAP_SWIZZLE_NONE, err, errlen, what);
}

FusedTmaPlan* make_fused_tma(const FusedArgs& a, const float* T_copy, char* err, size_t errlen) {
    const FusedGeom& g = a.g;
    const int N = g.N;
    FusedTmaPlan* p = new FusedTmaPlan();
    std::memset(&p->maps, 0, sizeof(p->maps));
    p->base = a;
    uint64_t dims[5];
    uint32_t box[5];
    for (int k = 0; k < N; ++k) { dims[k] = g.I[N - 1 - k]; box[k] = g.b[N - 1 - k]; }
    const float* xs[PASD_MAXN + 2];
    xs[0] = T_copy;
    xs[1] = a.E;
    for (int n = 0; n < N; ++n) xs[2 + n] = a.G[n];
    for (int i = 0; i < N + 2; ++i)
        if (!encode(&p->maps.tm_x[i], xs[i], N, dims, box, err, errlen, "element tile")) { delete p; return nullptr; }
    for (int n = 0; n < N; ++n) {
        for (int hh = 4; hh <= g.Rp[n]; hh += 4) {
            uint64_t ad[5];
            uint32_t ab[5];
            for (int k = 0; k < N; ++k) {
                int m = N - 1 - k;
                if (m == n) { ad[k] = g.Rp[n]; ab[k] = hh; }
                else { ad[k] = g.I[m]; ab[k] = g.b[m]; }
            }
            if (!encode(&p->maps.tm_a[n][hh / 4 - 1], a.A[n], N, ad, ab, err, errlen, "Vrot_n rows")) { delete p; return nullptr; }
            uint64_t wd[2] = {(uint64_t)g.Rp[n], (uint64_t)g.I[n]};
            uint32_t wb[2] = {(uint32_t)hh, (uint32_t)g.b[n]};
            if (!encode(&p->maps.tm_w[n][hh / 4 - 1], a.Wz[n], 2, wd, wb, err, errlen, "Urot_n rows")) { delete p; return nullptr; }
        }
    }
    return p;
}

void destroy_fused_tma(FusedTmaPlan* p) { delete p; }

template <int N, int SM>
static void launch_tma_n(FusedTmaPlan* p, int output, float* L, cudaStream_t s) {
    const FusedGeom& g = p->base.g;
    size_t smem = (size_t)g.smem_floats * 4 + 1024;
    set_smem_attr((const void*)fused_tma_kernel<N, SM>, (int)smem);
    fused_tma_kernel<N, SM><<<g.nregions, fused_block_threads(g), smem, s>>>(p->maps, p->base, output, L);
}

size_t fused_batch_entry_bytes() { return sizeof(FusedBatchEntry); }
int fused_batch_order(const FusedTmaPlan* p) { return p->base.g.N + 8 * p->base.g.split0; }
int fused_batch_ctas(const FusedTmaPlan* p) { return p->base.g.nregions; }
int fused_batch_threads(const FusedTmaPlan* p) { return fused_block_threads(p->base.g); }
size_t fused_batch_smem(const FusedTmaPlan* p) { return (size_t)p->base.g.smem_floats * 4 + 1024; }
void fused_batch_fill(void* entry, const FusedTmaPlan* p, int start) {
    // built in an aligned local and copied: `entry` points into a byte staging
    // buffer that need not meet the tensor maps' 64-byte alignment
    FusedBatchEntry e;
    std::memset(&e, 0, sizeof(e));
    e.maps = p->maps;
    e.args = p->base;
    e.start = start;
    std::memcpy(entry, &e, sizeof(e));
}
template <int N, int SM>
static void launch_batched_n(const void* entries, const int* block_entry, int grid, int threads, size_t smem,
                             cudaStream_t s) {
    set_smem_attr((const void*)fused_tma_kernel_batched<N, SM>, (int)smem);
    fused_tma_kernel_batched<N, SM><<<grid, threads, smem, s>>>(static_cast<const FusedBatchEntry*>(entries), block_entry);
}
// order = N + 8 split0 (fused_batch_order): every entry of one launch shares it
void launch_fused_batched(int order, const void* entries, const int* block_entry, int grid, int threads, size_t smem,
                          cudaStream_t s) {
    switch (order) {
        case 2: launch_batched_n<2, 0>(entries, block_entry, grid, threads, smem, s); break;
        case 3: launch_batched_n<3, 1>(entries, block_entry, grid, threads, smem, s); break;
        case 4: launch_batched_n<4, 2>(entries, block_entry, grid, threads, smem, s); break;
        case 8 + 3: launch_batched_n<3, 0>(entries, block_entry, grid, threads, smem, s); break;
        case 8 + 4: launch_batched_n<4, 0>(entries, block_entry, grid, threads, smem, s); break;
        default: break;
    }
}

void launch_fused_tma(FusedTmaPlan* p, int output, float* L, cudaStream_t s) {
    switch (p->base.g.N) {
        case 2: launch_tma_n<2, 0>(p, output, L, s); break;
        case 3: if (p->base.g.split0) launch_tma_n<3, 0>(p, output, L, s); else launch_tma_n<3, 1>(p, output, L, s); break;
        case 4: if (p->base.g.split0) launch_tma_n<4, 0>(p, output, L, s); else launch_tma_n<4, 2>(p, output, L, s); break;
        default: break;
    }
}

}  // namespace pasd
