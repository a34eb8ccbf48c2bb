// Fused elementwise pass of one PASD loop body (Algorithm 1, after the V-step).
// For every element x of the tensor, with z_n = Z_n(x) = fold_n(U_n V_n)(x):
//   H_n     = T - Z_n + Y_n/mu                       (Eq. 14)
//   E'      = prox_{1/(mu N)}(mean_n H_n)             (Eq. 15)
//   Y_n'    = Y_n + mu (T - Z_n - E')                 (multiplier update)
//   r_n     = T - Z_n - E'                            (stop test of Algorithm 1)
// The multipliers are stored as G_n = T - E + Y_n/mu, the argument of the next
// U- and V-steps, so H_n = G_n + E - Z_n and
//   G_n'    = T - E' + (mu/mu') (H_n - E'),  mu' = min(rho mu, mu_max).
// The next U-step's product G_n' Vrot_n^T is formed by the M-pass that follows.
//
// Z_n is rebuilt on the fly as Urot_n Vrot_n (Urot = U W, Vrot = diag(F) W^T A_n
// in the eigenbasis W of the SVT), a rank-R refold of the small factor; nothing
// of size D besides T, E, G_n is touched.
//
// Work decomposition: the tensor is cut into boxes ("tiles") of power-of-two
// extents b_n (B = prod b_n elements), tiles are grouped into regions, one CTA
// per region. Per tile, the CTA stages the Vrot_n columns and Urot_n rows the
// tile needs in shared memory; each thread owns a micro-box of 8 elements
// (2 along mode N-2, 4 along the contiguous mode N-1) and computes its Z_n in
// FP32 registers, reusing every loaded operand 2-8 times. Residual statistics
// are written once per region and reduced in a fixed order by the finalize
// kernel, so the pass is deterministic (no atomics).
#include "pasd_impl.cuh"
#include <algorithm>
#include <cmath>
#include <cstdint>

namespace pasd {

static inline int ilog2(int v) { int r = 0; while ((1 << r) < v) ++r; return r; }
static inline int pow2ceil(int64_t v) { int p = 1; while (p < v) p <<= 1; return p; }

static inline int round32(int x) { return (x + 31) / 32 * 32; }

// Chooses the tile box, the region grid and the shared-memory layout. `tma`
// selects the layout of fused_tma.cu (two stages of [Xs | As_n | Ws_n], dense
// boxes) instead of the single-buffer layout of this file.
bool plan_geom_impl(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                    size_t smem_limit, bool tma) {
    g = FusedGeom{};
    g.N = N;
    for (int n = 0; n < N; ++n) { g.I[n] = I[n]; g.Rp[n] = Rp[n]; }
    // element strides (C order)
    int64_t s = 1;
    for (int n = N - 1; n >= 0; --n) { g.stride[n] = s; s *= I[n]; }
    for (int n = 0; n < N; ++n) {
        int64_t a = 1;
        for (int m = n - 1; m >= 0; --m) { g.astr[n][m] = a; a *= I[m]; }
    }
    for (int target_bits = 11; target_bits >= 8; --target_bits) {
        int b[PASD_MAXN];
        // contiguous mode: >= 8 floats (a full 32-byte sector), least padding
        {
            int best = 8; double bw = 1e30;
            for (int c = 8; c <= 64; c <<= 1) {
                double w = (double)(((I[N - 1] + c - 1) / c) * c - I[N - 1]) / (double)I[N - 1];
                if (w < bw - 1e-12 || (std::fabs(w - bw) < 1e-12 && c > best)) { bw = w; best = c; }
                if (c >= I[N - 1]) break;
            }
            b[N - 1] = best;
        }
        for (int n = 0; n < N - 1; ++n) b[n] = 1;
        b[N - 2] = 2;
        int bits = ilog2(b[N - 1]) + 1;
        while (bits < target_bits) {
            int pick = -1; double pw = 1e30, pr = -1;
            for (int n = 0; n < N - 1; ++n) {
                if (b[n] >= pow2ceil(I[n])) continue;
                int c = 2 * b[n];
                double w = (double)(((I[n] + c - 1) / c) * c - I[n]) / (double)I[n];
                double room = (double)I[n] / b[n];
                if (w < pw - 1e-12 || (std::fabs(w - pw) < 1e-12 && room > pr)) { pw = w; pr = room; pick = n; }
            }
            if (pick < 0) break;
            b[pick] *= 2;
            ++bits;
        }
        int B = 1;
        for (int n = 0; n < N; ++n) { g.b[n] = b[n]; g.sh[n] = ilog2(b[n]); B *= b[n]; }
        if (B > 8 * FU_THREADS) continue;
        g.B = B;
        g.esh[N - 1] = 0;
        for (int n = N - 2; n >= 0; --n) g.esh[n] = g.esh[n + 1] + g.sh[n + 1];
        for (int n = 0; n < N; ++n)
            for (int m = 0; m < N; ++m) {
                if (m == n) { g.csh[n][m] = 0; continue; }
                g.csh[n][m] = (m > n) ? g.esh[m] : g.esh[m] - g.sh[n];
            }
        for (int n = 0; n < N; ++n) g.C[n] = B / b[n];
        for (int n = 0; n < N; ++n) g.mb[n] = (n == N - 1) ? 4 : (n == N - 2 ? 2 : 1);
        // thread-id bit offsets of the micro-box coordinates (last mode fastest)
        int off = 0;
        for (int n = N - 1; n >= 0; --n) { g.mbsh[n] = off; off += ilog2(b[n] / g.mb[n]); }
        // tiles and regions: one CTA per region, one resident CTA per SM, so the
        // kernel takes ceil(regions / SMs) waves, each as long as its largest
        // region. Pick the region grid Q minimising waves x max tiles per region.
        for (int n = 0; n < N; ++n) { g.nt[n] = (I[n] + b[n] - 1) / b[n]; g.Q[n] = 1; }
        {
            const int64_t cap = 4LL * num_sms;
            int64_t best_cost = INT64_MAX, best_reg = INT64_MAX;
            int q[PASD_MAXN], bq[PASD_MAXN];
            for (int n = 0; n < N; ++n) { q[n] = 1; bq[n] = 1; }
            // odometer over Q_n in [1, min(nt_n, cap)], pruned by the region cap
            for (;;) {
                int64_t reg = 1, mx = 1;
                for (int n = 0; n < N; ++n) {
                    reg *= q[n];
                    mx *= (g.nt[n] + q[n] - 1) / q[n];
                }
                if (reg <= cap) {
                    int64_t waves = (reg + num_sms - 1) / num_sms;
                    int64_t cost = waves * mx;
                    if (cost < best_cost || (cost == best_cost && reg < best_reg)) {
                        best_cost = cost; best_reg = reg;
                        for (int n = 0; n < N; ++n) bq[n] = q[n];
                    }
                }
                int k = N - 1;
                while (k >= 0) {
                    int64_t rest = 1;
                    for (int n = 0; n < N; ++n) rest *= (n == k) ? 1 : q[n];
                    if (q[k] < g.nt[k] && rest * (q[k] + 1) <= cap) { ++q[k]; break; }
                    q[k] = 1;
                    --k;
                }
                if (k < 0) break;
            }
            for (int n = 0; n < N; ++n) g.Q[n] = bq[n];
        }
        g.nregions = 1;
        for (int n = 0; n < N; ++n) g.nregions *= g.Q[n];
        g.nthreads = B / 8;
        if (tma) {
            bool fits = true;
            for (int n = 0; n < N; ++n) fits = fits && b[n] <= 256;
            if (!fits) continue;
            int o = 0;
            g.xs_off = o; o += round32((N + 2) * B);
            for (int n = 0; n < N; ++n) { g.as_off[n] = o; o += round32(g.C[n] * Rp[n]); }
            for (int n = 0; n < N; ++n) { g.ws_off[n] = o; o += round32(b[n] * Rp[n]); }
            g.stage_floats = round32(o);
            int64_t tx = (int64_t)(N + 2) * B, txo = 0;
            for (int n = 0; n < N; ++n) txo += (int64_t)g.C[n] * Rp[n] + (int64_t)b[n] * Rp[n];
            g.stage_tx_bytes = (uint32_t)(4 * (tx + txo));
            g.out_tx_bytes = (uint32_t)(4 * txo);
            g.smem_floats = 2 * g.stage_floats;
            g.tma = 1;
            // With (b_{N-1} / 4) (b_{N-2} / 2) < 8 the eight lanes of a quarter-warp
            // read element-tile rows 32 floats apart (the same banks): give each
            // thread groups 4 t and 4 t + B / 2 instead (split along mode 0).
            g.split0 = (N >= 3 && b[0] >= 2 && (b[N - 1] / 4) * (b[N - 2] / 2) < 8) ? 1 : 0;
            // +1 KB so the kernel can align its stages to 1024 bytes
            if ((size_t)g.smem_floats * 4 + 1024 <= smem_limit) return true;
            continue;
        }
        int o = 0;
        for (int n = 0; n < N; ++n) { g.as_off[n] = o; o += g.C[n] * (Rp[n] + 4); }
        for (int n = 0; n < N; ++n) { g.ws_off[n] = o; o += b[n] * Rp[n]; }
        g.smem_floats = o;
        if ((size_t)o * 4 <= smem_limit) return true;
    }
    return false;
}

bool plan_fused_geom(FusedGeom& g, int N, const int64_t* I, const int* Rp, int num_sms,
                     size_t smem_limit) {
    return plan_geom_impl(g, N, I, Rp, num_sms, smem_limit, false);
}

__device__ __forceinline__ float dot4(const float4& w, const float4& a, float acc) {
    acc = fmaf(w.x, a.x, acc);
    acc = fmaf(w.y, a.y, acc);
    acc = fmaf(w.z, a.z, acc);
    return fmaf(w.w, a.w, acc);
}

template <int N, bool VEC>
__global__ void __launch_bounds__(FU_THREADS, 1) fused_kernel(FusedArgs fa) {
    DevScalars* sc = fa.sc;
    if (!fa.output && sc->done) return;
    const FusedGeom& g = fa.g;
    extern __shared__ __align__(16) float sm[];
    const int t = threadIdx.x;
    const float* __restrict__ T = sc->T;

    // region of this CTA
    int q[N];
    {
        int r = blockIdx.x;
        for (int n = N - 1; n >= 0; --n) { q[n] = r % g.Q[n]; r /= g.Q[n]; }
    }
    int64_t ts[N], te[N];
#pragma unroll
    for (int n = 0; n < N; ++n) {
        ts[n] = (int64_t)q[n] * g.nt[n] / g.Q[n];
        te[n] = (int64_t)(q[n] + 1) * g.nt[n] / g.Q[n];
    }

    // micro-box of this thread
    int nmb = 1;
#pragma unroll
    for (int n = 0; n < N; ++n) nmb *= g.b[n] / g.mb[n];
    const bool active = t < nmb;
    int u0[N];   // micro-box origin (local element coordinates)
#pragma unroll
    for (int n = 0; n < N; ++n) u0[n] = ((t >> g.mbsh[n]) & (g.b[n] / g.mb[n] - 1)) * g.mb[n];
    int e0 = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) e0 += u0[n] << g.esh[n];
    int64_t toff = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) toff += (int64_t)u0[n] * g.stride[n];
    // per-mode column base of the micro-box origin
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

    float resmax = 0.f, l1 = 0.f, res2[N];
    int nonfin = 0;
#pragma unroll
    for (int n = 0; n < N; ++n) res2[n] = 0.f;

    // tiles of the region, C order
    int64_t ntile = 1;
#pragma unroll
    for (int n = 0; n < N; ++n) ntile *= te[n] - ts[n];
    for (int64_t tile = 0; tile < ntile; ++tile) {
        int64_t o[N];
        int ext[N];
        {
            int64_t r = tile;
#pragma unroll
            for (int n = N - 1; n >= 0; --n) {
                int64_t span = te[n] - ts[n];
                int64_t tc = ts[n] + r % span;
                r /= span;
                o[n] = tc * g.b[n];
                int64_t e = g.I[n] - o[n];
                ext[n] = e < g.b[n] ? (int)e : g.b[n];
            }
        }
        __syncthreads();   // previous tile's shared-memory readers are done
        // ---- stage Wz rows and A columns ----
#pragma unroll
        for (int n = 0; n < N; ++n) {
            // only the first round4(kept) rows of Vrot_n are current (the rest are zero
            // or left from an earlier body): stage and multiply those
            const int Rp = g.Rp[n], R4 = (sc->kept[n] + 3) >> 2;
            float* Ws = sm + g.ws_off[n];
            for (int idx = t; idx < g.b[n] * R4; idx += FU_THREADS) {
                int l = idx / R4, r4 = idx % R4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (l < ext[n]) v = *reinterpret_cast<const float4*>(fa.Wz[n] + (o[n] + l) * Rp + 4 * r4);
                *reinterpret_cast<float4*>(Ws + l * Rp + 4 * r4) = v;
            }
            float* As = sm + g.as_off[n];
            const int ald = Rp + 4;
            const int Cn = g.C[n];
            const float* __restrict__ An = fa.A[n];
            if (n < N - 1) {
                const int64_t post = g.stride[n];
                for (int idx = t; idx < Cn * R4; idx += FU_THREADS) {
                    int c = idx & (Cn - 1), r4 = idx / Cn;
                    bool ok = true;
                    int64_t a = 0, bb = 0;
#pragma unroll
                    for (int m = 0; m < N; ++m) {
                        if (m == n) continue;
                        int l = (c >> g.csh[n][m]) & (g.b[m] - 1);
                        ok = ok && (l < ext[m]);
                        if (m < n) a += (o[m] + l) * g.astr[n][m];
                        else bb += (o[m] + l) * g.stride[m];
                    }
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok) {
                        const float* src = An + (a * Rp + 4 * r4) * post + bb;
                        v.x = src[0];
                        v.y = src[post];
                        v.z = src[2 * post];
                        v.w = src[3 * post];
                    }
                    *reinterpret_cast<float4*>(As + c * ald + 4 * r4) = v;
                }
            } else {
                for (int idx = t; idx < Cn * R4; idx += FU_THREADS) {
                    int r4 = idx % R4, c = idx / R4;
                    bool ok = true;
                    int64_t a = 0;
#pragma unroll
                    for (int m = 0; m < N - 1; ++m) {
                        int l = (c >> g.csh[n][m]) & (g.b[m] - 1);
                        ok = ok && (l < ext[m]);
                        a += (o[m] + l) * g.astr[n][m];
                    }
                    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (ok) v = *reinterpret_cast<const float4*>(An + a * Rp + 4 * r4);
                    *reinterpret_cast<float4*>(As + c * ald + 4 * r4) = v;
                }
            }
        }
        __syncthreads();

        // ---- Z_n for the thread's 8 elements: j = d2 * 4 + d1 ----
        float z[N][8];
#pragma unroll
        for (int n = 0; n < N; ++n)
#pragma unroll
            for (int j = 0; j < 8; ++j) z[n][j] = 0.f;
        if (active) {
#pragma unroll
            for (int n = 0; n < N; ++n) {
                const int Rp = g.Rp[n], R4 = (sc->kept[n] + 3) >> 2, ald = Rp + 4;
                const float* Ws = sm + g.ws_off[n];
                const float* As = sm + g.as_off[n];
                if (n == N - 1) {
                    for (int r4 = 0; r4 < R4; ++r4) {
                        float4 w[4];
#pragma unroll
                        for (int d1 = 0; d1 < 4; ++d1)
                            w[d1] = *reinterpret_cast<const float4*>(Ws + (u0[n] + d1) * Rp + 4 * r4);
#pragma unroll
                        for (int d2 = 0; d2 < 2; ++d2) {
                            float4 a = *reinterpret_cast<const float4*>(As + (cb[n] + d2) * ald + 4 * r4);
#pragma unroll
                            for (int d1 = 0; d1 < 4; ++d1) z[n][d2 * 4 + d1] = dot4(w[d1], a, z[n][d2 * 4 + d1]);
                        }
                    }
                } else if (n == N - 2) {
                    for (int r4 = 0; r4 < R4; ++r4) {
                        float4 w0 = *reinterpret_cast<const float4*>(Ws + u0[n] * Rp + 4 * r4);
                        float4 w1 = *reinterpret_cast<const float4*>(Ws + (u0[n] + 1) * Rp + 4 * r4);
#pragma unroll
                        for (int d1 = 0; d1 < 4; ++d1) {
                            float4 a = *reinterpret_cast<const float4*>(As + (cb[n] + d1) * ald + 4 * r4);
                            z[n][d1] = dot4(w0, a, z[n][d1]);
                            z[n][4 + d1] = dot4(w1, a, z[n][4 + d1]);
                        }
                    }
                } else {
                    const int s2 = g.csh[n][N - 2];
                    for (int r4 = 0; r4 < R4; ++r4) {
                        float4 w = *reinterpret_cast<const float4*>(Ws + u0[n] * Rp + 4 * r4);
#pragma unroll
                        for (int d2 = 0; d2 < 2; ++d2)
#pragma unroll
                            for (int d1 = 0; d1 < 4; ++d1) {
                                int c = cb[n] + (d2 << s2) + d1;
                                float4 a = *reinterpret_cast<const float4*>(As + c * ald + 4 * r4);
                                z[n][d2 * 4 + d1] = dot4(w, a, z[n][d2 * 4 + d1]);
                            }
                    }
                }
            }
        }

        // ---- elementwise update ----
        bool vbase = active;
#pragma unroll
        for (int n = 0; n < N - 2; ++n) vbase = vbase && (u0[n] < ext[n]);
        int64_t tbase = toff;
#pragma unroll
        for (int n = 0; n < N; ++n) tbase += o[n] * g.stride[n];
#pragma unroll
        for (int d2 = 0; d2 < 2; ++d2) {
            const bool v2 = vbase && (u0[N - 2] + d2 < ext[N - 2]);
            const int64_t rowoff = tbase + (int64_t)d2 * g.stride[N - 2];
            const int ebase = e0 + (d2 << g.esh[N - 2]);
            float tv[4], ev[4], gv[N][4];
            bool ok[4];
#pragma unroll
            for (int d1 = 0; d1 < 4; ++d1) ok[d1] = v2 && (u0[N - 1] + d1 < ext[N - 1]);
            if (VEC && ok[0]) {
                float4 x = *reinterpret_cast<const float4*>(T + rowoff);
                tv[0] = x.x; tv[1] = x.y; tv[2] = x.z; tv[3] = x.w;
                if (!fa.output) {
                    x = *reinterpret_cast<const float4*>(fa.E + rowoff);
                    ev[0] = x.x; ev[1] = x.y; ev[2] = x.z; ev[3] = x.w;
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        x = *reinterpret_cast<const float4*>(fa.G[n] + rowoff);
                        gv[n][0] = x.x; gv[n][1] = x.y; gv[n][2] = x.z; gv[n][3] = x.w;
                    }
                }
            } else {
#pragma unroll
                for (int d1 = 0; d1 < 4; ++d1) {
                    tv[d1] = ok[d1] ? T[rowoff + d1] : 0.f;
                    if (!fa.output) {
                        ev[d1] = ok[d1] ? fa.E[rowoff + d1] : 0.f;
#pragma unroll
                        for (int n = 0; n < N; ++n) gv[n][d1] = ok[d1] ? fa.G[n][rowoff + d1] : 0.f;
                    }
                }
            }
            if (fa.output) {
                float lv[4];
#pragma unroll
                for (int d1 = 0; d1 < 4; ++d1) {
                    float s = 0.f;
#pragma unroll
                    for (int n = 0; n < N; ++n) s = fmaf(fa.alpha_w[n], z[n][d2 * 4 + d1], s);
                    lv[d1] = s;
                }
                if (VEC && ok[0]) {
                    *reinterpret_cast<float4*>(fa.L + rowoff) = make_float4(lv[0], lv[1], lv[2], lv[3]);
                } else {
#pragma unroll
                    for (int d1 = 0; d1 < 4; ++d1)
                        if (ok[d1]) fa.L[rowoff + d1] = lv[d1];
                }
                continue;
            }
            float en[4], gn[N][4];
#pragma unroll
            for (int d1 = 0; d1 < 4; ++d1) {
                float hs = 0.f;
#pragma unroll
                for (int n = 0; n < N; ++n) hs += (gv[n][d1] + ev[d1]) - z[n][d2 * 4 + d1];
                float eb = hs * invN;
                float mag = fabsf(eb) - thr;
                float e = mag > 0.f ? copysignf(mag, eb) : 0.f;
                en[d1] = e;
                bool fin = isfinite(e);
#pragma unroll
                for (int n = 0; n < N; ++n) {
                    float zz = z[n][d2 * 4 + d1];
                    float h = (gv[n][d1] + ev[d1]) - zz;
                    float r = (tv[d1] - zz) - e;
                    float gnew = (tv[d1] - e) + cfac * (h - e);
                    gn[n][d1] = gnew;
                    fin = fin && isfinite(gnew);
                    if (ok[d1]) {
                        resmax = fmaxf(resmax, fabsf(r));
                        res2[n] = fmaf(r, r, res2[n]);
                    }
                }
                if (ok[d1]) {
                    l1 += fabsf(e);
                    nonfin |= !fin;
                }
            }
            if (VEC && ok[0]) {
                *reinterpret_cast<float4*>(fa.E + rowoff) = make_float4(en[0], en[1], en[2], en[3]);
#pragma unroll
                for (int n = 0; n < N; ++n)
                    *reinterpret_cast<float4*>(fa.G[n] + rowoff) =
                        make_float4(gn[n][0], gn[n][1], gn[n][2], gn[n][3]);
            } else {
#pragma unroll
                for (int d1 = 0; d1 < 4; ++d1)
                    if (ok[d1]) {
                        fa.E[rowoff + d1] = en[d1];
#pragma unroll
                        for (int n = 0; n < N; ++n) fa.G[n][rowoff + d1] = gn[n][d1];
                    }
            }
        }
    }
    if (fa.output) return;

    // ---- block reductions of the residual statistics ----
    __shared__ float wred[FU_THREADS / 32][PASD_MAXN + 3];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        resmax = fmaxf(resmax, __shfl_down_sync(0xffffffffu, resmax, off));
        l1 += __shfl_down_sync(0xffffffffu, l1, off);
        nonfin |= __shfl_down_sync(0xffffffffu, nonfin, off);
#pragma unroll
        for (int n = 0; n < N; ++n) res2[n] += __shfl_down_sync(0xffffffffu, res2[n], off);
    }
    const int wid = t >> 5, lane = t & 31;
    if (lane == 0) {
        wred[wid][0] = resmax;
        wred[wid][1] = l1;
        wred[wid][2] = (float)nonfin;
#pragma unroll
        for (int n = 0; n < N; ++n) wred[wid][3 + n] = res2[n];
    }
    __syncthreads();
    if (t == 0) {
        float mx = 0.f, s1 = 0.f, nf = 0.f, s2[N];
#pragma unroll
        for (int n = 0; n < N; ++n) s2[n] = 0.f;
        for (int w = 0; w < FU_THREADS / 32; ++w) {
            mx = fmaxf(mx, wred[w][0]);
            s1 += wred[w][1];
            nf = fmaxf(nf, wred[w][2]);
#pragma unroll
            for (int n = 0; n < N; ++n) s2[n] += wred[w][3 + n];
        }
        float* p = fa.part + (size_t)blockIdx.x * fa.part_stride;
        p[0] = mx;
        p[1] = s1;
        p[2] = nf;
#pragma unroll
        for (int n = 0; n < N; ++n) p[3 + n] = s2[n];
    }
}

template <int N>
static void launch_n(const FusedArgs& a, cudaStream_t s) {
    bool vec = (a.g.I[N - 1] % 4) == 0;
    size_t smem = (size_t)a.g.smem_floats * 4;
    if (vec) {
        set_smem_attr((const void*)fused_kernel<N, true>, (int)smem);
        fused_kernel<N, true><<<a.g.nregions, FU_THREADS, smem, s>>>(a);
    } else {
        set_smem_attr((const void*)fused_kernel<N, false>, (int)smem);
        fused_kernel<N, false><<<a.g.nregions, FU_THREADS, smem, s>>>(a);
    }
}

void launch_fused(const FusedArgs& a, cudaStream_t s) {
    switch (a.g.N) {
        case 2: launch_n<2>(a, s); break;
        case 3: launch_n<3>(a, s); break;
        case 4: launch_n<4>(a, s); break;
        case 5: launch_n<5>(a, s); break;
        case 6: launch_n<6>(a, s); break;
        case 7: launch_n<7>(a, s); break;
        case 8: launch_n<8>(a, s); break;
        default: break;
    }
}

}  // namespace pasd
