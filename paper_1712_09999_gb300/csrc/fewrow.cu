// The two streaming products of a loop body for modes with few rows (I_n <= 8):
//   apass_small_kernel - the mode-n product A_n = U_n^T G_n of the V-step (Eq. 13)
//                        and per-CTA Gram partials of A_n A_n^T;
//   mpass_small_kernel - the next U-step's product G_n Vrot_n^T (Eq. 9) in the
//                        SVT eigenbasis, per-CTA partials over the columns.
//
// With I_n <= 8 a column of the unfolding [pre][I][post] holds at most 8 floats
// and U_n (I x Rp, Rp <= 8) fits in a few shared-memory lines, so one thread
// forms whole columns of A_n in registers: it loads the I entries of four
// consecutive columns (one 16-byte load per row along the contiguous index b
// when post % 4 == 0, four scalar loads otherwise), multiplies them by U
// (broadcast from shared memory), stores the four columns of A_n
// ([pre][Rp][post]) and adds their outer products to its Gram accumulators (the
// Rp (Rp + 1) / 2 entries on and above the diagonal). A fixed grid of CTAs walks
// the columns in a fixed order and each CTA writes one Gram partial, so the SVT
// sums a bounded number of partials in a fixed order.
//
// The TMA-fed kernels stage 16 rows per copy and tile 8 rows per thread; for a
// mode of three rows (the colour channel of a video) that is 13 rows of zero
// fill per stage, one CTA and one Gram partial per 256 columns in the A-pass,
// and 8 of 256 threads busy in the M-pass, which these kernels avoid.
#include "pasd_impl.cuh"

namespace pasd {

constexpr int AS_THREADS = 256;
constexpr int AS_IMAX = 8;

template <int RP, bool VEC>
__global__ void __launch_bounds__(AS_THREADS) apass_small_kernel(const ApassArgs a) {
    const DevScalars* sc = a.sc;
    if (sc->done) return;
    constexpr int NG = RP * (RP + 1) / 2;
    __shared__ __align__(16) float Us[AS_IMAX * RP];
    __shared__ float red[AS_THREADS / 32][NG];
    const int t = threadIdx.x;
    const int I = (int)a.I;
    for (int idx = t; idx < AS_IMAX * RP; idx += AS_THREADS) {
        const int i = idx / RP, r = idx % RP;
        Us[idx] = i < I ? a.U[i * RP + r] : 0.f;   // U is I x Rp (columns past R are zero)
    }
    __syncthreads();

    float gacc[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q) gacc[q] = 0.f;

    const int64_t post = a.post;
    // column groups of four (VEC: b, b + 1, b + 2, b + 3 inside one a-row)
    const int64_t per_row = VEC ? post / 4 : 0;
    const int64_t ngroups = VEC ? a.pre * per_row : (a.P + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * AS_THREADS;
    // (a-row, group within the row) of group g, advanced by `stride` groups at a
    // time without a division after the first
    const int64_t g0 = (int64_t)blockIdx.x * AS_THREADS + t;
    int64_t ar = VEC ? g0 / per_row : 0, gr = VEC ? g0 - ar * per_row : 0;
    const int64_t da = VEC ? stride / per_row : 0, dg = VEC ? stride - da * per_row : 0;
    for (int64_t g = g0; g < ngroups; g += stride) {
        float x[AS_IMAX][4];
        int64_t base[4];
        bool in[4];
        if (VEC) {
            const int64_t b = 4 * gr;
            const float* src = a.G + (ar * I) * post + b;
#pragma unroll
            for (int i = 0; i < AS_IMAX; ++i) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < I) v = *reinterpret_cast<const float4*>(src + (int64_t)i * post);
                x[i][0] = v.x; x[i][1] = v.y; x[i][2] = v.z; x[i][3] = v.w;
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) { base[c] = ar * RP * post + b + c; in[c] = true; }
            gr += dg;
            ar += da;
            if (gr >= per_row) { gr -= per_row; ++ar; }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t j = 4 * g + c;
                in[c] = j < a.P;
                const int64_t ac = in[c] ? j / post : 0, b = in[c] ? j - ac * post : 0;
                base[c] = ac * RP * post + b;
                const float* src = a.G + (ac * I) * post + b;
#pragma unroll
                for (int i = 0; i < AS_IMAX; ++i) x[i][c] = (in[c] && i < I) ? src[(int64_t)i * post] : 0.f;
            }
        }
        float av[RP][4];
#pragma unroll
        for (int r = 0; r < RP; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) av[r][c] = 0.f;
#pragma unroll
        for (int i = 0; i < AS_IMAX; ++i) {
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const float u = Us[i * RP + r];
#pragma unroll
                for (int c = 0; c < 4; ++c) av[r][c] = fmaf(u, x[i][c], av[r][c]);
            }
        }
        if (VEC) {
#pragma unroll
            for (int r = 0; r < RP; ++r)
                *reinterpret_cast<float4*>(a.A + base[0] + (int64_t)r * post) =
                    make_float4(av[r][0], av[r][1], av[r][2], av[r][3]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (in[c])
#pragma unroll
                    for (int r = 0; r < RP; ++r) a.A[base[c] + (int64_t)r * post] = av[r][c];
        }
        int q = 0;
#pragma unroll
        for (int r = 0; r < RP; ++r)
#pragma unroll
            for (int r2 = r; r2 < RP; ++r2, ++q)
#pragma unroll
                for (int c = 0; c < 4; ++c) gacc[q] = fmaf(av[r][c], av[r2][c], gacc[q]);
    }

    // CTA Gram partial: warp butterfly sums, then the warps' sums in order
#pragma unroll
    for (int q = 0; q < NG; ++q) {
        float v = gacc[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        gacc[q] = v;
    }
    const int w = t >> 5;
    if ((t & 31) == 0)
#pragma unroll
        for (int q = 0; q < NG; ++q) red[w][q] = gacc[q];
    __syncthreads();
    float* gp = a.gram_part + (size_t)blockIdx.x * RP * RP;
    if (t < NG) {
        int r = 0, rem = t;
        while (rem >= RP - r) { rem -= RP - r; ++r; }
        const int r2 = r + rem;
        float s = 0.f;
        for (int k = 0; k < AS_THREADS / 32; ++k) s += red[k][t];
        gp[r * RP + r2] = s;
        gp[r2 * RP + r] = s;
    }
}

// part[cta][I][Rp] = sum over this CTA's columns j of G_(n)[:, j] Vrot_n[:, j]^T,
// rows of Vrot past round4(s_n) being zero (not read). Same column walk as above.
template <int RP, bool VEC>
__global__ void __launch_bounds__(AS_THREADS) mpass_small_kernel(const MpassSmallArgs m) {
    const DevScalars* sc = m.sc;
    if (sc->done) return;
    const int s4 = (sc->kept[m.mode] + 3) & ~3;
    if (s4 == 0) return;                       // nothing kept: the U-step does not read M_n
    constexpr int NA = AS_IMAX * RP;
    __shared__ float red[AS_THREADS / 32][NA];
    const int t = threadIdx.x;
    const int I = (int)m.I;
    float acc[AS_IMAX][RP];
#pragma unroll
    for (int i = 0; i < AS_IMAX; ++i)
#pragma unroll
        for (int r = 0; r < RP; ++r) acc[i][r] = 0.f;
    const int64_t post = m.post;
    const int64_t per_row = VEC ? post / 4 : 0;
    const int64_t ngroups = VEC ? m.pre * per_row : (m.P + 3) / 4;
    const int64_t stride = (int64_t)gridDim.x * AS_THREADS;
    const int64_t g0 = (int64_t)blockIdx.x * AS_THREADS + t;
    int64_t ar = VEC ? g0 / per_row : 0, gr = VEC ? g0 - ar * per_row : 0;
    const int64_t da = VEC ? stride / per_row : 0, dg = VEC ? stride - da * per_row : 0;
    for (int64_t g = g0; g < ngroups; g += stride) {
        float x[AS_IMAX][4], v[RP][4];
        if (VEC) {
            const int64_t b = 4 * gr;
            const float* gs = m.G + (ar * I) * post + b;
            const float* vs = m.V + (ar * RP) * post + b;
#pragma unroll
            for (int i = 0; i < AS_IMAX; ++i) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i < I) q = *reinterpret_cast<const float4*>(gs + (int64_t)i * post);
                x[i][0] = q.x; x[i][1] = q.y; x[i][2] = q.z; x[i][3] = q.w;
            }
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (r < s4) q = *reinterpret_cast<const float4*>(vs + (int64_t)r * post);
                v[r][0] = q.x; v[r][1] = q.y; v[r][2] = q.z; v[r][3] = q.w;
            }
            gr += dg;
            ar += da;
            if (gr >= per_row) { gr -= per_row; ++ar; }
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int64_t j = 4 * g + c;
                const bool in = j < m.P;
                const int64_t ac = in ? j / post : 0, b = in ? j - ac * post : 0;
                const float* gs = m.G + (ac * I) * post + b;
                const float* vs = m.V + (ac * RP) * post + b;
#pragma unroll
                for (int i = 0; i < AS_IMAX; ++i) x[i][c] = (in && i < I) ? gs[(int64_t)i * post] : 0.f;
#pragma unroll
                for (int r = 0; r < RP; ++r) v[r][c] = (in && r < s4) ? vs[(int64_t)r * post] : 0.f;
            }
        }
#pragma unroll
        for (int i = 0; i < AS_IMAX; ++i)
#pragma unroll
            for (int r = 0; r < RP; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[i][r] = fmaf(x[i][c], v[r][c], acc[i][r]);
    }
#pragma unroll
    for (int i = 0; i < AS_IMAX; ++i)
#pragma unroll
        for (int r = 0; r < RP; ++r) {
            float q = acc[i][r];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) q += __shfl_xor_sync(0xffffffffu, q, off);
            acc[i][r] = q;
        }
    const int w = t >> 5;
    if ((t & 31) == 0)
#pragma unroll
        for (int i = 0; i < AS_IMAX; ++i)
#pragma unroll
            for (int r = 0; r < RP; ++r) red[w][i * RP + r] = acc[i][r];
    __syncthreads();
    float* dst = m.part + (size_t)blockIdx.x * I * RP;
    if (t < I * RP) {
        float q = 0.f;
        for (int k = 0; k < AS_THREADS / 32; ++k) q += red[k][t];
        dst[t] = q;
    }
}

bool apass_small_supported(int64_t I, int Rp) { return I <= AS_IMAX && Rp <= 8; }

// (up to 212 registers a thread at Rp = 8: one or two CTAs per SM, one wave)
int apass_small_grid(int num_sms, int64_t P) {
    const int64_t want = (P / 4 + AS_THREADS - 1) / AS_THREADS;
    const int64_t cap = 2LL * num_sms;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

void launch_apass_small(const ApassArgs& a, int grid, cudaStream_t s) {
    const bool vec = a.post % 4 == 0;
    if (a.Rp == 4) {
        if (vec) apass_small_kernel<4, true><<<grid, AS_THREADS, 0, s>>>(a);
        else apass_small_kernel<4, false><<<grid, AS_THREADS, 0, s>>>(a);
    } else {
        if (vec) apass_small_kernel<8, true><<<grid, AS_THREADS, 0, s>>>(a);
        else apass_small_kernel<8, false><<<grid, AS_THREADS, 0, s>>>(a);
    }
}

void launch_mpass_small(const MpassSmallArgs& m, int grid, cudaStream_t s) {
    const bool vec = m.post % 4 == 0;
    if (m.Rp == 4) {
        if (vec) mpass_small_kernel<4, true><<<grid, AS_THREADS, 0, s>>>(m);
        else mpass_small_kernel<4, false><<<grid, AS_THREADS, 0, s>>>(m);
    } else {
        if (vec) mpass_small_kernel<8, true><<<grid, AS_THREADS, 0, s>>>(m);
        else mpass_small_kernel<8, false><<<grid, AS_THREADS, 0, s>>>(m);
    }
}

}  // namespace pasd
