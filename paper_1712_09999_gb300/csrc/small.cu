// Per-mode R x R linear algebra of Algorithm 1, one CTA per mode:
//   svt_kernel   - V-step (Eq. 13): SVT of the R x P matrix A_n through its
//                  Gram matrix A_n A_n^T = W diag(sigma^2) W^T, so that
//                  SVT_tau(A_n) = W diag(max(1 - tau/sigma, 0)) W^T A_n;
//   polar_kernel - U-step (Eq. 9, Eq. 10): polar factor of M_n = G_n V_n^T with
//                  the null-space rule for a rank-deficient M_n;
//   finalize     - multipliers' side effects: residual norms, stop test, mu.
//
// Basis. PASD is invariant under U_n -> U_n Q, V_n -> Q^T V_n for orthogonal Q
// (the objective of Eq. 3 and every step depend on U_n V_n only). After each
// SVT the solver moves to the eigenbasis W of A_n A_n^T: the next U-step is
// solved for U_n W, so the next A_n has nearly orthogonal rows and its Gram
// matrix is nearly diagonal. That keeps the FP32 eigensolves relatively
// accurate for every singular value, including those near the threshold tau,
// and lets the cyclic Jacobi sweeps converge in one or two passes.
//
// Precision. GB300 issues FP64 at about 1/74 of the FP32 rate (1.0 vs 74
// TFLOP/s measured), so these kernels work in FP32; only scalar bookkeeping
// (objective, residual sums, mu) uses FP64.
#include "pasd_impl.cuh"
#include <cfloat>

namespace pasd {

constexpr int SM_THREADS = 512;

// ---------------------------------------------------------------------------
// Block-wide cyclic Jacobi eigen-solver for a symmetric n x n matrix.
//   A  (ld x ld, n x n used) is overwritten; eigenvalues end on the diagonal.
//   V  receives the eigenvectors (columns). A2, V2 are work buffers of the same
//   shape; pc (2 * ld ints) and cs (2 * ld floats) hold the per-round rotations.
// Pairs follow the round-robin (circle) ordering so that every round applies
// n/2 disjoint rotations at once. A rotation is skipped when
// |a_pq| <= tol * sqrt(|a_pp a_qq|), the relative criterion that preserves the
// relative accuracy of small eigenvalues of graded matrices. Sweeps stop when
// a sweep applies no rotation. Returns the pointer (A or A2, V or V2) holding
// the result through *Aout / *Vout.
// ---------------------------------------------------------------------------
__device__ void block_jacobi(float* A, float* V, float* A2, float* V2, int* pc, float* cs,
                             int n, int ld, float tol, int max_sweeps, float** Aout,
                             float** Vout) {
    const int t = threadIdx.x, nt = blockDim.x;
    int m = n + (n & 1);      // even size; index n (if odd) is a zero dummy
    for (int idx = t; idx < ld * ld; idx += nt) {
        int i = idx / ld, j = idx % ld;
        V[idx] = (i == j) ? 1.f : 0.f;
        if (i >= n || j >= n) A[idx] = 0.f;
    }
    __syncthreads();
    if (m < 2) { *Aout = A; *Vout = V; return; }
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated_any = 0;
        for (int round = 0; round < m - 1; ++round) {
            // rotation parameters, one thread per pair
            int rot = 0;
            if (t < m / 2) {
                int k = t;
                int p, q;
                if (k == 0) { p = 0; q = 1 + round; }
                else {
                    p = 1 + (round + k) % (m - 1);
                    q = 1 + (round - k + (m - 1)) % (m - 1);
                }
                float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
                float c = 1.f, s = 0.f;
                if (apq != 0.f && fabsf(apq) > tol * sqrtf(fabsf(app * aqq))) {
                    float theta = (aqq - app) / (2.f * apq);
                    float tt;
                    if (fabsf(theta) > 1e18f) tt = 0.5f / theta;
                    else tt = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(1.f + theta * theta));
                    c = rsqrtf(1.f + tt * tt);
                    s = tt * c;
                    rot = 1;
                }
                pc[p] = q; pc[q] = p;
                cs[2 * p] = c; cs[2 * p + 1] = -s;   // J[p][p] = c, J[q][p] = -s
                cs[2 * q] = c; cs[2 * q + 1] = s;    // J[q][q] = c, J[p][q] =  s
            }
            int any = __syncthreads_or(rot);
            if (!any) continue;
            rotated_any = 1;
            // A2 = J^T A J, V2 = V J
            for (int idx = t; idx < m * m; idx += nt) {
                int i = idx / m, j = idx % m;
                int pi = pc[i], pj = pc[j];
                float ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
                float v = ci * cj * A[i * ld + j] + ci * sj * A[i * ld + pj] +
                          si * cj * A[pi * ld + j] + si * sj * A[pi * ld + pj];
                if ((pi == j) && (si != 0.f)) v = 0.f;   // annihilated pair
                A2[i * ld + j] = v;
            }
            for (int idx = t; idx < n * m; idx += nt) {
                int i = idx / m, j = idx % m;
                int pj = pc[j];
                V2[i * ld + j] = V[i * ld + j] * cs[2 * j] + V[i * ld + pj] * cs[2 * j + 1];
            }
            __syncthreads();
            float* tA = A; A = A2; A2 = tA;
            float* tV = V; V = V2; V2 = tV;
        }
        if (!rotated_any) break;
    }
    *Aout = A;
    *Vout = V;
}

// Descending order of the diagonal of A (n x n, ld): perm[rank] = index.
__device__ void sort_desc(const float* A, int n, int ld, int* perm) {
    const int t = threadIdx.x;
    if (t < n) {
        // NaN sorts last, so the ranks always form a permutation
        float v = A[t * ld + t];
        if (v != v) v = -INFINITY;
        int r = 0;
        for (int j = 0; j < n; ++j) {
            float w = A[j * ld + j];
            if (w != w) w = -INFINITY;
            r += (w > v) || (w == v && j < t);
        }
        perm[r] = t;
    }
    __syncthreads();
}

// C (ca x cb, ldc) = X^T Y over `rows` rows; X (rows x ldx), Y (rows x ldy).
// One warp per output, lanes stride over the rows, shuffle reduction (fixed
// order, so the result is deterministic). With `sym` (X == Y, ca == cb) only
// the upper triangle is computed and mirrored.
__device__ void warp_AtB(const float* X, int ldx, const float* Y, int ldy, int64_t rows, int ca, int cb,
                         float* C, int ldc, bool sym) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = warp; o < ca * cb; o += nw) {
        const int a = o / cb, b = o % cb;
        if (sym && a > b) continue;
        float s = 0.f;
        for (int64_t r = lane; r < rows; r += 32) s = fmaf(X[r * ldx + a], Y[r * ldy + b], s);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) {
            C[a * ldc + b] = s;
            if (sym) C[b * ldc + a] = s;
        }
    }
}

// Y[:, y0 + c] (rows x cols) = X (rows x inner) * S (inner x cols); one thread per output.
__device__ void block_AB(const float* X, int ldx, const float* S, int lds, int64_t rows, int inner, int cols,
                         float* Y, int ldy) {
    for (int64_t idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
        const int64_t i = idx / cols;
        const int j = (int)(idx % cols);
        float s = 0.f;
        for (int k = 0; k < inner; ++k) s = fmaf(X[i * ldx + k], S[k * lds + j], s);
        Y[i * ldy + j] = s;
    }
}

// Z = Q diag(w^{-1/2}) Q^T for the n x n eigen-system (Q columns, eigenvalues w
// on the diagonal of D). Nonpositive eigenvalues (rank loss) map to 0.
__device__ void inv_sqrt_from_eig(const float* D, const float* Q, int n, int ld, float* Z) {
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        int i = idx / n, j = idx % n;
        float s = 0.f;
        for (int k = 0; k < n; ++k) {
            float w = D[k * ld + k];
            float f = w > 0.f ? rsqrtf(w) : 0.f;
            s = fmaf(Q[i * ld + k] * f, Q[j * ld + k], s);
        }
        Z[i * ld + j] = s;
    }
    __syncthreads();
}

struct JacobiBufs {
    float *A, *V, *A2, *V2, *cs;
    int* pc;
};

__device__ JacobiBufs carve_jacobi(float* base, int ld) {
    JacobiBufs b;
    b.A = base;
    b.V = b.A + ld * ld;
    b.A2 = b.V + ld * ld;
    b.V2 = b.A2 + ld * ld;
    b.cs = b.V2 + ld * ld;
    b.pc = reinterpret_cast<int*>(b.cs + 2 * ld);
    return b;
}
__host__ __device__ constexpr int jacobi_floats(int ld) { return 4 * ld * ld + 4 * ld; }

// ---------------------------------------------------------------------------
// SVT (Eq. 13 and the SVT definition after it), one CTA per mode.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SM_THREADS) svt_kernel(SmallArgs sa) {
    DevScalars* sc = sa.sc;
    if (sc->done) return;
    const SmallModeArgs& m = sa.m[blockIdx.x];
    const int R = m.R, Rp = m.Rp, ld = Rp;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    extern __shared__ __align__(16) float sm[];
    JacobiBufs jb = carve_jacobi(sm, ld);
    float* Smat = sm + jacobi_floats(ld);       // ld x ld (sorted eigenvectors)
    float* fsh = Smat + ld * ld;                // ld
    int* perm = reinterpret_cast<int*>(fsh + ld);
    float* red = reinterpret_cast<float*>(perm + ld);   // nw x 256

    // 1. Gram matrix = sum over the A-pass CTA partials: warp w owns partials
    //    w, w + nw, ...; lanes own outputs; then a fixed-order sum over warps.
    const int nout = Rp * Rp;
    for (int obase = 0; obase < nout; obase += 256) {
        float acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.f;
        for (int p = warp; p < m.n_gram; p += nw) {
            const float* src = m.gram_part + (size_t)p * nout + obase;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int o = lane + 32 * k;
                if (obase + o < nout) acc[k] += src[o];
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) red[warp * 256 + lane + 32 * k] = acc[k];
        __syncthreads();
        for (int o = t; o < 256 && obase + o < nout; o += blockDim.x) {
            float s = 0.f;
            for (int w = 0; w < nw; ++w) s += red[w * 256 + o];
            int oo = obase + o, i = oo / Rp, j = oo % Rp;
            if (i < R && j < R) jb.A[i * ld + j] = s;
        }
        __syncthreads();
    }
    // 2. eigen-decomposition
    float *Ae, *Ve;
    block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.pc, jb.cs, R, ld, 1e-6f, 30, &Ae, &Ve);
    sort_desc(Ae, R, ld, perm);
    // 3. thresholds
    const double mu = sc->mu;
    const float tau = (float)(m.lambda / mu);
    if (t < Rp) {
        float sig = 0.f, f = 0.f;
        if (t < R) {
            int src = perm[t];
            float lam = Ae[src * ld + src];
            sig = sqrtf(fmaxf(lam, 0.f));
            f = sig > tau ? 1.f - tau / sig : 0.f;
        }
        fsh[t] = f;
        m.sigma[t] = sig;
        m.F[t] = f;
    }
    for (int idx = t; idx < Rp * Rp; idx += blockDim.x) {
        int i = idx / Rp, j = idx % Rp;
        float v = 0.f;
        if (i < R && j < R) v = Ve[i * ld + perm[j]];
        else if (i == j) v = 1.f;
        m.W[idx] = v;
    }
    __syncthreads();
    if (t == 0) {
        int kept = 0;
        double nuc = 0.0;
        for (int i = 0; i < R; ++i) {
            float sig = m.sigma[i];
            if (sig > tau) { ++kept; nuc += (double)sig - (double)tau; }
        }
        *m.kept = kept;
        sc->kept[blockIdx.x] = kept;
        sc->nuclear[blockIdx.x] = nuc;
    }
    // 4. Urot = U W (I x Rp): the active subspace in the eigenbasis of the SVT.
    //    With Vrot = diag(F) W^T A_n (rows beyond the kept count are zero),
    //    fold_n(U_n V_n) = Urot[:, :s] Vrot[:s], the refold of rank s.
    for (int idx = t; idx < R * R; idx += blockDim.x) {
        int i = idx / R, j = idx % R;
        Smat[i * ld + j] = Ve[i * ld + perm[j]];
    }
    __syncthreads();
    for (int64_t idx = t; idx < m.I * Rp; idx += blockDim.x) {
        int64_t i = idx / Rp;
        int j = (int)(idx % Rp);
        float s = 0.f;
        if (j < R)
            for (int k = 0; k < R; ++k) s = fmaf(m.U[i * Rp + k], Smat[k * ld + j], s);
        m.Urot[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// U-step (Eq. 9, Eq. 10), one CTA per mode. In the eigenbasis W of the last
// SVT, V_n = diag(F) W^T A_n, so M_n = G_n V_n^T = (G_n A_n^T) W diag(F): its
// columns s..R-1 (F = 0, the null space of V_n^T) vanish. The result is
//   U = [ P1 , X ],  P1 = polar(M_n[:, :s]),  X = polar((I - P1 P1^T) (U W)[:, s:]),
// i.e. the unique polar factor on the range of M_n and, on its null space, the
// isometry closest to the previous iterate (identity at k = 0, where s = 0).
// A closing Newton-Schulz step re-orthonormalises U. The I x R matrices live in
// shared memory (row stride Rp + 1) when they fit, else in the global scratch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SM_THREADS) polar_kernel(SmallArgs sa) {
    DevScalars* sc = sa.sc;
    if (sc->done) return;
    const SmallModeArgs& m = sa.m[blockIdx.x];
    const int R = m.R, Rp = m.Rp, ld = Rp;
    const int64_t I = m.I;
    const int t = threadIdx.x;
    extern __shared__ __align__(16) float sm[];
    JacobiBufs jb = carve_jacobi(sm, ld);
    float* Z = sm + jacobi_floats(ld) + ld * ld;   // ld x ld
    float* K = Z + ld * ld;                        // ld x ld
    float* big = K + ld * ld + 2 * ld + 64;        // 3 x I x LD when it fits
    const bool in_smem = m.polar_in_smem != 0;
    const int LD = in_smem ? Rp + 1 : Rp;
    float* Mw = in_smem ? big : m.scratch;                 // [P1 | X]
    float* Pw = Mw + I * LD;                               // M in the W basis
    float* Bw = Pw + I * LD;                               // (U W)[:, s:], then B

    const int s = *m.kept;
    const int q = R - s;

    if (s > 0) {
        // M in the W basis: G_n Vrot^T, summed over regions by the finalize kernel
        for (int64_t idx = t; idx < I * s; idx += blockDim.x) {
            int64_t i = idx / s;
            int c = (int)(idx % s);
            Pw[i * LD + c] = m.Mred[i * Rp + c];
        }
        __syncthreads();
        // B1 = M^T M, Z1 = B1^{-1/2}, P1 = M Z1
        warp_AtB(Pw, LD, Pw, LD, I, s, s, jb.A, ld, true);
        __syncthreads();
        float *Ae, *Ve;
        block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.pc, jb.cs, s, ld, 1e-6f, 30, &Ae, &Ve);
        inv_sqrt_from_eig(Ae, Ve, s, ld, Z);
        block_AB(Pw, LD, Z, ld, I, s, s, Mw, LD);
        __syncthreads();
    }
    if (q > 0) {
        // (U W)[:, s:], from the SVT of the previous loop body (eye at k = 0)
        for (int64_t idx = t; idx < I * q; idx += blockDim.x) {
            int64_t i = idx / q;
            int c = (int)(idx % q);
            Bw[i * LD + c] = m.Urot[i * Rp + s + c];
        }
        __syncthreads();
        if (s > 0) {
            // K = P1^T Ur (s x q);  B = Ur - P1 K
            warp_AtB(Mw, LD, Bw, LD, I, s, q, K, ld, false);
            __syncthreads();
            for (int64_t idx = t; idx < I * q; idx += blockDim.x) {
                int64_t i = idx / q;
                int c = (int)(idx % q);
                float acc = Bw[i * LD + c];
                for (int k = 0; k < s; ++k) acc = fmaf(-Mw[i * LD + k], K[k * ld + c], acc);
                Bw[i * LD + c] = acc;
            }
            __syncthreads();
        }
        warp_AtB(Bw, LD, Bw, LD, I, q, q, jb.A, ld, true);
        __syncthreads();
        float *Ae, *Ve;
        block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.pc, jb.cs, q, ld, 1e-6f, 30, &Ae, &Ve);
        inv_sqrt_from_eig(Ae, Ve, q, ld, Z);
        block_AB(Bw, LD, Z, ld, I, q, q, Mw + s, LD);
        __syncthreads();
    }
    // Newton-Schulz: U = Un (3 I - Un^T Un) / 2
    warp_AtB(Mw, LD, Mw, LD, I, R, R, K, ld, true);
    __syncthreads();
    for (int idx = t; idx < R * R; idx += blockDim.x) {
        int i = idx / R, j = idx % R;
        Z[i * ld + j] = ((i == j) ? 1.5f : 0.f) - 0.5f * K[i * ld + j];
    }
    __syncthreads();
    for (int64_t idx = t; idx < I * Rp; idx += blockDim.x) {
        int64_t i = idx / Rp;
        int j = (int)(idx % Rp);
        float acc = 0.f;
        if (j < R)
            for (int k = 0; k < R; ++k) acc = fmaf(Mw[i * LD + k], Z[k * ld + j], acc);
        m.U[idx] = acc;
    }
}

static size_t small_base_floats(int maxRp) {
    int ld = maxRp;
    return (size_t)jacobi_floats(ld) + 3 * ld * ld + 2 * ld + 64;
}
static size_t svt_smem_bytes(int maxRp) {
    return 4 * (small_base_floats(maxRp) + (size_t)(SM_THREADS / 32) * 256);
}
// Bytes of shared memory the U-step needs with its I x R matrices resident.
size_t polar_smem_bytes(int maxRp, int64_t maxI) {
    return 4 * (small_base_floats(maxRp) + 3 * (size_t)maxI * (maxRp + 1));
}

void launch_svt(const SmallArgs& a, cudaStream_t s) {
    int maxRp = 4;
    for (int n = 0; n < a.N; ++n) maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
    size_t smem = svt_smem_bytes(maxRp);
    cudaFuncSetAttribute(svt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    svt_kernel<<<a.N, SM_THREADS, smem, s>>>(a);
}

void launch_polar(const SmallArgs& a, cudaStream_t s) {
    int maxRp = 4;
    int64_t maxI = 1;
    bool any_smem = false;
    for (int n = 0; n < a.N; ++n) {
        maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
        if (a.m[n].polar_in_smem) { any_smem = true; maxI = a.m[n].I > maxI ? a.m[n].I : maxI; }
    }
    size_t smem = any_smem ? polar_smem_bytes(maxRp, maxI) : 4 * small_base_floats(maxRp);
    cudaFuncSetAttribute(polar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    polar_kernel<<<a.N, SM_THREADS, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// Finalize one loop body. CTA 0: residual norms of T - Z_n - E (the stop test
// of Algorithm 1), objective of Eq. 3, mu schedule, iteration record. Other
// CTAs: the fixed-order sum of the per-region G_n A_n^T partials (one output
// per thread), which the next U-step reads.
// part layout per region: [0] max |T - Z_n - E|, [1] sum |E|, [2] non-finite
// flag, [3 + n] sum (T - Z_n - E)^2.
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(FinalizeArgs fa) {
    DevScalars* sc = fa.sc;
    if (sc->done) return;
    const int t = threadIdx.x, nt = blockDim.x;
    if (blockIdx.x > 0) {
        int64_t o = (int64_t)(blockIdx.x - 1) * nt + t;
        for (int n = 0; n < fa.N; ++n) {
            const int64_t cnt = fa.I[n] * fa.R[n];
            if (o < cnt) {
                const int64_t i = o / fa.R[n];
                const int r = (int)(o % fa.R[n]);
                float acc = 0.f;
                if (r < sc->kept[n]) {      // only the kept directions carry G V^T
                    const int64_t stride = fa.I[n] * fa.Rp[n];
                    const float* src = fa.mp_part[n] + i * fa.Rp[n] + r;
#pragma unroll 8
                    for (int p = 0; p < fa.n_mp[n]; ++p) acc += src[(int64_t)p * stride];
                }
                fa.Mred[n][i * fa.Rp[n] + r] = acc;
                return;
            }
            o -= cnt;
        }
        return;
    }
    __shared__ double sh[32][PASD_MAXN + 3];
    double mx = 0.0, l1 = 0.0, nf = 0.0;
    double r2[PASD_MAXN];
#pragma unroll
    for (int n = 0; n < PASD_MAXN; ++n) r2[n] = 0.0;
    for (int p = t; p < fa.nparts; p += nt) {
        const float* q = fa.part + (size_t)p * fa.stride;
        mx = fmax(mx, (double)q[0]);
        l1 += (double)q[1];
        nf = fmax(nf, (double)q[2]);
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) r2[n] += (double)q[3 + n];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
        l1 += __shfl_down_sync(0xffffffffu, l1, off);
        nf = fmax(nf, __shfl_down_sync(0xffffffffu, nf, off));
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n) r2[n] += __shfl_down_sync(0xffffffffu, r2[n], off);
    }
    const int w = t >> 5, lane = t & 31;
    if (lane == 0) {
        sh[w][0] = mx; sh[w][1] = l1; sh[w][2] = nf;
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n) sh[w][3 + n] = r2[n];
    }
    __syncthreads();
    if (t == 0) {
        const int nw = (nt + 31) / 32;
        for (int i = 1; i < nw; ++i) {
            mx = fmax(mx, sh[i][0]);
            l1 += sh[i][1];
            nf = fmax(nf, sh[i][2]);
#pragma unroll
            for (int n = 0; n < PASD_MAXN; ++n) r2[n] += sh[i][3 + n];
        }
        double r2max = 0.0;
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) r2max = fmax(r2max, r2[n]);
        const double tn = sc->t_norm_fro;
        const double fro_rel = tn > 0 ? sqrt(r2max) / tn : 0.0;
        double obj = l1;
        for (int n = 0; n < fa.N; ++n) obj += fa.lambda[n] * sc->nuclear[n];
        const double mu = sc->mu;
        sc->res_inf = mx;
        sc->res_fro_rel = fro_rel;
        sc->objective = obj;
        sc->l1_E = l1;
        sc->mu_used = mu;
        const double mun = fa.rho * mu;
        sc->mu = mun < fa.mu_max ? mun : fa.mu_max;
        const int k = sc->k + 1;
        sc->k = k;
        if (fa.trace && k <= fa.max_iter) {
            double* rec = fa.trace + (size_t)(k - 1) * 13;
            rec[0] = k; rec[1] = mx; rec[2] = fro_rel; rec[3] = obj; rec[4] = mu;
            for (int n = 0; n < 8; ++n) rec[5 + n] = n < fa.N ? sc->kept[n] : 0;
        }
        if (nf > 0.0 || !isfinite(mx)) {
            sc->nonfinite = 1;
            sc->status = -4;   // PASD_ERR_NONFINITE
            sc->done = 1;
        } else if ((fa.stop_rule == 0 && mx < fa.tol) || (fa.stop_rule == 1 && fro_rel < fa.tol)) {
            sc->status = 0;    // PASD_OK
            sc->done = 1;
        } else if (k >= fa.max_iter) {
            sc->status = fa.stop_rule == 2 ? 0 : 2;   // OK (fixed) / NOT_CONVERGED
            sc->done = 1;
        }
    }
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    int64_t tot = 0;
    for (int n = 0; n < a.N; ++n) tot += a.I[n] * a.R[n];
    int grid = 1 + (int)((tot + 255) / 256);
    finalize_kernel<<<grid, 256, 0, s>>>(a);
}

// ---------------------------------------------------------------------------
// Vrot_n = diag(F) W^T A_n: the small factor V_n of Eq. 13 in the eigenbasis of
// the SVT, stored like A_n ([pre][Rp][post]); rows at and beyond the kept
// count are zero. One thread per unfolding column, all modes in one launch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) vrot_kernel(VrotArgs va) {
    const DevScalars* sc = va.sc;
    if (sc->done) return;
    int k = 0;
    while (k + 1 < va.N && (int)blockIdx.x >= va.cta_start[k + 1]) ++k;
    const VrotMode& m = va.m[k];
    const int R = m.R, Rp = m.Rp;
    const int s = sc->kept[k];
    __shared__ float Wt[PASD_MAXR * PASD_MAXR];   // Wt[i][r] = F_i W[r][i]
    for (int idx = threadIdx.x; idx < s * R; idx += blockDim.x) {
        int i = idx / R, r = idx % R;
        Wt[i * R + r] = m.F[i] * m.W[r * Rp + i];
    }
    __syncthreads();
    const int64_t j = (int64_t)(blockIdx.x - va.cta_start[k]) * blockDim.x + threadIdx.x;
    if (j >= m.P) return;
    const int64_t a = j / m.post, b = j % m.post;
    const float* src = m.A + a * Rp * m.post + b;
    float* dst = m.V + a * Rp * m.post + b;
    float av[PASD_MAXR];
#pragma unroll 4
    for (int r = 0; r < R; ++r) av[r] = src[(int64_t)r * m.post];
    for (int i = 0; i < Rp; ++i) {
        float acc = 0.f;
        if (i < s)
            for (int r = 0; r < R; ++r) acc = fmaf(Wt[i * R + r], av[r], acc);
        dst[(int64_t)i * m.post] = acc;
    }
}

void launch_vrot(const VrotArgs& a, cudaStream_t s) {
    vrot_kernel<<<a.cta_start[a.N], 256, 0, s>>>(a);
}

// ---------------------------------------------------------------------------
// Initialisation of Algorithm 1 (U = eye(I, R), V = 0 i.e. F = 0 and W = I).
// ---------------------------------------------------------------------------
struct InitArgs {
    DevScalars* sc;
    const float* T;
    int R[PASD_MAXN];
    double mu0;
    int N;
    float* U[PASD_MAXN];
    int64_t I[PASD_MAXN];
    int Rp[PASD_MAXN];
    float* W[PASD_MAXN];
    float* F[PASD_MAXN];
    float* Urot[PASD_MAXN];
    int32_t* kept;
};

__global__ void init_kernel(InitArgs a) {
    int n = blockIdx.y;
    if (n >= a.N) return;
    int Rp = a.Rp[n];
    int64_t tot = a.I[n] * Rp;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = idx / Rp;
        int r = (int)(idx % Rp);
        const float v = (i == r && r < a.R[n]) ? 1.f : 0.f;   // eye(I_n, R_n), zero padding
        a.U[n][idx] = v;
        a.Urot[n][idx] = v;                                     // U W with W = I
    }
    if (blockIdx.x == 0) {
        for (int idx = threadIdx.x; idx < Rp * Rp; idx += blockDim.x)
            a.W[n][idx] = (idx / Rp == idx % Rp) ? 1.f : 0.f;
        for (int idx = threadIdx.x; idx < Rp; idx += blockDim.x) a.F[n][idx] = 0.f;
        if (threadIdx.x == 0) a.kept[n] = 0;
    }
    if (blockIdx.x == 0 && n == 0 && threadIdx.x == 0) {
        DevScalars* sc = a.sc;
        sc->T = a.T;
        sc->mu = a.mu0;
        sc->k = 0;
        sc->done = 0;
        sc->status = 2;
        sc->nonfinite = 0;
        for (int m = 0; m < PASD_MAXN; ++m) { sc->kept[m] = 0; sc->nuclear[m] = 0.0; }
        sc->res_inf = sc->res_fro_rel = sc->objective = sc->l1_E = 0.0;
        sc->mu_used = a.mu0;
    }
}

void launch_init_state(DevScalars* sc, const float* T, double mu0, int N, float** U,
                       const int64_t* I, const int* R, const int* Rp, float** W, float** F,
                       float** Urot, int32_t* kept, cudaStream_t s) {
    InitArgs a;
    a.sc = sc; a.T = T; a.mu0 = mu0; a.N = N; a.kept = kept;
    for (int n = 0; n < N; ++n) {
        a.U[n] = U[n]; a.I[n] = I[n]; a.R[n] = R[n]; a.Rp[n] = Rp[n]; a.W[n] = W[n]; a.F[n] = F[n];
        a.Urot[n] = Urot[n];
    }
    init_kernel<<<dim3(32, N), 256, 0, s>>>(a);
}

// ||T||_F: per-block FP32 partial sums of squares, then one block in FP64.
__global__ void sumsq_kernel(const float* __restrict__ T, int64_t D, float* part) {
    float s = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D;
         i += (int64_t)gridDim.x * blockDim.x) {
        float v = T[i];
        s = fmaf(v, v, s);
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    __shared__ float w[32];
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) tot += w[i];
        part[blockIdx.x] = tot;
    }
}
__global__ void sumsq_final(const float* part, int n, DevScalars* sc) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        sc->t_norm_fro = sqrt(s);
    }
}

void launch_norm_fro(const float* T, int64_t D, float* part, int nparts, DevScalars* sc,
                     cudaStream_t s) {
    sumsq_kernel<<<nparts, 256, 0, s>>>(T, D, part);
    sumsq_final<<<1, 32, 0, s>>>(part, nparts, sc);
}

// Y_n = mu (G_n - T + E)
__global__ void export_y_kernel(const float* G, const float* T, const float* E,
                                const DevScalars* sc, float* Y, int64_t D) {
    float mu = (float)sc->mu;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < D;
         i += (int64_t)gridDim.x * blockDim.x)
        Y[i] = mu * ((G[i] - T[i]) + E[i]);
}
void launch_export_y(const float* G, const float* T, const float* E, const DevScalars* sc,
                     float* Y, int64_t D, cudaStream_t s) {
    export_y_kernel<<<1024, 256, 0, s>>>(G, T, E, sc, Y, D);
}

}  // namespace pasd
