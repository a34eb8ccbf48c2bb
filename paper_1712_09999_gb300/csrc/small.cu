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
__device__ void block_AtB(const float* X, int ldx, const float* Y, int ldy, int64_t rows, int ca,
                          int cb, float* C, int ldc) {
    for (int idx = threadIdx.x; idx < ca * cb; idx += blockDim.x) {
        int i = idx / cb, j = idx % cb;
        float s = 0.f;
        for (int64_t r = 0; r < rows; ++r) s = fmaf(X[r * ldx + i], Y[r * ldy + j], s);
        C[i * ldc + j] = s;
    }
}

// Y (rows x cols, ldy) = X (rows x inner, ldx) * S (inner x cols, lds).
__device__ void block_AB(const float* X, int ldx, const float* S, int lds, int64_t rows, int inner,
                         int cols, float* Y, int ldy) {
    for (int64_t idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
        int64_t i = idx / cols;
        int j = (int)(idx % cols);
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
    const int t = threadIdx.x;
    extern __shared__ __align__(16) float sm[];
    JacobiBufs jb = carve_jacobi(sm, ld);
    float* Smat = sm + jacobi_floats(ld);       // ld x ld
    float* fsh = Smat + ld * ld;                // ld
    int* perm = reinterpret_cast<int*>(fsh + ld);

    // 1. Gram matrix C = sum over CTA partials (fixed order)
    for (int idx = t; idx < R * R; idx += blockDim.x) {
        int i = idx / R, j = idx % R;
        float s = 0.f;
        for (int p = 0; p < m.n_gram; ++p) s += m.gram_part[(size_t)p * Rp * Rp + i * Rp + j];
        jb.A[i * ld + j] = s;
    }
    __syncthreads();
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
    // W (sorted columns) -> global, padded
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
    // 4. S = W diag(F) W^T
    for (int idx = t; idx < R * R; idx += blockDim.x) {
        int i = idx / R, j = idx % R;
        float s = 0.f;
        for (int k = 0; k < R; ++k) s = fmaf(Ve[i * ld + perm[k]] * fsh[k], Ve[j * ld + perm[k]], s);
        Smat[i * ld + j] = s;
    }
    __syncthreads();
    // 5. Wz = U S (I x Rp, zero padding columns)
    for (int64_t idx = t; idx < m.I * Rp; idx += blockDim.x) {
        int64_t i = idx / Rp;
        int j = (int)(idx % Rp);
        float s = 0.f;
        if (j < R)
            for (int k = 0; k < R; ++k) s = fmaf(m.U[i * Rp + k], Smat[k * ld + j], s);
        m.Wz[idx] = s;
    }
}

// ---------------------------------------------------------------------------
// U-step (Eq. 9, Eq. 10), one CTA per mode. In the eigenbasis W of the last
// SVT, V_n = diag(F) W^T A_n, so M_n = G_n V_n^T = (G_n A_n^T) W diag(F): its
// columns s..R-1 (F = 0, the null space of V_n^T) vanish. The result is
//   U = [ P1 , X ],  P1 = polar(M_n[:, :s]),  X = polar((I - P1 P1^T) (U W)[:, s:]),
// i.e. the unique polar factor on the range of M_n and, on its null space, the
// isometry closest to the previous iterate (identity at k = 0, where s = 0).
// A closing Newton-Schulz step re-orthonormalises U.
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
    float* Wsh = sm + jacobi_floats(ld);   // ld x ld
    float* Z = Wsh + ld * ld;              // ld x ld
    float* K = Z + ld * ld;                // ld x ld
    float* fsh = K + ld * ld;              // ld

    const int s = *m.kept;
    const int q = R - s;
    float* Mp = m.scratch;                 // I x Rp : reduced G A^T
    float* Mr = Mp + I * Rp;               // I x Rp : M in the W basis, then B
    float* Ur = Mr + I * Rp;               // I x Rp : U W (null columns)
    float* Un = Ur + I * Rp;               // I x Rp : new U before re-orthonormalisation

    for (int idx = t; idx < Rp * Rp; idx += blockDim.x) Wsh[idx] = m.W[idx];
    if (t < Rp) fsh[t] = m.F[t];
    __syncthreads();

    if (s > 0) {
        // M' = sum of partials (fixed order), columns r < R
        for (int64_t idx = t; idx < I * R; idx += blockDim.x) {
            int64_t i = idx / R;
            int r = (int)(idx % R);
            float acc = 0.f;
            for (int p = 0; p < m.n_mp; ++p) acc += m.mp_part[(size_t)p * I * Rp + i * Rp + r];
            Mp[i * Rp + r] = acc;
        }
        __syncthreads();
        // M = M' W[:, :s] diag(F[:s])
        for (int64_t idx = t; idx < I * s; idx += blockDim.x) {
            int64_t i = idx / s;
            int c = (int)(idx % s);
            float acc = 0.f;
            for (int r = 0; r < R; ++r) acc = fmaf(Mp[i * Rp + r], Wsh[r * ld + c], acc);
            Mr[i * Rp + c] = acc * fsh[c];
        }
        __syncthreads();
        // B1 = M^T M (s x s), eigen -> Z1 = B1^{-1/2}; P1 = M Z1
        block_AtB(Mr, Rp, Mr, Rp, I, s, s, jb.A, ld);
        __syncthreads();
        float *Ae, *Ve;
        block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.pc, jb.cs, s, ld, 1e-6f, 30, &Ae, &Ve);
        inv_sqrt_from_eig(Ae, Ve, s, ld, Z);
        block_AB(Mr, Rp, Z, ld, I, s, s, Un, Rp);
        __syncthreads();
    }
    if (q > 0) {
        // Ur = U W[:, s:]
        for (int64_t idx = t; idx < I * q; idx += blockDim.x) {
            int64_t i = idx / q;
            int c = (int)(idx % q);
            float acc = 0.f;
            for (int r = 0; r < R; ++r) acc = fmaf(m.U[i * Rp + r], Wsh[r * ld + s + c], acc);
            Ur[i * Rp + c] = acc;
        }
        __syncthreads();
        float* Bm = Mr;   // reuse
        if (s > 0) {
            // K = P1^T Ur (s x q);  B = Ur - P1 K
            block_AtB(Un, Rp, Ur, Rp, I, s, q, K, ld);
            __syncthreads();
            for (int64_t idx = t; idx < I * q; idx += blockDim.x) {
                int64_t i = idx / q;
                int c = (int)(idx % q);
                float acc = Ur[i * Rp + c];
                for (int k = 0; k < s; ++k) acc = fmaf(-Un[i * Rp + k], K[k * ld + c], acc);
                Bm[i * Rp + c] = acc;
            }
        } else {
            for (int64_t idx = t; idx < I * q; idx += blockDim.x) {
                int64_t i = idx / q;
                int c = (int)(idx % q);
                Bm[i * Rp + c] = Ur[i * Rp + c];
            }
        }
        __syncthreads();
        block_AtB(Bm, Rp, Bm, Rp, I, q, q, jb.A, ld);
        __syncthreads();
        float *Ae, *Ve;
        block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.pc, jb.cs, q, ld, 1e-6f, 30, &Ae, &Ve);
        inv_sqrt_from_eig(Ae, Ve, q, ld, Z);
        block_AB(Bm, Rp, Z, ld, I, q, q, Un + s, Rp);
        __syncthreads();
    }
    // Newton-Schulz: U = Un (3 I - Un^T Un) / 2
    block_AtB(Un, Rp, Un, Rp, I, R, R, K, ld);
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
            for (int k = 0; k < R; ++k) acc = fmaf(Un[i * Rp + k], Z[k * ld + j], acc);
        m.U[idx] = acc;
    }
}

static size_t small_smem_bytes(int maxRp) {
    int ld = maxRp;
    return 4 * (size_t)(jacobi_floats(ld) + 3 * ld * ld + 2 * ld + 64);
}

void launch_svt(const SmallArgs& a, cudaStream_t s) {
    int maxRp = 4;
    for (int n = 0; n < a.N; ++n) maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
    size_t smem = small_smem_bytes(maxRp);
    cudaFuncSetAttribute(svt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    svt_kernel<<<a.N, SM_THREADS, smem, s>>>(a);
}

void launch_polar(const SmallArgs& a, cudaStream_t s) {
    int maxRp = 4;
    for (int n = 0; n < a.N; ++n) maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
    size_t smem = small_smem_bytes(maxRp);
    cudaFuncSetAttribute(polar_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    polar_kernel<<<a.N, SM_THREADS, smem, s>>>(a);
}

// ---------------------------------------------------------------------------
// Finalize one loop body: residual norms of T - Z_n - E (the stop test of
// Algorithm 1), objective of Eq. 3, mu schedule, iteration record.
// part layout per CTA: [0] max |T - Z_n - E|, [1] sum |E|, [2] non-finite flag,
// [3 + n] sum (T - Z_n - E)^2.
// ---------------------------------------------------------------------------
__global__ void finalize_kernel(FinalizeArgs fa) {
    DevScalars* sc = fa.sc;
    if (sc->done) return;
    __shared__ double sh[32][PASD_MAXN + 3];
    const int t = threadIdx.x, nt = blockDim.x;
    double mx = 0.0, l1 = 0.0, nf = 0.0;
    double r2[PASD_MAXN];
    for (int n = 0; n < PASD_MAXN; ++n) r2[n] = 0.0;
    // deterministic: thread t owns parts t, t + nt, ...; then a fixed tree
    for (int p = t; p < fa.nparts; p += nt) {
        const float* q = fa.part + (size_t)p * fa.stride;
        mx = fmax(mx, (double)q[0]);
        l1 += (double)q[1];
        nf = fmax(nf, (double)q[2]);
        for (int n = 0; n < fa.N; ++n) r2[n] += (double)q[3 + n];
    }
    // warp reduce
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
        l1 += __shfl_down_sync(0xffffffffu, l1, off);
        nf = fmax(nf, __shfl_down_sync(0xffffffffu, nf, off));
        for (int n = 0; n < fa.N; ++n) r2[n] += __shfl_down_sync(0xffffffffu, r2[n], off);
    }
    int w = t >> 5, lane = t & 31;
    if (lane == 0) {
        sh[w][0] = mx; sh[w][1] = l1; sh[w][2] = nf;
        for (int n = 0; n < fa.N; ++n) sh[w][3 + n] = r2[n];
    }
    __syncthreads();
    if (t == 0) {
        int nw = (nt + 31) / 32;
        for (int i = 1; i < nw; ++i) {
            mx = fmax(mx, sh[i][0]);
            l1 += sh[i][1];
            nf = fmax(nf, sh[i][2]);
            for (int n = 0; n < fa.N; ++n) r2[n] += sh[i][3 + n];
        }
        double r2max = 0.0;
        for (int n = 0; n < fa.N; ++n) r2max = fmax(r2max, r2[n]);
        double tn = sc->t_norm_fro;
        double fro_rel = tn > 0 ? sqrt(r2max) / tn : 0.0;
        double obj = l1;
        for (int n = 0; n < fa.N; ++n) obj += fa.lambda[n] * sc->nuclear[n];
        double mu = sc->mu;
        sc->res_inf = mx;
        sc->res_fro_rel = fro_rel;
        sc->objective = obj;
        sc->l1_E = l1;
        sc->mu_used = mu;
        double mun = fa.rho * mu;
        sc->mu = mun < fa.mu_max ? mun : fa.mu_max;
        int k = sc->k + 1;
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
    finalize_kernel<<<1, 256, 0, s>>>(a);
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
        a.U[n][idx] = (i == r && r < a.R[n]) ? 1.f : 0.f;   // eye(I_n, R_n), zero padding
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
                       int32_t* kept, cudaStream_t s) {
    InitArgs a;
    a.sc = sc; a.T = T; a.mu0 = mu0; a.N = N; a.kept = kept;
    for (int n = 0; n < N; ++n) {
        a.U[n] = U[n]; a.I[n] = I[n]; a.R[n] = R[n]; a.Rp[n] = Rp[n]; a.W[n] = W[n]; a.F[n] = F[n];
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
