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
//
// Latency. Each CTA works alone on an SM, so its time is the length of its
// dependency chain, not its arithmetic: matrices stay in shared memory, the
// products run as 4 x 4 register tiles over split row ranges (summed in a fixed
// order, so results do not depend on timing), global reads keep many loads in
// flight, and a Jacobi round costs one barrier.
#include "pasd_impl.cuh"
#include <cfloat>

namespace pasd {

constexpr int SM_THREADS = 512;
constexpr int TILE_SCRATCH = 4096;   // floats of split partial sums for tile_AtB

// ---------------------------------------------------------------------------
// Block-wide cyclic Jacobi eigen-solver for a symmetric n x n matrix.
//   A  (ld x ld, n x n used) is overwritten; eigenvalues end on the diagonal.
//   V  receives the eigenvectors (columns). A2, V2 are work buffers of the same
//   shape. Returns the buffers holding the result.
// Pairs follow the round-robin (circle) ordering, so every round applies m/2
// disjoint rotations at once (m = n rounded up to even; an odd n gets a zero
// dummy index). A rotation is skipped when |a_pq| <= tol * sqrt(|a_pp a_qq|),
// the relative criterion that keeps the relative accuracy of the small
// eigenvalues of graded matrices. A sweep starts only if some off-diagonal
// entry fails that test.
//
// A round computes the rotation of every index once (thread i < m, for the pair
// holding i; both members of a pair evaluate it identically from the smaller
// index p and the larger index q), then every thread updates its elements of
// A and V from the two rotations it needs; two barriers per round. The element
// update is evaluated in an order that is symmetric in (i, j) with explicit
// rounding, so A stays exactly symmetric.
// ---------------------------------------------------------------------------
struct JacobiBufs {
    float *A, *V, *A2, *V2, *cs;   // cs: 2 ld floats, the round's rotations
};
// Buffers holding the eigenvalues (diagonal) and eigenvectors (columns) on return.
struct EigBufs {
    float* A;
    float* V;
};

__device__ __forceinline__ int rr_partner(int i, int round, int m) {
    // index 0 stays fixed and meets 1 + round; index 1 + x (x != round) meets
    // 1 + y with x + y = 2 round (mod m - 1)
    if (i == 0) return 1 + round;
    const int x = i - 1, mm = m - 1;
    if (x == round) return 0;
    int y = 2 * round - x;
    if (y >= mm) y -= mm;
    if (y < 0) y += mm;
    return 1 + y;
}

// J restricted to the pair {i, pi}: J[i][i] = ci, J[pi][i] = si. The tangent is
// formed with the hardware's approximate reciprocal and reciprocal square root
// (a Jacobi round is a chain of dependent steps; the correctly rounded forms
// made it about a quarter slower); c and s come from the same t, so the
// rotation is orthogonal to rounding whatever t's last bits are.
// With `exact` the tangent and the cosine use correctly rounded division and
// square root instead: about a quarter of the error of each rotation, which a
// rank above 24 needs (there the many rotations of each entry add their
// rounding to the eigenvector directions; see sym_eig_orth).
__device__ __forceinline__ int pair_rotation(const float* A, int ld, int i, int pi, float tol, float& ci,
                                             float& si, bool exact = false) {
    const int p = min(i, pi), q = max(i, pi);
    const float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
    float c = 1.f, s = 0.f;
    int rot = 0;
    if (apq != 0.f && fabsf(apq) > tol * sqrtf(fabsf(app * aqq))) {
        float tt;
        if (exact) {
            const float theta = (aqq - app) / (2.f * apq);
            if (fabsf(theta) > 1e18f) tt = 0.5f / theta;
            else tt = copysignf(1.f / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f))), theta);
            c = 1.f / sqrtf(fmaf(tt, tt, 1.f));
        } else {
            const float theta = __fdividef(aqq - app, 2.f * apq);
            if (fabsf(theta) > 1e18f) {
                tt = __fdividef(0.5f, theta);
            } else {
                const float r = fmaf(theta, theta, 1.f);
                tt = copysignf(__fdividef(1.f, fabsf(theta) + r * rsqrtf(r)), theta);
            }
            c = rsqrtf(fmaf(tt, tt, 1.f));
        }
        s = tt * c;
        rot = 1;
    }
    ci = c;
    si = (i == p) ? -s : s;      // J[q][p] = -s, J[p][q] = s
    return rot;
}

// cs: 2 m floats of shared scratch for the round's rotations.
__device__ __forceinline__ EigBufs block_jacobi_body(float* A, float* V, float* A2, float* V2, float* cs, int n, int ld,
                                float tol, int max_sweeps) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int m = n + (n & 1);
    for (int idx = t; idx < ld * ld; idx += nt) {
        const int i = idx / ld, j = idx % ld;
        V[idx] = (i == j) ? 1.f : 0.f;
        if (i >= n || j >= n) A[idx] = 0.f;
    }
    __syncthreads();
    // this thread's first entry (i, j) of the m x m update, fixed for the solve
    const int fi = t / (m > 0 ? m : 1), fj = t - fi * (m > 0 ? m : 1);
    if (m >= 2) {
        for (int sweep = 0; sweep < max_sweeps; ++sweep) {
            int need = 0;
            for (int idx = t; idx < n * n; idx += nt) {
                const int i = idx / n, j = idx % n;
                if (i < j) {
                    const float apq = A[i * ld + j];
                    need |= (apq != 0.f && fabsf(apq) > tol * sqrtf(fabsf(A[i * ld + i] * A[j * ld + j])));
                }
            }
            if (!__syncthreads_or(need)) break;
            for (int round = 0; round < m - 1; ++round) {
                int rot = 0;
                if (t < m) {
                    const int pi = rr_partner(t, round, m);
                    float ci, si;
                    rot = pair_rotation(A, ld, t, pi, tol, ci, si, n > 24);
                    cs[2 * t] = ci;
                    cs[2 * t + 1] = si;
                }
                if (!__syncthreads_or(rot)) continue;
                // the partners come from the round-robin formula, not from a table, so
                // the loads below do not wait on another shared-memory load
                for (int idx = t; idx < m * m; idx += nt) {
                    const int i = idx < nt ? fi : idx / m, j = idx < nt ? fj : idx % m;
                    const int pi = rr_partner(i, round, m), pj = rr_partner(j, round, m);
                    const float ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
                    const float t1 = __fmul_rn(__fmul_rn(ci, cj), A[i * ld + j]);
                    const float t2 = __fmul_rn(__fmul_rn(ci, sj), A[i * ld + pj]);
                    const float t3 = __fmul_rn(__fmul_rn(si, cj), A[pi * ld + j]);
                    const float t4 = __fmul_rn(__fmul_rn(si, sj), A[pi * ld + pj]);
                    float v = __fadd_rn(__fadd_rn(t1, __fadd_rn(t2, t3)), t4);
                    if (pi == j && si != 0.f) v = 0.f;      // the annihilated pair
                    A2[i * ld + j] = v;
                    if (i < n) V2[i * ld + j] = fmaf(V[i * ld + pj], sj, V[i * ld + j] * cj);
                }
                __syncthreads();
                float* tA = A; A = A2; A2 = tA;
                float* tV = V; V = V2; V2 = tV;
            }
        }
    }
    return EigBufs{A, V};
}

// Out-of-line copy for the U-step, which runs two eigen-solves; the SVT inlines
// the body (one call site, and the call costs it more than the code size).
__device__ __noinline__ EigBufs block_jacobi(float* A, float* V, float* A2, float* V2, float* cs, int n,
                                            int ld, float tol, int max_sweeps) {
    return block_jacobi_body(A, V, A2, V2, cs, n, ld, tol, max_sweeps);
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

// The helpers below are out of line (__noinline__): the U-step calls them several
// times each, and inlined copies made that kernel wait on instruction fetch.
//
// C (na x nb, ldc) = X[:, :na]^T Y[:, :nb] over `rows` rows (row strides ldx,
// ldy, multiples of 4; 16-byte aligned bases). The entries of C up to the next
// multiples of 4 are written as zeros. 4 x 4 register tiles, rows split S ways,
// split sums added in a fixed order. With `sym` (X == Y, na == nb) only tiles
// on and above the diagonal are formed and mirrored. Ends with a barrier.
__device__ __noinline__ void tile_AtB(const float* X, int ldx, int na, const float* Y, int ldy, int nb, int64_t rows,
                         float* C, int ldc, bool sym, float* scratch) {
    const int t = threadIdx.x, nt = blockDim.x;
    const int ta = (na + 3) / 4, tb = (nb + 3) / 4;
    const int ntile = sym ? ta * (ta + 1) / 2 : ta * tb;
    int S = 1, lgS = 0;
    while (ntile * S * 2 <= TILE_SCRATCH / 16 && ntile * S * 2 <= nt && S * 2 <= rows) { S *= 2; ++lgS; }
    for (int w = t; w < ntile * S; w += nt) {
        const int tile = w >> lgS, sp = w & (S - 1);
        int a4, b4;
        if (sym) {
            a4 = 0;
            int rem = tile;
            while (rem >= ta - a4) { rem -= ta - a4; ++a4; }
            b4 = a4 + rem;
        } else {
            a4 = tile / tb;
            b4 = tile % tb;
        }
        const int r0 = (int)((rows * sp) >> lgS), r1 = (int)((rows * (sp + 1)) >> lgS);   // S is a power of two
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
        const float* xp = X + (int64_t)r0 * ldx + 4 * a4;
        const float* yp = Y + (int64_t)r0 * ldy + 4 * b4;
#pragma unroll 2
        for (int r = r0; r < r1; ++r, xp += ldx, yp += ldy) {
            const float4 x = *reinterpret_cast<const float4*>(xp);
            const float4 y = *reinterpret_cast<const float4*>(yp);
            const float xs[4] = {x.x, x.y, x.z, x.w}, ys[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xs[i], ys[j], acc[i][j]);
        }
        float4* dst = reinterpret_cast<float4*>(scratch + (size_t)w * 16);
#pragma unroll
        for (int i = 0; i < 4; ++i) dst[i] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    }
    __syncthreads();
    const int na4 = 4 * ta, nb4 = 4 * tb;
    for (int o = t; o < na4 * nb4; o += nt) {
        const int a = o / nb4, b = o % nb4;
        if (a >= na || b >= nb) {
            if (!sym || a <= b) C[a * ldc + b] = 0.f;
            if (sym && a <= b) C[b * ldc + a] = 0.f;
            continue;
        }
        if (sym && a > b) continue;
        const int a4 = a >> 2, b4 = b >> 2;
        const int tile = sym ? a4 * ta - a4 * (a4 - 1) / 2 + (b4 - a4) : a4 * tb + b4;
        const float* src = scratch + (size_t)tile * S * 16 + (a & 3) * 4 + (b & 3);
        // the split sums in order, loaded eight at a time ahead of their adds
        float s = 0.f;
        int sp = 0;
        for (; sp + 8 <= S; sp += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = src[(sp + u) * 16];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; sp < S; ++sp) s += src[sp * 16];
        C[a * ldc + b] = s;
        if (sym) C[b * ldc + a] = s;
    }
    __syncthreads();
}

// Y[:, :cols] = X[:, :inner] S  (or Y -= X S with `sub`), rows x cols, cols a
// multiple of 4; S is inner x cols (row stride lds, a multiple of 4). One
// thread per row and group of 4 columns. No barrier.
__device__ __noinline__ void tile_AB(const float* X, int ldx, int inner, const float* S, int lds, int cols, int64_t rows,
                        float* Y, int ldy, bool sub) {
    const int c4n = cols / 4;
    const int tot = (int)rows * c4n;
    for (int w = threadIdx.x; w < tot; w += blockDim.x) {
        const int i = w / c4n;
        const int c4 = w - i * c4n;
        float4* yp = reinterpret_cast<float4*>(Y + (int64_t)i * ldy + 4 * c4);
        float4 acc = sub ? *yp : make_float4(0.f, 0.f, 0.f, 0.f);
        const float sg = sub ? -1.f : 1.f;
        const float* xr = X + (int64_t)i * ldx;
        const float* sc = S + 4 * c4;
        int k = 0;
#pragma unroll 2
        for (; k + 4 <= inner; k += 4) {
            const float4 x4 = *reinterpret_cast<const float4*>(xr + k);
            const float xs[4] = {sg * x4.x, sg * x4.y, sg * x4.z, sg * x4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 sv = *reinterpret_cast<const float4*>(sc + (k + u) * lds);
                acc.x = fmaf(xs[u], sv.x, acc.x);
                acc.y = fmaf(xs[u], sv.y, acc.y);
                acc.z = fmaf(xs[u], sv.z, acc.z);
                acc.w = fmaf(xs[u], sv.w, acc.w);
            }
        }
        for (; k < inner; ++k) {
            const float xv = sg * xr[k];
            const float4 sv = *reinterpret_cast<const float4*>(sc + k * lds);
            acc.x = fmaf(xv, sv.x, acc.x);
            acc.y = fmaf(xv, sv.y, acc.y);
            acc.z = fmaf(xv, sv.z, acc.z);
            acc.w = fmaf(xv, sv.w, acc.w);
        }
        *yp = acc;
    }
}

// Symmetric eigen-solve whose eigenvector matrix, above kOrthMinN, is
// re-orthonormalised by one Newton-Schulz step V (3 I - V^T V) / 2. Each Jacobi
// rotation is orthogonal only to the rounding of its approximate reciprocal
// square root, and a high-rank Gram matrix formed in FP32 needs many sweeps of
// rotations, so V^T V drifts from I (by about 1e-6 at rank 60, enough to move L
// by 5e-5 over a few hundred loop bodies: the refold and the U-step are
// sensitive to that drift rather than to the last bits of the directions). At
// low rank the drift is far below that and the step is skipped. With no
// rotation at all V = I and the step returns I exactly. `scratch` holds
// TILE_SCRATCH floats.
constexpr int kOrthMinN = 24;
template <bool INLINE_SOLVE = false>
__device__ EigBufs sym_eig_orth(JacobiBufs& jb, int n, int ld, float tol, int max_sweeps, float* scratch);

// Z = Q diag(w^{-1/2}) Q^T for the n x n eigen-system (Q columns, eigenvalues w
// on the diagonal of D); entries up to the next multiple of 4 are zero.
// Nonpositive eigenvalues (rank loss) map to 0. Ends with a barrier.
__device__ __noinline__ void inv_sqrt_from_eig(const float* D, const float* Q, int n, int ld, float* Z) {
    const int n4 = (n + 3) & ~3;
    for (int idx = threadIdx.x; idx < n4 * n4; idx += blockDim.x) {
        const int i = idx / n4, j = idx % n4;
        float s = 0.f;
        if (i < n && j < n)
            for (int k = 0; k < n; ++k) {
                const float w = D[k * ld + k];
                const float f = w > 0.f ? rsqrtf(w) : 0.f;
                s = fmaf(Q[i * ld + k] * f, Q[j * ld + k], s);
            }
        Z[i * ld + j] = s;
    }
    __syncthreads();
}

// dst[i][c] = src[i][c0 + c] for c < w, 0 for w <= c < round4(w); rows x ...
// (eight elements per thread per pass, loaded before any is stored, so the
// global reads overlap instead of forming a chain)
// (32-bit index arithmetic: the planner accepts a mode only when
// I_n x (Rp_n + 4) stays below 2^31.)
__device__ __noinline__ void copy_cols(const float* src, int lds, int c0, int w, int64_t rows, float* dst, int ldd) {
    const int w4 = (w + 3) & ~3;
    const int tot = (int)rows * w4;
    const int step = blockDim.x;
    for (int base = threadIdx.x; base < tot; base += 8 * step) {
        float v[8];
        int off[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = base + u * step;
            const int i = idx / w4, c = idx - (idx / w4) * w4;
            off[u] = idx < tot ? i * ldd + c : -1;
            v[u] = (idx < tot && c < w) ? src[(int64_t)i * lds + c0 + c] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (off[u] >= 0) dst[off[u]] = v[u];
    }
}



__device__ JacobiBufs carve_jacobi(float* base, int ld) {
    JacobiBufs b;
    b.A = base;
    b.V = b.A + ld * ld;
    b.A2 = b.V + ld * ld;
    b.V2 = b.A2 + ld * ld;
    b.cs = b.V2 + ld * ld;
    return b;
}
// (a multiple of 4 floats, so what follows stays 16-byte aligned)
__host__ __device__ constexpr int jacobi_floats(int ld) { return 4 * ld * ld + 4 * ld; }   // A, V, A2, V2, cs (+ 2 ld spare)

template <bool INLINE_SOLVE>
__device__ EigBufs sym_eig_orth(JacobiBufs& jb, int n, int ld, float tol, int max_sweeps, float* scratch) {
    const EigBufs eb = INLINE_SOLVE ? block_jacobi_body(jb.A, jb.V, jb.A2, jb.V2, jb.cs, n, ld, tol, max_sweeps)
                                    : block_jacobi(jb.A, jb.V, jb.A2, jb.V2, jb.cs, n, ld, tol, max_sweeps);
    if (n <= kOrthMinN) return eb;
    // the pair of buffers the last round did not leave its result in
    float* K = eb.A == jb.A ? jb.A2 : jb.A;
    float* out = eb.V == jb.V ? jb.V2 : jb.V;
    const int n4 = (n + 3) & ~3;
    tile_AtB(eb.V, ld, n, eb.V, ld, n, n, K, ld, true, scratch);    // K = V^T V (zero padded to n4)
    for (int idx = threadIdx.x; idx < n4 * n4; idx += blockDim.x) {
        const int i = idx / n4, j = idx % n4;
        K[i * ld + j] = (i < n && j < n) ? ((i == j) ? 1.5f : 0.f) - 0.5f * K[i * ld + j] : 0.f;
    }
    __syncthreads();
    tile_AB(eb.V, ld, n, K, ld, n4, n, out, ld, false);            // rows < n, columns < n4
    __syncthreads();
    return EigBufs{eb.A, out};
}

// ---------------------------------------------------------------------------
// FP64 eigen-solve (PASD_F_FP64_EIG). The n x n float matrix in jb.A (an FP32
// Gram matrix) is solved in double: the same round-robin cyclic Jacobi, with
// correctly rounded rotations and the relative threshold 1e-13, then the
// eigenvalues and eigenvectors are rounded to float into jb.A / jb.V for the
// FP32 steps that follow (the double results stay in `dw` for
// inv_sqrt_from_eig_d). `dw` holds jacobi_d_floats(ld) floats (8-byte aligned).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int jacobi_d_floats(int ld) { return 8 * ld * ld + 4 * ld; }
struct EigBufsD {
    EigBufs f;               // float copies (jb.A, jb.V)
    const double* A;         // eigenvalues on the diagonal
    const double* V;         // eigenvectors (columns)
};
__device__ EigBufsD sym_eig_fp64(JacobiBufs& jb, int n, int ld, float* dwf) {
    const int t = threadIdx.x, nt = blockDim.x;
    double* A = reinterpret_cast<double*>(dwf);
    double* V = A + ld * ld;
    double* A2 = V + ld * ld;
    double* V2 = A2 + ld * ld;
    double* cs = V2 + ld * ld;
    const double tol = 1e-13;
    const int m = n + (n & 1);
    for (int idx = t; idx < ld * ld; idx += nt) {
        const int i = idx / ld, j = idx % ld;
        A[idx] = (i < n && j < n) ? (double)jb.A[idx] : 0.0;
        V[idx] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (m >= 2) {
        for (int sweep = 0; sweep < 40; ++sweep) {
            int need = 0;
            for (int idx = t; idx < n * n; idx += nt) {
                const int i = idx / n, j = idx % n;
                if (i < j) {
                    const double apq = A[i * ld + j];
                    need |= (apq != 0.0 && fabs(apq) > tol * sqrt(fabs(A[i * ld + i] * A[j * ld + j])));
                }
            }
            if (!__syncthreads_or(need)) break;
            for (int round = 0; round < m - 1; ++round) {
                int rot = 0;
                if (t < m) {
                    const int pi = rr_partner(t, round, m);
                    const int p = min(t, pi), q = max(t, pi);
                    const double app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
                    double c = 1.0, sn = 0.0;
                    if (apq != 0.0 && fabs(apq) > tol * sqrt(fabs(app * aqq))) {
                        const double theta = (aqq - app) / (2.0 * apq);
                        const double tt = fabs(theta) > 1e150 ? 0.5 / theta
                                                              : copysign(1.0 / (fabs(theta) + sqrt(fma(theta, theta, 1.0))), theta);
                        c = 1.0 / sqrt(fma(tt, tt, 1.0));
                        sn = tt * c;
                        rot = 1;
                    }
                    cs[2 * t] = c;
                    cs[2 * t + 1] = (t == p) ? -sn : sn;
                }
                if (!__syncthreads_or(rot)) continue;
                for (int idx = t; idx < m * m; idx += nt) {
                    const int i = idx / m, j = idx % m;
                    const int pi = rr_partner(i, round, m), pj = rr_partner(j, round, m);
                    const double ci = cs[2 * i], si = cs[2 * i + 1], cj = cs[2 * j], sj = cs[2 * j + 1];
                    // symmetric in (i, j) with explicit rounding: A stays exactly symmetric
                    const double t1 = __dmul_rn(__dmul_rn(ci, cj), A[i * ld + j]);
                    const double t2 = __dmul_rn(__dmul_rn(ci, sj), A[i * ld + pj]);
                    const double t3 = __dmul_rn(__dmul_rn(si, cj), A[pi * ld + j]);
                    const double t4 = __dmul_rn(__dmul_rn(si, sj), A[pi * ld + pj]);
                    double v = __dadd_rn(__dadd_rn(t1, __dadd_rn(t2, t3)), t4);
                    if (pi == j && si != 0.0) v = 0.0;
                    A2[i * ld + j] = v;
                    if (i < n) V2[i * ld + j] = fma(V[i * ld + pj], sj, V[i * ld + j] * cj);
                }
                __syncthreads();
                double* tA = A; A = A2; A2 = tA;
                double* tV = V; V = V2; V2 = tV;
            }
        }
    }
    for (int idx = t; idx < ld * ld; idx += nt) {
        jb.A[idx] = (float)A[idx];
        jb.V[idx] = (float)V[idx];
    }
    __syncthreads();
    return EigBufsD{EigBufs{jb.A, jb.V}, A, V};
}

// inv_sqrt_from_eig on the double eigen-system, rounded to float once.
__device__ void inv_sqrt_from_eig_d(const double* D, const double* Q, int n, int ld, float* Z) {
    const int n4 = (n + 3) & ~3;
    for (int idx = threadIdx.x; idx < n4 * n4; idx += blockDim.x) {
        const int i = idx / n4, j = idx % n4;
        double s = 0.0;
        if (i < n && j < n)
            for (int k = 0; k < n; ++k) {
                const double w = D[k * ld + k];
                const double f = w > 0.0 ? 1.0 / sqrt(w) : 0.0;
                s = fma(Q[i * ld + k] * f, Q[j * ld + k], s);
            }
        Z[i * ld + j] = (float)s;
    }
    __syncthreads();
}

// Row stride of the I x R matrices of the U-step in shared memory: a multiple of
// 4 with (stride / 4) odd, so float4 rows of consecutive rows hit distinct banks.
__host__ __device__ inline int polar_ld(int Rp) { return ((Rp / 4) & 1) ? Rp : Rp + 4; }

// ---------------------------------------------------------------------------
// SVT (Eq. 13 and the SVT definition after it), one CTA per mode.
// ---------------------------------------------------------------------------
// (also the scratch of the eigenvector re-orthonormalisation: TILE_SCRATCH floats)
__host__ __device__ inline int svt_red_floats(int Rp) { return Rp * Rp > TILE_SCRATCH ? Rp * Rp : TILE_SCRATCH; }

template <bool FP64>
__device__ __forceinline__ void svt_body(const SmallModeArgs& m, DevScalars* sc, const int mode) {
    if (sc->done) return;
    const double mu = sc->mu;
    const int R = m.R, Rp = m.Rp, ld = Rp;
    const int t = threadIdx.x;
    extern __shared__ __align__(16) float sm[];
    JacobiBufs jb = carve_jacobi(sm, ld);
    float* Smat = sm + jacobi_floats(ld);       // ld x ld (sorted eigenvectors, zero padded)
    float* sigsh = Smat + ld * ld;              // ld
    int* perm = reinterpret_cast<int*>(sigsh + ld);
    float* red = reinterpret_cast<float*>(perm + ld);   // svt_red_floats(Rp)

    // 1. Gram matrix = sum over the A-pass CTA partials. Thread (f, g) adds
    //    float4 f of partials g, g + G, ... (sixteen loads in flight), then the G
    //    group sums are added in order; the upper triangle is mirrored, so the
    //    matrix is exactly symmetric.
    {
        const int nf4 = Rp * Rp / 4;
        const int G = max(1, (int)blockDim.x / nf4);
        const float4* part = reinterpret_cast<const float4*>(m.gram_part);
        float4* red4 = reinterpret_cast<float4*>(red);
        for (int w = t; w < nf4 * G; w += blockDim.x) {
            const int f = w % nf4, g = w / nf4;
            // batches of 16 loads, the last one predicated (absent partials read as
            // zero, which leaves the in-order sums unchanged), so no load waits on an add
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int p = g; p < m.n_gram; p += 16 * G) {
                float4 v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    v[u] = p + u * G < m.n_gram ? part[(size_t)(p + u * G) * nf4 + f] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    acc.x += v[u].x; acc.y += v[u].y; acc.z += v[u].z; acc.w += v[u].w;
                }
            }
            red4[g * nf4 + f] = acc;
        }
        __syncthreads();
        for (int o = t; o < Rp * Rp; o += blockDim.x) {
            const int i = o / Rp, j = o % Rp;
            if (i > j || j >= R) continue;
            float s = 0.f;
            for (int g = 0; g < G; ++g) s += red[g * Rp * Rp + o];
            jb.A[i * ld + j] = s;
            jb.A[j * ld + i] = s;
        }
        __syncthreads();
    }
    // 2. eigen-decomposition
    const EigBufs eb = FP64 ? sym_eig_fp64(jb, R, ld, red + svt_red_floats(Rp)).f
                            : sym_eig_orth<true>(jb, R, ld, 1e-6f, 30, red);
    const float* Ae = eb.A;
    const float* Ve = eb.V;
    sort_desc(Ae, R, ld, perm);
    // 3. thresholds, sorted eigenvectors (W), kept count and nuclear norm
    const float tau = (float)(m.lambda / mu);
    if (t < Rp) {
        float sig = 0.f, f = 0.f;
        if (t < R) {
            const float lam = Ae[perm[t] * ld + perm[t]];
            sig = sqrtf(fmaxf(lam, 0.f));
            f = sig > tau ? 1.f - tau / sig : 0.f;
        }
        sigsh[t] = sig;
        m.sigma[t] = sig;
        m.F[t] = f;
    }
    int moved = 0;
    for (int idx = t; idx < Rp * Rp; idx += blockDim.x) {
        const int i = idx / Rp, j = idx % Rp;
        const bool in = i < R && j < R;
        const float v = in ? Ve[i * ld + perm[j]] : (i == j ? 1.f : 0.f);
        m.W[idx] = v;
        Smat[i * ld + j] = in ? v : 0.f;
        moved |= v != (i == j ? 1.f : 0.f);
    }
    // W exactly I (no rotation, order unchanged): Urot = U W below is an exact copy of U
    const int ident = !__syncthreads_or(moved);
    if (t == 0) sc->w_ident[mode] = ident;
    if (t < 32) {
        double nuc = 0.0;
        int kept = 0;
        for (int i = t; i < R; i += 32) {
            const float sig = sigsh[i];
            if (sig > tau) { ++kept; nuc += (double)sig - (double)tau; }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            nuc += __shfl_xor_sync(0xffffffffu, nuc, off);
            kept += __shfl_xor_sync(0xffffffffu, kept, off);
        }
        if (t == 0) {
            *m.kept = kept;
            sc->kept[mode] = kept;
            sc->nuclear[mode] = nuc;
        }
    }
    // 4. Urot = U W (I x Rp): the active subspace in the eigenbasis of the SVT.
    //    With Vrot = diag(F) W^T A_n (rows beyond the kept count are zero),
    //    fold_n(U_n V_n) = Urot[:, :s] Vrot[:s], the refold of rank s.
    //    U's padding columns are zero, so the product runs over Rp.
    tile_AB(m.U, Rp, Rp, Smat, ld, Rp, m.I, m.Urot, Rp, false);
}

template <bool FP64>
__global__ void __launch_bounds__(SM_THREADS, 1) svt_kernel(SmallArgs sa) {
    svt_body<FP64>(sa.m[blockIdx.x], sa.sc, blockIdx.x);
}
// one CTA per (solve, mode) entry of the batch
__global__ void __launch_bounds__(SM_THREADS, 1) svt_kernel_batched(const SmallBatchEntry* e) {
    const SmallBatchEntry& x = e[blockIdx.x];
    svt_body<false>(x.m, x.sc, x.mode);
}

// ---------------------------------------------------------------------------
// U-step (Eq. 9, Eq. 10), one CTA per mode. In the eigenbasis W of the last
// SVT, V_n = diag(F) W^T A_n, so M_n = G_n V_n^T = (G_n A_n^T) W diag(F): its
// columns s..R-1 (F = 0, the null space of V_n^T) vanish. The result is
//   U = [ P1 , X ],  P1 = polar(M_n[:, :s]),  X = polar((I - P1 P1^T) (U W)[:, s:]),
// i.e. the unique polar factor on the range of M_n and, on its null space, the
// isometry closest to the previous iterate (identity at k = 0, where s = 0).
// A closing Newton-Schulz step re-orthonormalises U. The I x R matrices live in
// shared memory when they fit, else in the global scratch.
// ---------------------------------------------------------------------------
template <bool FP64>
__device__ __forceinline__ void polar_body(const SmallModeArgs& m, DevScalars* sc, const int mode) {
    if (sc->done) return;
    const int R = m.R, Rp = m.Rp, ld = Rp;
    const int64_t I = m.I;
    extern __shared__ __align__(16) float sm[];
    JacobiBufs jb = carve_jacobi(sm, ld);
    float* Z = sm + jacobi_floats(ld);          // ld x ld
    float* K = Z + ld * ld;                     // ld x ld
    float* tsc = K + ld * ld;                   // TILE_SCRATCH
    float* big = tsc + TILE_SCRATCH;            // 4 x I x LD when it fits
    const bool in_smem = m.polar_in_smem != 0;
    const int LD = in_smem ? polar_ld(Rp) : Rp;
    float* dw = in_smem ? big + 4 * I * LD : big; // FP64 eigen-solve workspace (PASD_F_FP64_EIG)
    float* Mw = in_smem ? big : m.scratch;      // [P1 | X]
    float* Pw = Mw + I * LD;                    // M in the W basis
    float* Bw = Pw + I * LD;                    // (U W)[:, s:], then (I - P1 P1^T) of it
    float* Xb = Bw + I * LD;                    // X

    const int s = *m.kept;
    const int q = R - s;
    const int s4 = (s + 3) & ~3, q4 = (q + 3) & ~3;

    if (s == 0 && sc->w_ident[mode]) {
        // Nothing kept and the last SVT left the basis exactly as it was (W = I, so
        // Urot = U): Eq. 10 with M_n = 0 and every direction in the null space
        // returns the polar factor of U, which is U itself (a previous U-step's
        // orthonormal output, or eye at the start). U stays as it is.
        return;
    }
    if (s == 0) {
        // Nothing kept: the polar factor of Urot = U W. U and W are orthogonal to
        // rounding, so Urot^T Urot = I + O(1e-6) and one Newton-Schulz step gives
        // the polar factor to O(1e-12), the step the general path also ends with.
        // Urot's padding columns are zero, so the products run over Rp.
        tile_AtB(m.Urot, Rp, R, m.Urot, Rp, R, I, K, ld, true, tsc);
        int far = 0;
        for (int idx = threadIdx.x; idx < R * R; idx += blockDim.x) {
            const int i = idx / R, j = idx % R;
            far |= fabsf(K[i * ld + j] - (i == j ? 1.f : 0.f)) > 1e-3f;
        }
        if (!__syncthreads_or(far)) {
            for (int idx = threadIdx.x; idx < Rp * Rp; idx += blockDim.x) {
                const int i = idx / Rp, j = idx % Rp;
                Z[i * ld + j] = (i < R && j < R) ? ((i == j) ? 1.5f : 0.f) - 0.5f * K[i * ld + j] : 0.f;
            }
            __syncthreads();
            tile_AB(m.Urot, Rp, Rp, Z, ld, Rp, I, m.U, Rp, false);
            return;
        }
        // (not near-orthonormal: the general path below)
    }

    // both global inputs at once: M in the W basis (G_n Vrot^T, summed over
    // regions by the finalize kernel) and (U W)[:, s:] from the last SVT
    if (s > 0) copy_cols(m.Mred, Rp, 0, s, I, Pw, LD);
    if (q > 0) copy_cols(m.Urot, Rp, s, q, I, Bw, LD);
    __syncthreads();
    if (s > 0) {
        // B1 = M^T M, Z1 = B1^{-1/2}, P1 = M Z1
        tile_AtB(Pw, LD, s, Pw, LD, s, I, jb.A, ld, true, tsc);
        if (FP64) {
            const EigBufsD ed = sym_eig_fp64(jb, s, ld, dw);
            inv_sqrt_from_eig_d(ed.A, ed.V, s, ld, Z);
        } else {
            const EigBufs eb = sym_eig_orth(jb, s, ld, 1e-6f, 30, tsc);
            inv_sqrt_from_eig(eb.A, eb.V, s, ld, Z);
        }
        tile_AB(Pw, LD, s, Z, ld, s4, I, Mw, LD, false);
        __syncthreads();
    }
    if (q > 0) {
        // B = (U W)[:, s:] (eye at k = 0), less its part on the range of P1
        if (s > 0) {
            // K = P1^T Ur (s x q);  B = Ur - P1 K
            tile_AtB(Mw, LD, s, Bw, LD, q, I, K, ld, false, tsc);
            tile_AB(Mw, LD, s, K, ld, q4, I, Bw, LD, true);
            __syncthreads();
        }
        tile_AtB(Bw, LD, q, Bw, LD, q, I, jb.A, ld, true, tsc);
        if (FP64) {
            const EigBufsD ed = sym_eig_fp64(jb, q, ld, dw);
            inv_sqrt_from_eig_d(ed.A, ed.V, q, ld, Z);
        } else {
            const EigBufs eb = sym_eig_orth(jb, q, ld, 1e-6f, 30, tsc);
            inv_sqrt_from_eig(eb.A, eb.V, q, ld, Z);
        }
        tile_AB(Bw, LD, q, Z, ld, q4, I, Xb, LD, false);
        __syncthreads();
        for (int idx = threadIdx.x; idx < (int)I * q; idx += blockDim.x) {
            const int i = idx / q;
            const int c = idx - i * q;
            Mw[i * LD + s + c] = Xb[i * LD + c];
        }
        __syncthreads();
    }
    // Newton-Schulz: U = Un (3 I - Un^T Un) / 2, written with zero padding columns
    tile_AtB(Mw, LD, R, Mw, LD, R, I, K, ld, true, tsc);
    for (int idx = threadIdx.x; idx < Rp * Rp; idx += blockDim.x) {
        const int i = idx / Rp, j = idx % Rp;
        Z[i * ld + j] = (i < R && j < R) ? ((i == j) ? 1.5f : 0.f) - 0.5f * K[i * ld + j] : 0.f;
    }
    __syncthreads();
    tile_AB(Mw, LD, R, Z, ld, Rp, I, m.U, Rp, false);
}

template <bool FP64>
__global__ void __launch_bounds__(SM_THREADS, 1) polar_kernel(SmallArgs sa) {
    polar_body<FP64>(sa.m[blockIdx.x], sa.sc, blockIdx.x);
}
__global__ void __launch_bounds__(SM_THREADS, 1) polar_kernel_batched(const SmallBatchEntry* e) {
    const SmallBatchEntry& x = e[blockIdx.x];
    polar_body<false>(x.m, x.sc, x.mode);
}

static size_t small_base_floats(int maxRp) {
    const int ld = maxRp;
    return (size_t)jacobi_floats(ld) + 2 * (size_t)ld * ld + TILE_SCRATCH;
}
static size_t svt_smem_bytes(int maxRp, bool fp64) {
    const int ld = maxRp;
    return 4 * ((size_t)jacobi_floats(ld) + (size_t)ld * ld + 2 * (size_t)ld + svt_red_floats(maxRp) +
                (fp64 ? jacobi_d_floats(ld) : 0));
}
// Bytes of shared memory the U-step needs with its I x R matrices resident.
size_t polar_smem_bytes(int maxRp, int64_t maxI, bool fp64) {
    return 4 * (small_base_floats(maxRp) + 4 * (size_t)maxI * polar_ld(maxRp) + (fp64 ? jacobi_d_floats(maxRp) : 0));
}

size_t svt_launch_smem(const SmallArgs& a) {
    int maxRp = 4;
    bool fp64 = false;
    for (int n = 0; n < a.N; ++n) {
        maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
        fp64 = fp64 || a.m[n].fp64_eig;
    }
    return svt_smem_bytes(maxRp, fp64);
}

size_t polar_launch_smem(const SmallArgs& a) {
    int maxRp = 4;
    int64_t maxI = 1;
    bool any_smem = false, fp64 = false;
    for (int n = 0; n < a.N; ++n) {
        maxRp = a.m[n].Rp > maxRp ? a.m[n].Rp : maxRp;
        fp64 = fp64 || a.m[n].fp64_eig;
        if (a.m[n].polar_in_smem) { any_smem = true; maxI = a.m[n].I > maxI ? a.m[n].I : maxI; }
    }
    return any_smem ? polar_smem_bytes(maxRp, maxI, fp64)
                    : 4 * (small_base_floats(maxRp) + (fp64 ? jacobi_d_floats(maxRp) : 0));
}

void launch_svt(const SmallArgs& a, cudaStream_t s) {
    const size_t smem = svt_launch_smem(a);
    if (a.m[0].fp64_eig) {
        set_smem_attr((const void*)svt_kernel<true>, (int)smem);
        svt_kernel<true><<<a.N, SM_THREADS, smem, s>>>(a);
    } else {
        set_smem_attr((const void*)svt_kernel<false>, (int)smem);
        svt_kernel<false><<<a.N, SM_THREADS, smem, s>>>(a);
    }
}

void launch_polar(const SmallArgs& a, cudaStream_t s) {
    const size_t smem = polar_launch_smem(a);
    if (a.m[0].fp64_eig) {
        set_smem_attr((const void*)polar_kernel<true>, (int)smem);
        polar_kernel<true><<<a.N, SM_THREADS, smem, s>>>(a);
    } else {
        set_smem_attr((const void*)polar_kernel<false>, (int)smem);
        polar_kernel<false><<<a.N, SM_THREADS, smem, s>>>(a);
    }
}

void launch_polar_batched(const SmallBatchEntry* e, int n, size_t smem, cudaStream_t s) {
    set_smem_attr((const void*)polar_kernel_batched, (int)smem);
    polar_kernel_batched<<<n, SM_THREADS, smem, s>>>(e);
}

void launch_svt_batched(const SmallBatchEntry* e, int n, size_t smem, cudaStream_t s) {
    set_smem_attr((const void*)svt_kernel_batched, (int)smem);
    svt_kernel_batched<<<n, SM_THREADS, smem, s>>>(e);
}

// ---------------------------------------------------------------------------
// Finalize one loop body. CTA 0: residual norms of T - Z_n - E (the stop test
// of Algorithm 1), objective of Eq. 3, mu schedule, iteration record. Other
// CTAs: the fixed-order sum of the M-pass partials of G_n Vrot_n^T (64 outputs
// per CTA, four threads per output), which the next U-step reads.
// part layout per region: [0] max |T - Z_n - E|, [1] sum |E|, [2] non-finite
// flag, [3 + n] sum (T - Z_n - E)^2.
// ---------------------------------------------------------------------------
constexpr int FIN_THREADS = 256;
constexpr int FIN_OUT = FIN_THREADS / 4;

__device__ __forceinline__ void finalize_body(const FinalizeArgs& fa, const int block) {
    DevScalars* sc = fa.sc;
    if (sc->done) return;
    const int t = threadIdx.x, nt = blockDim.x;
    if (block > 0) {
        __shared__ float sub[4][FIN_OUT];
        const int ol = t % FIN_OUT, h = t / FIN_OUT;
        int64_t o = (int64_t)(block - 1) * FIN_OUT + ol;
        int mode = -1;
        int64_t i = 0;
        int r = 0;
        for (int n = 0; n < fa.N; ++n) {
            const int64_t cnt = fa.I[n] * fa.R[n];
            if (o < cnt) { mode = n; i = o / fa.R[n]; r = (int)(o % fa.R[n]); break; }
            o -= cnt;
        }
        float acc = 0.f;
        if (mode >= 0 && r < sc->kept[mode]) {      // only the kept directions carry G V^T
            const int64_t stride = fa.I[mode] * fa.Rp[mode];
            const float* src = fa.mp_part[mode] + i * fa.Rp[mode] + r;
            const int np = fa.n_mp[mode];
            const float* sp = src + (int64_t)h * stride;
            const int64_t st4 = 4 * stride;
            for (int p = h; p < np; p += 16, sp += 4 * st4) {   // 4 loads in flight (absent ones read as 0), added in order
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = p + 4 * u < np ? sp[u * st4] : 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u) acc += v[u];
            }
        }
        sub[h][ol] = acc;
        __syncthreads();
        if (h == 0 && mode >= 0)
            fa.Mred[mode][i * fa.Rp[mode] + r] = ((sub[0][ol] + sub[1][ol]) + sub[2][ol]) + sub[3][ol];
        return;
    }
    // scalars the tail needs, loaded first so that their latency overlaps the reduction
    double mu = 0.0, tn = 0.0, nuc[PASD_MAXN];
    int k0 = 0, kp[PASD_MAXN];
    if (t == 0) {
        mu = sc->mu;
        tn = sc->t_norm_fro;
        k0 = sc->k;
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n) {
            nuc[n] = n < fa.N ? sc->nuclear[n] : 0.0;
            kp[n] = n < fa.N ? sc->kept[n] : 0;
        }
    }
    // FP32 tree reductions over the region partials (fixed order)
    float mx = 0.f, l1 = 0.f, nf = 0.f;
    float r2[PASD_MAXN];
#pragma unroll
    for (int n = 0; n < PASD_MAXN; ++n) r2[n] = 0.f;
    for (int p = t; p < fa.nparts; p += nt) {
        const float* q = fa.part + (size_t)p * fa.stride;
        mx = fmaxf(mx, q[0]);
        l1 += q[1];
        nf = fmaxf(nf, q[2]);
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) r2[n] += q[3 + n];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        l1 += __shfl_xor_sync(0xffffffffu, l1, off);
        nf = fmaxf(nf, __shfl_xor_sync(0xffffffffu, nf, off));
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) r2[n] += __shfl_xor_sync(0xffffffffu, r2[n], off);
    }
    __shared__ float sh[FIN_THREADS / 32][PASD_MAXN + 3];
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
            mx = fmaxf(mx, sh[i][0]);
            l1 += sh[i][1];
            nf = fmaxf(nf, sh[i][2]);
#pragma unroll
            for (int n = 0; n < PASD_MAXN; ++n)
                if (n < fa.N) r2[n] += sh[i][3 + n];
        }
        float r2max = 0.f;
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) r2max = fmaxf(r2max, r2[n]);
        const double fro_rel = tn > 0 ? sqrt((double)r2max) / tn : 0.0;
        double obj = l1;
#pragma unroll
        for (int n = 0; n < PASD_MAXN; ++n)
            if (n < fa.N) obj += fa.lambda[n] * nuc[n];
        const double mxd = mx;
        sc->res_inf = mxd;
        sc->res_fro_rel = fro_rel;
        sc->objective = obj;
        sc->l1_E = l1;
        sc->mu_used = mu;
        const double mun = fa.rho * mu;
        sc->mu = mun < fa.mu_max ? mun : fa.mu_max;
        const int k = k0 + 1;
        sc->k = k;
        if (fa.trace && k <= fa.max_iter) {
            double* rec = fa.trace + (size_t)(k - 1) * 13;
            rec[0] = k; rec[1] = mxd; rec[2] = fro_rel; rec[3] = obj; rec[4] = mu;
#pragma unroll
            for (int n = 0; n < 8; ++n) rec[5 + n] = kp[n];
        }
        if (nf > 0.f || !isfinite(mx)) {
            sc->nonfinite = 1;
            sc->status = -4;   // PASD_ERR_NONFINITE
            sc->done = 1;
        } else if ((fa.stop_rule == 0 && mxd < fa.tol) || (fa.stop_rule == 1 && fro_rel < fa.tol)) {
            sc->status = 0;    // PASD_OK
            sc->done = 1;
        } else if (k >= fa.max_iter) {
            sc->status = fa.stop_rule == 2 ? 0 : 2;   // OK (fixed) / NOT_CONVERGED
            sc->done = 1;
        }
    }
}

__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel(FinalizeArgs fa) { finalize_body(fa, blockIdx.x); }
__global__ void __launch_bounds__(FIN_THREADS) finalize_kernel_batched(const FinBatchEntry* e, const int* block_entry) {
    const FinBatchEntry& x = e[block_entry[blockIdx.x]];
    finalize_body(x.a, blockIdx.x - x.start);
}

int finalize_ctas(const FinalizeArgs& a) {
    int64_t tot = 0;
    for (int n = 0; n < a.N; ++n) tot += a.I[n] * a.R[n];
    return 1 + (int)((tot + FIN_OUT - 1) / FIN_OUT);
}

void launch_finalize(const FinalizeArgs& a, cudaStream_t s) {
    finalize_kernel<<<finalize_ctas(a), FIN_THREADS, 0, s>>>(a);
}

void launch_finalize_batched(const FinBatchEntry* e, const int* block_entry, int grid, cudaStream_t s) {
    finalize_kernel_batched<<<grid, FIN_THREADS, 0, s>>>(e, block_entry);
}

// ---------------------------------------------------------------------------
// Vrot_n = diag(F) W^T A_n: the small factor V_n of Eq. 13 in the eigenbasis of
// the SVT, stored like A_n ([pre][Rp][post]); rows at and beyond the kept
// count are zero. All modes in one launch. A thread owns four consecutive
// columns b .. b + 3 of one a-row when post % 4 == 0 (one 16-byte load per row
// of A and one 16-byte store per row of Vrot), else one column (post == 1: the
// Rp contiguous floats of the column, as float4 moves).
// ---------------------------------------------------------------------------
// (four columns a thread only where there are enough columns to fill the GPU
// with the fatter threads)
__host__ __device__ inline int vrot_cols(int64_t P, int64_t post, int RB) {
    return (post % 4 == 0 && post > 1 && RB <= 32 && P >= (1 << 18)) ? 4 : 1;
}

template <int RB, bool V4>
__device__ __forceinline__ void vrot_body(const VrotArgs& va, const int block) {
    const DevScalars* sc = va.sc;
    if (sc->done) return;
    int k = 0;
    while (k + 1 < va.N && (int)block >= va.cta_start[k + 1]) ++k;
    const VrotMode& m = va.m[k];
    const int R = m.R, Rp = m.Rp;
    const int s = sc->kept[m.mode];
    // consumers read the first round4(s) rows only (rows s .. round4(s) - 1 are
    // zero); with nothing kept there is nothing to write
    const int s4 = (s + 3) & ~3;
    if (s4 == 0) return;
    // Wt[i][r] = F_i W[r][i] with row stride RB, zero for R <= r < RB: the
    // product below runs over the float4 groups r < Rp of a row as broadcasts,
    // and the padding terms are exact zeros, so each sum is the same as over r < R
    __shared__ __align__(16) float Wt[PASD_MAXR * PASD_MAXR];
    for (int idx = threadIdx.x; idx < s * RB; idx += blockDim.x) {
        const int i = idx / RB, r = idx % RB;
        Wt[idx] = r < R ? m.F[i] * m.W[r * Rp + i] : 0.f;
    }
    __syncthreads();
    const int64_t u = (int64_t)(block - va.cta_start[k]) * blockDim.x + threadIdx.x;
    if (V4 && vrot_cols(m.P, m.post, RB) == 4) {
        const int64_t per_row = m.post / 4;
        if (u >= m.P / 4) return;
        const int64_t a = u / per_row, b = 4 * (u - a * per_row);
        const float* src = m.A + a * Rp * m.post + b;
        float* dst = m.V + a * Rp * m.post + b;
        float av[RB][4];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < R) v = *reinterpret_cast<const float4*>(src + (int64_t)r * m.post);
            av[r][0] = v.x; av[r][1] = v.y; av[r][2] = v.z; av[r][3] = v.w;
        }
#pragma unroll
        for (int i = 0; i < RB; ++i) {
            if (i < s4) {
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
                if (i < s) {
                    const float4* w4 = reinterpret_cast<const float4*>(Wt + i * RB);
#pragma unroll
                    for (int r4 = 0; r4 < RB / 4; ++r4) {
                        if (4 * r4 < Rp) {
                            const float4 w = w4[r4];
                            const float ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q)
#pragma unroll
                                for (int c = 0; c < 4; ++c) acc[c] = fmaf(ws[q], av[4 * r4 + q][c], acc[c]);
                        }
                    }
                }
                *reinterpret_cast<float4*>(dst + (int64_t)i * m.post) = make_float4(acc[0], acc[1], acc[2], acc[3]);
            }
        }
        return;
    }
    const int64_t j = u;
    if (j >= m.P) return;
    const int64_t a = j / m.post, b = j % m.post;
    const float* src = m.A + a * Rp * m.post + b;
    float* dst = m.V + a * Rp * m.post + b;
    // the column of A_n in registers (RB >= Rp, fully unrolled), all loads in
    // flight; with post == 1 the column is Rp contiguous floats (float4 moves).
    // Entries past R are set to zero (A's padding rows are never multiplied).
    float av[RB];
    if (m.post == 1) {
#pragma unroll
        for (int r4 = 0; r4 < RB / 4; ++r4) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * r4 < Rp) v = reinterpret_cast<const float4*>(src)[r4];
            av[4 * r4] = v.x; av[4 * r4 + 1] = v.y; av[4 * r4 + 2] = v.z; av[4 * r4 + 3] = v.w;
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if (r >= R) av[r] = 0.f;
    } else {
#pragma unroll
        for (int r = 0; r < RB; ++r) av[r] = r < R ? src[(int64_t)r * m.post] : 0.f;
    }
    float out[RB];
#pragma unroll
    for (int i = 0; i < RB; ++i) {
        float acc = 0.f;
        if (i < s) {
            const float4* w4 = reinterpret_cast<const float4*>(Wt + i * RB);
#pragma unroll
            for (int r4 = 0; r4 < RB / 4; ++r4) {
                if (4 * r4 < Rp) {
                    const float4 w = w4[r4];
                    acc = fmaf(w.x, av[4 * r4], acc);
                    acc = fmaf(w.y, av[4 * r4 + 1], acc);
                    acc = fmaf(w.z, av[4 * r4 + 2], acc);
                    acc = fmaf(w.w, av[4 * r4 + 3], acc);
                }
            }
        }
        out[i] = acc;
    }
    if (m.post == 1) {
#pragma unroll
        for (int i4 = 0; i4 < RB / 4; ++i4)
            if (4 * i4 < s4)
                reinterpret_cast<float4*>(dst)[i4] = make_float4(out[4 * i4], out[4 * i4 + 1], out[4 * i4 + 2], out[4 * i4 + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < RB; ++i)
            if (i < s4) dst[(int64_t)i * m.post] = out[i];
    }
}

template <int RB, bool V4>
__global__ void __launch_bounds__(256) vrot_kernel(VrotArgs va) { vrot_body<RB, V4>(va, blockIdx.x); }
template <int RB, bool V4>
__global__ void __launch_bounds__(256) vrot_kernel_batched(const VrotBatchEntry* e, const int* block_entry) {
    const VrotBatchEntry& x = e[block_entry[blockIdx.x]];
    vrot_body<RB, V4>(x.a, blockIdx.x - x.start);
}

int vrot_rb(int maxRp) {
    return maxRp <= 8 ? 8 : maxRp <= 16 ? 16 : maxRp <= 24 ? 24 : maxRp <= 32 ? 32 : maxRp <= 48 ? 48 : 64;
}

// CTAs of mode n's part of the launch (256 threads, one or four columns each)
int vrot_ctas(int64_t P, int64_t post, int maxRp) {
    const int cols = vrot_cols(P, post, vrot_rb(maxRp));
    return (int)((P / cols + 255) / 256);
}

template <int RB>
static void launch_vrot_batched_rb(bool v4, const VrotBatchEntry* e, const int* block_entry, int grid, cudaStream_t s) {
    if (v4) vrot_kernel_batched<RB, true><<<grid, 256, 0, s>>>(e, block_entry);
    else vrot_kernel_batched<RB, false><<<grid, 256, 0, s>>>(e, block_entry);
}
// every entry of one launch has the same rank bucket rb and four-column flag v4 (vrot_split)
void launch_vrot_batched(int rb, bool v4, const VrotBatchEntry* e, const int* block_entry, int grid, cudaStream_t s) {
    switch (rb) {
        case 8: launch_vrot_batched_rb<8>(v4, e, block_entry, grid, s); break;
        case 16: launch_vrot_batched_rb<16>(v4, e, block_entry, grid, s); break;
        case 24: launch_vrot_batched_rb<24>(v4, e, block_entry, grid, s); break;
        case 32: launch_vrot_batched_rb<32>(v4, e, block_entry, grid, s); break;
        case 48: launch_vrot_batched_rb<48>(v4, e, block_entry, grid, s); break;
        default: launch_vrot_batched_rb<64>(v4, e, block_entry, grid, s); break;
    }
}

// The four-column path is compiled into the launch only when some mode takes it:
// its registers would otherwise slow every mode's one-column path.
template <int RB>
static void launch_vrot_rb(const VrotArgs& a, cudaStream_t s) {
    bool v4 = false;
    for (int n = 0; n < a.N; ++n) v4 = v4 || vrot_cols(a.m[n].P, a.m[n].post, RB) == 4;
    const int grid = a.cta_start[a.N];
    if (v4) vrot_kernel<RB, true><<<grid, 256, 0, s>>>(a);
    else vrot_kernel<RB, false><<<grid, 256, 0, s>>>(a);
}

int vrot_split(const VrotArgs& a, VrotArgs* out, int* rb_out, bool* v4_out) {
    int k = 0;
    for (const int rb : {8, 16, 24, 32, 48, 64}) {
        VrotArgs g = a;
        g.N = 0;
        g.cta_start[0] = 0;
        bool v4 = false;
        for (int n = 0; n < a.N; ++n) {
            if (vrot_rb(a.m[n].Rp) != rb) continue;
            g.m[g.N] = a.m[n];
            g.cta_start[g.N + 1] = g.cta_start[g.N] + vrot_ctas(a.m[n].P, a.m[n].post, rb);
            v4 = v4 || vrot_cols(a.m[n].P, a.m[n].post, rb) == 4;
            ++g.N;
        }
        if (g.N == 0) continue;
        out[k] = g;
        rb_out[k] = rb;
        v4_out[k] = v4;
        ++k;
    }
    return k;
}

int launch_vrot(const VrotArgs& a, cudaStream_t s) {
    VrotArgs sub[PASD_MAXN];
    int rbs[PASD_MAXN];
    bool v4s[PASD_MAXN];
    const int ns = vrot_split(a, sub, rbs, v4s);
    for (int k = 0; k < ns; ++k) {
        const VrotArgs& g = sub[k];
        switch (rbs[k]) {
            case 8: launch_vrot_rb<8>(g, s); break;
            case 16: launch_vrot_rb<16>(g, s); break;
            case 24: launch_vrot_rb<24>(g, s); break;
            case 32: launch_vrot_rb<32>(g, s); break;
            case 48: launch_vrot_rb<48>(g, s); break;
            default: launch_vrot_rb<64>(g, s); break;
        }
    }
    return ns;
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
        sc->skipped = 0;
        for (int m = 0; m < PASD_MAXN; ++m) { sc->kept[m] = 0; sc->nuclear[m] = 0.0; sc->w_ident[m] = 1; }
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
