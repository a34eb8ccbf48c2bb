// Closed form of the idle start of Algorithm 1.
//
// With V_n = 0 and E = 0 every sub-step of a loop body is determined: the
// U-step has M_n = G_n V_n^T = 0 and keeps U_n (Eq. 10 with the null-space
// reading), the V-step thresholds the singular values of U_n^T G_n, the E-step
// soft-thresholds mean_n G_n (Eq. 15) and every multiplier gains mu T. Starting
// from Y_n = 0, E = 0, the state at the start of iteration i is therefore
//     G_n^i = T - E + Y_n^i / mu^i = g_i T,   g_i = 1 + c_i,
//     c_0 = 0,  c_{i+1} = (c_i + 1) mu^i / mu^{i+1},
// (g_i = 1 + (1 - rho^-i) / (rho - 1) while mu^i = mu^0 rho^i), and iteration i
// stays idle exactly while
//     g_i sigma_max(U_n^T T_(n)) <= lambda_n / mu^i   for every n   (nothing kept)
//     g_i max|T|                 <= 1 / (N mu^i)                     (E stays 0).
// Both left sides grow and both right sides shrink with i, so the idle
// iterations are a prefix 0 .. i_a - 1. After the first loop body the device
// holds sigma_n(U_n^T T_(n)) (the SVT's singular values) and max|T| (the
// residual of that body), so the bodies 1 .. i_a - 2 can be replaced by
// G_n = g T and the matching mu: the solve resumes at iteration i_a - 1. A
// relative margin of 1e-3 on both tests keeps the decision on the safe side of
// FP32 rounding (a later resume only recomputes idle bodies).
#include "pasd_impl.cuh"

namespace pasd {

__global__ void idle_skip_decide_kernel(IdleSkipArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevScalars* sc = a.sc;
    *a.g = 0.f;
    if (sc->done || sc->k != 1 || sc->l1_E != 0.0) return;
    for (int n = 0; n < a.N; ++n)
        if (sc->kept[n] != 0) return;
    const double tmax = sc->res_inf;
    if (!(tmax > 0.0)) return;
    double smax[PASD_MAXN];
    for (int n = 0; n < a.N; ++n) smax[n] = (double)a.sigma[n][0];
    const double margin = 1.0 + 1e-3;
    // first non-idle iteration i_a (iteration 0 was computed and was idle)
    auto idle = [&](double g, double mu) {
        if (g * tmax * margin > 1.0 / (mu * a.N)) return false;
        for (int n = 0; n < a.N; ++n)
            if (g * smax[n] * margin > a.lambda[n] / mu) return false;
        return true;
    };
    double mu = sc->mu, c = sc->mu_used / sc->mu;   // mu^1, c_1
    int i = 1;
    while (i < a.max_iter && idle(1.0 + c, mu)) {
        const double mn = a.rho * mu < a.mu_max ? a.rho * mu : a.mu_max;
        c = (c + 1.0) * mu / mn;
        mu = mn;
        ++i;
    }
    const int resume = i - 1;   // computed normally, followed by i_a
    if (resume <= 1) return;
    // replay the scalars of the replaced bodies 2 .. resume (iterations 1 .. resume - 1)
    mu = sc->mu;
    c = sc->mu_used / sc->mu;
    double mu_last = mu;
    for (int it = 1; it < resume; ++it) {
        mu_last = mu;
        if (a.trace) {
            double* rec = a.trace + (size_t)it * 13;    // body it + 1
            rec[0] = it + 1;
            rec[1] = tmax;
            rec[2] = sc->res_fro_rel;
            rec[3] = sc->objective;
            rec[4] = mu;
            for (int n = 0; n < 8; ++n) rec[5 + n] = 0.0;
        }
        const double mn = a.rho * mu < a.mu_max ? a.rho * mu : a.mu_max;
        c = (c + 1.0) * mu / mn;
        mu = mn;
    }
    sc->mu = mu;                 // mu^resume
    sc->mu_used = mu_last;       // mu of the last replaced iteration
    sc->k = resume;
    sc->skipped = resume - 1;
    *a.g = (float)(1.0 + c);
}

// G_n = g T for every mode (no-op when the decision kernel left g = 0)
__global__ void idle_skip_apply_kernel(IdleSkipArgs a) {
    const float g = *a.g;
    if (g == 0.f) return;
    const int64_t n4 = a.D / 4;
    const float4* T4 = reinterpret_cast<const float4*>(a.T);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
        float4 v = T4[e];
        v.x *= g; v.y *= g; v.z *= g; v.w *= g;
        for (int n = 0; n < a.N; ++n) reinterpret_cast<float4*>(a.G[n])[e] = v;
    }
    for (int64_t e = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.D;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float v = a.T[e] * g;
        for (int n = 0; n < a.N; ++n) a.G[n][e] = v;
    }
}

void launch_idle_skip(const IdleSkipArgs& a, int num_sms, cudaStream_t s) {
    idle_skip_decide_kernel<<<1, 32, 0, s>>>(a);
    idle_skip_apply_kernel<<<num_sms * 4, 256, 0, s>>>(a);
}

}  // namespace pasd
