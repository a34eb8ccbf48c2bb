// Standalone operations exposed through the C ABI (outside the solve loop).
#include "../../include/pasd.h"
#include "pasd_impl.cuh"

#include <string>

namespace pasd {

// gram = sum over CTA partials, fixed order (deterministic).
__global__ void gram_reduce_kernel(const float* __restrict__ part, int ncta, int R, float* gram) {
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= R * R) return;
    float s = 0.f;
    for (int p = 0; p < ncta; ++p) s += part[(size_t)p * R * R + o];
    gram[o] = s;
}

void launch_gram_reduce(const float* part, int ncta, int R, float* gram, cudaStream_t s) {
    int n = R * R;
    gram_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(part, ncta, R, gram);
}

bool mode_product_rank_ok(int R) {
    static const int b[] = {4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 56, 64};
    for (int v : b)
        if (R == v) return true;
    return false;
}

}  // namespace pasd

using namespace pasd;

void pasd_set_error(const std::string& s);

extern "C" pasd_status pasd_mode_product(const float* X, int64_t pre, int64_t I, int64_t post,
                                         const float* U, int32_t R, float* A, float* gram,
                                         void* stream) {
    if (!X || !U || !A || pre < 1 || I < 1 || post < 1) {
        pasd_set_error("pasd_mode_product: NULL pointer or empty shape");
        return PASD_ERR_INVALID_ARG;
    }
    if (!mode_product_rank_ok(R)) {
        pasd_set_error("pasd_mode_product: R must be one of 4..32 (step 4), 40, 48, 56, 64");
        return PASD_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t P = pre * post;
    const int ncta = apass_ncta(P);
    const size_t part_bytes = (size_t)ncta * R * R * sizeof(float);
    char* scratch = nullptr;
    cudaError_t e = cudaMalloc(&scratch, 256 + part_bytes);
    if (e != cudaSuccess) {
        pasd_set_error(std::string("pasd_mode_product: cudaMalloc: ") + cudaGetErrorString(e));
        return PASD_ERR_OOM;
    }
    DevScalars* sc = reinterpret_cast<DevScalars*>(scratch);
    float* part = reinterpret_cast<float*>(scratch + 256);
    e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), s);
    if (e == cudaSuccess) {
        ApassArgs a{};
        a.G = X; a.U = U; a.A = A; a.gram_part = part; a.sc = sc;
        a.I = I; a.pre = pre; a.post = post; a.P = P; a.R = R; a.Rp = R; a.ncta = ncta;
        launch_apass(a, s);
        if (gram) launch_gram_reduce(part, ncta, R, gram, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(scratch);
    if (e != cudaSuccess) {
        pasd_set_error(std::string("pasd_mode_product: ") + cudaGetErrorString(e));
        return PASD_ERR_CUDA;
    }
    return PASD_OK;
}
