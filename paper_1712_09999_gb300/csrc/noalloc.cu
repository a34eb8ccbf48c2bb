// pasd_mode_product_noalloc: the mode-n product and Gram matrix of
// pasd_mode_product without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need this
// product: code running under a framework whose allocator must own every
// device byte (a raw cudaMalloc would be invisible to its accounting), and
// latency-critical loops where cudaMalloc/cudaFree would synchronise the
// device. For them the per-CTA Gram partial sums live in a fixed scratch array
// compiled into the library instead of being allocated per call.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchFloats floats
// (4 MiB). Every GPU that loads the library holds it until the process exits.
// In host code the array's name is only a host-side stand-in, not a device
// address, so the address handed to the kernels is taken with
// cudaGetSymbolAddress with that device current, on every call (a host-side
// lookup); the first call on a device (and the first after a cudaDeviceReset)
// also clears the flags and waits for that clear, so make it before any stream
// capture.
// Every call shares the one array and it keeps the last call's contents: two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller.
#include "../../include/pasd.h"
#include "pasd_impl.cuh"

#include <mutex>
#include <string>

namespace pasd {
void launch_gram_reduce(const float* part, int ncta, int R, float* gram, cudaStream_t s);
bool mode_product_rank_ok(int R);
}  // namespace pasd
void pasd_set_error(const std::string& msg);

using namespace pasd;

namespace {

constexpr size_t kNoAllocScratchFloats = size_t(1) << 20;   // 4 MiB of Gram partials

__device__ __align__(256) float g_mode_product_scratch[kNoAllocScratchFloats];
__device__ __align__(256) DevScalars g_mode_product_flags;   // "done" must read 0

struct DeviceScratch {
    float* part = nullptr;
    DevScalars* flags = nullptr;
    bool ready = false;
};
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
DeviceScratch g_scratch[kMaxDevices];

// Device addresses of the scratch on the current device. The addresses are
// looked up on every call (a host-side table lookup in the runtime) and compared
// with the cached ones: after a cudaDeviceReset the module is loaded again,
// possibly elsewhere, and the set-up (the flags clear) is then redone, so no call
// ever launches on a stale address. The set-up clears the flags on `stream` and
// waits for that clear.
pasd_status scratch_for_current_device(DeviceScratch** out, cudaStream_t stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        pasd_set_error(std::string("pasd_mode_product_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return PASD_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        pasd_set_error("pasd_mode_product_noalloc: device index out of range");
        return PASD_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DeviceScratch& d = g_scratch[dev];
    void* part = nullptr;
    void* flags = nullptr;
    e = cudaGetSymbolAddress(&part, g_mode_product_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&flags, g_mode_product_flags);
    if (e != cudaSuccess) {
        pasd_set_error(std::string("pasd_mode_product_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return PASD_ERR_CUDA;
    }
    if (!d.ready || d.part != part || d.flags != flags) {
        d.ready = false;
        d.part = static_cast<float*>(part);
        d.flags = static_cast<DevScalars*>(flags);
        // the product kernel returns early when flags->done is set: clear it once,
        // complete before any product is launched (on whatever stream)
        e = cudaMemsetAsync(d.flags, 0, sizeof(DevScalars), stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
        if (e != cudaSuccess) {
            pasd_set_error(std::string("pasd_mode_product_noalloc: clearing the flags: ") + cudaGetErrorString(e));
            return PASD_ERR_CUDA;
        }
        d.ready = true;
    }
    *out = &d;
    return PASD_OK;
}

}  // namespace

extern "C" pasd_status pasd_mode_product_noalloc(const float* X, int64_t pre, int64_t I, int64_t post,
                                                 const float* U, int32_t R, float* A, float* gram,
                                                 void* stream) {
    if (!X || !U || !A || pre < 1 || I < 1 || post < 1) {
        pasd_set_error("pasd_mode_product_noalloc: NULL pointer or empty shape");
        return PASD_ERR_INVALID_ARG;
    }
    if (!mode_product_rank_ok(R)) {
        pasd_set_error("pasd_mode_product_noalloc: R must be one of 4..32 (step 4), 40, 48, 56, 64");
        return PASD_ERR_UNSUPPORTED;
    }
    const int64_t P = pre * post;
    const int ncta = apass_ncta(P);
    if ((size_t)ncta * R * R > kNoAllocScratchFloats) {
        pasd_set_error("pasd_mode_product_noalloc: ceil(pre*post/256) * R * R exceeds the fixed scratch "
                       "of 1048576 floats; use pasd_mode_product");
        return PASD_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    DeviceScratch* d = nullptr;
    pasd_status st = scratch_for_current_device(&d, s);
    if (st != PASD_OK) return st;
    ApassArgs a{};
    a.G = X; a.U = U; a.A = A; a.gram_part = d->part; a.sc = d->flags;
    a.I = I; a.pre = pre; a.post = post; a.P = P; a.R = R; a.Rp = R; a.ncta = ncta;
    launch_apass(a, s);      // every CTA overwrites its whole R x R partial: nothing to clear
    if (gram) launch_gram_reduce(d->part, ncta, R, gram, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        pasd_set_error(std::string("pasd_mode_product_noalloc: ") + cudaGetErrorString(e));
        return PASD_ERR_CUDA;
    }
    return PASD_OK;
}
