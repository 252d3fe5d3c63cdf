// Allocation-free power spectrum (cwt_wavelet_power_noalloc in include/cwt.h).
//
// The partial sums of |W|^2 go to a fixed, file-scope device array instead of
// plan workspace, so the call needs neither a plan nor cudaMalloc.  In host
// code the array's name is only a host-side stand-in: its device address is
// looked up once per device with cudaGetSymbolAddress (that device current)
// and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/cwt.h"
#include "cwt_kernels.cuh"

using namespace cwtk;

namespace {

static __device__ __align__(256) double g_noalloc_partials[CWT_NOALLOC_MAX_PARTIALS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device (set up on the
// first call per device).
cwt_status scratch_address(double** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CWT_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess || !ptr) return CWT_ERR_CUDA;
        g_addr[dev] = (double*)ptr;
    }
    *out = g_addr[dev];
    return CWT_OK;
}

// True if q is device memory of the device `dev` (cudaPointerGetAttributes
// allocates nothing).  A pointer of another device, or host memory, would
// make the kernels read or write memory this device cannot address.
bool on_device(const void* q, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" cwt_status cwt_wavelet_power_noalloc(const void* W_dev, int64_t N, int32_t n_scales,
                                                int32_t is_complex, double* spectrum_dev, void* stream) {
    if (!W_dev || !spectrum_dev || N < 1 || n_scales < 1) return CWT_ERR_INVALID_ARG;
    if (((uintptr_t)W_dev % (is_complex ? 8 : 4)) != 0 || ((uintptr_t)spectrum_dev % 8) != 0)
        return CWT_ERR_INVALID_ARG;
    const int64_t chunks = (N + CWT_NOALLOC_CHUNK - 1) / CWT_NOALLOC_CHUNK;
    if (chunks * (int64_t)n_scales > CWT_NOALLOC_MAX_PARTIALS || n_scales > 65535) return CWT_ERR_UNSUPPORTED;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CWT_ERR_CUDA;
    if (!on_device(W_dev, dev) || !on_device(spectrum_dev, dev)) return CWT_ERR_INVALID_ARG;
    double* partials = nullptr;
    cwt_status st = scratch_address(&partials);
    if (st != CWT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((unsigned)chunks, (unsigned)n_scales);
    k_power_rows<256><<<grid, 256, 0, s>>>(W_dev, N, is_complex ? 1 : 0, CWT_NOALLOC_CHUNK, partials);
    if (cudaGetLastError() != cudaSuccess) return CWT_ERR_CUDA;
    k_power_finalize_uniform<<<n_scales, 32, 0, s>>>(partials, (int32_t)chunks, n_scales, N, spectrum_dev);
    if (cudaGetLastError() != cudaSuccess) return CWT_ERR_CUDA;
    return CWT_OK;
}
