// jac_sweep_dev_noalloc: the stateless sweep without a caller workspace.
//
// Some callers cannot allocate device memory at all: a plugin whose host
// application owns every byte of the GPU through its own pool allocator and
// hands the plugin only its input and output buffers, or a control loop that
// cannot afford the device-wide synchronisation that cudaMalloc/cudaFree may
// imply.  For them this entry point takes the same grid as jac_sweep_dev
// and keeps the sweep's scratch (error word, arrival counter, per-CTA
// residual partials) in a fixed-size array in this library's own device
// memory, reserved when the library's module is loaded onto a device.
//
// The array is a host-side stand-in in host code: its device address is
// fetched once per device with cudaGetSymbolAddress, with that device
// current, and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "jac_common.cuh"
#include "jac_internal.h"

namespace {

// Scratch: 256-byte header (error word, counter, default residual slot) plus
// one double per CTA of the last sweep's launch.
constexpr size_t kNoAllocScratchBytes = jac::kWsHeaderBytes + (size_t)JAC_NOALLOC_MAX_CTAS * sizeof(double);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

jac_status scratch_for_current_device(void **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        jac::set_thread_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return JAC_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        jac::set_thread_error("device ordinal out of range for the static scratch table");
        return JAC_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            jac::set_thread_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return JAC_ECUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return JAC_OK;
}

}  // namespace

extern "C" {

jac_status jac_sweep_dev_noalloc(const jac_grid *g, const jac_plan *plan, int n_iter, double *d_residual,
                                 void *stream)
{
    jac_status s = jac::validate_grid(g);
    if (s != JAC_OK) return s;
    if (n_iter < 0) {
        jac::set_thread_error("n_iter must be >= 0");
        return JAC_EINVAL;
    }
    if (n_iter == 0) return JAC_OK;
    const jac_plan p = jac::resolve_plan(g, plan);
    const size_t need = jac::sweep_workspace_bytes(g, p);
    if (need > kNoAllocScratchBytes) {
        jac::set_thread_error("launch needs " + std::to_string((need - jac::kWsHeaderBytes) / sizeof(double)) +
                              " CTAs but jac_sweep_dev_noalloc supports at most " +
                              std::to_string(JAC_NOALLOC_MAX_CTAS) + "; use a deeper kdepth or jac_sweep_dev");
        return JAC_EINVAL;
    }
    void *scratch = nullptr;
    if ((s = scratch_for_current_device(&scratch)) != JAC_OK) return s;
    // The header must start at zero; the previous call's contents are kept.
    cudaError_t e = cudaMemsetAsync(scratch, 0, jac::kWsHeaderBytes, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        jac::set_thread_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return JAC_ECUDA;
    }
    return jac::sweep_dev(g, &p, n_iter, d_residual, scratch, kNoAllocScratchBytes, stream);
}

}  // extern "C"
