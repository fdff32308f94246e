// fdtd_gradient_static: the gradient entry point without workspace scratch.
//
// fdtd_gradient stages the filter-transpose passes through two design-box
// sized FP64 arrays carved from the caller's workspace.  This variant uses a
// fixed array that the library itself owns in device memory instead, so the
// call touches nothing but the context's solver state and the caller's
// output.  It is meant for callers that cannot hand out or grow device
// memory at call time, for example code running inside a memory pool whose
// size was fixed up front, or a host component that only holds the device
// pointer of its output.  The paper has no counterpart: this is an
// integration aid, not part of the method.
//
// The array lives for the life of the process on every device that loads
// the library (FDTD_STATIC_DESIGN_MAX doubles twice, 16 MiB).  Calls share
// it: two calls that overlap on the GPU (different streams or contexts at
// the same time) race on it.  Each call overwrites the part it uses before
// reading it, so nothing has to start at zero.  Only a 2D E_z context with a
// design filter goes through the array, so only its design box is limited
// to FDTD_STATIC_DESIGN_MAX; the other contexts assemble their gradient
// directly and take any size.
#include <mutex>

#include "../../include/fdtd.h"
#include "fdtd_internal.h"

static __device__ __align__(256) double g_grad_scratch[2 * (size_t)FDTD_STATIC_DESIGN_MAX];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device; looked up once
// per device, with that device current.
fdtd_status scratch_on_current_device(double **out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FDTD_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_grad_scratch) != cudaSuccess || !p) return FDTD_ECUDA;
        g_scratch_ptr[dev] = (double *)p;
    }
    *out = g_scratch_ptr[dev];
    return FDTD_OK;
}

}  // namespace

extern "C" fdtd_status fdtd_gradient_static(fdtd_ctx *ctx, double *d_grad, size_t n)
{
    if (!ctx || !d_grad) return FDTD_EINVAL;
    // The array's address is looked up per device: the context's device must
    // be the current one, or the kernels would get another GPU's copy.
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FDTD_ECUDA;
    if (dev != fdtd::context_device(ctx)) return FDTD_EINVAL;
    double *scratch = nullptr;
    const fdtd_status s = scratch_on_current_device(&scratch);
    if (s != FDTD_OK) return s;
    return (fdtd_status)fdtd::gradient_into(ctx, d_grad, n, scratch, (size_t)FDTD_STATIC_DESIGN_MAX);
}
