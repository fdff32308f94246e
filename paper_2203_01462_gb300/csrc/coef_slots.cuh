// Per-context material coefficients in constant memory.
//
// Each context owns one slot of COEF_SLOTS; the host writes the slot (stream
// ordered) before a forward or adjoint pass and the step kernels take only
// the slot index.  A captured CUDA graph of a whole pass therefore stays
// valid when the damping level or the design changes, and the kernels still
// read every coefficient from the constant bank.  Included by each step-kernel
// translation unit, which gets its own copy of the arrays (internal linkage).
#pragma once

#include "fdtd_internal.h"

namespace fdtd {
namespace {

__constant__ Coef<float> c_coef_f[COEF_SLOTS];
__constant__ Coef<double> c_coef_d[COEF_SLOTS];

template <typename R>
__device__ __forceinline__ const Coef<R> &coef_at(int slot);
template <>
__device__ __forceinline__ const Coef<float> &coef_at<float>(int slot)
{
    return c_coef_f[slot];
}
template <>
__device__ __forceinline__ const Coef<double> &coef_at<double>(int slot)
{
    return c_coef_d[slot];
}

inline cudaError_t write_coef_slot(int slot, const Coef<float> &c, cudaStream_t st)
{
    return cudaMemcpyToSymbolAsync(c_coef_f, &c, sizeof c, (size_t)slot * sizeof c, cudaMemcpyHostToDevice, st);
}
inline cudaError_t write_coef_slot(int slot, const Coef<double> &c, cudaStream_t st)
{
    return cudaMemcpyToSymbolAsync(c_coef_d, &c, sizeof c, (size_t)slot * sizeof c, cudaMemcpyHostToDevice, st);
}

}  // namespace
}  // namespace fdtd
