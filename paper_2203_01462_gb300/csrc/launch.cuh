// Kernel launch with programmatic stream serialisation (programmatic
// dependent launch): the next kernel in the stream may be scheduled while
// this one drains, and every step kernel begins with griddepcontrol.wait,
// so no state is touched before the previous grid has completed.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace fdtd {

// `win` (may be null): an L2 access-policy window attached to this launch.
template <typename... KArgs, typename... Args>
inline void launch_pdl_win(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st,
                           const cudaAccessPolicyWindow *win, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (win) {
        attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
        attr[1].val.accessPolicyWindow = *win;
        cfg.numAttrs = 2;
    }
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args)
{
    launch_pdl_win(kern, grid, block, st, nullptr, std::forward<Args>(args)...);
}

}  // namespace fdtd
