// Kernel launch with programmatic stream serialisation (programmatic
// dependent launch): the next kernel in the stream may be scheduled while
// this one drains, and every step kernel begins with griddepcontrol.wait,
// so no state is touched before the previous grid has completed.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace fdtd {

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace fdtd
