// lbm_launch.cuh -- programmatic dependent launch of the step kernels: a
// step kernel may be scheduled onto SMs that the previous step kernel has
// already left (its tail), and waits on the device, before it touches any
// memory, until that kernel has completed and its writes are visible.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace tlv {

// First statement of a kernel launched by launch_pdl: wait for the grid
// before it in the stream (returns at once when launched without the
// attribute), then allow the next grid to be scheduled.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t st,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

} // namespace tlv
