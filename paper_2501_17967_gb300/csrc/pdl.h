// Programmatic dependent launch for the kernels of one apply.
//
// Every kernel of the library is launched with the programmatic stream
// serialisation attribute, so the GPU schedules the next kernel of the stream
// while the current one drains instead of after it has fully retired; and
// every kernel calls griddep_wait() before it touches global memory, which
// returns once the preceding kernel of the stream has completed and its writes
// are visible.  Because every kernel waits, the order is transitive: a kernel
// also sees everything written by the kernels before its predecessor.
// griddep_launch_dependents() lets the next kernel's CTAs start their own
// set-up (shared memory, tensor memory, barriers) before this one ends.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace bc {

__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace bc
