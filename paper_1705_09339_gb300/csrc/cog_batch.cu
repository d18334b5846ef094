// cog_batch.cu -- the per-step counter advance of a batch (one frame per
// stream per step), kept on the device so that a captured graph can be
// replayed without host-side parameter changes.
#include "cog_internal.h"

namespace cog {

__global__ void batch_advance_kernel(const BatchGroupDev g)
{
    asm volatile("griddepcontrol.wait;" ::: "memory");   // after the mixture stage
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < g.n && g.active[s]) {
        const uint32_t f = g.frame_no[s] + 1;
        g.frame_no[s] = f;
        g.descs[s].frame_no = f % 3;
        g.descs[s].frame_idx = f;
    }
}

cudaError_t launch_batch_advance(const BatchGroupDev &g, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cfg.stream = st;
    cfg.gridDim = dim3((unsigned)((g.n + 127) / 128));
    cfg.blockDim = dim3(128);
    return cudaLaunchKernelEx(&cfg, batch_advance_kernel, g);
}

}  // namespace cog
