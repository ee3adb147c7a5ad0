// Plain method frame (dense NeRF volume rendering of every culled pair).
#include "render_launch.h"

namespace nedf {

cudaError_t launch_march_frame(const Workspace &, const HostCamera *, int, int, int, int, int, float4 *, int,
                               cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace nedf
