// Launch sequences of the render path, called by the C-ABI layer.
#pragma once

#include "render_kernels.cuh"

namespace nedf {

struct FrameLaunch {
    Workspace ws;
    cudaStream_t stream;
    int W, H;
    int num_sms;
    int n_inst;
    int n_shade;
    const HostCamera *cam;   // device copy of this frame's camera
    cudaEvent_t *events;     // NULL, or kStages + 1 events recorded between the stages
    int launches;            // out: kernels launched
};

constexpr int kStages = 8;

cudaError_t launch_frame_f32(FrameLaunch &L);
cudaError_t launch_nedf_query_f32(const Workspace &ws, int type, const float *o, const float *d,
                                  float *out, int n, int num_sms, cudaStream_t st);
cudaError_t launch_march_frame(const Workspace &ws, const HostCamera *cam, int W, int H, int n_inst,
                               int n_samples, int early_stop, float4 *rgba, int num_sms,
                               cudaStream_t st);

}  // namespace nedf
