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
    int n_lights;
    int shade_resample;      // Step-2 outlier resampling: plain-method samples per pair (0 = off)
    int edit_mode;           // buffer reuse: 0 a whole frame, 1 the frozen part, 2 an edit frame
    const HostCamera *cam;   // device copy of this frame's camera
    cudaEvent_t *events;     // NULL, or kStages + 1 events recorded between the stages
    cudaEvent_t *engine_events;   // with events: 4 more, around the Step-1 and Step-3 NeDF engine launches
    bool engines_timed;      // out: the engine events were recorded
    int launches;            // out: kernels launched
};

constexpr int kStages = 8;
constexpr int kLightGridSize = 128;   // shadow-map camera grid (cells per side)

cudaError_t launch_frame(FrameLaunch &L);

// Tensor-core engine (render_pipe.cu): tiles of 256 rows, weight chunks streamed per layer; f8:
// hidden layers after the first in E4M3 with per-layer scales
constexpr int kPipeTileRows = 256;
size_t pipe_blob_size(int K0, int N, int L, int n_out, bool f8);
// pair: the SM-pair engine's layout (width 256 only; see k_pack_pipe)
cudaError_t launch_pack_pipe(const float *master, void *blob, int K_in, int K0, int N, int L, int n_out, bool f8,
                             bool pair, cudaStream_t st);
// mode 0: Step-1 pairs, 1: Step-3 pairs, 2: n caller rays (o, d) of `type` -> out float4[n]
cudaError_t launch_nedf_pipe(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out,
                             int n, int num_sms, cudaStream_t st);
cudaError_t launch_shade_pipe(const Workspace &ws, int npix, int num_sms, cudaStream_t st);
// The SM-pair NeRF engine (render_pair.cu), width 256: mode kModeShade or kModeMarch (pipe_common.cuh);
// cudaErrorInvalidConfiguration (nothing launched) when its shape does not fit
struct PipeArgs;
cudaError_t launch_pair_pipe(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a, int mode, int num_sms,
                             cudaStream_t st);
// The paper's classifier intersection network (render_cls.cu): packed FP32 master weights (head
// 1008 -> 256, 16 residual blocks, tails 256 -> 65 and 256 -> 128) -> per-type BF16 blob; the
// engine in the same three modes as launch_nedf_pipe, writing the same (m, a) outputs
constexpr int kClsIn = 1008;
constexpr long long kClsParams = 2413249;
size_t cls_blob_size();
cudaError_t launch_pack_cls(const float *master, void *blob, cudaStream_t st);
cudaError_t launch_cls_pipe(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out,
                            int n, int num_sms, cudaStream_t st);
// The same network on CUDA cores in FP32 (render_cls_f32.cu): per-type transposed FP32 blob, the
// same three modes and (m, a) outputs
size_t cls_f32_blob_size();
cudaError_t launch_pack_cls_f32(const float *master, void *blob, cudaStream_t st);
cudaError_t launch_cls_f32(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out,
                           int n, int num_sms, cudaStream_t st);
cudaError_t launch_march_colour_pipe(const Workspace &ws, const MarchBuffers &mb, int n_samples, int num_sms,
                                     cudaStream_t st);
cudaError_t launch_fallback(const Workspace &ws, int mode, int num_sms, cudaStream_t st);
// Step-2 outlier resampling (march.cu): the flagged pixels re-rendered by the plain method
cudaError_t launch_shade_resample(const FrameLaunch &L);
// decode of the tensor-core engine's outputs of every listed pair (mode 0: Step 1, 1: Step 3)
cudaError_t launch_nedf_decode(const Workspace &ws, int mode, int num_sms, cudaStream_t st);
// one bounded mbarrier wait that nothing completes (sets the timeout status after its limit)
cudaError_t launch_wait_check(uint32_t *status, cudaStream_t st);

// Step-3 binning through per-light shadow-map cameras (shadow_bin.cu); its shadow-ray passes run
// shadow_bin_blocks(num_sms) blocks (Workspace::sblk holds a range per type and block)
inline int shadow_bin_blocks(int num_sms) { return num_sms * 6; }   // one wave at 6 blocks per SM
// edit_frame: buffer reuse's edit frame (the frozen pixels' shadow rays against the manipulated instance too)
cudaError_t launch_shadow_binning(const Workspace &ws, int npix, int n_lights, int n_inst, int rows_per_tile,
                                  int num_sms, cudaStream_t st, int *launches, bool edit_frame = false);
cudaError_t launch_nedf_query_f32(const Workspace &ws, int type, const float *o, const float *d,
                                  float *out, int n, int num_sms, cudaStream_t st);
cudaError_t launch_primary_binning(FrameLaunch &L);
size_t march_bytes(int npix, long long pairs, int n_samples);
cudaError_t launch_march_colour_frame(const FrameLaunch &L, void *scratch, long long pairs_cap, int n_samples,
                                      int early_stop, float4 *rgba);

}  // namespace nedf
