// Launch sequences of the learned part (NeDF training), called by the C-ABI layer.
#pragma once

#include "nedf_device.cuh"

namespace nedf {

struct TrainLaunch {
    const DevType *type;     // device record of the type being trained
    float rb;
    int hidden, width;
    long long n_params;
    float *master;           // packed FP32 weights, W[out][in] then b per layer
    float *kernel_w;         // the renderer's copy (per layer Wt[in][out] then b)
    float *scratch;          // activations, deltas, gradient (train_scratch_bytes)
    float *loss;             // device float[4]: loss, hit count, row count
    uint32_t *status;        // device status word (bounded waits of the tensor-core path)
    int num_sms;
    cudaStream_t stream;
};

size_t train_scratch_bytes(int batch, int hidden, int width, long long n_params);

// Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected) on the master weights with the given gradient;
// the renderer's FP32 copy is rewritten in the same pass.
cudaError_t launch_adam(const TrainLaunch &L, const float *grad, float *adam_m, float *adam_v, int step, float lr);

// The same step with BF16 operands on the tensor cores (train_tc.cu), widths 64 and 128: products
// in tcgen05 GEMMs with FP32 accumulation, FP32 master weights and Adam.
bool train_tc_supported(int width, int hidden);
size_t train_tc_scratch_bytes(int batch, int hidden, int width, long long n_params);
cudaError_t launch_loss_grad_tc(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                                const float *hit_star, int n, float *grad);
cudaError_t launch_train_step_tc(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                                 const float *hit_star, long long n_rays, long long start, int batch, float *adam_m,
                                 float *adam_v, int step, float lr);

cudaError_t launch_make_labels(const DevType *type, float rb, long long n_rays, uint64_t seed, int steps,
                               int bisect, float *o, float *d, float *m_star, float *hit_star, int num_sms,
                               cudaStream_t st);

// The same rays labelled by a density network [63, width x hidden, 1] (kernel layout: per layer
// Wt[in][out] then b; width 64 or 128) through Eq. 5 over n_samples chord midpoints (<= 1024).
constexpr int kDensIn = 63;
constexpr int kMaxDensSamples = 1024;
cudaError_t launch_density_labels(const float *wk, int hidden, int width, float rb, long long n_rays, uint64_t seed,
                                  int n_samples, float *o, float *d, float *m_star, float *hit_star, int num_sms,
                                  cudaStream_t st);

// Loss and gradient on rows [0, n) of (o, d, m_star, hit_star); gradient written to grad (packed).
cudaError_t launch_loss_grad(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                             const float *hit_star, int n, float *grad);

// One Adam step on rows start .. start+batch-1 (mod n_rays) of the training set.
cudaError_t launch_train_step(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                              const float *hit_star, long long n_rays, long long start, int batch,
                              float *adam_m, float *adam_v, int step, float lr);

// The paper's classifier network (train_cls.cu): Eq. 6 and its gradient by hand, the dense
// products as BF16 tcgen05 GEMMs with FP32 accumulation, Adam; the scratch holds a batch's
// activations (cls_train_scratch_bytes).
struct ClsTrainLaunch {
    float rb;
    float *master;           // packed FP32 weights (head, 16 x (W1, b1, W2, b2), tail A, tail B)
    float *scratch;
    float *loss;             // device float[4]: loss, hit rows
    uint32_t *status;        // device status word (bounded waits)
    int num_sms;
    cudaStream_t stream;
};
size_t cls_train_scratch_bytes(long long batch);
cudaError_t launch_cls_loss_grad(const ClsTrainLaunch &L, const float *o, const float *d, const float *m_star,
                                 const float *hit_star, int n, float *grad);
cudaError_t launch_cls_train_step(const ClsTrainLaunch &L, const float *o, const float *d, const float *m_star,
                                  const float *hit_star, long long n_rays, long long start, int batch, float *adam_m,
                                  float *adam_v, int step, float lr);

// Re-derives the renderer's copy of the weights from the master weights.
cudaError_t launch_refresh_weights(const TrainLaunch &L);

}  // namespace nedf
