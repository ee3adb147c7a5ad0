// FP32 tile MLP on CUDA cores (reference-precision path of every network in the renderer).
#pragma once

#include "nedf_device.cuh"

namespace nedf {

constexpr int kTileRows = 64;        // rows per SIMT MLP tile
constexpr int kXStride = kTileRows + 4;
constexpr int kThreads = 256;

// ---------------------------------------------------------------------------------------------
// FP32 tile MLP on CUDA cores.  X is a feature-major tile [K][kXStride] in shared memory;
// a layer overwrites it with its N outputs.  256 threads: 16 column groups x 16 row groups,
// each thread computes 4 rows x N/16 columns.
// ---------------------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ void dense_f32(float *X, int K, const float *__restrict__ Wt,
                                          const float *__restrict__ b, bool relu)
{
    constexpr int NC = N / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        float bj = __ldg(b + tx + 16 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
    const float *xp = X + ty * 4;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        float4 xv = *reinterpret_cast<const float4 *>(xp + k * kXStride);
        const float *wr = Wt + (size_t)k * N + tx;
        float w[NC];
#pragma unroll
        for (int j = 0; j < NC; ++j) w[j] = __ldg(wr + 16 * j);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            acc[0][j] = fmaf(xv.x, w[j], acc[0][j]);
            acc[1][j] = fmaf(xv.y, w[j], acc[1][j]);
            acc[2][j] = fmaf(xv.z, w[j], acc[2][j]);
            acc[3][j] = fmaf(xv.w, w[j], acc[3][j]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            X[(tx + 16 * j) * kXStride + ty * 4 + i] = relu ? fmaxf(acc[i][j], 0.0f) : acc[i][j];
    __syncthreads();
}

template <int N>
__device__ __forceinline__ void mlp_hidden_f32(float *X, int K0, int hidden, const float *w)
{
    // layer 0: K0 -> N, then hidden-1 layers N -> N; w advanced past each (Wt, b)
    dense_f32<N>(X, K0, w, w + (size_t)K0 * N, true);
    w += (size_t)K0 * N + N;
    for (int l = 1; l < hidden; ++l) {
        dense_f32<N>(X, N, w, w + (size_t)N * N, true);
        w += (size_t)N * N + N;
    }
}

// Output layer with n_out <= 4 outputs: y[r][o] for the tile's rows.
__device__ __forceinline__ void out_layer_f32(const float *X, int K, const float *__restrict__ Wt,
                                              const float *__restrict__ b, int n_out, float (*y)[4])
{
    for (int e = threadIdx.x; e < kTileRows * n_out; e += blockDim.x) {
        int r = e / n_out, o = e - r * n_out;
        float acc = __ldg(b + o);
        for (int k = 0; k < K; ++k) acc = fmaf(X[k * kXStride + r], __ldg(Wt + k * n_out + o), acc);
        y[r][o] = acc;
    }
    __syncthreads();
}

// gamma(x) of an n-wide input with L frequencies written as features [f0, f0 + n (1 + 2L)).
__device__ __forceinline__ float posenc_feature(const float *x, int n, int L, int f)
{
    if (f < n) return x[f];
    f -= n;
    int blk = f / n, c = f - blk * n;
    if (blk < L) return sinf(ldexpf(x[c], blk));
    return cosf(ldexpf(x[c], blk - L));
}

}  // namespace nedf
