// Pieces shared by the tensor-core training of both networks (train_tc.cu: the regression NeDF;
// train_cls.cu: the paper's classifier network): the GEMM epilogues of the forward and backward
// passes, the row-GEMM kernel and the weight-gradient kernel over a list of output tiles.
//
// Activations and error signals are BF16 operands, every sum FP32 (tc_gemm.cuh).  A weight
// gradient [dW | db] = dZ^T [H | 1] is split over the batch rows (fixed splits, each writing its
// own partial in the packed parameter layout), and the partials are summed in split order, so a
// training step is deterministic.
#pragma once

#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace nedf {
namespace trn {

using tcg::Operand;

// a BF16 value (raw bits in the low or high half of a word) is positive iff its sign bit is clear
// and it is not zero
__device__ __forceinline__ float pos_lo(uint32_t w) { return ((w & 0xFFFFu) != 0u && !(w & 0x8000u)) ? 1.0f : 0.0f; }
__device__ __forceinline__ float pos_hi(uint32_t w) { return ((w >> 16) != 0u && !(w & 0x80000000u)) ? 1.0f : 0.0f; }
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

__device__ __forceinline__ void store32_bf16(__nv_bfloat16 *dst, const uint32_t (&pk)[16])
{
    uint4 *d = reinterpret_cast<uint4 *>(dst);
#pragma unroll
    for (int q = 0; q < 4; ++q) d[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
}

// forward: out[row][n] = BF16(act(acc + bias[n] (+ skip[row][n]))), act = ReLU or identity
template <bool RELU, bool SKIP>
struct EpiForward {
    __nv_bfloat16 *out;
    const float *bias;
    const __nv_bfloat16 *skip;   // the block input h (SKIP)
    int M, N, ld;                // rows, valid columns, row stride (elements) of out and skip
    __device__ __forceinline__ void operator()(int row, int c0, const uint32_t (&v)[32]) const
    {
        if (row >= M || c0 >= N) return;
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(v[i]) + __ldg(bias + c0 + i);
        if (SKIP) {
            const uint4 *s = reinterpret_cast<const uint4 *>(skip + (size_t)row * ld + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 sv = s[q];
                const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    x[8 * q + 2 * j] += bf_lo(sw[j]);
                    x[8 * q + 2 * j + 1] += bf_hi(sw[j]);
                }
            }
        }
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            pk[i] = RELU ? tc::pack_bf16_relu(x[2 * i], x[2 * i + 1]) : tc::pack_bf16(x[2 * i], x[2 * i + 1]);
        store32_bf16(out + (size_t)row * ld + c0, pk);
    }
};

// FP32 outputs: out[row][n] = acc + bias[n] for n < N (the classifier's logits)
struct EpiLogits {
    float *out;
    const float *bias;
    int M, N, ld;
    __device__ __forceinline__ void operator()(int row, int c0, const uint32_t (&v)[32]) const
    {
        if (row >= M) return;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (c0 + i < N) out[(size_t)row * ld + c0 + i] = __uint_as_float(v[i]) + __ldg(bias + c0 + i);
    }
};

// backward: out[row][n] = BF16((acc (+ add[row][n])) * [mask[row][n] > 0]); no mask when mask is
// null (a linear layer's input gradient)
template <bool ADD>
struct EpiBackward {
    __nv_bfloat16 *out;
    const __nv_bfloat16 *mask;   // the layer input's activations (positive: ReLU passed)
    const __nv_bfloat16 *add;    // the skip connection's gradient (ADD)
    int M, N, ld;
    __device__ __forceinline__ void operator()(int row, int c0, const uint32_t (&v)[32]) const
    {
        if (row >= M || c0 >= N) return;
        float x[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) x[i] = __uint_as_float(v[i]);
        if (ADD) {
            const uint4 *s = reinterpret_cast<const uint4 *>(add + (size_t)row * ld + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 sv = s[q];
                const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    x[8 * q + 2 * j] += bf_lo(sw[j]);
                    x[8 * q + 2 * j + 1] += bf_hi(sw[j]);
                }
            }
        }
        if (mask) {
            const uint4 *s = reinterpret_cast<const uint4 *>(mask + (size_t)row * ld + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 sv = s[q];
                const uint32_t sw[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    x[8 * q + 2 * j] *= pos_lo(sw[j]);
                    x[8 * q + 2 * j + 1] *= pos_hi(sw[j]);
                }
            }
        }
        uint32_t pk[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) pk[i] = tc::pack_bf16(x[2 * i], x[2 * i + 1]);
        store32_bf16(out + (size_t)row * ld + c0, pk);
    }
};

template <int BN, int S, class Epi>
__global__ void __launch_bounds__(tcg::kThreads) k_rows(Operand A, Operand B, long long k_total, Epi epi, uint32_t *status,
                                                        uint32_t flag)
{
    tcg::gemm_tile<BN, S>(A, B, blockIdx.x * tcg::kBM, 0, 0, k_total, epi, status, flag);
}

// M = rows of A (batch), N = BN (one tile), all of K: one launch, one CTA per 128 rows
template <int BN, int S, class Epi>
cudaError_t rows_gemm(const Operand &A, const Operand &B, int M, long long K, const Epi &epi, uint32_t *status,
                      uint32_t flag, cudaStream_t st)
{
    using SM = tcg::GemmSmem<BN, S>;
    cudaError_t e = cudaFuncSetAttribute(k_rows<BN, S, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::BYTES);
    if (e != cudaSuccess) return e;
    k_rows<BN, S, Epi><<<(M + tcg::kBM - 1) / tcg::kBM, tcg::kThreads, SM::BYTES, st>>>(A, B, K, epi, status, flag);
    return cudaGetLastError();
}

// One output tile of a weight gradient: rows m0 .. m0 + 127 of dZ^T (output features), rows
// n0 .. n0 + BN - 1 of [H | 1] (input features, the ones row giving the bias gradient).  Columns
// [c_lo, c_hi) and the ones column of the tile are written into the split's partial: output
// feature o (< fo) of segment s (o < seg_split: s = 0, else s = 1 counting from seg_split) at
// w_off[s] + o' * fi + n and its bias at b_off[s] + o'.
struct WgradJob {
    Operand a, b;
    int m0, n0, c_lo, c_hi, fo, fi, ones, seg_split;
    long long w_off[2], b_off[2];
};

struct EpiWgrad {
    const WgradJob *job;
    float *partial;
    long long split_stride;
    // c0: the absolute first column (the tile's n0 included)
    __device__ __forceinline__ void operator()(int row, int c0, const uint32_t (&v)[32]) const
    {
        const WgradJob &J = *job;
        if (row >= J.fo) return;
        const int s = row < J.seg_split ? 0 : 1;
        const int o = s ? row - J.seg_split : row;
        float *p = partial + blockIdx.z * split_stride;                 // blockIdx.z: the split
#pragma unroll 4
        for (int i = 0; i < 32; ++i) {
            const int n = c0 + i;
            if (n >= J.c_lo && n < J.c_hi && n < J.fi) p[J.w_off[s] + (long long)o * J.fi + n] = __uint_as_float(v[i]);
            else if (n == J.ones) p[J.b_off[s] + o] = __uint_as_float(v[i]);
        }
    }
};

// blockIdx.y = job, blockIdx.z = split of the batch (rows z * split_rows ..)
template <int BN, int S>
__global__ void __launch_bounds__(tcg::kThreads) k_wgrad(const WgradJob *jobs, long long k_total, int split_rows,
                                                         float *partial, long long split_stride, uint32_t *status,
                                                         uint32_t flag)
{
    __shared__ WgradJob J;
    if (threadIdx.x == 0) J = jobs[blockIdx.y];
    __syncthreads();
    const long long kb = (long long)blockIdx.z * split_rows;
    const long long ke = kb + split_rows < k_total ? kb + split_rows : k_total;
    const EpiWgrad epi{&J, partial, split_stride};
    tcg::gemm_tile<BN, S>(J.a, J.b, J.m0, J.n0, kb, ke, epi, status, flag);
}

template <int BN, int S>
cudaError_t wgrad(const WgradJob *jobs_dev, int n_jobs, long long B, int split_rows, float *partial, long long split_stride,
                  uint32_t *status, uint32_t flag, cudaStream_t st)
{
    using SM = tcg::GemmSmem<BN, S>;
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<BN, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM::BYTES);
    if (e != cudaSuccess) return e;
    const int splits = (int)((B + split_rows - 1) / split_rows);
    k_wgrad<BN, S><<<dim3(1, n_jobs, splits), tcg::kThreads, SM::BYTES, st>>>(jobs_dev, B, split_rows, partial, split_stride,
                                                                               status, flag);
    return cudaGetLastError();
}

// grad[i] = partial[0][i] + partial[1][i] + ... in split order
__global__ void k_sum_splits(const float *partial, int splits, long long n, float *grad);

}  // namespace trn
}  // namespace nedf
