// The paper's intersection network on CUDA cores in FP32 (Section "Intersection network", Eq. 3-4,
// Appendix A): the reference-precision counterpart of the tensor-core engine k_nedfc, selected by
// precision NEDF_PREC_FP32 with nedf_arch NEDF_ARCH_CLASSIFIER, so that whole frames of the
// classifier can be checked against the FP64 oracle at FP32 tolerance.
//
// It works on the same tiles as the engine (256 rows of one type's pair list, or of the caller's
// queries), 64 rows at a time, and writes the same (m, a) per pair, so the decode, fallback and
// z-min that follow are shared.  Per 64-row sub-tile: the 16 chord points encoded one at a time
// (63 features each) and accumulated into the head's 256 outputs; 16 residual blocks h' =
// ReLU(h + W2 ReLU(W1 h + b1) + b2) with h and the first layer's output in shared memory; the two
// tails into 193 logits; the first maximum of the coarse and of the fine logits gives m (Eq. 4).
// Each of the 256 threads owns an 8 x 8 block of outputs (rows 8 ty .. 8 ty + 7, columns tx + 32 j)
// and reads the layer's weights transposed (input-major), so a warp's weight loads for one input
// are 8 coalesced 128-byte rows, shared through L1 by the 8 warps of the block.
#include "pipe_common.cuh"
#include "render_launch.h"
#include "mlp_f32.cuh"

namespace nedf {

namespace {

constexpr int W = 256, NC = 64, NF = 128, NOUT = 1 + NC + NF, NBLK = 16, NPT = 16, NFEAT = 63;
constexpr int kRows = 64, kThreads = 256, kXLd = 64;
// packed FP32 master layout (W[out][in] then b[out] per layer)
constexpr long long kHeadW = (long long)kClsIn * W;
constexpr long long kBlock0 = kHeadW + W;
constexpr long long kLayer = (long long)W * W + W;
constexpr long long kTailA = kBlock0 + 2LL * NBLK * kLayer;
constexpr long long kTailB = kTailA + (long long)(1 + NC) * (W + 1);
// transposed blob (floats): head Wt[1008][256], b[256]; 32 body layers Wt[256][256], b[256]; the
// tail Wt[256][256] (outputs 0: hit logit, 1..64 coarse, 65..192 fine, zero beyond), b[256]
constexpr long long kTHead = (long long)kClsIn * W + W;
constexpr long long kTLayer = (long long)W * W + W;
constexpr long long kTTail = kTHead + 2LL * NBLK * kTLayer;
constexpr long long kTFloats = kTTail + kTLayer;
constexpr size_t kSmem = (size_t)(2 * kRows * W + kRows * kXLd) * sizeof(float);

__global__ void k_pack_cls_f32(const float *w, float *out)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < kTFloats; e += (long long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (e < kTHead) {
            const long long q = e;
            if (q < (long long)kClsIn * W) v = w[(q % W) * kClsIn + q / W];   // Wt[i][o] = W[o][i]
            else v = w[kHeadW + (q - (long long)kClsIn * W)];
        } else if (e < kTTail) {
            const long long q = e - kTHead, layer = q / kTLayer, k = q % kTLayer;
            const float *L = w + kBlock0 + layer * kLayer;
            v = k < (long long)W * W ? L[(k % W) * W + k / W] : L[(long long)W * W + (k - (long long)W * W)];
        } else {
            const long long k = e - kTTail;
            if (k < (long long)W * W) {
                const long long i = k / W, o = k % W;
                if (o < 1 + NC) v = w[kTailA + o * W + i];
                else if (o < NOUT) v = w[kTailB + (o - 1 - NC) * W + i];
            } else {
                const long long o = k - (long long)W * W;
                if (o < 1 + NC) v = w[kTailA + (long long)(1 + NC) * W + o];
                else if (o < NOUT) v = w[kTailB + (long long)NF * W + (o - 1 - NC)];
            }
        }
        out[e] = v;
    }
}

// acc[i][j] += sum_k in[8 ty + i][k] * Wt[k][tx + 32 j] over k < K (in: shared, leading dimension ld)
__device__ __forceinline__ void layer_acc(float (&acc)[8][8], const float *in, int ld, const float *Wt, int K, int ty, int tx)
{
    const float *a0 = in + (size_t)(8 * ty) * ld;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        float wv[8], av[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) wv[j] = __ldg(Wt + (size_t)k * W + tx + 32 * j);
#pragma unroll
        for (int i = 0; i < 8; ++i) av[i] = a0[(size_t)i * ld + k];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
    }
}

__device__ __forceinline__ void zero(float (&acc)[8][8])
{
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_nedfc_f32(Workspace ws, PipeArgs a)
{
    extern __shared__ float cf_smem[];
    float *H = cf_smem;                      // [64][256] the residual stream
    float *Tb = H + kRows * W;               // [64][256] a block's first-layer output, then the logits
    float *X = Tb + kRows * W;               // [64][64] one encoded chord point per row
    __shared__ float s_pe[kRows][3], s_stp[kRows][3];
    __shared__ unsigned long long s_idx[kRows];
    __shared__ int s_valid[kRows], s_kept[kRows];
    __shared__ float s_tp[kRows];
    const MarchBuffers none{};
    const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
    const unsigned long long n_tiles = pipe_n_tiles<kPipeRows, MODE>(ws, none, a);
    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int t = pipe_tile_type<MODE>(ws, none, a, tile);
        const DevType T = ws.types[t];
        const float *Wb = reinterpret_cast<const float *>(a.blobs + (size_t)t * a.blob_stride);
        for (int sub = 0; sub < kPipeRows / kRows; ++sub) {
            int any = 0;
            if (tid < kRows) {
                unsigned long long idx;
                bool valid;
                PairRay pr{};
                nedf_row<MODE>(ws, a, T, t, tile, sub * kRows + tid, idx, valid, pr);
                s_idx[tid] = idx;
                s_valid[tid] = valid;
                s_kept[tid] = valid && pr.kept;
                s_tp[tid] = pr.tp;
                // 16 points uniform over the chord [t_e, t_x] (reading 23), t_x = 2 t_perp - t_e
                const float te = pr.te, span = 2.0f * (pr.tp - pr.te);
                s_pe[tid][0] = pr.ol.x + te * pr.dl.x;
                s_pe[tid][1] = pr.ol.y + te * pr.dl.y;
                s_pe[tid][2] = pr.ol.z + te * pr.dl.z;
                s_stp[tid][0] = span * pr.dl.x;
                s_stp[tid][1] = span * pr.dl.y;
                s_stp[tid][2] = span * pr.dl.z;
                any = valid;
            }
            if (!__syncthreads_or(any)) break;            // past the end of the type's list
            float acc[8][8];
            zero(acc);
            // head: the 16 points, 63 features each, accumulated point by point
            for (int j = 0; j < NPT; ++j) {
                const float fj = (float)j / 15.0f;
                for (int e = tid; e < kRows * NFEAT; e += kThreads) {
                    const int r = e / NFEAT, f = e - r * NFEAT;
                    float v = 0.0f;
                    if (s_kept[r]) {
                        const float xs[3] = {s_pe[r][0] + fj * s_stp[r][0], s_pe[r][1] + fj * s_stp[r][1],
                                             s_pe[r][2] + fj * s_stp[r][2]};
                        v = posenc_feature(xs, 3, 10, f);
                    }
                    X[r * kXLd + f] = v;
                }
                __syncthreads();
                layer_acc(acc, X, kXLd, Wb + (size_t)j * NFEAT * W, NFEAT, ty, tx);
                __syncthreads();
            }
            {
                const float *b = Wb + (size_t)kClsIn * W;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) H[(8 * ty + i) * W + tx + 32 * j] = acc[i][j] + __ldg(b + tx + 32 * j);
            }
            __syncthreads();
            // residual blocks
            for (int k = 0; k < NBLK; ++k) {
                const float *W1 = Wb + kTHead + 2LL * k * kTLayer, *W2 = W1 + kTLayer;
                const float *b1 = W1 + (size_t)W * W, *b2 = W2 + (size_t)W * W;
                zero(acc);
                layer_acc(acc, H, W, W1, W, ty, tx);
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        Tb[(8 * ty + i) * W + tx + 32 * j] = fmaxf(acc[i][j] + __ldg(b1 + tx + 32 * j), 0.0f);
                __syncthreads();
                zero(acc);
                layer_acc(acc, Tb, W, W2, W, ty, tx);
                // the skip sum reads the elements this thread overwrites; H as an operand was last
                // read before the barrier above
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        float &h = H[(8 * ty + i) * W + tx + 32 * j];
                        h = fmaxf(h + acc[i][j] + __ldg(b2 + tx + 32 * j), 0.0f);
                    }
                __syncthreads();
            }
            // tails: 193 logits (hit, 64 coarse, 128 fine) into Tb
            zero(acc);
            layer_acc(acc, H, W, Wb + kTTail, W, ty, tx);
            {
                const float *b = Wb + kTTail + (size_t)W * W;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) Tb[(8 * ty + i) * W + tx + 32 * j] = acc[i][j] + __ldg(b + tx + 32 * j);
            }
            __syncthreads();
            // Eq. 4: the first maximum of the coarse and of the fine logits
            if (tid < kRows && s_valid[tid]) {
                const float *l = Tb + (size_t)tid * W;
                float bc = -INFINITY, bf = -INFINITY;
                int ic = 0, jf = 0;
                for (int c = 0; c < NC; ++c)
                    if (l[1 + c] > bc) { bc = l[1 + c]; ic = c; }
                for (int c = 0; c < NF; ++c)
                    if (l[1 + NC + c] > bf) { bf = l[1 + NC + c]; jf = c; }
                const float m_out = (float)(ic * NF + jf) * (1.0f / (NC * NF / 2)) - 1.0f, a_out = l[0];
                const unsigned long long idx = s_idx[tid];
                if (MODE == kModeQuery) {
                    float4 res = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
                    if (s_kept[tid]) {
                        const float Dl = s_tp[tid] - T.rb * m_out;
                        res = make_float4(m_out, a_out, Dl, (a_out > 0.f && Dl > 0.f) ? 1.f : 0.f);
                    }
                    a.qout[idx] = res;
                } else {
                    ws.nout[MODE == kModeShadow ? 1 : 0][idx] = make_float2(m_out, a_out);
                }
            }
            __syncthreads();
        }
    }
}

template <int MODE>
cudaError_t launch_mode(const Workspace &ws, const PipeArgs &a, int grid, cudaStream_t st)
{
    if (grid < 1) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_nedfc_f32<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    k_nedfc_f32<MODE><<<grid, kThreads, kSmem, st>>>(ws, a);
    return cudaGetLastError();
}

}  // namespace

size_t cls_f32_blob_size() { return ((size_t)kTFloats * sizeof(float) + 1023) & ~(size_t)1023; }

cudaError_t launch_pack_cls_f32(const float *master, void *blob, cudaStream_t st)
{
    k_pack_cls_f32<<<1024, 256, 0, st>>>(master, reinterpret_cast<float *>(blob));
    return cudaGetLastError();
}

cudaError_t launch_cls_f32(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out, int n,
                           int num_sms, cudaStream_t st)
{
    PipeArgs a{};
    a.blobs = ws.nedf_tc;
    a.blob_stride = ws.nedf_tc_stride;
    a.query_type = type;
    a.qo = o;
    a.qd = d;
    a.qout = reinterpret_cast<float4 *>(out);
    a.qn = n;
    if (mode == 0) return launch_mode<kModePrimary>(ws, a, num_sms, st);
    if (mode == 1) return launch_mode<kModeShadow>(ws, a, num_sms, st);
    const int grid = (int)std::min<long long>(num_sms, ((long long)n + kPipeRows - 1) / kPipeRows);
    return launch_mode<kModeQuery>(ws, a, grid, st);
}

}  // namespace nedf
