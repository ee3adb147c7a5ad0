// Learned part on the tensor cores: BF16 NeDF training with FP32 accumulation, FP32 master weights
// and Adam (Section "Intersection network": supervision of F_Phi through Eq. 2 and Eq. 5; the
// regression form of Eq. 6; "Training details": Adam).
//
// A step on a batch of B rows, width W, L hidden layers (all products tcgen05 GEMMs, tc_gemm.cuh):
//   encode    X0[b] = BF16(gamma([p_e, d])) (78 features, 2 zero pads)              CUDA cores
//   forward   H_{l+1} = BF16(ReLU(H_l Wb_l^T + b_l)),  l = 0 .. L-1                   M = B, N = W
//   loss      y = W_out H_L + b_out (FP32), the loss of Eq. 6 (regression form), dy,
//             dZ_{L-1} = BF16((W_out^T dy) * [H_L > 0]), and dW_out, db_out per split  CUDA cores
//   backward  dZ_{l-1} = BF16((dZ_l Wb_l) * [H_l > 0]),  l = L-1 .. 1                 M = B, N = W
//   weights   [dW_l | db_l] = dZ_l^T [H_l | 1]  (split-K over the batch, all layers in one launch)
//   then the split partials are summed in a fixed order and Adam updates the FP32 master.
// Activations and error signals are BF16 operands (reading 29 of the oracle: the error signal of a
// hidden layer is rounded to BF16 where it enters a product); every sum is FP32.  The split sums
// keep a step deterministic, so a resumed run repeats an uninterrupted one bit for bit.
#include <algorithm>
#include <cmath>

#include "mlp_f32.cuh"
#include "tc_gemm.cuh"
#include "train_launch.h"
#include "train_tc.cuh"

namespace nedf {

using tcg::Operand;

constexpr int kTcSplitRows = 1024;       // batch rows per weight-gradient split (a multiple of 64)
constexpr int kTcStagesRow = 2;          // row GEMMs (K = 80 or W: at most two 64-deep blocks)
constexpr int kTcStagesWgrad = 3;        // weight gradients (K = the split's rows)

// ---- scratch ----------------------------------------------------------------------------------
struct TcTrainScratch {
    __nv_bfloat16 *x0;           // [B][80]
    __nv_bfloat16 *h[17];        // h[l]: [B][W], l = 1 .. L
    __nv_bfloat16 *dz[16];       // dz[l]: [B][W], l = 0 .. L-1
    __nv_bfloat16 *wb;           // BF16 weights: layer 0 [W][80], layers 1 .. L-1 [W][W], output [2][W]
    float *dy;                   // [B][2]
    float *grad;                 // [n_params]
    trn::WgradJob *jobs;         // the weight-gradient tiles (device copy)
    float *partial;              // [splits][n_params]
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__host__ __device__ __forceinline__ long long wb_elems(int L, int W) { return (long long)W * kNedfInPad + (long long)(L - 1) * W * W + 2LL * W; }

size_t train_tc_scratch_bytes(int batch, int hidden, int width, long long n_params)
{
    const size_t B = (size_t)batch, splits = (B + kTcSplitRows - 1) / kTcSplitRows;
    size_t bytes = align256(B * kNedfInPad * 2) + 2 * (size_t)hidden * align256(B * width * 2) +
                   align256((size_t)wb_elems(hidden, width) * 2) + align256(B * 2 * 4) + align256(n_params * 4) +
                   align256(sizeof(trn::WgradJob) * 16) + splits * (size_t)n_params * 4;
    return bytes + 256;
}

static TcTrainScratch carve_tc(void *base, int B, int L, int W, long long n_params)
{
    TcTrainScratch s{};
    uint8_t *p = reinterpret_cast<uint8_t *>(align256(reinterpret_cast<size_t>(base)));
    s.x0 = reinterpret_cast<__nv_bfloat16 *>(p); p += align256((size_t)B * kNedfInPad * 2);
    for (int l = 1; l <= L; ++l) { s.h[l] = reinterpret_cast<__nv_bfloat16 *>(p); p += align256((size_t)B * W * 2); }
    for (int l = 0; l < L; ++l) { s.dz[l] = reinterpret_cast<__nv_bfloat16 *>(p); p += align256((size_t)B * W * 2); }
    s.wb = reinterpret_cast<__nv_bfloat16 *>(p); p += align256((size_t)wb_elems(L, W) * 2);
    s.dy = reinterpret_cast<float *>(p); p += align256((size_t)B * 2 * 4);
    s.grad = reinterpret_cast<float *>(p); p += align256((size_t)n_params * 4);
    s.jobs = reinterpret_cast<trn::WgradJob *>(p); p += align256(sizeof(trn::WgradJob) * 16);
    s.partial = reinterpret_cast<float *>(p);
    return s;
}

// offset of layer l's weights in the packed layout (W[out][in] then b[out] per layer)
__host__ __device__ __forceinline__ long long packed_off(int l, int W)
{
    return l == 0 ? 0 : (long long)kNedfIn * W + W + (long long)(l - 1) * (W * W + W);
}
// offset of layer l's BF16 weights in wb
__host__ __device__ __forceinline__ long long wb_off(int l, int W)
{
    return l == 0 ? 0 : (long long)W * kNedfInPad + (long long)(l - 1) * W * W;
}

// ---- BF16 weights from the FP32 master ----------------------------------------------------------
__global__ void k_tc_pack_weights(const float *master, __nv_bfloat16 *wb, int L, int W)
{
    const long long n = wb_elems(L, W);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (e < (long long)W * kNedfInPad) {                        // layer 0, padded to 80 inputs
            const int o = (int)(e / kNedfInPad), i = (int)(e % kNedfInPad);
            v = i < kNedfIn ? master[(long long)o * kNedfIn + i] : 0.0f;
        } else {
            long long r = e - (long long)W * kNedfInPad;
            const long long hid = (long long)(L - 1) * W * W;
            if (r < hid) {
                const int l = 1 + (int)(r / ((long long)W * W));
                v = master[packed_off(l, W) + r % ((long long)W * W)];
            } else {
                v = master[packed_off(L, W) + (r - hid)];            // output layer [2][W]
            }
        }
        wb[e] = __float2bfloat16_rn(v);
    }
}

// ---- encoding ------------------------------------------------------------------------------------
__global__ void k_tc_encode(float rb, const float *o, const float *d, long long start, long long n, int B,
                            __nv_bfloat16 *x0, float *loss_hits, const float *hit_star)
{
    float hits = 0.0f;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
        const long long i = (start + b) % n;
        const V3 ol = v3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        const V3 dl = normalized(v3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
        Chord ch;
        float x6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (bound_chord(ol, dl, rb, ch)) {
            const V3 pe = madd(ol, ch.te, dl);
            x6[0] = pe.x; x6[1] = pe.y; x6[2] = pe.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
        }
        uint32_t pk[kNedfInPad / 2];
        for (int f = 0; f < kNedfInPad; f += 2) {
            const float a = f < kNedfIn ? posenc_feature(x6, 6, 6, f) : 0.0f;
            const float c = f + 1 < kNedfIn ? posenc_feature(x6, 6, 6, f + 1) : 0.0f;
            pk[f / 2] = tc::pack_bf16(a, c);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(x0 + b * kNedfInPad);
        for (int q = 0; q < kNedfInPad / 8; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        hits += hit_star[i];
    }
    for (int off = 16; off; off >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, off);
    if ((threadIdx.x & 31) == 0 && hits != 0.0f) atomicAdd(loss_hits, hits);
}

// ---- loss, output layer, first error signal ----------------------------------------------------
// One thread per row: y = W_out h_L + b_out with the BF16 output weights, the loss terms and
// dL/dy, and dZ_{L-1} = BF16((W_out^T dy) * [h_L > 0]).
template <int W>
__global__ void k_tc_loss(const __nv_bfloat16 *hL, const __nv_bfloat16 *wout, const float *bout, const float *o,
                          const float *d, const float *m_star, const float *hit_star, float rb, long long start,
                          long long n, int B, float *dy, __nv_bfloat16 *dz, float *loss)
{
    __shared__ float wsm[2][W];
    __shared__ float red[32];
    for (int k = threadIdx.x; k < 2 * W; k += blockDim.x) wsm[k / W][k % W] = __bfloat162float(wout[k]);
    __syncthreads();
    const float n_hit = loss[1];
    float part = 0.0f;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < B; b += (long long)gridDim.x * blockDim.x) {
        const long long i = (start + b) % n;
        const V3 ol = v3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
        const V3 dl = normalized(v3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
        Chord ch;
        const bool kept = bound_chord(ol, dl, rb, ch);
        const uint4 *hrow = reinterpret_cast<const uint4 *>(hL + (size_t)b * W);
        float y0 = bout[0], y1 = bout[1];
        for (int q = 0; q < W / 8; ++q) {
            const uint4 hv = hrow[q];
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
            for (int j = 0; j < 4; ++j) {
                const float a = __uint_as_float(hw[j] << 16), c = __uint_as_float(hw[j] & 0xFFFF0000u);
                const int k = 8 * q + 2 * j;
                y0 = fmaf(wsm[0][k], a, fmaf(wsm[0][k + 1], c, y0));
                y1 = fmaf(wsm[1][k], a, fmaf(wsm[1][k + 1], c, y1));
            }
        }
        float dm = 0.0f, da = 0.0f;
        if (kept) {
            const float al = hit_star[i];
            const float bce = fmaxf(y1, 0.0f) - al * y1 + log1pf(expf(-fabsf(y1)));
            part += 0.1f * bce / (float)B;
            if (al > 0.5f) {
                const float e = y0 - m_star[i];
                part += e * e / n_hit;
                dm = 2.0f * e / n_hit;
            }
            da = 0.1f * (1.0f / (1.0f + expf(-y1)) - al) / (float)B;
        }
        dy[2 * b] = dm;
        dy[2 * b + 1] = da;
        uint4 *dst = reinterpret_cast<uint4 *>(dz + (size_t)b * W);
        for (int q = 0; q < W / 8; ++q) {
            const uint4 hv = hrow[q];
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
            uint32_t pk[4];
            for (int j = 0; j < 4; ++j) {
                const int k = 8 * q + 2 * j;
                const float g0 = (hw[j] & 0xFFFFu) != 0u && !(hw[j] & 0x8000u) ? wsm[0][k] * dm + wsm[1][k] * da : 0.0f;
                const float g1 = (hw[j] >> 16) != 0u && !(hw[j] & 0x80000000u) ? wsm[0][k + 1] * dm + wsm[1][k + 1] * da
                                                                                 : 0.0f;
                pk[j] = tc::pack_bf16(g0, g1);
            }
            dst[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
    for (int off = 16; off; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(&loss[0], t);
    }
}

// Output-layer gradient of one split (blockIdx.x) and 32 of the W columns (blockIdx.y):
// dW_out[o][k] = sum_b dy[b][o] h_L[b][k] and (column block 0) db_out[o] = sum_b dy[b][o] over the
// split's rows into the split's partial.  Warp w sums rows w, w + 8, ... of the split (lane = column),
// then the eight warps are added in order: a fixed summation order, deterministic.
template <int W>
__global__ void __launch_bounds__(256) k_tc_out_grad(const __nv_bfloat16 *hL, const float *dy, int B, int rows_per_split,
                                                     float *partial, long long split_stride, long long off)
{
    __shared__ float red[8][2][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r0 = blockIdx.x * rows_per_split, r1 = min(B, r0 + rows_per_split);
    const int c = blockIdx.y * 32 + lane;
    float a0 = 0.0f, a1 = 0.0f, s0 = 0.0f, s1 = 0.0f;
    for (int b = r0 + warp; b < r1; b += 8) {
        const float2 g = *reinterpret_cast<const float2 *>(dy + 2 * (size_t)b);
        const float h = __bfloat162float(hL[(size_t)b * W + c]);
        a0 = fmaf(g.x, h, a0);
        a1 = fmaf(g.y, h, a1);
        s0 += g.x;
        s1 += g.y;
    }
    red[warp][0][lane] = a0;
    red[warp][1][lane] = a1;
    if (lane == 0) { red[warp][0][32] = s0; red[warp][1][32] = s1; }
    __syncthreads();
    float *p = partial + blockIdx.x * split_stride + off;
    if (threadIdx.x < 64) {
        const int o = threadIdx.x >> 5, l = threadIdx.x & 31;
        float acc = 0.0f;
        for (int w = 0; w < 8; ++w) acc += red[w][o][l];
        p[(long long)o * W + blockIdx.y * 32 + l] = acc;
    } else if (threadIdx.x < 66 && blockIdx.y == 0) {
        const int o = threadIdx.x - 64;
        float acc = 0.0f;
        for (int w = 0; w < 8; ++w) acc += red[w][o][32];
        p[2LL * W + o] = acc;
    }
}

namespace trn {
__global__ void k_sum_splits(const float *partial, int splits, long long n, float *grad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int z = 0; z < splits; ++z) acc += partial[(size_t)z * n + i];
        grad[i] = acc;
    }
}
}  // namespace trn

// ---- one forward / backward pass ----------------------------------------------------------------
template <int W>
static cudaError_t run_tc(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                          const float *hit_star, long long start, long long n, int B, TcTrainScratch s)
{
    cudaStream_t st = L.stream;
    const int nl = L.hidden;
    uint32_t *status = L.status;
    const uint32_t flag = kStatusTimeout;
    cudaError_t e = cudaMemsetAsync(L.loss, 0, sizeof(float) * 4, st);
    if (e != cudaSuccess) return e;
#define CK_(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    k_tc_pack_weights<<<L.num_sms * 2, 256, 0, st>>>(L.master, s.wb, nl, W);
    const int eb = (int)std::min<long long>((B + 255) / 256, (long long)L.num_sms * 8);
    k_tc_encode<<<eb, 256, 0, st>>>(L.rb, o, d, start, n, B, s.x0, L.loss + 1, hit_star);
    // forward: H_{l+1} = BF16(ReLU(H_l Wb_l^T + b_l))
    for (int l = 0; l < nl; ++l) {
        const int fi = l == 0 ? kNedfInPad : W;
        const Operand A{l == 0 ? s.x0 : s.h[l], fi, B, fi, tcg::kKMajor, -1};
        const Operand Bw{s.wb + wb_off(l, W), fi, W, fi, tcg::kKMajor, -1};
        const float *bias = L.master + packed_off(l, W) + (long long)(l == 0 ? kNedfIn : W) * W;
        CK_((trn::rows_gemm<W, kTcStagesRow>(A, Bw, B, fi, trn::EpiForward<true, false>{s.h[l + 1], bias, nullptr, B, W, W},
                                             status, flag, st)));
    }
    // loss, dy, first error signal
    k_tc_loss<W><<<eb, 256, 0, st>>>(s.h[nl], s.wb + wb_off(nl, W), L.master + packed_off(nl, W) + 2LL * W, o, d, m_star,
                                     hit_star, L.rb, start, n, B, s.dy, s.dz[nl - 1], L.loss);
    // backward through the hidden layers: dZ_{l-1} = BF16((dZ_l Wb_l) * [H_l > 0])
    for (int l = nl - 1; l >= 1; --l) {
        const Operand A{s.dz[l], W, B, W, tcg::kKMajor, -1};
        const Operand Bw{s.wb + wb_off(l, W), W, W, W, tcg::kMNMajor, -1};       // element (i, o) = W_l[o][i]
        CK_((trn::rows_gemm<W, kTcStagesRow>(A, Bw, B, W, trn::EpiBackward<false>{s.dz[l - 1], s.h[l], nullptr, B, W, W},
                                             status, flag, st)));
    }
    // weight and bias gradients of every hidden layer, split over the batch, one launch: per layer
    // one tile [dW | db] = dZ^T [H | 1], the ones row after the layer's inputs
    trn::WgradJob jobs[16];
    for (int l = 0; l < nl; ++l) {
        const int fi = l == 0 ? kNedfIn : W, fip = l == 0 ? kNedfInPad : W;
        trn::WgradJob j{};
        j.a = Operand{s.dz[l], W, W, B, tcg::kMNMajor, -1};                      // (o, b) = dZ_l[b][o]
        j.b = Operand{l == 0 ? s.x0 : s.h[l], fip, fip, B, tcg::kMNMajor, fip};  // (i, b) = H_l[b][i]; row fip = 1
        j.m0 = 0; j.n0 = 0; j.c_lo = 0; j.c_hi = fi; j.fo = W; j.fi = fi; j.ones = fip; j.seg_split = W;
        j.w_off[0] = packed_off(l, W); j.b_off[0] = packed_off(l, W) + (long long)fi * W;
        jobs[l] = j;
    }
    CK_(cudaMemcpyAsync(s.jobs, jobs, sizeof(trn::WgradJob) * nl, cudaMemcpyHostToDevice, st));
    // the widest B operand: 80 inputs of layer 0 or W, then the 8-row group of the ones row
    constexpr int BN = (W > kNedfInPad ? W : kNedfInPad) + 16;
    CK_((trn::wgrad<BN, kTcStagesWgrad>(s.jobs, nl, B, kTcSplitRows, s.partial, L.n_params, status, flag, st)));
    const int splits = (B + kTcSplitRows - 1) / kTcSplitRows;
    k_tc_out_grad<W><<<dim3(splits, W / 32), 256, 0, st>>>(s.h[nl], s.dy, B, kTcSplitRows, s.partial, L.n_params,
                                                            packed_off(nl, W));
    trn::k_sum_splits<<<(int)std::min<long long>((L.n_params + 255) / 256, (long long)L.num_sms * 8), 256, 0, st>>>(
        s.partial, splits, L.n_params, s.grad);
#undef CK_
    return cudaGetLastError();
}

static cudaError_t tc_fwd_bwd(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                              const float *hit_star, long long start, long long n, int B, TcTrainScratch s)
{
    switch (L.width) {
    case 64: return run_tc<64>(L, o, d, m_star, hit_star, start, n, B, s);
    case 128: return run_tc<128>(L, o, d, m_star, hit_star, start, n, B, s);
    default: return cudaErrorInvalidValue;
    }
}

bool train_tc_supported(int width, int hidden) { return (width == 64 || width == 128) && hidden >= 1 && hidden <= 16; }

cudaError_t launch_loss_grad_tc(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                                const float *hit_star, int n, float *grad)
{
    TcTrainScratch s = carve_tc(L.scratch, n, L.hidden, L.width, L.n_params);
    cudaError_t e = tc_fwd_bwd(L, o, d, m_star, hit_star, 0, n, n, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(grad, s.grad, sizeof(float) * L.n_params, cudaMemcpyDeviceToDevice, L.stream);
}

cudaError_t launch_train_step_tc(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                                 const float *hit_star, long long n_rays, long long start, int batch, float *adam_m,
                                 float *adam_v, int step, float lr)
{
    TcTrainScratch s = carve_tc(L.scratch, batch, L.hidden, L.width, L.n_params);
    cudaError_t e = tc_fwd_bwd(L, o, d, m_star, hit_star, start, n_rays, batch, s);
    if (e != cudaSuccess) return e;
    return launch_adam(L, s.grad, adam_m, adam_v, step, lr);
}

}  // namespace nedf
