// Training of the paper's classifier intersection network (Section "Intersection network",
// Eq. 3-4 and the BCE loss of Eq. 6; "Training details": Adam) on the tensor cores.
//
// A batch of B labelled rays: the 16 encoded chord points of each (B x 1008, BF16), the forward
// pass with every block's input h, its ReLU'd first-layer output t and (through h_{k+1}) its skip
// sum's sign kept, the logits (FP32), Eq. 6's loss and its gradient with respect to the logits,
// then the backward pass by hand (ReLU masks, the skip connection, dW = delta^T input, db = column
// sums of delta, d input = delta W) and one Adam step on the packed FP32 master weights.  Every
// dense product is a tcgen05 GEMM (tc_gemm.cuh, train_tc.cuh) with BF16 operands and FP32
// accumulation: the residual stream and the error signals are BF16 between products, as in the
// BF16 inference engine; the encoding, the loss, the split sums and Adam are kernels of this file.
#include <algorithm>
#include <cmath>

#include "mlp_f32.cuh"
#include "render_launch.h"
#include "train_launch.h"
#include "train_tc.cuh"

namespace nedf {

namespace {

using trn::Operand;
using trn::WgradJob;

constexpr int W = 256, NC = 64, NF = 128, NOUT = 1 + NC + NF, NOUT_PAD = 208, NBLK = 16;
constexpr long long kHeadW = (long long)kClsIn * W;
constexpr long long kBlock0 = kHeadW + W;
constexpr long long kLayer = (long long)W * W + W;
constexpr long long kTailA = kBlock0 + 2 * NBLK * kLayer;
constexpr long long kTailB = kTailA + (long long)(1 + NC) * (W + 1);
constexpr int kClsSplitRows = 8192;      // batch rows per weight-gradient split
constexpr int kRowStages = 2, kHeadStages = 3, kWgradStages = 3;
constexpr int kJobs = 2 * 8 + NBLK * 2 * 4 + 4;
// BF16 weights: head [256][1008], then W1, W2 of each block [256][256], then the tails [208][256]
// (tail A's 65 rows, tail B's 128, 15 zero rows)
constexpr long long kWbHead = 0, kWbBlock0 = (long long)W * kClsIn;
constexpr long long kWbTail = kWbBlock0 + 2LL * NBLK * W * W;
constexpr long long kWbElems = kWbTail + (long long)NOUT_PAD * W;

struct ClsScratch {
    __nv_bfloat16 *X, *H, *T, *DZ, *DU, *DH0, *G, *wb;
    float *L, *valid, *btail, *grad, *partial;
    WgradJob *jobs;
    long long B;
    __host__ __device__ __nv_bfloat16 *h(int k) const { return H + (size_t)k * B * W; }
    __host__ __device__ __nv_bfloat16 *t(int k) const { return T + (size_t)k * B * W; }
    __host__ __device__ __nv_bfloat16 *dz(int k) const { return DZ + (size_t)k * B * W; }
    __host__ __device__ __nv_bfloat16 *du(int k) const { return DU + (size_t)k * B * W; }
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t scratch_bytes(long long B)
{
    const size_t splits = (size_t)((B + kClsSplitRows - 1) / kClsSplitRows);
    return 256 + a256((size_t)B * kClsIn * 2) + a256((size_t)(NBLK + 1) * B * W * 2) + 3 * a256((size_t)NBLK * B * W * 2) +
           a256((size_t)B * W * 2) + a256((size_t)B * NOUT_PAD * 2) + a256((size_t)kWbElems * 2) + a256((size_t)B * NOUT * 4) +
           a256((size_t)B * 4) + a256((size_t)NOUT * 4) + a256((size_t)kClsParams * 4) + splits * (size_t)kClsParams * 4 +
           a256(sizeof(WgradJob) * kJobs);
}

ClsScratch carve(void *base, long long B)
{
    ClsScratch s;
    s.B = B;
    uint8_t *p = reinterpret_cast<uint8_t *>(a256(reinterpret_cast<size_t>(base)));
    auto take = [&](size_t bytes) { uint8_t *q = p; p += a256(bytes); return q; };
    s.X = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * kClsIn * 2));
    s.H = reinterpret_cast<__nv_bfloat16 *>(take((size_t)(NBLK + 1) * B * W * 2));
    s.T = reinterpret_cast<__nv_bfloat16 *>(take((size_t)NBLK * B * W * 2));
    s.DZ = reinterpret_cast<__nv_bfloat16 *>(take((size_t)NBLK * B * W * 2));
    s.DU = reinterpret_cast<__nv_bfloat16 *>(take((size_t)NBLK * B * W * 2));
    s.DH0 = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * W * 2));
    s.G = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * NOUT_PAD * 2));
    s.wb = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kWbElems * 2));
    s.L = reinterpret_cast<float *>(take((size_t)B * NOUT * 4));
    s.valid = reinterpret_cast<float *>(take((size_t)B * 4));
    s.btail = reinterpret_cast<float *>(take((size_t)NOUT * 4));
    s.grad = reinterpret_cast<float *>(take((size_t)kClsParams * 4));
    s.jobs = reinterpret_cast<WgradJob *>(take(sizeof(WgradJob) * kJobs));
    s.partial = reinterpret_cast<float *>(p);
    return s;
}

// ---- kernels ------------------------------------------------------------------------------------
// Row r = training-set row (start + r) mod n: the 16 chord points, each [x, sin(2^k x), cos(2^k x)],
// rounded to BF16.
__global__ void k_cls_encode(const float *o, const float *d, long long n_rows, long long start, long long B, float rb,
                             __nv_bfloat16 *X, float *valid)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * 16; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e >> 4;
        const int j = (int)(e & 15);
        const long long q = (start + r) % n_rows;
        const V3 ol = v3(o[3 * q], o[3 * q + 1], o[3 * q + 2]);
        const V3 dl = normalized(v3(d[3 * q], d[3 * q + 1], d[3 * q + 2]));
        Chord ch;
        const bool kept = bound_chord(ol, dl, rb, ch);
        const V3 x = madd(ol, ch.te + (ch.tx - ch.te) * (float)j / 15.0f, dl);
        const float xs[3] = {x.x, x.y, x.z};
        __nv_bfloat16 *row = X + (size_t)r * kClsIn + 63 * j;
        for (int f = 0; f < 63; ++f) row[f] = __float2bfloat16_rn(kept ? posenc_feature(xs, 3, 10, f) : 0.0f);
        if (j == 0) valid[r] = kept ? 1.0f : 0.0f;
    }
}

// The BF16 weights and the tails' FP32 bias row from the packed FP32 master.
__global__ void k_cls_pack(const float *w, __nv_bfloat16 *wb, float *btail)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < kWbElems; e += (long long)gridDim.x * blockDim.x) {
        float v = 0.0f;
        if (e < kWbBlock0) {
            v = w[e];                                                      // head [256][1008]
        } else if (e < kWbTail) {
            const long long q = e - kWbBlock0, layer = q / ((long long)W * W), k = q % ((long long)W * W);
            v = w[kBlock0 + layer * kLayer + k];                            // W1 / W2 of block layer / 2
        } else {
            const long long q = e - kWbTail, o = q / W, i = q % W;
            if (o < 1 + NC) v = w[kTailA + o * W + i];
            else if (o < NOUT) v = w[kTailB + (o - 1 - NC) * W + i];
        }
        wb[e] = __float2bfloat16_rn(v);
    }
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < NOUT; o += gridDim.x * blockDim.x)
        btail[o] = o < 1 + NC ? w[kTailA + (long long)(1 + NC) * W + o] : w[kTailB + (long long)NF * W + (o - 1 - NC)];
}

__device__ __forceinline__ float bce(float x, float y) { return fmaxf(x, 0.0f) - x * y + log1pf(expf(-fabsf(x))); }
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Hit rows of the batch (the bin terms of Eq. 6 are averaged over them).
__global__ void k_count_hits(const float *hit_star, const float *valid, long long n_rows, long long start, long long B,
                             float *loss)
{
    float c = 0.0f;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < B; r += (long long)gridDim.x * blockDim.x)
        c += (valid[r] > 0.5f && hit_star[(start + r) % n_rows] > 0.5f) ? 1.0f : 0.0f;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c > 0.0f) atomicAdd(&loss[1], c);
}

// Eq. 6 per row and its gradient with respect to the logits (one warp per row), the gradient as
// BF16 rows of NOUT_PAD (zero beyond the 193 logits).  Segment
// operator S: u = (m* + 1) N_c / 2, c = floor(u), f = floor((u - c) N_f), clamped.
__global__ void k_cls_loss(const float *L, __nv_bfloat16 *G, const float *m_star, const float *hit_star, const float *valid,
                           long long n_rows, long long start, long long B, float *loss)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const float n_hit = fmaxf(loss[1], 1.0f);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < B; r += warps) {
        const long long q = (start + r) % n_rows;
        const bool ok = valid[r] > 0.5f;
        const bool hit = ok && hit_star[q] > 0.5f;
        int cs = 0, fs = 0;
        if (hit) {
            const float u = (m_star[q] + 1.0f) * 0.5f * NC;
            cs = min(max((int)floorf(u), 0), NC - 1);
            fs = min(max((int)floorf((u - cs) * NF), 0), NF - 1);
        }
        const float *l = L + (size_t)r * NOUT;
        __nv_bfloat16 *g = G + (size_t)r * NOUT_PAD;
        float acc = 0.0f;
        for (int i = lane; i < NOUT; i += 32) {
            float gi = 0.0f;
            if (!ok) {
                gi = 0.0f;
            } else if (i == 0) {
                const float y = hit ? 1.0f : 0.0f;
                acc += 0.1f * bce(l[0], y) / B;
                gi = 0.1f * (sigm(l[0]) - y) / B;
            } else if (hit && i <= NC) {
                const float y = i - 1 == cs ? 1.0f : 0.0f;
                acc += bce(l[i], y) / NC / n_hit;
                gi = (sigm(l[i]) - y) / NC / n_hit;
            } else if (hit) {
                const float y = i - 1 - NC == fs ? 1.0f : 0.0f;
                acc += bce(l[i], y) / NF / n_hit;
                gi = (sigm(l[i]) - y) / NF / n_hit;
            }
            g[i] = __float2bfloat16_rn(gi);     // the logit gradient enters the products in BF16
        }
        for (int i = NOUT + lane; i < NOUT_PAD; i += 32) g[i] = __float2bfloat16_rn(0.0f);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) atomicAdd(&loss[0], acc);
    }
}

// Adam (Kingma & Ba 2015) with bias correction.
__global__ void k_adam(float *theta, const float *g, float *m, float *v, long long n, float lr, float c1, float c2)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float gi = g[e];
        const float mi = 0.9f * m[e] + 0.1f * gi, vi = 0.999f * v[e] + 0.001f * gi * gi;
        m[e] = mi;
        v[e] = vi;
        theta[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    }
}

int grid_for(long long n, int num_sms) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 16)); }

Operand kop(const __nv_bfloat16 *p, long long ld, int rows, long long k) { return Operand{p, ld, rows, k, tcg::kKMajor, -1}; }
Operand mnop(const __nv_bfloat16 *p, long long ld, int rows, long long k, int ones = -1)
{
    return Operand{p, ld, rows, k, tcg::kMNMajor, ones};
}

// The weight-gradient tiles of one batch (see trn::WgradJob).
int make_jobs(const ClsScratch &s, WgradJob *J)
{
    int n = 0;
    const long long B = s.B;
    auto job = [&](Operand a, Operand b, int m0, int n0, int fo, int fi, int ones, long long w0, long long b0,
                   int seg, long long w1, long long b1) {
        WgradJob j{};
        j.a = a; j.b = b; j.m0 = m0; j.n0 = n0; j.c_lo = n0; j.c_hi = n0 + 128; j.fo = fo; j.fi = fi;
        j.ones = (ones >= n0 && ones < n0 + 144) ? ones : -1;
        j.seg_split = seg; j.w_off[0] = w0; j.b_off[0] = b0; j.w_off[1] = w1; j.b_off[1] = b1;
        J[n++] = j;
    };
    // head: dW = dH0^T X (1008 inputs in eight 128-column tiles, the ones row at 1008)
    for (int mb = 0; mb < 2; ++mb)
        for (int nb = 0; nb < 8; ++nb)
            job(mnop(s.DH0, W, W, B), mnop(s.X, kClsIn, kClsIn, B, kClsIn), mb * 128, nb * 128, W, kClsIn, kClsIn, 0,
                kHeadW, W, 0, 0);
    // blocks: dW1 = dU^T h, dW2 = dZ^T t
    for (int k = 0; k < NBLK; ++k)
        for (int layer = 0; layer < 2; ++layer) {
            const long long off = kBlock0 + (2LL * k + layer) * kLayer;
            const __nv_bfloat16 *A = layer == 0 ? s.du(k) : s.dz(k), *Bm = layer == 0 ? s.h(k) : s.t(k);
            for (int mb = 0; mb < 2; ++mb)
                for (int nb = 0; nb < 2; ++nb)
                    job(mnop(A, W, W, B), mnop(Bm, W, W, B, W), mb * 128, nb * 128, W, W, W, off, off + (long long)W * W, W,
                        0, 0);
        }
    // tails: dW = G^T h_16 (rows 0 .. 64 tail A, 65 .. 192 tail B)
    for (int mb = 0; mb < 2; ++mb)
        for (int nb = 0; nb < 2; ++nb)
            job(mnop(s.G, NOUT_PAD, NOUT_PAD, B), mnop(s.h(NBLK), W, W, B, W), mb * 128, nb * 128, NOUT, W, W, kTailA,
                kTailA + (long long)(1 + NC) * W, 1 + NC, kTailB, kTailB + (long long)NF * W);
    return n;
}

// Forward, loss and gradient of one batch; the gradient lands in s.grad.
cudaError_t loss_grad(const ClsTrainLaunch &L, const ClsScratch &s, const float *o, const float *d, const float *m_star,
                      const float *hit_star, long long n_rows, long long start)
{
    cudaStream_t st = L.stream;
    const long long B = s.B;
    const int M = (int)B;
    const int gsm = L.num_sms;
    const float *w = L.master;
    uint32_t *status = L.status;
    const uint32_t flag = kStatusTimeout;
    cudaError_t e = cudaMemsetAsync(L.loss, 0, sizeof(float) * 4, st);
    if (e != cudaSuccess) return e;
    k_cls_pack<<<gsm * 4, 256, 0, st>>>(w, s.wb, s.btail);
    k_cls_encode<<<grid_for(B * 16, gsm), 256, 0, st>>>(o, d, n_rows, start, B, L.rb, s.X, s.valid);
    // forward
#define CK_(x) do { if ((e = (x)) != cudaSuccess) return e; } while (0)
    CK_((trn::rows_gemm<W, kHeadStages>(kop(s.X, kClsIn, M, kClsIn), kop(s.wb + kWbHead, kClsIn, W, kClsIn), M, kClsIn,
                                       trn::EpiForward<false, false>{s.h(0), w + kHeadW, nullptr, M, W, W}, status, flag, st)));
    for (int k = 0; k < NBLK; ++k) {
        const __nv_bfloat16 *W1 = s.wb + kWbBlock0 + 2LL * k * W * W, *W2 = W1 + (long long)W * W;
        const float *b1 = w + kBlock0 + 2LL * k * kLayer + (long long)W * W, *b2 = b1 + kLayer;
        CK_((trn::rows_gemm<W, kRowStages>(kop(s.h(k), W, M, W), kop(W1, W, W, W), M, W,
                                           trn::EpiForward<true, false>{s.t(k), b1, nullptr, M, W, W}, status, flag, st)));
        CK_((trn::rows_gemm<W, kRowStages>(kop(s.t(k), W, M, W), kop(W2, W, W, W), M, W,
                                           trn::EpiForward<true, true>{s.h(k + 1), b2, s.h(k), M, W, W}, status, flag, st)));
    }
    CK_((trn::rows_gemm<NOUT_PAD, kRowStages>(kop(s.h(NBLK), W, M, W), kop(s.wb + kWbTail, W, NOUT_PAD, W), M, W,
                                              trn::EpiLogits{s.L, s.btail, M, NOUT, NOUT}, status, flag, st)));
    // Eq. 6 and its gradient
    k_count_hits<<<grid_for(B, gsm), 256, 0, st>>>(hit_star, s.valid, n_rows, start, B, L.loss);
    k_cls_loss<<<grid_for(B * 32, gsm), 256, 0, st>>>(s.L, s.G, m_star, hit_star, s.valid, n_rows, start, B, L.loss);
    // backward: tails, then the blocks last to first: dz = dh [z > 0]; du = (dz W2) [u > 0];
    // dh = dz + du W1 (masked by the block input for the next dz; unmasked at the linear head)
    CK_((trn::rows_gemm<W, kRowStages>(kop(s.G, NOUT_PAD, M, NOUT_PAD), mnop(s.wb + kWbTail, W, W, NOUT_PAD), M, NOUT_PAD,
                                       trn::EpiBackward<false>{s.dz(NBLK - 1), s.h(NBLK), nullptr, M, W, W}, status, flag, st)));
    for (int k = NBLK - 1; k >= 0; --k) {
        const __nv_bfloat16 *W1 = s.wb + kWbBlock0 + 2LL * k * W * W, *W2 = W1 + (long long)W * W;
        CK_((trn::rows_gemm<W, kRowStages>(kop(s.dz(k), W, M, W), mnop(W2, W, W, W), M, W,
                                           trn::EpiBackward<false>{s.du(k), s.t(k), nullptr, M, W, W}, status, flag, st)));
        CK_((trn::rows_gemm<W, kRowStages>(kop(s.du(k), W, M, W), mnop(W1, W, W, W), M, W,
                                           trn::EpiBackward<true>{k > 0 ? s.dz(k - 1) : s.DH0, k > 0 ? s.h(k) : nullptr,
                                                                  s.dz(k), M, W, W},
                                           status, flag, st)));
    }
    // weight and bias gradients of every layer, split over the batch, one launch
    WgradJob jobs[kJobs];
    const int n_jobs = make_jobs(s, jobs);
    CK_(cudaMemcpyAsync(s.jobs, jobs, sizeof(WgradJob) * n_jobs, cudaMemcpyHostToDevice, st));
    CK_((trn::wgrad<144, kWgradStages>(s.jobs, n_jobs, B, kClsSplitRows, s.partial, kClsParams, status, flag, st)));
    const int splits = (int)((B + kClsSplitRows - 1) / kClsSplitRows);
    trn::k_sum_splits<<<grid_for(kClsParams, gsm), 256, 0, st>>>(s.partial, splits, kClsParams, s.grad);
#undef CK_
    return cudaGetLastError();
}

}  // namespace

size_t cls_train_scratch_bytes(long long batch) { return scratch_bytes(batch); }

cudaError_t launch_cls_loss_grad(const ClsTrainLaunch &L, const float *o, const float *d, const float *m_star,
                                 const float *hit_star, int n, float *grad)
{
    const ClsScratch s = carve(L.scratch, n);
    cudaError_t e = loss_grad(L, s, o, d, m_star, hit_star, n, 0);
    if (e == cudaSuccess && grad != s.grad)
        e = cudaMemcpyAsync(grad, s.grad, sizeof(float) * kClsParams, cudaMemcpyDeviceToDevice, L.stream);
    return e;
}

cudaError_t launch_cls_train_step(const ClsTrainLaunch &L, const float *o, const float *d, const float *m_star,
                                  const float *hit_star, long long n_rays, long long start, int batch, float *adam_m,
                                  float *adam_v, int step, float lr)
{
    const ClsScratch s = carve(L.scratch, batch);
    cudaError_t e = loss_grad(L, s, o, d, m_star, hit_star, n_rays, start);
    if (e != cudaSuccess) return e;
    const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
    k_adam<<<grid_for(kClsParams, L.num_sms), 256, 0, L.stream>>>(L.master, s.grad, adam_m, adam_v, kClsParams, lr, c1, c2);
    return cudaGetLastError();
}

}  // namespace nedf
