// Training of the paper's classifier intersection network (Section "Intersection network",
// Eq. 3-4 and the BCE loss of Eq. 6; "Training details": Adam), FP32.
//
// A batch of B labelled rays: the 16 encoded chord points of each (B x 1008), the forward pass
// with every block's input h, pre-activation u = W1 h + b1 and skip sum z = h + W2 ReLU(u) + b2
// kept, the logits, Eq. 6's loss and its gradient with respect to the logits, then the backward
// pass by hand (ReLU masks, the skip connection, dW = delta^T input, db = column sums of delta,
// d input = delta W) and one Adam step on the packed FP32 master weights.  The dense products are
// plain GEMMs and go to cuBLAS (row-major operands passed as their column-major transposes); the
// encoding, the loss, the masks and Adam are kernels of this file.
#include <cublas_v2.h>

#include <algorithm>
#include <cmath>

#include "mlp_f32.cuh"
#include "render_launch.h"
#include "train_launch.h"

namespace nedf {

namespace {

constexpr int W = 256, NC = 64, NF = 128, NOUT = 1 + NC + NF, NBLK = 16;
constexpr long long kHeadW = (long long)kClsIn * W;
constexpr long long kBlock0 = kHeadW + W;
constexpr long long kLayer = (long long)W * W + W;
constexpr long long kTailA = kBlock0 + 2 * NBLK * kLayer;
constexpr long long kTailB = kTailA + (long long)(1 + NC) * (W + 1);

// Scratch of a batch of B rows (floats, all row-major): X B x 1008; H[17], U[16], T[16], Z[16]
// B x 256 each; logits and G B x 193; dH, dZ, dT, dU B x 256; ones B; grad kClsParams; flags B.
struct ClsScratch {
    float *X, *H, *U, *T, *Z, *L, *G, *dH, *dZ, *dT, *dU, *ones, *grad, *valid;
    long long B;
    __host__ __device__ float *h(int k) const { return H + (size_t)k * B * W; }
    __host__ __device__ float *u(int k) const { return U + (size_t)k * B * W; }
    __host__ __device__ float *t(int k) const { return T + (size_t)k * B * W; }
    __host__ __device__ float *z(int k) const { return Z + (size_t)k * B * W; }
};

ClsScratch carve(float *base, long long B)
{
    ClsScratch s;
    s.B = B;
    float *p = base;
    auto take = [&](size_t n) { float *q = p; p += (n + 63) & ~(size_t)63; return q; };
    s.X = take((size_t)B * kClsIn);
    s.H = take((size_t)(NBLK + 1) * B * W);
    s.U = take((size_t)NBLK * B * W);
    s.T = take((size_t)NBLK * B * W);
    s.Z = take((size_t)NBLK * B * W);
    s.L = take((size_t)B * NOUT);
    s.G = take((size_t)B * NOUT);
    s.dH = take((size_t)B * W);
    s.dZ = take((size_t)B * W);
    s.dT = take((size_t)B * W);
    s.dU = take((size_t)B * W);
    s.ones = take((size_t)B);
    s.grad = take((size_t)kClsParams);
    s.valid = take((size_t)B);
    return s;
}

size_t scratch_floats(long long B)
{
    auto r = [](size_t n) { return (n + 63) & ~(size_t)63; };
    return r((size_t)B * kClsIn) + r((size_t)(NBLK + 1) * B * W) + 3 * r((size_t)NBLK * B * W) + 2 * r((size_t)B * NOUT) +
           4 * r((size_t)B * W) + r((size_t)B) + r((size_t)kClsParams) + r((size_t)B);
}

// ---- kernels ------------------------------------------------------------------------------------
// Row r = training-set row (start + r) mod n: the 16 chord points, each [x, sin(2^k x), cos(2^k x)].
__global__ void k_cls_encode(const float *o, const float *d, long long n_rows, long long start, long long B, float rb,
                             float *X, float *valid, float *ones)
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
        float *row = X + (size_t)r * kClsIn + 63 * j;
        for (int f = 0; f < 63; ++f) row[f] = kept ? posenc_feature(xs, 3, 10, f) : 0.0f;
        if (j == 0) {
            valid[r] = kept ? 1.0f : 0.0f;
            ones[r] = 1.0f;
        }
    }
}

// y[r][c] += b[c] (bias of a B x N output), optionally ReLU'd into a second buffer
__global__ void k_bias(float *y, const float *b, long long B, int N, int ldy, float *relu_out)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * N; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / N;
        const int c = (int)(e - r * N);
        const float v = y[r * ldy + c] + b[c];
        y[r * ldy + c] = v;
        if (relu_out) relu_out[r * N + c] = fmaxf(v, 0.0f);
    }
}

// z = z + h + b2 (z holds W2 t), h_next = ReLU(z)
__global__ void k_skip(float *z, const float *h, const float *b2, float *h_next, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float v = z[e] + h[e] + b2[e % W];
        z[e] = v;
        h_next[e] = fmaxf(v, 0.0f);
    }
}

// out = in * [pre > 0]
__global__ void k_mask(float *out, const float *in, const float *pre, long long n)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        out[e] = pre[e] > 0.0f ? in[e] : 0.0f;
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

// Eq. 6 per row and its gradient with respect to the logits (one warp per row).  Segment
// operator S: u = (m* + 1) N_c / 2, c = floor(u), f = floor((u - c) N_f), clamped.
__global__ void k_cls_loss(const float *L, float *G, const float *m_star, const float *hit_star, const float *valid,
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
        float *g = G + (size_t)r * NOUT;
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
            g[i] = gi;
        }
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

// ---- cuBLAS wrappers on row-major operands ------------------------------------------------------
struct Gemm {
    cublasHandle_t h;
    cublasStatus_t st = CUBLAS_STATUS_SUCCESS;
    // Y[B x N] (ldy) = X[B x K] W^T, W row-major N x K (the packed layout)
    void fwd(const float *X, int K, const float *Wt, int N, float *Y, int ldy, long long B)
    {
        const float one = 1.0f, zero = 0.0f;
        if (st == CUBLAS_STATUS_SUCCESS)
            st = cublasSgemm(h, CUBLAS_OP_T, CUBLAS_OP_N, N, (int)B, K, &one, Wt, K, X, K, &zero, Y, ldy);
    }
    // dW[N x K] (+)= G[B x N]^T X[B x K]
    void wgrad(const float *G, int ldg, int N, const float *X, int K, float *dW, long long B, float beta)
    {
        const float one = 1.0f;
        if (st == CUBLAS_STATUS_SUCCESS)
            st = cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_T, K, N, (int)B, &one, X, K, G, ldg, &beta, dW, K);
    }
    // dX[B x K] (+)= G[B x N] W[N x K]
    void dgrad(const float *G, int ldg, int N, const float *Wt, int K, float *dX, long long B, float beta)
    {
        const float one = 1.0f;
        if (st == CUBLAS_STATUS_SUCCESS)
            st = cublasSgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, K, (int)B, N, &one, Wt, K, G, ldg, &beta, dX, K);
    }
    // db[N] = column sums of G[B x N]
    void bgrad(const float *G, int ldg, int N, const float *ones, float *db, long long B)
    {
        const float one = 1.0f, zero = 0.0f;
        if (st == CUBLAS_STATUS_SUCCESS) st = cublasSgemv(h, CUBLAS_OP_N, N, (int)B, &one, G, ldg, ones, 1, &zero, db, 1);
    }
};

int grid_for(long long n, int num_sms) { return (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, (long long)num_sms * 16)); }

// Forward, loss and gradient of one batch; the gradient lands in s.grad.
cudaError_t loss_grad(const ClsTrainLaunch &L, const ClsScratch &s, const float *o, const float *d, const float *m_star,
                      const float *hit_star, long long n_rows, long long start)
{
    cudaStream_t st = L.stream;
    const long long B = s.B;
    const int gsm = L.num_sms;
    Gemm g{static_cast<cublasHandle_t>(L.cublas)};
    const float *w = L.master;
    float *gr = s.grad;
    cudaMemsetAsync(L.loss, 0, sizeof(float) * 4, st);
    k_cls_encode<<<grid_for(B * 16, gsm), 256, 0, st>>>(o, d, n_rows, start, B, L.rb, s.X, s.valid, s.ones);
    // forward
    g.fwd(s.X, kClsIn, w, W, s.h(0), W, B);
    k_bias<<<grid_for(B * W, gsm), 256, 0, st>>>(s.h(0), w + kHeadW, B, W, W, nullptr);
    for (int k = 0; k < NBLK; ++k) {
        const float *W1 = w + kBlock0 + 2 * k * kLayer, *W2 = W1 + kLayer;
        g.fwd(s.h(k), W, W1, W, s.u(k), W, B);
        k_bias<<<grid_for(B * W, gsm), 256, 0, st>>>(s.u(k), W1 + (size_t)W * W, B, W, W, s.t(k));
        g.fwd(s.t(k), W, W2, W, s.z(k), W, B);
        k_skip<<<grid_for(B * W, gsm), 256, 0, st>>>(s.z(k), s.h(k), W2 + (size_t)W * W, s.h(k + 1), B * W);
    }
    g.fwd(s.h(NBLK), W, w + kTailA, 1 + NC, s.L, NOUT, B);
    g.fwd(s.h(NBLK), W, w + kTailB, NF, s.L + 1 + NC, NOUT, B);
    k_bias<<<grid_for(B * (1 + NC), gsm), 256, 0, st>>>(s.L, w + kTailA + (size_t)(1 + NC) * W, B, 1 + NC, NOUT, nullptr);
    k_bias<<<grid_for(B * NF, gsm), 256, 0, st>>>(s.L + 1 + NC, w + kTailB + (size_t)NF * W, B, NF, NOUT, nullptr);
    // Eq. 6 and its gradient
    k_count_hits<<<grid_for(B, gsm), 256, 0, st>>>(hit_star, s.valid, n_rows, start, B, L.loss);
    k_cls_loss<<<grid_for(B * 32, gsm), 256, 0, st>>>(s.L, s.G, m_star, hit_star, s.valid, n_rows, start, B, L.loss);
    // backward: tails
    g.wgrad(s.G, NOUT, 1 + NC, s.h(NBLK), W, gr + kTailA, B, 0.0f);
    g.bgrad(s.G, NOUT, 1 + NC, s.ones, gr + kTailA + (size_t)(1 + NC) * W, B);
    g.wgrad(s.G + 1 + NC, NOUT, NF, s.h(NBLK), W, gr + kTailB, B, 0.0f);
    g.bgrad(s.G + 1 + NC, NOUT, NF, s.ones, gr + kTailB + (size_t)NF * W, B);
    g.dgrad(s.G, NOUT, 1 + NC, w + kTailA, W, s.dH, B, 0.0f);
    g.dgrad(s.G + 1 + NC, NOUT, NF, w + kTailB, W, s.dH, B, 1.0f);
    // blocks, last to first: dz = dh [z > 0]; dW2 = dz^T t; dt = dz W2; du = dt [u > 0];
    // dW1 = du^T h; dh = dz + du W1
    for (int k = NBLK - 1; k >= 0; --k) {
        const long long o1 = kBlock0 + 2 * k * kLayer, o2 = o1 + kLayer;
        k_mask<<<grid_for(B * W, gsm), 256, 0, st>>>(s.dZ, s.dH, s.z(k), B * W);
        g.wgrad(s.dZ, W, W, s.t(k), W, gr + o2, B, 0.0f);
        g.bgrad(s.dZ, W, W, s.ones, gr + o2 + (size_t)W * W, B);
        g.dgrad(s.dZ, W, W, w + o2, W, s.dT, B, 0.0f);
        k_mask<<<grid_for(B * W, gsm), 256, 0, st>>>(s.dU, s.dT, s.u(k), B * W);
        g.wgrad(s.dU, W, W, s.h(k), W, gr + o1, B, 0.0f);
        g.bgrad(s.dU, W, W, s.ones, gr + o1 + (size_t)W * W, B);
        cudaMemcpyAsync(s.dH, s.dZ, sizeof(float) * B * W, cudaMemcpyDeviceToDevice, st);
        g.dgrad(s.dU, W, W, w + o1, W, s.dH, B, 1.0f);
    }
    // head (linear)
    g.wgrad(s.dH, W, W, s.X, kClsIn, gr, B, 0.0f);
    g.bgrad(s.dH, W, W, s.ones, gr + kHeadW, B);
    if (g.st != CUBLAS_STATUS_SUCCESS) return cudaErrorUnknown;
    return cudaGetLastError();
}

}  // namespace

size_t cls_train_scratch_bytes(long long batch) { return scratch_floats(batch) * sizeof(float); }

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
