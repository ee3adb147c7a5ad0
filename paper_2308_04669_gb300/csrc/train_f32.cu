// Learned part: training-set generation, NeDF forward with saved activations, hand-written
// backward, split-K weight-gradient GEMMs and fused Adam (FP32 on CUDA cores).
//
// Method: arXiv 2308.04669, Section "Intersection network" (supervision of F_Phi by the
// radiance field's depth, converted to mu through Eq. 2), Eq. 5-6, "Training details" (Adam).
// Labels come from the plain method on the analytic density; the loss is the regression form
// of Eq. 6 for a (depth, hit logit) network.
#include <algorithm>
#include <cmath>

#include "mlp_f32.cuh"
#include "train_launch.h"

namespace nedf {

// ---------------------------------------------------------------------------------------------
// training set: rays entering the bound sphere, labelled by the plain method
// ---------------------------------------------------------------------------------------------
// Ray r of a training set: entry point uniform on the bound sphere, cosine-weighted inward
// direction, from four counter-based uniforms.
__device__ __forceinline__ void label_ray(uint64_t seed, long long r, float rb, V3 &org, V3 &dir)
{
    float u0 = uniform24(seed, 4ull * r), u1 = uniform24(seed, 4ull * r + 1);
    float u2 = uniform24(seed, 4ull * r + 2), u3 = uniform24(seed, 4ull * r + 3);
    // entry point uniform on the sphere
    float z = 1.0f - 2.0f * u0, phi = 6.283185307179586f * u1;
    float rho = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincosf(phi, &sp, &cp);
    V3 nrm = v3(rho * cp, rho * sp, z);
    V3 w = v3(-nrm.x, -nrm.y, -nrm.z);
    // tangent frame about the inward normal (Duff et al., JCGT 2017)
    float sg = w.z >= 0.0f ? 1.0f : -1.0f;
    float a = -1.0f / (sg + w.z), b = w.x * w.y * a;
    V3 b1 = v3(1.0f + sg * w.x * w.x * a, sg * b, -sg * w.x);
    V3 b2 = v3(b, sg + w.y * w.y * a, -w.y);
    // cosine-weighted direction
    float rr = sqrtf(u2), st, ct;
    sincosf(6.283185307179586f * u3, &st, &ct);
    float lx = rr * ct, ly = rr * st, lz = sqrtf(fmaxf(0.0f, 1.0f - u2));
    dir = v3(lx * b1.x + ly * b2.x + lz * w.x, lx * b1.y + ly * b2.y + lz * w.y, lx * b1.z + ly * b2.z + lz * w.z);
    org = v3(rb * nrm.x, rb * nrm.y, rb * nrm.z);
}

__global__ void k_make_labels(const DevType *type_p, float rb, long long n, uint64_t seed, int steps, int bisect,
                              float *o, float *d, float *m_star, float *hit_star)
{
    const DevType T = *type_p;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
        V3 org, dir;
        label_ray(seed, r, rb, org, dir);
        o[3 * r] = org.x; o[3 * r + 1] = org.y; o[3 * r + 2] = org.z;
        d[3 * r] = dir.x; d[3 * r + 1] = dir.y; d[3 * r + 2] = dir.z;
        V3 dl = normalized(dir);
        Chord ch;
        float ms = 0.0f, hs = 0.0f;
        if (bound_chord(org, dl, rb, ch)) {
            bool hit;
            float D = march_crossing(T, org, dl, ch.te, ch.tx, steps, bisect, hit);
            if (hit) {
                hs = 1.0f;
                ms = (ch.tp - D) / rb;
            }
        }
        m_star[r] = ms;
        hit_star[r] = hs;
    }
}

cudaError_t launch_make_labels(const DevType *type, float rb, long long n_rays, uint64_t seed, int steps,
                               int bisect, float *o, float *d, float *m_star, float *hit_star, int num_sms,
                               cudaStream_t st)
{
    long long blocks = (n_rays + 255) / 256;
    if (blocks > (long long)num_sms * 32) blocks = (long long)num_sms * 32;
    k_make_labels<<<(int)blocks, 256, 0, st>>>(type, rb, n_rays, seed, steps, bisect, o, d, m_star, hit_star);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// training set labelled by a generic radiance field's density network (plugin mode): the same
// rays; per ray, sigma = ReLU(MLP(gamma_10(x))) at n_samples chord midpoints (64-row FP32 tiles),
// then Eq. 5's weights w_i = T_i (1 - exp(-sigma_i delta)).  Label depth: the opacity-normalised
// Eq. 5 depth; hit: opacity > 0.5; m* = (t_perp - D) / rb.  One block per ray.
// ---------------------------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(kThreads) k_density_labels(const float *wk, int hidden, float rb, long long n,
                                                             uint64_t seed, int n_samples, float *o, float *d,
                                                             float *m_star, float *hit_star)
{
    __shared__ __align__(16) float X[(W > kDensIn ? W : kDensIn) * kXStride];
    __shared__ float y[kTileRows][4];
    __shared__ float sig[kMaxDensSamples];
    const float *wo = wk + (size_t)kDensIn * W + W + (size_t)(hidden - 1) * (W * W + W);
    for (long long r = blockIdx.x; r < n; r += gridDim.x) {
        V3 org, dir;
        label_ray(seed, r, rb, org, dir);
        if (threadIdx.x == 0) {
            o[3 * r] = org.x; o[3 * r + 1] = org.y; o[3 * r + 2] = org.z;
            d[3 * r] = dir.x; d[3 * r + 1] = dir.y; d[3 * r + 2] = dir.z;
        }
        const V3 dl = normalized(dir);
        Chord ch;
        const bool kept = bound_chord(org, dl, rb, ch);      // the same outcome in every thread
        if (!kept) {
            if (threadIdx.x == 0) { m_star[r] = 0.0f; hit_star[r] = 0.0f; }
            continue;
        }
        const float delta = (ch.tx - ch.te) / n_samples;
        for (int t0 = 0; t0 < n_samples; t0 += kTileRows) {
            for (int e = threadIdx.x; e < kTileRows * kDensIn; e += blockDim.x) {
                const int rr = e % kTileRows, fi = e / kTileRows;
                const V3 x = madd(org, ch.te + (t0 + rr + 0.5f) * delta, dl);
                const float xs[3] = {x.x, x.y, x.z};
                X[fi * kXStride + rr] = posenc_feature(xs, 3, 10, fi);
            }
            __syncthreads();
            mlp_hidden_f32<W>(X, kDensIn, hidden, wk);
            out_layer_f32(X, W, wo, wo + W, 1, y);
            if (threadIdx.x < kTileRows && t0 + (int)threadIdx.x < n_samples)
                sig[t0 + threadIdx.x] = fmaxf(y[threadIdx.x][0], 0.0f);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            float T = 1.0f, A = 0.0f, Dw = 0.0f;
            for (int i = 0; i < n_samples; ++i) {
                const float alpha = 1.0f - expf(-sig[i] * delta);
                const float wi = T * alpha;
                A += wi;
                Dw += wi * (ch.te + (i + 0.5f) * delta);
                T *= 1.0f - alpha;
            }
            const bool hit = A > 0.5f;
            m_star[r] = hit ? (ch.tp - Dw / A) / rb : 0.0f;
            hit_star[r] = hit ? 1.0f : 0.0f;
        }
        __syncthreads();
    }
}

cudaError_t launch_density_labels(const float *wk, int hidden, int width, float rb, long long n_rays, uint64_t seed,
                                  int n_samples, float *o, float *d, float *m_star, float *hit_star, int num_sms,
                                  cudaStream_t st)
{
    if (n_samples < 1 || n_samples > kMaxDensSamples || hidden < 1) return cudaErrorInvalidValue;
    const int blocks = (int)std::min<long long>(n_rays, (long long)num_sms * 8);
    if (width == 64)
        k_density_labels<64><<<blocks, kThreads, 0, st>>>(wk, hidden, rb, n_rays, seed, n_samples, o, d, m_star, hit_star);
    else if (width == 128)
        k_density_labels<128><<<blocks, kThreads, 0, st>>>(wk, hidden, rb, n_rays, seed, n_samples, o, d, m_star, hit_star);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// scratch layout for a batch of B rows (all row-major [B][width]):
//   h[0]: B x 80 (encoded input), h[1..L]: B x w (hidden activations),
//   dz[0..L-1]: B x w (gradient w.r.t. hidden pre-activations), dy: B x 2, valid: B, then grad.
// ---------------------------------------------------------------------------------------------
// Weight and bias gradients are summed over the batch in splits of kSplitRows rows; each split
// writes its own partial gradient and k_sum_splits adds the splits in a fixed order, so a training
// step is deterministic (and a resumed run repeats an uninterrupted one bit for bit).
constexpr int kSplitRows = 512;          // 128 splits at a batch of 65536

struct TrainScratch {
    float *h[17];
    float *dz[16];
    float *dy;
    float *valid;
    float *grad;
    float *zero;                 // 512 zeros (bias operand of the backward products)
    float *partial;              // [splits][n_params]
};

static TrainScratch carve(float *base, int B, int L, int w, long long n_params)
{
    TrainScratch s{};
    float *p = base;
    s.h[0] = p; p += (size_t)B * kNedfInPad;
    for (int l = 1; l <= L; ++l) { s.h[l] = p; p += (size_t)B * w; }
    for (int l = 0; l < L; ++l) { s.dz[l] = p; p += (size_t)B * w; }
    s.dy = p; p += (size_t)B * 2;
    s.valid = p; p += (size_t)B;
    s.grad = p; p += n_params;
    s.zero = p; p += 512;
    s.partial = p;
    return s;
}

size_t train_scratch_bytes(int batch, int hidden, int width, long long n_params)
{
    const size_t splits = ((size_t)batch + kSplitRows - 1) / kSplitRows;
    size_t floats = (size_t)batch * (kNedfInPad + 2 * (size_t)hidden * width + 3) + n_params + 512 + splits * n_params;
    return floats * sizeof(float);
}

// rows of the batch: b -> dataset index (start + b) mod n
__device__ __forceinline__ long long row_index(long long start, long long b, long long n) { return (start + b) % n; }

// hit count of the batch (the mean of the depth term runs over labelled hits)
__global__ void k_count_hits(const float *hit_star, long long start, long long n, int B, float *loss)
{
    float c = 0.0f;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x)
        c += hit_star[row_index(start, b, n)];
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c != 0.0f) atomicAdd(&loss[1], c);
}

template <int W>
__global__ void __launch_bounds__(kThreads) k_train_fwd(const DevType *type_p, float rb, int L, const float *w,
                                                        const float *o, const float *d, const float *m_star,
                                                        const float *hit_star, long long start, long long n, int B,
                                                        TrainScratch s, float *loss)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ float x6[kTileRows][6];
    __shared__ int kept[kTileRows];
    __shared__ float y[kTileRows][4];
    __shared__ float red[kThreads / 32];
    (void)type_p;
    const float n_hit = loss[1];
    for (long long tile = blockIdx.x; tile * kTileRows < B; tile += gridDim.x) {
        const long long b0 = tile * kTileRows;
        if (threadIdx.x < kTileRows) {
            long long b = b0 + threadIdx.x;
            kept[threadIdx.x] = 0;
            for (int c = 0; c < 6; ++c) x6[threadIdx.x][c] = 0.0f;
            if (b < B) {
                long long i = row_index(start, b, n);
                V3 ol = v3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
                V3 dl = normalized(v3(d[3 * i], d[3 * i + 1], d[3 * i + 2]));
                Chord ch;
                if (bound_chord(ol, dl, rb, ch)) {
                    kept[threadIdx.x] = 1;
                    V3 pe = madd(ol, ch.te, dl);
                    x6[threadIdx.x][0] = pe.x; x6[threadIdx.x][1] = pe.y; x6[threadIdx.x][2] = pe.z;
                    x6[threadIdx.x][3] = dl.x; x6[threadIdx.x][4] = dl.y; x6[threadIdx.x][5] = dl.z;
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRows * kNedfInPad; e += blockDim.x) {
            int r = e % kTileRows, fi = e / kTileRows;
            float v = fi < kNedfIn ? posenc_feature(x6[r], 6, 6, fi) : 0.0f;
            X[fi * kXStride + r] = v;
            long long b = b0 + r;
            if (b < B) s.h[0][(size_t)b * kNedfInPad + fi] = v;
        }
        __syncthreads();
        // hidden layers, each output saved for the backward pass
        const float *wp = w;
        int K = kNedfIn;
        for (int l = 0; l < L; ++l) {
            dense_f32<W>(X, K, wp, wp + (size_t)K * W, true);
            wp += (size_t)K * W + W;
            K = W;
            for (int e = threadIdx.x; e < kTileRows * W; e += blockDim.x) {
                int fi = e / kTileRows, r = e - fi * kTileRows;
                long long b = b0 + r;
                if (b < B) s.h[l + 1][(size_t)b * W + fi] = X[fi * kXStride + r];
            }
        }
        out_layer_f32(X, W, wp, wp + 2 * W, 2, y);
        // loss terms and dL/dy
        float part = 0.0f;
        if (threadIdx.x < kTileRows) {
            long long b = b0 + threadIdx.x;
            if (b < B) {
                long long i = row_index(start, b, n);
                float dm = 0.0f, da = 0.0f;
                if (kept[threadIdx.x]) {
                    float m = y[threadIdx.x][0], a = y[threadIdx.x][1], al = hit_star[i];
                    float bce = fmaxf(a, 0.0f) - al * a + log1pf(expf(-fabsf(a)));
                    part = 0.1f * bce / (float)B;
                    if (al > 0.5f) {
                        float e = m - m_star[i];
                        part += e * e / n_hit;
                        dm = 2.0f * e / n_hit;
                    }
                    da = 0.1f * (1.0f / (1.0f + expf(-a)) - al) / (float)B;
                }
                s.dy[2 * b] = dm;
                s.dy[2 * b + 1] = da;
                s.valid[b] = kept[threadIdx.x] ? 1.0f : 0.0f;
            }
        }
        for (int off = 16; off; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
            for (int k = 0; k < kThreads / 32; ++k) t += red[k];
            atomicAdd(&loss[0], t);
        }
        __syncthreads();
    }
}

// Backward through the hidden layers: dz_{L-1} = (W_L^T dy) * [h_L > 0], then
// dz_{l-1} = (W_l^T dz_l) * [h_l > 0].  W (packed, [out][in]) is the [K][N] operand here.
template <int W>
__global__ void __launch_bounds__(kThreads) k_train_bwd(int L, const float *master, int B, TrainScratch s,
                                                        const float *zero_bias)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    // offsets of each layer's W in the packed layout
    long long off[17];
    off[0] = 0;
    int K = kNedfIn;
    for (int l = 0; l < L; ++l) { off[l + 1] = off[l] + (long long)K * W + W; K = W; }
    const float *WL = master + off[L];   // output layer [2][W]
    for (long long tile = blockIdx.x; tile * kTileRows < B; tile += gridDim.x) {
        const long long b0 = tile * kTileRows;
        // dz_{L-1}
        for (int e = threadIdx.x; e < kTileRows * W; e += blockDim.x) {
            int k = e / kTileRows, r = e - k * kTileRows;
            long long b = b0 + r;
            float v = 0.0f;
            if (b < B) {
                float g = WL[k] * s.dy[2 * b] + WL[W + k] * s.dy[2 * b + 1];
                v = s.h[L][(size_t)b * W + k] > 0.0f ? g : 0.0f;
                s.dz[L - 1][(size_t)b * W + k] = v;
            }
            X[k * kXStride + r] = v;
        }
        __syncthreads();
        for (int l = L - 1; l >= 1; --l) {
            dense_f32<W>(X, W, master + off[l], zero_bias, false);   // X <- X W_l  (rows x in)
            for (int e = threadIdx.x; e < kTileRows * W; e += blockDim.x) {
                int k = e / kTileRows, r = e - k * kTileRows;
                long long b = b0 + r;
                float v = 0.0f;
                if (b < B) {
                    v = s.h[l][(size_t)b * W + k] > 0.0f ? X[k * kXStride + r] : 0.0f;
                    s.dz[l - 1][(size_t)b * W + k] = v;
                }
                X[k * kXStride + r] = v;
            }
            __syncthreads();
        }
        __syncthreads();
    }
}

// dW[out][in] = sum_b A[b][out] * Bm[b][in] over split z's rows, stored at dW + z * split_stride;
// 64x64 output tile per block.
__global__ void __launch_bounds__(256) k_grad_atb(const float *A, int lda, const float *Bm, int ldb, int n_out, int n_in,
                                                  int rows, int rows_per_split, float *dW, long long split_stride)
{
    dW += blockIdx.z * split_stride;
    __shared__ float As[32][64 + 4];
    __shared__ float Bs[32][64 + 4];
    const int o0 = blockIdx.x * 64, i0 = blockIdx.y * 64;
    const int r0 = blockIdx.z * rows_per_split, r1 = min(rows, r0 + rows_per_split);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][4] = {};
    for (int rc = r0; rc < r1; rc += 32) {
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            int rr = e / 64, c = e - rr * 64;
            int r = rc + rr;
            As[rr][c] = (r < r1 && o0 + c < n_out) ? A[(size_t)r * lda + o0 + c] : 0.0f;
            Bs[rr][c] = (r < r1 && i0 + c < n_in) ? Bm[(size_t)r * ldb + i0 + c] : 0.0f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            float a[4], b[4];
            for (int q = 0; q < 4; ++q) { a[q] = As[k][ty * 4 + q]; b[q] = Bs[k][tx * 4 + q]; }
            for (int p = 0; p < 4; ++p)
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            int oo = o0 + ty * 4 + p, ii = i0 + tx * 4 + q;
            if (oo < n_out && ii < n_in) dW[(size_t)oo * n_in + ii] = acc[p][q];
        }
}

// db[out] = sum_b A[b][out] over split y's rows, stored at db + y * split_stride.  A block takes
// 128 columns: lane j sums columns 4j..4j+3 over every eighth row, then the eight warps are added in
// order (fixed order: deterministic).
__global__ void __launch_bounds__(256) k_grad_bias(const float *A, int lda, int n_out, int rows, int rows_per_split,
                                                   float *db, long long split_stride)
{
    __shared__ float red[8][128];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 128 + lane * 4;
    const int r0 = blockIdx.y * rows_per_split, r1 = min(rows, r0 + rows_per_split);
    const bool vec = (lda & 3) == 0 && c + 3 < n_out;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int r = r0 + warp; r < r1; r += 8) {
        const float *row = A + (size_t)r * lda + c;
        if (vec) {
            const float4 v = *reinterpret_cast<const float4 *>(row);
            a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
        } else {
            if (c < n_out) a0 += row[0];
            if (c + 1 < n_out) a1 += row[1];
            if (c + 2 < n_out) a2 += row[2];
            if (c + 3 < n_out) a3 += row[3];
        }
    }
    red[warp][lane * 4] = a0; red[warp][lane * 4 + 1] = a1; red[warp][lane * 4 + 2] = a2; red[warp][lane * 4 + 3] = a3;
    __syncthreads();
    if (threadIdx.x < 128) {
        const int o = blockIdx.x * 128 + threadIdx.x;
        float acc = 0.f;
        for (int w = 0; w < 8; ++w) acc += red[w][threadIdx.x];
        if (o < n_out) db[blockIdx.y * split_stride + o] = acc;
    }
}

// grad[i] = partial[0][i] + partial[1][i] + ... in split order
__global__ void k_sum_splits(const float *partial, int splits, long long n, float *grad)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int z = 0; z < splits; ++z) acc += partial[(size_t)z * n + i];
        grad[i] = acc;
    }
}

// Adam (Kingma & Ba 2015) on the packed master weights; the renderer's transposed copy is
// written in the same pass.
__global__ void k_adam(float *master, float *kernel_w, const float *grad, float *m, float *v, long long n, int L, int W,
                       float lr, float c1, float c2, int do_update)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float th = master[i];
        if (do_update) {
            float g = grad[i];
            float mi = 0.9f * m[i] + 0.1f * g;
            float vi = 0.999f * v[i] + 0.001f * g * g;
            m[i] = mi;
            v[i] = vi;
            th -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
            master[i] = th;
        }
        // packed index -> kernel layout index
        long long off = 0, j = i;
        int fi = kNedfIn;
        for (int l = 0; l <= L; ++l) {
            int fo = l < L ? W : 2;
            long long sz = (long long)fi * fo + fo;
            if (j < sz) {
                long long dst = j < (long long)fi * fo ? off + (j % fi) * fo + j / fi : off + j;
                kernel_w[dst] = th;
                break;
            }
            j -= sz;
            off += sz;
            fi = W;
        }
    }
}

template <int W>
static cudaError_t run_fwd_bwd(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                               const float *hit_star, long long start, long long n, int B, TrainScratch s)
{
    cudaStream_t st = L.stream;
    cudaError_t e = cudaMemsetAsync(L.loss, 0, sizeof(float) * 4, st);
    if (e != cudaSuccess) return e;
    k_count_hits<<<std::min(1024, (B + 255) / 256), 256, 0, st>>>(hit_star, start, n, B, L.loss);
    size_t sm = (size_t)(W > kNedfInPad ? W : kNedfInPad) * kXStride * sizeof(float);
    if ((e = cudaFuncSetAttribute(k_train_fwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_train_bwd<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
        return e;
    int tiles = (B + kTileRows - 1) / kTileRows;
    int grid = std::min(tiles, L.num_sms * 4);
    k_train_fwd<W><<<grid, kThreads, sm, st>>>(L.type, L.rb, L.hidden, L.kernel_w, o, d, m_star, hit_star, start, n,
                                                B, s, L.loss);
    // zero bias vector for the backward products
    float *zero = s.zero;
    if ((e = cudaMemsetAsync(zero, 0, sizeof(float) * 512, st)) != cudaSuccess)
        return e;
    k_train_bwd<W><<<grid, kThreads, sm, st>>>(L.hidden, L.master, B, s, zero);
    // weight gradients: layer l uses dz_l (or dy for the output layer) against h_l
    const int split_rows = kSplitRows;
    int splits = (B + split_rows - 1) / split_rows;
    long long off = 0;
    int fi = kNedfIn;
    for (int l = 0; l <= L.hidden; ++l) {
        int fo = l < L.hidden ? W : 2;
        const float *A = l < L.hidden ? s.dz[l] : s.dy;
        int lda = fo;
        const float *Bm = s.h[l];
        int ldb = l == 0 ? kNedfInPad : W;
        dim3 g((fo + 63) / 64, (fi + 63) / 64, splits);
        k_grad_atb<<<g, 256, 0, st>>>(A, lda, Bm, ldb, fo, fi, B, split_rows, s.partial + off, L.n_params);
        dim3 gb((fo + 127) / 128, splits);
        k_grad_bias<<<gb, 256, 0, st>>>(A, lda, fo, B, split_rows, s.partial + off + (long long)fi * fo, L.n_params);
        off += (long long)fi * fo + fo;
        fi = W;
    }
    k_sum_splits<<<(int)std::min<long long>((L.n_params + 255) / 256, (long long)L.num_sms * 8), 256, 0, st>>>(
        s.partial, splits, L.n_params, s.grad);
    return cudaGetLastError();
}

static cudaError_t fwd_bwd(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                           const float *hit_star, long long start, long long n, int B, TrainScratch s)
{
    switch (L.width) {
    case 64: return run_fwd_bwd<64>(L, o, d, m_star, hit_star, start, n, B, s);
    case 128: return run_fwd_bwd<128>(L, o, d, m_star, hit_star, start, n, B, s);
    case 256: return run_fwd_bwd<256>(L, o, d, m_star, hit_star, start, n, B, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_loss_grad(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                             const float *hit_star, int n, float *grad)
{
    TrainScratch s = carve(L.scratch, n, L.hidden, L.width, L.n_params);
    cudaError_t e = fwd_bwd(L, o, d, m_star, hit_star, 0, n, n, s);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(grad, s.grad, sizeof(float) * L.n_params, cudaMemcpyDeviceToDevice, L.stream);
}

cudaError_t launch_train_step(const TrainLaunch &L, const float *o, const float *d, const float *m_star,
                              const float *hit_star, long long n_rays, long long start, int batch, float *adam_m,
                              float *adam_v, int step, float lr)
{
    TrainScratch s = carve(L.scratch, batch, L.hidden, L.width, L.n_params);
    cudaError_t e = fwd_bwd(L, o, d, m_star, hit_star, start, n_rays, batch, s);
    if (e != cudaSuccess) return e;
    return launch_adam(L, s.grad, adam_m, adam_v, step, lr);
}

cudaError_t launch_adam(const TrainLaunch &L, const float *grad, float *adam_m, float *adam_v, int step, float lr)
{
    float c1 = (float)(1.0 - std::pow(0.9, step)), c2 = (float)(1.0 - std::pow(0.999, step));
    int blocks = (int)std::min<long long>((L.n_params + 255) / 256, (long long)L.num_sms * 8);
    k_adam<<<blocks, 256, 0, L.stream>>>(L.master, L.kernel_w, grad, adam_m, adam_v, L.n_params, L.hidden, L.width,
                                         lr, c1, c2, 1);
    return cudaGetLastError();
}

cudaError_t launch_refresh_weights(const TrainLaunch &L)
{
    int blocks = (int)std::min<long long>((L.n_params + 255) / 256, (long long)L.num_sms * 8);
    k_adam<<<blocks, 256, 0, L.stream>>>(L.master, L.kernel_w, nullptr, nullptr, nullptr, L.n_params, L.hidden,
                                         L.width, 0.0f, 1.0f, 1.0f, 0);
    return cudaGetLastError();
}

}  // namespace nedf
