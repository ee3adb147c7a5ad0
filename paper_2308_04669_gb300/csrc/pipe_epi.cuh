// Pieces of the tensor-core MLP engines shared by the one-SM engines (render_pipe.cu) and the
// SM-pair NeRF engine (render_pair.cu): tile shapes, the weight-blob offsets, the input encodings,
// the A-operand row stores and the layer epilogues (TMEM -> ReLU / rounding -> next A operand, or
// the output-layer fold).
#pragma once

#include "pipe_common.cuh"

namespace nedf {

using namespace tc;

// NERF: the colour network (90 inputs padded to 96, 3 outputs); otherwise the NeDF (78 -> 80, 2).
// F8: hidden layers after the first in E4M3 (first layer BF16; output layer on CUDA cores).
template <int N, bool NERF, bool F8>
struct PipeShape {
    static constexpr int K0 = NERF ? kNerfInPad : kNedfInPad;        // input width of layer 0
    // BF16: the bias of every layer is folded into its MMAs: two constant-one input columns times
    // the bias split into BF16 high and low parts.  Layer 0 has them inside its input padding;
    // hidden layers read them from a 16-column block at ONES, after every column a layer writes.
    // F8: layer 0 as in BF16; later biases are added (with the layer's scale) in the epilogue.
    static constexpr int ONES = K0 > N ? K0 : N;
    static constexpr int A_ROW = F8 ? (2 * K0 > N ? 2 * K0 : N) : 2 * (ONES + kKC);   // A bytes per row
    static constexpr int CHUNK = N * 32;                             // N x 16 BF16 or N x 32 E4M3
    static constexpr int RING = F8 ? (N == 64 ? 65536 : 131072) : (N == 128 ? 98304 : 65536);   // ring bytes
    static constexpr int SMAX = RING / CHUNK;                        // stages at one chunk per stage
    static constexpr int NOUT = NERF ? 3 : 2;
    static constexpr size_t A_BYTES = (size_t)kHalf * A_ROW;
    static constexpr size_t FIXED = 2 * A_BYTES + (size_t)RING;      // + the fp32 block (depends on L)
};

// ---- weight blobs: per layer, chunks of 32 bytes of input per output row, each chunk N rows in the
// core-matrix layout (SBO 256 bytes).  Layer 0 (BF16) has K0 / 16 chunks with the bias in input
// columns K_in, K_in + 1 (high and low BF16 parts).  A BF16 hidden layer has N / 16 chunks plus
// one bias chunk (columns 0, 1); an E4M3 hidden layer has N / 32 chunks of W / s_l.  Then the fp32
// block: [w_out n_out x N (BF16 values)][b_out], and for E4M3 at pipe_f8_bias_off
// [bias L x N (row 0 unused)][s_l, L values (s_0 unused)].
__host__ __device__ inline size_t pipe_layer_off(int K0, int N, int l, bool f8)
{
    return l == 0 ? 0 : (size_t)K0 * N * 2 + (size_t)(l - 1) * (f8 ? (size_t)N * N : (size_t)(N + kKC) * N * 2);
}
__host__ __device__ inline size_t pipe_w_bytes(int K0, int N, int L, bool f8) { return pipe_layer_off(K0, N, L, f8); }
__host__ __device__ inline size_t pipe_f8_bias_off(int N, int n_out) { return ((size_t)n_out * N + n_out + 3) & ~(size_t)3; }
__host__ __device__ inline size_t pipe_f32_floats(int N, int L, int n_out, bool f8)
{
    const size_t b = pipe_f8_bias_off(N, n_out);
    return f8 ? (b + (size_t)L * N + L + 3) & ~(size_t)3 : b;
}
// ---- encodings into a BF16 A row (identity, sine blocks, cosine blocks; 2^k frequencies from the
// double-angle identities applied to sincos(x)) ---------------------------------------------------
template <int NIN, int F>
__device__ __forceinline__ void pipe_encode(const float *x, float *out)
{
#pragma unroll
    for (int c = 0; c < NIN; ++c) out[c] = x[c];
#pragma unroll
    for (int c = 0; c < NIN; ++c) {
        float s, co;
        sincosf(x[c], &s, &co);
#pragma unroll
        for (int k = 0; k < F; ++k) {
            out[NIN + k * NIN + c] = s;
            out[NIN + F * NIN + k * NIN + c] = co;
            float s2 = 2.0f * s * co;
            float c2 = (co - s) * (co + s);
            s = s2;
            co = c2;
        }
    }
}


// The same layout for E4M3 activations: 16 columns per 16-byte slice, slice stride 2048; one
// K = 32 MMA step again reads two slices (4 KB).
__device__ __forceinline__ uint32_t a_offset8(int r, int k)
{
    return (uint32_t)((k >> 4) * 2048 + (r >> 3) * 128 + (r & 7) * 16 + (k & 15));
}

// KG: bytes between 8-column groups (2048 for a 128-row half; 4096 for the 256 rows of a swapped
// NeDF tile, whose B operand spans both halves)
template <int K, int KG = 2048>
__device__ __forceinline__ void pipe_store_row(uint8_t *A, int r, const float *f, int n_valid)
{
#pragma unroll
    for (int c = 0; c < K / 8; ++c) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = c * 8 + 2 * e;
            // inputs, then the two constant-one columns the layer-0 bias is folded into, then zeros
            const float v0 = k < n_valid ? f[k] : (k < n_valid + 2 ? 1.0f : 0.0f);
            const float v1 = k + 1 < n_valid ? f[k + 1] : (k + 1 < n_valid + 2 ? 1.0f : 0.0f);
            p[e] = pack_bf16(v0, v1);
        }
        *reinterpret_cast<uint4 *>(A + (uint32_t)(c * KG + (r >> 3) * 128 + (r & 7) * 16)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
}

// ReLU and BF16 of 32 accumulator columns of this thread's row (the bias is already in them),
// stored as A columns [c0, c0 + 32) of row r.
__device__ __forceinline__ void epi_convert(const uint32_t (&v)[32], uint8_t *A, int r, int c0)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t *u = v + 8 * q;
        uint4 pk;
        pk.x = pack_bf16_relu(__uint_as_float(u[0]), __uint_as_float(u[1]));
        pk.y = pack_bf16_relu(__uint_as_float(u[2]), __uint_as_float(u[3]));
        pk.z = pack_bf16_relu(__uint_as_float(u[4]), __uint_as_float(u[5]));
        pk.w = pack_bf16_relu(__uint_as_float(u[6]), __uint_as_float(u[7]));
        *reinterpret_cast<uint4 *>(A + a_offset(r, c0 + 8 * q)) = pk;
    }
}

// E4M3 activations: x = acc (AFF false: bias already in it) or acc * s + bias (AFF), then ReLU and
// E4M3 of 32 columns, stored as A columns [c0, c0 + 32) of row r.
template <bool AFF>
__device__ __forceinline__ float epi_affine(uint32_t u, const float *bias, int j, float s)
{
    return AFF ? fmaf(__uint_as_float(u), s, bias[j]) : __uint_as_float(u);
}

template <bool AFF>
__device__ __forceinline__ void epi_convert8(const uint32_t (&v)[32], const float *bias, float s, uint8_t *A, int r, int c0)
{
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int j = 4 * q;
        w[q] = pack_e4m3_relu(epi_affine<AFF>(v[j], bias, j, s), epi_affine<AFF>(v[j + 1], bias, j + 1, s)) |
               (pack_e4m3_relu(epi_affine<AFF>(v[j + 2], bias, j + 2, s), epi_affine<AFF>(v[j + 3], bias, j + 3, s)) << 16);
    }
    *reinterpret_cast<uint4 *>(A + a_offset8(r, c0)) = make_uint4(w[0], w[1], w[2], w[3]);
    *reinterpret_cast<uint4 *>(A + a_offset8(r, c0 + 16)) = make_uint4(w[4], w[5], w[6], w[7]);
}

// Last hidden layer: ReLU and BF16 rounding of 32 columns, folded into the NOUT outputs (w_out
// rows of length N; 16-byte aligned at every multiple of 4 columns).  The weights are read four
// columns per load; the FMAs run in column order, so the sums are those of a column-by-column loop.
template <int NOUT, int N>
__device__ __forceinline__ void epi_output(const uint32_t (&v)[32], const float *wout, float *out)
{
#pragma unroll
    for (int jj = 0; jj < 32; jj += 4) {
        float4 w[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) w[o] = *reinterpret_cast<const float4 *>(wout + o * N + jj);
        const uint32_t p0 = pack_bf16_relu(__uint_as_float(v[jj]), __uint_as_float(v[jj + 1]));
        const uint32_t p1 = pack_bf16_relu(__uint_as_float(v[jj + 2]), __uint_as_float(v[jj + 3]));
        const float h0 = __uint_as_float(p0 << 16), h1 = __uint_as_float(p0 & 0xFFFF0000u);
        const float h2 = __uint_as_float(p1 << 16), h3 = __uint_as_float(p1 & 0xFFFF0000u);
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            out[o] = fmaf(h1, w[o].y, fmaf(h0, w[o].x, out[o]));
            out[o] = fmaf(h3, w[o].w, fmaf(h2, w[o].z, out[o]));
        }
    }
}

// The same with E4M3 rounding of the last hidden activation (bias and weights four columns per
// load).
template <int NOUT, int N, bool AFF>
__device__ __forceinline__ void epi_output8(const uint32_t (&v)[32], const float *bias, float s, const float *wout, float *out)
{
#pragma unroll
    for (int jj = 0; jj < 32; jj += 4) {
        float4 w[NOUT];
#pragma unroll
        for (int o = 0; o < NOUT; ++o) w[o] = *reinterpret_cast<const float4 *>(wout + o * N + jj);
        const float4 b = AFF ? *reinterpret_cast<const float4 *>(bias + jj) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float x0 = AFF ? fmaf(__uint_as_float(v[jj]), s, b.x) : __uint_as_float(v[jj]);
        const float x1 = AFF ? fmaf(__uint_as_float(v[jj + 1]), s, b.y) : __uint_as_float(v[jj + 1]);
        const float x2 = AFF ? fmaf(__uint_as_float(v[jj + 2]), s, b.z) : __uint_as_float(v[jj + 2]);
        const float x3 = AFF ? fmaf(__uint_as_float(v[jj + 3]), s, b.w) : __uint_as_float(v[jj + 3]);
        float h0, h1, h2, h3;
        unpack_e4m3(pack_e4m3_relu(x0, x1), h0, h1);
        unpack_e4m3(pack_e4m3_relu(x2, x3), h2, h3);
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            out[o] = fmaf(h1, w[o].y, fmaf(h0, w[o].x, out[o]));
            out[o] = fmaf(h3, w[o].w, fmaf(h2, w[o].z, out[o]));
        }
    }
}

// One layer's epilogue over the N accumulator columns of this thread's row, TMEM loads
// double-buffered (block b + 1 loads while block b is converted).  LAST: fold into the outputs;
// otherwise write the next layer's A operand (BF16, or E4M3 when F8).
template <int N, int NOUT, bool F8, bool AFF, bool LAST>
__device__ __forceinline__ void epi_layer(uint32_t tmem_row, uint8_t *Ag, int r, const float *bias, float s,
                                          const float *wout, float *out)
{
    uint32_t va[32], vb[32];
    tmem_ld32(tmem_row, va);
    tmem_wait_ld(va);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 64) {
        tmem_ld32(tmem_row + c0 + 32, vb);
        if (LAST) {
            if (F8) epi_output8<NOUT, N, AFF>(va, bias + c0, s, wout + c0, out);
            else epi_output<NOUT, N>(va, wout + c0, out);
        } else {
            if (F8) epi_convert8<AFF>(va, bias + c0, s, Ag, r, c0);
            else epi_convert(va, Ag, r, c0);
        }
        tmem_wait_ld(vb);
        if (c0 + 64 < N) tmem_ld32(tmem_row + c0 + 64, va);
        if (LAST) {
            if (F8) epi_output8<NOUT, N, AFF>(vb, bias + c0 + 32, s, wout + c0 + 32, out);
            else epi_output<NOUT, N>(vb, wout + c0 + 32, out);
        } else {
            if (F8) epi_convert8<AFF>(vb, bias + c0 + 32, s, Ag, r, c0 + 32);
            else epi_convert(vb, Ag, r, c0 + 32);
        }
        if (c0 + 64 < N) tmem_wait_ld(va);
    }
}

// 32 rows of one feature (ReLU, BF16): four 16-byte vectors of eight rows, 128 bytes apart.
__device__ __forceinline__ void epi_rows8(const uint32_t (&v)[32], uint8_t *dst)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t *u = v + 8 * b;
        uint4 pk;
        pk.x = pack_bf16_relu(__uint_as_float(u[0]), __uint_as_float(u[1]));
        pk.y = pack_bf16_relu(__uint_as_float(u[2]), __uint_as_float(u[3]));
        pk.z = pack_bf16_relu(__uint_as_float(u[4]), __uint_as_float(u[5]));
        pk.w = pack_bf16_relu(__uint_as_float(u[6]), __uint_as_float(u[7]));
        *reinterpret_cast<uint4 *>(dst + b * 128) = pk;
    }
}

// Epilogue of a swapped NeDF layer (D = W H^T: TMEM lane = output feature f, column = tile row):
// the 128 columns from tcol are rows row0 .. row0 + 127.  Each value is ReLU'd, rounded to BF16 and
// stored as the next layer's B operand, MN-major: 16-feature chunk f / 16 at 8 KB steps, 8-feature
// group at 4 KB, feature f % 8 at 16 bytes, rows contiguous in 16-byte vectors of eight (128 bytes
// per 8-row group).  TMEM loads double-buffered as in epi_layer.
__device__ __forceinline__ void epi_swapped(uint32_t tcol, uint8_t *H, int f, int row0)
{
    uint8_t *dst = H + (f >> 4) * 8192 + ((f >> 3) & 1) * 4096 + (f & 7) * 16 + (row0 >> 3) * 128;
    uint32_t va[32], vb[32];
    tmem_ld32(tcol, va);
    tmem_wait_ld(va);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 64) {
        tmem_ld32(tcol + c0 + 32, vb);
        epi_rows8(va, dst + (c0 >> 3) * 128);
        tmem_wait_ld(vb);
        if (c0 + 64 < 128) tmem_ld32(tcol + c0 + 64, va);
        epi_rows8(vb, dst + ((c0 + 32) >> 3) * 128);
        if (c0 + 64 < 128) tmem_wait_ld(va);
    }
}
}  // namespace nedf
