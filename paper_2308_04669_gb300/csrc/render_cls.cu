// The paper's intersection network on the tensor cores (tcgen05/TMEM, BF16 operands, FP32
// accumulation): Section "Intersection network" (Eq. 3-4) and Appendix A.
//
// Network: 16 points on the ray's chord through the bound, each encoded with 10 frequencies
// (1008 inputs); a linear head to 256 features; 16 residual blocks h' = ReLU(h + W2 ReLU(W1 h + b1)
// + b2); two linear tails, 256 -> 65 (hit logit, 64 coarse bins) and 256 -> 128 (fine bins); the
// output is m = mu / l from the argmax bins (Eq. 4) and the hit logit, the same (m, a) pair the
// regression NeDF engine writes, so the decode, fallback and z-min that follow are shared.
//
// k_nedfc works on tiles of 256 rows held as two 128-row halves (one TMEM accumulator of 256
// columns each; all 512 columns), one tile at a time per CTA, in 37 steps of K = 256: four head
// passes (the 1008 inputs, padded to 16 x 64, do not fit the A buffer, so the epilogue encodes four
// points at a time), 32 body layers and the tail.  Every weight chunk (256 outputs x 16 inputs,
// 8 KB) feeds one M = 128, N = 256 MMA per half.
//   warps 0-3 / 4-7  epilogue of rows 0..127 / 128..255: encoding, then per step tcgen05.ld of
//                    the accumulator, bias (the tile type's FP32 biases, kept in shared memory),
//                    ReLU, BF16, next A operand in shared memory;
//   warp 8           producer: the type's weight chunks, step after step, through the stage ring;
//   warp 9           MMA issuer and TMEM owner.
// Residual stream: a block's input h is the A operand of W1 (BF16).  W1's epilogue reads it back
// from shared memory, writes h + b2 into the accumulator columns it has just read (tcgen05.st),
// and overwrites h with t = BF16(ReLU(W1 h + b1)); W2's MMAs then accumulate onto h + b2, so the
// skip connection costs no shared memory (one A buffer per half) and the sum is FP32.  Every wait
// is bounded, as in the other engines.
#include "pipe_common.cuh"
#include "render_launch.h"

#include <algorithm>

namespace nedf {

constexpr int kClsSteps = 37;               // 4 head passes, 32 body layers, the tail
constexpr int kClsHeadPasses = 4;
constexpr int kClsChunks = 16;              // chunks per step (K = 256)
constexpr int kClsChunkBytes = 8192;        // 256 outputs x 16 BF16 inputs
constexpr int kClsW = 256;
constexpr int kClsNC = 64, kClsNF = 128;
constexpr size_t kClsWBytes = (size_t)kClsSteps * kClsChunks * kClsChunkBytes;
constexpr int kClsBiasRows = 34;            // head, 32 body layers, tail (193 of 256 used)
constexpr size_t kClsABytes = 65536;        // one half's A operand: 128 rows x 256 BF16
constexpr int kClsRing = 65536;
constexpr int kClsSMax = kClsRing / kClsChunkBytes;
constexpr size_t kClsBiasBytes = (size_t)kClsBiasRows * kClsW * 4;
constexpr size_t kClsSmem = 2 * kClsABytes + kClsRing + kClsBiasBytes;   // + the type's FP32 biases

// Packed FP32 master layout (W[out][in] then b[out]): head, 16 x (W1, b1, W2, b2), tail A, tail B.
constexpr long long kClsHeadW = (long long)kClsIn * kClsW;
constexpr long long kClsBlock0 = kClsHeadW + kClsW;
constexpr long long kClsLayer = (long long)kClsW * kClsW + kClsW;
constexpr long long kClsTailA = kClsBlock0 + 32 * kClsLayer;
constexpr long long kClsTailB = kClsTailA + (long long)(1 + kClsNC) * (kClsW + 1);
static_assert(kClsTailB + (long long)kClsNF * (kClsW + 1) == kClsParams, "classifier parameter count");

size_t cls_blob_size() { return (kClsWBytes + (size_t)kClsBiasRows * kClsW * 4 + 1023) & ~(size_t)1023; }

// Blob: step s, chunk c = 16 consecutive inputs of the step, in the core-matrix layout of a B
// operand (256 output rows, SBO 256, LBO 128).  Head pass s covers input columns 256 s .. 256 s + 255
// of the padded input (point j at columns 64 j .. 64 j + 62, column 64 j + 63 zero).  The tail's 256
// outputs: hit logit, 64 coarse, 128 fine, 63 zero rows.  Then FP32 biases, one row of 256 per
// step after the head passes (row 0: head; 1..32: body layers; 33: tail).
__global__ void k_pack_cls(const float *master, uint8_t *blob)
{
    const long long n_w = (long long)kClsSteps * kClsChunks * 256 * 16;
    const long long total = n_w + (long long)kClsBiasRows * kClsW;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < n_w) {
            const int k = (int)(e & 15), n = (int)((e >> 4) & 255);
            const long long sc = e >> 12;
            const int c = (int)(sc % kClsChunks), s = (int)(sc / kClsChunks);
            const int kk = 16 * c + k;                   // input column within the step
            float v = 0.0f;
            if (s < kClsHeadPasses) {
                const int col = 256 * s + kk, j = col >> 6, f = col & 63;
                if (f < 63) v = master[(long long)n * kClsIn + 63 * j + f];
            } else if (s < kClsSteps - 1) {
                const int l = s - kClsHeadPasses;
                v = master[kClsBlock0 + (long long)l * kClsLayer + (long long)n * kClsW + kk];
            } else if (n < 1 + kClsNC) {
                v = master[kClsTailA + (long long)n * kClsW + kk];
            } else if (n < 1 + kClsNC + kClsNF) {
                v = master[kClsTailB + (long long)(n - 1 - kClsNC) * kClsW + kk];
            }
            *reinterpret_cast<__nv_bfloat16 *>(blob + (size_t)sc * kClsChunkBytes + cm_offset(n, k, kKC)) =
                __float2bfloat16_rn(v);
        } else {
            const long long q = e - n_w;
            const int row = (int)(q / kClsW), n = (int)(q % kClsW);
            float v = 0.0f;
            if (row == 0) v = master[kClsHeadW + n];
            else if (row <= 32) v = master[kClsBlock0 + (long long)(row - 1) * kClsLayer + (long long)kClsW * kClsW + n];
            else if (n < 1 + kClsNC) v = master[kClsTailA + (long long)(1 + kClsNC) * kClsW + n];
            else if (n < 1 + kClsNC + kClsNF) v = master[kClsTailB + (long long)kClsNF * kClsW + (n - 1 - kClsNC)];
            reinterpret_cast<float *>(blob + kClsWBytes)[q] = v;
        }
    }
}

cudaError_t launch_pack_cls(const float *master, void *blob, cudaStream_t st)
{
    k_pack_cls<<<2048, 256, 0, st>>>(master, (uint8_t *)blob);
    return cudaGetLastError();
}

// ---- epilogue pieces (one thread = one row of its half) -------------------------------------------
// Encoded points 4p .. 4p + 3 of this row as A columns 0..255: per point [x, sin(2^k x), cos(2^k x)]
// (k = 0..9, coordinate fastest) and a zero.  sin/cos of 2^k x come from sincosf at k = 0 and 5 and
// the double-angle identities in between (at most four doublings: about 16 ulp, far below a BF16
// step).
__device__ __forceinline__ void cls_encode_pass(uint8_t *A, int r, V3 pe, V3 step, int p, bool valid)
{
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        float f[64];
        const V3 x = madd(pe, (float)(4 * p + q), step);
        const float xs[3] = {x.x, x.y, x.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            f[c] = xs[c];
            float s = 0.f, co = 1.f;
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                if (k == 0 || k == 5) {
                    sincosf(ldexpf(xs[c], k), &s, &co);
                } else {
                    const float s2 = 2.0f * s * co, c2 = (co - s) * (co + s);
                    s = s2;
                    co = c2;
                }
                f[3 + 3 * k + c] = s;
                f[33 + 3 * k + c] = co;
            }
        }
        f[63] = 0.0f;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
            uint4 pk;
            pk.x = valid ? pack_bf16(f[8 * g + 0], f[8 * g + 1]) : 0u;
            pk.y = valid ? pack_bf16(f[8 * g + 2], f[8 * g + 3]) : 0u;
            pk.z = valid ? pack_bf16(f[8 * g + 4], f[8 * g + 5]) : 0u;
            pk.w = valid ? pack_bf16(f[8 * g + 6], f[8 * g + 7]) : 0u;
            *reinterpret_cast<uint4 *>(A + a_offset(r, 64 * q + 8 * g)) = pk;
        }
    }
}

// The 256 accumulator columns of this thread's row, 32 at a time, TMEM loads double-buffered;
// fn(c0, v) gets columns c0 .. c0 + 31.
template <typename F>
__device__ __forceinline__ void cls_rows(uint32_t trow, F &&fn)
{
    uint32_t va[32], vb[32];
    tmem_ld32(trow, va);
    tmem_wait_ld(va);
#pragma unroll 1
    for (int c0 = 0; c0 < kClsW; c0 += 64) {
        tmem_ld32(trow + c0 + 32, vb);
        fn(c0, va);
        tmem_wait_ld(vb);
        if (c0 + 64 < kClsW) tmem_ld32(trow + c0 + 64, va);
        fn(c0 + 32, vb);
        if (c0 + 64 < kClsW) tmem_wait_ld(va);
    }
}

__device__ __forceinline__ float u2f(uint32_t u) { return __uint_as_float(u); }

// 32 values (plus bias, optional ReLU) rounded to BF16 as A columns c0 .. c0 + 31 of row r.
template <bool RELU>
__device__ __forceinline__ void cls_store(uint8_t *A, int r, int c0, const uint32_t (&v)[32], const float *b)
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float x[8];
        float4 b0 = make_float4(0.f, 0.f, 0.f, 0.f), b1 = b0;
        if (b) {
            b0 = *reinterpret_cast<const float4 *>(b + c0 + 8 * q);
            b1 = *reinterpret_cast<const float4 *>(b + c0 + 8 * q + 4);
        }
        const float bb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = u2f(v[8 * q + e]) + bb[e];
        uint4 pk;
        if (RELU) {
            pk.x = pack_bf16_relu(x[0], x[1]); pk.y = pack_bf16_relu(x[2], x[3]);
            pk.z = pack_bf16_relu(x[4], x[5]); pk.w = pack_bf16_relu(x[6], x[7]);
        } else {
            pk.x = pack_bf16(x[0], x[1]); pk.y = pack_bf16(x[2], x[3]);
            pk.z = pack_bf16(x[4], x[5]); pk.w = pack_bf16(x[6], x[7]);
        }
        *reinterpret_cast<uint4 *>(A + a_offset(r, c0 + 8 * q)) = pk;
    }
}

// W1's epilogue for columns c0 .. c0 + 31: h (this block's input, BF16 in A) + b2 into the
// accumulator columns just read, then t = BF16(ReLU(acc + b1)) over h in A.
__device__ __forceinline__ void cls_block_first(uint8_t *A, int r, int c0, const uint32_t (&v)[32], const float *b1,
                                                const float *b2, uint32_t tcol)
{
    uint32_t res[32];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 h = *reinterpret_cast<const uint4 *>(A + a_offset(r, c0 + 8 * q));
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        const float4 p0 = *reinterpret_cast<const float4 *>(b2 + c0 + 8 * q);
        const float4 p1 = *reinterpret_cast<const float4 *>(b2 + c0 + 8 * q + 4);
        const float bb[8] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 8 * q + 2 * e;
            res[j] = __float_as_uint(__uint_as_float(hw[e] << 16) + bb[2 * e]);
            res[j + 1] = __float_as_uint(__uint_as_float(hw[e] & 0xFFFF0000u) + bb[2 * e + 1]);
        }
    }
    cls_store<true>(A, r, c0, v, b1);
    tmem_st32(tcol, res);    // the caller waits for all of the layer's stores at once
}

// ---- the engine ------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1) k_nedfc(Workspace ws, PipeArgs a)
{
    static_assert(MODE == kModePrimary || MODE == kModeShadow || MODE == kModeQuery, "NeDF modes");
    const int GC = max(1, min(a.stage_bytes / kClsChunkBytes, kClsSMax / 2));
    const int STAGE = GC * kClsChunkBytes, S = kClsRing / STAGE;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ PipeShared P;
    __shared__ uint64_t w_full[kClsSMax], w_empty[kClsSMax];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint8_t *A[2] = {smem, smem + kClsABytes};
    uint8_t *ring = smem + 2 * kClsABytes;
    volatile int *abort = &P.abort;
    const MarchBuffers none{};

    if (warp == 9) tmem_alloc(&P.tmem_base, 2 * kClsW);
    if (threadIdx.x == 0) {
        mbar_init(&P.a_ready, 2 * kHalf);
        mbar_init(&P.acc_full, 1);
        mbar_init(&P.fin, 1);
        for (int s = 0; s < S; ++s) {
            mbar_init(&w_full[s], 1);
            mbar_init(&w_empty[s], 1);
        }
        P.abort = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = P.tmem_base;
    const unsigned long long n_tiles = pipe_n_tiles<kClsW, MODE>(ws, none, a);

    if (warp == 8) {
        // ------------------------------ producer ------------------------------------------------
        if (lane == 0) {
            unsigned long long q = 0;
            RingPos rp;
            for (unsigned long long tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
                const uint8_t *blob = a.blobs + (size_t)pipe_tile_type<MODE>(ws, none, a, tile) * a.blob_stride;
                for (int s = 0; s < kClsSteps && !*abort; ++s) {
                    const uint8_t *src = blob + (size_t)s * kClsChunks * kClsChunkBytes;
                    for (int c0 = 0; c0 < kClsChunks; c0 += GC, ++q, rp.next(S)) {
                        const int st = rp.st;
                        const uint32_t bytes = (uint32_t)(min(GC, kClsChunks - c0) * kClsChunkBytes);
                        if (!pipe_wait(&w_empty[st], rp.ph ^ 1u, abort, ws.status)) break;
                        mbar_arrive_expect_tx(&w_full[st], bytes);
                        bulk_g2s(ring + (size_t)st * STAGE, src + (size_t)c0 * kClsChunkBytes, bytes, &w_full[st]);
                    }
                }
            }
            const unsigned long long q0 = q > (unsigned long long)S ? q - S : 0;
            for (unsigned long long k = q0; k < q; ++k) pipe_drain(&w_full[k % S], (uint32_t)((k / S) & 1u), ws.status);
        }
    } else if (warp == 9) {
        // ------------------------------ MMA issuer ----------------------------------------------
        if (lane == 0) {
            unsigned long long ja = 0;
            RingPos rp;
            const uint32_t idesc = idesc_bf16(128, kClsW);
            const uint32_t ax = smem_addr(A[0]), ay = smem_addr(A[1]);
            bool issued_any = false;
            for (unsigned long long tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
                for (int s = 0; s < kClsSteps && !*abort; ++s, ++ja) {
                    if (!pipe_wait(&P.a_ready, (uint32_t)(ja & 1u), abort, ws.status)) break;
                    tc_fence_after();
                    // accumulate from the first chunk: later head passes, and W2 (onto h + b2)
                    const bool second = s >= kClsHeadPasses && s < kClsSteps - 1 && ((s - kClsHeadPasses) & 1);
                    const bool keep = (s > 0 && s < kClsHeadPasses) || second;
                    for (int c0 = 0; c0 < kClsChunks; c0 += GC, rp.next(S)) {
                        const int st = rp.st;
                        if (!pipe_wait(&w_full[st], rp.ph, abort, ws.status)) break;
                        const int c1 = min(kClsChunks, c0 + GC);
                        uint64_t bd = smem_desc(smem_addr(ring + (size_t)st * STAGE), 128, 256);
                        uint64_t adx = smem_desc(ax + (uint32_t)c0 * 4096u, 2048, 128);
                        uint64_t ady = smem_desc(ay + (uint32_t)c0 * 4096u, 2048, 128);
                        for (int c = c0; c < c1; ++c) {
                            const uint32_t acc = (keep || c > 0) ? 1u : 0u;
                            mma_bf16(tmem, adx, bd, idesc, acc);
                            mma_bf16(tmem + kClsW, ady, bd, idesc, acc);
                            adx += 4096u >> 4;
                            ady += 4096u >> 4;
                            bd += kClsChunkBytes >> 4;
                        }
                        mma_commit(&w_empty[st]);
                        issued_any = true;
                    }
                    mma_commit(&P.acc_full);
                }
            }
            if (issued_any) {
                mma_commit(&P.fin);
                pipe_drain(&P.fin, 0u, ws.status);
            }
        }
    } else {
        // ------------------------------ epilogue groups -----------------------------------------
        const int g = warp >> 2;
        const int r = threadIdx.x & 127;
        const int R = g * kHalf + r;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * kClsW);
        uint8_t *Ag = A[g];
        float *bias = reinterpret_cast<float *>(smem + 2 * kClsABytes + kClsRing);   // the tile type's biases
        int bias_type = -1;
        unsigned long long jb = 0;
        for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            if (epilogue_any(*abort != 0)) break;
            const int t = pipe_tile_type<MODE>(ws, none, a, tile);
            const DevType T = ws.types[t];
            if (t != bias_type) {
                // both groups are past every read of the previous type's biases before they are replaced
                asm volatile("bar.sync 3, 256;" ::: "memory");
                const float4 *src = reinterpret_cast<const float4 *>(a.blobs + (size_t)t * a.blob_stride + kClsWBytes);
                for (int i = threadIdx.x; i < kClsBiasRows * kClsW / 4; i += 2 * kHalf)
                    reinterpret_cast<float4 *>(bias)[i] = __ldg(src + i);
                asm volatile("bar.sync 3, 256;" ::: "memory");
                bias_type = t;
            }
            unsigned long long idx;
            bool valid;
            PairRay pr{};
            nedf_row<MODE>(ws, a, T, t, tile, R, idx, valid, pr);
            const bool enc = valid && pr.kept;
            // 16 points uniform over the chord [t_e, t_x] (t_x = 2 t_perp - t_e)
            const V3 pe = madd(pr.ol, pr.te, pr.dl);
            const V3 stp = enc ? v3(pr.dl.x * (2.0f / 15.0f) * (pr.tp - pr.te), pr.dl.y * (2.0f / 15.0f) * (pr.tp - pr.te),
                                    pr.dl.z * (2.0f / 15.0f) * (pr.tp - pr.te))
                               : v3(0.f, 0.f, 0.f);
            cls_encode_pass(Ag, r, pe, stp, 0, enc);
            fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(&P.a_ready);
            bool ok = true;
            float m_out = 0.f, a_out = 0.f;
            for (int s = 0; s < kClsSteps; ++s, ++jb) {
                ok = __all_sync(0xffffffffu, pipe_wait(&P.acc_full, (uint32_t)(jb & 1u), abort, ws.status));
                if (!ok) {
                    *abort = 1;
                    break;
                }
                tc_fence_after();
                if (s + 1 < kClsHeadPasses) {
                    cls_encode_pass(Ag, r, pe, stp, s + 1, enc);
                } else if (s + 1 == kClsHeadPasses) {
                    cls_rows(trow, [&](int c0, const uint32_t (&v)[32]) { cls_store<false>(Ag, r, c0, v, bias); });
                } else if (s + 1 < kClsSteps) {
                    const int l = s - kClsHeadPasses;              // body layer just computed
                    const float *bl = bias + (size_t)(1 + l) * kClsW;
                    if ((l & 1) == 0) {
                        cls_rows(trow, [&](int c0, const uint32_t (&v)[32]) {
                            cls_block_first(Ag, r, c0, v, bl, bl + kClsW, trow + c0);
                        });
                        tmem_wait_st();
                    } else {
                        cls_rows(trow, [&](int c0, const uint32_t (&v)[32]) { cls_store<true>(Ag, r, c0, v, nullptr); });
                    }
                } else {
                    // tail: hit logit, first maximum of the coarse and of the fine logits (Eq. 4)
                    const float *bt = bias + (size_t)33 * kClsW;       // shared memory
                    float bc = -INFINITY, bf = -INFINITY, al = 0.f;
                    int ic = 0, jf = 0;
                    cls_rows(trow, [&](int c0, const uint32_t (&v)[32]) {
#pragma unroll
                        for (int e = 0; e < 32; ++e) {
                            const int col = c0 + e;
                            const float x = u2f(v[e]) + bt[col];
                            if (col == 0) al = x;
                            else if (col <= kClsNC) { if (x > bc) { bc = x; ic = col - 1; } }
                            else if (col <= kClsNC + kClsNF) { if (x > bf) { bf = x; jf = col - 1 - kClsNC; } }
                        }
                    });
                    m_out = (float)(ic * kClsNF + jf) * (1.0f / (kClsNC * kClsNF / 2)) - 1.0f;
                    a_out = al;
                }
                if (s + 1 < kClsSteps) {
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(&P.a_ready);
                } else {
                    tc_fence_before();
                }
            }
            if (epilogue_any(!ok || *abort)) break;
            if (valid) {
                if (MODE == kModeQuery) {
                    float4 res = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
                    if (pr.kept) {
                        const float Dl = pr.tp - T.rb * m_out;
                        res = make_float4(m_out, a_out, Dl, (a_out > 0.f && Dl > 0.f) ? 1.f : 0.f);
                    }
                    a.qout[idx] = res;
                } else {
                    ws.nout[MODE == kModeShadow ? 1 : 0][idx] = make_float2(m_out, a_out);
                }
            }
        }
    }
    // ---- teardown ------------------------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 9) tmem_dealloc(tmem, 2 * kClsW);
}

template <int MODE>
static cudaError_t launch_cls(const Workspace &ws, const PipeArgs &a, int grid, cudaStream_t st)
{
    if (grid < 1) return cudaSuccess;
    PipeArgs args = a;
    args.stage_bytes = ws.pipe_stage_bytes[MODE] > 0 ? ws.pipe_stage_bytes[MODE] : kDefaultStageBytes;
    cudaError_t e = cudaFuncSetAttribute(k_nedfc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClsSmem);
    if (e != cudaSuccess) return e;
    k_nedfc<MODE><<<grid, kPipeThreads, kClsSmem, st>>>(ws, args);
    return cudaGetLastError();
}

cudaError_t launch_cls_pipe(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out, int n,
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
    if (mode == 0) return launch_cls<kModePrimary>(ws, a, num_sms, st);
    if (mode == 1) return launch_cls<kModeShadow>(ws, a, num_sms, st);
    const int grid = (int)std::min<long long>(num_sms, ((long long)n + kPipeRows - 1) / kPipeRows);
    return launch_cls<kModeQuery>(ws, a, grid, st);
}

}  // namespace nedf
