// Warp-specialised tensor-core MLP engines (tcgen05/TMEM; BF16, or E4M3 hidden layers) for every
// render-time network.
//
// Method: arXiv 2308.04669, Eq. 1-2 and 7 (NeDF queries of Steps 1 and 3), Eq. 8 with the sample
// window (the radiance field of Step 2), and the plain method's colour frame (its NeRF at every
// sample).
//
// k_pipe (the NeRF: shading and plain-method colour rows) works on tiles of 256 rows held as two
// 128-row halves X and Y, with one TMEM accumulator per half.  Each hidden layer is two tcgen05
// MMAs per weight chunk (M = 128, N = width), one per half, so every chunk fetched from L2 serves
// 256 rows.  Roles:
//   warps 0-3   epilogue group X: row set-up of rows 0..127, layer epilogues (tcgen05.ld, ReLU,
//               rounding, A operand in shared memory), output layer and tail;
//   warps 4-7   epilogue group Y: the same for rows 128..255 (TMEM lane quarter = warp % 4);
//   warp 8      producer: streams the weight chunks of every layer of every tile, in MMA order,
//               through a ring of shared-memory stages (one bulk asynchronous copy each: a copy
//               costs its issuing thread a few hundred cycles whatever its size);
//   warp 9      MMA issuer (and TMEM owner);
//   warps 10-11 (shading) prefetch: the next tile's row inputs (pixel, instance, depth, sample
//               position and density) into shared memory while the current tile's layers run.
// k_nedf2 (the NeDF, widths up to 128) keeps two such tiles in flight (see its own comment).
// The producer only waits for free stages, so while the epilogue warps work on layer l it is
// already loading layer l+1.  Every wait is bounded: a timeout sets the status word and an abort
// flag that ends every role's loop, and the teardown drains the kernel's own copies and MMAs
// (again bounded) before TMEM is freed.
#include "pipe_epi.cuh"
#include "render_launch.h"

#include <cuda_fp8.h>

#include <algorithm>

namespace nedf {

using namespace tc;

size_t pipe_blob_size(int K0, int N, int L, int n_out, bool f8)
{
    size_t b = pipe_w_bytes(K0, N, L, f8) + pipe_f32_floats(N, L, n_out, f8) * 4;
    return (b + 1023) & ~(size_t)1023;
}

// E4M3 layer scales: s_l = the power of two with max|W_l| / s_l in (224, 448] (1 for a zero layer),
// from the exponent of max|W_l| alone, so it is exact.  One block per hidden layer l >= 1.
__global__ void k_fp8_scales(const float *master, uint8_t *blob, int K_in, int K0, int N, int L, int n_out)
{
    const int l = 1 + blockIdx.x;
    const float *W = master + (size_t)K_in * N + N + (size_t)(l - 1) * ((size_t)N * N + N);
    float m = 0.0f;
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) m = fmaxf(m, fabsf(W[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
        float s = 1.0f;
        if (m > 0.0f) {
            int e;
            const float fm = frexpf(m, &e);         // m = fm 2^e, fm in [0.5, 1)
            // m / 2^k in (224, 448]: k = e - 9 when fm <= 7/8 (fm 512 <= 448), else e - 8
            s = ldexpf(1.0f, fm <= 0.875f ? e - 9 : e - 8);
        }
        float *f32 = reinterpret_cast<float *>(blob + pipe_w_bytes(K0, N, L, true));
        f32[pipe_f8_bias_off(N, n_out) + (size_t)L * N + l] = s;
        if (l == 1) f32[pipe_f8_bias_off(N, n_out) + (size_t)L * N] = 1.0f;
    }
}

// packed FP32 master (W[out][in] then b per layer) -> chunked blob; one thread per element.
// pair (width 256, the SM-pair engine): within each layer, the first 128 output rows of every
// chunk come first (chunk after chunk, 4 KB each), then the last 128 rows, so each SM of the pair
// streams its half of a layer from one contiguous range; each half-chunk keeps the core-matrix
// layout of 128 rows.
__global__ void k_pack_pipe(const float *master, uint8_t *blob, int K_in, int K0, int N, int L, int n_out, bool f8,
                            bool pair)
{
    const size_t wb = pipe_w_bytes(K0, N, L, f8);
    float *f32 = reinterpret_cast<float *>(blob + wb);
    const size_t boff = pipe_f8_bias_off(N, n_out);
    const long long KH = f8 ? N : N + kKC;
    const long long total_w = (long long)N * K0 + (long long)(L - 1) * N * KH;
    const long long n_f32 = (long long)n_out * N + n_out + (f8 ? (long long)L * N : 0);
    const long long total = total_w + n_f32;
    const long long off_out = (long long)K_in * N + N + (long long)(L - 1) * (N * N + N);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < total_w) {
            int l, K, Kin;
            long long j, off_w;
            if (e < (long long)N * K0) {
                l = 0; j = e; K = K0; Kin = K_in; off_w = 0;
            } else {
                const long long e2 = e - (long long)N * K0;
                l = 1 + (int)(e2 / ((long long)N * KH));
                j = e2 - (long long)(l - 1) * N * KH;
                K = (int)KH; Kin = N;
                off_w = (long long)K_in * N + N + (long long)(l - 1) * (N * N + N);
            }
            const int n = (int)(j / K), k = (int)(j - (long long)n * K);
            if (f8 && l > 0) {
                const float sc = f32[boff + (size_t)L * N + l];
                const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(master[off_w + (long long)n * Kin + k] / sc,
                                                                    __NV_SATFINITE, __NV_E4M3);
                const size_t in_chunk = ((size_t)(pair ? n & 127 : n) >> 3) * 256 + ((k & 31) >> 4) * 128 + (n & 7) * 16 + (k & 15);
                const size_t dst = pipe_layer_off(K0, N, l, true) +
                                   (pair ? (size_t)(n >> 7) * (N / 32) * 4096 + (size_t)(k / 32) * 4096
                                         : (size_t)(k / 32) * N * 32) + in_chunk;
                blob[dst] = (uint8_t)q;
                continue;
            }
            float v = 0.0f;
            if (k < Kin) {
                v = master[off_w + (long long)n * Kin + k];
            } else if (k < Kin + 2) {
                const float b = master[off_w + (long long)N * Kin + n];
                const float hi = round_bf16(b);
                v = k == Kin ? hi : b - hi;
            }
            const size_t dst = pipe_layer_off(K0, N, l, false) +
                               (pair ? (size_t)(n >> 7) * (K / kKC) * 4096 + (size_t)(k / kKC) * 4096 + cm_offset(n & 127, k % kKC, kKC)
                                     : (size_t)(k / kKC) * N * kKC * 2 + cm_offset(n, k % kKC, kKC));
            *reinterpret_cast<__nv_bfloat16 *>(blob + dst) = __float2bfloat16_rn(v);
        } else {
            const long long q = e - total_w;
            if (q < (long long)n_out * N) f32[q] = round_bf16(master[off_out + q]);
            else if (q < (long long)n_out * N + n_out) f32[q] = master[off_out + (long long)n_out * N + (q - (long long)n_out * N)];
            else {
                // E4M3 mode: the hidden biases, row l of [L x N] (row 0 is folded into layer 0)
                const long long qq = q - ((long long)n_out * N + n_out);
                const int l = (int)(qq / N), n = (int)(qq - (long long)l * N);
                f32[boff + qq] = l == 0 ? 0.0f : master[(long long)K_in * N + N + (long long)(l - 1) * (N * N + N) + (long long)N * N + n];
            }
        }
    }
}

cudaError_t launch_pack_pipe(const float *master, void *blob, int K_in, int K0, int N, int L, int n_out, bool f8,
                             bool pair, cudaStream_t st)
{
    if (f8 && L > 1) {
        k_fp8_scales<<<L - 1, 256, 0, st>>>(master, (uint8_t *)blob, K_in, K0, N, L, n_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long KH = f8 ? N : N + kKC;
    const long long total = (long long)N * K0 + (long long)(L - 1) * N * KH + (long long)n_out * N + n_out +
                            (f8 ? (long long)L * N : 0);
    k_pack_pipe<<<(int)std::min<long long>((total + 255) / 256, 4096), 256, 0, st>>>(master, (uint8_t *)blob, K_in, K0, N,
                                                                                     L, n_out, f8, pair && N == 256);
    return cudaGetLastError();
}


// MMAs of chunks [c0, c1) of one layer for the two 128-row halves (accumulators dx, dy; A operands
// at ax, ay; the stage's first chunk at `stage`).  Descriptors advance by constant steps of their
// start-address field (16-byte units), so the issuing thread spends a few instructions per MMA;
// chunk 0 overwrites the accumulators.  bias_chunk (-1: none) reads A at ones_off instead.
template <bool E4M3>
__device__ __forceinline__ void issue_chunks(uint32_t dx, uint32_t dy, uint32_t ax, uint32_t ay, uint32_t stage, int c0,
                                             int c1, int chunk_bytes, uint32_t idesc, int bias_chunk, uint32_t ones_off)
{
    uint64_t bd = smem_desc(stage, 128, 256);
    uint64_t adx = smem_desc(ax + (uint32_t)c0 * 4096u, 2048, 128), ady = smem_desc(ay + (uint32_t)c0 * 4096u, 2048, 128);
    const uint64_t bstep = (uint64_t)(chunk_bytes >> 4), astep = 4096u >> 4;
    for (int c = c0; c < c1; ++c) {
        if (c == bias_chunk) {
            adx = smem_desc(ax + ones_off, 2048, 128);
            ady = smem_desc(ay + ones_off, 2048, 128);
        }
        const uint32_t acc = c > 0 ? 1u : 0u;
        if (E4M3) {
            mma_e4m3(dx, adx, bd, idesc, acc);
            mma_e4m3(dy, ady, bd, idesc, acc);
        } else {
            mma_bf16(dx, adx, bd, idesc, acc);
            mma_bf16(dy, ady, bd, idesc, acc);
        }
        adx += astep;
        ady += astep;
        bd += bstep;
    }
}


// Inputs of row R of a NeRF tile: the sample's local position and direction (x6), its density
// (shade) or sample weight (march), and the keys the tail needs: for shading, the pixel and its
// sample length at slot [half * 128 + pixel-in-half] (written by the pixel's first sample row);
// for the plain method's colour rows, the row's pair (0xFFFFFFFF: none).  Invalid rows get zeros.
template <int MODE>
__device__ __forceinline__ void pipe_row_inputs(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a,
                                                const DevFrame &f, const DevType &T, int t, unsigned long long tile,
                                                int R, float *x6, float &sig, uint32_t *key, float *wd)
{
    for (int c = 0; c < 6; ++c) x6[c] = 0.f;
    sig = 0.f;
    const int g = R / kHalf, r = R - g * kHalf;
    if (MODE == kModeShade) {
        const int ns = f.n_shade;
        const int ppg = kHalf / ns;           // pixels per half
        const unsigned long long first = (tile - ws.cnt->h_tile[t]) * (unsigned long long)(2 * ppg) + g * ppg;
        const int q = r / ns, j = r - q * ns;
        if (q < ppg && first + q < ws.cnt->h_count[t]) {
            const uint32_t p = ws.hlist[(size_t)t * a.npix + first + q];
            const DevInst I = ws.inst[ws.id[p]];
            V3 o, d, ol, dl;
            camera_ray(f, p % f.W, p / f.W, o, d);
            to_local(I, o, d, ol, dl);
            const float Dl = ws.depth[p] / I.s;
            const float delta = 2.0f * f.shade_half / ns;
            const V3 x = madd(ol, Dl - f.shade_half + (j + 0.5f) * delta, dl);
            x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
            sig = density(T, x, f.sigma_max, f.sdf_width);
            if (j == 0) { key[g * kHalf + q] = p; wd[g * kHalf + q] = I.s * delta; }
        }
    } else {
        const unsigned long long end = min(mb.row_cursor[t], mb.row_off[t + 1]);
        const unsigned long long idx = mb.row_off[t] + (tile - mb.row_tile[t]) * kPipeRows + R;
        uint32_t pair = 0xFFFFFFFFu;
        if (idx < end) {
            const uint2 row = mb.rows[idx];
            const uint2 pp = ws.ppairs[row.x];
            const DevInst I = ws.inst[pp.y];
            V3 o, d, ol, dl;
            camera_ray(f, pp.x % f.W, pp.x / f.W, o, d);
            to_local(I, o, d, ol, dl);
            Chord ch;
            bound_chord(ol, dl, T.rb, ch);
            const float dt = (ch.tx - ch.te) / a.n_samples;
            float Tr = mb.T_first[row.x];
            for (int jj = mb.k_first[row.x]; jj < (int)row.y; ++jj)
                Tr *= expf(-density(T, madd(ol, ch.te + (jj + 0.5f) * dt, dl), f.sigma_max, f.sdf_width) * I.s * dt);
            const V3 x = madd(ol, ch.te + (row.y + 0.5f) * dt, dl);
            x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
            sig = Tr * (1.0f - expf(-density(T, x, f.sigma_max, f.sdf_width) * I.s * dt));
            pair = row.x;
        }
        key[R] = pair;
    }
}

template <int N, int MODE, bool F8>
__global__ void __launch_bounds__(kPipeThreadsPf, 1) k_pipe(Workspace ws, MarchBuffers mb, PipeArgs a)
{
    static_assert(MODE == kModeShade || MODE == kModeMarch, "the NeDF modes run in k_nedf2");
    constexpr bool NERF = true;
    using SH = PipeShape<N, NERF, F8>;
    constexpr int K0 = SH::K0, NOUT = SH::NOUT;
    // schedule: GC chunks per stage (at least 2 stages in the ring), S stages
    const int GC = max(1, min(a.stage_bytes / SH::CHUNK, SH::SMAX / 2));
    const int STAGE = GC * SH::CHUNK, S = SH::RING / STAGE;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ PipeShared P;
    __shared__ uint64_t w_full[SH::SMAX], w_empty[SH::SMAX];
    // tail scratch of the two groups (shading composite; plain-method per-pair sums)
    __shared__ float t_sig[kPipeRows], t_rgb[kPipeRows][3];
    __shared__ uint32_t t_key[kPipeRows];
    __shared__ float t_wd[kPipeRows];
    // the next tile's row inputs, computed by the prefetch warps while this tile's layers run
    __shared__ float pf_x[kPipeRows][6], pf_sig[kPipeRows], pf_wd[kPipeRows];
    __shared__ uint32_t pf_key[kPipeRows];
    __shared__ uint64_t pf_full, pf_empty;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = NERF ? ws.nerf_hidden : ws.nedf_hidden;
    uint8_t *A[2] = {smem, smem + SH::A_BYTES};
    uint8_t *ring = smem + 2 * SH::A_BYTES;
    float *f32s = reinterpret_cast<float *>(smem + SH::FIXED);       // output layer of one type
    const int n_f32 = (int)pipe_f32_floats(N, L, NOUT, F8);
    volatile int *abort = &P.abort;

    if (warp == 9) tmem_alloc(&P.tmem_base, 2 * N);
    if (threadIdx.x == 0) {
        mbar_init(&P.a_ready, 2 * kHalf);
        mbar_init(&P.acc_full, 1);
        mbar_init(&P.fin, 1);
        mbar_init(&pf_full, kPipeThreadsPf - kPipeThreads);
        mbar_init(&pf_empty, 2 * kHalf);
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
    const unsigned long long n_tiles = pipe_n_tiles<N, MODE>(ws, mb, a);
    const DevFrame &f = *ws.frame;

    if (warp == 8) {
        // ------------------------------ producer ------------------------------------------------
        if (lane == 0) {
            unsigned long long q = 0;
            RingPos rp;
            for (unsigned long long tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
                const uint8_t *blob = a.blobs + (size_t)pipe_tile_type<MODE>(ws, mb, a, tile) * a.blob_stride;
                for (int l = 0; l < L && !*abort; ++l) {
                    const uint8_t *src = blob + pipe_layer_off(K0, N, l, F8);
                    const int nk = l == 0 ? K0 / kKC : (F8 ? N / 32 : N / kKC + 1);
                    for (int c0 = 0; c0 < nk; c0 += GC, ++q, rp.next(S)) {
                        const int s = rp.st;
                        const uint32_t bytes = (uint32_t)(min(GC, nk - c0) * SH::CHUNK);
                        if (!pipe_wait(&w_empty[s], rp.ph ^ 1u, abort, ws.status)) break;
                        mbar_arrive_expect_tx(&w_full[s], bytes);
                        bulk_g2s(ring + (size_t)s * STAGE, src + (size_t)c0 * SH::CHUNK, bytes, &w_full[s]);
                    }
                }
            }
            // drain: the last (up to S) copies may still be landing
            const unsigned long long q0 = q > (unsigned long long)S ? q - S : 0;
            for (unsigned long long k = q0; k < q; ++k) pipe_drain(&w_full[k % S], (uint32_t)((k / S) & 1u), ws.status);
        }
    } else if (warp == 9) {
        // ------------------------------ MMA issuer ----------------------------------------------
        if (lane == 0) {
            unsigned long long ja = 0;
            RingPos rp;
            const uint32_t idesc = idesc_bf16(128, N), idesc8 = idesc_e4m3(128, N);
            bool issued_any = false;
            for (unsigned long long tile = blockIdx.x; tile < n_tiles && !*abort; tile += gridDim.x) {
                for (int l = 0; l < L && !*abort; ++l, ++ja) {
                    if (!pipe_wait(&P.a_ready, (uint32_t)(ja & 1u), abort, ws.status)) break;
                    tc_fence_after();
                    const uint32_t ax = smem_addr(A[0]), ay = smem_addr(A[1]);
                    const int nk = l == 0 ? K0 / kKC : (F8 ? N / 32 : N / kKC + 1);
                    const bool e4m3 = F8 && l > 0;
                    for (int c0 = 0; c0 < nk; c0 += GC, rp.next(S)) {
                        const int s = rp.st;
                        if (!pipe_wait(&w_full[s], rp.ph, abort, ws.status)) break;
                        const uint32_t stage = smem_addr(ring + (size_t)s * STAGE);
                        const int c1 = min(nk, c0 + GC);
                        if (e4m3) issue_chunks<true>(tmem, tmem + N, ax, ay, stage, c0, c1, SH::CHUNK, idesc8, -1, 0u);
                        else      // a BF16 hidden layer's last chunk is its bias, against the constant-one block
                            issue_chunks<false>(tmem, tmem + N, ax, ay, stage, c0, c1, SH::CHUNK, idesc,
                                                l > 0 ? N / kKC : -1, (uint32_t)(SH::ONES / kKC) * 4096u);
                        mma_commit(&w_empty[s]);      // the stage is free once its MMAs have read it
                        issued_any = true;
                    }
                    mma_commit(&P.acc_full);
                }
            }
            if (issued_any) {                         // everything issued has completed before TMEM goes
                mma_commit(&P.fin);
                pipe_drain(&P.fin, 0u, ws.status);
            }
        }
    } else if (warp >= 10) {
        // ------------------------------ prefetch warps ------------------------------------------
        // shading: each tile's row inputs (the global-load chain pixel -> instance -> depth, the
        // sample geometry and density) one tile ahead of the epilogue, into pf_*: 4 rows per thread.
        // The plain method's colour rows carry a transmittance loop over their earlier samples, too
        // much for 64 threads: their epilogue threads compute their own rows.
        const int pt = threadIdx.x - kPipeThreads;
        uint32_t ph = 0;
        for (unsigned long long tile = blockIdx.x; MODE == kModeShade && tile < n_tiles && !*abort;
             tile += gridDim.x, ph ^= 1u) {
            if (!pipe_wait(&pf_empty, ph ^ 1u, abort, ws.status)) break;
            const int t = pipe_tile_type<MODE>(ws, mb, a, tile);
            const DevType T = ws.types[t];
#pragma unroll
            for (int k = 0; k < kPipeRows / (kPipeThreadsPf - kPipeThreads); ++k) {
                const int R = pt + k * (kPipeThreadsPf - kPipeThreads);
                pipe_row_inputs<MODE>(ws, mb, a, f, T, t, tile, R, pf_x[R], pf_sig[R], pf_key, pf_wd);
            }
            mbar_arrive(&pf_full);
        }
    } else {
        // ------------------------------ epilogue groups -----------------------------------------
        const int g = warp >> 2;                      // 0: rows 0..127 (X), 1: rows 128..255 (Y)
        const int r = threadIdx.x & 127;              // row within the half
        const int R = g * kHalf + r;                  // row within the tile
        const uint32_t tmem_row = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(g * N);
        uint8_t *Ag = A[g];
        if (!F8) {
            // the constant-one block BF16 hidden-layer biases are folded into: columns ONES, ONES + 1
            *reinterpret_cast<uint4 *>(Ag + a_offset(r, SH::ONES)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
            *reinterpret_cast<uint4 *>(Ag + a_offset(r, SH::ONES + 8)) = make_uint4(0u, 0u, 0u, 0u);
        }
        unsigned long long jb = 0, pf_ph = 0;
        const int ns = f.n_shade;
        int f32_type = -1;
        const float *f32 = f32s;
        for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
            if (epilogue_any(*abort != 0)) break;
            const int t = pipe_tile_type<MODE>(ws, mb, a, tile);
            const DevType T = ws.types[t];
            if (t != f32_type) {
                // both groups are past every read of the previous type's block before it is replaced
                asm volatile("bar.sync 3, 256;" ::: "memory");
                const float4 *src = reinterpret_cast<const float4 *>(a.blobs + (size_t)t * a.blob_stride +
                                                                     pipe_w_bytes(K0, N, L, F8));
                for (int i = threadIdx.x; i < n_f32 / 4; i += 2 * kHalf)
                    reinterpret_cast<float4 *>(f32s)[i] = src[i];
                asm volatile("bar.sync 3, 256;" ::: "memory");
                f32_type = t;
            }
            // ---- row set-up: the prefetch warps' inputs for this tile ----------------------------
            float x6[6];
            float sig;                                // shade: density; march: sample weight
            if (MODE == kModeShade) {
                const bool okp = pipe_wait(&pf_full, (uint32_t)(pf_ph & 1u), abort, ws.status);
                ++pf_ph;
                if (epilogue_any(!okp)) {
                    *abort = 1;
                    break;
                }
#pragma unroll
                for (int c = 0; c < 6; ++c) x6[c] = pf_x[R][c];
                sig = pf_sig[R];
                t_key[R] = pf_key[R];
                t_wd[R] = pf_wd[R];
                mbar_arrive(&pf_empty);               // this thread is done with the buffer
            } else {
                pipe_row_inputs<MODE>(ws, mb, a, f, T, t, tile, R, x6, sig, t_key, t_wd);
            }
            {
                float feat[K0];
                pipe_encode<3, 10>(x6, feat);
                pipe_encode<3, 4>(x6 + 3, feat + 63);
                pipe_store_row<K0>(Ag, r, feat, kNerfIn);
            }
            fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(&P.a_ready);
            // ---- layers -------------------------------------------------------------------------
            float out[NOUT];
#pragma unroll
            for (int o = 0; o < NOUT; ++o) out[o] = f32[NOUT * N + o];
            bool ok = true;
            for (int l = 0; l < L; ++l, ++jb) {
                // a warp-uniform outcome: the tcgen05.ld below is warp-collective
                ok = __all_sync(0xffffffffu, pipe_wait(&P.acc_full, (uint32_t)(jb & 1u), abort, ws.status));
                if (!ok) {
                    *abort = 1;
                    break;
                }
                tc_fence_after();
                // E4M3 layers after the first take their scale and bias here (layer 0's bias rides in its MMA)
                const float *bias = f32 + pipe_f8_bias_off(N, NOUT) + (size_t)l * N;
                const float sc = F8 && l > 0 ? f32[pipe_f8_bias_off(N, NOUT) + (size_t)L * N + l] : 1.0f;
                if (l + 1 < L) {
                    if (F8 && l > 0) epi_layer<N, NOUT, F8, true, false>(tmem_row, Ag, r, bias, sc, f32, out);
                    else epi_layer<N, NOUT, F8, false, false>(tmem_row, Ag, r, bias, sc, f32, out);
                    fence_proxy_async_smem();
                    tc_fence_before();
                    mbar_arrive(&P.a_ready);
                } else {
                    if (F8 && l > 0) epi_layer<N, NOUT, F8, true, true>(tmem_row, Ag, r, bias, sc, f32, out);
                    else epi_layer<N, NOUT, F8, false, true>(tmem_row, Ag, r, bias, sc, f32, out);
                    tc_fence_before();
                }
            }
            // one outcome for both groups: the tails use named barriers and ballots
            if (epilogue_any(!ok || *abort)) break;
            // ---- tail ---------------------------------------------------------------------------
            {
                const float wr = MODE == kModeShade ? 1.0f : sig;
#pragma unroll
                for (int c = 0; c < 3; ++c) t_rgb[R][c] = wr / (1.0f + expf(-out[c]));
                t_sig[R] = sig;
                asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kHalf) : "memory");
                if (MODE == kModeShade) {
                    const int ppg = kHalf / ns;
                    const unsigned long long first = (tile - ws.cnt->h_tile[t]) * (unsigned long long)(2 * ppg) + g * ppg;
                    if (r < ppg && first + r < ws.cnt->h_count[t]) {
                        float Tr = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, Aa = 0.f, smax = 0.f;
                        const float wd = t_wd[g * kHalf + r];
                        for (int k = 0; k < ns; ++k) {
                            const int rr = g * kHalf + r * ns + k;
                            const float alpha = 1.0f - expf(-t_sig[rr] * wd);
                            const float w = Tr * alpha;
                            cr += w * t_rgb[rr][0]; cg += w * t_rgb[rr][1]; cb += w * t_rgb[rr][2]; Aa += w;
                            Tr *= 1.0f - alpha;
                            smax = fmaxf(smax, t_sig[rr]);
                        }
                        const uint32_t pix = t_key[g * kHalf + r];
                        ws.rgba[pix] = make_float4(cr, cg, cb, Aa);
                        flag_shade_outlier(ws, f, pix, smax);
                    }
                } else {
                    // one sum per run of rows of the same pair (runs are contiguous within a half)
                    const uint32_t pair = t_key[R];
                    if (pair != 0xFFFFFFFFu && (r == 0 || t_key[R - 1] != pair)) {
                        float sa = 0.f, sb = 0.f, sc = 0.f;
                        for (int k = R; k < (g + 1) * kHalf && t_key[k] == pair; ++k) {
                            sa += t_rgb[k][0]; sb += t_rgb[k][1]; sc += t_rgb[k][2];
                        }
                        atomicAdd(&mb.C[pair].x, sa);
                        atomicAdd(&mb.C[pair].y, sb);
                        atomicAdd(&mb.C[pair].z, sc);
                    }
                }
                asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kHalf) : "memory");
            }
        }
    }
    // ---- teardown ------------------------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 9) tmem_dealloc(tmem, 2 * N);
}

// ---------------------------------------------------------------------------------------------------
// NeDF engine with two tiles in flight (widths 64 and 128): TMEM holds the accumulators of two
// 256-row tiles (slots), so the tensor pipe works on one slot's layer while the epilogue warps
// convert the other slot's previous layer, and a slot's tail and next set-up overlap the other
// slot's MMAs.  The CTA's tiles alternate between the slots; the producer, the MMA issuer and the
// epilogue walk the same sequence (round r: for each layer l, slot 0 then slot 1).
//
// BF16 width 128 swaps the operands of every layer but the last: D^T = W H^T with the weight chunk
// as A (M = 128 output features) and the tile's 256 rows as B (N = 256), one MMA per chunk.  A
// thread issues a tcgen05.mma about every 50 cycles, so M = N = 128 MMAs (64 cycles of the pipe)
// leave the issuer no room for its waits and commits; N = 256 MMAs (128 cycles) do.  The swapped
// accumulator has a feature per TMEM lane and a tile row per column, so the epilogue thread of
// feature f writes the next layer's activations MN-major (eight rows per 16-byte vector).  Layer 0
// reads the encoded rows K-major (as the set-up writes them, one thread per row), and the last
// hidden layer runs unswapped (A = the MN-major activations of each half, B = the weight chunk) so
// that its accumulator is row-per-lane for the output fold and the tail.  The hidden biases fold
// into one more chunk whose B (or, unswapped, A) operand is a constant block of ones shared by both
// slots.
// ---------------------------------------------------------------------------------------------------
// SWAP (BF16 width 128 only): the operand order above; the autotuner picks it per NeDF mode (the
// unswapped order: A = each half's activations, B = the weight chunk, as at width 64 and in E4M3).
template <int N, bool F8, bool SWAP = (N == 128 && !F8)>
struct NedfShape2 {
    static_assert(!SWAP || (N == 128 && !F8), "swapped operands: BF16 width 128 only");
    using B = PipeShape<N, false, F8>;
    static constexpr bool SW = SWAP;                                         // swapped operands
    static constexpr size_t H_BYTES = 65536;        // swapped: 8 chunks x 256 rows x 16 BF16 columns
    static constexpr size_t ONES_BYTES = 8192;      // swapped: the bias chunk's constant operand
    // BF16 width 128: room for two whole 9-chunk layers (36 KB each), so a layer can be one stage
    static constexpr int RING = SW ? 81920 : F8 ? 131072 : (N == 128 ? 73728 : 65536);
    static constexpr int SMAX = RING / B::CHUNK;
    static constexpr size_t ACT = SW ? 2 * H_BYTES + ONES_BYTES : 4 * B::A_BYTES;
    static constexpr size_t FIXED = ACT + (size_t)RING;                     // + two fp32 blocks
};


// ---------------------------------------------------------------------------------------------------
// Decode of the NeDF outputs of every listed pair (Eq. 2 and 7): depth and hit, the confidence
// fallback, refinement and outlier re-answering, then the z-min (Step 1) or the occlusion bit
// (Step 3); pairs deferred to the plain method go to its list.  One thread per pair, after the
// engine (which only stores each pair's two outputs, keeping this work off its epilogue warps).
// ---------------------------------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256) k_nedf_decode(Workspace ws)
{
    static_assert(MODE == kModePrimary || MODE == kModeShadow, "listed pairs only");
    constexpr bool SHADOW = MODE == kModeShadow;
    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    const unsigned long long *off = SHADOW ? C.s_off : C.p_off;
    const int nt = f.n_types;
    const unsigned long long n = off[nt];
    const float4 *geo = SHADOW ? ws.sgeo : ws.pgeo;
    const uint2 *pairs = SHADOW ? ws.spairs : ws.ppairs;
    const float2 *nout = ws.nout[SHADOW ? 1 : 0];
    const int lane = threadIdx.x & 31;
    __shared__ unsigned s_cnt;
    __shared__ unsigned long long s_base;
    // the trip count is uniform within a block, so the ballot and the barriers below see whole
    // warps; deferred pairs are ranked inside the block (shared-memory atomics) and the block's
    // range of the plain method's list is reserved with one global atomic
    for (unsigned long long base = blockIdx.x * (unsigned long long)blockDim.x; base < n;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long idx = base + threadIdx.x;
        if (threadIdx.x == 0) s_cnt = 0u;
        __syncthreads();
        bool defer = false;
        if (idx < n) {
            int t = 0;
            while (t + 1 < nt && off[t + 1] <= idx) ++t;
            const DevType T = ws.types[t];
            const float4 g0 = geo[2 * idx], g1 = geo[2 * idx + 1];
            const uint2 pp = pairs[idx];
            const float2 o = nout[idx];
            PairRay pr;
            pr.ol = v3(g0.x, g0.y, g0.z);
            pr.te = g0.w;
            pr.dl = v3(g1.x, g1.y, g1.z);
            pr.tp = g1.w;
            pr.key = pp.x;
            pr.inst = pp.y;
            pr.s = ws.inst[pp.y].s;
            pr.ell = SHADOW ? ws.sell[idx] : 0.0f;
            pr.kept = true;
            float Dl;
            bool hit;
            defer = nedf_decode(f, T, pr.ol, pr.dl, pr.tp, o.x, o.y, Dl, hit);
            if (!defer && hit) apply_hit(ws, f, SHADOW, pr, Dl);
        }
        const unsigned m = __ballot_sync(0xffffffffu, defer);
        unsigned pos = 0;
        if (m) {
            const int leader = __ffs(m) - 1;
            if (lane == leader) pos = atomicAdd(&s_cnt, (unsigned)__popc(m));
            pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(m & ((1u << lane) - 1u));
        }
        __syncthreads();
        if (threadIdx.x == 0 && s_cnt) s_base = atomicAdd(&ws.cnt->fb_count[SHADOW ? 1 : 0], (unsigned long long)s_cnt);
        __syncthreads();
        if (defer) ws.fb_list[SHADOW ? 1 : 0][s_base + pos] = (uint32_t)idx;
    }
}

cudaError_t launch_nedf_decode(const Workspace &ws, int mode, int num_sms, cudaStream_t st)
{
    if (mode == 1) k_nedf_decode<kModeShadow><<<num_sms * 8, 256, 0, st>>>(ws);
    else k_nedf_decode<kModePrimary><<<num_sms * 8, 256, 0, st>>>(ws);
    return cudaGetLastError();
}

// A whole NeDF layer (one weight stage holds it) issued as a straight run of MMAs: descriptors
// advance by constant steps of their start-address field, with no per-MMA address selection (a
// per-chunk branch and descriptor rebuild in the issuing thread cost ≈ 40 cycles per MMA, enough
// to starve the tensor pipe).  Swapped operands: D^T (dx, 128 features x 256 rows) += W_c H_c^T with
// weight chunk c of the stage (A, 4 KB apart) and the slot's activation chunk c (B, 8 KB apart);
// BIAS: the last chunk reads the constant-one block instead.
template <int NK, bool BIAS>
__device__ __forceinline__ void issue_layer_swapped(uint32_t dx, uint64_t wd, uint32_t hs, uint32_t ones, uint32_t id)
{
    const uint64_t bd = smem_desc(hs, 4096, 128);
#pragma unroll
    for (int c = 0; c < (BIAS ? NK - 1 : NK); ++c)
        mma_bf16(dx, wd + (uint64_t)(c * (4096 >> 4)), bd + (uint64_t)(c * (8192 >> 4)), id, c > 0 ? 1u : 0u);
    if (BIAS) mma_bf16(dx, wd + (uint64_t)((NK - 1) * (4096 >> 4)), smem_desc(ones, 4096, 128), id, 1u);
}

// The same for the unswapped last hidden layer: each 128-row half (A: the MN-major activations,
// halves 2 KB apart) against weight chunk c (B), into dx and dy; the last chunk is the bias chunk.
template <int NK>
__device__ __forceinline__ void issue_layer_unswapped(uint32_t dx, uint32_t dy, uint64_t wd, uint32_t hs, uint32_t ones,
                                                      uint32_t id)
{
    const uint64_t ax = smem_desc(hs, 4096, 128), ay = smem_desc(hs + 2048u, 4096, 128);
#pragma unroll
    for (int c = 0; c < NK - 1; ++c) {
        mma_bf16(dx, ax + (uint64_t)(c * (8192 >> 4)), wd + (uint64_t)(c * (4096 >> 4)), id, c > 0 ? 1u : 0u);
        mma_bf16(dy, ay + (uint64_t)(c * (8192 >> 4)), wd + (uint64_t)(c * (4096 >> 4)), id, c > 0 ? 1u : 0u);
    }
    const uint64_t wl = wd + (uint64_t)((NK - 1) * (4096 >> 4));
    mma_bf16(dx, smem_desc(ones, 4096, 128), wl, id, 1u);
    mma_bf16(dy, smem_desc(ones + 2048u, 4096, 128), wl, id, 1u);
}

// The same straight run for the unswapped engine (128-row halves as A, weight chunks as B; E4M3
// hidden layers or width 64): NK chunks of chunk_bytes each; BIAS: the last chunk reads A from the
// constant-one columns at ones_off.
template <bool E4M3, int NK, bool BIAS>
__device__ __forceinline__ void issue_layer_halves(uint32_t dx, uint32_t dy, uint32_t ax, uint32_t ay, uint32_t stage,
                                                   uint32_t chunk_bytes, uint32_t idesc, uint32_t ones_off)
{
    const uint64_t bd = smem_desc(stage, 128, 256), adx = smem_desc(ax, 2048, 128), ady = smem_desc(ay, 2048, 128);
    const uint64_t bstep = (uint64_t)(chunk_bytes >> 4);
#pragma unroll
    for (int c = 0; c < NK; ++c) {
        const bool bias = BIAS && c == NK - 1;
        const uint64_t a0 = bias ? smem_desc(ax + ones_off, 2048, 128) : adx + (uint64_t)(c * (4096 >> 4));
        const uint64_t a1 = bias ? smem_desc(ay + ones_off, 2048, 128) : ady + (uint64_t)(c * (4096 >> 4));
        const uint32_t acc = c > 0 ? 1u : 0u;
        if (E4M3) {
            mma_e4m3(dx, a0, bd + (uint64_t)c * bstep, idesc, acc);
            mma_e4m3(dy, a1, bd + (uint64_t)c * bstep, idesc, acc);
        } else {
            mma_bf16(dx, a0, bd + (uint64_t)c * bstep, idesc, acc);
            mma_bf16(dy, a1, bd + (uint64_t)c * bstep, idesc, acc);
        }
    }
}

template <int N, int MODE, bool F8, bool SWAP>
__global__ void __launch_bounds__(kPipeThreads, 1) k_nedf2(Workspace ws, MarchBuffers mb, PipeArgs a)
{
    using SH = PipeShape<N, false, F8>;
    using S2 = NedfShape2<N, F8, SWAP>;
    constexpr int K0 = SH::K0, NOUT = 2;
    const int GC = max(1, min(a.stage_bytes / SH::CHUNK, S2::SMAX / 2));
    const int STAGE = GC * SH::CHUNK, S = S2::RING / STAGE;
    // When a round's two tiles have the same type, one copy of each layer's weights serves both
    // slots: the stages stay until the second slot's MMAs have read them, so the ring must hold
    // every stage of a layer at once.
    const int NK_MAX = max(K0 / kKC, F8 ? N / 32 : N / kKC + 1);
    const bool can_share = S >= (NK_MAX + GC - 1) / GC;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t a_ready[2], acc_full[2], fin;
    __shared__ uint64_t w_full[S2::SMAX], w_empty[S2::SMAX];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    constexpr bool SW = S2::SW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = ws.nedf_hidden;
    uint8_t *ring = smem + S2::ACT;
    uint8_t *ones_blk = smem + 2 * S2::H_BYTES;                 // swapped only
    const int n_f32 = (int)pipe_f32_floats(N, L, NOUT, F8);
    const size_t f32_bytes = ((size_t)n_f32 * 4 + 15) & ~(size_t)15;
    volatile int *abort = &abort_flag;

    if (warp == 9) tmem_alloc(&tmem_base, 4 * N);
    if (threadIdx.x == 0) {
        for (int j = 0; j < 2; ++j) {
            mbar_init(&a_ready[j], 2 * kHalf);
            mbar_init(&acc_full[j], 1);
        }
        mbar_init(&fin, 1);
        for (int q = 0; q < S; ++q) {
            mbar_init(&w_full[q], 1);
            mbar_init(&w_empty[q], 1);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const unsigned long long n_tiles = pipe_n_tiles<N, MODE>(ws, mb, a);
    const unsigned long long gx = gridDim.x;
    const DevFrame &f = *ws.frame;
    auto A_of = [&](int s, int h) { return smem + (size_t)(2 * s + h) * SH::A_BYTES; };   // unswapped
    auto H_of = [&](int s) { return smem + (size_t)s * S2::H_BYTES; };                     // swapped

    if (warp == 8) {
        // ------------------------------ producer ------------------------------------------------
        if (lane == 0) {
            unsigned long long q = 0;
            RingPos rp;
            for (unsigned long long t0 = blockIdx.x; t0 < n_tiles && !*abort; t0 += 2 * gx) {
                const bool two = t0 + gx < n_tiles;
                const int ty0 = pipe_tile_type<MODE>(ws, mb, a, t0), ty1 = two ? pipe_tile_type<MODE>(ws, mb, a, t0 + gx) : ty0;
                const bool share = can_share && ty0 == ty1;
                for (int l = 0; l < L && !*abort; ++l)
                    for (int s = 0; s < 2 && !*abort; ++s) {
                        const unsigned long long tile = t0 + s * gx;
                        if (tile >= n_tiles || (s == 1 && share)) continue;
                        const uint8_t *src = a.blobs + (size_t)(s ? ty1 : ty0) * a.blob_stride + pipe_layer_off(K0, N, l, F8);
                        const int nk = l == 0 ? K0 / kKC : (F8 ? N / 32 : N / kKC + 1);
                        for (int c0 = 0; c0 < nk; c0 += GC, ++q, rp.next(S)) {
                            const int st = rp.st;
                            const uint32_t bytes = (uint32_t)(min(GC, nk - c0) * SH::CHUNK);
                            if (!pipe_wait(&w_empty[st], rp.ph ^ 1u, abort, ws.status)) break;
                            mbar_arrive_expect_tx(&w_full[st], bytes);
                            bulk_g2s(ring + (size_t)st * STAGE, src + (size_t)c0 * SH::CHUNK, bytes, &w_full[st]);
                        }
                    }
            }
            const unsigned long long q0 = q > (unsigned long long)S ? q - S : 0;
            for (unsigned long long k = q0; k < q; ++k) pipe_drain(&w_full[k % S], (uint32_t)((k / S) & 1u), ws.status);
        }
    } else if (warp == 9) {
        // ------------------------------ MMA issuer ----------------------------------------------
        if (lane == 0) {
            unsigned long long ja[2] = {0, 0};
            RingPos rp;
            const uint32_t idesc = idesc_bf16(128, N), idesc8 = idesc_e4m3(128, N);
            bool issued_any = false;
            for (unsigned long long t0 = blockIdx.x; t0 < n_tiles && !*abort; t0 += 2 * gx) {
                // the same decision as the producer's: shared stages are walked twice and released
                // by the second slot
                const bool two = t0 + gx < n_tiles;
                const bool share = can_share && (!two || pipe_tile_type<MODE>(ws, mb, a, t0) == pipe_tile_type<MODE>(ws, mb, a, t0 + gx));
                for (int l = 0; l < L && !*abort; ++l) {
                    const RingPos rp_layer = rp;
                    for (int s = 0; s < 2 && !*abort; ++s) {
                        if (t0 + s * gx >= n_tiles) continue;
                        if (!pipe_wait(&a_ready[s], (uint32_t)(ja[s]++ & 1u), abort, ws.status)) break;
                        tc_fence_after();
                        if (share) rp = rp_layer;
                        const bool release = !share || s == 1 || !two;
                        const uint32_t ax = smem_addr(A_of(s, 0)), ay = smem_addr(A_of(s, 1));
                        const uint32_t dx = tmem + (uint32_t)(2 * s) * N, dy = dx + N;
                        const uint32_t hs = smem_addr(H_of(s)), ones = smem_addr(ones_blk);
                        // swapped layers: N = 256 rows, B MN-major (bit 16) after layer 0; the last
                        // layer unswapped: A MN-major (bit 15) after layer 0
                        const bool swapped = SW && l + 1 < L;
                        const uint32_t id_sw = swapped ? idesc_bf16(128, 256) | (l > 0 ? 1u << 16 : 0u)
                                                       : idesc_bf16(128, N) | (l > 0 ? 1u << 15 : 0u);
                        const int nk = l == 0 ? K0 / kKC : (F8 ? N / 32 : N / kKC + 1);
                        const bool e4m3 = F8 && l > 0;
                        for (int c0 = 0; c0 < nk; c0 += GC, rp.next(S)) {
                            const int st = rp.st;
                            if (!pipe_wait(&w_full[st], rp.ph, abort, ws.status)) break;
                            const uint32_t stage = smem_addr(ring + (size_t)st * STAGE);
                            const int c1 = min(nk, c0 + GC);
                            if (SW) {
                                // chunk c: input columns 16c..16c+15, 8 KB of the slot's
                                // activations (8-column groups 4 KB apart, 8-row groups 128 bytes
                                // apart); a hidden layer's bias chunk reads the ones block
                                uint64_t wd = smem_desc(stage, 128, 256);
                                if (c0 == 0 && c1 == nk && (swapped || l > 0)) {
                                    // the whole layer in this stage (the autotuner's stages of >= 36 KB)
                                    if constexpr (SW) {
                                        if (!swapped) issue_layer_unswapped<N / kKC + 1>(dx, dy, wd, hs, ones, id_sw);
                                        else if (l == 0) issue_layer_swapped<K0 / kKC, false>(dx, wd, hs, ones, id_sw);
                                        else issue_layer_swapped<N / kKC + 1, true>(dx, wd, hs, ones, id_sw);
                                    }
                                } else
                                for (int c = c0; c < c1; ++c) {
                                    const uint32_t src = (l > 0 && c == N / kKC) ? ones : hs + (uint32_t)c * 8192u;
                                    const uint32_t acc = c > 0 ? 1u : 0u;
                                    if (swapped) {
                                        mma_bf16(dx, wd, smem_desc(src, 4096, 128), id_sw, acc);
                                    } else {
                                        mma_bf16(dx, smem_desc(src, 4096, 128), wd, id_sw, acc);
                                        mma_bf16(dy, smem_desc(src + 2048u, 4096, 128), wd, id_sw, acc);
                                    }
                                    wd += (uint64_t)(SH::CHUNK >> 4);
                                }
                            } else if (c0 == 0 && c1 == nk) {
                                // the whole layer in this stage: a straight run
                                if (l == 0) issue_layer_halves<false, K0 / kKC, false>(dx, dy, ax, ay, stage, SH::CHUNK, idesc, 0u);
                                else if (e4m3) issue_layer_halves<true, N / 32, false>(dx, dy, ax, ay, stage, SH::CHUNK, idesc8, 0u);
                                else issue_layer_halves<false, N / kKC + 1, true>(dx, dy, ax, ay, stage, SH::CHUNK, idesc,
                                                                                  (uint32_t)(SH::ONES / kKC) * 4096u);
                            } else if (e4m3) {
                                issue_chunks<true>(dx, dy, ax, ay, stage, c0, c1, SH::CHUNK, idesc8, -1, 0u);
                            } else {
                                issue_chunks<false>(dx, dy, ax, ay, stage, c0, c1, SH::CHUNK, idesc,
                                                    l > 0 ? N / kKC : -1, (uint32_t)(SH::ONES / kKC) * 4096u);
                            }
                            if (release) mma_commit(&w_empty[st]);
                            issued_any = true;
                        }
                        mma_commit(&acc_full[s]);
                    }
                }
            }
            if (issued_any) {
                mma_commit(&fin);
                pipe_drain(&fin, 0u, ws.status);
            }
        }
    } else {
        // ------------------------------ epilogue groups -----------------------------------------
        const int g = warp >> 2;                      // half: rows 0..127 (X) or 128..255 (Y)
        const int r = threadIdx.x & 127;
        const int R = g * kHalf + r;
        const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
        float *f32s[2] = {reinterpret_cast<float *>(smem + S2::FIXED),
                          reinterpret_cast<float *>(smem + S2::FIXED + f32_bytes)};
        int f32_type[2] = {-1, -1};
        unsigned long long jb[2] = {0, 0};
        if (SW) {
            // the ones block, MN-major like the activations: input columns 0 and 1 are 1 for all 256
            // rows (the 16-byte vectors 0 and 1 of each 8-row group), the rest 0
            for (int u = threadIdx.x; u < (int)(S2::ONES_BYTES / 16); u += 2 * kHalf) {
                const bool one = u * 16 < 4096 && ((u * 16) & 127) < 32;
                const uint32_t w = one ? pack_bf16(1.0f, 1.0f) : 0u;
                reinterpret_cast<uint4 *>(ones_blk)[u] = make_uint4(w, w, w, w);
            }
        } else if (!F8) {
            for (int s = 0; s < 2; ++s) {
                *reinterpret_cast<uint4 *>(A_of(s, g) + a_offset(r, SH::ONES)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(A_of(s, g) + a_offset(r, SH::ONES + 8)) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        // set-up of slot s for `tile`: its type's fp32 block, the encoded rows, then a_ready
        auto setup = [&](int s, unsigned long long tile) {
            const int t = pipe_tile_type<MODE>(ws, mb, a, tile);
            if (t != f32_type[s]) {
                asm volatile("bar.sync 3, 256;" ::: "memory");   // every reader of the old block is done
                const float4 *src = reinterpret_cast<const float4 *>(a.blobs + (size_t)t * a.blob_stride +
                                                                     pipe_w_bytes(K0, N, L, F8));
                for (int i = threadIdx.x; i < n_f32 / 4; i += 2 * kHalf) reinterpret_cast<float4 *>(f32s[s])[i] = src[i];
                asm volatile("bar.sync 3, 256;" ::: "memory");
                f32_type[s] = t;
            }
            const DevType T = ws.types[t];
            unsigned long long idx;
            bool valid;
            PairRay pr;
            nedf_row<MODE>(ws, a, T, t, tile, R, idx, valid, pr);
            float x6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid && pr.kept) {
                const V3 pe = madd(pr.ol, pr.te, pr.dl);
                x6[0] = pe.x; x6[1] = pe.y; x6[2] = pe.z; x6[3] = pr.dl.x; x6[4] = pr.dl.y; x6[5] = pr.dl.z;
            }
            float feat[K0];
            pipe_encode<6, 6>(x6, feat);
            if (SW) pipe_store_row<K0, 4096>(H_of(s), R, feat, kNedfIn);
            else pipe_store_row<K0>(A_of(s, g), r, feat, kNedfIn);
            fence_proxy_async_smem();
            tc_fence_before();
            mbar_arrive(&a_ready[s]);
        };
        // output of a finished tile's row: a query's (m, a, D_l, hit), or a listed pair's (m, a) for
        // the decode pass
        auto emit = [&](unsigned long long tile, const float *out) {
            const int t = pipe_tile_type<MODE>(ws, mb, a, tile);
            unsigned long long idx;
            if (MODE == kModeQuery) {
                const DevType T = ws.types[t];
                bool valid;
                PairRay pr;
                nedf_row<MODE>(ws, a, T, t, tile, R, idx, valid, pr);
                if (valid) {
                    float4 res = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
                    if (pr.kept) {
                        const float Dl = pr.tp - T.rb * out[0];
                        res = make_float4(out[0], out[1], Dl, (out[1] > 0.f && Dl > 0.f) ? 1.f : 0.f);
                    }
                    a.qout[idx] = res;
                }
            } else if (nedf_row_index<MODE>(ws, a, t, tile, R, idx)) {
                ws.nout[MODE == kModeShadow ? 1 : 0][idx] = make_float2(out[0], out[1]);
            }
        };
        if (blockIdx.x < n_tiles) setup(0, blockIdx.x);
        if (blockIdx.x + gx < n_tiles) setup(1, blockIdx.x + gx);
        bool stop = false;
        for (unsigned long long t0 = blockIdx.x; t0 < n_tiles && !stop; t0 += 2 * gx) {
            for (int l = 0; l < L && !stop; ++l)
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    if (stop) continue;
                    const unsigned long long tile = t0 + s * gx;
                    if (tile >= n_tiles) continue;
                    // a warp-uniform outcome (tcgen05.ld is warp-collective);
                    // the last layer's step also synchronises the 256 epilogue threads (set-up), so
                    // its outcome, and the decision to stop, are made for all of them there
                    const bool last = l + 1 == L;
                    const bool okw = __all_sync(0xffffffffu, pipe_wait(&acc_full[s], (uint32_t)(jb[s]++ & 1u), abort, ws.status));
                    const bool ok = last ? !epilogue_any(!okw) : okw;
                    if (ok) {
                        tc_fence_after();
                        const float *f32 = f32s[s];
                        const uint32_t trow = tmem + lane_q + (uint32_t)(2 * s + g) * N;
                        const float *bias = f32 + pipe_f8_bias_off(N, NOUT) + (size_t)l * N;
                        const float sc = F8 && l > 0 ? f32[pipe_f8_bias_off(N, NOUT) + (size_t)L * N + l] : 1.0f;
                        float out[NOUT] = {f32[NOUT * N], f32[NOUT * N + 1]};
                        if (l + 1 < L) {
                            if (SW) epi_swapped(tmem + lane_q + (uint32_t)(2 * s * N + g * kHalf), H_of(s), (warp & 3) * 32 + lane, g * kHalf);
                            else if (F8 && l > 0) epi_layer<N, NOUT, F8, true, false>(trow, A_of(s, g), r, bias, sc, f32, out);
                            else epi_layer<N, NOUT, F8, false, false>(trow, A_of(s, g), r, bias, sc, f32, out);
                            fence_proxy_async_smem();
                            tc_fence_before();
                            mbar_arrive(&a_ready[s]);
                        } else {
                            if (F8 && l > 0) epi_layer<N, NOUT, F8, true, true>(trow, A_of(s, g), r, bias, sc, f32, out);
                            else epi_layer<N, NOUT, F8, false, true>(trow, A_of(s, g), r, bias, sc, f32, out);
                            tc_fence_before();
                        }
                        if (l + 1 == L) {
                            emit(tile, out);
                            const unsigned long long nxt = tile + 2 * gx;
                            if (!epilogue_any(*abort != 0) && nxt < n_tiles) setup(s, nxt);
                        }
                    } else {
                        *abort = 1;
                    }
                    if (last) stop = epilogue_any(!ok || *abort);
                }
        }
    }
    // ---- teardown ------------------------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 9) tmem_dealloc(tmem, 4 * N);
}

// ---------------------------------------------------------------------------------------------------
// Wait-limit check: one thread waits on an mbarrier phase that nothing completes, with the same
// bounded wait as the engine; the wait gives up after its limit and sets the timeout status.
// ---------------------------------------------------------------------------------------------------
__global__ void k_wait_check(uint32_t *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_wait(&bar, 0u, status, kStatusTimeout);      // phase 0 never completes
    }
}

cudaError_t launch_wait_check(uint32_t *status, cudaStream_t st)
{
    k_wait_check<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// Deferred plain-method pairs (low confidence, outliers, checked misses), one thread per pair: the
// plain method's march with the samples the SDF proves on one side skipped (march_crossing_skip:
// the same crossing and bisection as the uniform march)
// ---------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fallback(Workspace ws, int mode)
{
    const DevFrame &f = *ws.frame;
    const unsigned long long n = ws.cnt->fb_count[mode];
    const uint2 *pairs = mode == 1 ? ws.spairs : ws.ppairs;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        const uint2 pr = pairs[ws.fb_list[mode][e]];
        const DevType T = ws.types[ws.inst[pr.y].type];
        PairRay R;
        setup_pair_ray(ws, f, mode == 1, pr, T.rb, R);
        bool hit = false;
        const float Dl = march_crossing_skip(T, R.ol, R.dl, R.te, R.tx, f.march_steps, f.march_bisect, hit);
        if (hit) apply_hit(ws, f, mode == 1, R, Dl);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ws.cnt->fallback, n);
}

cudaError_t launch_fallback(const Workspace &ws, int mode, int num_sms, cudaStream_t st)
{
    k_fallback<<<num_sms * 8, 256, 0, st>>>(ws, mode);
    return cudaGetLastError();
}

template <int N, int MODE, bool F8>
static cudaError_t launch_pipe_n(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a, int grid, cudaStream_t st)
{
    constexpr bool NERF = MODE == kModeShade || MODE == kModeMarch;
    const int L = NERF ? ws.nerf_hidden : ws.nedf_hidden;
    const size_t sm = PipeShape<N, NERF, F8>::FIXED + ((pipe_f32_floats(N, L, NERF ? 3 : 2, F8) * 4 + 1023) & ~(size_t)1023);
    if (sm > 227 * 1024 - 8192) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_pipe<N, MODE, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_pipe<N, MODE, F8><<<grid, kPipeThreadsPf, sm, st>>>(ws, mb, a);
    return cudaGetLastError();
}

// precision 1: BF16 layers; precision 2: first layer BF16, later hidden layers E4M3
template <int MODE>
static cudaError_t launch_pipe(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a, int width, int grid,
                               cudaStream_t st)
{
    if (grid < 1) return cudaSuccess;
    const bool f8 = ws.precision == 2;
    PipeArgs args = a;
    args.stage_bytes = ws.pipe_stage_bytes[MODE] > 0 ? ws.pipe_stage_bytes[MODE] : kDefaultStageBytes;
    if (width == 256 && ws.nerf_pair_off && ws.pipe_order[MODE] == 1) {
        // the SM-pair engine (its own blob layout); the one-SM engine when the pair shape does not fit
        PipeArgs pa = args;
        pa.blobs = a.blobs + ws.nerf_pair_off;
        const cudaError_t e = launch_pair_pipe(ws, mb, pa, MODE, grid, st);
        if (e != cudaErrorInvalidConfiguration) return e;
    }
    switch (width) {
    case 64: return f8 ? launch_pipe_n<64, MODE, true>(ws, mb, args, grid, st) : launch_pipe_n<64, MODE, false>(ws, mb, args, grid, st);
    case 128: return f8 ? launch_pipe_n<128, MODE, true>(ws, mb, args, grid, st) : launch_pipe_n<128, MODE, false>(ws, mb, args, grid, st);
    case 256: return f8 ? launch_pipe_n<256, MODE, true>(ws, mb, args, grid, st) : launch_pipe_n<256, MODE, false>(ws, mb, args, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int MODE, bool F8, bool SWAP = (N == 128 && !F8)>
static cudaError_t launch_nedf2_n(const Workspace &ws, const PipeArgs &a, int grid, cudaStream_t st)
{
    const size_t f32b = (pipe_f32_floats(N, ws.nedf_hidden, 2, F8) * 4 + 15) & ~(size_t)15;
    const size_t sm = NedfShape2<N, F8, SWAP>::FIXED + 2 * f32b;
    if (sm > 227 * 1024 - 8192) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_nedf2<N, MODE, F8, SWAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    MarchBuffers none{};
    k_nedf2<N, MODE, F8, SWAP><<<grid, kPipeThreads, sm, st>>>(ws, none, a);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_nedf2(const Workspace &ws, const PipeArgs &a, int grid, cudaStream_t st)
{
    if (grid < 1) return cudaSuccess;
    const bool f8 = ws.precision == 2;
    PipeArgs args = a;
    args.stage_bytes = ws.pipe_stage_bytes[MODE] > 0 ? ws.pipe_stage_bytes[MODE] : kDefaultStageBytes;
    switch (ws.nedf_width) {
    case 64: return f8 ? launch_nedf2_n<64, MODE, true>(ws, args, grid, st) : launch_nedf2_n<64, MODE, false>(ws, args, grid, st);
    case 128:
        if (f8) return launch_nedf2_n<128, MODE, true>(ws, args, grid, st);
        // operand order 2: unswapped (activations as A); 0 (default) and 1: swapped
        return ws.pipe_order[MODE] == 2 ? launch_nedf2_n<128, MODE, false, false>(ws, args, grid, st)
                                        : launch_nedf2_n<128, MODE, false, true>(ws, args, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_nedf_pipe(const Workspace &ws, int mode, int type, const float *o, const float *d, float *out, int n,
                             int num_sms, cudaStream_t st)
{
    if (ws.nedf_arch == 1) return launch_cls_pipe(ws, mode, type, o, d, out, n, num_sms, st);
    PipeArgs a{};
    a.blobs = ws.nedf_tc;
    a.blob_stride = ws.nedf_tc_stride;
    a.query_type = type;
    a.qo = o;
    a.qd = d;
    a.qout = reinterpret_cast<float4 *>(out);
    a.qn = n;
    if (mode == 0) return launch_nedf2<kModePrimary>(ws, a, num_sms, st);
    if (mode == 1) return launch_nedf2<kModeShadow>(ws, a, num_sms, st);
    const int grid = (int)std::min<long long>(num_sms, ((long long)n + kPipeRows - 1) / kPipeRows);
    return launch_nedf2<kModeQuery>(ws, a, grid, st);
}

cudaError_t launch_shade_pipe(const Workspace &ws, int npix, int num_sms, cudaStream_t st)
{
    PipeArgs a{};
    a.blobs = ws.nerf_tc;
    a.blob_stride = ws.nerf_tc_stride;
    a.npix = npix;
    MarchBuffers none{};
    return launch_pipe<kModeShade>(ws, none, a, ws.nerf_width, num_sms, st);
}

cudaError_t launch_march_colour_pipe(const Workspace &ws, const MarchBuffers &mb, int n_samples, int num_sms, cudaStream_t st)
{
    PipeArgs a{};
    a.blobs = ws.nerf_tc;
    a.blob_stride = ws.nerf_tc_stride;
    a.n_samples = n_samples;
    return launch_pipe<kModeMarch>(ws, mb, a, ws.nerf_width, num_sms, st);
}

}  // namespace nedf
