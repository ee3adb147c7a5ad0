// BF16 tensor-core (tcgen05 / TMEM) path of the render-time networks.
//
// Method: arXiv 2308.04669, Eq. 1-2 and 7 (NeDF queries of Step 1 and Step 3), Eq. 8 with the
// sample window (the radiance field of Step 2).
//
// One CTA of 128 threads runs 128-row tiles; thread r owns row r from its ray set-up through
// the decode.  Hidden layers are single-CTA tcgen05 MMAs (M = 128, N = width, K = 16 per
// instruction) from shared-memory operands into a TMEM accumulator; the epilogue reads the
// accumulator with tcgen05.ld (warp w sees lanes 32w .. 32w+31, i.e. its own rows), adds the
// bias, applies ReLU and writes the next layer's BF16 A operand back to shared memory.  The
// last hidden layer's epilogue also evaluates the small output layer (2 or 3 outputs) on CUDA
// cores from BF16-rounded activations and weights, so no output MMA is needed.
//
// NeDF weights (6 x 128: 180 KB in BF16) stay resident in shared memory across the tiles of a
// type; NeRF weights (8 x 256: 944 KB) are streamed layer by layer with bulk asynchronous
// copies, the copy of layer l+1 overlapping the epilogue of layer l.
#include "render_kernels.cuh"
#include "render_launch.h"
#include "tc_ptx.cuh"

#include <algorithm>

namespace nedf {

using namespace tc;

constexpr int kTcRows = kTcTileRows;
constexpr int kTcThreads = 128;

// ---- per-type BF16 weight blobs -----------------------------------------------------------------
// [W_0: N x K0 bf16][W_1..W_{L-1}: N x N bf16][bias: L x N f32][w_out: n_out x N f32 (bf16
// values)][b_out: n_out f32], every part 16-byte aligned, W parts in the core-matrix layout.
__host__ __device__ inline size_t tc_w_bytes(int K0, int N, int L) { return ((size_t)K0 * N + (size_t)(L - 1) * N * N) * 2; }
__host__ __device__ inline size_t tc_f32_floats(int N, int L, int n_out) { return ((size_t)L * N + (size_t)n_out * N + n_out + 3) & ~(size_t)3; }
__host__ __device__ inline size_t tc_blob_bytes(int K0, int N, int L, int n_out)
{
    size_t b = tc_w_bytes(K0, N, L) + tc_f32_floats(N, L, n_out) * 4;
    return (b + 1023) & ~(size_t)1023;
}

// packed FP32 master (W[out][in], b per layer) -> BF16 blob; one thread per element
__global__ void k_pack_tc(const float *master, uint8_t *blob, int K_in, int K0, int N, int L, int n_out)
{
    size_t wb = tc_w_bytes(K0, N, L);
    float *f32 = reinterpret_cast<float *>(blob + wb);
    long long total_w = (long long)N * K0 + (long long)(L - 1) * N * N;
    long long total = total_w + (long long)L * N + (long long)n_out * N + n_out;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        if (e < total_w) {
            int l, n, k, K, Kin;
            long long off_src, off_dst, j;
            if (e < (long long)N * K0) {
                l = 0; j = e; K = K0; Kin = K_in; off_src = 0; off_dst = 0;
            } else {
                long long e2 = e - (long long)N * K0;
                l = 1 + (int)(e2 / ((long long)N * N));
                j = e2 - (long long)(l - 1) * N * N;
                K = N; Kin = N;
                off_src = (long long)K_in * N + N + (long long)(l - 1) * (N * N + N);
                off_dst = (long long)N * K0 * 2 + (long long)(l - 1) * N * N * 2;
            }
            n = (int)(j / K);
            k = (int)(j - (long long)n * K);
            float v = k < Kin ? master[off_src + (long long)n * Kin + k] : 0.0f;
            *reinterpret_cast<__nv_bfloat16 *>(blob + off_dst + cm_offset(n, k, K)) = __float2bfloat16_rn(v);
        } else {
            long long j = e - total_w;
            if (j < (long long)L * N) {          // hidden biases
                int l = (int)(j / N), n = (int)(j - (long long)l * N);
                long long off = l == 0 ? (long long)K_in * N : (long long)K_in * N + N + (long long)(l - 1) * (N * N + N) + (long long)N * N;
                f32[j] = master[off + n];
            } else {
                long long q = j - (long long)L * N;
                long long off_out = (long long)K_in * N + N + (long long)(L - 1) * (N * N + N);
                if (q < (long long)n_out * N) f32[j] = round_bf16(master[off_out + q]);
                else f32[j] = master[off_out + (long long)n_out * N + (q - (long long)n_out * N)];
            }
        }
    }
}

cudaError_t launch_pack_tc(const float *master, void *blob, int K_in, int K0, int N, int L, int n_out, cudaStream_t st)
{
    long long total = (long long)N * K0 + (long long)(L - 1) * N * N + (long long)L * N + (long long)n_out * N + n_out;
    int blocks = (int)std::min<long long>((total + 255) / 256, 4096);
    k_pack_tc<<<blocks, 256, 0, st>>>(master, (uint8_t *)blob, K_in, K0, N, L, n_out);
    return cudaGetLastError();
}

size_t tc_blob_size(int K0, int N, int L, int n_out) { return tc_blob_bytes(K0, N, L, n_out); }

// ---- encodings into a BF16 A row ------------------------------------------------------------------
// gamma of an n-wide input with F frequencies, identity first, then sine blocks, then cosine
// blocks (frequency 2^k).  sin / cos of 2^k x come from the double-angle identities applied to
// sincos(x); the values are rounded to BF16 afterwards.
template <int NIN, int F>
__device__ __forceinline__ void encode(const float *x, float *out)
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

template <int K>
__device__ __forceinline__ void store_row_bf16(uint8_t *A, int r, const float *f, int n_valid)
{
#pragma unroll
    for (int c = 0; c < K / 8; ++c) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int k = c * 8 + 2 * e;
            p[e] = pack_bf16(k < n_valid ? f[k] : 0.0f, k + 1 < n_valid ? f[k + 1] : 0.0f);
        }
        *reinterpret_cast<uint4 *>(A + cm_offset(r, c * 8, K)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
}

// ---- one layer on the tensor cores ---------------------------------------------------------------
__device__ __forceinline__ void issue_layer(uint32_t tmem, const uint8_t *A, const uint8_t *W, int K, int N,
                                            uint64_t *bar)
{
    tc_fence_after();
    const uint32_t a0 = smem_addr(A), b0 = smem_addr(W), sbo = (uint32_t)(K / 8) * 128;
    const uint32_t id = (N == 256) ? idesc_bf16(128, 256) : (N == 128 ? idesc_bf16(128, 128) : idesc_bf16(128, 64));
    for (int s = 0; s < K / 16; ++s)
        mma_bf16(tmem, smem_desc(a0 + s * 256, 128, sbo), smem_desc(b0 + s * 256, 128, sbo), id, s > 0 ? 1u : 0u);
    mma_commit(bar);
}

// Accumulator row -> bias + ReLU -> BF16 A row of the next layer (K = N).
template <int N>
__device__ __forceinline__ void epilogue_hidden(uint32_t tmem_row, const float *bias, uint8_t *A, int r)
{
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem_row + c0, v);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t p[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int j = q * 8 + 2 * e;
                float x0 = fmaxf(__uint_as_float(v[j]) + bias[c0 + j], 0.0f);
                float x1 = fmaxf(__uint_as_float(v[j + 1]) + bias[c0 + j + 1], 0.0f);
                p[e] = pack_bf16(x0, x1);
            }
            *reinterpret_cast<uint4 *>(A + cm_offset(r, c0 + q * 8, N)) = make_uint4(p[0], p[1], p[2], p[3]);
        }
    }
}

// Accumulator row -> bias + ReLU -> BF16 -> output layer (n_out outputs) on CUDA cores.
template <int N, int NOUT>
__device__ __forceinline__ void epilogue_out(uint32_t tmem_row, const float *bias, const float *wout,
                                             const float *bout, float *y)
{
#pragma unroll
    for (int o = 0; o < NOUT; ++o) y[o] = bout[o];
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
        uint32_t v[32];
        tmem_ld32(tmem_row + c0, v);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            float h = round_bf16(fmaxf(__uint_as_float(v[j]) + bias[c0 + j], 0.0f));
#pragma unroll
            for (int o = 0; o < NOUT; ++o) y[o] = fmaf(h, wout[o * N + c0 + j], y[o]);
        }
    }
}

struct TcSmem {
    uint64_t bar_w;      // weight bytes landed
    uint64_t bar_f;      // fp32 block (biases, output layer) landed
    uint64_t bar_mma;    // MMAs of a layer completed
    uint32_t tmem_base;
    int pad;
};

struct TcSync {
    uint32_t w_phase = 0, f_phase = 0, mma_phase = 0;
    bool w_pending = false, f_pending = false, mma_pending = false;
    bool ok = true;
};

__device__ __forceinline__ void tc_setup(TcSmem &S, uint32_t ncols)
{
    if ((threadIdx.x >> 5) == 0) tmem_alloc(&S.tmem_base, ncols);
    if (threadIdx.x == 0) {
        mbar_init(&S.bar_w, 1);
        mbar_init(&S.bar_f, 1);
        mbar_init(&S.bar_mma, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// Waits on one barrier phase; a timeout flags the status word and clears ok.
__device__ __forceinline__ void tc_wait(uint64_t *bar, uint32_t &phase, bool &pending, TcSync &y, uint32_t *status)
{
    if (!pending) return;
    if (!mbar_wait(bar, phase, status, kStatusTimeout)) y.ok = false;
    phase ^= 1;
    pending = false;
}

// Drains whatever async work is still outstanding (bounded), then frees TMEM.
__device__ __forceinline__ void tc_teardown(TcSmem &S, TcSync &y, uint32_t ncols, uint32_t *status)
{
    tc_wait(&S.bar_mma, y.mma_phase, y.mma_pending, y, status);
    tc_wait(&S.bar_w, y.w_phase, y.w_pending, y, status);
    tc_wait(&S.bar_f, y.f_phase, y.f_pending, y, status);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_dealloc(S.tmem_base, ncols);
}

// ---------------------------------------------------------------------------------------------------
// NeDF tiles: mode 0 = Step-1 primary pairs, 1 = Step-3 shadow pairs, 2 = caller rays of one type
// ---------------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(kTcThreads, 1)
k_nedf_tc(Workspace ws, const uint8_t *blobs, size_t blob_stride, int mode, int query_type, const float *qo,
          const float *qd, float4 *qout, int qn)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcSmem S;
    const int L = ws.nedf_hidden;
    constexpr int K0 = kNedfInPad;
    const size_t blob_bytes = tc_blob_bytes(K0, N, L, 2);
    uint8_t *Wsm = smem;
    const float *f32 = reinterpret_cast<const float *>(smem + tc_w_bytes(K0, N, L));
    uint8_t *A = smem + blob_bytes;
    const int r = threadIdx.x, warp = threadIdx.x >> 5;
    constexpr uint32_t kCols = N < 32 ? 32 : N;

    tc_setup(S, kCols);
    const uint32_t tmem = S.tmem_base;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    TcSync y;
    int loaded = -1;

    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    unsigned long long n_tiles;
    if (mode == 2) n_tiles = ((unsigned long long)qn + kTcRows - 1) / kTcRows;
    else n_tiles = (mode ? C.s_tile : C.p_tile)[f.n_types];
    const unsigned long long *tile_off = mode == 1 ? C.s_tile : C.p_tile;
    const unsigned long long *pair_off = mode == 1 ? C.s_off : C.p_off;
    const uint2 *pairs = mode == 1 ? ws.spairs : ws.ppairs;

    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int t = query_type;
        unsigned long long begin = tile * kTcRows, end = (unsigned long long)qn;
        if (mode != 2) {
            t = 0;
            while (t + 1 < f.n_types && tile_off[t + 1] <= tile) ++t;
            begin = pair_off[t] + (tile - tile_off[t]) * kTcRows;
            end = pair_off[t + 1];
        }
        const DevType T = ws.types[t];
        if (t != loaded) {
            // the previous tile's MMAs and epilogues are complete: the weights can be replaced
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&S.bar_w, (uint32_t)blob_bytes);
                const uint8_t *src = blobs + (size_t)t * blob_stride;
                for (size_t off = 0; off < blob_bytes; off += 65536)
                    bulk_g2s(Wsm + off, src + off, (uint32_t)min((size_t)65536, blob_bytes - off), &S.bar_w);
            }
            y.w_pending = true;
            loaded = t;
        }
        // ---- row set-up: ray, local frame, bound chord, encoding -------------------------------
        const unsigned long long idx = begin + r;
        const bool valid = idx < end;
        PairRay R;
        R.kept = false;
        R.te = R.tx = R.tp = 0.f;
        R.ol = v3(0, 0, 0);
        R.dl = v3(0, 0, 1);
        if (valid) {
            if (mode == 2) {
                R.ol = v3(qo[3 * idx], qo[3 * idx + 1], qo[3 * idx + 2]);
                R.dl = normalized(v3(qd[3 * idx], qd[3 * idx + 1], qd[3 * idx + 2]));
                Chord ch;
                R.kept = bound_chord(R.ol, R.dl, T.rb, ch);
                R.te = ch.te; R.tx = ch.tx; R.tp = ch.tp;
            } else {
                setup_pair_ray(ws, f, mode == 1, pairs[idx], T.rb, R);
            }
        }
        float out[2] = {0.f, 0.f};
        {
            float feat[K0];
            float x6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (valid && R.kept) {
                V3 pe = madd(R.ol, R.te, R.dl);
                x6[0] = pe.x; x6[1] = pe.y; x6[2] = pe.z; x6[3] = R.dl.x; x6[4] = R.dl.y; x6[5] = R.dl.z;
            }
            encode<6, 6>(x6, feat);
            store_row_bf16<K0>(A, r, feat, kNedfIn);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_wait(&S.bar_w, y.w_phase, y.w_pending, y, ws.status);
        // ---- hidden layers on the tensor cores, output layer fused into the last epilogue -----
        for (int l = 0; l < L; ++l) {
            const int K = l == 0 ? K0 : N;
            const uint8_t *Wl = Wsm + (l == 0 ? 0 : (size_t)K0 * N * 2 + (size_t)(l - 1) * N * N * 2);
            if (threadIdx.x == 0 && y.ok) issue_layer(tmem, A, Wl, K, N, &S.bar_mma);
            y.mma_pending = y.ok;
            tc_wait(&S.bar_mma, y.mma_phase, y.mma_pending, y, ws.status);
            tc_fence_after();
            if (l + 1 < L) {
                epilogue_hidden<N>(tmem_row, f32 + l * N, A, r);
                fence_proxy_async_smem();
            } else {
                epilogue_out<N, 2>(tmem_row, f32 + l * N, f32 + L * N, f32 + L * N + 2 * N, out);
            }
            tc_fence_before();
            __syncthreads();
        }
        // ---- decode (Eq. 2, 7) and checks; plain-method pairs are deferred to their own pass ---
        bool defer = false;
        if (valid) {
            if (mode == 2) {
                float4 res = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
                if (R.kept) {
                    float Dl = R.tp - T.rb * out[0];
                    res = make_float4(out[0], out[1], Dl, (out[1] > 0.f && Dl > 0.f) ? 1.f : 0.f);
                }
                qout[idx] = res;
            } else {
                float Dl;
                bool hit;
                defer = nedf_decode(f, T, R.ol, R.dl, R.tp, out[0], out[1], Dl, hit);
                if (!defer && hit) apply_hit(ws, f, mode == 1, R, Dl);
            }
        }
        if (mode != 2) {
            const int lane = threadIdx.x & 31;
            unsigned m = __ballot_sync(0xffffffffu, defer);
            if (m) {
                int leader = __ffs(m) - 1;
                unsigned long long start = 0;
                if (lane == leader) start = atomicAdd(&ws.cnt->fb_count[mode], (unsigned long long)__popc(m));
                start = __shfl_sync(0xffffffffu, start, leader);
                if (defer) ws.fb_list[mode][start + __popc(m & ((1u << lane) - 1u))] = (uint32_t)idx;
            }
        }
        if (!__syncthreads_and(y.ok)) break;
    }
    tc_teardown(S, y, kCols, ws.status);
}

// ---------------------------------------------------------------------------------------------------
// Step 2 tiles: rows = pixels x n_shade samples; NeRF weights streamed layer by layer through one
// shared-memory slot.  The copy of layer l+1 (or of the next tile's layer 0) is issued as soon
// as the MMAs of layer l have completed and overlaps the epilogue of layer l.
// ---------------------------------------------------------------------------------------------------
template <int N>
__device__ __forceinline__ int shade_tile_type(const Counters &C, int n_types, unsigned long long tile)
{
    int t = 0;
    while (t + 1 < n_types && C.h_tile[t + 1] <= tile) ++t;
    return t;
}

// MODE 0: rows of Step 2 (pixels x n_shade samples around the stored depth), composited per
//         pixel.  MODE 1: sample rows of the plain method's colour frame (runs of samples of
//         one (ray, instance) pair), weighted by T * alpha and summed per pair.
template <int N, int MODE>
__global__ void __launch_bounds__(kTcThreads, 1)
k_shade_tc(Workspace ws, MarchBuffers mb, const uint8_t *blobs, size_t blob_stride, int npix, int n_samples)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ TcSmem S;
    __shared__ float sig_s[kTcRows], rgb_s[kTcRows][3];
    __shared__ uint32_t pix_s[kTcRows];
    __shared__ float wdelta_s[kTcRows];
    const int L = ws.nerf_hidden;
    constexpr int K0 = kNerfInPad;
    constexpr int KA = K0 > N ? K0 : N;
    const size_t wbytes = tc_w_bytes(K0, N, L);
    const uint32_t f32_bytes = (uint32_t)(tc_f32_floats(N, L, 3) * 4);
    const size_t slot_bytes = (size_t)N * KA * 2;
    uint8_t *Wslot = smem;
    float *f32 = reinterpret_cast<float *>(smem + ((slot_bytes + 1023) & ~(size_t)1023));
    uint8_t *A = reinterpret_cast<uint8_t *>(f32) + ((f32_bytes + 1023) & ~(size_t)1023);
    const int r = threadIdx.x, warp = threadIdx.x >> 5;
    constexpr uint32_t kCols = N < 32 ? 32 : N;

    tc_setup(S, kCols);
    const uint32_t tmem = S.tmem_base;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    TcSync y;
    int f32_type = -1, prefetched = -1;

    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    const int ns = f.n_shade;
    const int ppt = kTcRows / ns;
    const unsigned long long *tile_off = MODE == 0 ? C.h_tile : mb.row_tile;
    const unsigned long long n_tiles = tile_off[f.n_types];
    auto tile_type = [&](unsigned long long tile) {
        int t = 0;
        while (t + 1 < f.n_types && tile_off[t + 1] <= tile) ++t;
        return t;
    };
    auto layer_off = [&](int l) -> size_t { return l == 0 ? 0 : (size_t)K0 * N * 2 + (size_t)(l - 1) * N * N * 2; };
    auto layer_bytes = [&](int l) -> uint32_t { return (uint32_t)((size_t)N * (l == 0 ? K0 : N) * 2); };

    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int t = tile_type(tile);
        const DevType T = ws.types[t];
        const uint8_t *blob = blobs + (size_t)t * blob_stride;
        // weights of layer 0 (unless prefetched) and, on a type change, the fp32 block
        if (prefetched != t) {
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&S.bar_w, layer_bytes(0));
                bulk_g2s(Wslot, blob, layer_bytes(0), &S.bar_w);
            }
            y.w_pending = true;
        }
        if (f32_type != t) {
            if (threadIdx.x == 0) {
                mbar_arrive_expect_tx(&S.bar_f, f32_bytes);
                bulk_g2s(f32, blob + wbytes, f32_bytes, &S.bar_f);
            }
            y.f_pending = true;
            f32_type = t;
        }
        prefetched = -1;
        // ---- row set-up: sample position and its density / weight ----------------------------
        float x6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        float sig = 0.f;
        int n_pix = 0;                       // MODE 0: pixels in the tile
        uint32_t pair = 0xFFFFFFFFu;         // MODE 1: the row's pair
        if (MODE == 0) {
            const unsigned long long first = (tile - C.h_tile[t]) * ppt;
            n_pix = first < C.h_count[t] ? (int)min((unsigned long long)ppt, C.h_count[t] - first) : 0;
            const int q = r / ns, j = r - q * ns;
            if (q < n_pix) {
                uint32_t p = ws.hlist[(size_t)t * npix + first + q];
                DevInst I = ws.inst[ws.id[p]];
                V3 o, d, ol, dl;
                camera_ray(f, p % f.W, p / f.W, o, d);
                to_local(I, o, d, ol, dl);
                float Dl = ws.depth[p] / I.s;
                float delta = 2.0f * f.shade_half / ns;
                float tj = Dl - f.shade_half + (j + 0.5f) * delta;
                V3 x = madd(ol, tj, dl);
                x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
                sig = density(T, x, f.sigma_max, f.sdf_width);
                if (j == 0) { pix_s[q] = p; wdelta_s[q] = I.s * delta; }
            }
        } else {
            const unsigned long long end = min(mb.row_cursor[t], mb.row_off[t + 1]);
            const unsigned long long row_i = mb.row_off[t] + (tile - mb.row_tile[t]) * kTcRows + r;
            if (row_i < end) {
                uint2 row = mb.rows[row_i];
                uint2 pr = ws.ppairs[row.x];
                DevInst I = ws.inst[pr.y];
                V3 o, d, ol, dl;
                camera_ray(f, pr.x % f.W, pr.x / f.W, o, d);
                to_local(I, o, d, ol, dl);
                Chord ch;
                bound_chord(ol, dl, T.rb, ch);
                float dt = (ch.tx - ch.te) / n_samples;
                float Tr = mb.T_first[row.x];      // transmittance at sample k from the pair's first row
                for (int jj = mb.k_first[row.x]; jj < (int)row.y; ++jj) {
                    float sj = density(T, madd(ol, ch.te + (jj + 0.5f) * dt, dl), f.sigma_max, f.sdf_width);
                    Tr *= expf(-sj * I.s * dt);
                }
                V3 x = madd(ol, ch.te + (row.y + 0.5f) * dt, dl);
                x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
                sig = Tr * (1.0f - expf(-density(T, x, f.sigma_max, f.sdf_width) * I.s * dt));   // weight
                pair = row.x;
            }
            pix_s[r] = pair;
        }
        sig_s[r] = sig;
        {
            float feat[K0];
            encode<3, 10>(x6, feat);
            encode<3, 4>(x6 + 3, feat + 63);
            store_row_bf16<K0>(A, r, feat, kNerfIn);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_wait(&S.bar_f, y.f_phase, y.f_pending, y, ws.status);
        float out[3] = {0.f, 0.f, 0.f};
        for (int l = 0; l < L; ++l) {
            const int K = l == 0 ? K0 : N;
            tc_wait(&S.bar_w, y.w_phase, y.w_pending, y, ws.status);          // layer l landed
            if (threadIdx.x == 0 && y.ok) issue_layer(tmem, A, Wslot, K, N, &S.bar_mma);
            y.mma_pending = y.ok;
            tc_wait(&S.bar_mma, y.mma_phase, y.mma_pending, y, ws.status);
            tc_fence_after();
            // the slot is free again: fetch the next layer, or the next tile's layer 0
            int next_t = -1;
            const uint8_t *next_src = nullptr;
            if (l + 1 < L) {
                next_src = blob + layer_off(l + 1);
            } else {
                unsigned long long nt = tile + gridDim.x;
                if (nt < n_tiles) {
                    next_t = tile_type(nt);
                    next_src = blobs + (size_t)next_t * blob_stride;
                }
            }
            if (next_src && y.ok) {
                if (threadIdx.x == 0) {
                    uint32_t nb = layer_bytes(l + 1 < L ? l + 1 : 0);
                    mbar_arrive_expect_tx(&S.bar_w, nb);
                    bulk_g2s(Wslot, next_src, nb, &S.bar_w);
                }
                y.w_pending = true;
                if (l + 1 == L) prefetched = next_t;
            }
            if (l + 1 < L) {
                epilogue_hidden<N>(tmem_row, f32 + l * N, A, r);
                fence_proxy_async_smem();
            } else {
                epilogue_out<N, 3>(tmem_row, f32 + l * N, f32 + L * N, f32 + L * N + 3 * N, out);
            }
            tc_fence_before();
            __syncthreads();
        }
        const float wr = MODE == 0 ? 1.0f : sig;
#pragma unroll
        for (int c = 0; c < 3; ++c) rgb_s[r][c] = wr / (1.0f + expf(-out[c]));
        __syncthreads();
        if (MODE == 0) {
            // front-to-back composite over each pixel's samples (Eq. 8 over the window)
            if (r < n_pix) {
                float Tr = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, Aa = 0.f;
                for (int k = 0; k < ns; ++k) {
                    int rr = r * ns + k;
                    float alpha = 1.0f - expf(-sig_s[rr] * wdelta_s[r]);
                    float w = Tr * alpha;
                    cr += w * rgb_s[rr][0]; cg += w * rgb_s[rr][1]; cb += w * rgb_s[rr][2]; Aa += w;
                    Tr *= 1.0f - alpha;
                }
                ws.rgba[pix_s[r]] = make_float4(cr, cg, cb, Aa);
            }
        } else {
            // one sum per run of rows of the same pair (runs are contiguous)
            if (pair != 0xFFFFFFFFu && (r == 0 || pix_s[r - 1] != pair)) {
                float a = 0.f, b = 0.f, c = 0.f;
                for (int k = r; k < kTcRows && pix_s[k] == pair; ++k) { a += rgb_s[k][0]; b += rgb_s[k][1]; c += rgb_s[k][2]; }
                atomicAdd(&mb.C[pair].x, a);
                atomicAdd(&mb.C[pair].y, b);
                atomicAdd(&mb.C[pair].z, c);
            }
        }
        if (!__syncthreads_and(y.ok)) break;
    }
    tc_teardown(S, y, kCols, ws.status);
}

// ---------------------------------------------------------------------------------------------------
// Deferred plain-method pairs (low confidence or outliers), one thread per pair
// ---------------------------------------------------------------------------------------------------
__global__ void k_fallback(Workspace ws, int mode)
{
    const DevFrame &f = *ws.frame;
    const unsigned long long n = ws.cnt->fb_count[mode];
    const uint2 *pairs = mode == 1 ? ws.spairs : ws.ppairs;
    for (unsigned long long e = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; e < n;
         e += (unsigned long long)gridDim.x * blockDim.x) {
        uint2 pr = pairs[ws.fb_list[mode][e]];
        const DevType T = ws.types[ws.inst[pr.y].type];
        PairRay R;
        setup_pair_ray(ws, f, mode == 1, pr, T.rb, R);
        bool hit = false;
        float Dl = march_crossing(T, R.ol, R.dl, R.te, R.tx, f.march_steps, f.march_bisect, hit);
        if (hit) apply_hit(ws, f, mode == 1, R, Dl);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ws.cnt->fallback, n);
}

cudaError_t launch_fallback(const Workspace &ws, int mode, int num_sms, cudaStream_t st)
{
    k_fallback<<<num_sms * 8, 128, 0, st>>>(ws, mode);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------
// launches
// ---------------------------------------------------------------------------------------------------
template <int N>
static size_t nedf_tc_smem(int L)
{
    constexpr int KA = kNedfInPad > N ? kNedfInPad : N;
    return tc_blob_bytes(kNedfInPad, N, L, 2) + (size_t)kTcRows * KA * 2;
}

template <int N>
static size_t shade_tc_smem(int L)
{
    constexpr int KA = kNerfInPad > N ? kNerfInPad : N;
    size_t slot = ((size_t)N * KA * 2 + 1023) & ~(size_t)1023;
    size_t f = (tc_f32_floats(N, L, 3) * 4 + 1023) & ~(size_t)1023;
    return slot + f + (size_t)kTcRows * KA * 2;
}

template <int N>
static cudaError_t launch_nedf_tc_n(const Workspace &ws, const uint8_t *blobs, size_t stride, int mode, int type,
                                    const float *o, const float *d, float4 *out, int n, int grid, cudaStream_t st)
{
    size_t sm = nedf_tc_smem<N>(ws.nedf_hidden);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_nedf_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_nedf_tc<N><<<grid, kTcThreads, sm, st>>>(ws, blobs, stride, mode, type, o, d, out, n);
    return cudaGetLastError();
}

cudaError_t launch_nedf_tc(const Workspace &ws, const void *blobs, size_t stride, int mode, int type, const float *o,
                           const float *d, float *out, int n, int num_sms, cudaStream_t st)
{
    int grid = num_sms;
    if (mode == 2) grid = (int)std::min<long long>(num_sms, (n + kTcRows - 1) / kTcRows);
    if (grid < 1) return cudaSuccess;
    const uint8_t *b = (const uint8_t *)blobs;
    float4 *o4 = reinterpret_cast<float4 *>(out);
    switch (ws.nedf_width) {
    case 64: return launch_nedf_tc_n<64>(ws, b, stride, mode, type, o, d, o4, n, grid, st);
    case 128: return launch_nedf_tc_n<128>(ws, b, stride, mode, type, o, d, o4, n, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int N, int MODE>
static cudaError_t launch_shade_tc_n(const Workspace &ws, const MarchBuffers &mb, const uint8_t *blobs, size_t stride,
                                     int npix, int n_samples, int grid, cudaStream_t st)
{
    size_t sm = shade_tc_smem<N>(ws.nerf_hidden);
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_shade_tc<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_shade_tc<N, MODE><<<grid, kTcThreads, sm, st>>>(ws, mb, blobs, stride, npix, n_samples);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_colour_tc(const Workspace &ws, const MarchBuffers &mb, int npix, int n_samples, int num_sms,
                                    cudaStream_t st)
{
    const uint8_t *b = ws.nerf_tc;
    const size_t stride = ws.nerf_tc_stride;
    switch (ws.nerf_width) {
    case 64: return launch_shade_tc_n<64, MODE>(ws, mb, b, stride, npix, n_samples, num_sms, st);
    case 128: return launch_shade_tc_n<128, MODE>(ws, mb, b, stride, npix, n_samples, num_sms, st);
    case 256: return launch_shade_tc_n<256, MODE>(ws, mb, b, stride, npix, n_samples, num_sms, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_shade_tc(const Workspace &ws, const void *, size_t, int npix, int num_sms, cudaStream_t st)
{
    MarchBuffers none{};
    return launch_colour_tc<0>(ws, none, npix, 0, num_sms, st);
}

cudaError_t launch_march_colour_tc(const Workspace &ws, const MarchBuffers &mb, int n_samples, int num_sms,
                                   cudaStream_t st)
{
    return launch_colour_tc<1>(ws, mb, 0, n_samples, num_sms, st);
}

}  // namespace nedf
