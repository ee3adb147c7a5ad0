// SM-pair NeRF engine (width 256; shading and plain-method colour rows): a cluster of two CTAs on
// two SMs runs each hidden layer as tcgen05 MMAs of cta_group::2, M = 256 rows (128 per SM) x
// N = 256 outputs x K = 16 (BF16) or 32 (E4M3).
//
// Method: arXiv 2308.04669, Eq. 8 with the sample window (the radiance field of Step 2 evaluated at
// the samples around the NeDF depth) and the plain method's colour frame.
//
// Why a pair: a one-SM M = 128, N = 256 MMA reads 4 KB of A and 8 KB of B from shared memory every
// 128 cycles, and the weight stream and the epilogue's activation stores come on top, which keeps
// the one-SM engine near the shared-memory bandwidth.  In a pair MMA each SM reads its own 128
// rows of A and only its half of B (128 of the N outputs), so each SM streams half of every layer's
// weights, and the shared memory this frees holds two 256-row tiles ("slots") per cluster, which
// take turns on the tensor pipe: one slot's epilogue (TMEM -> ReLU / rounding -> next A operand)
// runs under the other slot's MMAs.
//
// Per CTA: warps 0-7 epilogue (lane quarter = warp % 4, column half = warp / 4: each thread one
// row and 128 of the 256 columns), warp 8 producer (its own half of each weight chunk, one bulk copy
// per stage, into its own ring), warp 9 the MMA issuer in the even CTA and, in the odd CTA, a relay
// that forwards each filled stage to the even CTA (an arrival on its peer_full barrier).  The even
// CTA's issuer starts a slot's layer once all 16 epilogue warps of both CTAs have arrived on its
// a_ready barrier, and commits each stage's release and each slot's accumulator to the barriers of
// both CTAs.  Every wait is bounded; a timeout sets the status word and ends the CTA's loops, and
// the other CTA's waits then run out as well.
#include "pipe_epi.cuh"
#include "render_launch.h"

#include <algorithm>

namespace nedf {

using namespace tc;

template <bool F8>
struct PairShape {
    static constexpr int N = 256;
    static constexpr int K0 = kNerfInPad;                       // layer-0 input (BF16)
    static constexpr int ONES = N;                              // BF16 hidden-layer bias columns
    static constexpr int A_ROW = F8 ? N : 2 * (ONES + kKC);     // bytes per row of one slot's A
    static constexpr size_t A_BYTES = (size_t)kHalf * A_ROW;   // one slot: this CTA's 128 rows
    static constexpr int HCHUNK = 4096;                         // this CTA's half of a weight chunk
    static constexpr int NH = 18;                               // ring: half-chunks (a layer has <= 17)
    static constexpr int RING = NH * HCHUNK;
    static constexpr int NOUT = 3;
    static constexpr size_t FIXED = 2 * A_BYTES + (size_t)RING;   // + two fp32 blocks
};

// chunks (of K = 16 BF16 or 32 E4M3 inputs) of layer l
template <bool F8>
__device__ __forceinline__ int pair_nk(int l)
{
    return l == 0 ? kNerfInPad / kKC : (F8 ? 256 / 32 : 256 / kKC + 1);
}

// Slices [C0, C1) (8 columns each) of a layer-0 input row, as pipe_store_row writes them.
template <int C0, int C1>
__device__ __forceinline__ void pair_store_slices(uint8_t *A, int r, const float *f, int n_valid)
{
#pragma unroll
    for (int c = C0; c < C1; ++c) {
        uint32_t p[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = c * 8 + 2 * e;
            const float v0 = k < n_valid ? f[k] : (k < n_valid + 2 ? 1.0f : 0.0f);
            const float v1 = k + 1 < n_valid ? f[k + 1] : (k + 1 < n_valid + 2 ? 1.0f : 0.0f);
            p[e] = pack_bf16(v0, v1);
        }
        *reinterpret_cast<uint4 *>(A + a_offset(r, c * 8)) = make_uint4(p[0], p[1], p[2], p[3]);
    }
}

// A hidden layer's epilogue over this thread's 128 columns [cb, cb + 128) of its row: ReLU and
// rounding (BF16, or E4M3 after acc * s + bias when AFF), stored as the next layer's A columns.
template <bool F8, bool AFF>
__device__ __forceinline__ void pair_epi_cols(uint32_t taddr, uint8_t *A, int r, int cb, const float *bias, float s)
{
    uint32_t va[32], vb[32];
    tmem_ld32(taddr, va);
    tmem_wait_ld(va);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 64) {
        tmem_ld32(taddr + c0 + 32, vb);
        if (F8) epi_convert8<AFF>(va, bias + cb + c0, s, A, r, cb + c0);
        else epi_convert(va, A, r, cb + c0);
        tmem_wait_ld(vb);
        if (c0 + 64 < 128) tmem_ld32(taddr + c0 + 64, va);
        if (F8) epi_convert8<AFF>(vb, bias + cb + c0 + 32, s, A, r, cb + c0 + 32);
        else epi_convert(vb, A, r, cb + c0 + 32);
        if (c0 + 64 < 128) tmem_wait_ld(va);
    }
}

// The last hidden layer over the same 128 columns, folded into the three outputs (w_out rows of
// length 256 at wout).
template <bool F8, bool AFF>
__device__ __forceinline__ void pair_epi_fold(uint32_t taddr, int cb, const float *bias, float s, const float *wout,
                                              float *out)
{
    uint32_t va[32], vb[32];
    tmem_ld32(taddr, va);
    tmem_wait_ld(va);
#pragma unroll 1
    for (int c0 = 0; c0 < 128; c0 += 64) {
        tmem_ld32(taddr + c0 + 32, vb);
        if (F8) epi_output8<3, 256, AFF>(va, bias + cb + c0, s, wout + cb + c0, out);
        else epi_output<3, 256>(va, wout + cb + c0, out);
        tmem_wait_ld(vb);
        if (c0 + 64 < 128) tmem_ld32(taddr + c0 + 64, va);
        if (F8) epi_output8<3, 256, AFF>(vb, bias + cb + c0 + 32, s, wout + cb + c0 + 32, out);
        else epi_output<3, 256>(vb, wout + cb + c0 + 32, out);
        if (c0 + 64 < 128) tmem_wait_ld(va);
    }
}

// Bounded wait on a phase completed by arrivals of the other CTA (acquire at cluster scope).
__device__ __forceinline__ bool pair_wait(uint64_t *bar, uint32_t parity, volatile int *abort, uint32_t *status)
{
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!*abort) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if (globaltimer_ns() - t0 > 1000000000ull) {
            atomicOr(status, kStatusTimeout);
            *abort = 1;
            return false;
        }
    }
    return false;
}

template <int MODE, bool F8>
__global__ void __launch_bounds__(kPipeThreads, 1) k_pair(Workspace ws, MarchBuffers mb, PipeArgs a)
{
    static_assert(MODE == kModeShade || MODE == kModeMarch, "NeRF modes only");
    using SH = PairShape<F8>;
    constexpr int N = SH::N, K0 = SH::K0, NOUT = SH::NOUT;
    // stages of GC half-chunks, S = 18 / GC of them; a layer (at most 17 half-chunks) always fits,
    // so a round's two tiles of one type share every stage
    const int want = a.stage_bytes / SH::HCHUNK;
    const int GC = want >= 9 ? 9 : want >= 6 ? 6 : want >= 3 ? 3 : want >= 2 ? 2 : 1;
    const int STAGE = GC * SH::HCHUNK, S = SH::NH / GC;
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ uint64_t a_ready[2], acc_full[2], fin;
    __shared__ uint64_t w_full[SH::NH], w_empty[SH::NH], peer_full[SH::NH];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    // tail scratch: per slot the rows' densities (shade) or sample weights (march), their pixel or
    // pair keys and the pixels' sample lengths; per row the colour and the second column half's sums
    __shared__ float t_sig[2][kHalf], t_wd[2][kHalf];
    __shared__ uint32_t t_key[2][kHalf];
    __shared__ float t_rgb[kHalf][3], t_part[kHalf][3];

    const uint32_t rank = cluster_ctarank();
    const unsigned long long cid = blockIdx.x >> 1, nc = gridDim.x >> 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = ws.nerf_hidden;
    uint8_t *ring = smem + 2 * SH::A_BYTES;
    const int n_f32 = (int)pipe_f32_floats(N, L, NOUT, F8);
    const size_t f32_bytes = ((size_t)n_f32 * 4 + 15) & ~(size_t)15;
    volatile int *abort = &abort_flag;
    auto A_of = [&](int s) { return smem + (size_t)s * SH::A_BYTES; };

    if (warp == 9) tmem_alloc_pair(&tmem_base, 2 * N);
    if (threadIdx.x == 0) {
        for (int j = 0; j < 2; ++j) {
            mbar_init(&a_ready[j], 16);                  // 8 epilogue warps of each CTA
            mbar_init(&acc_full[j], 1);
        }
        mbar_init(&fin, 1);
        for (int q = 0; q < S; ++q) {
            mbar_init(&w_full[q], 1);
            mbar_init(&w_empty[q], 1);
            mbar_init(&peer_full[q], 1);
        }
        abort_flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    cluster_sync();                                      // both CTAs' barriers exist, TMEM allocated
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const unsigned long long n_tiles = pipe_n_tiles<N, MODE>(ws, mb, a);
    const DevFrame &f = *ws.frame;

    if (warp == 8) {
        // ------------------------------ producer (both CTAs: their own halves) ------------------
        if (lane == 0) {
            unsigned long long q = 0;
            RingPos rp;
            for (unsigned long long t0 = cid; t0 < n_tiles && !*abort; t0 += 2 * nc) {
                const bool two = t0 + nc < n_tiles;
                const int ty0 = pipe_tile_type<MODE>(ws, mb, a, t0), ty1 = two ? pipe_tile_type<MODE>(ws, mb, a, t0 + nc) : ty0;
                const bool share = ty0 == ty1;
                for (int l = 0; l < L && !*abort; ++l)
                    for (int s = 0; s < 2 && !*abort; ++s) {
                        if (t0 + s * nc >= n_tiles || (s == 1 && share)) continue;
                        const int nk = pair_nk<F8>(l);
                        const uint8_t *src = a.blobs + (size_t)(s ? ty1 : ty0) * a.blob_stride +
                                             pipe_layer_off(K0, N, l, F8) + (size_t)rank * nk * SH::HCHUNK;
                        for (int c0 = 0; c0 < nk; c0 += GC, ++q, rp.next(S)) {
                            const int st = rp.st;
                            const uint32_t bytes = (uint32_t)(min(GC, nk - c0) * SH::HCHUNK);
                            if (!pipe_wait(&w_empty[st], rp.ph ^ 1u, abort, ws.status)) break;
                            mbar_arrive_expect_tx(&w_full[st], bytes);
                            bulk_g2s(ring + (size_t)st * STAGE, src + (size_t)c0 * SH::HCHUNK, bytes, &w_full[st]);
                        }
                    }
            }
            const unsigned long long q0 = q > (unsigned long long)S ? q - S : 0;
            for (unsigned long long k = q0; k < q; ++k) pipe_drain(&w_full[k % S], (uint32_t)((k / S) & 1u), ws.status);
        }
    } else if (warp == 9) {
        if (lane == 0 && rank == 1) {
            // ------------------------------ relay (odd CTA) -------------------------------------
            // the same fill sequence as this CTA's producer: each completed fill is forwarded to
            // the even CTA's peer_full barrier of that stage
            RingPos rp;
            for (unsigned long long t0 = cid; t0 < n_tiles && !*abort; t0 += 2 * nc) {
                const bool two = t0 + nc < n_tiles;
                const bool share = !two || pipe_tile_type<MODE>(ws, mb, a, t0) == pipe_tile_type<MODE>(ws, mb, a, t0 + nc);
                for (int l = 0; l < L && !*abort; ++l)
                    for (int s = 0; s < 2 && !*abort; ++s) {
                        if (t0 + s * nc >= n_tiles || (s == 1 && share)) continue;
                        const int nk = pair_nk<F8>(l);
                        for (int c0 = 0; c0 < nk; c0 += GC, rp.next(S)) {
                            if (!pipe_wait(&w_full[rp.st], rp.ph, abort, ws.status)) break;
                            mbar_arrive_cluster(mapa_shared(smem_addr(&peer_full[rp.st]), 0));
                        }
                    }
            }
            if (cid < n_tiles) pipe_drain(&fin, 0u, ws.status);   // the even CTA's last MMAs used this SM
        } else if (lane == 0) {
            // ------------------------------ MMA issuer (even CTA) -------------------------------
            unsigned long long ja[2] = {0, 0};
            RingPos rp;
            const uint32_t idb = idesc_bf16(256, N), id8 = idesc_e4m3(256, N);
            for (unsigned long long t0 = cid; t0 < n_tiles && !*abort; t0 += 2 * nc) {
                const bool two = t0 + nc < n_tiles;
                const bool share = !two || pipe_tile_type<MODE>(ws, mb, a, t0) == pipe_tile_type<MODE>(ws, mb, a, t0 + nc);
                for (int l = 0; l < L && !*abort; ++l) {
                    const RingPos rp_layer = rp;
                    for (int s = 0; s < 2 && !*abort; ++s) {
                        if (t0 + s * nc >= n_tiles) continue;
                        if (!pair_wait(&a_ready[s], (uint32_t)(ja[s]++ & 1u), abort, ws.status)) break;
                        tc_fence_after();
                        if (share) rp = rp_layer;
                        const bool release = !share || s == 1 || !two;
                        const int nk = pair_nk<F8>(l);
                        const bool e4m3 = F8 && l > 0;
                        const uint32_t ax = smem_addr(A_of(s)), d = tmem + (uint32_t)(s * N);
                        for (int c0 = 0; c0 < nk; c0 += GC, rp.next(S)) {
                            const int st = rp.st;
                            if (!pipe_wait(&w_full[st], rp.ph, abort, ws.status)) break;
                            if (!pair_wait(&peer_full[st], rp.ph, abort, ws.status)) break;
                            tc_fence_after();
                            uint64_t bd = smem_desc(smem_addr(ring + (size_t)st * STAGE), 128, 256);
                            const int c1 = min(nk, c0 + GC);
                            // chunk c reads A columns [16c, 16c + 16) (BF16) or [32c, 32c + 32)
                            // (E4M3): 4 KB at c * 4096; a BF16 hidden layer's chunk 16 is its bias,
                            // against the constant-one columns at 256 = the same offset
                            // descriptors advance by constant steps of their start-address field (a
                            // per-MMA rebuild in the issuing thread starves the pipe)
                            uint64_t ad = smem_desc(ax + (uint32_t)c0 * 4096u, 2048, 128);
                            if (e4m3) {
                                for (int c = c0; c < c1; ++c) {
                                    mma_e4m3_pair(d, ad, bd, id8, c > 0 ? 1u : 0u);
                                    ad += (uint64_t)(4096 >> 4);
                                    bd += (uint64_t)(SH::HCHUNK >> 4);
                                }
                            } else {
                                for (int c = c0; c < c1; ++c) {
                                    mma_bf16_pair(d, ad, bd, idb, c > 0 ? 1u : 0u);
                                    ad += (uint64_t)(4096 >> 4);
                                    bd += (uint64_t)(SH::HCHUNK >> 4);
                                }
                            }
                            if (release) {
                                mma_commit_pair(smem_addr(&w_empty[st]));
                                mma_commit_pair(mapa_shared(smem_addr(&w_empty[st]), 1));
                            }
                        }
                        mma_commit_pair(smem_addr(&acc_full[s]));
                        mma_commit_pair(mapa_shared(smem_addr(&acc_full[s]), 1));
                    }
                }
            }
            if (cid < n_tiles) {                         // every MMA has completed before TMEM goes
                mma_commit_pair(smem_addr(&fin));
                mma_commit_pair(mapa_shared(smem_addr(&fin), 1));
                pipe_drain(&fin, 0u, ws.status);
            }
        }
    } else {
        // ------------------------------ epilogue (both CTAs) ------------------------------------
        const int ch = warp >> 2;                        // column half: outputs [128 ch, 128 ch + 128)
        const int r = (warp & 3) * 32 + lane;            // row among this CTA's 128 (TMEM lane)
        const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
        float *f32s[2] = {reinterpret_cast<float *>(smem + SH::FIXED),
                          reinterpret_cast<float *>(smem + SH::FIXED + f32_bytes)};
        int f32_type[2] = {-1, -1};
        unsigned long long jb[2] = {0, 0};
        const uint32_t a_ready_even[2] = {mapa_shared(smem_addr(&a_ready[0]), 0), mapa_shared(smem_addr(&a_ready[1]), 0)};
        const Counters &C = *ws.cnt;
        if (!F8 && ch == 0) {
            // the constant-one columns the BF16 hidden-layer biases are folded into: 256 and 257
            for (int s = 0; s < 2; ++s) {
                *reinterpret_cast<uint4 *>(A_of(s) + a_offset(r, SH::ONES)) = make_uint4(pack_bf16(1.0f, 1.0f), 0u, 0u, 0u);
                *reinterpret_cast<uint4 *>(A_of(s) + a_offset(r, SH::ONES + 8)) = make_uint4(0u, 0u, 0u, 0u);
            }
        }
        // this warp's A writes are done: one arrival per warp on the even CTA's a_ready
        auto arrive_a = [&](int s) {
            fence_proxy_async_smem();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(a_ready_even[s]);
        };
        // set-up of slot s for `tile`: its type's fp32 block, the rows' samples, the encoded input
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
            float x6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            float sig = 0.f;                             // shade: density; march: sample weight
            uint32_t key = 0xFFFFFFFFu;
            if (MODE == kModeShade) {
                const int ns = f.n_shade;
                const int ppg = kHalf / ns;              // pixels per CTA and tile
                const unsigned long long first = (tile - C.h_tile[t]) * (unsigned long long)(2 * ppg) + rank * ppg;
                const int qq = r / ns, j = r - qq * ns;
                if (qq < ppg && first + qq < C.h_count[t]) {
                    const uint32_t p = ws.hlist[(size_t)t * a.npix + first + qq];
                    const DevInst I = ws.inst[ws.id[p]];
                    V3 o, d, ol, dl;
                    camera_ray(f, p % f.W, p / f.W, o, d);
                    to_local(I, o, d, ol, dl);
                    const float Dl = ws.depth[p] / I.s;
                    const float delta = 2.0f * f.shade_half / ns;
                    const V3 x = madd(ol, Dl - f.shade_half + (j + 0.5f) * delta, dl);
                    x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
                    sig = density(T, x, f.sigma_max, f.sdf_width);
                    if (j == 0 && ch == 0) {
                        t_key[s][qq] = p;
                        t_wd[s][qq] = I.s * delta;
                    }
                }
            } else {
                const unsigned long long end = min(mb.row_cursor[t], mb.row_off[t + 1]);
                const unsigned long long idx = mb.row_off[t] + (tile - mb.row_tile[t]) * kPipeRows + rank * kHalf + r;
                if (idx < end) {
                    const uint2 row = mb.rows[idx];
                    const uint2 pp = ws.ppairs[row.x];
                    const DevInst I = ws.inst[pp.y];
                    V3 o, d, ol, dl;
                    camera_ray(f, pp.x % f.W, pp.x / f.W, o, d);
                    to_local(I, o, d, ol, dl);
                    Chord chd;
                    bound_chord(ol, dl, T.rb, chd);
                    const float dt = (chd.tx - chd.te) / a.n_samples;
                    float Tr = mb.T_first[row.x];
                    for (int jj = mb.k_first[row.x]; jj < (int)row.y; ++jj)
                        Tr *= expf(-density(T, madd(ol, chd.te + (jj + 0.5f) * dt, dl), f.sigma_max, f.sdf_width) * I.s * dt);
                    const V3 x = madd(ol, chd.te + (row.y + 0.5f) * dt, dl);
                    x6[0] = x.x; x6[1] = x.y; x6[2] = x.z; x6[3] = dl.x; x6[4] = dl.y; x6[5] = dl.z;
                    sig = Tr * (1.0f - expf(-density(T, x, f.sigma_max, f.sdf_width) * I.s * dt));
                    key = row.x;
                }
            }
            if (ch == 0) {
                t_sig[s][r] = sig;
                if (MODE == kModeMarch) t_key[s][r] = key;
            }
            float feat[K0];
            pipe_encode<3, 10>(x6, feat);
            pipe_encode<3, 4>(x6 + 3, feat + 63);
            if (ch == 0) pair_store_slices<0, K0 / 16>(A_of(s), r, feat, kNerfIn);
            else pair_store_slices<K0 / 16, K0 / 8>(A_of(s), r, feat, kNerfIn);
            arrive_a(s);
        };
        // tail of slot s's tile: colour per row, then the shading composite per pixel (or the plain
        // method's per-pair sums); out holds this thread's partial output sums
        auto tail = [&](int s, unsigned long long tile, const float *out) {
            if (ch == 1)
                for (int c = 0; c < 3; ++c) t_part[r][c] = out[c];
            asm volatile("bar.sync 4, 256;" ::: "memory");
            if (ch == 0) {
                const float wr = MODE == kModeShade ? 1.0f : t_sig[s][r];
                for (int c = 0; c < 3; ++c) t_rgb[r][c] = wr / (1.0f + expf(-(out[c] + t_part[r][c])));
            }
            asm volatile("bar.sync 4, 256;" ::: "memory");
            if (ch == 0) {
                const int t = pipe_tile_type<MODE>(ws, mb, a, tile);
                if (MODE == kModeShade) {
                    const int ns = f.n_shade, ppg = kHalf / ns;
                    const unsigned long long first = (tile - C.h_tile[t]) * (unsigned long long)(2 * ppg) + rank * ppg;
                    if (r < ppg && first + r < C.h_count[t]) {
                        float Tr = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, Aa = 0.f, smax = 0.f;
                        const float wd = t_wd[s][r];
                        for (int k = 0; k < ns; ++k) {
                            const int rr = r * ns + k;
                            const float alpha = 1.0f - expf(-t_sig[s][rr] * wd);
                            const float w = Tr * alpha;
                            cr += w * t_rgb[rr][0]; cg += w * t_rgb[rr][1]; cb += w * t_rgb[rr][2]; Aa += w;
                            Tr *= 1.0f - alpha;
                            smax = fmaxf(smax, t_sig[s][rr]);
                        }
                        const uint32_t pix = t_key[s][r];
                        ws.rgba[pix] = make_float4(cr, cg, cb, Aa);
                        flag_shade_outlier(ws, f, pix, smax);
                    }
                } else {
                    // one sum per run of rows of the same pair (runs are contiguous within the CTA's rows)
                    const uint32_t pair = t_key[s][r];
                    if (pair != 0xFFFFFFFFu && (r == 0 || t_key[s][r - 1] != pair)) {
                        float sa = 0.f, sb = 0.f, sc = 0.f;
                        for (int k = r; k < kHalf && t_key[s][k] == pair; ++k) {
                            sa += t_rgb[k][0]; sb += t_rgb[k][1]; sc += t_rgb[k][2];
                        }
                        atomicAdd(&mb.C[pair].x, sa);
                        atomicAdd(&mb.C[pair].y, sb);
                        atomicAdd(&mb.C[pair].z, sc);
                    }
                }
            }
            asm volatile("bar.sync 4, 256;" ::: "memory");
        };
        if (cid < n_tiles) setup(0, cid);
        if (cid + nc < n_tiles) setup(1, cid + nc);
        bool stop = false;
        for (unsigned long long t0 = cid; t0 < n_tiles && !stop; t0 += 2 * nc) {
            for (int l = 0; l < L && !stop; ++l)
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    if (stop) continue;
                    const unsigned long long tile = t0 + s * nc;
                    if (tile >= n_tiles) continue;
                    // tcgen05.ld is warp-collective: a warp-uniform outcome; the last layer's step
                    // (tail, set-up: named barriers) decides for all 256 epilogue threads
                    const bool last = l + 1 == L;
                    const bool okw = __all_sync(0xffffffffu, pipe_wait(&acc_full[s], (uint32_t)(jb[s]++ & 1u), abort, ws.status));
                    const bool ok = last ? !epilogue_any(!okw) : okw;
                    if (ok) {
                        tc_fence_after();
                        const float *f32 = f32s[s];
                        const uint32_t taddr = tmem + lane_q + (uint32_t)(s * N + ch * 128);
                        const float *bias = f32 + pipe_f8_bias_off(N, NOUT) + (size_t)l * N;
                        const float sc = F8 && l > 0 ? f32[pipe_f8_bias_off(N, NOUT) + (size_t)L * N + l] : 1.0f;
                        if (!last) {
                            if (F8 && l > 0) pair_epi_cols<F8, true>(taddr, A_of(s), r, ch * 128, bias, sc);
                            else pair_epi_cols<F8, false>(taddr, A_of(s), r, ch * 128, bias, sc);
                            arrive_a(s);
                        } else {
                            float out[NOUT];
#pragma unroll
                            for (int o = 0; o < NOUT; ++o) out[o] = ch == 0 ? f32[NOUT * N + o] : 0.0f;
                            if (F8 && l > 0) pair_epi_fold<F8, true>(taddr, ch * 128, bias, sc, f32, out);
                            else pair_epi_fold<F8, false>(taddr, ch * 128, bias, sc, f32, out);
                            tc_fence_before();
                            tail(s, tile, out);
                            const unsigned long long nxt = tile + 2 * nc;
                            if (!epilogue_any(*abort != 0) && nxt < n_tiles) setup(s, nxt);
                        }
                    } else {
                        *abort = 1;
                    }
                    if (last) stop = epilogue_any(!ok || *abort);
                }
        }
    }
    // ---- teardown: no CTA of the pair leaves while the other may still reach its shared memory,
    // its barriers or its TMEM ----------------------------------------------------------------------
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (warp == 9) tmem_dealloc_pair(tmem, 2 * N);
}

// ---------------------------------------------------------------------------------------------------
// Launch: clusters of two CTAs, as many as can be resident at once (one CTA per SM), each cluster
// walking tiles cid, cid + nc, ... in rounds of two.  Returns cudaErrorInvalidConfiguration, before
// launching anything, when the shape does not fit (the caller then runs the one-SM engine).
// ---------------------------------------------------------------------------------------------------
template <int MODE, bool F8>
static cudaError_t launch_pair_n(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a, int num_sms,
                                 cudaStream_t st)
{
    using SH = PairShape<F8>;
    const size_t f32b = (pipe_f32_floats(256, ws.nerf_hidden, 3, F8) * 4 + 15) & ~(size_t)15;
    const size_t sm = SH::FIXED + 2 * f32b;
    if (sm > 227 * 1024 - 8192) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_pair<MODE, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2, 1, 1);
    cfg.blockDim = dim3(kPipeThreads, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    e = cudaOccupancyMaxActiveClusters(&clusters, k_pair<MODE, F8>, &cfg);
    if (e != cudaSuccess) return e;
    clusters = std::min(clusters, num_sms / 2);
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    e = cudaLaunchKernelEx(&cfg, k_pair<MODE, F8>, ws, mb, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// mode kModeShade or kModeMarch; a.blobs points at type 0's SM-pair layout
cudaError_t launch_pair_pipe(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a, int mode, int num_sms,
                             cudaStream_t st)
{
    const bool f8 = ws.precision == 2;
    if (mode == kModeShade) return f8 ? launch_pair_n<kModeShade, true>(ws, mb, a, num_sms, st)
                                      : launch_pair_n<kModeShade, false>(ws, mb, a, num_sms, st);
    return f8 ? launch_pair_n<kModeMarch, true>(ws, mb, a, num_sms, st)
              : launch_pair_n<kModeMarch, false>(ws, mb, a, num_sms, st);
}

}  // namespace nedf
