// FP32 render path on CUDA cores: the reference-precision implementation of Steps 1-3.
//
// Method: arXiv 2308.04669, Algorithm 1 and Algorithm 2, Eq. 1-2, 7, 8.
#include "render_kernels.cuh"
#include "mlp_f32.cuh"
#include "render_launch.h"

#include <algorithm>

namespace nedf {

// ---------------------------------------------------------------------------------------------
// frame setup: camera basis (look-at with world up +y) and counter reset
// ---------------------------------------------------------------------------------------------
__global__ void k_setup(Workspace ws, const HostCamera *cam)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        DevFrame &f = *ws.frame;
        V3 eye = v3(cam->eye[0], cam->eye[1], cam->eye[2]);
        V3 fwd = normalized(sub(v3(cam->target[0], cam->target[1], cam->target[2]), eye));
        V3 right = normalized(v3(-fwd.z, 0.0f, fwd.x));          // fwd x (0,1,0)
        V3 up = v3(right.y * fwd.z - right.z * fwd.y, right.z * fwd.x - right.x * fwd.z,
                   right.x * fwd.y - right.y * fwd.x);           // right x fwd
        f.eye[0] = eye.x; f.eye[1] = eye.y; f.eye[2] = eye.z;
        f.fwd[0] = fwd.x; f.fwd[1] = fwd.y; f.fwd[2] = fwd.z;
        f.right[0] = right.x; f.right[1] = right.y; f.right[2] = right.z;
        f.up[0] = up.x; f.up[1] = up.y; f.up[2] = up.z;
        f.tan_h = tanf(0.5f * cam->fov_y_deg * 0.017453292519943295f);
        f.aspect = (float)f.W / (float)f.H;
    }
    unsigned long long *c = reinterpret_cast<unsigned long long *>(ws.cnt);
    for (int i = threadIdx.x; i < (int)(sizeof(Counters) / 8); i += blockDim.x) c[i] = 0ull;
    if (ws.rs_cnt) {
        unsigned long long *cr = reinterpret_cast<unsigned long long *>(ws.rs_cnt);
        for (int i = threadIdx.x; i < (int)(sizeof(Counters) / 8); i += blockDim.x) cr[i] = 0ull;
    }
}

__global__ void k_clear(Workspace ws, int npix)
{
    const bool edit = ws.frame->edit_mode == 2;            // an edit frame starts from the frozen part
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        ws.keys[p] = edit ? ws.edit_keys[p] : ~0ull;
        ws.occl[p] = edit ? ws.edit_occl[p] : 0u;
        if (ws.rs_mask) ws.rs_mask[p] = 0u;
    }
}

// ---------------------------------------------------------------------------------------------
// Step 1 binning: conservative screen rectangle of each instance's bound sphere, exact cull of
// every pixel ray inside it.  pass 0 counts pairs per type, pass 1 writes them.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool screen_rect(const DevFrame &f, V3 c, float r, int &i0, int &i1, int &j0, int &j1)
{
    V3 e = sub(c, v3(f.eye[0], f.eye[1], f.eye[2]));
    float cx = dot(e, v3(f.right[0], f.right[1], f.right[2]));
    float cy = dot(e, v3(f.up[0], f.up[1], f.up[2]));
    float cz = dot(e, v3(f.fwd[0], f.fwd[1], f.fwd[2]));
    if (cz <= r * 1.001f + 1e-6f) {           // bound reaches behind the eye plane: whole image
        i0 = 0; i1 = f.W - 1; j0 = 0; j1 = f.H - 1;
        return true;
    }
    // Tangent planes through the eye: (c_a - u c_z)^2 = r^2 (1 + u^2).
    float den = cz * cz - r * r;
    float sx = r * sqrtf(fmaxf(cx * cx + cz * cz - r * r, 0.f));
    float sy = r * sqrtf(fmaxf(cy * cy + cz * cz - r * r, 0.f));
    float u0 = (cx * cz - sx) / den, u1 = (cx * cz + sx) / den;
    float v0 = (cy * cz - sy) / den, v1 = (cy * cz + sy) / den;
    float su = f.W * 0.5f / (f.tan_h * f.aspect), sv = f.H * 0.5f / f.tan_h;
    float fi0 = u0 * su + f.W * 0.5f - 0.5f, fi1 = u1 * su + f.W * 0.5f - 0.5f;
    float fj0 = -v1 * sv + f.H * 0.5f - 0.5f, fj1 = -v0 * sv + f.H * 0.5f - 0.5f;
    if (!(fi1 >= -2.f && fi0 <= f.W + 1.f && fj1 >= -2.f && fj0 <= f.H + 1.f)) return false;
    i0 = max(0, (int)floorf(fi0) - 2); i1 = min(f.W - 1, (int)ceilf(fi1) + 2);
    j0 = max(0, (int)floorf(fj0) - 2); j1 = min(f.H - 1, (int)ceilf(fj1) + 2);
    return i0 <= i1 && j0 <= j1;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// One block per instance: the pixels of the conservative screen rectangle of its bound sphere,
// each culled exactly.  PASS 0 counts the kept pairs (pinst[2 i], and the type's total); after the
// scan (pinst[2 i + 1] = the first index of the instance's range in its type's segment) PASS 1
// writes them there with a shared-memory cursor, so no global counter is contended.
template <int PASS>
__global__ void __launch_bounds__(kThreads) k_bin_primary(Workspace ws)
{
    const DevFrame &f = *ws.frame;
    int inst = blockIdx.x;
    if (inst >= f.n_inst) return;
    // buffer reuse: the frozen part leaves the manipulated instance out, an edit frame has only it
    const bool skip = (f.edit_mode == 1 && inst == f.edit_inst) || (f.edit_mode == 2 && inst != f.edit_inst);
    DevInst I = ws.inst[inst];
    DevType T = ws.types[I.type];
    int i0 = 0, i1 = -1, j0 = 0, j1 = -1;
    if (skip || !screen_rect(f, v3(I.T[0], I.T[1], I.T[2]), T.rb * I.s, i0, i1, j0, j1)) {
        if (PASS == 0 && threadIdx.x == 0) ws.pinst[2 * inst] = 0;
        return;
    }
    int bw = i1 - i0 + 1, npx = bw * (j1 - j0 + 1);
    __shared__ unsigned long long blk_count, s_cur, s_beg, s_end;
    if (threadIdx.x == 0) {
        if (PASS == 0) {
            blk_count = 0;
        } else {
            s_beg = s_cur = ws.pinst[2 * inst + 1];
            s_end = min(s_beg + ws.pinst[2 * inst], ws.cnt->p_off[I.type + 1]);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned local = 0;
    for (int base = 0; base < npx; base += blockDim.x) {
        int p = base + threadIdx.x;
        bool keep = false;
        int i = 0, j = 0;
        V3 ol = v3(0, 0, 0), dl = v3(0, 0, 0);
        Chord c{};
        if (p < npx) {
            i = i0 + p % bw; j = j0 + p / bw;
            V3 o, d;
            camera_ray(f, i, j, o, d);
            to_local(I, o, d, ol, dl);
            keep = bound_chord(ol, dl, T.rb, c);
        }
        if (PASS == 0) {
            local += keep;
        } else {
            const unsigned mask = __ballot_sync(0xffffffffu, keep);
            if (!mask) continue;
            const int leader = __ffs(mask) - 1;
            unsigned long long start = 0;
            if (lane == leader) start = atomicAdd(&s_cur, (unsigned long long)__popc(mask));
            start = __shfl_sync(0xffffffffu, start, leader);
            if (keep) {
                const unsigned long long idx = start + __popc(mask & lanemask_lt());
                if (idx < s_end) {
                    ws.ppairs[idx] = make_uint2((uint32_t)(j * f.W + i), (uint32_t)inst);
                    if (ws.pair_geo) {
                        ws.pgeo[2 * idx] = make_float4(ol.x, ol.y, ol.z, c.te);
                        ws.pgeo[2 * idx + 1] = make_float4(dl.x, dl.y, dl.z, c.tp);
                    }
                } else {
                    atomicOr(ws.status, kStatusPrimaryOverflow);
                }
            }
        }
    }
    if (PASS == 0) {
        for (int o = 16; o; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
        if (lane == 0 && local) atomicAdd(&blk_count, (unsigned long long)local);
        __syncthreads();
        if (threadIdx.x == 0) {
            ws.pinst[2 * inst] = blk_count;
            if (blk_count) atomicAdd(&ws.cnt->p_count[I.type], blk_count);
        }
    } else {
        __syncthreads();
        if (threadIdx.x == 0 && s_end > s_beg) atomicAdd(&ws.cnt->p_cursor[I.type], min(s_cur, s_end) - s_beg);
    }
}

// Prefix sums of a list's per-type counts (clamped to the capacity) and of its tiles.
__device__ void scan_list(unsigned long long *count, unsigned long long *cursor, unsigned long long *off,
                          unsigned long long *tile, int n_types, long long cap, int rows_per_tile,
                          uint32_t *status, uint32_t flag, unsigned long long *requested)
{
    unsigned long long o = 0, t = 0, req = 0;
    for (int k = 0; k < n_types; ++k) {
        req += count[k];
        unsigned long long c = count[k];
        if (o + c > (unsigned long long)cap) {
            c = (unsigned long long)cap - o;
            *status |= flag;
        }
        count[k] = c;
        off[k] = o;
        cursor[k] = o;
        tile[k] = t;
        o += c;
        t += (c + rows_per_tile - 1) / rows_per_tile;
    }
    off[n_types] = o;
    tile[n_types] = t;
    if (requested) *requested = req;
}

// The type segments (thread 0), then each instance's range inside its type's segment (any
// disjoint order: a shared-memory running offset per type).
__global__ void __launch_bounds__(1024) k_scan_primary(Workspace ws, int rows_per_tile)
{
    __shared__ unsigned long long s_run[kMaxTypes];
    const DevFrame &f = *ws.frame;
    if (threadIdx.x == 0)
        scan_list(ws.cnt->p_count, ws.cnt->p_cursor, ws.cnt->p_off, ws.cnt->p_tile, f.n_types, ws.pcap,
                  rows_per_tile, ws.status, kStatusPrimaryOverflow, &ws.cnt->p_total_requested);
    __syncthreads();
    if (threadIdx.x < f.n_types) s_run[threadIdx.x] = ws.cnt->p_off[threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.x; i < f.n_inst; i += blockDim.x) {
        const unsigned long long c = ws.pinst[2 * i];
        ws.pinst[2 * i + 1] = c ? atomicAdd(&s_run[ws.inst[i].type], c) : 0ull;
    }
}

__global__ void k_scan_shade(Workspace ws, int pixels_per_tile)
{
    const DevFrame &f = *ws.frame;
    unsigned long long t = 0;
    for (int k = 0; k < f.n_types; ++k) {
        ws.cnt->h_tile[k] = t;
        t += (ws.cnt->h_count[k] + pixels_per_tile - 1) / pixels_per_tile;
    }
    ws.cnt->h_tile[f.n_types] = t;
}

// ---------------------------------------------------------------------------------------------
// NeDF tiles (Step 1 primary pairs, Step 3 shadow pairs)
// ---------------------------------------------------------------------------------------------
struct RowInfo {
    float x6[6];     // entry point on the bound, local direction
    float ol[3], dl[3];
    float te, tx, tp, s, rb;
    float ell;       // shadow: distance light -> surface point
    uint32_t key;    // primary: pixel; shadow: pixel * n_lights + light
    uint32_t inst;
    int valid;
};

template <int W_HID>
__global__ void __launch_bounds__(kThreads) k_nedf_tiles(Workspace ws, int shadow_pass)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ RowInfo rows[kTileRows];
    __shared__ float y[kTileRows][4];
    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    const unsigned long long *tile_off = shadow_pass ? C.s_tile : C.p_tile;
    const unsigned long long *pair_off = shadow_pass ? C.s_off : C.p_off;
    const uint2 *pairs = shadow_pass ? ws.spairs : ws.ppairs;
    const int n_types = f.n_types;
    const unsigned long long n_tiles = tile_off[n_types];
    const bool use_march = f.depth_source == 1;

    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int t = 0;
        while (t + 1 < n_types && tile_off[t + 1] <= tile) ++t;
        unsigned long long begin = pair_off[t] + (tile - tile_off[t]) * kTileRows;
        unsigned long long end = pair_off[t + 1];
        const DevType T = ws.types[t];
        // rays of the tile's rows
        if (threadIdx.x < kTileRows) {
            RowInfo &ri = rows[threadIdx.x];
            unsigned long long idx = begin + threadIdx.x;
            ri.valid = idx < end;
            for (int c = 0; c < 6; ++c) ri.x6[c] = 0.0f;
            if (ri.valid) {
                uint2 pr = pairs[idx];
                DevInst I = ws.inst[pr.y];
                V3 o, d;
                if (!shadow_pass) {
                    camera_ray(f, pr.x % f.W, pr.x / f.W, o, d);
                } else {
                    uint32_t pix = pr.x / f.n_lights, l = pr.x - pix * f.n_lights;
                    V3 oc, dc;
                    camera_ray(f, pix % f.W, pix / f.W, oc, dc);
                    V3 x = madd(oc, ws.depth[pix], dc);
                    light_ray(ws.lcam, f, (int)l, x, o, d, ri.ell);
                }
                V3 ol, dl;
                to_local(I, o, d, ol, dl);
                Chord ch;
                bound_chord(ol, dl, T.rb, ch);
                V3 pe = madd(ol, ch.te, dl);
                ri.x6[0] = pe.x; ri.x6[1] = pe.y; ri.x6[2] = pe.z;
                ri.x6[3] = dl.x; ri.x6[4] = dl.y; ri.x6[5] = dl.z;
                ri.ol[0] = ol.x; ri.ol[1] = ol.y; ri.ol[2] = ol.z;
                ri.dl[0] = dl.x; ri.dl[1] = dl.y; ri.dl[2] = dl.z;
                ri.te = ch.te; ri.tx = ch.tx; ri.tp = ch.tp; ri.s = I.s; ri.rb = T.rb;
                ri.key = pr.x; ri.inst = pr.y;
            }
        }
        __syncthreads();
        if (!use_march) {
            // features: identity, 6 sine blocks, 6 cosine blocks of the 6-D input
            for (int e = threadIdx.x; e < kTileRows * kNedfIn; e += blockDim.x) {
                int r = e % kTileRows, fi = e / kTileRows;
                X[fi * kXStride + r] = posenc_feature(rows[r].x6, 6, 6, fi);
            }
            __syncthreads();
            const float *w = ws.nedf_w + (size_t)t * ws.nedf_stride;
            mlp_hidden_f32<W_HID>(X, kNedfIn, ws.nedf_hidden, w);
            const float *wo = w + (size_t)kNedfIn * W_HID + W_HID + (size_t)(ws.nedf_hidden - 1) * (W_HID * W_HID + W_HID);
            out_layer_f32(X, W_HID, wo, wo + W_HID * 2, 2, y);
        }
        // decode (Eq. 2, Eq. 7), fallback, refinement, then z-min or occlusion
        if (threadIdx.x < kTileRows && rows[threadIdx.x].valid) {
            const RowInfo &ri = rows[threadIdx.x];
            V3 ol = v3(ri.ol[0], ri.ol[1], ri.ol[2]), dl = v3(ri.dl[0], ri.dl[1], ri.dl[2]);
            float Dl;
            bool hit;
            if (use_march) {
                Dl = march_crossing_skip(T, ol, dl, ri.te, ri.tx, f.march_steps, f.march_bisect, hit);
            } else {
                if (nedf_decode(f, T, ol, dl, ri.tp, y[threadIdx.x][0], y[threadIdx.x][1], Dl, hit)) {
                    Dl = march_crossing_skip(T, ol, dl, ri.te, ri.tx, f.march_steps, f.march_bisect, hit);
                    atomicAdd(&ws.cnt->fallback, 1ull);
                }
            }
            if (hit) {
                float D = ri.s * Dl;
                if (!shadow_pass) {
                    unsigned long long key = ((unsigned long long)__float_as_uint(D) << 32) | ri.inst;
                    atomicMin(&ws.keys[ri.key], key);
                } else if (D + f.eps < ri.ell) {
                    uint32_t pix = ri.key / f.n_lights, l = ri.key - pix * f.n_lights;
                    atomicOr(&ws.occl[pix], 1u << l);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Step 1 resolve: packed keys -> depth / id buffers, per-type lists of pixels to shade
// ---------------------------------------------------------------------------------------------
// Each block resolves kResolvePix x 256 pixels at a time: every thread takes kResolvePix pixels
// 256 apart (coalesced key reads and depth / id writes), ranks its listed pixels inside the
// block's per-type counts with shared-memory atomics (one per warp and type), and the block then
// reserves its range of each type's shading list and adds its hit count with one global atomic
// each, so the frame's few per-type counters see a few hundred atomics instead of one per warp.
constexpr int kResolvePix = 8;

__global__ void __launch_bounds__(256) k_resolve(Workspace ws, int npix)
{
    __shared__ unsigned s_cnt[kMaxTypes];
    __shared__ unsigned long long s_base[kMaxTypes];
    __shared__ unsigned s_hits;
    const DevFrame &f = *ws.frame;
    const int lane = threadIdx.x & 31;
    const int n_types = f.n_types;
    const long long per_block = (long long)kResolvePix * blockDim.x;
    for (long long b0 = (long long)blockIdx.x * per_block; b0 < npix; b0 += (long long)gridDim.x * per_block) {
        if (threadIdx.x < kMaxTypes) s_cnt[threadIdx.x] = 0u;
        if (threadIdx.x == 0) s_hits = 0u;
        __syncthreads();
        // every load first (the keys, then their instances' types), so that each thread has
        // kResolvePix independent loads in flight instead of a chain per pixel
        unsigned long long key[kResolvePix];
        uint32_t ty[kResolvePix], pos[kResolvePix];
#pragma unroll
        for (int i = 0; i < kResolvePix; ++i) {
            const long long p = b0 + (long long)i * blockDim.x + threadIdx.x;
            key[i] = p < npix ? ws.keys[p] : ~0ull;
        }
#pragma unroll
        for (int i = 0; i < kResolvePix; ++i) ty[i] = key[i] != ~0ull ? ws.inst[(uint32_t)key[i]].type : 0xFFFFFFFFu;
#pragma unroll
        for (int i = 0; i < kResolvePix; ++i) {
            const long long p = b0 + (long long)i * blockDim.x + threadIdx.x;
            const bool in = p < npix;
            const unsigned long long k = key[i];
            float D = __int_as_float(0x7f800000);
            uint32_t id = kNoId;
            const bool hit = k != ~0ull;
            uint32_t t = ty[i];
            if (hit) {
                D = __uint_as_float((uint32_t)(k >> 32));
                id = (uint32_t)(k & 0xffffffffu);
            }
            // an edit frame shades and fully re-shadows only the pixels the manipulated instance
            // wins; every other pixel keeps the frozen part's colour and occlusion bits
            if (f.edit_mode == 2 && hit) {
                const bool listed = id == (uint32_t)f.edit_inst;
                if (listed) ws.occl[p] = 0u;
                else ws.rgba[p] = ws.edit_rgba[p];
                if (!listed) t = 0xFFFFFFFFu;
            }
            const unsigned peers = __match_any_sync(0xffffffffu, t);
            const unsigned hits = __ballot_sync(0xffffffffu, hit);
            uint32_t r = 0u;
            if (t != 0xFFFFFFFFu) {
                const int leader = __ffs(peers) - 1;
                if (lane == leader) r = atomicAdd(&s_cnt[t], (unsigned)__popc(peers));
                r = __shfl_sync(peers, r, leader) + __popc(peers & ((1u << lane) - 1u));
            }
            if (lane == 0 && hits) atomicAdd(&s_hits, (unsigned)__popc(hits));
            ty[i] = t;
            pos[i] = r;
            if (in) {
                ws.depth[p] = D;
                ws.id[p] = id;
                if (!hit) ws.rgba[p] = make_float4(0.f, 0.f, 0.f, 0.f);   // hit pixels are written by Step 2
            }
        }
        __syncthreads();
        if (threadIdx.x < n_types) {
            const unsigned c = s_cnt[threadIdx.x];
            s_base[threadIdx.x] = c ? atomicAdd(&ws.cnt->h_count[threadIdx.x], (unsigned long long)c) : 0ull;
        }
        if (threadIdx.x == 32 && s_hits) atomicAdd(&ws.cnt->hit_pixels, (unsigned long long)s_hits);
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kResolvePix; ++i)
            if (ty[i] != 0xFFFFFFFFu)
                ws.hlist[(size_t)ty[i] * npix + s_base[ty[i]] + pos[i]] = (uint32_t)(b0 + (long long)i * blockDim.x + threadIdx.x);
        __syncthreads();                          // s_cnt / s_base are reset for the next chunk
    }
}

// ---------------------------------------------------------------------------------------------
// Step 2: deferred shading.  Tile rows = pixels x n_shade samples of the winning instance.
// ---------------------------------------------------------------------------------------------
template <int W_NERF>
__global__ void __launch_bounds__(kThreads) k_shade_tiles(Workspace ws, int npix)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ float xs[kTileRows][6];     // local sample position, local direction
    __shared__ float sig[kTileRows];
    __shared__ float y[kTileRows][4];
    __shared__ uint32_t tile_pix[kTileRows];
    __shared__ float tile_ws[kTileRows];    // world length of one sample interval
    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    const int ns = f.n_shade;
    const int ppt = kTileRows / ns;
    const int n_types = f.n_types;
    const unsigned long long n_tiles = C.h_tile[n_types];
    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int t = 0;
        while (t + 1 < n_types && C.h_tile[t + 1] <= tile) ++t;
        unsigned long long first = (tile - C.h_tile[t]) * ppt;
        int n_pix = first < C.h_count[t] ? (int)min((unsigned long long)ppt, C.h_count[t] - first) : 0;
        const DevType T = ws.types[t];
        if (threadIdx.x < ppt * ns) {
            int q = threadIdx.x / ns, j = threadIdx.x - q * ns;
            for (int c = 0; c < 6; ++c) xs[threadIdx.x][c] = 0.0f;
            sig[threadIdx.x] = 0.0f;
            if (q < n_pix) {
                uint32_t p = ws.hlist[(size_t)t * npix + first + q];
                if (j == 0) tile_pix[q] = p;
                DevInst I = ws.inst[ws.id[p]];
                V3 o, d, ol, dl;
                camera_ray(f, p % f.W, p / f.W, o, d);
                to_local(I, o, d, ol, dl);
                float Dl = ws.depth[p] / I.s;
                float delta = 2.0f * f.shade_half / ns;
                float tj = Dl - f.shade_half + (j + 0.5f) * delta;
                V3 x = madd(ol, tj, dl);
                xs[threadIdx.x][0] = x.x; xs[threadIdx.x][1] = x.y; xs[threadIdx.x][2] = x.z;
                xs[threadIdx.x][3] = dl.x; xs[threadIdx.x][4] = dl.y; xs[threadIdx.x][5] = dl.z;
                sig[threadIdx.x] = density(T, x, f.sigma_max, f.sdf_width);
                if (j == 0) tile_ws[q] = I.s * delta;
            }
        }
        __syncthreads();
        if (T.nerf) {
            for (int e = threadIdx.x; e < kTileRows * kNerfIn; e += blockDim.x) {
                int r = e % kTileRows, fi = e / kTileRows;
                float v = fi < 63 ? posenc_feature(&xs[r][0], 3, 10, fi) : posenc_feature(&xs[r][3], 3, 4, fi - 63);
                X[fi * kXStride + r] = v;
            }
            __syncthreads();
            const float *w = ws.nerf_w + (size_t)t * ws.nerf_stride;
            mlp_hidden_f32<W_NERF>(X, kNerfIn, ws.nerf_hidden, w);
            const float *wo = w + (size_t)kNerfIn * W_NERF + W_NERF + (size_t)(ws.nerf_hidden - 1) * (W_NERF * W_NERF + W_NERF);
            out_layer_f32(X, W_NERF, wo, wo + W_NERF * 3, 3, y);
        }
        // front-to-back composite of each pixel's samples (Eq. 8 over the window)
        if (threadIdx.x < n_pix) {
            int q = threadIdx.x;
            float Tr = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f, A = 0.f, smax = 0.f;
            for (int j = 0; j < ns; ++j) {
                int r = q * ns + j;
                smax = fmaxf(smax, sig[r]);
                float alpha = 1.0f - expf(-sig[r] * tile_ws[q]);
                float R, G, B;
                if (T.nerf) {
                    R = 1.0f / (1.0f + expf(-y[r][0]));
                    G = 1.0f / (1.0f + expf(-y[r][1]));
                    B = 1.0f / (1.0f + expf(-y[r][2]));
                } else {
                    R = T.albedo[0]; G = T.albedo[1]; B = T.albedo[2];
                }
                float wgt = Tr * alpha;
                cr += wgt * R; cg += wgt * G; cb += wgt * B; A += wgt;
                Tr *= 1.0f - alpha;
            }
            ws.rgba[tile_pix[q]] = make_float4(cr, cg, cb, A);
            flag_shade_outlier(ws, f, tile_pix[q], smax);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------------
// Composite: shadow buffer = mean over lights of (occluded ? beta : 1); out = rgb * shadow
// ---------------------------------------------------------------------------------------------
// Four pixels a grid stride apart per thread and iteration, their loads issued together, so that
// enough bytes are in flight to cover the HBM latency.
__global__ void __launch_bounds__(256) k_composite(Workspace ws, int npix)
{
    const DevFrame &f = *ws.frame;
    const int nl = f.n_lights;
    const float beta = f.beta;
    const int stride = gridDim.x * blockDim.x;
    for (int p0 = blockIdx.x * blockDim.x + threadIdx.x; p0 < npix; p0 += 4 * stride) {
        uint32_t id[4], m[4];
        float4 c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * stride;
            id[u] = p < npix ? ws.id[p] : kNoId;
            c[u] = p < npix ? ws.rgba[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) m[u] = id[u] != kNoId ? ws.occl[p0 + u * stride] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * stride;
            if (p >= npix) break;
            float S = 1.0f;
            if (id[u] != kNoId) {
                const int occ = __popc(m[u]);
                S = ((nl - occ) * 1.0f + occ * beta) / nl;
            }
            ws.shadow[p] = S;
            ws.out[p] = make_float4(c[u].x * S, c[u].y * S, c[u].z * S, c[u].w);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// host-side launch sequence of one FP32 frame
// ---------------------------------------------------------------------------------------------
template <int W>
static size_t nedf_smem() { return (size_t)(W > kNedfInPad ? W : kNedfInPad) * kXStride * sizeof(float); }
template <int W>
static size_t nerf_smem() { return (size_t)(W > kNerfInPad ? W : kNerfInPad) * kXStride * sizeof(float); }

template <int W>
static cudaError_t launch_nedf(const Workspace &ws, int grid, int shadow_pass, cudaStream_t st)
{
    size_t sm = nedf_smem<W>();
    cudaError_t e = cudaFuncSetAttribute(k_nedf_tiles<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_nedf_tiles<W><<<grid, kThreads, sm, st>>>(ws, shadow_pass);
    return cudaGetLastError();
}

template <int W>
static cudaError_t launch_shade(const Workspace &ws, int grid, int npix, cudaStream_t st)
{
    size_t sm = nerf_smem<W>();
    cudaError_t e = cudaFuncSetAttribute(k_shade_tiles<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_shade_tiles<W><<<grid, kThreads, sm, st>>>(ws, npix);
    return cudaGetLastError();
}

static cudaError_t nedf_dispatch(const Workspace &ws, int grid, int shadow_pass, cudaStream_t st)
{
    switch (ws.nedf_width) {
    case 64: return launch_nedf<64>(ws, grid, shadow_pass, st);
    case 128: return launch_nedf<128>(ws, grid, shadow_pass, st);
    case 256: return launch_nedf<256>(ws, grid, shadow_pass, st);
    default: return cudaErrorInvalidValue;
    }
}

static cudaError_t shade_dispatch(const Workspace &ws, int grid, int npix, cudaStream_t st)
{
    switch (ws.nerf_width) {
    case 0:
    case 64: return launch_shade<64>(ws, grid, npix, st);
    case 128: return launch_shade<128>(ws, grid, npix, st);
    case 256: return launch_shade<256>(ws, grid, npix, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_primary_binning(FrameLaunch &L)
{
    const Workspace &ws = L.ws;
    cudaStream_t st = L.stream;
    int npix = L.W * L.H;
    k_setup<<<1, 256, 0, st>>>(ws, L.cam);
    k_clear<<<L.num_sms * 4, 256, 0, st>>>(ws, npix);
    k_bin_primary<0><<<L.n_inst, kThreads, 0, st>>>(ws);
    k_scan_primary<<<1, 1024, 0, st>>>(ws, kTileRows);
    k_bin_primary<1><<<L.n_inst, kThreads, 0, st>>>(ws);
    return cudaGetLastError();
}

cudaError_t launch_frame(FrameLaunch &L)
{
    const Workspace &ws = L.ws;
    cudaStream_t st = L.stream;
    int npix = L.W * L.H;
    int gsm = L.num_sms;
    int stage = 0;
    // the tensor-core kernels take 256-row tiles (shading: two 128-row halves of n_shade-sample
    // pixels), the CUDA-core kernels 64-row tiles; the work-list scans must use the tile size of
    // the kernel that consumes the list
    const bool tc_nedf = ws.precision >= 1 && ws.depth_source == 0;      // BF16 or E4M3 tensor-core layers
    const bool tc_shade = ws.precision >= 1 && ws.nerf_hidden > 0;
    // the classifier network in FP32 on CUDA cores: the engines' tiles, decode and fallback
    const bool cls_f32 = ws.precision == 0 && ws.nedf_arch == 1 && ws.depth_source == 0;
    const bool listed_nedf = tc_nedf || cls_f32;                         // (m, a) per pair, then decode
    const int nedf_rows = listed_nedf ? kPipeTileRows : kTileRows;
    // the engine shades (128 / n_shade) pixels per 128-row half, two halves per tile
    const int shade_ppt = tc_shade ? 2 * (kTcTileRows / L.n_shade) : kTileRows / L.n_shade;
    // inside a captured graph the records are external (they still mark the stage boundaries for
    // timing when the graph runs); on an uncaptured stream they are plain records
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (L.events) cudaStreamIsCapturing(st, &cap);
    auto mark = [&]() {
        if (L.events) {
            if (cap == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(L.events[stage], st, cudaEventRecordExternal);
            else cudaEventRecord(L.events[stage], st);
        }
        ++stage;
    };
    mark();
    k_setup<<<1, 256, 0, st>>>(ws, L.cam);
    k_clear<<<gsm * 4, 256, 0, st>>>(ws, npix);
    mark();
    k_bin_primary<0><<<L.n_inst, kThreads, 0, st>>>(ws);
    k_scan_primary<<<1, 1024, 0, st>>>(ws, nedf_rows);
    k_bin_primary<1><<<L.n_inst, kThreads, 0, st>>>(ws);
    // the engine launch alone, inside its stage (the stage also holds the decode and fallback)
    auto mark_engine = [&](int k) {
        if (!L.events || !L.engine_events || !listed_nedf) return;
        if (cap == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(L.engine_events[k], st, cudaEventRecordExternal);
        else cudaEventRecord(L.engine_events[k], st);
        L.engines_timed = true;
    };
    mark();
    mark_engine(0);
    cudaError_t e = tc_nedf   ? launch_nedf_pipe(ws, 0, 0, nullptr, nullptr, nullptr, 0, gsm, st)
                    : cls_f32 ? launch_cls_f32(ws, 0, 0, nullptr, nullptr, nullptr, 0, gsm, st)
                              : nedf_dispatch(ws, gsm * 4, 0, st);
    mark_engine(1);
    if (e != cudaSuccess) return e;
    int launches = 6;
    if (listed_nedf) {                    // decode, then the pairs deferred to the plain method
        if ((e = launch_nedf_decode(ws, 0, gsm, st)) != cudaSuccess) return e;
        if ((e = launch_fallback(ws, 0, gsm, st)) != cudaSuccess) return e;
        launches += 2;
    }
    mark();
    k_resolve<<<gsm * 4, 256, 0, st>>>(ws, npix);
    k_scan_shade<<<1, 1, 0, st>>>(ws, shade_ppt);
    mark();
    e = tc_shade ? launch_shade_pipe(ws, npix, gsm, st) : shade_dispatch(ws, gsm * 4, npix, st);
    if (e != cudaSuccess) return e;
    if (L.shade_resample > 0 && ws.rs_mask) {       // Step-2 outliers: the plain method's colour
        if ((e = launch_shade_resample(L)) != cudaSuccess) return e;
        launches += ws.nerf_hidden > 0 ? 7 : 6;
    }
    mark();
    int nbin = 0;
    e = launch_shadow_binning(ws, npix, L.n_lights, L.n_inst, nedf_rows, gsm, st, &nbin, L.edit_mode == 2);
    if (e != cudaSuccess) return e;
    mark();
    mark_engine(2);
    e = tc_nedf   ? launch_nedf_pipe(ws, 1, 0, nullptr, nullptr, nullptr, 0, gsm, st)
        : cls_f32 ? launch_cls_f32(ws, 1, 0, nullptr, nullptr, nullptr, 0, gsm, st)
                  : nedf_dispatch(ws, gsm * 4, 1, st);
    mark_engine(3);
    if (e != cudaSuccess) return e;
    if (listed_nedf) {
        if ((e = launch_nedf_decode(ws, 1, gsm, st)) != cudaSuccess) return e;
        if ((e = launch_fallback(ws, 1, gsm, st)) != cudaSuccess) return e;
        launches += 2;
    }
    mark();
    k_composite<<<gsm * 8, 256, 0, st>>>(ws, npix);
    mark();
    L.launches = launches + 4 + nbin;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// NeDF queries on caller-given local rays (the network in isolation)
// ---------------------------------------------------------------------------------------------
template <int W_HID>
__global__ void __launch_bounds__(kThreads) k_nedf_query(Workspace ws, int type, const float *o,
                                                         const float *d, float *out, int n)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ float x6[kTileRows][6];
    __shared__ float tp[kTileRows];
    __shared__ int kept[kTileRows];
    __shared__ float y[kTileRows][4];
    const DevType T = ws.types[type];
    const float *w = ws.nedf_w + (size_t)type * ws.nedf_stride;
    for (long long tile = blockIdx.x; tile * kTileRows < n; tile += gridDim.x) {
        if (threadIdx.x < kTileRows) {
            long long idx = tile * kTileRows + threadIdx.x;
            for (int c = 0; c < 6; ++c) x6[threadIdx.x][c] = 0.0f;
            kept[threadIdx.x] = 0;
            if (idx < n) {
                V3 ol = v3(o[3 * idx], o[3 * idx + 1], o[3 * idx + 2]);
                V3 dl = normalized(v3(d[3 * idx], d[3 * idx + 1], d[3 * idx + 2]));
                Chord ch;
                kept[threadIdx.x] = bound_chord(ol, dl, T.rb, ch);
                V3 pe = madd(ol, ch.te, dl);
                if (kept[threadIdx.x]) {
                    x6[threadIdx.x][0] = pe.x; x6[threadIdx.x][1] = pe.y; x6[threadIdx.x][2] = pe.z;
                    x6[threadIdx.x][3] = dl.x; x6[threadIdx.x][4] = dl.y; x6[threadIdx.x][5] = dl.z;
                }
                tp[threadIdx.x] = ch.tp;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRows * kNedfIn; e += blockDim.x) {
            int r = e % kTileRows, fi = e / kTileRows;
            X[fi * kXStride + r] = posenc_feature(x6[r], 6, 6, fi);
        }
        __syncthreads();
        mlp_hidden_f32<W_HID>(X, kNedfIn, ws.nedf_hidden, w);
        const float *wo = w + (size_t)kNedfIn * W_HID + W_HID + (size_t)(ws.nedf_hidden - 1) * (W_HID * W_HID + W_HID);
        out_layer_f32(X, W_HID, wo, wo + W_HID * 2, 2, y);
        if (threadIdx.x < kTileRows) {
            long long idx = tile * kTileRows + threadIdx.x;
            if (idx < n) {
                float4 r = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
                if (kept[threadIdx.x]) {
                    float m = y[threadIdx.x][0], a = y[threadIdx.x][1];
                    float Dl = tp[threadIdx.x] - T.rb * m;
                    r = make_float4(m, a, Dl, (a > 0.f && Dl > 0.f) ? 1.f : 0.f);
                }
                reinterpret_cast<float4 *>(out)[idx] = r;
            }
        }
        __syncthreads();
    }
}

template <int W>
static cudaError_t launch_query(const Workspace &ws, int type, const float *o, const float *d, float *out,
                                int n, int grid, cudaStream_t st)
{
    size_t sm = nedf_smem<W>();
    cudaError_t e = cudaFuncSetAttribute(k_nedf_query<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_nedf_query<W><<<grid, kThreads, sm, st>>>(ws, type, o, d, out, n);
    return cudaGetLastError();
}

cudaError_t launch_nedf_query_f32(const Workspace &ws, int type, const float *o, const float *d, float *out,
                                  int n, int num_sms, cudaStream_t st)
{
    int grid = (int)std::min<long long>((long long)num_sms * 4, (n + kTileRows - 1) / kTileRows);
    if (grid < 1) return cudaSuccess;
    switch (ws.nedf_width) {
    case 64: return launch_query<64>(ws, type, o, d, out, n, grid, st);
    case 128: return launch_query<128>(ws, type, o, d, out, n, grid, st);
    case 256: return launch_query<256>(ws, type, o, d, out, n, grid, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nedf
