// Step-3 binning: shadow rays grouped with the instances that can occlude them.
//
// Method: arXiv 2308.04669, Algorithm 2 (shadow rays from the point light L towards the surface
// point x, answered "like in STEP 1") and the shadow-mapping idea it builds on (Section "Fast
// Dynamic shadows Casting").  Every shadow ray of a light starts at L, so each light gets a
// pinhole "shadow-map camera" at L aimed at the scene bound: a G x G grid of direction cells.
// An instance's bound sphere, seen from L, covers exactly the directions inside its tangent
// cone; the cone's section with the image plane has the bounding rectangle given by the two
// tangent planes per axis, so the instance is listed in every cell of that rectangle (plus one
// cell of margin).  A shadow ray then looks up the single cell its direction falls in, and the
// exact bound-sphere test decides.  Instances whose rectangle is too large (close to the
// light) go to a per-light list every ray checks; a light inside the scene bound uses all
// instances.  The per-type pair lists are then built by a count pass, a scan and a fill pass
// over the same rays, each block placing its pairs in its own range.
#include "render_kernels.cuh"
#include "render_launch.h"

#include <algorithm>

namespace nedf {

constexpr int kMaxCellsPerInstance = 1024;
constexpr int kScanBlock = 4096;        // elements per block of the grid scan (1024 threads x 4)

// ---- scene bound of the instance spheres, one shadow-map camera per light --------------------------
__global__ void __launch_bounds__(256) k_light_setup(Workspace ws)
{
    __shared__ float red[6][256];
    const DevFrame &f = *ws.frame;
    float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
    for (int i = threadIdx.x; i < f.n_inst; i += blockDim.x) {
        DevInst I = ws.inst[i];
        float r = I.s * ws.types[I.type].rb;
        for (int c = 0; c < 3; ++c) {
            lo[c] = fminf(lo[c], I.T[c] - r);
            hi[c] = fmaxf(hi[c], I.T[c] + r);
        }
    }
    for (int c = 0; c < 3; ++c) {
        red[c][threadIdx.x] = lo[c];
        red[3 + c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int c = 0; c < 3; ++c) {
                red[c][threadIdx.x] = fminf(red[c][threadIdx.x], red[c][threadIdx.x + s]);
                red[3 + c][threadIdx.x] = fmaxf(red[3 + c][threadIdx.x], red[3 + c][threadIdx.x + s]);
            }
        __syncthreads();
    }
    if (threadIdx.x < kMaxLights) ws.lg_big_count[threadIdx.x] = 0;
    const int l = threadIdx.x;
    if (l >= f.n_lights) return;
    float blo[3] = {red[0][0], red[1][0], red[2][0]}, bhi[3] = {red[3][0], red[4][0], red[5][0]};
    V3 L = v3(f.lights[l][0], f.lights[l][1], f.lights[l][2]);
    LightCam cam{};
    V3 ctr = v3(0.5f * (blo[0] + bhi[0]), 0.5f * (blo[1] + bhi[1]), 0.5f * (blo[2] + bhi[2]));
    const V3 half = v3(0.5f * (bhi[0] - blo[0]), 0.5f * (bhi[1] - blo[1]), 0.5f * (bhi[2] - blo[2]));
    cam.ctr[0] = ctr.x; cam.ctr[1] = ctr.y; cam.ctr[2] = ctr.z;
    cam.rad = sqrtf(dot(half, half)) * 1.001f + 1e-3f;   // contains every instance's bound sphere
    if ((f.parallel_mask >> l) & 1u) {
        // a parallel light: an orthographic grid across its direction, over the bound sphere
        const V3 w = L;
        const V3 a0 = fabsf(w.y) < 0.9f ? v3(0.f, 1.f, 0.f) : v3(1.f, 0.f, 0.f);
        const V3 rt = normalized(v3(w.y * a0.z - w.z * a0.y, w.z * a0.x - w.x * a0.z, w.x * a0.y - w.y * a0.x));
        const V3 u2 = v3(rt.y * w.z - rt.z * w.y, rt.z * w.x - rt.x * w.z, rt.x * w.y - rt.y * w.x);
        cam.valid = f.n_inst > 0;
        cam.ortho = 1;
        cam.tan_h = 1.0f;
        cam.fwd[0] = w.x; cam.fwd[1] = w.y; cam.fwd[2] = w.z;
        cam.right[0] = rt.x; cam.right[1] = rt.y; cam.right[2] = rt.z;
        cam.up[0] = u2.x; cam.up[1] = u2.y; cam.up[2] = u2.z;
        ws.lcam[l] = cam;
        return;
    }
    bool inside = L.x >= blo[0] && L.x <= bhi[0] && L.y >= blo[1] && L.y <= bhi[1] && L.z >= blo[2] && L.z <= bhi[2];
    cam.valid = !inside && f.n_inst > 0;
    V3 fwd = normalized(sub(ctr, L));
    V3 up0 = fabsf(fwd.y) < 0.9f ? v3(0.f, 1.f, 0.f) : v3(1.f, 0.f, 0.f);
    V3 right = normalized(v3(fwd.y * up0.z - fwd.z * up0.y, fwd.z * up0.x - fwd.x * up0.z, fwd.x * up0.y - fwd.y * up0.x));
    V3 up = v3(right.y * fwd.z - right.z * fwd.y, right.z * fwd.x - right.x * fwd.z, right.x * fwd.y - right.y * fwd.x);
    float tmax = 0.0f;
    for (int k = 0; k < 8 && cam.valid; ++k) {
        V3 corner = v3((k & 1) ? bhi[0] : blo[0], (k & 2) ? bhi[1] : blo[1], (k & 4) ? bhi[2] : blo[2]);
        V3 e = sub(corner, L);
        float z = dot(e, fwd);
        if (z <= 1e-3f * sqrtf(dot(e, e))) { cam.valid = 0; break; }
        tmax = fmaxf(tmax, fmaxf(fabsf(dot(e, right)), fabsf(dot(e, up))) / z);
    }
    cam.tan_h = tmax * 1.05f + 1e-3f;
    if (cam.tan_h > 4.0f) cam.valid = 0;
    cam.eye[0] = L.x; cam.eye[1] = L.y; cam.eye[2] = L.z;
    cam.fwd[0] = fwd.x; cam.fwd[1] = fwd.y; cam.fwd[2] = fwd.z;
    cam.right[0] = right.x; cam.right[1] = right.y; cam.right[2] = right.z;
    cam.up[0] = up.x; cam.up[1] = up.y; cam.up[2] = up.z;
    ws.lcam[l] = cam;
}

__device__ __forceinline__ int cell_of(float u, float tan_h, int G)
{
    int c = (int)floorf((u / tan_h + 1.0f) * 0.5f * G);
    return min(max(c, 0), G - 1);
}

// Cell rectangle of a sphere (centre c, radius r) in a light's grid; false when the sphere
// reaches the light's image plane (then it goes to the per-light list).
__device__ __forceinline__ bool light_rect(const LightCam &cam, int G, V3 c, float r, int &i0, int &i1, int &j0,
                                           int &j1)
{
    if (cam.ortho) {                 // a parallel light: the sphere's orthographic shadow is a disc
        const V3 p = sub(c, v3(cam.ctr[0], cam.ctr[1], cam.ctr[2]));
        const float cu = dot(p, v3(cam.right[0], cam.right[1], cam.right[2])) / cam.rad;
        const float cv = dot(p, v3(cam.up[0], cam.up[1], cam.up[2])) / cam.rad, rr = r / cam.rad;
        i0 = max(cell_of(cu - rr, 1.0f, G) - 1, 0);
        i1 = min(cell_of(cu + rr, 1.0f, G) + 1, G - 1);
        j0 = max(cell_of(cv - rr, 1.0f, G) - 1, 0);
        j1 = min(cell_of(cv + rr, 1.0f, G) + 1, G - 1);
        return true;
    }
    V3 e = sub(c, v3(cam.eye[0], cam.eye[1], cam.eye[2]));
    float cx = dot(e, v3(cam.right[0], cam.right[1], cam.right[2]));
    float cy = dot(e, v3(cam.up[0], cam.up[1], cam.up[2]));
    float cz = dot(e, v3(cam.fwd[0], cam.fwd[1], cam.fwd[2]));
    if (cz <= r * 1.001f + 1e-6f) return false;
    // tangent planes through L: (c_a - u c_z)^2 = r^2 (1 + u^2)
    float den = cz * cz - r * r;
    float sx = r * sqrtf(fmaxf(cx * cx + cz * cz - r * r, 0.f));
    float sy = r * sqrtf(fmaxf(cy * cy + cz * cz - r * r, 0.f));
    i0 = max(cell_of((cx * cz - sx) / den, cam.tan_h, G) - 1, 0);
    i1 = min(cell_of((cx * cz + sx) / den, cam.tan_h, G) + 1, G - 1);
    j0 = max(cell_of((cy * cz - sy) / den, cam.tan_h, G) - 1, 0);
    j1 = min(cell_of((cy * cz + sy) / den, cam.tan_h, G) + 1, G - 1);
    return true;
}

__global__ void k_zero_u32(uint32_t *p, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// One warp per (light, instance): the lanes share the instance's cell rectangle, one cell each,
// so an instance covering tens of cells costs one round of atomics instead of a serial loop.
template <int PASS>
__global__ void __launch_bounds__(256) k_light_bin(Workspace ws, int n_lights)
{
    const DevFrame &f = *ws.frame;
    const int G = ws.lg_G, n_inst = f.n_inst, lane = threadIdx.x & 31;
    const long long total = (long long)n_lights * n_inst;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long e = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < total; e += warps) {
        const int l = (int)(e / n_inst), i = (int)(e - (long long)l * n_inst);
        const LightCam cam = ws.lcam[l];
        if (!cam.valid) continue;
        if (f.edit_mode == 1 && i == f.edit_inst) continue;     // the frozen part has no manipulated instance
        const DevInst I = ws.inst[i];
        const float r = I.s * ws.types[I.type].rb;
        int i0, i1, j0, j1;
        const bool ok = light_rect(cam, G, v3(I.T[0], I.T[1], I.T[2]), r, i0, i1, j0, j1);
        if (!ok || (i1 - i0 + 1) * (j1 - j0 + 1) > kMaxCellsPerInstance) {
            if (PASS == 1 && lane == 0) {
                const uint32_t pos = atomicAdd(&ws.lg_big_count[l], 1u);
                ws.lg_big[(size_t)l * ws.max_inst + pos] = (uint32_t)i;
            }
            continue;
        }
        const int wdt = i1 - i0 + 1, n_cells = wdt * (j1 - j0 + 1);
        for (int c = lane; c < n_cells; c += 32) {
            const int jr = c / wdt;
            const size_t cell = ((size_t)l * G + (j0 + jr)) * G + (i0 + c - jr * wdt);
            if (PASS == 0) {
                atomicAdd(&ws.lg_count[cell], 1u);
            } else {
                const uint32_t pos = atomicAdd(&ws.lg_cursor[cell], 1u);
                if ((long long)pos < ws.lg_cap) ws.lg_items[pos] = (uint32_t)i;
                else atomicOr(ws.status, kStatusShadowOverflow);
            }
        }
    }
}

// ---- exclusive scan of the grid counts (3 kernels) ----------------------------------------------
__global__ void __launch_bounds__(1024) k_scan_blocks(const uint32_t *in, uint32_t *out, uint32_t *block_sums, long long n)
{
    __shared__ uint32_t wsum[32];
    const long long base = (long long)blockIdx.x * kScanBlock + threadIdx.x * 4;
    uint32_t v[4], t = 0;
    for (int k = 0; k < 4; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        t += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = t;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - t;
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = run;
}

__global__ void __launch_bounds__(1024) k_scan_sums(uint32_t *block_sums, int nb, uint32_t *total_out)
{
    __shared__ uint32_t wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t t = threadIdx.x < nb ? block_sums[threadIdx.x] : 0u, incl = t;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = wsum[lane], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t excl = wsum[warp] + incl - t;
    if (threadIdx.x < nb) block_sums[threadIdx.x] = excl;
    if (threadIdx.x == nb - 1) *total_out = excl + t;
}

__global__ void k_scan_add(uint32_t *out, uint32_t *cursor, const uint32_t *block_sums, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        uint32_t v = out[i] + block_sums[i / kScanBlock];
        out[i] = v;
        cursor[i] = v;
    }
}

// ---- shadow rays against the instances listed in their cell --------------------------------------
__device__ __forceinline__ unsigned lane_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// The shadow rays of the hit pixels (the per-type hit lists of the resolve, one after another),
// lane-coherent: the 32 lanes of a warp take 32 consecutive hit pixels (neighbours on screen)
// for one light, so that they mostly fall in the same light-grid cell, read the same candidate
// instances (broadcast loads) and run the same number of candidate tests.  Flat index rr ->
// q = rr / 32, light l = q % n_lights, hit h = (q / n_lights) * 32 + rr % 32.
//
// PASS 0 counts each block's kept pairs per type (shared-memory atomics) into sblk; after the
// scan, PASS 1 runs the same rays in the same blocks and places each block's pairs in its own
// range of each type's list with shared-memory cursors, so no global counter is contended.
template <int PASS>
__global__ void __launch_bounds__(256, 6) k_bin_shadow_grid(Workspace ws, int npix)
{
    __shared__ unsigned long long hit_pre[kMaxTypes + 1];   // first flat hit index of each type's list
    __shared__ unsigned long long s_cur[kMaxTypes];         // PASS 0: count; PASS 1: cursor
    __shared__ unsigned long long s_beg[kMaxTypes], s_end[kMaxTypes], s_lim[kMaxTypes];
    const DevFrame &f = *ws.frame;
    const int nl = f.n_lights, n_inst = f.n_inst, G = ws.lg_G, n_types = f.n_types;
    const int lane = threadIdx.x & 31, nb = ws.sblk_nb;
    if (threadIdx.x < n_types) {
        const int t = threadIdx.x;
        if (PASS == 0) {
            s_cur[t] = 0;
        } else {
            s_beg[t] = s_cur[t] = ws.sblk[(size_t)t * (nb + 1) + blockIdx.x];
            s_end[t] = ws.sblk[(size_t)t * (nb + 1) + blockIdx.x + 1];
            s_lim[t] = ws.cnt->s_off[t + 1];
        }
    }
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int t = 0; t < n_types; ++t) {
            hit_pre[t] = acc;
            acc += ws.cnt->h_count[t];
        }
        hit_pre[n_types] = acc;
    }
    __syncthreads();
    const unsigned long long n_hit = hit_pre[n_types];
    const long long n_rays = (long long)((n_hit + 31) / 32) * 32 * nl;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n_rays; base += (long long)gridDim.x * blockDim.x) {
        const long long rr = base + threadIdx.x;
        const long long q = rr >> 5;
        const uint32_t l = (uint32_t)(q % nl);
        const unsigned long long h = (unsigned long long)(q / nl) * 32 + (unsigned long long)(rr & 31);
        const bool valid = h < n_hit;
        uint32_t pix = 0;
        V3 o = v3(0, 0, 0), d = v3(0, 0, 1);
        float ell = 0.0f;
        int count = 0, nc = 0;
        uint32_t c0 = 0;
        bool grid = false;
        if (valid) {
            int t = 0;
            while (t + 1 < n_types && hit_pre[t + 1] <= h) ++t;
            pix = ws.hlist[(size_t)t * npix + (h - hit_pre[t])];
            V3 oc, dc;
            camera_ray(f, pix % f.W, pix / f.W, oc, dc);
            V3 x = madd(oc, ws.depth[pix], dc);
            light_ray(ws.lcam, f, (int)l, x, o, d, ell);
            const LightCam &cam = ws.lcam[l];
            grid = cam.valid;
            if (grid) {
                float u, w;
                if (cam.ortho) {                 // a parallel light: where the ray crosses the grid
                    const V3 p = sub(o, v3(cam.ctr[0], cam.ctr[1], cam.ctr[2]));
                    u = dot(p, v3(cam.right[0], cam.right[1], cam.right[2])) / cam.rad;
                    w = dot(p, v3(cam.up[0], cam.up[1], cam.up[2])) / cam.rad;
                } else {
                    const float z = dot(d, v3(cam.fwd[0], cam.fwd[1], cam.fwd[2]));
                    u = dot(d, v3(cam.right[0], cam.right[1], cam.right[2])) / z;
                    w = dot(d, v3(cam.up[0], cam.up[1], cam.up[2])) / z;
                }
                size_t cell = ((size_t)l * G + cell_of(w, cam.tan_h, G)) * G + cell_of(u, cam.tan_h, G);
                c0 = ws.lg_off[cell];
                long long end = min((long long)ws.lg_off[cell + 1], ws.lg_cap);   // overflow: flagged in the fill
                nc = (int)max(0ll, end - (long long)c0);
                count = nc + (int)ws.lg_big_count[l];
            } else {
                count = n_inst;
            }
        }
        // the fill pass walks only the candidates the count pass kept (their bits in the ray's
        // mask, lowest first), re-testing each exactly as the count pass did; rays of more than 32
        // candidates (or frames beyond the mask buffer) walk all of them again
        const bool masked = PASS == 1 && count <= 32 && n_rays <= ws.smask_cap;
        uint32_t kmask = masked && valid ? ws.smask[rr] : 0u;
        const int items = masked ? __popc(kmask) : count;
        const int maxc = __reduce_max_sync(0xffffffffu, items);
        uint32_t kept_bits = 0u;
        for (int j = 0; j < maxc; ++j) {
            bool keep = false;
            uint32_t inst = 0, ty = 0;
            V3 ol = v3(0, 0, 0), dl = v3(0, 0, 0);
            Chord ch{};
            int k = j;
            if (masked && j < items) {
                k = __ffs(kmask) - 1;
                kmask &= kmask - 1u;
            }
            if (j < items) {
                inst = grid ? (k < nc ? ws.lg_items[c0 + k] : ws.lg_big[(size_t)l * ws.max_inst + (k - nc)]) : (uint32_t)k;
                DevInst I = ws.inst[inst];
                ty = I.type;
                to_local(I, o, d, ol, dl);
                keep = bound_chord(ol, dl, ws.types[ty].rb, ch) && (ch.te * I.s < ell) &&
                       !(f.edit_mode == 1 && inst == (uint32_t)f.edit_inst);
            }
            if (PASS == 0 && keep && k < 32) kept_bits |= 1u << k;
            const unsigned active = __ballot_sync(0xffffffffu, keep);
            if (!keep) continue;
            const unsigned peers = __match_any_sync(active, ty);
            const int leader = __ffs(peers) - 1;
            if (PASS == 0) {
                if (lane == leader) atomicAdd(&s_cur[ty], (unsigned long long)__popc(peers));
                continue;
            }
            unsigned long long start = 0;
            if (lane == leader) start = atomicAdd(&s_cur[ty], (unsigned long long)__popc(peers));
            start = __shfl_sync(peers, start, leader);
            const unsigned long long idx = start + __popc(peers & lane_lt());
            if (idx < s_end[ty] && idx < s_lim[ty]) {
                ws.spairs[idx] = make_uint2(pix * nl + l, inst);
                if (ws.pair_geo) {
                    ws.sgeo[2 * idx] = make_float4(ol.x, ol.y, ol.z, ch.te);
                    ws.sgeo[2 * idx + 1] = make_float4(dl.x, dl.y, dl.z, ch.tp);
                    ws.sell[idx] = ell;
                }
            } else {
                atomicOr(ws.status, kStatusShadowOverflow);    // the list's capacity (or a count/fill mismatch)
            }
        }
        if (PASS == 0 && valid && count <= 32 && n_rays <= ws.smask_cap) ws.smask[rr] = kept_bits;
    }
    __syncthreads();
    if (threadIdx.x < n_types) {
        const int t = threadIdx.x;
        if (PASS == 0) {
            ws.sblk[(size_t)t * (nb + 1) + blockIdx.x] = s_cur[t];
        } else {
            const unsigned long long filled = min(s_cur[t], min(s_end[t], s_lim[t]));
            if (filled > s_beg[t]) atomicAdd(&ws.cnt->s_cursor[t], filled - s_beg[t]);
        }
    }
}

// Buffer reuse, edit frame: the shadow rays of the pixels the frozen part wins (their surface
// points and their occlusion by the frozen instances are unchanged) tested against the
// manipulated instance alone; the pairs join the same per-type lists (count pass, then fill).
template <int PASS>
__global__ void __launch_bounds__(256) k_edit_shadow(Workspace ws, int npix)
{
    const DevFrame &f = *ws.frame;
    const int nl = f.n_lights, lane = threadIdx.x & 31;
    const uint32_t e = (uint32_t)f.edit_inst;
    const DevInst I = ws.inst[e];
    const uint32_t ty = I.type;
    const float rb = ws.types[ty].rb;
    const long long n_rays = (long long)npix * nl;
    // the trip count is uniform within a block, so the ballots below see whole warps
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n_rays; base += (long long)gridDim.x * blockDim.x) {
        const long long rr = base + threadIdx.x;
        bool keep = false;
        uint32_t pix = 0, l = 0;
        V3 ol = v3(0, 0, 0), dl = v3(0, 0, 0);
        Chord ch{};
        float ell = 0.0f;
        if (rr < n_rays) {
            pix = (uint32_t)(rr / nl);
            l = (uint32_t)(rr - (long long)pix * nl);
            const uint32_t id = ws.id[pix];
            if (id != kNoId && id != e) {
                V3 oc, dc;
                camera_ray(f, pix % f.W, pix / f.W, oc, dc);
                const V3 x = madd(oc, ws.depth[pix], dc);
                V3 o, d;
                light_ray(ws.lcam, f, (int)l, x, o, d, ell);
                to_local(I, o, d, ol, dl);
                keep = bound_chord(ol, dl, rb, ch) && (ch.te * I.s < ell);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        unsigned long long start = 0;
        if (PASS == 0) {
            if (lane == __ffs(m) - 1) atomicAdd(&ws.cnt->s_count[ty], (unsigned long long)__popc(m));
            continue;
        }
        if (lane == __ffs(m) - 1) start = atomicAdd(&ws.cnt->s_cursor[ty], (unsigned long long)__popc(m));
        start = __shfl_sync(0xffffffffu, start, __ffs(m) - 1);
        if (keep) {
            const unsigned long long idx = start + __popc(m & lane_lt());
            if (idx < ws.cnt->s_off[ty + 1]) {
                ws.spairs[idx] = make_uint2(pix * nl + l, e);
                if (ws.pair_geo) {
                    ws.sgeo[2 * idx] = make_float4(ol.x, ol.y, ol.z, ch.te);
                    ws.sgeo[2 * idx + 1] = make_float4(dl.x, dl.y, dl.z, ch.tp);
                    ws.sell[idx] = ell;
                }
            } else {
                atomicOr(ws.status, kStatusShadowOverflow);
            }
        }
    }
}

// The per-type shadow lists: type t holds its grid pairs (block after block) and then its edit
// frame's pairs.  One warp per type sums the blocks' counts; thread 0 lays out the segments (the
// capacity clamps the last ones) and their tiles; one warp per type then scans the blocks' counts
// into their first indices.  s_cursor[t] starts at the segment: the fill pass adds each block's
// pairs to it, the edit frame's appends continue from there, so a segment filled exactly ends at
// the next segment.
__global__ void __launch_bounds__(1024) k_scan_shadow_pairs(Workspace ws, int rows_per_tile)
{
    __shared__ unsigned long long s_grid[kMaxTypes];
    const DevFrame &f = *ws.frame;
    Counters &C = *ws.cnt;
    const int nb = ws.sblk_nb, T = f.n_types;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int t = warp; t < T; t += nw) {
        unsigned long long s = 0;
        for (int b = lane; b < nb; b += 32) s += ws.sblk[(size_t)t * (nb + 1) + b];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) s_grid[t] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long o = 0, tl = 0, req = 0;
        for (int k = 0; k < T; ++k) {
            unsigned long long c = s_grid[k] + C.s_count[k];       // grid pairs + edit-frame pairs
            req += c;
            if (o + c > (unsigned long long)ws.scap) {
                c = (unsigned long long)ws.scap - o;
                *ws.status |= kStatusShadowOverflow;
            }
            C.s_count[k] = c;
            C.s_off[k] = o;
            C.s_cursor[k] = o;
            C.s_tile[k] = tl;
            o += c;
            tl += (c + rows_per_tile - 1) / rows_per_tile;
        }
        C.s_off[T] = o;
        C.s_tile[T] = tl;
        C.s_total_requested = req;
    }
    __syncthreads();
    for (int t = warp; t < T; t += nw) {
        unsigned long long run = C.s_off[t];
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            const unsigned long long v = b < nb ? ws.sblk[(size_t)t * (nb + 1) + b] : 0ull;
            unsigned long long incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (b < nb) ws.sblk[(size_t)t * (nb + 1) + b] = run + incl - v;
            run += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) ws.sblk[(size_t)t * (nb + 1) + nb] = run;      // the end of the grid pairs
    }
}

cudaError_t launch_shadow_binning(const Workspace &ws, int npix, int n_lights, int n_inst, int rows_per_tile,
                                  int num_sms, cudaStream_t st, int *launches, bool edit_frame)
{
    const int G = ws.lg_G;
    const long long cells = (long long)n_lights * G * G;
    const int nb = (int)((cells + kScanBlock - 1) / kScanBlock);
    if (nb > 1024) return cudaErrorInvalidValue;
    const long long pairs = (long long)n_lights * n_inst;
    const int gb = (int)std::min<long long>((pairs + 7) / 8, (long long)num_sms * 8);     // a warp per pair
    k_light_setup<<<1, 256, 0, st>>>(ws);
    k_zero_u32<<<num_sms * 2, 256, 0, st>>>(ws.lg_count, cells);
    k_light_bin<0><<<gb, 256, 0, st>>>(ws, n_lights);
    k_scan_blocks<<<nb, 1024, 0, st>>>(ws.lg_count, ws.lg_off, ws.scan_tmp, cells);
    k_scan_sums<<<1, 1024, 0, st>>>(ws.scan_tmp, nb, ws.lg_off + cells);
    k_scan_add<<<num_sms * 2, 256, 0, st>>>(ws.lg_off, ws.lg_cursor, ws.scan_tmp, cells);
    k_light_bin<1><<<gb, 256, 0, st>>>(ws, n_lights);
    k_bin_shadow_grid<0><<<ws.sblk_nb, 256, 0, st>>>(ws, npix);
    if (edit_frame) k_edit_shadow<0><<<num_sms * 8, 256, 0, st>>>(ws, npix);
    k_scan_shadow_pairs<<<1, 1024, 0, st>>>(ws, rows_per_tile);
    k_bin_shadow_grid<1><<<ws.sblk_nb, 256, 0, st>>>(ws, npix);
    if (edit_frame) k_edit_shadow<1><<<num_sms * 8, 256, 0, st>>>(ws, npix);
    *launches = edit_frame ? 12 : 10;
    return cudaGetLastError();
}

}  // namespace nedf
