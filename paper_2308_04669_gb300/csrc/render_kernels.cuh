// Render-path kernels: work lists, NeDF queries, z-min, deferred shading, shadows, composite.
//
// Method: arXiv 2308.04669, Algorithm 1 (Steps 1-2) and Algorithm 2 (Step 3).
//
// Work is organised as lists of (ray, instance) pairs grouped by object type, so that every
// tile of rows handed to an MLP shares one set of weights.  Each list is built in two passes
// (count, then fill) over identical cull arithmetic, so sizes are exact and deterministic
// while the order inside a type is not; nothing downstream depends on that order (the z-min
// is an atomic minimum of a packed (depth, id) key; occlusion is an atomic OR).
#pragma once

#include "nedf_device.cuh"
#include "mlp_f32.cuh"

namespace nedf {

constexpr int kTcTileRows = 128;     // rows per tensor-core MLP tile (M of the MMA)

struct LightCam;

struct Counters {
    unsigned long long p_count[kMaxTypes];
    unsigned long long p_cursor[kMaxTypes];
    unsigned long long p_off[kMaxTypes + 1];     // pair offsets of each type's segment
    unsigned long long p_tile[kMaxTypes + 1];    // first tile of each type
    unsigned long long s_count[kMaxTypes];
    unsigned long long s_cursor[kMaxTypes];
    unsigned long long s_off[kMaxTypes + 1];
    unsigned long long s_tile[kMaxTypes + 1];
    unsigned long long h_count[kMaxTypes];       // valid pixels per type (shading lists)
    unsigned long long h_tile[kMaxTypes + 1];
    unsigned long long fallback;
    unsigned long long hit_pixels;
    unsigned long long rs_pixels;                // Step-2 outliers re-rendered by the plain method
    unsigned long long p_total_requested;
    unsigned long long s_total_requested;
    unsigned long long fb_count[2];              // deferred plain-method pairs (primary, shadow)
    unsigned long long lg_total;                 // shadow light-grid entries requested
};

struct Workspace {
    DevFrame *frame;
    const DevType *types;
    const DevInst *inst;
    unsigned long long *keys;    // [W*H] packed (depth bits << 32 | id)
    float *depth;                // [W*H]
    uint32_t *id;                // [W*H]
    float4 *rgba;                // [W*H]
    float *shadow;               // [W*H]
    float4 *out;                 // [W*H]
    uint32_t *occl;              // [W*H] bit l set = light l occluded
    uint2 *ppairs;               // primary (pixel, instance)
    long long pcap;
    uint2 *spairs;               // shadow (pixel * n_lights + light, instance)
    long long scap;
    // pair geometry from the binning passes, for the NeDF engines that read it (pair_geo): per
    // pair (local origin, t_entry) and (local direction, t_perp); per shadow pair the world length
    // from the light to the lit point
    float4 *pgeo;                // [2 * pcap]
    float4 *sgeo;                // [2 * scap]
    float *sell;                 // [scap]
    float2 *nout[2];             // the engine's NeDF outputs (m, a) per listed pair: primary, shadow
    // Step-2 outlier resampling: per-pixel outlier flags, and the outliers' primary pairs as a list
    // of their own with its own counters (the plain method's colour kernels then run on it as on
    // the whole frame's pairs), plus their scratch
    uint32_t *rs_mask;           // [W*H], or null while resampling was never enabled
    uint2 *rs_pairs;             // [rs_cap]
    Counters *rs_cnt;
    void *rs_scratch;
    long long rs_cap;
    // buffer reuse: the frozen part's packed depth/id keys, colours and occlusion bits [W*H]
    const unsigned long long *edit_keys;
    const float4 *edit_rgba;
    const uint32_t *edit_occl;
    uint32_t *hlist;             // [n_types][W*H] valid pixels per type
    Counters *cnt;
    uint32_t *status;
    // weights (FP32, per type, kernel layout: per layer Wt[in][out] then b[out])
    const float *nedf_w;
    long long nedf_stride;
    const float *nerf_w;
    long long nerf_stride;
    int nedf_hidden, nedf_width, nerf_hidden, nerf_width;
    int nedf_arch;               // 0: regression MLP, 1: the paper's classifier network (nedf_tc only)
    int pair_geo;                // the binning passes store each pair's local ray (pgeo / sgeo)
    // BF16 tensor-core weight blobs (per type, fixed stride); precision 1 selects them
    int precision;
    int depth_source;            // host copy of the frame option (selects kernels)
    const uint8_t *nedf_tc;
    size_t nedf_tc_stride;
    const uint8_t *nerf_tc;
    size_t nerf_tc_stride;
    size_t nerf_pair_off;        // width 256: offset of the SM-pair layout inside each type's blob (0: none)
    // pairs deferred to the plain method by the tensor-core NeDF kernels (indices into the lists)
    uint32_t *fb_list[2];
    // shadow-map cameras: per light a G x G grid of direction cells with instance lists
    struct LightCam *lcam;       // [kMaxLights]
    uint32_t *lg_count;          // [n_lights * G * G]
    uint32_t *lg_off;            // [n_lights * G * G + 1] (exclusive scan), reused as cursors
    uint32_t *lg_cursor;         // [n_lights * G * G]
    uint32_t *lg_items;          // instance ids, cell after cell
    long long lg_cap;
    uint32_t *lg_big;            // [n_lights][max_instances] instances too large for cell lists
    uint32_t *lg_big_count;      // [kMaxLights]
    int lg_G;
    int max_inst;
    uint32_t *scan_tmp;          // block sums of the grid scan
    // shadow-ray binning: per type t and block b of the binning grid, the block's pair count (count
    // pass), then the first index of its range ([t][nb] = the end of the type's grid pairs)
    unsigned long long *sblk;    // [kMaxTypes][sblk_nb + 1]
    // shadow-ray binning: per shadow ray (of at most 32 candidates) the candidates the count pass
    // kept, bit k = candidate k, so the fill pass tests only those
    uint32_t *smask;
    long long smask_cap;
    // primary binning: per instance its pair count (count pass) and the first index of its range
    unsigned long long *pinst;   // [max_instances][2]
    int sblk_nb;                 // blocks of the shadow-ray binning grid
    // tensor-core schedule: weight bytes per bulk copy of each engine mode (shade, march colour,
    // primary NeDF, shadow NeDF, NeDF query); picked by the autotuner or set by the caller
    int pipe_stage_bytes[5];
    // operand order of the NeDF engines at BF16 width 128 (same kernel index): 0 default, 1 swapped
    // (weights as A, D^T = W H^T), 2 unswapped (activations as A); results do not depend on it.
    // NeRF kernels (0, 1) at width 256: 1 the SM-pair engine, 0 (default) and 2 the one-SM engine
    int pipe_order[5];
};

struct LightCam {
    float eye[3], right[3], up[3], fwd[3];
    float tan_h;
    int valid;                   // 0: light inside the scene bound or too wide a view -> all instances
    int ortho;                   // a parallel light: an orthographic grid across its direction
    float ctr[3], rad;           // the scene's bound sphere (parallel lights' rays start on it)
};

// The shadow ray of light l towards the surface point x (Algorithm 2): o = the light, d = the unit
// direction from o to x, ell = |x - o|.  A parallel light (unit travel direction w) reaches x from
// infinity; its ray starts where the line x - t w leaves the scene's bound sphere (just outside,
// so outside every object's bound): the same entry points, directions and order along the ray as
// from infinity.
__device__ __forceinline__ void light_ray(const LightCam *lcam, const DevFrame &f, int l, V3 x, V3 &o, V3 &d, float &ell)
{
    if ((f.parallel_mask >> l) & 1u) {
        const LightCam &cam = lcam[l];
        d = v3(f.lights[l][0], f.lights[l][1], f.lights[l][2]);
        const V3 p = sub(x, v3(cam.ctr[0], cam.ctr[1], cam.ctr[2]));
        const float b = dot(p, d);                       // |p - t d| = rad at t = b + sqrt(...)
        const float disc = fmaxf(b * b - dot(p, p) + cam.rad * cam.rad, 0.0f);
        ell = fmaxf(b + sqrtf(disc), 0.0f) + 1e-3f * cam.rad + 1e-3f;
        o = madd(x, -ell, d);
    } else {
        o = v3(f.lights[l][0], f.lights[l][1], f.lights[l][2]);
        const V3 v = sub(x, o);
        ell = sqrtf(dot(v, v));
        d = normalized(v);
    }
}

// Plain-method colour frame buffers (march.cu): per pair, its samples' transmittance and the
// weighted colour accumulated by the colour-network tiles over its run of sample rows.
struct MarchBuffers {
    int *head;            // [npix] first pair of the pixel's list (-1 = none)
    int *next;            // [pairs] next pair of the same pixel
    float *te_world;      // [pairs]
    float *T_pair;        // [pairs] transmittance through the pair's samples
    float *T_first;       // [pairs] transmittance before the pair's first sample row
    int *k_first;         // [pairs]
    float4 *C;            // [pairs] accumulated weighted colour (xyz)
    uint2 *rows;          // [pairs * n] (pair, k)
    unsigned long long *row_cursor;   // [kMaxTypes]
    unsigned long long *row_off;      // [kMaxTypes + 1]
    unsigned long long *row_tile;     // [kMaxTypes + 1]
    long long row_cap;
};

// ---------------------------------------------------------------------------------------------
// (ray, instance) pair set-up shared by the NeDF kernels and the deferred plain-method pass
// ---------------------------------------------------------------------------------------------
struct PairRay {
    V3 ol, dl;
    float te, tx, tp, s, ell;
    uint32_t key, inst;
    bool kept;
};

// Step-2 outlier test ("rs", Section "Deferred Shading"): an extremely small density at every
// sample around the predicted depth says the depth missed the surface; the pixel is flagged for
// the plain method's volume rendering.  Called by the lanes that composite a pixel (any subset of
// the warp); the count is warp-aggregated.
__device__ __forceinline__ void flag_shade_outlier(const Workspace &ws, const DevFrame &f, uint32_t pix, float smax)
{
    const bool rs = f.shade_resample > 0 && smax < f.shade_sigma_min;
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, rs);
    if (!m) return;
    if (rs) ws.rs_mask[pix] = 1u;
    if ((threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&ws.cnt->rs_pixels, (unsigned long long)__popc(m));
}

__device__ __forceinline__ void setup_pair_ray(const Workspace &ws, const DevFrame &f, bool shadow, uint2 pr,
                                               float rb, PairRay &R)
{
    R.key = pr.x;
    R.inst = pr.y;
    DevInst I = ws.inst[pr.y];
    R.s = I.s;
    R.ell = 0.0f;
    V3 o, d;
    if (!shadow) {
        camera_ray(f, pr.x % f.W, pr.x / f.W, o, d);
    } else {
        uint32_t pix = pr.x / f.n_lights, l = pr.x - pix * f.n_lights;
        V3 oc, dc;
        camera_ray(f, pix % f.W, pix / f.W, oc, dc);
        V3 x = madd(oc, ws.depth[pix], dc);
        light_ray(ws.lcam, f, (int)l, x, o, d, R.ell);
    }
    to_local(I, o, d, R.ol, R.dl);
    Chord ch;
    R.kept = bound_chord(R.ol, R.dl, rb, ch);
    R.te = ch.te;
    R.tx = ch.tx;
    R.tp = ch.tp;
}

// Step 1: packed atomic minimum (strict '<' in id order on ties).  Step 3: occlusion bit when
// the hit lies closer to the light than the surface point by more than eps (Algorithm 2).
__device__ __forceinline__ void apply_hit(const Workspace &ws, const DevFrame &f, bool shadow, const PairRay &R,
                                          float Dl)
{
    float D = R.s * Dl;
    if (!shadow) {
        atomicMin(&ws.keys[R.key], ((unsigned long long)__float_as_uint(D) << 32) | R.inst);
    } else if (D + f.eps < R.ell) {
        uint32_t pix = R.key / f.n_lights, l = R.key - pix * f.n_lights;
        atomicOr(&ws.occl[pix], 1u << l);
    }
}

}  // namespace nedf
