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
    unsigned long long p_total_requested;
    unsigned long long s_total_requested;
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
    uint32_t *hlist;             // [n_types][W*H] valid pixels per type
    Counters *cnt;
    uint32_t *status;
    // weights (FP32, per type, kernel layout: per layer Wt[in][out] then b[out])
    const float *nedf_w;
    long long nedf_stride;
    const float *nerf_w;
    long long nerf_stride;
    int nedf_hidden, nedf_width, nerf_hidden, nerf_width;
    // BF16 tensor-core weight blobs (per type, fixed stride); precision 1 selects them
    int precision;
    int depth_source;            // host copy of the frame option (selects kernels)
    const uint8_t *nedf_tc;
    size_t nedf_tc_stride;
    const uint8_t *nerf_tc;
    size_t nerf_tc_stride;
};

}  // namespace nedf
