// C-ABI entry points of libnedf_compose (declared in include/nedf_compose.h).
//
// Host side of the renderer: argument checks, ownership of device workspace, weight layout
// conversion, and the launch sequence of each call.  All arithmetic of the method runs in the
// kernels; this file only moves and validates data.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/nedf_compose.h"
#include "render_launch.h"
#include "train_launch.h"

using namespace nedf;

struct TrainState {
    float *o = nullptr, *d = nullptr, *m_star = nullptr, *hit_star = nullptr;  // training set
    long long n_rays = 0;
    long long cursor = 0;
    float *master = nullptr;   // packed FP32 weights (W[out][in], b)
    float *adam_m = nullptr, *adam_v = nullptr;
    int step = 0;
};

struct nedf_handle {
    nedf_config cfg{};
    nedf_options opt{};
    // buffer reuse (an edit session): frozen buffers, the session's camera, lights and instances
    std::vector<DevInst> h_inst;                 // host copy of the current instances
    bool edit_active = false;
    int edit_inst = -1, edit_mode = 0, last_mode = 0;
    std::vector<DevInst> edit_inst_snapshot;
    nedf_camera edit_cam{};
    std::vector<nedf_light> edit_lights;
    unsigned long long version = 0, edit_version = 0;   // bumped by anything that changes a frame's result
    unsigned long long *d_edit_keys = nullptr;
    float4 *d_edit_rgba = nullptr;
    uint32_t *d_edit_occl = nullptr;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    std::string err;
    int n_types = 0, n_inst = 0;
    long long nedf_params = 0, nerf_params = 0;
    // device memory
    DevFrame *d_frame = nullptr;
    HostCamera *d_cam = nullptr;
    DevFrame *h_frame = nullptr;     // pinned staging
    HostCamera *h_cam = nullptr;     // pinned staging
    DevType *d_types = nullptr;
    DevInst *d_inst = nullptr;
    float *d_nedf_w = nullptr, *d_nerf_w = nullptr;
    unsigned long long *d_keys = nullptr;
    float *d_depth = nullptr, *d_shadow = nullptr;
    uint32_t *d_id = nullptr, *d_occl = nullptr, *d_hlist = nullptr, *d_status = nullptr;
    float4 *d_rgba = nullptr, *d_out = nullptr;
    uint2 *d_ppairs = nullptr, *d_spairs = nullptr;
    float4 *d_pgeo = nullptr, *d_sgeo = nullptr;
    float *d_sell = nullptr;
    float2 *d_nout[2] = {nullptr, nullptr};
    Counters *d_cnt = nullptr;
    float *d_train_scratch = nullptr;
    size_t train_scratch_bytes = 0;
    float *d_loss = nullptr;
    std::vector<TrainState> train;
    std::vector<DevType> types_host;
    uint8_t *d_nedf_tc = nullptr, *d_nerf_tc = nullptr;   // BF16 blobs
    uint32_t *d_fb[2] = {nullptr, nullptr};
    LightCam *d_lcam = nullptr;
    uint32_t *d_lg_count = nullptr, *d_lg_off = nullptr, *d_lg_cursor = nullptr, *d_lg_items = nullptr;
    uint32_t *d_lg_big = nullptr, *d_lg_big_count = nullptr, *d_scan_tmp = nullptr;
    unsigned long long *d_sblk = nullptr, *d_pinst = nullptr;
    uint32_t *d_smask = nullptr;
    long long lg_cap = 0, smask_cap = 0;
    size_t nedf_tc_stride = 0, nerf_tc_stride = 0, nerf_pair_off = 0;
    void *d_march_scratch = nullptr;
    size_t march_scratch_bytes = 0;
    uint32_t *d_rs_mask = nullptr;
    uint2 *d_rs_pairs = nullptr;
    Counters *d_rs_cnt = nullptr;
    void *d_rs_scratch = nullptr;
    size_t rs_scratch_bytes = 0;
    long long rs_cap = 0;
    bool profiling = false, profiled = false;
    // CUDA graph of one frame, relaunched while its shape key is unchanged
    struct FrameKey {
        int n_inst, n_lights, depth_source, n_shade, profiling, shade_resample, edit_mode;
        const void *out[5];
        bool operator==(const FrameKey &o) const
        {
            if (n_inst != o.n_inst || n_lights != o.n_lights || depth_source != o.depth_source ||
                n_shade != o.n_shade || profiling != o.profiling || shade_resample != o.shade_resample ||
                edit_mode != o.edit_mode)
                return false;
            for (int i = 0; i < 5; ++i)
                if (out[i] != o.out[i]) return false;
            return true;
        }
    } gkey{};
    cudaGraphExec_t gexec = nullptr;
    int glaunches = 0;
    bool graphs = true;
    cudaEvent_t ev[kStages + 1] = {};
    cudaEvent_t eng_ev[4] = {};       // around the Step-1 and Step-3 tensor-core NeDF engine launches
    bool engines_timed = false, gengines = false;
    int last_launches = 0;
    int stage_bytes[NEDF_N_SCHEDULE] = {0, 0, 0, 0, 0};   // tensor-core schedule (0 = default)
    int operand_order[NEDF_N_SCHEDULE] = {0, 0, 0, 0, 0};
    // guard bytes after every buffer allocated at create: (buffer, its size)
    std::vector<std::pair<const uint8_t *, size_t>> guards;
};

// Bytes of a known pattern after each buffer allocated at create; nedf_compose_validate checks them.
static constexpr size_t kGuardBytes = 256;
static constexpr unsigned char kGuardByte = 0xA5;

// NVTX range over one API call (shows the call in profilers' timelines; free without one)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

static thread_local std::string g_create_error;

namespace nedf {
// Error text of calls that have no handle (returned by nedf_compose_last_error(NULL)).
void set_thread_error(const std::string &msg) { g_create_error = msg; }
}  // namespace nedf

static int fail(nedf_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    else g_create_error = msg;
    return code;
}

static int cuda_fail(nedf_handle *h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? NEDF_ERR_OOM : NEDF_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(h, call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);      \
    } while (0)

static long long mlp_params(int n_in, int hidden, int width, int n_out)
{
    if (hidden <= 0) return 0;
    long long p = (long long)n_in * width + width;
    p += (long long)(hidden - 1) * ((long long)width * width + width);
    p += (long long)width * n_out + n_out;
    return p;
}

// packed W[out][in], b  ->  per layer Wt[in][out], b (the SIMT kernels' layout)
static void to_kernel_layout(const float *src, float *dst, int n_in, int hidden, int width, int n_out)
{
    std::vector<int> dims;
    dims.push_back(n_in);
    for (int l = 0; l < hidden; ++l) dims.push_back(width);
    dims.push_back(n_out);
    size_t off = 0;
    for (size_t l = 0; l + 1 < dims.size(); ++l) {
        int fi = dims[l], fo = dims[l + 1];
        for (int o = 0; o < fo; ++o)
            for (int i = 0; i < fi; ++i) dst[off + (size_t)i * fo + o] = src[off + (size_t)o * fi + i];
        for (int o = 0; o < fo; ++o) dst[off + (size_t)fi * fo + o] = src[off + (size_t)fi * fo + o];
        off += (size_t)fi * fo + fo;
    }
}

static Workspace make_ws(nedf_handle *h)
{
    Workspace ws{};
    ws.frame = h->d_frame;
    ws.types = h->d_types;
    ws.inst = h->d_inst;
    ws.keys = h->d_keys;
    ws.depth = h->d_depth;
    ws.id = h->d_id;
    ws.rgba = h->d_rgba;
    ws.shadow = h->d_shadow;
    ws.out = h->d_out;
    ws.occl = h->d_occl;
    ws.ppairs = h->d_ppairs;
    ws.pcap = h->cfg.primary_pair_capacity;
    ws.spairs = h->d_spairs;
    ws.pgeo = h->d_pgeo;
    ws.sgeo = h->d_sgeo;
    ws.sell = h->d_sell;
    ws.nout[0] = h->d_nout[0];
    ws.nout[1] = h->d_nout[1];
    ws.rs_mask = h->d_rs_mask;
    ws.rs_pairs = h->d_rs_pairs;
    ws.rs_cnt = h->d_rs_cnt;
    ws.rs_scratch = h->d_rs_scratch;
    ws.rs_cap = h->rs_cap;
    ws.edit_keys = h->d_edit_keys;
    ws.edit_rgba = h->d_edit_rgba;
    ws.edit_occl = h->d_edit_occl;
    ws.scap = h->cfg.shadow_pair_capacity;
    ws.hlist = h->d_hlist;
    ws.cnt = h->d_cnt;
    ws.status = h->d_status;
    ws.nedf_w = h->d_nedf_w;
    ws.nedf_stride = h->nedf_params;
    ws.nerf_w = h->d_nerf_w;
    ws.nerf_stride = h->nerf_params;
    ws.nedf_hidden = h->cfg.nedf_hidden;
    ws.nedf_width = h->cfg.nedf_width;
    ws.nedf_arch = h->cfg.nedf_arch;
    ws.pair_geo = h->cfg.precision != NEDF_PREC_FP32 || h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER;
    ws.nerf_hidden = h->cfg.nerf_hidden;
    ws.nerf_width = h->cfg.nerf_width;
    ws.precision = h->cfg.precision;
    ws.depth_source = h->opt.depth_source;
    ws.nedf_tc = h->d_nedf_tc;
    ws.nedf_tc_stride = h->nedf_tc_stride;
    for (int k = 0; k < NEDF_N_SCHEDULE; ++k) ws.pipe_stage_bytes[k] = h->stage_bytes[k];
    for (int k = 0; k < NEDF_N_SCHEDULE; ++k) ws.pipe_order[k] = h->operand_order[k];
    ws.nerf_tc = h->d_nerf_tc;
    ws.nerf_tc_stride = h->nerf_tc_stride;
    ws.nerf_pair_off = h->nerf_pair_off;
    ws.fb_list[0] = h->d_fb[0];
    ws.fb_list[1] = h->d_fb[1];
    ws.lcam = h->d_lcam;
    ws.lg_count = h->d_lg_count;
    ws.lg_off = h->d_lg_off;
    ws.lg_cursor = h->d_lg_cursor;
    ws.lg_items = h->d_lg_items;
    ws.lg_cap = h->lg_cap;
    ws.lg_big = h->d_lg_big;
    ws.lg_big_count = h->d_lg_big_count;
    ws.lg_G = kLightGridSize;
    ws.max_inst = h->cfg.max_instances;
    ws.scan_tmp = h->d_scan_tmp;
    ws.sblk = h->d_sblk;
    ws.smask = h->d_smask;
    ws.smask_cap = h->smask_cap;
    ws.pinst = h->d_pinst;
    ws.sblk_nb = shadow_bin_blocks(h->num_sms);
    return ws;
}

static bool finite3(const float *v, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

extern "C" {

const char *nedf_compose_last_error(const nedf_handle *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

int nedf_compose_create(const nedf_config *cfg, void *cuda_stream, nedf_handle **out)
{
    if (!cfg || !out) return fail(nullptr, NEDF_ERR_ARG, "null argument");
    *out = nullptr;
    const nedf_config &c = *cfg;
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
        return fail(nullptr, NEDF_ERR_ARG, "width/height out of range");
    if (c.max_instances < 1 || c.max_types < 1 || c.max_types > NEDF_MAX_TYPES)
        return fail(nullptr, NEDF_ERR_ARG, "max_instances/max_types out of range");
    if (c.nedf_arch != NEDF_ARCH_REGRESSION && c.nedf_arch != NEDF_ARCH_CLASSIFIER)
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "nedf_arch");
    if (c.nedf_arch == NEDF_ARCH_CLASSIFIER && c.precision == NEDF_PREC_FP8)
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "the classifier network runs in BF16 or FP32 precision");
    if (c.nedf_arch == NEDF_ARCH_REGRESSION &&
        (c.nedf_hidden < 1 || c.nedf_hidden > 16 || (c.nedf_width != 64 && c.nedf_width != 128 && c.nedf_width != 256)))
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "NeDF shape: hidden 1..16, width 64/128/256");
    if (c.nerf_hidden < 0 || c.nerf_hidden > 16 ||
        (c.nerf_hidden > 0 && c.nerf_width != 64 && c.nerf_width != 128 && c.nerf_width != 256))
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "NeRF shape: hidden 0..16, width 64/128/256");
    if (c.precision != NEDF_PREC_FP32 && c.precision != NEDF_PREC_BF16 && c.precision != NEDF_PREC_FP8)
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "precision");
    if (c.nedf_arch == NEDF_ARCH_REGRESSION && c.precision != NEDF_PREC_FP32 && c.nedf_width > 128)
        return fail(nullptr, NEDF_ERR_UNSUPPORTED, "tensor-core NeDF width must be 64 or 128");
    if (c.primary_pair_capacity < 0 || c.shadow_pair_capacity < 0)
        return fail(nullptr, NEDF_ERR_ARG, "negative capacity");

    nedf_handle *h = new nedf_handle();
    h->cfg = c;
    long long npix = (long long)c.width * c.height;
    if (h->cfg.primary_pair_capacity == 0) h->cfg.primary_pair_capacity = 8 * npix;
    if (h->cfg.shadow_pair_capacity == 0) h->cfg.shadow_pair_capacity = 4 * npix * NEDF_MAX_LIGHTS / 8;
    h->stream = (cudaStream_t)cuda_stream;
    h->opt = nedf_options{8, 0.05f, 0.5f, 0.02f, 50.0f, 0.01f, NEDF_DEPTH_NEDF, 128, 4, 0.0f, 0, 0, 0, 1.0f};
    if (c.nedf_arch == NEDF_ARCH_CLASSIFIER) {     // the fixed shape; the regression kernels are unused
        h->cfg.nedf_hidden = 1;
        h->cfg.nedf_width = 64;
    }
    h->nedf_params = c.nedf_arch == NEDF_ARCH_CLASSIFIER ? kClsParams : mlp_params(kNedfIn, c.nedf_hidden, c.nedf_width, 2);
    h->nerf_params = mlp_params(kNerfIn, c.nerf_hidden, c.nerf_width, 3);
    auto bail = [&](cudaError_t e, const char *what) {
        int code = e == cudaErrorMemoryAllocation ? NEDF_ERR_OOM : NEDF_ERR_CUDA;
        g_create_error = std::string(what) + ": " + cudaGetErrorString(e);
        nedf_compose_destroy(h);
        return code;
    };
    cudaError_t e;
#define CA(ptr, bytes)                                                                      \
    do {                                                                                    \
        const size_t nb_ = (bytes);                                                         \
        e = cudaMalloc((void **)&(ptr), nb_ + kGuardBytes);                                 \
        if (e != cudaSuccess) return bail(e, "cudaMalloc " #ptr);                           \
        e = cudaMemset(reinterpret_cast<uint8_t *>(ptr) + nb_, kGuardByte, kGuardBytes);    \
        if (e != cudaSuccess) return bail(e, "cudaMemset guard " #ptr);                     \
        h->guards.emplace_back(reinterpret_cast<const uint8_t *>(ptr), nb_);               \
    } while (0)
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) return bail(e, "cudaGetDevice");
    if ((e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess)
        return bail(e, "cudaDeviceGetAttribute");
    CA(h->d_frame, sizeof(DevFrame));
    CA(h->d_cam, sizeof(HostCamera));
    if ((e = cudaMallocHost((void **)&h->h_frame, sizeof(DevFrame))) != cudaSuccess) return bail(e, "cudaMallocHost");
    if ((e = cudaMallocHost((void **)&h->h_cam, sizeof(HostCamera))) != cudaSuccess) return bail(e, "cudaMallocHost");
    CA(h->d_types, sizeof(DevType) * c.max_types);
    CA(h->d_inst, sizeof(DevInst) * c.max_instances);
    CA(h->d_nedf_w, sizeof(float) * h->nedf_params * c.max_types);
    if (h->nerf_params) CA(h->d_nerf_w, sizeof(float) * h->nerf_params * c.max_types);
    CA(h->d_keys, sizeof(unsigned long long) * npix);
    CA(h->d_depth, sizeof(float) * npix);
    CA(h->d_shadow, sizeof(float) * npix);
    CA(h->d_id, sizeof(uint32_t) * npix);
    CA(h->d_occl, sizeof(uint32_t) * npix);
    CA(h->d_hlist, sizeof(uint32_t) * npix * c.max_types);
    CA(h->d_rgba, sizeof(float4) * npix);
    CA(h->d_out, sizeof(float4) * npix);
    CA(h->d_ppairs, sizeof(uint2) * h->cfg.primary_pair_capacity);
    CA(h->d_spairs, sizeof(uint2) * h->cfg.shadow_pair_capacity);
    CA(h->d_pgeo, 2 * sizeof(float4) * h->cfg.primary_pair_capacity);
    CA(h->d_sgeo, 2 * sizeof(float4) * h->cfg.shadow_pair_capacity);
    CA(h->d_sell, sizeof(float) * h->cfg.shadow_pair_capacity);
    CA(h->d_nout[0], sizeof(float2) * h->cfg.primary_pair_capacity);
    CA(h->d_nout[1], sizeof(float2) * h->cfg.shadow_pair_capacity);
    CA(h->d_cnt, sizeof(Counters));
    CA(h->d_status, sizeof(uint32_t));
    CA(h->d_loss, sizeof(float) * 4);
    CA(h->d_fb[0], sizeof(uint32_t) * h->cfg.primary_pair_capacity);
    CA(h->d_fb[1], sizeof(uint32_t) * h->cfg.shadow_pair_capacity);
    {
        const size_t cells = (size_t)NEDF_MAX_LIGHTS * kLightGridSize * kLightGridSize;
        // grid items over all lights: 512 cells per instance per light on average (one instance
        // covers at most 1024 of a light's cells; larger ones are listed apart)
        h->lg_cap = (long long)c.max_instances * 512 * NEDF_MAX_LIGHTS;
        CA(h->d_lcam, sizeof(LightCam) * NEDF_MAX_LIGHTS);
        CA(h->d_lg_count, sizeof(uint32_t) * cells);
        CA(h->d_lg_off, sizeof(uint32_t) * (cells + 1));
        CA(h->d_lg_cursor, sizeof(uint32_t) * cells);
        CA(h->d_lg_items, sizeof(uint32_t) * h->lg_cap);
        CA(h->d_lg_big, sizeof(uint32_t) * (size_t)NEDF_MAX_LIGHTS * c.max_instances);
        CA(h->d_lg_big_count, sizeof(uint32_t) * NEDF_MAX_LIGHTS);
        CA(h->d_scan_tmp, sizeof(uint32_t) * 1024);
        CA(h->d_sblk, sizeof(unsigned long long) * kMaxTypes * (shadow_bin_blocks(h->num_sms) + 1));
        CA(h->d_pinst, sizeof(unsigned long long) * 2 * c.max_instances);
        // shadow rays' kept-candidate masks (count pass -> fill pass), for up to 8 lights per pixel;
        // frames with more shadow rays fill without them
        h->smask_cap = (npix + 32) * 8;
        CA(h->d_smask, sizeof(uint32_t) * h->smask_cap);
    }
    if (c.precision == NEDF_PREC_FP32 && c.nedf_arch == NEDF_ARCH_CLASSIFIER) {
        h->nedf_tc_stride = cls_f32_blob_size();          // the CUDA-core classifier's FP32 weights
        CA(h->d_nedf_tc, h->nedf_tc_stride * c.max_types);
    }
    if (c.precision != NEDF_PREC_FP32) {
        const bool f8 = c.precision == NEDF_PREC_FP8;
        h->nedf_tc_stride = c.nedf_arch == NEDF_ARCH_CLASSIFIER ? cls_blob_size()
                                                                : pipe_blob_size(kNedfInPad, c.nedf_width, c.nedf_hidden, 2, f8);
        CA(h->d_nedf_tc, h->nedf_tc_stride * c.max_types);
        if (c.nerf_hidden > 0) {
            // width 256: each type's blob holds the one-SM layout, then the SM-pair layout
            h->nerf_pair_off = c.nerf_width == 256 ? pipe_blob_size(kNerfInPad, c.nerf_width, c.nerf_hidden, 3, f8) : 0;
            h->nerf_tc_stride = pipe_blob_size(kNerfInPad, c.nerf_width, c.nerf_hidden, 3, f8) + h->nerf_pair_off;
            CA(h->d_nerf_tc, h->nerf_tc_stride * c.max_types);
        }
    }
#undef CA
    if ((e = cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), h->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaMemsetAsync(h->d_cnt, 0, sizeof(Counters), h->stream)) != cudaSuccess) return bail(e, "memset");
    if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(e, "sync");
    h->train.resize(c.max_types);
    *out = h;
    return NEDF_OK;
}

void nedf_compose_destroy(nedf_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    void *dev[] = {h->d_frame, h->d_cam, h->d_types, h->d_inst, h->d_nedf_w, h->d_nerf_w, h->d_keys,
                   h->d_depth, h->d_shadow, h->d_id, h->d_occl, h->d_hlist, h->d_rgba, h->d_out,
                   h->d_ppairs, h->d_spairs, h->d_pgeo, h->d_sgeo, h->d_sell, h->d_nout[0], h->d_nout[1], h->d_rs_mask, h->d_rs_pairs, h->d_rs_cnt, h->d_rs_scratch, h->d_edit_keys, h->d_edit_rgba, h->d_edit_occl, h->d_cnt, h->d_status, h->d_loss, h->d_train_scratch,
                   h->d_march_scratch, h->d_nedf_tc, h->d_nerf_tc, h->d_fb[0], h->d_fb[1], h->d_lcam,
                   h->d_lg_count, h->d_lg_off, h->d_lg_cursor, h->d_lg_items, h->d_lg_big,
                   h->d_lg_big_count, h->d_scan_tmp, h->d_sblk, h->d_pinst, h->d_smask};
    for (void *p : dev)
        if (p) cudaFree(p);
    for (TrainState &t : h->train) {
        void *tp[] = {t.o, t.d, t.m_star, t.hit_star, t.master, t.adam_m, t.adam_v};
        for (void *p : tp)
            if (p) cudaFree(p);
    }
    if (h->h_frame) cudaFreeHost(h->h_frame);
    if (h->h_cam) cudaFreeHost(h->h_cam);
    for (cudaEvent_t e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    delete h;
}

int nedf_compose_set_options(nedf_handle *h, const nedf_options *o)
{
    if (!h || !o) return fail(h, NEDF_ERR_ARG, "null argument");
    if (o->n_shade < 1 || o->n_shade > 32) return fail(h, NEDF_ERR_ARG, "n_shade must be 1..32");
    if (!(o->shade_half > 0.f) || !(o->shadow_beta > 0.f && o->shadow_beta < 1.f) || !(o->shadow_eps >= 0.f) ||
        !(o->sigma_max > 0.f) || !(o->sdf_width > 0.f) || !std::isfinite(o->shade_half) || !std::isfinite(o->shadow_eps))
        return fail(h, NEDF_ERR_ARG, "option out of range");
    if (o->depth_source != NEDF_DEPTH_NEDF && o->depth_source != NEDF_DEPTH_MARCH)
        return fail(h, NEDF_ERR_ARG, "depth_source");
    if (o->march_steps < 1 || o->march_steps > 65536 || o->march_bisect < 0 || o->march_bisect > 64)
        return fail(h, NEDF_ERR_ARG, "march_steps 1..65536, march_bisect 0..64");
    if (!(o->fallback_conf >= 0.f && o->fallback_conf <= 1.f) || o->refine_steps < 0 || o->refine_steps > 64)
        return fail(h, NEDF_ERR_ARG, "fallback_conf / refine_steps");
    if (o->shade_resample < 0 || o->shade_resample > 1024 || !(o->shade_sigma_min >= 0.f) || !std::isfinite(o->shade_sigma_min))
        return fail(h, NEDF_ERR_ARG, "shade_resample 0..1024, shade_sigma_min >= 0");
    if (o->miss_check < 0 || o->miss_check > 64) return fail(h, NEDF_ERR_ARG, "miss_check 0..64");
    if (o->shade_resample > 0) {
        // buffers of Step-2 resampling: outlier flags, a pair list of up to a quarter of the
        // pixels' worth of pairs and the plain method's scratch for it (grown with the samples)
        const long long npix = (long long)h->cfg.width * h->cfg.height;
        const long long cap = std::max<long long>(1 << 16, std::min<long long>(h->cfg.primary_pair_capacity, npix / 4));
        const size_t need = march_bytes((int)npix, cap, o->shade_resample);
        if (!h->d_rs_mask) {
            cudaError_t e = cudaMalloc((void **)&h->d_rs_mask, sizeof(uint32_t) * npix);
            if (e == cudaSuccess) e = cudaMemset(h->d_rs_mask, 0, sizeof(uint32_t) * npix);
            if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_rs_pairs, sizeof(uint2) * cap);
            if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_rs_cnt, sizeof(Counters));
            if (e != cudaSuccess) return cuda_fail(h, e, "resampling buffers");
            h->rs_cap = cap;
        }
        if (need > h->rs_scratch_bytes) {
            cudaStreamSynchronize(h->stream);
            if (h->d_rs_scratch) cudaFree(h->d_rs_scratch);
            h->d_rs_scratch = nullptr;
            h->rs_scratch_bytes = 0;
            cudaError_t e = cudaMalloc(&h->d_rs_scratch, need);
            if (e != cudaSuccess) return cuda_fail(h, e, "resampling scratch");
            h->rs_scratch_bytes = need;
        }
    }
    h->opt = *o;
    ++h->version;
    return NEDF_OK;
}

int nedf_compose_get_options(const nedf_handle *h, nedf_options *o)
{
    if (!h || !o) return NEDF_ERR_ARG;
    *o = h->opt;
    return NEDF_OK;
}

int nedf_compose_sync(nedf_handle *h)
{
    if (!h) return NEDF_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    uint32_t st = 0;
    CK(h, cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st) {
        CK(h, cudaMemset(h->d_status, 0, sizeof(uint32_t)));
        if (st & kStatusTimeout) return fail(h, NEDF_ERR_TIMEOUT, "a bounded device wait gave up");
        return fail(h, NEDF_ERR_CAPACITY, st & kStatusPrimaryOverflow ? "primary pair list overflowed"
                                          : st & kStatusShadowOverflow ? "shadow pair list overflowed"
                                                                       : "resampling pair list overflowed");
    }
    return NEDF_OK;
}

// Packs one type's FP32 master weights (device) into its tensor-core blob.
static cudaError_t pack_nedf(nedf_handle *h, const float *master, uint8_t *blob)
{
    if (h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER)
        return h->cfg.precision == NEDF_PREC_FP32 ? launch_pack_cls_f32(master, blob, h->stream)
                                                  : launch_pack_cls(master, blob, h->stream);
    return launch_pack_pipe(master, blob, kNedfIn, kNedfInPad, h->cfg.nedf_width, h->cfg.nedf_hidden, 2,
                            h->cfg.precision == NEDF_PREC_FP8, false, h->stream);
}

int nedf_compose_set_types(nedf_handle *h, int n_types, const nedf_type_desc *types)
{
    if (h) ++h->version;
    NvtxRange nvtx_("nedf_compose_set_types");
    if (!h || !types) return fail(h, NEDF_ERR_ARG, "null argument");
    if (n_types < 1 || n_types > h->cfg.max_types) return fail(h, NEDF_ERR_ARG, "n_types out of range");
    std::vector<DevType> dt(n_types);
    std::vector<float> nedf((size_t)h->nedf_params * n_types), nerf((size_t)h->nerf_params * n_types);
    for (int k = 0; k < n_types; ++k) {
        const nedf_type_desc &t = types[k];
        if (t.sdf_kind < 0 || t.sdf_kind > 7) return fail(h, NEDF_ERR_ARG, "unknown sdf_kind");
        if (!(t.rb > 0.f) || !std::isfinite(t.rb) || !finite3(t.sdf_params, 8) || !finite3(t.albedo, 3))
            return fail(h, NEDF_ERR_ARG, "type parameters must be finite, rb > 0");
        if (!t.nedf_weights) return fail(h, NEDF_ERR_ARG, "missing NeDF weights");
        if (h->cfg.nerf_hidden > 0 && !t.nerf_weights) return fail(h, NEDF_ERR_ARG, "missing NeRF weights");
        if (!finite3(t.nedf_weights, (int)h->nedf_params)) return fail(h, NEDF_ERR_ARG, "non-finite NeDF weight");
        if (h->nerf_params && !finite3(t.nerf_weights, (int)h->nerf_params))
            return fail(h, NEDF_ERR_ARG, "non-finite NeRF weight");
        dt[k].kind = t.sdf_kind;
        for (int i = 0; i < 8; ++i) dt[k].p[i] = t.sdf_params[i];
        dt[k].rb = t.rb;
        for (int i = 0; i < 3; ++i) dt[k].albedo[i] = t.albedo[i];
        dt[k].nerf = h->cfg.nerf_hidden > 0;
        if (h->cfg.nedf_arch == NEDF_ARCH_REGRESSION)
            to_kernel_layout(t.nedf_weights, nedf.data() + (size_t)k * h->nedf_params, kNedfIn, h->cfg.nedf_hidden,
                             h->cfg.nedf_width, 2);
        if (h->nerf_params)
            to_kernel_layout(t.nerf_weights, nerf.data() + (size_t)k * h->nerf_params, kNerfIn,
                             h->cfg.nerf_hidden, h->cfg.nerf_width, 3);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(h->d_types, dt.data(), sizeof(DevType) * n_types, cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->d_nedf_w, nedf.data(), sizeof(float) * nedf.size(), cudaMemcpyHostToDevice));
    if (h->nerf_params)
        CK(h, cudaMemcpy(h->d_nerf_w, nerf.data(), sizeof(float) * nerf.size(), cudaMemcpyHostToDevice));
    h->types_host = dt;
    h->n_types = n_types;
    // training state: master weights = the given packed weights, fresh moments
    for (int k = 0; k < n_types; ++k) {
        TrainState &ts = h->train[k];
        size_t bytes = sizeof(float) * h->nedf_params;
        if (!ts.master) {
            CK(h, cudaMalloc((void **)&ts.master, bytes));
            CK(h, cudaMalloc((void **)&ts.adam_m, bytes));
            CK(h, cudaMalloc((void **)&ts.adam_v, bytes));
        }
        CK(h, cudaMemcpy(ts.master, types[k].nedf_weights, bytes, cudaMemcpyHostToDevice));
        CK(h, cudaMemset(ts.adam_m, 0, bytes));
        CK(h, cudaMemset(ts.adam_v, 0, bytes));
        ts.step = 0;
        ts.cursor = 0;
        if (h->d_nedf_tc)
            CK(h, pack_nedf(h, ts.master, h->d_nedf_tc + (size_t)k * h->nedf_tc_stride));
    }
    if (h->d_nerf_tc) {
        float *tmp = nullptr;
        CK(h, cudaMalloc((void **)&tmp, sizeof(float) * h->nerf_params));
        for (int k = 0; k < n_types; ++k) {
            cudaError_t e = cudaMemcpy(tmp, types[k].nerf_weights, sizeof(float) * h->nerf_params,
                                       cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = launch_pack_pipe(tmp, h->d_nerf_tc + (size_t)k * h->nerf_tc_stride, kNerfIn, kNerfInPad,
                                   h->cfg.nerf_width, h->cfg.nerf_hidden, 3, h->cfg.precision == NEDF_PREC_FP8, false,
                                   h->stream);
            if (e == cudaSuccess && h->nerf_pair_off)
                e = launch_pack_pipe(tmp, h->d_nerf_tc + (size_t)k * h->nerf_tc_stride + h->nerf_pair_off, kNerfIn,
                                     kNerfInPad, h->cfg.nerf_width, h->cfg.nerf_hidden, 3,
                                     h->cfg.precision == NEDF_PREC_FP8, true, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) {
                cudaFree(tmp);
                return cuda_fail(h, e, "NeRF weight packing");
            }
        }
        cudaFree(tmp);
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return NEDF_OK;
}

int nedf_compose_set_instances(nedf_handle *h, int n, const nedf_instance *inst)
{
    NvtxRange nvtx_("nedf_compose_set_instances");
    if (!h || (!inst && n > 0)) return fail(h, NEDF_ERR_ARG, "null argument");
    if (h->n_types == 0) return fail(h, NEDF_ERR_STATE, "set_types first");
    if (n < 0 || n > h->cfg.max_instances) return fail(h, NEDF_ERR_ARG, "instance count out of range");
    std::vector<DevInst> di(n > 0 ? n : 1);
    for (int i = 0; i < n; ++i) {
        const nedf_instance &s = inst[i];
        if (s.type >= (uint32_t)h->n_types) return fail(h, NEDF_ERR_ARG, "instance type out of range");
        if (!finite3(s.R, 9) || !finite3(s.T, 3) || !std::isfinite(s.s) || !(s.s > 0.f))
            return fail(h, NEDF_ERR_ARG, "instance transform must be finite with s > 0");
        std::memcpy(di[i].R, s.R, sizeof(s.R));
        std::memcpy(di[i].T, s.T, sizeof(s.T));
        di[i].s = s.s;
        di[i].type = s.type;
        di[i].pad[0] = di[i].pad[1] = 0.f;
    }
    if (n > 0)
        CK(h, cudaMemcpyAsync(h->d_inst, di.data(), sizeof(DevInst) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));   // di is a host temporary
    h->n_inst = n;
    di.resize(n);
    h->h_inst = std::move(di);
    return NEDF_OK;
}

static int check_frame_args(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights)
{
    if (!h || !cam || (!lights && n_lights > 0)) return fail(h, NEDF_ERR_ARG, "null argument");
    if (h->n_types == 0 || h->n_inst == 0) return fail(h, NEDF_ERR_STATE, "set_types and set_instances first");
    if (n_lights < 1 || n_lights > NEDF_MAX_LIGHTS) return fail(h, NEDF_ERR_ARG, "n_lights must be 1..32");
    if (!finite3(cam->eye, 3) || !finite3(cam->target, 3) || !(cam->fov_y_deg > 0.f && cam->fov_y_deg < 180.f))
        return fail(h, NEDF_ERR_ARG, "camera");
    float dx = cam->target[0] - cam->eye[0], dz = cam->target[2] - cam->eye[2];
    float dy = cam->target[1] - cam->eye[1];
    if (dx * dx + dz * dz <= 1e-12f * (dx * dx + dy * dy + dz * dz) || (dx == 0.f && dy == 0.f && dz == 0.f))
        return fail(h, NEDF_ERR_ARG, "camera must not look along the up axis");
    for (int l = 0; l < n_lights; ++l) {
        if (!finite3(lights[l].pos, 3)) return fail(h, NEDF_ERR_ARG, "light");
        if (lights[l].parallel && !(std::fabs(lights[l].pos[0]) + std::fabs(lights[l].pos[1]) + std::fabs(lights[l].pos[2]) > 0.f))
            return fail(h, NEDF_ERR_ARG, "a parallel light needs a non-zero direction");
    }
    return NEDF_OK;
}

// Writes this frame's camera, lights and options into the pinned staging records (the copies
// to the device are part of the frame's launch sequence).
static cudaError_t stage_frame(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights)
{
    cudaError_t e = cudaStreamSynchronize(h->stream);   // the previous frame may still read the staging
    if (e != cudaSuccess) return e;
    DevFrame &f = *h->h_frame;
    std::memset(&f, 0, sizeof(f));
    f.W = h->cfg.width;
    f.H = h->cfg.height;
    f.n_lights = n_lights;
    f.parallel_mask = 0u;
    for (int l = 0; l < n_lights; ++l) {
        float p[3] = {lights[l].pos[0], lights[l].pos[1], lights[l].pos[2]};
        if (lights[l].parallel) {                  // a parallel light's direction, normalised
            const float n = std::sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
            for (float &v : p) v /= n;
            f.parallel_mask |= 1u << l;
        }
        for (int c = 0; c < 3; ++c) f.lights[l][c] = p[c];
    }
    f.n_shade = h->opt.n_shade;
    f.shade_half = h->opt.shade_half;
    f.beta = h->opt.shadow_beta;
    f.eps = h->opt.shadow_eps;
    f.sigma_max = h->opt.sigma_max;
    f.sdf_width = h->opt.sdf_width;
    f.depth_source = h->opt.depth_source;
    f.march_steps = h->opt.march_steps;
    f.march_bisect = h->opt.march_bisect;
    f.fallback_conf = h->opt.fallback_conf;
    f.refine_steps = h->opt.refine_steps;
    f.outlier_resample = h->opt.outlier_resample;
    f.shade_resample = h->opt.shade_resample;
    f.shade_sigma_min = h->opt.shade_sigma_min;
    f.miss_check = h->opt.miss_check;
    f.edit_mode = h->edit_mode;
    f.edit_inst = h->edit_inst;
    f.n_inst = h->n_inst;
    f.n_types = h->n_types;
    std::memcpy(h->h_cam->eye, cam->eye, sizeof(cam->eye));
    std::memcpy(h->h_cam->target, cam->target, sizeof(cam->target));
    h->h_cam->fov_y_deg = cam->fov_y_deg;
    return cudaSuccess;
}

static cudaError_t enqueue_upload(nedf_handle *h)
{
    cudaError_t e = cudaMemcpyAsync(h->d_frame, h->h_frame, sizeof(DevFrame), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(h->d_cam, h->h_cam, sizeof(HostCamera), cudaMemcpyHostToDevice, h->stream);
}

static cudaError_t upload_frame(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights)
{
    cudaError_t e = stage_frame(h, cam, lights, n_lights);
    return e != cudaSuccess ? e : enqueue_upload(h);
}

static int fill_stats(nedf_handle *h, nedf_frame_stats *stats)
{
    CK(h, cudaStreamSynchronize(h->stream));
    Counters c;
    uint32_t st = 0;
    CK(h, cudaMemcpy(&c, h->d_cnt, sizeof(c), cudaMemcpyDeviceToHost));
    CK(h, cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    stats->primary_pairs = (int64_t)c.p_off[h->n_types];
    stats->shadow_pairs = (int64_t)c.s_off[h->n_types];
    stats->hit_pixels = (int64_t)c.hit_pixels;
    stats->fallback_pairs = (int64_t)c.fallback;
    stats->kernel_launches = h->last_launches;
    stats->status = st;
    stats->resampled_pixels = (int64_t)c.rs_pixels;
    return nedf_compose_sync(h);
}

// One frame.  Caller device buffers (any may be NULL) receive the outputs directly.  On a
// stream other than the legacy default stream the upload and the launch sequence are captured
// into a CUDA graph, relaunched while the shape key (instance and light counts, depth source,
// samples per pixel, profiling, output buffers) stays the same.
static int render_impl(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights,
                       float *depth = nullptr, uint32_t *id = nullptr, float *rgba = nullptr, float *shadow = nullptr,
                       float *out = nullptr)
{
    CK(h, stage_frame(h, cam, lights, n_lights));
    FrameLaunch L;
    L.ws = make_ws(h);
    if (depth) L.ws.depth = depth;
    if (id) L.ws.id = id;
    if (rgba) L.ws.rgba = reinterpret_cast<float4 *>(rgba);
    if (shadow) L.ws.shadow = shadow;
    if (out) L.ws.out = reinterpret_cast<float4 *>(out);
    L.stream = h->stream;
    L.W = h->cfg.width;
    L.H = h->cfg.height;
    L.num_sms = h->num_sms;
    L.n_inst = h->n_inst;
    L.n_shade = h->opt.n_shade;
    L.n_lights = n_lights;
    L.shade_resample = h->opt.shade_resample;
    L.edit_mode = h->edit_mode;
    h->last_mode = h->edit_mode;
    L.cam = h->d_cam;
    L.events = h->profiling ? h->ev : nullptr;
    L.engine_events = h->profiling ? h->eng_ev : nullptr;
    L.launches = 0;
    L.engines_timed = false;
    if (!h->graphs || h->stream == nullptr) {
        CK(h, enqueue_upload(h));
        CK(h, launch_frame(L));
        h->last_launches = L.launches;
        h->engines_timed = L.engines_timed;
    } else {
        nedf_handle::FrameKey key{h->n_inst, n_lights, h->opt.depth_source, h->opt.n_shade, h->profiling ? 1 : 0,
                                  h->opt.shade_resample, h->edit_mode, {depth, id, rgba, shadow, out}};
        if (!h->gexec || !(key == h->gkey)) {
            if (h->gexec) {
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
            CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = enqueue_upload(h);
            if (e == cudaSuccess) e = launch_frame(L);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                h->gexec = nullptr;
                return cuda_fail(h, e, "frame graph capture");
            }
            h->gkey = key;
            h->glaunches = L.launches;
            h->gengines = L.engines_timed;
        }
        CK(h, cudaGraphLaunch(h->gexec, h->stream));
        h->last_launches = h->glaunches;
        h->engines_timed = h->gengines;
    }
    if (h->profiling) h->profiled = true;
    return NEDF_OK;
}

int nedf_compose_render(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights,
                        float *depth, uint32_t *id, float *rgba, float *shadow, float *out,
                        nedf_frame_stats *stats)
{
    NvtxRange nvtx_("nedf_compose_render");
    int r = check_frame_args(h, cam, lights, n_lights);
    if (r != NEDF_OK) return r;
    r = render_impl(h, cam, lights, n_lights, depth, id, rgba, shadow, out);
    if (r != NEDF_OK) return r;
    if (stats) return fill_stats(h, stats);
    return NEDF_OK;
}

int nedf_compose_begin_edit(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights, int inst)
{
    NvtxRange nvtx_("nedf_compose_begin_edit");
    int r = check_frame_args(h, cam, lights, n_lights);
    if (r != NEDF_OK) return r;
    if (inst < 0 || inst >= h->n_inst) return fail(h, NEDF_ERR_ARG, "inst out of range");
    if (h->opt.shade_resample > 0)
        return fail(h, NEDF_ERR_UNSUPPORTED, "buffer reuse with Step-2 outlier resampling (its pixels depend on every object)");
    const size_t npix = (size_t)h->cfg.width * h->cfg.height;
    if (!h->d_edit_keys) {
        cudaError_t e = cudaMalloc((void **)&h->d_edit_keys, sizeof(unsigned long long) * npix);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_edit_rgba, sizeof(float4) * npix);
        if (e == cudaSuccess) e = cudaMalloc((void **)&h->d_edit_occl, sizeof(uint32_t) * npix);
        if (e != cudaSuccess) return cuda_fail(h, e, "buffer reuse buffers");
    }
    h->edit_active = false;
    h->edit_inst = inst;
    h->edit_mode = 1;                                      // the frozen part, into the handle's buffers
    r = render_impl(h, cam, lights, n_lights);
    h->edit_mode = 0;
    if (r != NEDF_OK) return r;
    CK(h, cudaMemcpyAsync(h->d_edit_keys, h->d_keys, sizeof(unsigned long long) * npix, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->d_edit_rgba, h->d_rgba, sizeof(float4) * npix, cudaMemcpyDeviceToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->d_edit_occl, h->d_occl, sizeof(uint32_t) * npix, cudaMemcpyDeviceToDevice, h->stream));
    r = nedf_compose_sync(h);                              // the frozen frame's device status
    if (r != NEDF_OK) return r;
    h->edit_active = true;
    h->edit_inst_snapshot = h->h_inst;
    h->edit_cam = *cam;
    h->edit_lights.assign(lights, lights + n_lights);
    h->edit_version = h->version;
    return NEDF_OK;
}

int nedf_compose_render_edit(nedf_handle *h, float *depth, uint32_t *id, float *rgba, float *shadow, float *out,
                             nedf_frame_stats *stats)
{
    NvtxRange nvtx_("nedf_compose_render_edit");
    if (!h) return NEDF_ERR_ARG;
    if (!h->edit_active) return fail(h, NEDF_ERR_STATE, "no edit session (nedf_compose_begin_edit)");
    if (h->opt.shade_resample > 0)
        return fail(h, NEDF_ERR_UNSUPPORTED, "buffer reuse with Step-2 outlier resampling (its pixels depend on every object)");
    if (h->version != h->edit_version || h->h_inst.size() != h->edit_inst_snapshot.size())
        return fail(h, NEDF_ERR_STATE, "types, options, weights or the instance count changed since begin_edit");
    for (size_t i = 0; i < h->h_inst.size(); ++i)
        if ((int)i != h->edit_inst && std::memcmp(&h->h_inst[i], &h->edit_inst_snapshot[i], sizeof(DevInst)) != 0)
            return fail(h, NEDF_ERR_STATE, "an instance other than the manipulated one changed");
    h->edit_mode = 2;
    int r = render_impl(h, &h->edit_cam, h->edit_lights.data(), (int)h->edit_lights.size(), depth, id, rgba, shadow, out);
    h->edit_mode = 0;
    if (r != NEDF_OK) return r;
    if (stats) return fill_stats(h, stats);
    return NEDF_OK;
}

int nedf_compose_end_edit(nedf_handle *h)
{
    if (!h) return NEDF_ERR_ARG;
    h->edit_active = false;
    h->edit_inst = -1;
    return NEDF_OK;
}

int nedf_compose_render_host(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights,
                             float *depth, uint32_t *id, float *rgba, float *shadow, float *out,
                             nedf_frame_stats *stats)
{
    NvtxRange nvtx_("nedf_compose_render_host");
    int r = check_frame_args(h, cam, lights, n_lights);
    if (r != NEDF_OK) return r;
    r = render_impl(h, cam, lights, n_lights);
    if (r != NEDF_OK) return r;
    size_t npix = (size_t)h->cfg.width * h->cfg.height;
    cudaMemcpyKind k = cudaMemcpyDeviceToHost;
    if (depth) CK(h, cudaMemcpyAsync(depth, h->d_depth, npix * 4, k, h->stream));
    if (id) CK(h, cudaMemcpyAsync(id, h->d_id, npix * 4, k, h->stream));
    if (rgba) CK(h, cudaMemcpyAsync(rgba, h->d_rgba, npix * 16, k, h->stream));
    if (shadow) CK(h, cudaMemcpyAsync(shadow, h->d_shadow, npix * 4, k, h->stream));
    if (out) CK(h, cudaMemcpyAsync(out, h->d_out, npix * 16, k, h->stream));
    if (stats) return fill_stats(h, stats);
    return nedf_compose_sync(h);
}

int nedf_compose_render_march(nedf_handle *h, const nedf_camera *cam, int n_samples, int early_stop, float *rgba)
{
    NvtxRange nvtx_("nedf_compose_render_march");
    nedf_light dummy{{0.f, 10.f, 0.f}};
    int r = check_frame_args(h, cam, &dummy, 1);
    if (r != NEDF_OK) return r;
    if (!rgba || n_samples < 1 || n_samples > 4096) return fail(h, NEDF_ERR_ARG, "rgba / n_samples 1..4096");
    CK(h, upload_frame(h, cam, &dummy, 1));
    FrameLaunch L{};
    L.ws = make_ws(h);
    L.stream = h->stream;
    L.W = h->cfg.width;
    L.H = h->cfg.height;
    L.num_sms = h->num_sms;
    L.n_inst = h->n_inst;
    L.n_shade = h->opt.n_shade;
    L.cam = h->d_cam;
    CK(h, launch_primary_binning(L));
    // the pair count sizes the sample-row workspace (this path synchronises once)
    unsigned long long pairs = 0;
    CK(h, cudaMemcpyAsync(&pairs, &h->d_cnt->p_off[h->n_types], sizeof(pairs), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    size_t need = march_bytes(h->cfg.width * h->cfg.height, (long long)pairs, n_samples);
    if (need > h->march_scratch_bytes) {
        if (h->d_march_scratch) cudaFree(h->d_march_scratch);
        h->d_march_scratch = nullptr;
        h->march_scratch_bytes = 0;
        CK(h, cudaMalloc(&h->d_march_scratch, need));
        h->march_scratch_bytes = need;
    }
    CK(h, launch_march_colour_frame(L, h->d_march_scratch, (long long)pairs, n_samples, early_stop,
                                    reinterpret_cast<float4 *>(rgba)));
    return NEDF_OK;
}

const char *nedf_compose_stage_name(int stage)
{
    static const char *names[kStages] = {"setup", "step1_bin", "step1_nedf", "step1_resolve",
                                         "step2_shade", "step3_bin", "step3_nedf", "composite"};
    return (stage >= 0 && stage < kStages) ? names[stage] : "";
}

int nedf_compose_set_profiling(nedf_handle *h, int on)
{
    if (!h) return NEDF_ERR_ARG;
    if (on && !h->ev[0]) {
        for (cudaEvent_t &e : h->ev) CK(h, cudaEventCreate(&e));
        for (cudaEvent_t &e : h->eng_ev) CK(h, cudaEventCreate(&e));
    }
    h->profiling = on != 0;
    return NEDF_OK;
}

int nedf_compose_get_stage_times(nedf_handle *h, float *ms, int n)
{
    if (!h || !ms || n < kStages) return fail(h, NEDF_ERR_ARG, "ms must hold NEDF_N_STAGES floats");
    if (!h->profiled) return fail(h, NEDF_ERR_STATE, "no profiled render");
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < kStages; ++i) CK(h, cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
    return NEDF_OK;
}

int nedf_compose_get_engine_times(nedf_handle *h, float *ms, int n)
{
    if (!h || !ms || n < NEDF_N_ENGINE_TIMES) return fail(h, NEDF_ERR_ARG, "ms must hold NEDF_N_ENGINE_TIMES floats");
    if (!h->profiled) return fail(h, NEDF_ERR_STATE, "no profiled render");
    CK(h, cudaStreamSynchronize(h->stream));
    for (int i = 0; i < NEDF_N_ENGINE_TIMES; ++i) {
        ms[i] = 0.0f;
        if (h->engines_timed) CK(h, cudaEventElapsedTime(&ms[i], h->eng_ev[2 * i], h->eng_ev[2 * i + 1]));
    }
    return NEDF_OK;
}

int nedf_compose_validate(nedf_handle *h)
{
    if (!h) return NEDF_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    std::vector<uint8_t> g(kGuardBytes);
    for (const auto &b : h->guards) {
        CK(h, cudaMemcpy(g.data(), b.first + b.second, kGuardBytes, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < kGuardBytes; ++i)
            if (g[i] != kGuardByte) {
                char msg[160];
                snprintf(msg, sizeof msg, "guard bytes after a %zu-byte device buffer were overwritten", b.second);
                return fail(h, NEDF_ERR_STATE, msg);
            }
    }
    if (!h->n_types) return NEDF_OK;
    Counters c;
    CK(h, cudaMemcpy(&c, h->d_cnt, sizeof(c), cudaMemcpyDeviceToHost));
    uint32_t st = 0;
    CK(h, cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st) return NEDF_OK;      // an overflow or timeout is reported by sync; the lists are then partial
    const int T = h->n_types;
    const bool tc_nedf = (h->cfg.precision != NEDF_PREC_FP32 || h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER) &&
                         h->opt.depth_source == NEDF_DEPTH_NEDF;      // listed pairs, decode and fallback
    const bool tc_shade = h->cfg.precision != NEDF_PREC_FP32 && h->cfg.nerf_hidden > 0;
    const unsigned long long rows = tc_nedf ? kPipeTileRows : 64;
    const unsigned long long ppt = tc_shade ? 2 * (128 / h->opt.n_shade) : 64 / h->opt.n_shade;
    unsigned long long hits = 0;
    auto bad = [&](const char *what, int t) {
        char msg[160];
        snprintf(msg, sizeof msg, "work-list invariant violated: %s (type %d)", what, t);
        return fail(h, NEDF_ERR_STATE, msg);
    };
    if (c.p_off[0] != 0 || c.p_tile[0] != 0 || c.s_off[0] != 0 || c.s_tile[0] != 0 || c.h_tile[0] != 0)
        return bad("segments do not start at 0", 0);
    for (int t = 0; t < T; ++t) {
        const unsigned long long pn = c.p_off[t + 1] - c.p_off[t], sn = c.s_off[t + 1] - c.s_off[t];
        if (c.p_off[t + 1] < c.p_off[t] || c.s_off[t + 1] < c.s_off[t]) return bad("pair offsets decrease", t);
        if (c.p_cursor[t] != c.p_off[t + 1]) return bad("primary segment not filled exactly", t);
        if (c.s_cursor[t] != c.s_off[t + 1]) return bad("shadow segment not filled exactly", t);
        if (c.p_tile[t + 1] - c.p_tile[t] != (pn + rows - 1) / rows) return bad("primary tiles do not cover the pairs", t);
        if (c.s_tile[t + 1] - c.s_tile[t] != (sn + rows - 1) / rows) return bad("shadow tiles do not cover the pairs", t);
        if (c.h_tile[t + 1] - c.h_tile[t] != (c.h_count[t] + ppt - 1) / ppt) return bad("shading tiles", t);
        hits += c.h_count[t];
    }
    // an edit frame lists only the pixels the manipulated instance wins
    if (h->last_mode != 2 && hits != c.hit_pixels) return bad("shading lists do not sum to the hit pixels", -1);
    if (c.fb_count[0] > c.p_off[T] || c.fb_count[1] > c.s_off[T]) return bad("more deferred pairs than pairs", -1);
    if (c.fallback != c.fb_count[0] + c.fb_count[1] && tc_nedf) return bad("deferred pairs not all answered", -1);
    return NEDF_OK;
}

int nedf_compose_inject_status(nedf_handle *h, uint32_t bits)
{
    if (!h) return NEDF_ERR_ARG;
    uint32_t st = 0;
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost));
    st |= bits;
    CK(h, cudaMemcpy(h->d_status, &st, sizeof(st), cudaMemcpyHostToDevice));
    return NEDF_OK;
}

int nedf_compose_check_wait_limit(nedf_handle *h)
{
    if (!h) return NEDF_ERR_ARG;
    CK(h, launch_wait_check(h->d_status, h->stream));
    const int r = nedf_compose_sync(h);
    if (r == NEDF_ERR_TIMEOUT) {
        h->err.clear();
        return NEDF_OK;                              // the wait gave up and reported it
    }
    return r != NEDF_OK ? r : fail(h, NEDF_ERR_STATE, "the bounded wait did not report its timeout");
}

static void drop_graph(nedf_handle *h)
{
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
}

int nedf_compose_set_schedule(nedf_handle *h, const nedf_schedule *s)
{
    if (!h || !s) return fail(h, NEDF_ERR_ARG, "null argument");
    for (int k = 0; k < NEDF_N_SCHEDULE; ++k) {
        const int b = s->stage_bytes[k];
        if (b != 0 && (b < 1024 || b > 262144 || b % 1024 != 0))
            return fail(h, NEDF_ERR_ARG, "stage_bytes: 0 or a multiple of 1024 in [1024, 262144]");
        if (s->operand_order[k] < 0 || s->operand_order[k] > 2) return fail(h, NEDF_ERR_ARG, "operand_order: 0, 1 or 2");
    }
    for (int k = 0; k < NEDF_N_SCHEDULE; ++k) {
        h->stage_bytes[k] = s->stage_bytes[k];
        h->operand_order[k] = s->operand_order[k];
    }
    drop_graph(h);
    return NEDF_OK;
}

int nedf_compose_get_schedule(nedf_handle *h, nedf_schedule *s)
{
    if (!h || !s) return fail(h, NEDF_ERR_ARG, "null argument");
    for (int k = 0; k < NEDF_N_SCHEDULE; ++k) {
        s->stage_bytes[k] = h->stage_bytes[k];
        s->tuned_ms[k] = 0.0f;
        s->operand_order[k] = h->operand_order[k];
    }
    return NEDF_OK;
}

int nedf_compose_autotune(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights, int reps,
                          nedf_schedule *chosen)
{
    NvtxRange nvtx_("nedf_compose_autotune");
    int r = check_frame_args(h, cam, lights, n_lights);
    if (r != NEDF_OK) return r;
    if (reps < 1) return fail(h, NEDF_ERR_ARG, "reps < 1");
    if (h->cfg.precision != NEDF_PREC_FP32) {
        // stage sizes: the kernels round to whole weight chunks (2-8 KB), so 12 and 24 KB give stages
        // of three and six chunks, which divide the 9-chunk NeDF layers evenly
        static const int cand[8] = {8192, 12288, 16384, 24576, 32768, 36864, 49152, 65536};
        constexpr int n_cand = 8;
        // operand orders of the NeDF engines: both at BF16 width 128 (swapped, unswapped), else the one
        const bool orders = h->cfg.nedf_arch == NEDF_ARCH_REGRESSION && h->cfg.precision == NEDF_PREC_BF16 &&
                            h->cfg.nedf_width == 128 && h->opt.depth_source == NEDF_DEPTH_NEDF;
        const int n_order = orders ? 2 : 1;
        // stage index of each tuned kernel: Step-2 shading, Step-1 NeDF, Step-3 NeDF
        static const int kern[3] = {0, 2, 3}, stage[3] = {4, 2, 6};
        float best[3] = {1e30f, 1e30f, 1e30f};
        int pick[3] = {cand[1], cand[1], cand[1]}, pick_order[3] = {0, 0, 0};
        const bool was_profiling = h->profiling;
        r = nedf_compose_set_profiling(h, 1);
        if (r != NEDF_OK) return r;
        for (int o = 0; o < n_order; ++o) {
            const int order = orders ? 1 + o : 0;
            for (int k = 2; k < NEDF_N_SCHEDULE; ++k) h->operand_order[k] = order;
            for (int c = 0; c < n_cand; ++c) {
                for (int k = 0; k < NEDF_N_SCHEDULE; ++k) h->stage_bytes[k] = cand[c];
                drop_graph(h);
                float t[3] = {1e30f, 1e30f, 1e30f};
                for (int i = 0; i <= reps; ++i) {              // the first render captures the graph
                    r = render_impl(h, cam, lights, n_lights);
                    if (r != NEDF_OK) return r;
                    float ms[kStages];
                    r = nedf_compose_get_stage_times(h, ms, kStages);
                    if (r != NEDF_OK) return r;
                    if (i == 0) continue;
                    for (int j = 0; j < 3; ++j) t[j] = std::min(t[j], ms[stage[j]]);
                }
                for (int j = 0; j < 3; ++j)
                    if (t[j] < best[j]) {
                        best[j] = t[j];
                        pick[j] = cand[c];
                        pick_order[j] = order;
                    }
            }
        }
        h->stage_bytes[0] = pick[0];
        h->stage_bytes[1] = pick[0];
        h->stage_bytes[2] = pick[1];
        h->stage_bytes[3] = pick[2];
        h->stage_bytes[4] = pick[1];
        h->operand_order[2] = pick_order[1];
        h->operand_order[3] = pick_order[2];
        h->operand_order[4] = pick_order[1];
        drop_graph(h);
        h->profiling = was_profiling;
        if (chosen) {
            for (int k = 0; k < NEDF_N_SCHEDULE; ++k) {
                chosen->stage_bytes[k] = h->stage_bytes[k];
                chosen->operand_order[k] = h->operand_order[k];
                chosen->tuned_ms[k] = 0.0f;
            }
            for (int j = 0; j < 3; ++j) chosen->tuned_ms[kern[j]] = best[j];
        }
        return NEDF_OK;
    }
    if (chosen) return nedf_compose_get_schedule(h, chosen);
    return NEDF_OK;
}

int nedf_compose_nedf_query(nedf_handle *h, int type, int n, const float *o, const float *d, float *out)
{
    if (!h || !o || !d || !out) return fail(h, NEDF_ERR_ARG, "null argument");
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    if (n < 0) return fail(h, NEDF_ERR_ARG, "n < 0");
    if (h->cfg.precision != NEDF_PREC_FP32)
        CK(h, launch_nedf_pipe(make_ws(h), 2, type, o, d, out, n, h->num_sms, h->stream));
    else if (h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER)
        CK(h, launch_cls_f32(make_ws(h), 2, type, o, d, out, n, h->num_sms, h->stream));
    else
        CK(h, launch_nedf_query_f32(make_ws(h), type, o, d, out, n, h->num_sms, h->stream));
    return NEDF_OK;
}

}  // extern "C"

// ---- learned part -------------------------------------------------------------------------------
extern "C" {

// The type's training set sized for n_rays rows (reallocated when the size changes).
static int ensure_train_set(nedf_handle *h, int type, int64_t n_rays)
{
    TrainState &ts = h->train[type];
    if (ts.n_rays != n_rays) {
        float *p[] = {ts.o, ts.d, ts.m_star, ts.hit_star};
        for (float *q : p)
            if (q) cudaFree(q);
        ts.o = ts.d = ts.m_star = ts.hit_star = nullptr;
        ts.n_rays = 0;
        CK(h, cudaMalloc((void **)&ts.o, sizeof(float) * 3 * n_rays));
        CK(h, cudaMalloc((void **)&ts.d, sizeof(float) * 3 * n_rays));
        CK(h, cudaMalloc((void **)&ts.m_star, sizeof(float) * n_rays));
        CK(h, cudaMalloc((void **)&ts.hit_star, sizeof(float) * n_rays));
        ts.n_rays = n_rays;
    }
    ts.cursor = 0;
    return NEDF_OK;
}

// Copies of the training set to the caller's device buffers (any may be NULL).
static int copy_train_set(nedf_handle *h, int type, int64_t n_rays, float *o, float *d, float *m_star, float *hit_star)
{
    TrainState &ts = h->train[type];
    size_t b3 = sizeof(float) * 3 * n_rays, b1 = sizeof(float) * n_rays;
    if (o) CK(h, cudaMemcpyAsync(o, ts.o, b3, cudaMemcpyDeviceToDevice, h->stream));
    if (d) CK(h, cudaMemcpyAsync(d, ts.d, b3, cudaMemcpyDeviceToDevice, h->stream));
    if (m_star) CK(h, cudaMemcpyAsync(m_star, ts.m_star, b1, cudaMemcpyDeviceToDevice, h->stream));
    if (hit_star) CK(h, cudaMemcpyAsync(hit_star, ts.hit_star, b1, cudaMemcpyDeviceToDevice, h->stream));
    return NEDF_OK;
}

int nedf_compose_make_labels(nedf_handle *h, int type, int64_t n_rays, uint64_t seed, int march_steps,
                             int march_bisect, float *o, float *d, float *m_star, float *hit_star)
{
    NvtxRange nvtx_("nedf_compose_make_labels");
    if (!h) return NEDF_ERR_ARG;
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    if (n_rays < 1 || n_rays > (1ll << 30)) return fail(h, NEDF_ERR_ARG, "n_rays 1..2^30");
    if (march_steps < 1 || march_steps > 65536 || march_bisect < 0 || march_bisect > 64)
        return fail(h, NEDF_ERR_ARG, "march parameters");
    int r = ensure_train_set(h, type, n_rays);
    if (r != NEDF_OK) return r;
    TrainState &ts = h->train[type];
    CK(h, launch_make_labels(h->d_types + type, h->types_host[type].rb, n_rays, seed, march_steps, march_bisect,
                             ts.o, ts.d, ts.m_star, ts.hit_star, h->num_sms, h->stream));
    return copy_train_set(h, type, n_rays, o, d, m_star, hit_star);
}

int nedf_compose_make_labels_density(nedf_handle *h, int type, int64_t n_rays, uint64_t seed, int n_samples,
                                     int dens_hidden, int dens_width, const float *dens_weights, float *o, float *d,
                                     float *m_star, float *hit_star)
{
    NvtxRange nvtx_("nedf_compose_make_labels_density");
    if (!h || !dens_weights) return fail(h, NEDF_ERR_ARG, "null argument");
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    if (n_rays < 1 || n_rays > (1ll << 30)) return fail(h, NEDF_ERR_ARG, "n_rays 1..2^30");
    if (n_samples < 1 || n_samples > kMaxDensSamples) return fail(h, NEDF_ERR_ARG, "n_samples 1..1024");
    if (dens_hidden < 1 || dens_hidden > 8 || (dens_width != 64 && dens_width != 128))
        return fail(h, NEDF_ERR_UNSUPPORTED, "density network: hidden 1..8, width 64 or 128");
    const long long np = mlp_params(kDensIn, dens_hidden, dens_width, 1);
    if (!finite3(dens_weights, (int)np)) return fail(h, NEDF_ERR_ARG, "non-finite density weight");
    int r = ensure_train_set(h, type, n_rays);
    if (r != NEDF_OK) return r;
    std::vector<float> wk((size_t)np);
    to_kernel_layout(dens_weights, wk.data(), kDensIn, dens_hidden, dens_width, 1);
    float *dw = nullptr;
    CK(h, cudaMalloc((void **)&dw, sizeof(float) * np));
    cudaError_t e = cudaMemcpy(dw, wk.data(), sizeof(float) * np, cudaMemcpyHostToDevice);
    TrainState &ts = h->train[type];
    if (e == cudaSuccess)
        e = launch_density_labels(dw, dens_hidden, dens_width, h->types_host[type].rb, n_rays, seed, n_samples, ts.o,
                                  ts.d, ts.m_star, ts.hit_star, h->num_sms, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dw);
    if (e != cudaSuccess) return cuda_fail(h, e, "density labels");
    return copy_train_set(h, type, n_rays, o, d, m_star, hit_star);
}

// BF16 and E4M3 handles train the regression NeDF with BF16 operands on the tensor cores; FP32
// handles (and shapes the tensor-core path does not take) keep the FP32 CUDA-core path.
static bool train_on_tensor_cores(const nedf_handle *h)
{
    return h->cfg.nedf_arch != NEDF_ARCH_CLASSIFIER && h->cfg.precision != NEDF_PREC_FP32 &&
           train_tc_supported(h->cfg.nedf_width, h->cfg.nedf_hidden);
}

static int ensure_train_scratch(nedf_handle *h, int batch)
{
    const bool cls = h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER;
    size_t need = cls ? cls_train_scratch_bytes(batch)
                  : train_on_tensor_cores(h) ? train_tc_scratch_bytes(batch, h->cfg.nedf_hidden, h->cfg.nedf_width, h->nedf_params)
                                             : train_scratch_bytes(batch, h->cfg.nedf_hidden, h->cfg.nedf_width, h->nedf_params);
    if (need > h->train_scratch_bytes) {
        if (h->d_train_scratch) cudaFree(h->d_train_scratch);
        h->d_train_scratch = nullptr;
        h->train_scratch_bytes = 0;
        CK(h, cudaMalloc((void **)&h->d_train_scratch, need));
        h->train_scratch_bytes = need;
    }
    return NEDF_OK;
}

static ClsTrainLaunch make_cls_train_launch(nedf_handle *h, int type)
{
    ClsTrainLaunch L{};
    L.rb = h->types_host[type].rb;
    L.master = h->train[type].master;
    L.scratch = h->d_train_scratch;
    L.loss = h->d_loss;
    L.status = h->d_status;
    L.num_sms = h->num_sms;
    L.stream = h->stream;
    return L;
}

static TrainLaunch make_train_launch(nedf_handle *h, int type)
{
    TrainLaunch L{};
    L.type = h->d_types + type;
    L.rb = h->types_host[type].rb;
    L.hidden = h->cfg.nedf_hidden;
    L.width = h->cfg.nedf_width;
    L.n_params = h->nedf_params;
    L.master = h->train[type].master;
    L.kernel_w = h->d_nedf_w + (size_t)type * h->nedf_params;
    L.scratch = h->d_train_scratch;
    L.loss = h->d_loss;
    L.status = h->d_status;
    L.num_sms = h->num_sms;
    L.stream = h->stream;
    return L;
}

int nedf_compose_loss_grad(nedf_handle *h, int type, int n, const float *o, const float *d, const float *m_star,
                           const float *hit_star, float *grad, float *loss_host)
{
    if (!h || !o || !d || !m_star || !hit_star || !grad) return fail(h, NEDF_ERR_ARG, "null argument");
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    if (n < 1 || n > (1 << 24)) return fail(h, NEDF_ERR_ARG, "n out of range");
    int r = ensure_train_scratch(h, n);
    if (r != NEDF_OK) return r;
    if (h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER) {
        CK(h, launch_cls_loss_grad(make_cls_train_launch(h, type), o, d, m_star, hit_star, n, grad));
    } else if (train_on_tensor_cores(h)) {
        CK(h, launch_loss_grad_tc(make_train_launch(h, type), o, d, m_star, hit_star, n, grad));
    } else {
        TrainLaunch L = make_train_launch(h, type);
        CK(h, launch_loss_grad(L, o, d, m_star, hit_star, n, grad));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    if (loss_host) CK(h, cudaMemcpy(loss_host, h->d_loss, sizeof(float), cudaMemcpyDeviceToHost));
    return nedf_compose_sync(h);
}

int nedf_compose_train_step(nedf_handle *h, int type, int batch, float lr, float *loss_host)
{
    if (h) ++h->version;                           // the weights change
    NvtxRange nvtx_("nedf_compose_train_step");
    if (!h) return NEDF_ERR_ARG;
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    TrainState &ts = h->train[type];
    if (ts.n_rays == 0) return fail(h, NEDF_ERR_STATE, "make_labels first");
    if (batch < 1 || batch > (1 << 22) || batch > ts.n_rays) return fail(h, NEDF_ERR_ARG, "batch out of range");
    if (!(lr > 0.f) || !std::isfinite(lr)) return fail(h, NEDF_ERR_ARG, "lr");
    int r = ensure_train_scratch(h, batch);
    if (r != NEDF_OK) return r;
    ts.step += 1;
    if (h->cfg.nedf_arch == NEDF_ARCH_CLASSIFIER) {
        CK(h, launch_cls_train_step(make_cls_train_launch(h, type), ts.o, ts.d, ts.m_star, ts.hit_star, ts.n_rays,
                                    ts.cursor, batch, ts.adam_m, ts.adam_v, ts.step, lr));
    } else if (train_on_tensor_cores(h)) {
        CK(h, launch_train_step_tc(make_train_launch(h, type), ts.o, ts.d, ts.m_star, ts.hit_star, ts.n_rays,
                                   ts.cursor, batch, ts.adam_m, ts.adam_v, ts.step, lr));
    } else {
        TrainLaunch L = make_train_launch(h, type);
        CK(h, launch_train_step(L, ts.o, ts.d, ts.m_star, ts.hit_star, ts.n_rays, ts.cursor, batch, ts.adam_m,
                                ts.adam_v, ts.step, lr));
    }
    ts.cursor = (ts.cursor + batch) % ts.n_rays;
    if (h->d_nedf_tc)
        CK(h, pack_nedf(h, ts.master, h->d_nedf_tc + (size_t)type * h->nedf_tc_stride));
    if (loss_host) {
        CK(h, cudaStreamSynchronize(h->stream));
        CK(h, cudaMemcpy(loss_host, h->d_loss, sizeof(float), cudaMemcpyDeviceToHost));
    }
    return NEDF_OK;
}

int nedf_compose_get_nedf_weights(nedf_handle *h, int type, float *host_out, int64_t n_floats)
{
    if (!h || !host_out) return fail(h, NEDF_ERR_ARG, "null argument");
    if (type < 0 || type >= h->n_types) return fail(h, NEDF_ERR_ARG, "type out of range");
    if (n_floats < h->nedf_params) return fail(h, NEDF_ERR_ARG, "buffer too small");
    CK(h, cudaStreamSynchronize(h->stream));
    CK(h, cudaMemcpy(host_out, h->train[type].master, sizeof(float) * h->nedf_params, cudaMemcpyDeviceToHost));
    return NEDF_OK;
}

// blob: magic, version, n_types, n_params, then per type: step, master, m, v
int nedf_compose_save_state(nedf_handle *h, void *buf, size_t *size)
{
    if (!h || !size) return fail(h, NEDF_ERR_ARG, "null argument");
    size_t per = sizeof(int32_t) + sizeof(int64_t) + 3 * sizeof(float) * h->nedf_params;
    size_t need = 4 * sizeof(int64_t) + per * h->n_types;
    if (!buf) {
        *size = need;
        return NEDF_OK;
    }
    if (*size < need) return fail(h, NEDF_ERR_ARG, "buffer too small");
    CK(h, cudaStreamSynchronize(h->stream));
    char *p = (char *)buf;
    int64_t hdr[4] = {0x4e45444653544154ll, 2, h->n_types, h->nedf_params};
    std::memcpy(p, hdr, sizeof(hdr));
    p += sizeof(hdr);
    size_t wb = sizeof(float) * h->nedf_params;
    for (int k = 0; k < h->n_types; ++k) {
        int32_t st = h->train[k].step;
        int64_t cur = h->train[k].cursor;
        std::memcpy(p, &st, sizeof(st));
        p += sizeof(st);
        std::memcpy(p, &cur, sizeof(cur));
        p += sizeof(cur);
        CK(h, cudaMemcpy(p, h->train[k].master, wb, cudaMemcpyDeviceToHost)); p += wb;
        CK(h, cudaMemcpy(p, h->train[k].adam_m, wb, cudaMemcpyDeviceToHost)); p += wb;
        CK(h, cudaMemcpy(p, h->train[k].adam_v, wb, cudaMemcpyDeviceToHost)); p += wb;
    }
    *size = need;
    return NEDF_OK;
}

int nedf_compose_load_state(nedf_handle *h, const void *buf, size_t size)
{
    if (h) ++h->version;
    if (!h || !buf) return fail(h, NEDF_ERR_ARG, "null argument");
    int64_t hdr[4];
    if (size < sizeof(hdr)) return fail(h, NEDF_ERR_ARG, "blob too small");
    std::memcpy(hdr, buf, sizeof(hdr));
    size_t per = sizeof(int32_t) + sizeof(int64_t) + 3 * sizeof(float) * h->nedf_params;
    if (hdr[0] != 0x4e45444653544154ll || hdr[1] != 2 || hdr[2] != h->n_types || hdr[3] != h->nedf_params ||
        size < sizeof(hdr) + per * h->n_types)
        return fail(h, NEDF_ERR_ARG, "blob does not match this handle");
    CK(h, cudaStreamSynchronize(h->stream));
    const char *p = (const char *)buf + sizeof(hdr);
    size_t wb = sizeof(float) * h->nedf_params;
    for (int k = 0; k < h->n_types; ++k) {
        int32_t st;
        int64_t cur;
        std::memcpy(&st, p, sizeof(st));
        p += sizeof(st);
        std::memcpy(&cur, p, sizeof(cur));
        p += sizeof(cur);
        h->train[k].step = st;
        h->train[k].cursor = cur;
        CK(h, cudaMemcpy(h->train[k].master, p, wb, cudaMemcpyHostToDevice)); p += wb;
        CK(h, cudaMemcpy(h->train[k].adam_m, p, wb, cudaMemcpyHostToDevice)); p += wb;
        CK(h, cudaMemcpy(h->train[k].adam_v, p, wb, cudaMemcpyHostToDevice)); p += wb;
        TrainLaunch L = make_train_launch(h, k);
        CK(h, launch_refresh_weights(L));
        if (h->d_nedf_tc)
            CK(h, pack_nedf(h, h->train[k].master, h->d_nedf_tc + (size_t)k * h->nedf_tc_stride));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return NEDF_OK;
}

}  // extern "C"
