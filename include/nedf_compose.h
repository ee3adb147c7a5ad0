/* nedf_compose.h -- C ABI of the GB300 (sm_103a) NeDF composition renderer.
 *
 * Method: arXiv 2308.04669, "A General Implicit Framework for Fast NeRF Composition and
 * Rendering".  One render call runs the paper's three render-time steps on one GPU:
 *   Step 1, NeDF generation (Algorithm 1, first half; Eq. 1, 2, 7): every pixel ray is taken
 *     into each instance's local frame, culled against the instance's bound sphere and answered
 *     by the type's Neural Depth Field network; a per-pixel minimum fills the depth and ID
 *     buffers.
 *   Step 2, deferred shading (Algorithm 1, second half; Eq. 8): only the winning instance's
 *     radiance field is evaluated, at samples bracketing the stored depth, into the colour
 *     buffer.
 *   Step 3, shadows (Algorithm 2): shadow rays from each light towards the surface point (from
 *     a point light's position, or from infinity along a parallel light's direction) are
 *     answered by NeDF queries into a shadow buffer that multiplies the colour.
 * The learned part (Section "Intersection network", Eq. 5-6, "Training details") trains each
 * type's NeDF on depth / hit labels that the plain ray-marching method computes on the device.
 *
 * Conventions shared by every call:
 *   - All calls return NEDF_OK (0) or a negative NEDF_ERR_* code and never throw.  The text of
 *     the last error is available from nedf_compose_last_error().
 *   - A handle is bound to one CUDA stream (given at create) and is not thread safe.
 *   - "host" pointers point to ordinary CPU memory; "device" pointers to memory of the GPU that
 *     was current at create.  Unless stated otherwise the caller owns every buffer it passes;
 *     the library copies what it keeps and owns all of its own workspace.
 *   - Device work is asynchronous on the handle's stream.  Errors found by kernels (a full work
 *     list, a wait that gave up) are recorded in a device status word and returned by the next
 *     nedf_compose_sync() (and by any call that synchronises).
 *   - Images are row-major, pixel p = j * width + i with row j = 0 at the top.
 *   - Instance i of the last set_instances() call has id i (Algorithm 1's unique model id).
 *   - Packed MLP weights (float32): for each layer in order, W[out][in] row-major, then b[out].
 *     Hidden layers use ReLU, the output layer is linear.
 *       NeDF dims: [78, nedf_width x nedf_hidden, 2]  input = 6-frequency encoding of
 *                  (entry point on the bound sphere, local direction); outputs (m, a) with
 *                  mu = rb * m (Eq. 1) and hit logit a.
 *       NeRF dims: [90, nerf_width x nerf_hidden, 3]  input = [10-frequency encoding of the
 *                  local position (63), 4-frequency encoding of the local direction (27)];
 *                  outputs are RGB logits (sigmoid applied).
 */
#ifndef NEDF_COMPOSE_H
#define NEDF_COMPOSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------------- */
#define NEDF_OK 0
#define NEDF_ERR_ARG (-1)          /* invalid argument (null, out of range, non-finite)          */
#define NEDF_ERR_CUDA (-2)         /* a CUDA runtime call failed                                 */
#define NEDF_ERR_OOM (-3)          /* device allocation failed                                   */
#define NEDF_ERR_UNSUPPORTED (-4)  /* configuration the library does not implement              */
#define NEDF_ERR_CAPACITY (-5)     /* a device work list overflowed; the frame is incomplete     */
#define NEDF_ERR_TIMEOUT (-6)      /* a bounded device wait gave up                              */
#define NEDF_ERR_STATE (-7)        /* call out of order (e.g. render before set_types)           */

#define NEDF_MAX_LIGHTS 32
#define NEDF_MAX_TYPES 64

/* ---- enums --------------------------------------------------------------------------------- */
enum nedf_precision {       /* arithmetic of the NeDF and NeRF layers (accumulation is FP32)   */
    NEDF_PREC_FP32 = 0,     /* CUDA cores                                                      */
    NEDF_PREC_BF16 = 1,     /* tensor cores, BF16 weights and activations                      */
    NEDF_PREC_FP8 = 2       /* tensor cores: first layer BF16, later hidden layers E4M3 weights
                               (W / s_l, s_l a per-layer power of two) and E4M3 activations;
                               the output layer in FP32 with BF16 weights                       */
};
enum nedf_arch {            /* the NeDF network of every type                                   */
    NEDF_ARCH_REGRESSION = 0, /* a ReLU MLP (nedf_hidden x nedf_width) on the entry point and
                               direction (78 encoded inputs) regressing m = mu / l and a hit logit */
    NEDF_ARCH_CLASSIFIER = 1  /* the paper's intersection network (Section "Intersection network",
                               Appendix A): 16 chord points x 10-frequency encoding (1008 inputs),
                               linear head to 256, 16 residual blocks
                               h' = ReLU(h + W2 ReLU(W1 h + b1) + b2), tails 256 -> 1 + 64 (hit
                               logit, coarse bins) and 256 -> 128 (fine bins), argmax decode of
                               Eq. 4.  Packed weights W[out][in] then b[out]: head, per block W1,
                               b1, W2, b2, tail A, tail B (2,413,249 floats).  Renders in BF16
                               (tensor cores) or FP32 (CUDA cores, the reference precision; FP8
                               is refused); training (loss_grad, train_step) uses the BCE loss of
                               Eq. 6 with every dense product a BF16 tensor-core GEMM (FP32
                               accumulation, FP32 master weights) */
};
enum nedf_depth_source {    /* what answers the (ray, instance) depth queries of Steps 1 and 3 */
    NEDF_DEPTH_NEDF = 0,    /* the Neural Depth Field (the method)                             */
    NEDF_DEPTH_MARCH = 1    /* the plain method: density ray-marching plus bisection           */
};
enum nedf_sdf_kind {        /* analytic object densities sigma = sigma_max * sigmoid(-sdf/w)   */
    NEDF_SDF_SPHERE = 0,    /* params: radius                                                  */
    NEDF_SDF_TORUS = 1,     /* params: R, r (ring in the xz plane)                             */
    NEDF_SDF_BOX = 2,       /* params: half extents x, y, z                                    */
    NEDF_SDF_CAPSULE = 3,   /* params: half length (y), radius                                 */
    NEDF_SDF_ROUNDCONE = 4, /* params: r1, y1, r2, y2                                          */
    NEDF_SDF_TWOSPHERE = 5, /* params: centre offset along x, radius                           */
    NEDF_SDF_TWISTTORUS = 6,/* params: R, r (ring in the xy plane), twist rad per unit y       */
    NEDF_SDF_OCTA = 7       /* params: a in |x|+|y|+|z| = a                                    */
};

/* ---- records ------------------------------------------------------------------------------- */
typedef struct nedf_config {
    int width, height;             /* framebuffer size, 1 .. 16384 each                         */
    int max_instances;             /* capacity of set_instances(); the shadow-map binning keeps */
                                   /* 64 KiB per instance (grid cells over all lights)          */
    int max_types;                 /* capacity of set_types(), <= NEDF_MAX_TYPES                */
    int nedf_hidden, nedf_width;   /* NeDF shape shared by all types: hidden layers, width      */
    int nerf_hidden, nerf_width;   /* NeRF shape shared by all types; nerf_hidden = 0 means a   */
                                   /* constant albedo per type instead of a colour network      */
    int precision;                 /* enum nedf_precision                                       */
    int64_t primary_pair_capacity; /* (ray, instance) pairs of Step 1; 0 = 8 * width * height   */
    int64_t shadow_pair_capacity;  /* pairs of Step 3; 0 = 4 * width * height * NEDF_MAX_LIGHTS/8 */
    int nedf_arch;                 /* enum nedf_arch; with NEDF_ARCH_CLASSIFIER nedf_hidden and */
                                   /* nedf_width are ignored                                    */
} nedf_config;

typedef struct nedf_options {
    int n_shade;             /* samples per pixel in Step 2 (1 .. 32); default 8                */
    float shade_half;        /* half width h of the sample window, object-local; default 0.05   */
    float shadow_beta;       /* darkening factor beta of Algorithm 2, (0,1); default 0.5        */
    float shadow_eps;        /* epsilon of Algorithm 2's test D + eps < |L - x|, world; 0.02    */
    float sigma_max;         /* peak density of the analytic objects; default 50                */
    float sdf_width;         /* width w of the density's sigmoid; default 0.01                  */
    int depth_source;        /* enum nedf_depth_source; default NEDF_DEPTH_NEDF                 */
    int march_steps;         /* plain method: uniform steps over the bound chord; default 128   */
    int march_bisect;        /* plain method: bisection steps after the crossing; default 4     */
    float fallback_conf;     /* NeDF pairs with max(p, 1-p) < this (p = sigmoid(a)) are         */
                             /* re-answered by the plain method; 0 disables; default 0          */
    int refine_steps;        /* density bisection steps in [D - h, D + h] after a NeDF hit; 0   */
    int outlier_resample;    /* with refine_steps > 0: a NeDF hit whose window [D - h, D + h] has */
                             /* no crossing of the half-density level is an outlier (the density */
                             /* check of Section "Deferred Shading") and is re-answered by the   */
                             /* plain method; default 0                                          */
    int shade_resample;      /* Step-2 outlier resampling ("rs", Section "Deferred Shading"): a     */
                             /* shaded pixel whose largest density over its n_shade samples is    */
                             /* below shade_sigma_min (its depth missed the surface) is re-rendered */
                             /* by the plain method's volume rendering of every object on its ray  */
                             /* with this many samples per pair (1 .. 1024); 0 = off (default)     */
    float shade_sigma_min;   /* the outlier threshold ("extremely small" density); default 1.0,   */
                             /* 2 % of the default peak density                                   */
    int miss_check;          /* a NeDF miss kept by the confidence test is checked at this many   */
                             /* midpoints of its bound chord (0 .. 64); if the density there      */
                             /* reaches the half level anywhere, the pair is re-answered by the   */
                             /* plain method (a confidently wrong miss would let a farther object */
                             /* win the pixel); 0 = off (default)                                 */
} nedf_options;

typedef struct nedf_type_desc {
    int sdf_kind;                  /* enum nedf_sdf_kind                                        */
    float sdf_params[8];           /* shape parameters, unused entries ignored                  */
    float rb;                      /* bound-sphere radius l (object-local); mu in [-l, l]        */
    float albedo[3];               /* colour when nerf_hidden == 0                              */
    const float *nedf_weights;     /* host, packed NeDF weights (copied)                        */
    const float *nerf_weights;     /* host, packed NeRF weights (copied); NULL iff nerf_hidden==0 */
} nedf_type_desc;

typedef struct nedf_instance {
    uint32_t type;                 /* index into the types of set_types()                       */
    float R[9];                    /* rotation, row-major: world = s * R * local + T (Eq. 7's G) */
    float T[3];                    /* translation                                               */
    float s;                       /* uniform scale, > 0                                        */
} nedf_instance;

typedef struct nedf_camera {
    float eye[3];                  /* pinhole position (all primary rays start here)            */
    float target[3];               /* look-at point; up is +y                                   */
    float fov_y_deg;               /* vertical field of view, (0, 180)                          */
} nedf_camera;

typedef struct nedf_light {
    float pos[3];                  /* point light: its position, world; parallel light: the     */
                                   /* direction its light travels (any non-zero length)         */
    int parallel;                  /* 0: point light; non-zero: parallel light (Section 1's      */
                                   /* "parallel light sources"; rays from infinity along pos)   */
} nedf_light;

typedef struct nedf_frame_stats {
    int64_t primary_pairs;         /* (pixel ray, instance) pairs that survived the bound cull  */
    int64_t shadow_pairs;          /* (shadow ray, instance) pairs queried                      */
    int64_t hit_pixels;            /* pixels with a valid id                                    */
    int64_t fallback_pairs;        /* pairs re-answered by the plain method                     */
    int64_t kernel_launches;       /* kernels this library launched for the frame               */
    uint32_t status;               /* device status bits (0 = clean)                            */
    int64_t resampled_pixels;      /* pixels re-rendered by Step-2 outlier resampling           */
} nedf_frame_stats;

typedef struct nedf_handle nedf_handle;

/* ---- lifecycle ----------------------------------------------------------------------------- */

/* Creates a renderer for `cfg` on `cuda_stream` (a cudaStream_t; NULL = the legacy default
 * stream) on the current device and allocates all workspace.  *out receives the handle.
 * Errors: NEDF_ERR_ARG (bad sizes, null), NEDF_ERR_UNSUPPORTED (shape or precision this
 * build lacks), NEDF_ERR_OOM, NEDF_ERR_CUDA. */
int nedf_compose_create(const nedf_config *cfg, void *cuda_stream, nedf_handle **out);

/* Frees everything the handle owns.  Synchronises its stream first.  NULL is a no-op. */
void nedf_compose_destroy(nedf_handle *h);

/* Text of the last error on this handle ("" if none); valid until the next call.  With
 * h == NULL, the last error of a failed nedf_compose_create on this thread. */
const char *nedf_compose_last_error(const nedf_handle *h);

/* Replaces the rendering options (host struct, copied).  Defaults are set at create. */
int nedf_compose_set_options(nedf_handle *h, const nedf_options *opt);
int nedf_compose_get_options(const nedf_handle *h, nedf_options *opt);

/* Waits for the handle's stream and returns the first recorded device status as an error code
 * (NEDF_ERR_CAPACITY, NEDF_ERR_TIMEOUT), clearing it; NEDF_OK if clean. */
int nedf_compose_sync(nedf_handle *h);

/* ---- scene --------------------------------------------------------------------------------- */

/* Object types (Section "Manipulating Objects": instances of a type share its NeDF and NeRF
 * weights).  `types` is a host array of n_types records; every pointed-to weight array is
 * copied, converted to the configured precision and laid out for the kernels.  Resets the
 * training state of every type.  Errors: NEDF_ERR_ARG (n_types out of range, unknown kind,
 * rb <= 0, missing weights), NEDF_ERR_CUDA. */
int nedf_compose_set_types(nedf_handle *h, int n_types, const nedf_type_desc *types);

/* Instances (Section "Manipulating Objects", Eq. 7: each model is a type placed by a rigid
 * transform G(R, T, s)).  `inst` is a host array of n records, copied.  The id of instance i
 * is i.  Errors: NEDF_ERR_ARG for n > max_instances, a type index >= n_types, s <= 0 or any
 * non-finite number (nothing is changed then). */
int nedf_compose_set_instances(nedf_handle *h, int n, const nedf_instance *inst);

/* ---- render -------------------------------------------------------------------------------- */

/* One frame: Steps 1-3 and the composite.  cam and lights are host records (n_lights in
 * 1 .. NEDF_MAX_LIGHTS).  Output buffers are caller-owned DEVICE arrays of width*height
 * elements (rgba and out: 4 floats per pixel); `out` is an addition to the paper's colour,
 * depth and id outputs so that the frame a viewer shows (colour times shadow) needs no extra pass:
 *   depth   float  Step 1 depth buffer: world distance along the unit pixel ray, +inf if empty
 *   id      uint32 Step 1 id buffer: winning instance index, 0xFFFFFFFF if empty
 *   rgba    float4 Step 2 colour buffer (premultiplied RGB, opacity), (0,0,0,0) if empty
 *   shadow  float  Step 3 shadow buffer: mean over lights of (occluded ? beta : 1); 1 if empty
 *   out     float4 composite: (rgba.rgb * shadow, rgba.a)
 * Any of depth / id / rgba / shadow / out may be NULL (the library then keeps its own copy);
 * given buffers are written by the kernels directly and must stay valid until the frame is done.
 * stats (host) may be NULL; when given, the call synchronises and fills it.
 * On a stream other than the legacy default stream the frame (uploads and every kernel) is
 * captured into a CUDA graph on first use and relaunched while the instance count, the light
 * count, depth_source, n_shade, profiling and the output buffers stay the same.
 * Ties in depth go to the lowest instance id (Algorithm 1's strict '<' in id order).
 * Errors: NEDF_ERR_STATE (no types or instances yet), NEDF_ERR_ARG, NEDF_ERR_CUDA, and with
 * stats given NEDF_ERR_CAPACITY when a pair list overflowed. */
int nedf_compose_render(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights,
                        int n_lights, float *depth, uint32_t *id, float *rgba, float *shadow,
                        float *out, nedf_frame_stats *stats);

/* The same frame written to HOST buffers (any may be NULL): the library renders into its own
 * device buffers, copies the requested ones to the host and synchronises. */
int nedf_compose_render_host(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights,
                             int n_lights, float *depth, uint32_t *id, float *rgba, float *shadow,
                             float *out, nedf_frame_stats *stats);

/* ---- buffer reuse while one object is manipulated (Section "CUDA implementation") ----------
 * While the user moves one instance the other objects' work is frozen and their buffers reused.
 * nedf_compose_begin_edit renders the frozen part of the frame — every instance but `inst` — for
 * this camera and these lights into the handle's reuse buffers (packed depth/id keys, colours,
 * per-light occlusion bits; 28 bytes per pixel, allocated on first use).  After the caller moves
 * `inst` (nedf_compose_set_instances with every other record unchanged),
 * nedf_compose_render_edit renders the whole frame from those buffers plus `inst` alone: Step 1
 * for inst's pairs only (z-min against the frozen keys), Step 2 only for the pixels inst wins
 * (every other pixel keeps its frozen colour), Step 3 with full shadow queries for those pixels
 * and, for every other pixel, its frozen occlusion bits plus a test against inst alone.  Its
 * buffers equal nedf_compose_render's for the same scene bit for bit.  Outputs as in
 * nedf_compose_render (caller device buffers, any may be NULL).  nedf_compose_end_edit ends the
 * session (any number of ordinary renders may happen during it).
 * Errors: NEDF_ERR_ARG (inst out of range), NEDF_ERR_STATE (render_edit without a session, or
 * another instance, the instance count or the type set changed), NEDF_ERR_UNSUPPORTED (Step-2
 * outlier resampling on: its re-rendered pixels depend on every object). */
int nedf_compose_begin_edit(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights,
                            int inst);
int nedf_compose_render_edit(nedf_handle *h, float *depth, uint32_t *id, float *rgba, float *shadow,
                             float *out, nedf_frame_stats *stats);
int nedf_compose_end_edit(nedf_handle *h);

/* Plain method colour (the baseline of the paper's speed comparison, Section "Storage and
 * Speed"): every (pixel ray, instance) pair that survives the bound cull is volume rendered
 * with n_samples midpoint samples of its NeRF over the bound chord, pairs composited front to
 * back by entry distance.  rgba: caller-owned device float4[width*height].  With
 * early_stop != 0, a ray stops once its transmittance is below 1e-4 and colour networks are
 * skipped where the sample weight is below 1e-6. */
int nedf_compose_render_march(nedf_handle *h, const nedf_camera *cam, int n_samples,
                              int early_stop, float *rgba);

/* ---- per-stage timing (the per-step breakdown of the paper's Fig. 5) ----------------------- */

#define NEDF_N_STAGES 8
/* Stage i of a frame: 0 setup and clear, 1 Step-1 binning, 2 Step-1 NeDF, 3 Step-1 resolve
 * (z-min to buffers), 4 Step-2 shading, 5 Step-3 binning, 6 Step-3 NeDF, 7 composite. */
const char *nedf_compose_stage_name(int stage);

/* on != 0: every later render records CUDA events between its stages on the handle's stream.
 * Costs a few microseconds per frame; off by default. */
int nedf_compose_set_profiling(nedf_handle *h, int on);

/* Device milliseconds of each stage of the last profiled render (synchronises).  ms is a host
 * array of n >= NEDF_N_STAGES floats.  Errors: NEDF_ERR_STATE when nothing was profiled. */
int nedf_compose_get_stage_times(nedf_handle *h, float *ms, int n);

#define NEDF_N_ENGINE_TIMES 2
/* Device milliseconds of the tensor-core NeDF engine launch alone within the Step-1 and the
 * Step-3 stage of the last profiled render (the stages also hold the output decode and the
 * plain-method pairs): ms[0] Step 1, ms[1] Step 3; 0 where the frame ran no such launch (FP32
 * precision or plain-method depth).  ms is a host array of n >= NEDF_N_ENGINE_TIMES floats;
 * synchronises.  Errors: NEDF_ERR_STATE when nothing was profiled. */
int nedf_compose_get_engine_times(nedf_handle *h, float *ms, int n);

/* ---- checks (debug and tests; none of them faults, traps or hangs the GPU) -----------------------
 * nedf_compose_validate: synchronises, then checks the 256 guard bytes the library places after
 * every buffer it allocated at create (a kernel that wrote past a buffer's end shows here) and the
 * last frame's work lists: per-type pair segments ordered and filled exactly (each type's write
 * cursor ends at its segment's end), tile tables covering each segment at the consuming kernel's
 * tile size, shading lists summing to the hit-pixel count, every deferred pair answered.  Returns
 * NEDF_OK, or NEDF_ERR_STATE naming the first violation.  Skips the list checks when the frame
 * reported an overflow or timeout (those come back through nedf_compose_sync).
 * nedf_compose_inject_status: ORs bits into the device status word (host-side fault injection: the
 * next nedf_compose_sync reports the error and clears the word).  Bits: 1 primary list overflow,
 * 2 shadow list overflow, 4 timeout.
 * nedf_compose_check_wait_limit: launches one kernel whose mbarrier wait can never complete; the
 * wait gives up after its ~1 s limit and sets the timeout status.  Returns NEDF_OK when that timeout
 * was reported (and clears it), so the handle and context remain usable; NEDF_ERR_STATE otherwise. */
int nedf_compose_validate(nedf_handle *h);
int nedf_compose_inject_status(nedf_handle *h, uint32_t bits);
int nedf_compose_check_wait_limit(nedf_handle *h);

/* ---- schedule of the tensor-core MLP kernels and its autotuner ----------------------------------
 * The tensor-core engine streams each type's weights through a fixed shared-memory ring in stages,
 * one bulk copy per stage; the stage size trades copy-issue cost against how far ahead the ring
 * reads.  The NeDF engine at BF16 width 128 can also run its layers with either operand order:
 * swapped (the weight chunk as A, 128 output features x the tile's 256 rows, one MMA per chunk)
 * or unswapped (each 128-row half of the tile as A, the weight chunk as B, two MMAs per chunk).
 * The NeRF kernels at width 256 can also run on SM pairs (operand order 1: clusters of two CTAs
 * whose MMAs span both SMs, M = 256 rows), whose colours differ from the one-SM engine's only by
 * the FP32 order of the output layer's sum.  The stage size and the NeDF operand order change
 * timing, not results.  Kernel index k of the arrays below:
 * 0 Step-2 shading, 1 plain-method colour rows, 2 Step-1 NeDF, 3 Step-3 NeDF, 4 NeDF query. */
#define NEDF_N_SCHEDULE 5
typedef struct {
    int stage_bytes[NEDF_N_SCHEDULE];  /* weight bytes per bulk copy; 0 = default (16384); the
                                          kernel clamps to a whole number of weight chunks and to
                                          at least two stages in its ring                          */
    float tuned_ms[NEDF_N_SCHEDULE];   /* set by nedf_compose_autotune: the chosen schedule's best
                                          time for kernels 0, 2 and 3 (0 elsewhere)                */
    int operand_order[NEDF_N_SCHEDULE];/* NeDF kernels 2-4 at BF16 width 128: 0 = default
                                          (swapped), 1 = swapped, 2 = unswapped; NeRF kernels 0-1
                                          at width 256: 0 = default (one SM), 1 = SM pair, 2 = one
                                          SM; ignored elsewhere                                    */
} nedf_schedule;

/* Replaces the schedule (host struct, copied).  stage_bytes must be 0 or a multiple of 1024 in
 * [1024, 262144], operand_order 0, 1 or 2.  The next render re-captures its CUDA graph.  Errors:
 * NEDF_ERR_ARG. */
int nedf_compose_set_schedule(nedf_handle *h, const nedf_schedule *s);
int nedf_compose_get_schedule(nedf_handle *h, nedf_schedule *s);

/* Autotuner: renders the given frame (into the handle's own buffers) with each candidate stage
 * size (8, 12, 16, 24, 32, 36, 48, 64 KB) for every tensor-core kernel and, at BF16 width 128,
 * each operand order of the NeDF engines, reps timed frames per candidate with stage events, and
 * keeps per kernel the candidate with the smallest time (the plain-method colour rows take the
 * shading kernel's choice, NeDF queries Step 1's).  Synchronises; leaves profiling as it was.
 * chosen (may be NULL) receives the result.  With FP32 precision there is nothing to tune and the
 * schedule is left unchanged.  Errors: those of nedf_compose_render, NEDF_ERR_ARG for reps < 1. */
int nedf_compose_autotune(nedf_handle *h, const nedf_camera *cam, const nedf_light *lights, int n_lights,
                          int reps, nedf_schedule *chosen);

/* ---- kernels in isolation (for tests and tools) ------------------------------------------- */

/* NeDF queries on n arbitrary object-local rays of one type (Eq. 1-2): o, d are device
 * float[n][3] (d need not be unit).  out is device float[n][4] = (m, a, D_local, hit) with
 * D_local = t_perp - rb * m and hit = (a > 0 && D_local > 0); culled rays give (0, 0, +inf, 0). */
int nedf_compose_nedf_query(nedf_handle *h, int type, int n, const float *o, const float *d,
                            float *out);

/* ---- Step 1 without allocations ------------------------------------------------------------ */

/* Depth and id buffers of Step 1 (the same method as nedf_compose_render with default options,
 * in FP32 with its own summation order: depths agree within the render tolerance, ids wherever
 * the two nearest hits are not tied to within that tolerance) for callers that cannot allocate device memory: code embedded in a host whose device memory
 * belongs to that host's own pool, real-time loops that must not block on or fail in an
 * allocation, or phases in which the allocator may not be touched.  No handle is needed and
 * nothing is allocated (no cudaMalloc, cudaFree or allocating library call); the caller passes
 * every input and output, and the call's only scratch is a fixed array inside the library of
 * 512 x 512 packed (depth, id) keys (2 MiB, held on every GPU that loads the library until
 * the process exits).  The paper has no counterpart for this entry point.
 *   width, height    framebuffer size; width * height must not exceed 512 * 512 (NEDF_ERR_ARG)
 *   cam              host camera record
 *   inst_dev         device array of n_inst nedf_instance records (id = index); each record's
 *                    type must be < n_types and its s a positive finite number: the records are
 *                    in device memory where the call cannot check them, so an instance that breaks
 *                    this is skipped (it writes no pixel) rather than reported
 *   rb_host          host array of n_types bound radii
 *   nedf_hidden, nedf_width, nedf_weights_dev
 *                    NeDF shape and device array of n_types packed NeDF weight sets, back to back
 *   depth_dev, id_dev  device outputs of width * height floats / uint32 (as in render)
 *   cuda_stream      stream the work is queued on (asynchronous; NULL = legacy default stream)
 * Every call shares the scratch array and clears the part it uses first; calls whose work
 * overlaps on the GPU (other streams or threads) race on it and must be serialised by the caller.
 * The first successful call on each device looks up the scratch array's device address (with
 * that device current; a failed lookup is retried by the next call); make that first call before
 * any stream capture.  Errors (null pointers,
 * sizes, shapes, a CUDA failure) return a NEDF_ERR_* code; the text is available from
 * nedf_compose_last_error(NULL) on the calling thread. */
int nedf_compose_depth_noalloc(int width, int height, const nedf_camera *cam, int n_inst,
                               const nedf_instance *inst_dev, int n_types, const float *rb_host,
                               int nedf_hidden, int nedf_width, const float *nedf_weights_dev,
                               float *depth_dev, uint32_t *id_dev, void *cuda_stream);

/* ---- learned part -------------------------------------------------------------------------- */

/* Builds the training set of one type on the device: n_rays rays with entry points uniform on
 * the bound sphere and directions cosine-weighted about the inward normal (counter-based
 * SplitMix64 draws 4r .. 4r+3 of `seed` for ray r), labelled by the plain method
 * (march_steps uniform steps, march_bisect bisection steps): hit* and m* = (t_perp - D*) / rb
 * (Eq. 2 inverted, Eq. 5's depth replaced by the half-density crossing).  Optional device
 * outputs (each may be NULL): o, d float[n][3], m_star float[n], hit_star float[n]. */
int nedf_compose_make_labels(nedf_handle *h, int type, int64_t n_rays, uint64_t seed,
                             int march_steps, int march_bisect, float *o, float *d,
                             float *m_star, float *hit_star);

/* The same training set (same rays for the same seed) labelled by a generic radiance field's
 * density network instead of the type's analytic density (Section "Intersection network": the
 * NeDF is supervised with a pre-trained NeRF through Eq. 5; plugin mode).  dens_weights: host,
 * packed W[out][in] then b[out] per layer with dims [63, dens_width x dens_hidden, 1]
 * (dens_hidden 1..8, dens_width 64 or 128); the input is the object-local position encoded with
 * 10 frequencies (identity, sin block, cos block) and sigma = ReLU(output).  Per ray, n_samples
 * (1..1024) midpoints of the chord through the bound give Eq. 5's weights w_i = T_i (1 -
 * exp(-sigma_i delta)); the label depth D is Eq. 5's sum normalised by the opacity A = sum w_i,
 * hit* = A > 0.5 and m* = (t_perp - D) / rb.  FP32 on CUDA cores; synchronous.  Outputs as for
 * nedf_compose_make_labels.  Errors: NEDF_ERR_ARG (range, null, non-finite weight),
 * NEDF_ERR_UNSUPPORTED (network shape), NEDF_ERR_CUDA. */
int nedf_compose_make_labels_density(nedf_handle *h, int type, int64_t n_rays, uint64_t seed,
                                     int n_samples, int dens_hidden, int dens_width,
                                     const float *dens_weights, float *o, float *d, float *m_star,
                                     float *hit_star);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8) of the type's NeDF on `batch`
 * consecutive rays of its training set (wrapping around), starting where the previous step
 * ended.  The random seed of a step is not an argument: the rays and labels are drawn once per
 * training set by nedf_compose_make_labels (its `seed`), and a step is a deterministic function
 * of the training set, the weights and the cursor (so a saved state resumes bit for bit).
 * Loss, NEDF_ARCH_REGRESSION (regression form of Eq. 6): mean over labelled hits of
 * (m - m*)^2 plus 0.1 * mean BCE(a, hit*).  NEDF_ARCH_CLASSIFIER (Eq. 6 itself): mean over
 * labelled hits of BCE(coarse logits, one-hot S_c(m*)) + BCE(fine logits, one-hot S_f(m*)), each
 * the mean over its bins, plus 0.1 * mean BCE(hit logit, hit*); the segment operator S takes
 * u = (m* + 1) 32 to c = floor(u), f = floor((u - c) 128).  Products: FP32 on CUDA cores for an
 * FP32 handle's regression NeDF; otherwise BF16 operands on the tensor cores with FP32 accumulation
 * (activations and error signals rounded to BF16 between products).  FP32 master weights and
 * moments; the rendering copy is refreshed.  loss_host (host float, may be NULL)
 * receives the loss of this batch; giving it synchronises.  Errors: NEDF_ERR_STATE (no training
 * set for the type), NEDF_ERR_ARG, NEDF_ERR_CUDA. */
int nedf_compose_train_step(nedf_handle *h, int type, int batch, float lr, float *loss_host);

/* Loss and gradient of the type's current NeDF weights on n caller rays / labels (all device:
 * o, d float[n][3], m_star, hit_star float[n]); grad is device float[n_params] in the packed
 * layout.  loss_host may be NULL.  Synchronises. */
int nedf_compose_loss_grad(nedf_handle *h, int type, int n, const float *o, const float *d,
                           const float *m_star, const float *hit_star, float *grad,
                           float *loss_host);

/* Copies the type's current FP32 NeDF weights (packed layout) to host memory. */
int nedf_compose_get_nedf_weights(nedf_handle *h, int type, float *host_out, int64_t n_floats);

/* Training state of every type (weights, Adam moments, step count, position in the training set)
 * as one little-endian blob: header {magic, version 2, n_types, n_params} (int64 each), then per
 * type int32 step, int64 batch cursor, FP32 master weights, Adam m, Adam v.  Training steps are
 * deterministic (gradient splits summed in a fixed order), so a run resumed from a saved state
 * repeats the uninterrupted run bit for bit on the same GPU.
 * save: with buf == NULL only *size is set; otherwise *size is the capacity in bytes.
 * load: the blob must come from a handle with the same config and types. */
int nedf_compose_save_state(nedf_handle *h, void *buf, size_t *size);
int nedf_compose_load_state(nedf_handle *h, const void *buf, size_t size);

#ifdef __cplusplus
}
#endif
#endif /* NEDF_COMPOSE_H */
