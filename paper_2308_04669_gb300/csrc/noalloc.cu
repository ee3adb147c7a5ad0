// Step 1 (NeDF generation: depth and id buffers) for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: a renderer embedded in a host application whose
// device memory is owned by that application's own pool, a real-time loop that must not block
// on or fail in an allocation mid-frame, or code that runs while the host is forbidden from
// touching the allocator.  For them, nedf_compose_depth_noalloc runs the same Step-1 method as
// the handle-based renderer (ray transform, bound cull, NeDF MLP, strict-'<' z-min; FP32, with its
// own loop order, so results agree within the render tolerance) with only
// caller-owned inputs and outputs and one fixed scratch array that lives in this file:
// the packed (depth, id) keys of at most kNoAllocMaxPixels pixels.
//
// The scratch array belongs to every GPU that loads the library, for the life of the process,
// and every call shares it: calls whose work overlaps on the GPU (two streams, or two threads)
// race on it.  Each call clears the part it uses before writing.
//
// The first successful call on a device looks up the device address of the array
// (cudaGetSymbolAddress, with that device current); make that first call before any stream
// capture.
// The paper has no counterpart for this entry point.
#include <mutex>
#include <string>

#include "../../include/nedf_compose.h"
#include "mlp_f32.cuh"

namespace nedf {

constexpr int kNoAllocMaxPixels = 512 * 512;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned long long g_noalloc_keys[kNoAllocMaxPixels];

// Device address of g_noalloc_keys per device, looked up on the first call that succeeds; a
// failed lookup is not remembered, so a later call (for example once a context is current)
// tries again.
static unsigned long long *g_keys_dev[kNoAllocMaxDevices];
static std::mutex g_keys_mutex;
void set_thread_error(const std::string &msg);   // api.cu

struct NoAllocParams {
    DevFrame f;                  // camera basis filled in by each block
    HostCamera cam;
    const nedf_instance *inst;
    const float *w;              // packed NeDF weights, n_types x n_params
    long long n_params;
    int n_types;                 // instances with type >= n_types are skipped (never read)
    float rb[kMaxTypes];
    int hidden, width;
    unsigned long long *keys;
    float *depth;
    uint32_t *id;
};

__global__ void k_na_clear(unsigned long long *keys, int npix)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) keys[p] = ~0ull;
}

__device__ __forceinline__ void na_camera(const HostCamera &c, DevFrame &f)
{
    V3 eye = v3(c.eye[0], c.eye[1], c.eye[2]);
    V3 fwd = normalized(sub(v3(c.target[0], c.target[1], c.target[2]), eye));
    V3 right = normalized(v3(-fwd.z, 0.0f, fwd.x));
    V3 up = v3(right.y * fwd.z - right.z * fwd.y, right.z * fwd.x - right.x * fwd.z, right.x * fwd.y - right.y * fwd.x);
    f.eye[0] = eye.x; f.eye[1] = eye.y; f.eye[2] = eye.z;
    f.fwd[0] = fwd.x; f.fwd[1] = fwd.y; f.fwd[2] = fwd.z;
    f.right[0] = right.x; f.right[1] = right.y; f.right[2] = right.z;
    f.up[0] = up.x; f.up[1] = up.y; f.up[2] = up.z;
    f.tan_h = tanf(0.5f * c.fov_y_deg * 0.017453292519943295f);
    f.aspect = (float)f.W / (float)f.H;
}

// Y = act(X W^T + b) with W in the ABI's packed layout W[out][in]; X feature-major in shared memory.
template <int N>
__device__ __forceinline__ void dense_packed(float *X, int K, const float *__restrict__ W, const float *__restrict__ b,
                                             bool relu)
{
    constexpr int NC = N / 16;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float acc[4][NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        float bj = __ldg(b + tx + 16 * j);
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i][j] = bj;
    }
    const float *xp = X + ty * 4;
    for (int k = 0; k < K; ++k) {
        float4 xv = *reinterpret_cast<const float4 *>(xp + k * kXStride);
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            float w = __ldg(W + (size_t)(tx + 16 * j) * K + k);
            acc[0][j] = fmaf(xv.x, w, acc[0][j]);
            acc[1][j] = fmaf(xv.y, w, acc[1][j]);
            acc[2][j] = fmaf(xv.z, w, acc[2][j]);
            acc[3][j] = fmaf(xv.w, w, acc[3][j]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NC; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            X[(tx + 16 * j) * kXStride + ty * 4 + i] = relu ? fmaxf(acc[i][j], 0.0f) : acc[i][j];
    __syncthreads();
}

// One block per instance: the pixels of its screen rectangle are culled, the survivors are
// packed into 64-row tiles in shared memory, each tile runs the NeDF, and hits go into the
// packed (depth, id) keys with an atomic minimum.
struct NaTile {
    float x6[kTileRows][6];
    float tp[kTileRows];
    uint32_t pix[kTileRows];
    float y[kTileRows][4];
    int fill;
};

template <int N>
__device__ void na_run_tile(float *X, NaTile &T, int n, const float *w, int hidden, float rb, float s, int inst,
                            unsigned long long *keys)
{
    for (int e = threadIdx.x; e < kTileRows * kNedfIn; e += blockDim.x) {
        int r = e % kTileRows, fi = e / kTileRows;
        X[fi * kXStride + r] = r < n ? posenc_feature(T.x6[r], 6, 6, fi) : 0.0f;
    }
    __syncthreads();
    const float *wp = w;
    int K = kNedfIn;
    for (int l = 0; l < hidden; ++l) {
        dense_packed<N>(X, K, wp, wp + (size_t)N * K, true);
        wp += (size_t)N * K + N;
        K = N;
    }
    for (int e = threadIdx.x; e < kTileRows * 2; e += blockDim.x) {
        int r = e >> 1, o = e & 1;
        float acc = __ldg(wp + 2 * N + o);
        for (int k = 0; k < N; ++k) acc = fmaf(X[k * kXStride + r], __ldg(wp + o * N + k), acc);
        T.y[r][o] = acc;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        float Dl = T.tp[threadIdx.x] - rb * T.y[threadIdx.x][0];
        if (T.y[threadIdx.x][1] > 0.0f && Dl > 0.0f) {
            float D = s * Dl;
            atomicMin(&keys[T.pix[threadIdx.x]], ((unsigned long long)__float_as_uint(D) << 32) | (uint32_t)inst);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) T.fill = 0;
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(kThreads) k_na_step1(NoAllocParams P)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ DevFrame f;
    __shared__ NaTile T;
    const int inst = blockIdx.x;
    if (threadIdx.x == 0) {
        f = P.f;
        na_camera(P.cam, f);
        T.fill = 0;
    }
    __syncthreads();
    const nedf_instance src = P.inst[inst];
    // The records live in device memory, so the host cannot check them; an instance of an unknown
    // type or with a scale that is not a positive finite number is skipped (the test is uniform over the block, which returns as a whole).
    if (src.type >= (uint32_t)P.n_types || !(src.s > 0.0f) || !isfinite(src.s)) return;
    DevInst I;
    for (int c = 0; c < 9; ++c) I.R[c] = src.R[c];
    for (int c = 0; c < 3; ++c) I.T[c] = src.T[c];
    I.s = src.s;
    I.type = src.type;
    const float rb = P.rb[src.type];
    const float *w = P.w + (size_t)src.type * P.n_params;
    // conservative screen rectangle of the bound sphere (tangent planes through the eye)
    int i0 = 0, i1 = f.W - 1, j0 = 0, j1 = f.H - 1;
    {
        V3 e = sub(v3(I.T[0], I.T[1], I.T[2]), v3(f.eye[0], f.eye[1], f.eye[2]));
        float r = rb * I.s;
        float cx = dot(e, v3(f.right[0], f.right[1], f.right[2]));
        float cy = dot(e, v3(f.up[0], f.up[1], f.up[2]));
        float cz = dot(e, v3(f.fwd[0], f.fwd[1], f.fwd[2]));
        if (cz > r * 1.001f + 1e-6f) {
            float den = cz * cz - r * r;
            float sx = r * sqrtf(fmaxf(cx * cx + cz * cz - r * r, 0.f));
            float sy = r * sqrtf(fmaxf(cy * cy + cz * cz - r * r, 0.f));
            float su = f.W * 0.5f / (f.tan_h * f.aspect), sv = f.H * 0.5f / f.tan_h;
            float fi0 = (cx * cz - sx) / den * su + f.W * 0.5f - 0.5f, fi1 = (cx * cz + sx) / den * su + f.W * 0.5f - 0.5f;
            float fj0 = -(cy * cz + sy) / den * sv + f.H * 0.5f - 0.5f, fj1 = -(cy * cz - sy) / den * sv + f.H * 0.5f - 0.5f;
            if (!(fi1 >= -2.f && fi0 <= f.W + 1.f && fj1 >= -2.f && fj0 <= f.H + 1.f)) return;   // whole block
            i0 = max(0, (int)floorf(fi0) - 2); i1 = min(f.W - 1, (int)ceilf(fi1) + 2);
            j0 = max(0, (int)floorf(fj0) - 2); j1 = min(f.H - 1, (int)ceilf(fj1) + 2);
        }
    }
    const int bw = i1 - i0 + 1, npx = bw * (j1 - j0 + 1);
    for (int base = 0; base < npx; base += blockDim.x) {
        const int p = base + threadIdx.x;
        bool keep = false;
        V3 ol = v3(0, 0, 0), dl = v3(0, 0, 1);
        Chord ch{};
        int i = 0, j = 0;
        if (p < npx) {
            i = i0 + p % bw;
            j = j0 + p / bw;
            V3 o, d;
            camera_ray(f, i, j, o, d);
            to_local(I, o, d, ol, dl);
            keep = bound_chord(ol, dl, rb, ch);
        }
        // compaction: every round places survivors into free rows; a full tile is run at once
        while (__syncthreads_or(keep)) {
            if (keep) {
                int slot = atomicAdd(&T.fill, 1);
                if (slot < kTileRows) {
                    V3 pe = madd(ol, ch.te, dl);
                    T.x6[slot][0] = pe.x; T.x6[slot][1] = pe.y; T.x6[slot][2] = pe.z;
                    T.x6[slot][3] = dl.x; T.x6[slot][4] = dl.y; T.x6[slot][5] = dl.z;
                    T.tp[slot] = ch.tp;
                    T.pix[slot] = (uint32_t)(j * f.W + i);
                    keep = false;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0 && T.fill > kTileRows) T.fill = kTileRows;   // claims past a full tile
            __syncthreads();
            if (T.fill == kTileRows) na_run_tile<N>(X, T, kTileRows, w, P.hidden, rb, I.s, inst, P.keys);
        }
    }
    __syncthreads();
    const int n = T.fill;
    if (n > 0) na_run_tile<N>(X, T, n, w, P.hidden, rb, I.s, inst, P.keys);
}

__global__ void k_na_resolve(const unsigned long long *keys, float *depth, uint32_t *id, int npix)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        unsigned long long k = keys[p];
        depth[p] = k == ~0ull ? __int_as_float(0x7f800000) : __uint_as_float((uint32_t)(k >> 32));
        id[p] = k == ~0ull ? kNoId : (uint32_t)(k & 0xffffffffu);
    }
}

template <int N>
static cudaError_t launch_na(const NoAllocParams &P, int n_inst, int npix, cudaStream_t st)
{
    size_t sm = (size_t)(N > kNedfInPad ? N : kNedfInPad) * kXStride * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_na_step1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_na_clear<<<64, 256, 0, st>>>(P.keys, npix);
    k_na_step1<N><<<n_inst, kThreads, sm, st>>>(P);
    k_na_resolve<<<64, 256, 0, st>>>(P.keys, P.depth, P.id, npix);
    return cudaGetLastError();
}

}  // namespace nedf

using namespace nedf;

extern "C" int nedf_compose_depth_noalloc(int width, int height, const nedf_camera *cam, int n_inst,
                                          const nedf_instance *inst_dev, int n_types, const float *rb_host,
                                          int nedf_hidden, int nedf_width, const float *nedf_weights_dev,
                                          float *depth_dev, uint32_t *id_dev, void *cuda_stream)
{
    auto fail = [](int code, const char *msg) {
        set_thread_error(msg);
        return code;
    };
    if (!cam || !inst_dev || !rb_host || !nedf_weights_dev || !depth_dev || !id_dev)
        return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: null argument");
    if (width < 1 || height < 1 || (long long)width * height > kNoAllocMaxPixels)
        return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: width * height must be 1 .. 262144 (512 x 512), "
                                  "the size of its built-in scratch");
    if (n_inst < 1 || n_inst > (1 << 20)) return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: n_inst 1 .. 2^20");
    if (n_types < 1 || n_types > kMaxTypes) return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: n_types 1 .. 64");
    if (nedf_hidden < 1 || nedf_hidden > 16 || (nedf_width != 64 && nedf_width != 128 && nedf_width != 256))
        return fail(NEDF_ERR_UNSUPPORTED, "nedf_compose_depth_noalloc: hidden 1 .. 16, width 64 / 128 / 256");
    if (!(cam->fov_y_deg > 0.f && cam->fov_y_deg < 180.f))
        return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: fov_y_deg must be in (0, 180)");
    for (int t = 0; t < n_types; ++t)
        if (!(rb_host[t] > 0.f)) return fail(NEDF_ERR_ARG, "nedf_compose_depth_noalloc: rb must be > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
        return fail(NEDF_ERR_CUDA, "nedf_compose_depth_noalloc: cudaGetDevice failed");
    // once per device, with that device current: the device address of the scratch array
    unsigned long long *keys = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_keys_mutex);
        if (!g_keys_dev[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_keys);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                return fail(NEDF_ERR_CUDA, "nedf_compose_depth_noalloc: cudaGetSymbolAddress of the scratch array failed");
            }
            g_keys_dev[dev] = static_cast<unsigned long long *>(p);
        }
        keys = g_keys_dev[dev];
    }
    NoAllocParams P{};
    P.f.W = width;
    P.f.H = height;
    for (int c = 0; c < 3; ++c) {
        P.cam.eye[c] = cam->eye[c];
        P.cam.target[c] = cam->target[c];
    }
    P.cam.fov_y_deg = cam->fov_y_deg;
    P.inst = inst_dev;
    P.w = nedf_weights_dev;
    P.n_params = (long long)kNedfIn * nedf_width + nedf_width +
                 (long long)(nedf_hidden - 1) * ((long long)nedf_width * nedf_width + nedf_width) +
                 (long long)nedf_width * 2 + 2;
    P.n_types = n_types;
    for (int t = 0; t < n_types; ++t) P.rb[t] = rb_host[t];
    P.hidden = nedf_hidden;
    P.width = nedf_width;
    P.keys = keys;
    P.depth = depth_dev;
    P.id = id_dev;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int npix = width * height;
    switch (nedf_width) {
    case 64: e = launch_na<64>(P, n_inst, npix, st); break;
    case 128: e = launch_na<128>(P, n_inst, npix, st); break;
    default: e = launch_na<256>(P, n_inst, npix, st); break;
    }
    if (e != cudaSuccess) return fail(NEDF_ERR_CUDA, cudaGetErrorString(e));
    return NEDF_OK;
}
