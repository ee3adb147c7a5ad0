// Plain method colour frame: every (pixel ray, instance) pair that survives the bound cull is
// volume rendered with n midpoint samples of its radiance field over the bound chord, and the
// pairs of a pixel are composited front to back by entry distance.  This is the naive
// composition the paper measures its speed-up against (Section "Storage and Speed", Table 1's
// base column, Table 2's ground truth) with the analytic density of the workloads.
//
// Work layout: pairs come from the Step-1 binning lists.  A pass over pairs evaluates the
// densities of their samples and reserves a contiguous run of "sample rows" per pair (all n in
// the dense variant; in the early-stop variant only the run whose weight T*alpha reaches 1e-6,
// stopping once T < 1e-4).  Colour-network tiles then run over sample rows grouped by type and
// reduce each pair's weighted colour; a last pass composites the pairs of every pixel.
#include "mlp_f32.cuh"
#include "render_launch.h"

namespace nedf {

constexpr float kEsWeight = 1e-6f;
constexpr float kEsTransmittance = 1e-4f;

__device__ __forceinline__ void pair_ray(const DevFrame &f, const DevInst &I, uint32_t pix, V3 &ol, V3 &dl)
{
    V3 o, d;
    camera_ray(f, pix % f.W, pix / f.W, o, d);
    to_local(I, o, d, ol, dl);
}

__global__ void k_march_clear(Workspace ws, MarchBuffers mb, int npix, int n_samples)
{
    const DevFrame &f = *ws.frame;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) mb.head[p] = -1;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long o = 0;
        for (int t = 0; t < f.n_types; ++t) {
            mb.row_off[t] = o;
            mb.row_cursor[t] = o;
            o += ws.cnt->p_count[t] * (unsigned long long)n_samples;   // at most n rows per pair
        }
        mb.row_off[f.n_types] = o;
    }
}

template <bool ES>
__global__ void k_march_pairs(Workspace ws, MarchBuffers mb, int n_samples)
{
    const DevFrame &f = *ws.frame;
    const unsigned long long n_pairs = ws.cnt->p_off[f.n_types];
    for (unsigned long long q = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; q < n_pairs;
         q += (unsigned long long)gridDim.x * blockDim.x) {
        uint2 pr = ws.ppairs[q];
        DevInst I = ws.inst[pr.y];
        DevType T = ws.types[I.type];
        V3 ol, dl;
        pair_ray(f, I, pr.x, ol, dl);
        Chord ch;
        bound_chord(ol, dl, T.rb, ch);
        float dt = (ch.tx - ch.te) / n_samples;
        float Tr = 1.0f, T_first = 1.0f, wsum = 0.0f;
        int k_first = -1, k_last = -1;
        for (int k = 0; k < n_samples; ++k) {
            float tk = ch.te + (k + 0.5f) * dt;
            float sig = density(T, madd(ol, tk, dl), f.sigma_max, f.sdf_width);
            float alpha = 1.0f - expf(-sig * I.s * dt);
            float w = Tr * alpha;
            if (!ES || w >= kEsWeight) {
                if (k_first < 0) { k_first = k; T_first = Tr; }
                k_last = k;
                wsum += w;
            }
            Tr *= 1.0f - alpha;
            if (ES && Tr < kEsTransmittance) break;
        }
        int count = k_first < 0 ? 0 : k_last - k_first + 1;
        mb.te_world[q] = ch.te * I.s;
        mb.T_pair[q] = Tr;
        mb.T_first[q] = T_first;
        mb.k_first[q] = k_first;
        if (T.nerf) {
            mb.C[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (count > 0) {
                unsigned long long pos = atomicAdd(&mb.row_cursor[I.type], (unsigned long long)count);
                if (pos + count <= mb.row_off[I.type + 1])
                    for (int i = 0; i < count; ++i) mb.rows[pos + i] = make_uint2((uint32_t)q, (uint32_t)(k_first + i));
                else
                    atomicOr(ws.status, kStatusPrimaryOverflow);
            }
        } else {
            mb.C[q] = make_float4(wsum * T.albedo[0], wsum * T.albedo[1], wsum * T.albedo[2], 0.f);
        }
        mb.next[q] = atomicExch(&mb.head[pr.x], (int)q);
    }
}

__global__ void k_march_scan(Workspace ws, MarchBuffers mb, int rows_per_tile)
{
    const DevFrame &f = *ws.frame;
    unsigned long long t = 0;
    for (int k = 0; k < f.n_types; ++k) {
        mb.row_tile[k] = t;
        unsigned long long rows = min(mb.row_cursor[k], mb.row_off[k + 1]) - mb.row_off[k];
        t += (rows + rows_per_tile - 1) / rows_per_tile;
    }
    mb.row_tile[f.n_types] = t;
}

template <int W_NERF>
__global__ void __launch_bounds__(kThreads) k_march_colour(Workspace ws, MarchBuffers mb, int n_samples)
{
    extern __shared__ float4 smem4[];
    float *X = reinterpret_cast<float *>(smem4);
    __shared__ float xs[kTileRows][6];
    __shared__ float wrow[kTileRows];
    __shared__ uint32_t prow[kTileRows];
    __shared__ float y[kTileRows][4];
    const DevFrame &f = *ws.frame;
    const int n_types = f.n_types;
    const unsigned long long n_tiles = mb.row_tile[n_types];
    for (unsigned long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        int t = 0;
        while (t + 1 < n_types && mb.row_tile[t + 1] <= tile) ++t;
        unsigned long long end = min(mb.row_cursor[t], mb.row_off[t + 1]);
        unsigned long long r0 = mb.row_off[t] + (tile - mb.row_tile[t]) * kTileRows;
        const DevType T = ws.types[t];
        if (threadIdx.x < kTileRows) {
            int r = threadIdx.x;
            for (int c = 0; c < 6; ++c) xs[r][c] = 0.0f;
            wrow[r] = 0.0f;
            prow[r] = 0xFFFFFFFFu;
            if (r0 + r < end) {
                uint2 row = mb.rows[r0 + r];
                uint2 pr = ws.ppairs[row.x];
                DevInst I = ws.inst[pr.y];
                V3 ol, dl;
                pair_ray(f, I, pr.x, ol, dl);
                Chord ch;
                bound_chord(ol, dl, T.rb, ch);
                float dt = (ch.tx - ch.te) / n_samples;
                // transmittance at sample k from the pair's first row
                float Tr = mb.T_first[row.x];
                for (int j = mb.k_first[row.x]; j < (int)row.y; ++j) {
                    float sj = density(T, madd(ol, ch.te + (j + 0.5f) * dt, dl), f.sigma_max, f.sdf_width);
                    Tr *= expf(-sj * I.s * dt);
                }
                float tk = ch.te + (row.y + 0.5f) * dt;
                V3 x = madd(ol, tk, dl);
                float sig = density(T, x, f.sigma_max, f.sdf_width);
                wrow[r] = Tr * (1.0f - expf(-sig * I.s * dt));
                prow[r] = row.x;
                xs[r][0] = x.x; xs[r][1] = x.y; xs[r][2] = x.z;
                xs[r][3] = dl.x; xs[r][4] = dl.y; xs[r][5] = dl.z;
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRows * kNerfIn; e += blockDim.x) {
            int r = e % kTileRows, fi = e / kTileRows;
            X[fi * kXStride + r] = fi < 63 ? posenc_feature(&xs[r][0], 3, 10, fi) : posenc_feature(&xs[r][3], 3, 4, fi - 63);
        }
        __syncthreads();
        const float *w = ws.nerf_w + (size_t)t * ws.nerf_stride;
        mlp_hidden_f32<W_NERF>(X, kNerfIn, ws.nerf_hidden, w);
        const float *wo = w + (size_t)kNerfIn * W_NERF + W_NERF + (size_t)(ws.nerf_hidden - 1) * (W_NERF * W_NERF + W_NERF);
        out_layer_f32(X, W_NERF, wo, wo + W_NERF * 3, 3, y);
        // weighted colour per row, then one reduction per run of rows of the same pair
        if (threadIdx.x < kTileRows) {
            int r = threadIdx.x;
            float wr = wrow[r];
            y[r][0] = wr / (1.0f + expf(-y[r][0]));
            y[r][1] = wr / (1.0f + expf(-y[r][1]));
            y[r][2] = wr / (1.0f + expf(-y[r][2]));
        }
        __syncthreads();
        if (threadIdx.x < kTileRows) {
            int r = threadIdx.x;
            uint32_t p = prow[r];
            if (p != 0xFFFFFFFFu && (r == 0 || prow[r - 1] != p)) {
                float a = 0.f, b = 0.f, c = 0.f;
                for (int s = r; s < kTileRows && prow[s] == p; ++s) { a += y[s][0]; b += y[s][1]; c += y[s][2]; }
                atomicAdd(&mb.C[p].x, a);
                atomicAdd(&mb.C[p].y, b);
                atomicAdd(&mb.C[p].z, c);
            }
        }
        __syncthreads();
    }
}

// Front-to-back over the pixel's pairs in (entry distance, instance id) order.  LISTED: only the
// pixels that have pairs in the list are written (Step-2 resampling runs on a subset).
template <bool LISTED>
__global__ void k_march_composite(Workspace ws, MarchBuffers mb, float4 *rgba, int npix)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
        if (LISTED && mb.head[p] < 0) continue;
        float Tr = 1.0f, r = 0.f, g = 0.f, b = 0.f;
        float last_te = -1.0f;
        uint32_t last_id = 0;
        bool first = true;
        int n = 0;
        for (int q = mb.head[p]; q >= 0; q = mb.next[q]) ++n;
        for (int it = 0; it < n; ++it) {
            int best = -1;
            float bte = 0.f;
            uint32_t bid = 0;
            for (int q = mb.head[p]; q >= 0; q = mb.next[q]) {
                float te = mb.te_world[q];
                uint32_t id = ws.ppairs[q].y;
                bool after = first || te > last_te || (te == last_te && id > last_id);
                if (!after) continue;
                if (best < 0 || te < bte || (te == bte && id < bid)) { best = q; bte = te; bid = id; }
            }
            if (best < 0) break;
            float4 c = mb.C[best];
            r += Tr * c.x; g += Tr * c.y; b += Tr * c.z;
            Tr *= mb.T_pair[best];
            last_te = bte; last_id = bid; first = false;
        }
        rgba[p] = make_float4(r, g, b, 1.0f - Tr);
    }
}

size_t march_bytes(int npix, long long pairs, int n_samples)
{
    return (size_t)npix * 4 + (size_t)pairs * (4 + 4 + 4 + 4 + 4 + 16) + (size_t)pairs * n_samples * 8 +
           3 * (kMaxTypes + 1) * 8 + 1024;
}

static MarchBuffers carve_march(void *base, int npix, long long pairs, int n_samples)
{
    MarchBuffers mb{};
    char *p = (char *)base;
    auto take = [&](size_t bytes) { char *q = p; p += (bytes + 255) & ~(size_t)255; return (void *)q; };
    mb.C = (float4 *)take((size_t)pairs * 16);
    mb.rows = (uint2 *)take((size_t)pairs * n_samples * 8);
    mb.head = (int *)take((size_t)npix * 4);
    mb.next = (int *)take((size_t)pairs * 4);
    mb.te_world = (float *)take((size_t)pairs * 4);
    mb.T_pair = (float *)take((size_t)pairs * 4);
    mb.T_first = (float *)take((size_t)pairs * 4);
    mb.k_first = (int *)take((size_t)pairs * 4);
    mb.row_cursor = (unsigned long long *)take((kMaxTypes + 1) * 8);
    mb.row_off = (unsigned long long *)take((kMaxTypes + 1) * 8);
    mb.row_tile = (unsigned long long *)take((kMaxTypes + 1) * 8);
    mb.row_cap = pairs * n_samples;
    return mb;
}

template <int W>
static cudaError_t launch_colour(const Workspace &ws, const MarchBuffers &mb, int n_samples, int grid, cudaStream_t st)
{
    size_t sm = (size_t)(W > kNerfInPad ? W : kNerfInPad) * kXStride * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_march_colour<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_march_colour<W><<<grid, kThreads, sm, st>>>(ws, mb, n_samples);
    return cudaGetLastError();
}

cudaError_t launch_march_colour_frame(const FrameLaunch &L, void *scratch, long long pairs_cap, int n_samples,
                                      int early_stop, float4 *rgba)
{
    const Workspace &ws = L.ws;
    cudaStream_t st = L.stream;
    int npix = L.W * L.H;
    int g = L.num_sms * 4;
    MarchBuffers mb = carve_march(scratch, npix, pairs_cap, n_samples);
    k_march_clear<<<g, 256, 0, st>>>(ws, mb, npix, n_samples);
    if (early_stop) k_march_pairs<true><<<g * 2, 128, 0, st>>>(ws, mb, n_samples);
    else k_march_pairs<false><<<g * 2, 128, 0, st>>>(ws, mb, n_samples);
    const bool tc = ws.precision >= 1 && ws.nerf_hidden > 0;
    k_march_scan<<<1, 1, 0, st>>>(ws, mb, tc ? kPipeTileRows : kTileRows);
    cudaError_t e = cudaSuccess;
    if (tc) {
        e = launch_march_colour_pipe(ws, mb, n_samples, L.num_sms, st);
        if (e != cudaSuccess) return e;
    } else if (ws.nerf_hidden > 0) {
        switch (ws.nerf_width) {
        case 64: e = launch_colour<64>(ws, mb, n_samples, g, st); break;
        case 128: e = launch_colour<128>(ws, mb, n_samples, g, st); break;
        case 256: e = launch_colour<256>(ws, mb, n_samples, g, st); break;
        default: e = cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    k_march_composite<false><<<g, 256, 0, st>>>(ws, mb, rgba, npix);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Step-2 outlier resampling ("rs", Section "Deferred Shading"): the primary pairs of every pixel
// the shading flagged (an extremely small density around its depth) become a pair list of their
// own, with its own counters, and the kernels above render exactly those pixels by the plain
// method (dense, n samples per pair, front to back) into the colour buffer.
// ---------------------------------------------------------------------------------------------
__global__ void k_rs_collect(Workspace ws)
{
    const DevFrame &f = *ws.frame;
    const unsigned long long n = ws.cnt->p_off[f.n_types];
    const int lane = threadIdx.x & 31;
    // the trip count is uniform within a block, so the ballots below see whole warps
    for (unsigned long long base = blockIdx.x * (unsigned long long)blockDim.x; base < n;
         base += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long q = base + threadIdx.x;
        bool keep = false;
        uint2 pp = make_uint2(0u, 0u);
        uint32_t ty = 0;
        if (q < n) {
            pp = ws.ppairs[q];
            keep = ws.rs_mask[pp.x] != 0u;
            if (keep) ty = ws.inst[pp.y].type;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (!m) continue;
        unsigned long long start = 0;
        if (lane == __ffs(m) - 1) start = atomicAdd(&ws.rs_cnt->p_cursor[0], (unsigned long long)__popc(m));
        start = __shfl_sync(0xffffffffu, start, __ffs(m) - 1);
        if (keep) {
            const unsigned long long idx = start + __popc(m & ((1u << lane) - 1u));
            const bool fits = idx < (unsigned long long)ws.rs_cap;
            if (fits) ws.rs_pairs[idx] = pp;
            else atomicOr(ws.status, kStatusResampleOverflow);
            // per-type counts of the kept pairs (they size the plain method's sample rows)
            const unsigned kept = __ballot_sync(m, fits);
            if (fits) {
                const unsigned peers = __match_any_sync(kept, ty);
                if (lane == __ffs(peers) - 1) atomicAdd(&ws.rs_cnt->p_count[ty], (unsigned long long)__popc(peers));
            }
        }
    }
}

__global__ void k_rs_close(Workspace ws)
{
    const DevFrame &f = *ws.frame;
    Counters &C = *ws.rs_cnt;
    unsigned long long o = 0;
    for (int t = 0; t < f.n_types; ++t) {
        C.p_off[t] = o;
        o += C.p_count[t];
    }
    C.p_off[f.n_types] = o;                  // = min(collected, capacity)
}

cudaError_t launch_shade_resample(const FrameLaunch &L)
{
    const Workspace &ws = L.ws;
    cudaStream_t st = L.stream;
    const int npix = L.W * L.H, g = L.num_sms * 4, n = L.shade_resample;
    k_rs_collect<<<g * 2, 256, 0, st>>>(ws);
    k_rs_close<<<1, 1, 0, st>>>(ws);
    Workspace wr = ws;                       // the same frame, the resampling list as its pairs
    wr.ppairs = ws.rs_pairs;
    wr.pcap = ws.rs_cap;
    wr.cnt = ws.rs_cnt;
    MarchBuffers mb = carve_march(ws.rs_scratch, npix, ws.rs_cap, n);
    k_march_clear<<<g, 256, 0, st>>>(wr, mb, npix, n);
    k_march_pairs<false><<<g * 2, 128, 0, st>>>(wr, mb, n);
    const bool tc = ws.precision >= 1 && ws.nerf_hidden > 0;
    k_march_scan<<<1, 1, 0, st>>>(wr, mb, tc ? kPipeTileRows : kTileRows);
    cudaError_t e = cudaSuccess;
    if (tc) {
        e = launch_march_colour_pipe(wr, mb, n, L.num_sms, st);
    } else if (ws.nerf_hidden > 0) {
        switch (ws.nerf_width) {
        case 64: e = launch_colour<64>(wr, mb, n, g, st); break;
        case 128: e = launch_colour<128>(wr, mb, n, g, st); break;
        case 256: e = launch_colour<256>(wr, mb, n, g, st); break;
        default: e = cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess) return e;
    k_march_composite<true><<<g, 256, 0, st>>>(wr, mb, ws.rgba, npix);
    return cudaGetLastError();
}

}  // namespace nedf
