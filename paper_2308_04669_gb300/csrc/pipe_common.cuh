// Pieces shared by the tensor-core engines (render_pipe.cu: the NeRF and regression-NeDF engines;
// render_cls.cu: the classifier intersection network): tile geometry, the A-operand layout, the
// kernel arguments, the bounded waits and the row look-ups of listed pairs.
#pragma once

#include "render_kernels.cuh"
#include "tc_ptx.cuh"

namespace nedf {

using namespace tc;

constexpr int kPipeRows = 256;              // rows per tile (two MMA halves of 128)
constexpr int kHalf = 128;
constexpr int kPipeThreads = 320;           // 8 epilogue warps, producer, MMA issuer
constexpr int kPipeThreadsPf = 384;         // the NeRF engine: + 2 warps preparing the next tile's rows
constexpr int kKC = 16;                     // K columns per weight chunk (one MMA K step)
// A bulk copy costs its issuing thread a few hundred cycles whatever its size, so weights move in
// stages of several chunks (one copy, one full and one empty barrier phase each).  The stage size
// is a run-time schedule parameter, the autotuner's; a shape's ring bytes are fixed.
constexpr int kDefaultStageBytes = 16384;

enum PipeMode { kModeShade = 0, kModeMarch = 1, kModePrimary = 2, kModeShadow = 3, kModeQuery = 4 };

// A operand of one 128-row half, K-major without swizzle, with the 8-row groups of one 8-column
// slice adjacent: element (r, k) at (k / 8) * 2048 + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
// (leading byte offset 2048 to the next 8 columns, stride byte offset 128 to the next 8 rows), so
// the 4 KB one MMA K step reads are contiguous.
__device__ __forceinline__ uint32_t a_offset(int r, int k)
{
    return (uint32_t)((k >> 3) * 2048 + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct PipeArgs {
    int stage_bytes;              // schedule: weight bytes per bulk copy
    const uint8_t *blobs;
    size_t blob_stride;
    int npix;
    int n_samples;
    int query_type;
    const float *qo, *qd;
    float4 *qout;
    int qn;
};

// Position in a ring of S weight stages: the stage and the parity of its current fill, kept by
// increments (a 64-bit division by the run-time S would cost the issuing thread hundreds of cycles
// per stage).
struct RingPos {
    int st = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int S)
    {
        if (++st == S) {
            st = 0;
            ph ^= 1u;
        }
    }
};

struct PipeShared {
    uint64_t a_ready, acc_full, fin;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ bool pipe_wait(uint64_t *bar, uint32_t parity, volatile int *abort, uint32_t *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    while (!*abort) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > 1000000000ull) {
            atomicOr(status, kStatusTimeout);
            *abort = 1;
            return false;
        }
    }
    return false;
}

// Same wait without the abort shortcut: used by the teardown to drain in-flight work.
__device__ __forceinline__ void pipe_drain(uint64_t *bar, uint32_t parity, uint32_t *status)
{
    mbar_wait(bar, parity, status, kStatusTimeout);
}

// OR of v over the 256 epilogue threads (named barrier 3); every one of them gets the result, so
// both groups leave their loops at the same point.
__device__ __forceinline__ bool epilogue_any(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 3, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

template <int N, int MODE>
__device__ __forceinline__ unsigned long long pipe_n_tiles(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a)
{
    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    if (MODE == kModeQuery) return ((unsigned long long)a.qn + kPipeRows - 1) / kPipeRows;
    if (MODE == kModeShade) return C.h_tile[f.n_types];
    if (MODE == kModeMarch) return mb.row_tile[f.n_types];
    if (MODE == kModePrimary) return C.p_tile[f.n_types];
    return C.s_tile[f.n_types];
}

template <int MODE>
__device__ __forceinline__ int pipe_tile_type(const Workspace &ws, const MarchBuffers &mb, const PipeArgs &a,
                                              unsigned long long tile)
{
    if (MODE == kModeQuery) return a.query_type;
    const DevFrame &f = *ws.frame;
    const Counters &C = *ws.cnt;
    const unsigned long long *off = MODE == kModeShade ? C.h_tile
                                  : MODE == kModeMarch ? mb.row_tile
                                  : MODE == kModePrimary ? C.p_tile : C.s_tile;
    int t = 0;
    while (t + 1 < f.n_types && off[t + 1] <= tile) ++t;
    return t;
}

// Pair index of row R of a NeDF tile of type t (Step-1 pairs, Step-3 pairs or caller queries);
// false past the end of the type's list (or of the queries).
template <int MODE>
__device__ __forceinline__ bool nedf_row_index(const Workspace &ws, const PipeArgs &a, int t, unsigned long long tile, int R,
                                               unsigned long long &idx)
{
    if (MODE == kModeQuery) {
        idx = tile * kPipeRows + R;
        return idx < (unsigned long long)a.qn;
    }
    const Counters &C = *ws.cnt;
    const unsigned long long *toff = MODE == kModePrimary ? C.p_tile : C.s_tile;
    const unsigned long long *poff = MODE == kModePrimary ? C.p_off : C.s_off;
    idx = poff[t] + (tile - toff[t]) * kPipeRows + R;
    return idx < poff[t + 1];
}

// Validity and local ray of row R of a NeDF tile, for its set-up (and a query's output).  A listed
// pair's local ray and chord come from the binning pass: one coalesced load, no chain of dependent
// loads through the pair and instance records.
template <int MODE>
__device__ __forceinline__ void nedf_row(const Workspace &ws, const PipeArgs &a, const DevType &T, int t,
                                         unsigned long long tile, int R, unsigned long long &idx, bool &valid, PairRay &pr)
{
    pr.kept = false;
    valid = nedf_row_index<MODE>(ws, a, t, tile, R, idx);
    if (!valid) return;
    if (MODE == kModeQuery) {
        pr.ol = v3(a.qo[3 * idx], a.qo[3 * idx + 1], a.qo[3 * idx + 2]);
        pr.dl = normalized(v3(a.qd[3 * idx], a.qd[3 * idx + 1], a.qd[3 * idx + 2]));
        Chord ch;
        pr.kept = bound_chord(pr.ol, pr.dl, T.rb, ch);
        pr.te = ch.te; pr.tx = ch.tx; pr.tp = ch.tp;
    } else {
        const float4 *geo = MODE == kModePrimary ? ws.pgeo : ws.sgeo;
        const float4 g0 = __ldg(&geo[2 * idx]), g1 = __ldg(&geo[2 * idx + 1]);
        pr.ol = v3(g0.x, g0.y, g0.z);
        pr.te = g0.w;
        pr.dl = v3(g1.x, g1.y, g1.z);
        pr.tp = g1.w;
        pr.kept = true;                          // the binning lists only pairs that meet the bound
    }
}

}  // namespace nedf
