// A tcgen05 GEMM engine for the learned part: D[M][N] = sum_k A(m, k) B(n, k) with BF16 operands
// read from global memory in either major order, FP32 accumulation in TMEM and a fused epilogue.
//
// One CTA computes one 128 x BN output tile over a K range (the caller maps its grid to tiles,
// N blocks and K splits).  Four warps stage K in blocks of 64 through an S-deep ring of shared-memory stages with 16-byte cp.async
// copies (zero-filled outside the operands); thread 0 issues four M = 128, N = BN, K = 16 MMAs per
// block and commits them to the stage's barrier, which the copies into that stage wait for before
// they overwrite it.  The epilogue warps read the accumulator back with tcgen05.ld (warp w: rows
// 32w .. 32w + 31) and apply the epilogue functor.
//
// Shared-memory layout of an operand block of R rows (M or N) by 64 K, no swizzle, both orders:
//   K-major  (rows whose K is contiguous in global memory): element (r, k) at
//            (k / 8) * 16R + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
//   MN-major (K rows whose M or N is contiguous):          element (r, k) at
//            (k / 8) * 16R + (r / 8) * 128 + (k % 8) * 16 + (r % 8) * 2
// so that a K step of 16 is two 8-column groups 16R bytes apart (leading byte offset 16R) of
// 8-row core matrices 128 bytes apart (stride byte offset 128) in either order, the order being
// told to the MMA by the instruction descriptor (bit 15 for A, bit 16 for B).  Consecutive 16-byte
// vectors of a stage are copies of consecutive threads, so the stores into shared
// memory are conflict-free.
#pragma once

#include <cuda_bf16.h>

#include "tc_ptx.cuh"

namespace nedf {
namespace tcg {

using namespace tc;

constexpr int kBM = 128;          // rows of the output tile (TMEM lanes)
constexpr int kBK = 64;           // K per stage
constexpr int kThreads = 128;

enum Major : int { kKMajor = 0, kMNMajor = 1 };

// A global BF16 operand.  K-major: element (r, k) at p[r * ld + k]; MN-major: at p[k * ld + r].
// rows / k_len bound the valid region (outside reads as zero).  ones_row (B operands only): a
// synthesized row index >= rows whose elements are 1 inside the valid K range (a bias column).
struct Operand {
    const __nv_bfloat16 *p;
    long long ld;
    int rows;
    long long k_len;
    int major;
    int ones_row;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stages rows [r0, r0 + R) x K [k0, k0 + 64) of op into the block at `dst` (layout above).
template <int R>
__device__ __forceinline__ void load_block(const Operand &op, int r0, long long k0, uint8_t *dst)
{
    const uint32_t base = smem_addr(dst);
    constexpr int NV = R * kBK / 8;              // 16-byte vectors
    for (int v = threadIdx.x; v < NV; v += kThreads) {
        int r, kk;
        if (op.major == kKMajor) {
            r = v % R;                           // conflict-free: vector v at byte 16 v
            kk = (v / R) * 8;
        } else {
            kk = (v / R) * 8 + (v & 7);
            r = ((v % R) >> 3) * 8;
        }
        const int gr = r0 + r;
        const long long gk = k0 + kk;
        const uint32_t d = base + (uint32_t)v * 16u;
        if (op.major == kKMajor) {
            const bool ok = gr < op.rows && gk < op.k_len;
            const __nv_bfloat16 *src = ok ? op.p + (long long)gr * op.ld + gk : op.p;
            cp_async16(d, src, ok ? 16u : 0u);
        } else if (gr < op.rows || op.ones_row < 0 || op.ones_row < gr || op.ones_row >= gr + 8) {
            const bool ok = gr < op.rows && gk < op.k_len;
            const __nv_bfloat16 *src = ok ? op.p + gk * op.ld + gr : op.p;
            cp_async16(d, src, ok ? 16u : 0u);
        } else {
            // the 8-row group holding the synthesized bias row (MN-major B operands only)
            const uint32_t one = gk < op.k_len ? 0x3F80u : 0u;        // BF16 1.0
            uint32_t w[4] = {0u, 0u, 0u, 0u};
            const int j = op.ones_row - gr;
            w[j >> 1] = one << ((j & 1) * 16);
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(d), "r"(w[0]), "r"(w[1]), "r"(w[2]),
                         "r"(w[3])
                         : "memory");
        }
    }
}

struct GemmShared {
    uint64_t mma_done[8];
    uint64_t acc_full;
    uint32_t tmem_base;
};

template <int BN, int S>
struct GemmSmem {
    static constexpr int A_BYTES = kBM * kBK * 2;
    static constexpr int B_BYTES = BN * kBK * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    static constexpr int BYTES = S * STAGE + 1024;        // + alignment slack
    static constexpr int TMEM_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
};

// The D tile with rows m0 .. m0 + 127 of M and columns n0 .. n0 + BN - 1 of N over K [kb, ke)
// (kb a multiple of 64).  The epilogue is called as epi(row, first column, 32 values) for every
// row of the tile and every 32 columns.  Waits are bounded (timeout_flag set in *status).
template <int BN, int S, class Epi>
__device__ __forceinline__ void gemm_tile(const Operand &A, const Operand &B, int m0, int n0, long long kb, long long ke,
                                          const Epi &epi, uint32_t *status, uint32_t timeout_flag)
{
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "tcgen05 kind::f16 with M = 128 needs N = 16 .. 256");
    static_assert(S >= 2 && S <= 8, "stages");
    using SM = GemmSmem<BN, S>;
    extern __shared__ uint8_t gsm_raw[];
    __shared__ GemmShared sh;
    uint8_t *ring = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nk = ke > kb ? (int)((ke - kb + kBK - 1) / kBK) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&sh.mma_done[s], 1);
        mbar_init(&sh.acc_full, 1);
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&sh.tmem_base, SM::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh.tmem_base;

    // operands with the split's K range
    Operand a = A, b = B;
    a.k_len = ke;
    b.k_len = ke;
    uint32_t idesc = idesc_bf16(kBM, BN);
    if (A.major == kMNMajor) idesc |= 1u << 15;
    if (B.major == kMNMajor) idesc |= 1u << 16;
    bool ok = true;

    // prologue: blocks 0 .. S-2
    for (int i = 0; i < S - 1; ++i) {
        if (i < nk) {
            uint8_t *st = ring + (size_t)i * SM::STAGE;
            load_block<kBM>(a, m0, kb + (long long)i * kBK, st);
            load_block<BN>(b, n0, kb + (long long)i * kBK, st + SM::A_BYTES);
        }
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S;
        cp_async_wait<S - 2>();                  // this thread's copies of block kt have landed
        fence_proxy_async_smem();                // ... and are visible to the tensor core
        __syncthreads();
        if (threadIdx.x == 0 && ok) {
            tc_fence_after();
            const uint32_t sa = smem_addr(ring + (size_t)s * SM::STAGE), sb = sa + SM::A_BYTES;
            for (int j = 0; j < kBK / 16; ++j) {
                const uint64_t da = smem_desc(sa + (uint32_t)j * 2u * kBM * 16u, kBM * 16, 128);
                const uint64_t db = smem_desc(sb + (uint32_t)j * 2u * BN * 16u, BN * 16, 128);
                mma_bf16(tmem, da, db, idesc, (kt > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(&sh.mma_done[s]);
        }
        // refill the stage block kt - 1 used, once its MMAs are done
        const int nt = kt + S - 1;
        if (nt < nk) {
            const int sn = nt % S;
            if (kt >= 1 && ok) ok = mbar_wait(&sh.mma_done[sn], (uint32_t)(((kt - 1) / S) & 1), status, timeout_flag);
            if (ok) {
                uint8_t *st = ring + (size_t)sn * SM::STAGE;
                load_block<kBM>(a, m0, kb + (long long)nt * kBK, st);
                load_block<BN>(b, n0, kb + (long long)nt * kBK, st + SM::A_BYTES);
            }
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (threadIdx.x == 0) {
        if (nk > 0) mma_commit(&sh.acc_full);
        else mbar_arrive(&sh.acc_full);          // nothing to accumulate: the epilogue sees zeros
    }
    if (!mbar_wait(&sh.acc_full, 0u, status, timeout_flag)) {
        ok = false;
        mbar_wait(&sh.acc_full, 0u, status, timeout_flag);   // drain before TMEM is released
    }
    tc_fence_after();

    // epilogue: warp w reads lanes (rows) 32w .. 32w + 31, 32 columns at a time
    const int row = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
    for (int c = 0; c < BN; c += 32) {
        uint32_t v[32];
        if (nk > 0) {
            tmem_ld32(tl + (uint32_t)c, v);
            tmem_wait_ld(v);
        } else {
            for (int i = 0; i < 32; ++i) v[i] = 0u;
        }
        if (ok) epi(row, n0 + c, v);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, SM::TMEM_COLS);
}

}  // namespace tcg
}  // namespace nedf
