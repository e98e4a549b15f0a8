// Anti-distance semiring product and pivot-block kernels (u8: S = 255, u16: S = 65535;
// the u32 kernels, S = 2^32 − 1, are in antidist32.cu).  The closure schedules that
// drive them are in closure.cu.
//
// Product (Section 2 formula, Section 3 ⊗, Section 4 listings):
//   C := (accumulate ? C : 0) ⊕ A ⊗ B,   (A ⊗ B)_ij = max_k max(A_ik + B_kj − S, 0).
// The paper computes it as a running ⊕ of column-times-row outer products,
// k outermost ("Floyd-Warshall-abc").  Here each CTA owns a BM×BN tile of C in
// registers and streams BK-deep k-panels of A and B through shared memory; per
// k every thread applies the outer product of its TM entries of column k of A
// with its TN entries of row k of B (two 16-bit lanes per register, one DPX
// add-max per lane pair; see sr_common.cuh for the exact lane arithmetic).
//
// Pivot block (phase 1 of the blocked closure, Section 2 Warshall / Section 3 Floyd):
// one CTA closes a 128×128 diagonal block in shared memory and registers, optionally
// after applying its update from the previous pivot block's panels.

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "antidist_tile.cuh"
#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

template <class KD, int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(MulCfg<KD, BM, BN, BK, TM, TN>::THREADS, MulCfg<KD, BM, BN, BK, TM, TN>::MIN_BLOCKS)
antidist_mul_kernel(MulArgs p)
{
    // one tile per CTA; a grid short of the tile count leaves the rest to the split kernel
    mul_tiles<KD, BM, BN, BK, TM, TN, VEC>(p, blockIdx.x, 1 << 30);
}

// The last, partial wave of a deep product split along K: cluster c (of n CTAs) computes
// tile base + c, CTA rank r of it the k-slice [r·kslice, (r+1)·kslice) (kslice a multiple of
// BK, so every slice starts 16-byte aligned); rank 0 merges and stores.
template <class KD, int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(MulCfg<KD, BM, BN, BK, TM, TN>::THREADS, MulCfg<KD, BM, BN, BK, TM, TN>::MIN_BLOCKS)
antidist_mul_split_kernel(MulArgs p, int base, int kslice)
{
    mul_tiles<KD, BM, BN, BK, TM, TN, VEC, false, 0, true>(p, base + (int)(blockIdx.x / cluster_size()), 1 << 30,
                                                           0x7fffffff, kslice);
}

// Many independent products in one launch (the batched closure's grouped schedule):
// CTA b computes tile b - start[i] of product i, i the last product with start[i] <= b.
template <class KD, int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(MulCfg<KD, BM, BN, BK, TM, TN>::THREADS, MulCfg<KD, BM, BN, BK, TM, TN>::MIN_BLOCKS)
antidist_mul_grouped_kernel(const MulArgs *args, const int *start, int n)
{
    const int b = blockIdx.x;
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const MulArgs p = args[lo];
    // many small products: their ragged edge tiles skip the empty half (128-wide tiles)
    constexpr bool kRagged = TM % 8 == 0 && (TN / 2) % 8 == 0;
    mul_tiles<KD, BM, BN, BK, TM, TN, VEC, false, 0, false, kRagged>(p, b - start[lo], 1 << 30);
}

// -------------------------------------------------------------------------
// Phase 1 of the blocked closure: close one pivot block on one CTA
// -------------------------------------------------------------------------
// One CTA of 256 threads; the 128×128 block lives in shared memory as 16-bit lane
// pairs (rows padded to 65 words, so a column of lanes falls in distinct banks),
// loaded and stored in coalesced 16-byte chunks.  With kprev >= 0 the block first
// receives its phase-3 update from the previous pivot block, T_kk ⊕= T_k,prev ⊗
// T_prev,k: a 128-deep product, thread (r0, c0), r0, c0 in [0,16), holding rows
// r0 + 16 j and lane pairs c0 + 16 m in registers.
//
// The closure itself is the three-phase blocked scheme once more, on 32×32
// sub-blocks.  For each sub-block s:
//   1. one warp closes the diagonal sub-block D: lane = row, the 16 lane pairs of a
//      row in registers, the pivot row shuffled from its lane (32 steps, no barrier);
//   2. the column panel (rows outside s, columns of s) becomes x ⊗ (I ⊕ D) row by
//      row in registers (threads 0-95), while threads 128-255 update the row panel
//      (rows of s, columns outside s) in place: X_rj ⊕= D_rk ⊗ X_kj;
//   3. every entry outside row and column s: X_ij ⊕= X_ik ⊗ X_kj over k in s.
// Three barriers per sub-block instead of one per pivot.  Entries outside the block
// width bw are zero and stay zero (0 ⊗ x = 0), so ragged blocks need no special case.
// The in-place row panel may read entries other threads already updated; any mix of
// old and new values gives the same result because D is closed and ⊗ is monotone.
template <class KD, int PB>
struct PivotCfg {
    static constexpr int TRN = PB / 16, TCN = PB / 32;
    static constexpr int SB = 32, NP = PB / 2, LDX = NP + 1;         // lane pairs per row, padded
    static constexpr size_t SX = (size_t)PB * LDX * 4;                // the block
    static constexpr size_t KPREV = (size_t)KD::AW * PB * PB * 4      // sY: [k][row] broadcast words
                                    + (size_t)PB * NP * 4;             // sZ: [k][lane pair]
    static constexpr size_t CLOSE = (size_t)KD::AW * SB * PB * 4      // sA: [SB][PB] broadcast column panel
                                    + (size_t)KD::AW * SB * SB * 4    // sD: [SB][SB] broadcast diagonal
                                    + (size_t)SB * (SB / 2) * 4;      // sDp: [SB][SB/2] diagonal lane pairs
    static constexpr size_t SMEM = SX + (KPREV > CLOSE ? KPREV : CLOSE);
    static_assert(PB == 128, "four 32-wide sub-blocks");
    static_assert(SX % 16 == 0, "16-byte aligned staging after the block");
};

// rows [i0, i0+h) × columns [j0, j0+w) of T (zero outside) -> dst[r * ldd + pair] as
// 16-bit lane pairs, PB columns, one 16-byte chunk of a row per thread and step
template <class E, int PB, bool VEC>
__device__ __forceinline__ void pivot_stage(const E *T, int64_t ldt, int i0, int j0, int h, int w, uint32_t *dst,
                                            int ldd)
{
    constexpr int CH = 16 / (int)sizeof(E), CPR = PB / CH;          // entries per chunk, chunks per row
    for (int c = threadIdx.x; c < PB * CPR; c += blockDim.x) {
        const int r = c / CPR, col = (c % CPR) * CH;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < h) {
            const E *src = T + (int64_t)(i0 + r) * ldt + j0 + col;
            if (VEC && col + CH <= w) {
                v = *reinterpret_cast<const uint4 *>(src);
            } else {
                uint32_t q[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int t = 0; t < CH; ++t)
                    if (col + t < w)
                        q[(t * sizeof(E)) / 4] |= (uint32_t)src[t] << (8 * ((t * sizeof(E)) % 4));
                v = make_uint4(q[0], q[1], q[2], q[3]);
            }
        }
        uint32_t *d = dst + r * ldd + col / 2;
        if (sizeof(E) == 1) {
            d[0] = u8x2_lo(v.x); d[1] = u8x2_hi(v.x); d[2] = u8x2_lo(v.y); d[3] = u8x2_hi(v.y);
            d[4] = u8x2_lo(v.z); d[5] = u8x2_hi(v.z); d[6] = u8x2_lo(v.w); d[7] = u8x2_hi(v.w);
        } else {
            d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
        }
    }
}

// rows [i0, i0+h) × columns [j0, j0+w) of T (zero outside), each entry a broadcast
// to its A-operand words: y0[col * PB + row] (and y1 for u16)
template <class KD, int PB, bool VEC>
__device__ __forceinline__ void pivot_stage_bcast(const typename KD::elem *T, int64_t ldt, int i0, int j0, int h,
                                                  int w, uint32_t *y0, uint32_t *y1)
{
    using E = typename KD::elem;
    constexpr int CH = 16 / (int)sizeof(E), CPR = PB / CH;
    for (int c = threadIdx.x; c < PB * CPR; c += blockDim.x) {
        const int r = c / CPR, col = (c % CPR) * CH;
        uint32_t q[4] = {0u, 0u, 0u, 0u};
        if (r < h) {
            const E *src = T + (int64_t)(i0 + r) * ldt + j0 + col;
            if (VEC && col + CH <= w) {
                const uint4 v = *reinterpret_cast<const uint4 *>(src);
                q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
            } else {
#pragma unroll
                for (int t = 0; t < CH; ++t)
                    if (col + t < w)
                        q[(t * sizeof(E)) / 4] |= (uint32_t)src[t] << (8 * ((t * sizeof(E)) % 4));
            }
        }
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const uint32_t a = (q[(t * sizeof(E)) / 4] >> (8 * ((t * sizeof(E)) % 4))) & (sizeof(E) == 1 ? 0xFFu : 0xFFFFu);
            uint32_t a0, a1;
            KD::bcast(a, a0, a1);
            y0[(col + t) * PB + r] = a0;
            if (KD::AW == 2) y1[(col + t) * PB + r] = a1;
        }
    }
}

template <class KD, int PB, bool VEC>
__device__ __forceinline__ void pivot_block(void *Tv, int64_t ldt, int D, int kb, int kprev)
{
    using E = typename KD::elem;
    using Cfg = PivotCfg<KD, PB>;
    constexpr int TRN = Cfg::TRN, TCN = Cfg::TCN, SB = Cfg::SB, LDX = Cfg::LDX, NP = Cfg::NP;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sX = smem;                                    // [PB][LDX] lane pairs
    uint32_t *stage = smem + Cfg::SX / 4;                   // kprev operands, then closure staging

    E *T = static_cast<E *>(Tv);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int r0 = tid >> 4, c0 = tid & 15;
    const int k0 = kb * PB, bw = min(PB, D - k0);

    pivot_stage<E, PB, VEC>(T, ldt, k0, k0, bw, bw, sX, LDX);

    if (kprev >= 0) {
        uint32_t *sY0 = stage;                              // [PB][PB]: broadcast T_k,prev at [k][row]
        uint32_t *sY1 = stage + PB * PB;
        uint32_t *sZ = stage + KD::AW * PB * PB;            // [PB][NP]: T_prev,k lane pairs
        const int p0 = kprev * PB, pw = min(PB, D - p0);
        pivot_stage<E, PB, VEC>(T, ldt, p0, k0, pw, bw, sZ, NP);
        pivot_stage_bcast<KD, PB, VEC>(T, ldt, k0, p0, bw, pw, sY0, sY1);
        __syncthreads();
        uint32_t X[TRN][TCN];
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) X[j][m] = sX[(r0 + 16 * j) * LDX + c0 + 16 * m];
        for (int kk = 0; kk < pw; ++kk) {
            uint32_t bv[TCN], a0[TRN], a1[TRN];
#pragma unroll
            for (int m = 0; m < TCN; ++m) bv[m] = sZ[kk * NP + c0 + 16 * m];
#pragma unroll
            for (int j = 0; j < TRN; ++j) {
                a0[j] = sY0[kk * PB + r0 + 16 * j];
                a1[j] = KD::AW == 2 ? sY1[kk * PB + r0 + 16 * j] : 0u;
            }
#pragma unroll
            for (int j = 0; j < TRN; ++j)
#pragma unroll
                for (int m = 0; m < TCN; ++m) X[j][m] = KD::op(X[j][m], bv[m], a0[j], a1[j]);
        }
        __syncthreads();                                    // all reads of sX and the staging done
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) sX[(r0 + 16 * j) * LDX + c0 + 16 * m] = X[j][m];
    }
    __syncthreads();

    uint32_t *sA0 = stage;                                  // [SB][PB]: broadcast X_i,32s+k
    uint32_t *sA1 = sA0 + SB * PB;
    uint32_t *sD0 = sA0 + KD::AW * SB * PB;                 // [SB][SB]: broadcast D_r,k at [k][r]
    uint32_t *sD1 = sD0 + SB * SB;
    uint32_t *sDp = sD0 + KD::AW * SB * SB;                 // [SB][SB/2]: D rows as lane pairs

    for (int s = 0; s < PB / SB && SB * s < bw; ++s) {
        const int rs = SB * s, ps = (SB / 2) * s;           // first row / lane pair of sub-block s
        // 1. close the diagonal sub-block (one warp)
        if (warp == 0) {
            uint32_t d[16];
#pragma unroll
            for (int p = 0; p < 16; ++p) d[p] = sX[(rs + lane) * LDX + ps + p];
#pragma unroll
            for (int kk = 0; kk < SB; ++kk) {
                uint32_t piv[16];
#pragma unroll
                for (int p = 0; p < 16; ++p) piv[p] = __shfl_sync(0xffffffffu, d[p], kk);
                uint32_t a0, a1;
                KD::bcast((d[kk >> 1] >> (16 * (kk & 1))) & 0xFFFFu, a0, a1);
#pragma unroll
                for (int p = 0; p < 16; ++p) d[p] = KD::op(d[p], piv[p], a0, a1);
            }
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                sX[(rs + lane) * LDX + ps + p] = d[p];
                sDp[lane * 16 + p] = d[p];
            }
#pragma unroll
            for (int kk = 0; kk < SB; ++kk) {
                uint32_t a0, a1;
                KD::bcast((d[kk >> 1] >> (16 * (kk & 1))) & 0xFFFFu, a0, a1);
                sD0[kk * SB + lane] = a0;
                if (KD::AW == 2) sD1[kk * SB + lane] = a1;
            }
        }
        __syncthreads();
        // 2a. column panel, one row per thread: x := x ⊗ (I ⊕ D)
        if (tid < PB - SB) {
            const int i = tid < rs ? tid : tid + SB;
            uint32_t x[16], y[16];
#pragma unroll
            for (int p = 0; p < 16; ++p) y[p] = x[p] = sX[i * LDX + ps + p];
#pragma unroll
            for (int kk = 0; kk < SB; ++kk) {
                uint32_t a0, a1;
                KD::bcast((x[kk >> 1] >> (16 * (kk & 1))) & 0xFFFFu, a0, a1);
                const uint4 *drow = reinterpret_cast<const uint4 *>(sDp + kk * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 v = drow[q];
                    y[4 * q] = KD::op(y[4 * q], v.x, a0, a1);
                    y[4 * q + 1] = KD::op(y[4 * q + 1], v.y, a0, a1);
                    y[4 * q + 2] = KD::op(y[4 * q + 2], v.z, a0, a1);
                    y[4 * q + 3] = KD::op(y[4 * q + 3], v.w, a0, a1);
                }
            }
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                sX[i * LDX + ps + p] = y[p];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t a0, a1;
                    KD::bcast((y[p] >> (16 * h)) & 0xFFFFu, a0, a1);
                    sA0[(2 * p + h) * PB + i] = a0;
                    if (KD::AW == 2) sA1[(2 * p + h) * PB + i] = a1;
                }
            }
        } else if (tid >= 128) {
            // 2b. row panel (in place): row rs + (tid & 31), 12 lane pairs outside s
            const int r = rs + (tid & 31), g = (tid >> 5) - 4;
            uint32_t acc[12];
            int pc[12];
#pragma unroll
            for (int u = 0; u < 12; ++u) {
                const int jq = g + 4 * u;                   // 0..47
                pc[u] = jq < ps ? jq : jq + SB / 2;
                acc[u] = sX[r * LDX + pc[u]];
            }
            for (int kk = 0; kk < SB; ++kk) {
                const uint32_t a0 = sD0[kk * SB + (tid & 31)];
                const uint32_t a1 = KD::AW == 2 ? sD1[kk * SB + (tid & 31)] : 0u;
#pragma unroll
                for (int u = 0; u < 12; ++u)
                    acc[u] = KD::op(acc[u], sX[(rs + kk) * LDX + pc[u]], a0, a1);
            }
#pragma unroll
            for (int u = 0; u < 12; ++u) sX[r * LDX + pc[u]] = acc[u];
        }
        __syncthreads();
        // 3. everything outside row and column s: 96 rows × 48 lane pairs, 6 × 3 per thread
        {
            const int tr = tid >> 4, tc = tid & 15;
            int ri[6], pj[3];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const int i = tr + 16 * q;
                ri[q] = i < rs ? i : i + SB;
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int j = tc + 16 * u;
                pj[u] = j < ps ? j : j + SB / 2;
            }
            uint32_t acc[6][3];
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
                for (int u = 0; u < 3; ++u) acc[q][u] = sX[ri[q] * LDX + pj[u]];
            for (int kk = 0; kk < SB; ++kk) {
                uint32_t a0[6], a1[6], b[3];
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    a0[q] = sA0[kk * PB + ri[q]];
                    a1[q] = KD::AW == 2 ? sA1[kk * PB + ri[q]] : 0u;
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) b[u] = sX[(rs + kk) * LDX + pj[u]];
#pragma unroll
                for (int q = 0; q < 6; ++q)
#pragma unroll
                    for (int u = 0; u < 3; ++u) acc[q][u] = KD::op(acc[q][u], b[u], a0[q], a1[q]);
            }
#pragma unroll
            for (int q = 0; q < 6; ++q)
#pragma unroll
                for (int u = 0; u < 3; ++u) sX[ri[q] * LDX + pj[u]] = acc[q][u];
        }
        __syncthreads();
    }

    // write back in 16-byte chunks
    constexpr int CH = 16 / (int)sizeof(E), CPR = PB / CH;
    for (int c = tid; c < PB * CPR; c += 256) {
        const int r = c / CPR, col = (c % CPR) * CH;
        if (r >= bw || col >= bw)
            continue;
        const uint32_t *q = sX + r * LDX + col / 2;
        E *dst = T + (int64_t)(k0 + r) * ldt + k0 + col;
        uint4 v;
        if (sizeof(E) == 1)
            v = make_uint4(pack_u8x4(q[0], q[1]), pack_u8x4(q[2], q[3]), pack_u8x4(q[4], q[5]), pack_u8x4(q[6], q[7]));
        else
            v = make_uint4(q[0], q[1], q[2], q[3]);
        if (VEC && col + CH <= bw) {
            *reinterpret_cast<uint4 *>(dst) = v;
        } else {
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < CH; ++t)
                if (col + t < bw) dst[t] = (E)((w4[(t * sizeof(E)) / 4] >> (8 * ((t * sizeof(E)) % 4))) & (sizeof(E) == 1 ? 0xFFu : 0xFFFFu));
        }
    }
}

template <class KD, int PB, bool VEC>
__global__ void __launch_bounds__(256) antidist_pivot_kernel(void *Tv, int64_t ldt, int D, int kb, int kprev)
{
    pivot_block<KD, PB, VEC>(Tv, ldt, D, kb, kprev);
}

// Pivot block kb of many graphs in one launch (the batched closure's grouped schedule):
// CTA b closes block kb of graph active[b]; phase 3 of kb-1 has already updated it.
template <class KD, int PB>
__global__ void __launch_bounds__(256) antidist_pivot_grouped_kernel(const BatchGraph *graphs, const int *active, int kb)
{
    const BatchGraph g = graphs[active[blockIdx.x]];
    if (g.pad)
        pivot_block<KD, PB, true>(g.T, g.ldt, g.D, kb, -1);
    else
        pivot_block<KD, PB, false>(g.T, g.ldt, g.D, kb, -1);
}

// -------------------------------------------------------------------------
// Host launchers
// -------------------------------------------------------------------------
template <class KD, int BM, int BN, int BK, int TM, int TN>
static sr_status launch_mul_cfg(const MulArgs &a, bool vec, cudaStream_t s)
{
    using Cfg = MulCfg<KD, BM, BN, BK, TM, TN>;
    const int64_t tiles = (int64_t)((a.N + BN - 1) / BN) * ((a.R + BM - 1) / BM);
    if (tiles > 0x7fffffffLL)
        return fail(SR_EINVAL, "antidist_mul: too many tiles (%lld)", (long long)tiles);
    auto kern = vec ? antidist_mul_kernel<KD, BM, BN, BK, TM, TN, true>
                    : antidist_mul_kernel<KD, BM, BN, BK, TM, TN, false>;
    constexpr bool kSplits = TN == 16;                  // the 128×128 tiles of deep products
    static bool attr[2][kMaxDevices] = {};
    static int slots[kMaxDevices] = {}, sm_count[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[vec][dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        if constexpr (kSplits) {
            auto split = vec ? antidist_mul_split_kernel<KD, BM, BN, BK, TM, TN, true>
                             : antidist_mul_split_kernel<KD, BM, BN, BK, TM, TN, false>;
            SR_CUDA_CHECK(cudaFuncSetAttribute(split, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        }
        int per_sm = 0, sms = 0, d = 0;
        SR_CUDA_CHECK(cudaGetDevice(&d));
        SR_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::THREADS, Cfg::SMEM));
        SR_CUDA_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d));
        slots[dev] = per_sm * sms;
        sm_count[dev] = sms;
        attr[vec][dev] = true;
    }
    // One tile per CTA: the hardware block scheduler balances a sparse last wave better than
    // a persistent grid or smaller tail tiles on a second stream (both measured slower).
    // A CTA alone on an SM runs its tile about as fast as the SM runs three (the k-loop has
    // ILP enough), so a last wave of up to one tile per SM costs a whole tile time however
    // few its tiles.  When the last wave is that sparse, its tiles go to clusters of split_k
    // CTAs over slices of K instead, with split_k as large as keeps one CTA per SM (a 6144³
    // u8 product on GB300: 2304 tiles on 456 slots leave 24, split 4 ways: 6.70 -> 6.44 ms).
    // Where split CTAs would share SMs the split gains nothing (4096³: 112 tail tiles;
    // 2.00 ms unsplit, 2.03 ms as 112 clusters of 4).
    const int nkt = (a.K + BK - 1) / BK;
    const int tail = slots[dev] > 0 ? (int)(tiles % slots[dev]) : 0;
    int split_k = 0;
    if (kSplits && a.K >= 1024 && a.skip_tile < 0 && a.rskipw == 0 && a.cskipw == 0 && tail > 0 && a.split)
        split_k = std::min(std::min(4, sm_count[dev] / tail), nkt / 4);
    if (split_k < 2) {
        kern<<<(unsigned)tiles, Cfg::THREADS, Cfg::SMEM, s>>>(a);
        SR_CUDA_CHECK(cudaGetLastError());
        count_launches();
        return SR_OK;
    }
    if (tiles > tail) {
        kern<<<(unsigned)(tiles - tail), Cfg::THREADS, Cfg::SMEM, s>>>(a);
        SR_CUDA_CHECK(cudaGetLastError());
        count_launches();
    }
    if constexpr (kSplits) {
        auto split = vec ? antidist_mul_split_kernel<KD, BM, BN, BK, TM, TN, true>
                         : antidist_mul_split_kernel<KD, BM, BN, BK, TM, TN, false>;
        const int kslice = (nkt + split_k - 1) / split_k * BK;
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(tail * split_k));
        lc.blockDim = dim3(Cfg::THREADS);
        lc.dynamicSmemBytes = Cfg::SMEM;
        lc.stream = s;
        cudaLaunchAttribute la[1];
        la[0].id = cudaLaunchAttributeClusterDimension;
        la[0].val.clusterDim.x = (unsigned)split_k;
        la[0].val.clusterDim.y = 1;
        la[0].val.clusterDim.z = 1;
        lc.attrs = la;
        lc.numAttrs = 1;
        SR_CUDA_CHECK(cudaLaunchKernelEx(&lc, split, a, (int)(tiles - tail), kslice));
        count_launches();
    }
    return SR_OK;
}

// Tile rows per group of the tile order for a deep product: enough that a wave of CTAs
// reuses A's row panels from L2, few enough that the group's panels of A (g · 128 rows · K)
// stay within about 32 MB of L2 beside the column panels of B streaming through.  Shallow
// products (the closure's K = 128..512 passes) keep the row-major order: their operands
// are small and stay in L2 anyway.
int group_rows(int R, int K, int esize, int bm)
{
    if (K < 1024) return 0;
    const int64_t per_row = (int64_t)bm * K * esize;
    const int tiles_m = (R + bm - 1) / bm;
    const int g = (int)std::max<int64_t>(1, ((int64_t)32 << 20) / per_row);
    return g >= tiles_m ? 0 : g;
}

sr_status launch_antidist_mul(const MulArgs &a0, sr_dtype dt, bool vec, cudaStream_t s, int tiles)
{
    if (a0.R <= 0 || a0.N <= 0)
        return SR_OK;
    MulArgs a = a0;
    if (a.group_m == 0 && a.skip_tile < 0)
        a.group_m = group_rows(a.R, a.K, dt == SR_U8 ? 1 : dt == SR_U16 ? 2 : 4, tiles == 1 ? 64 : 128);
    if (dt == SR_U32)
        return launch_antidist32_mul(a, vec, s, tiles);
    if (tiles == 1)
        return dt == SR_U8 ? launch_mul_cfg<KindU8, 64, 64, 32, 4, 8>(a, vec, s)
                           : launch_mul_cfg<KindU16, 64, 64, 32, 4, 8>(a, vec, s);
    return dt == SR_U8 ? launch_mul_cfg<KindU8, 128, 128, 32, 8, 16>(a, vec, s)
                       : launch_mul_cfg<KindU16, 128, 128, 32, 8, 16>(a, vec, s);
}

template <class KD, int PB>
static sr_status launch_pivot(void *T, int64_t ldt, int D, int kb, int kprev, bool vec, cudaStream_t s)
{
    if constexpr (std::is_same<KD, KindU32>::value) {
        static_assert(PB == 128, "u32 pivot block");
        return launch_antidist32_pivot(T, ldt, D, kb, kprev, s);
    } else {
    using Cfg = PivotCfg<KD, PB>;
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(antidist_pivot_kernel<KD, PB, true>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        SR_CUDA_CHECK(cudaFuncSetAttribute(antidist_pivot_kernel<KD, PB, false>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr[dev] = true;
    }
    if (vec)
        antidist_pivot_kernel<KD, PB, true><<<1, 256, Cfg::SMEM, s>>>(T, ldt, D, kb, kprev);
    else
        antidist_pivot_kernel<KD, PB, false><<<1, 256, Cfg::SMEM, s>>>(T, ldt, D, kb, kprev);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
    }
}

// ---- grouped launches (the batched closure's per-pivot-block schedule)
template <class KD, int BM, int BN, int BK, int TM, int TN>
static sr_status launch_grouped_cfg(const MulArgs *args, const int *start, int n, int tiles, bool vec,
                                    cudaStream_t s)
{
    using Cfg = MulCfg<KD, BM, BN, BK, TM, TN>;
    auto kern = vec ? antidist_mul_grouped_kernel<KD, BM, BN, BK, TM, TN, true>
                    : antidist_mul_grouped_kernel<KD, BM, BN, BK, TM, TN, false>;
    static bool attr[2][kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[vec][dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr[vec][dev] = true;
    }
    kern<<<tiles, Cfg::THREADS, Cfg::SMEM, s>>>(args, start, n);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_antidist_mul_grouped(const MulArgs *args, const int *start, int n, int tiles, sr_dtype dt,
                                      bool vec, bool thin, cudaStream_t s)
{
    if (n <= 0 || tiles <= 0)
        return SR_OK;
    if (thin)
        return dt == SR_U8 ? launch_grouped_cfg<KindU8, 64, 64, 32, 4, 8>(args, start, n, tiles, vec, s)
                           : launch_grouped_cfg<KindU16, 64, 64, 32, 4, 8>(args, start, n, tiles, vec, s);
    return dt == SR_U8 ? launch_grouped_cfg<KindU8, 128, 128, 32, 8, 16>(args, start, n, tiles, vec, s)
                       : launch_grouped_cfg<KindU16, 128, 128, 32, 8, 16>(args, start, n, tiles, vec, s);
}

template <class KD>
static sr_status launch_pivot_grouped_t(const BatchGraph *graphs, const int *active, int n, int kb, cudaStream_t s)
{
    constexpr int PB = 128;
    using Cfg = PivotCfg<KD, PB>;
    constexpr size_t SMEM = Cfg::SX + Cfg::CLOSE;          // no previous-block operands
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(antidist_pivot_grouped_kernel<KD, PB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
        attr[dev] = true;
    }
    antidist_pivot_grouped_kernel<KD, PB><<<n, 256, SMEM, s>>>(graphs, active, kb);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_antidist_pivot_grouped(const BatchGraph *graphs, const int *active, int n, int kb, sr_dtype dt,
                                        cudaStream_t s)
{
    if (n <= 0)
        return SR_OK;
    return dt == SR_U8 ? launch_pivot_grouped_t<KindU8>(graphs, active, n, kb, s)
                       : launch_pivot_grouped_t<KindU16>(graphs, active, n, kb, s);
}

sr_status launch_antidist_pivot(void *T, int64_t ldt, int D, int kb, int kprev, sr_dtype dt, bool vec,
                                cudaStream_t s)
{
    if (dt == SR_U8)
        return launch_pivot<KindU8, 128>(T, ldt, D, kb, kprev, vec, s);
    if (dt == SR_U32)
        return launch_pivot<KindU32, 128>(T, ldt, D, kb, kprev, vec, s);
    return launch_pivot<KindU16, 128>(T, ldt, D, kb, kprev, vec, s);
}

// -------------------------------------------------------------------------
// Encoding: T = S − w for 0 < w < S, else 0 (Section 3)
// -------------------------------------------------------------------------
// One 32-bit word of entries: S − w is the bitwise complement of w for every S here
// (2^bits − 1), w = S encodes to 0 by itself, and w = 0 ("no edge") is masked to 0.
template <class E>
__device__ __forceinline__ uint32_t encode_word(uint32_t x)
{
    if (sizeof(E) == 1) return ~x & __vcmpne4(x, 0u);
    if (sizeof(E) == 2) return ~x & __vcmpne2(x, 0u);
    return x ? ~x : 0u;
}

// 16-byte chunks of a row per thread (vector loads and stores when the rows are aligned)
template <class E, bool VEC>
__global__ void antidist_encode_kernel(const E *W, int64_t ldw, E *T, int64_t ldt, int R, int C)
{
    constexpr int CH = 16 / (int)sizeof(E);
    const int cpr = (C + CH - 1) / CH;
    const int64_t n = (int64_t)R * cpr;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / cpr), c = (int)(t % cpr) * CH;
        const E *src = W + (int64_t)r * ldw + c;
        E *dst = T + (int64_t)r * ldt + c;
        if (VEC && c + CH <= C) {
            uint4 v = *reinterpret_cast<const uint4 *>(src);
            v.x = encode_word<E>(v.x); v.y = encode_word<E>(v.y);
            v.z = encode_word<E>(v.z); v.w = encode_word<E>(v.w);
            *reinterpret_cast<uint4 *>(dst) = v;
        } else {
            for (int k = 0; k < CH && c + k < C; ++k) {
                const uint32_t w = src[k];
                dst[k] = (E)(w == 0u ? 0u : ~w);
            }
        }
    }
}

template <class E>
static void launch_encode_t(const void *W, int64_t ldw, void *T, int64_t ldt, int R, int C, int num_sms,
                            cudaStream_t s)
{
    constexpr int CH = 16 / (int)sizeof(E);
    const int64_t n = (int64_t)R * ((C + CH - 1) / CH);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
    const bool vec = aligned16(W) && aligned16(T) && ((ldw * (int64_t)sizeof(E)) & 15) == 0 &&
                     ((ldt * (int64_t)sizeof(E)) & 15) == 0;
    auto Wt = static_cast<const E *>(W);
    auto Tt = static_cast<E *>(T);
    if (vec)
        antidist_encode_kernel<E, true><<<blocks, 256, 0, s>>>(Wt, ldw, Tt, ldt, R, C);
    else
        antidist_encode_kernel<E, false><<<blocks, 256, 0, s>>>(Wt, ldw, Tt, ldt, R, C);
}

sr_status launch_antidist_encode(const void *W, int64_t ldw, void *T, int64_t ldt, int R, int C,
                                 sr_dtype dt, int num_sms, cudaStream_t s)
{
    if (dt == SR_U8)
        launch_encode_t<uint8_t>(W, ldw, T, ldt, R, C, num_sms, s);
    else if (dt == SR_U16)
        launch_encode_t<uint16_t>(W, ldw, T, ldt, R, C, num_sms, s);
    else
        launch_encode_t<uint32_t>(W, ldw, T, ldt, R, C, num_sms, s);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
