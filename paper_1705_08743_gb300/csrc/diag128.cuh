// Phase 1 of the blocked closure on one 128×128 diagonal block, in shared memory, by 128
// threads: Section 2's Warshall loop with Section 3's Floyd ⊕/⊗ on the anti-distance
// lanes (u8 and u16 as 16-bit lane pairs, see sr_common.cuh).  Used by the persistent
// schedule and by the fused-pass schedule.
#pragma once

#include "antidist_tile.cuh"
#include "sr_common.cuh"

namespace sr {
namespace diag {

// The block sits in shared memory as 16-bit lane pairs (entry c of row r in the low or
// high half of word r·kDiagLdx + c/2; rows padded to kDiagLdx words).  It is closed by the same
// three phases once more on its two 64-wide halves: close X00; X01 ⊕= X00 ⊗ X01 and
// X10 ⊕= X10 ⊗ X00; X11 ⊕= X10 ⊗ X01; close X11; X10 ⊕= X11 ⊗ X10 and X01 ⊕= X01 ⊗ X11;
// X00 ⊕= X01 ⊗ X10.  Entries outside the block (a ragged last block) are 0, and 0 ⊗ x =
// x ⊗ 0 = 0, so every step may run over the full 64 pivots.
constexpr int kDiagW = 128;                 // block side
constexpr int kDiagLdx = 68;                // words per staged row (16-byte aligned rows)
constexpr int kDiagThreads = 128;           // threads that run the routines
constexpr size_t kDiagSmem = (size_t)(kDiagW * kDiagLdx + 64) * sizeof(uint32_t);

// thread (r, h) = (tid / 2, tid % 2) holds row r, lane pairs [16h, 16h + 16) of a 64-wide half
__device__ __forceinline__ void load16(const uint32_t *src, uint32_t (&x)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 v = reinterpret_cast<const uint4 *>(src)[q];
        x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void store16(uint32_t *dst, const uint32_t (&x)[16])
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        reinterpret_cast<uint4 *>(dst)[q] = make_uint4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}

// Warshall/Floyd over the 64 pivots of the half-block at (o, o), o in {0, 64}: before pivot k
// the two threads of row k publish it (double-buffered), one barrier per pivot; entry (r, k)
// comes from the thread of row r that holds column k, by a shuffle within the lane pair.
template <class KD, int SYNC>
__device__ void close64(uint32_t *X, uint32_t *piv, int o)
{
    const int tid = threadIdx.x, r = tid >> 1, h = tid & 1;
    uint32_t x[16];
    uint32_t *row = X + (o + r) * kDiagLdx + o / 2 + 16 * h;
    load16(row, x);
#pragma unroll
    for (int k = 0; k < 64; ++k) {
        uint32_t *pb = piv + (k & 1) * 32;
        if (r == k) store16(pb + 16 * h, x);
        tile_sync<SYNC>();
        const uint32_t mine = x[(k >> 1) & 15];
        const uint32_t other = __shfl_xor_sync(0xffffffffu, mine, 1);
        const uint32_t w = h == (k >> 5) ? mine : other;
        uint32_t a0, a1;
        KD::bcast((w >> (16 * (k & 1))) & 0xFFFFu, a0, a1);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = reinterpret_cast<const uint4 *>(pb + 16 * h)[q];
            x[4 * q] = KD::op(x[4 * q], v.x, a0, a1);
            x[4 * q + 1] = KD::op(x[4 * q + 1], v.y, a0, a1);
            x[4 * q + 2] = KD::op(x[4 * q + 2], v.z, a0, a1);
            x[4 * q + 3] = KD::op(x[4 * q + 3], v.w, a0, a1);
        }
    }
    store16(row, x);
}

// C ⊕= A ⊗ B on 64-wide halves: C at (cr, cc), A at (ar, ac), B at (br, bc) (entry offsets).
// A in-place update (C sharing rows with A or B) reads a mix of old and new entries, which
// the monotone ⊗ makes harmless.
template <class KD>
__device__ void mul64(uint32_t *X, int cr, int cc, int ar, int ac, int br, int bc)
{
    const int tid = threadIdx.x, r = tid >> 1, h = tid & 1;
    uint32_t x[16];
    uint32_t *crow = X + (cr + r) * kDiagLdx + cc / 2 + 16 * h;
    const uint32_t *arow = X + (ar + r) * kDiagLdx + ac / 2;
    const uint32_t *b0 = X + br * kDiagLdx + bc / 2 + 16 * h;
    load16(crow, x);
#pragma unroll 4
    for (int k = 0; k < 64; ++k) {
        uint32_t a0, a1;
        KD::bcast((arow[k >> 1] >> (16 * (k & 1))) & 0xFFFFu, a0, a1);
        const uint4 *bv = reinterpret_cast<const uint4 *>(b0 + k * kDiagLdx);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 v = bv[q];
            x[4 * q] = KD::op(x[4 * q], v.x, a0, a1);
            x[4 * q + 1] = KD::op(x[4 * q + 1], v.y, a0, a1);
            x[4 * q + 2] = KD::op(x[4 * q + 2], v.z, a0, a1);
            x[4 * q + 3] = KD::op(x[4 * q + 3], v.w, a0, a1);
        }
    }
    store16(crow, x);
}

// Closes the diagonal block at (k0, k0) of the D×D matrix T (row stride ldt) in place, on
// threads 0..kDiagThreads-1 with SYNC their barrier (tile_sync) and X the first kDiagSmem
// bytes of shared memory.  T is read through L2 (other CTAs of the launch may have written it).
template <class KD, int SYNC>
__device__ void close_diag128(typename KD::elem *T, int64_t ldt, int D, int k0, uint32_t *X)
{
    using E = typename KD::elem;
    uint32_t *piv = X + kDiagW * kDiagLdx;
    const int tid = threadIdx.x;
    const int bw = min(kDiagW, D - k0);
    constexpr int CH = 16 / (int)sizeof(E), CPR = kDiagW / CH;       // entries per chunk, chunks per row
    // stage: 16-byte chunks through L2, zero outside the block
    for (int c = tid; c < kDiagW * CPR; c += kDiagThreads) {
        const int r = c / CPR, col = (c % CPR) * CH;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (r < bw && col < bw) {
            const E *src = T + (int64_t)(k0 + r) * ldt + k0 + col;
            if (col + CH <= bw) {
                v = __ldcg(reinterpret_cast<const uint4 *>(src));
            } else {
                uint32_t w[4] = {0u, 0u, 0u, 0u};
                for (int t = 0; t < CH; ++t)
                    if (col + t < bw) w[(t * sizeof(E)) / 4] |= (uint32_t)__ldcg(src + t) << (8 * ((t * sizeof(E)) % 4));
                v = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        uint32_t *d = X + r * kDiagLdx + col / 2;
        if (sizeof(E) == 1) {
            reinterpret_cast<uint4 *>(d)[0] = make_uint4(u8x2_lo(v.x), u8x2_hi(v.x), u8x2_lo(v.y), u8x2_hi(v.y));
            reinterpret_cast<uint4 *>(d)[1] = make_uint4(u8x2_lo(v.z), u8x2_hi(v.z), u8x2_lo(v.w), u8x2_hi(v.w));
        } else {
            reinterpret_cast<uint4 *>(d)[0] = v;
        }
    }
    tile_sync<SYNC>();
    close64<KD, SYNC>(X, piv, 0);
    tile_sync<SYNC>();
    mul64<KD>(X, 0, 64, 0, 0, 0, 64);                      // X01 ⊕= X00 ⊗ X01
    mul64<KD>(X, 64, 0, 64, 0, 0, 0);                      // X10 ⊕= X10 ⊗ X00
    tile_sync<SYNC>();
    mul64<KD>(X, 64, 64, 64, 0, 0, 64);                    // X11 ⊕= X10 ⊗ X01
    tile_sync<SYNC>();
    close64<KD, SYNC>(X, piv, 64);
    tile_sync<SYNC>();
    mul64<KD>(X, 64, 0, 64, 64, 64, 0);                    // X10 ⊕= X11 ⊗ X10
    mul64<KD>(X, 0, 64, 0, 64, 64, 64);                    // X01 ⊕= X01 ⊗ X11
    tile_sync<SYNC>();
    mul64<KD>(X, 0, 0, 0, 64, 64, 0);                      // X00 ⊕= X01 ⊗ X10
    tile_sync<SYNC>();
    for (int c = tid; c < kDiagW * CPR; c += kDiagThreads) {
        const int r = c / CPR, col = (c % CPR) * CH;
        if (r >= bw || col >= bw) continue;
        const uint32_t *q = X + r * kDiagLdx + col / 2;
        E *dst = T + (int64_t)(k0 + r) * ldt + k0 + col;
        uint4 v;
        if (sizeof(E) == 1)
            v = make_uint4(pack_u8x4(q[0], q[1]), pack_u8x4(q[2], q[3]), pack_u8x4(q[4], q[5]), pack_u8x4(q[6], q[7]));
        else
            v = make_uint4(q[0], q[1], q[2], q[3]);
        if (col + CH <= bw) {
            *reinterpret_cast<uint4 *>(dst) = v;
        } else {
            const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
            for (int t = 0; t < CH; ++t)
                if (col + t < bw)
                    dst[t] = (E)((w4[(t * sizeof(E)) / 4] >> (8 * ((t * sizeof(E)) % 4))) & (sizeof(E) == 1 ? 0xFFu : 0xFFFFu));
        }
    }
}

}  // namespace diag
}  // namespace sr
