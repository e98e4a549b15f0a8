// Anti-distance semiring product and closure (u8: S = 255, u16: S = 65535).
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
// Closure (Section 2 Warshall, Section 3 Floyd): three-phase blocked form of
//   T := A;  for k = 1..D:  T := T ⊕ (T_col k ⊗ T_row k).
// For each k-block of width PB:
//   phase 1: T_kk := closure of the diagonal block (PB sequential pivots, one CTA);
//   phase 2: T_kj := T_kj ⊕ T_kk ⊗ T_kj,  T_ik := T_ik ⊕ T_ik ⊗ T_kk (panels);
//   phase 3: T_ij := T_ij ⊕ T_ik ⊗ T_kj for all other blocks (the product kernel
//            with K = PB, panel rows/columns excluded).
// Every pivot order gives the same fixed point, and rows/columns of the pivot
// block do not change in their own step, so the blocked order is exact.
// Phases 1 and 2 run fused in one launch: each panel CTA closes the diagonal
// block itself (all CTAs of the launch compute the identical T_kk).

#include <algorithm>
#include <cstdio>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

__device__ __forceinline__ int remap(int x, int skip0, int skipw) { return x < skip0 ? x : x + skipw; }

// -------------------------------------------------------------------------
// 16-byte chunk loads with zero fill outside [0, nrow) × [0, ncol)
// -------------------------------------------------------------------------
template <class E, bool VEC>
__device__ __forceinline__ uint4 load_chunk(const E *base, int64_t ld, int r, int c, int nrow, int ncol)
{
    constexpr int CH = 16 / sizeof(E);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= nrow || c >= ncol)
        return v;
    const E *p = base + (int64_t)r * ld + c;
    if (VEC && c + CH <= ncol)
        return *reinterpret_cast<const uint4 *>(p);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int t = 0; t < CH; ++t)
        if (c + t < ncol)
            w[(t * sizeof(E)) / 4] |= (uint32_t)p[t] << (8 * ((t * sizeof(E)) % 4));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ uint32_t u4get(const uint4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// element t of a 16-byte chunk
template <class E>
__device__ __forceinline__ uint32_t chunk_elem(const uint4 &v, int t)
{
    if (sizeof(E) == 1)
        return __byte_perm(u4get(v, t / 4), 0u, 0x4440 | (t % 4));
    return (u4get(v, t / 2) >> (16 * (t % 2))) & 0xFFFFu;
}

// -------------------------------------------------------------------------
// Product kernel (also phase 3 of the closure)
// -------------------------------------------------------------------------
template <class KD, int BM, int BN, int BK, int TM, int TN>
struct MulCfg {
    using E = typename KD::elem;
    static constexpr int TR = BM / TM, TC = BN / TN, THREADS = TR * TC;
    static constexpr int CH = 16 / (int)sizeof(E);
    static constexpr int NP = TN / 2;
    static constexpr int A_CHUNKS = BM * BK / CH / THREADS;
    static constexpr int B_CHUNKS = BK * BN / CH / THREADS;
    static constexpr size_t SMEM = (size_t)2 * BK * (KD::AW * BM + BN / 2) * sizeof(uint32_t);
    static_assert(TM % 4 == 0 && TN % 8 == 0, "thread tile");
    static_assert(BK % CH == 0 && BN % CH == 0, "chunking");
    static_assert(A_CHUNKS * CH * THREADS == BM * BK && B_CHUNKS * CH * THREADS == BK * BN, "chunks");
    static_assert(THREADS % 32 == 0 && BM % 32 == 0, "warps");
};

template <class KD, int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(MulCfg<KD, BM, BN, BK, TM, TN>::THREADS)
antidist_mul_kernel(MulArgs p)
{
    using Cfg = MulCfg<KD, BM, BN, BK, TM, TN>;
    using E = typename KD::elem;
    constexpr int TR = Cfg::TR, TC = Cfg::TC, THREADS = Cfg::THREADS, CH = Cfg::CH, NP = Cfg::NP;
    constexpr int BN2 = BN / 2;

    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA0 = smem;                               // [2][BK][BM]  broadcast word 0
    uint32_t *sA1 = smem + 2 * BK * BM;                 // [2][BK][BM]  broadcast word 1 (u16)
    uint32_t *sB = smem + KD::AW * 2 * BK * BM;          // [2][BK][BN/2] lane pairs

    const E *__restrict__ A = static_cast<const E *>(p.A);
    const E *__restrict__ B = static_cast<const E *>(p.B);
    E *C = static_cast<E *>(p.C);

    const int tid = threadIdx.x;
    const int tc = tid % TC, tr = tid / TC;
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;

    uint32_t acc[TM][NP];

    // ---- initial accumulator: C tile or the semiring zero
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + tr * 4 + (i % 4);
#pragma unroll
        for (int g = 0; g < NP / 4; ++g) {
            const int c = col0 + g * (8 * TC) + tc * 8;
            uint32_t q[4] = {0u, 0u, 0u, 0u};
            if (p.accumulate && r < p.R && c < p.N) {
                const int pr = remap(r, p.skip0, p.skipw), pc = remap(c, p.skip0, p.skipw);
                const E *src = C + (int64_t)pr * p.ldc + pc;
                if (sizeof(E) == 1) {
                    uint32_t w0 = 0u, w1 = 0u;
                    if (VEC && c + 8 <= p.N) {
                        uint2 v = *reinterpret_cast<const uint2 *>(src);
                        w0 = v.x; w1 = v.y;
                    } else {
                        for (int t = 0; t < 8; ++t)
                            if (c + t < p.N) {
                                uint32_t e = (uint32_t)src[t] << (8 * (t % 4));
                                if (t < 4) w0 |= e; else w1 |= e;
                            }
                    }
                    q[0] = u8x2_lo(w0); q[1] = u8x2_hi(w0); q[2] = u8x2_lo(w1); q[3] = u8x2_hi(w1);
                } else {
                    if (VEC && c + 8 <= p.N) {
                        uint4 v = *reinterpret_cast<const uint4 *>(src);
                        q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
                    } else {
                        for (int t = 0; t < 8; ++t)
                            if (c + t < p.N)
                                q[t / 2] |= (uint32_t)src[t] << (16 * (t % 2));
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                acc[i][g * 4 + u] = q[u];
        }
    }

    // ---- staging of one BK-deep k-panel: global -> registers -> shared
    uint4 ra[Cfg::A_CHUNKS], rb[Cfg::B_CHUNKS];
    auto gload = [&](int k0) {
#pragma unroll
        for (int u = 0; u < Cfg::A_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int i = ch % BM, kc = ch / BM;
            const int r = row0 + i;
            ra[u] = r < p.R ? load_chunk<E, VEC>(A, p.lda, remap(r, p.skip0, p.skipw), k0 + kc * CH,
                                                 0x7fffffff, p.K)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < Cfg::B_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int jc = ch % (BN / CH), kr = ch / (BN / CH);
            const int c = col0 + jc * CH;
            const int pc = c < p.N ? remap(c, p.skip0, p.skipw) : 0;
            // column bound checked on the logical index; the chunk never straddles the gap
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (c < p.N && k0 + kr < p.K) {
                const int lim = p.N - c;   // valid elements in this chunk
                v = load_chunk<E, VEC>(B, p.ldb, k0 + kr, pc, p.K, pc + lim);
            }
            rb[u] = v;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int u = 0; u < Cfg::A_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int i = ch % BM, kc = ch / BM;
#pragma unroll
            for (int t = 0; t < CH; ++t) {
                uint32_t a0, a1;
                KD::bcast(chunk_elem<E>(ra[u], t), a0, a1);
                const int k = kc * CH + t;
                sA0[(buf * BK + k) * BM + i] = a0;
                if (KD::AW == 2)
                    sA1[(buf * BK + k) * BM + i] = a1;
            }
        }
#pragma unroll
        for (int u = 0; u < Cfg::B_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int jc = ch % (BN / CH), kr = ch / (BN / CH);
            uint32_t *dst = sB + (buf * BK + kr) * BN2 + jc * (CH / 2);
            if (sizeof(E) == 1) {
                const uint4 v = rb[u];
                reinterpret_cast<uint4 *>(dst)[0] = make_uint4(u8x2_lo(v.x), u8x2_hi(v.x), u8x2_lo(v.y), u8x2_hi(v.y));
                reinterpret_cast<uint4 *>(dst)[1] = make_uint4(u8x2_lo(v.z), u8x2_hi(v.z), u8x2_lo(v.w), u8x2_hi(v.w));
            } else {
                reinterpret_cast<uint4 *>(dst)[0] = rb[u];
            }
        }
    };

    const int nkt = (p.K + BK - 1) / BK;
    gload(0);
    sstore(0);
    __syncthreads();

    for (int kt = 0; kt < nkt; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nkt)
            gload((kt + 1) * BK);
        const uint32_t *a0p = sA0 + buf * BK * BM + tr * 4;
        const uint32_t *a1p = sA1 + buf * BK * BM + tr * 4;
        const uint32_t *bp = sB + buf * BK * BN2 + tc * 4;
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            uint32_t a0[TM], a1[TM], b[NP];
#pragma unroll
            for (int g = 0; g < TM / 4; ++g) {
                const uint4 v = *reinterpret_cast<const uint4 *>(a0p + k * BM + g * 4 * TR);
                a0[4 * g] = v.x; a0[4 * g + 1] = v.y; a0[4 * g + 2] = v.z; a0[4 * g + 3] = v.w;
                if (KD::AW == 2) {
                    const uint4 w = *reinterpret_cast<const uint4 *>(a1p + k * BM + g * 4 * TR);
                    a1[4 * g] = w.x; a1[4 * g + 1] = w.y; a1[4 * g + 2] = w.z; a1[4 * g + 3] = w.w;
                } else {
                    a1[4 * g] = a1[4 * g + 1] = a1[4 * g + 2] = a1[4 * g + 3] = 0u;
                }
            }
#pragma unroll
            for (int g = 0; g < NP / 4; ++g) {
                const uint4 v = *reinterpret_cast<const uint4 *>(bp + k * BN2 + g * 4 * TC);
                b[4 * g] = v.x; b[4 * g + 1] = v.y; b[4 * g + 2] = v.z; b[4 * g + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < NP; ++j)
                    acc[i][j] = KD::op(acc[i][j], b[j], a0[i], a1[i]);
        }
        if (kt + 1 < nkt)
            sstore(buf ^ 1);
        __syncthreads();
    }

    // ---- epilogue
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + tr * 4 + (i % 4);
        if (r >= p.R)
            continue;
        const int pr = remap(r, p.skip0, p.skipw);
#pragma unroll
        for (int g = 0; g < NP / 4; ++g) {
            const int c = col0 + g * (8 * TC) + tc * 8;
            if (c >= p.N)
                continue;
            E *dst = C + (int64_t)pr * p.ldc + remap(c, p.skip0, p.skipw);
            const uint32_t *q = &acc[i][g * 4];
            if (sizeof(E) == 1) {
                const uint32_t w0 = pack_u8x4(q[0], q[1]), w1 = pack_u8x4(q[2], q[3]);
                if (VEC && c + 8 <= p.N) {
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(w0, w1);
                } else {
                    for (int t = 0; t < 8; ++t)
                        if (c + t < p.N)
                            dst[t] = (E)(((t < 4 ? w0 : w1) >> (8 * (t % 4))) & 0xFFu);
                }
            } else {
                if (VEC && c + 8 <= p.N) {
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
                } else {
                    for (int t = 0; t < 8; ++t)
                        if (c + t < p.N)
                            dst[t] = (E)((q[t / 2] >> (16 * (t % 2))) & 0xFFFFu);
                }
            }
        }
    }
}

// -------------------------------------------------------------------------
// Fused phases 1 + 2 of the blocked closure
// -------------------------------------------------------------------------
// 256 threads; thread (r0, c0), r0, c0 in [0,16), owns rows r0 + 16 j (j < TRN)
// and lane-pair columns c0 + 16 m (m < TCN) of a PB×PB block, so pivot kk =
// 16 j + q lives in register row j of threads r0 == q, and in register column
// m = j/2, half q&1, of threads c0 == 8 (j&1) + q/2: every register index is a
// compile-time constant while the pivot loop over q stays rolled.
template <class KD, int PB>
struct PanelCfg {
    static constexpr int TRN = PB / 16, TCN = PB / 32;
    static constexpr size_t SMEM = (size_t)KD::AW * PB * PB * 4   // sAt: [PB][PB] broadcast words
                                   + (size_t)PB * (PB / 2) * 4    // sBp: [PB][PB/2] lane pairs
                                   + 2 * (PB / 2) * 4             // rowbuf[2][PB/2]
                                   + 2 * PB * 2;                  // colbuf[2][PB] (u16)
    static_assert(PB % 32 == 0 && PB >= 32, "panel");
};

template <class KD, int PB>
__global__ void __launch_bounds__(256) antidist_panel_kernel(void *Tv, int64_t ldt, int D, int kb)
{
    using E = typename KD::elem;
    using Cfg = PanelCfg<KD, PB>;
    constexpr int TRN = Cfg::TRN, TCN = Cfg::TCN;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sAt0 = smem;                                  // [PB][PB]: row kk, slot r0*TRN + j
    uint32_t *sAt1 = smem + PB * PB;                        // second broadcast word (u16)
    uint32_t *sBp = smem + KD::AW * PB * PB;                // [PB][PB/2]: row kk, slot c0*TCN + m
    uint32_t *rowbuf = sBp + PB * (PB / 2);                 // [2][PB/2]
    uint16_t *colbuf = reinterpret_cast<uint16_t *>(rowbuf + 2 * (PB / 2));  // [2][PB]

    E *T = static_cast<E *>(Tv);
    const int tid = threadIdx.x;
    const int r0 = tid >> 4, c0 = tid & 15;
    const int nb = (D + PB - 1) / PB;
    const int k0 = kb * PB, bw = min(PB, D - k0);

    // which block this CTA updates besides the diagonal one
    int role = 0, bi = kb, bj = kb;               // 0: diagonal, 1: row panel, 2: column panel
    if (blockIdx.x >= 1 && blockIdx.x < (unsigned)nb) {
        role = 1;
        bj = (int)blockIdx.x - 1;
        if (bj >= kb) ++bj;
    } else if (blockIdx.x >= (unsigned)nb) {
        role = 2;
        bi = (int)blockIdx.x - nb;
        if (bi >= kb) ++bi;
    }

    auto load_block = [&](int i0, int j0, int h, int w, uint32_t (&R)[TRN][TCN]) {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) {
                const int r = r0 + 16 * j, c = 2 * (c0 + 16 * m);
                uint32_t v = 0u;
                if (r < h) {
                    const E *src = T + (int64_t)(i0 + r) * ldt + j0 + c;
                    if (c < w) v = (uint32_t)src[0];
                    if (c + 1 < w) v |= (uint32_t)src[1] << 16;
                }
                R[j][m] = v;
            }
    };
    auto store_block = [&](int i0, int j0, int h, int w, const uint32_t (&R)[TRN][TCN]) {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) {
                const int r = r0 + 16 * j, c = 2 * (c0 + 16 * m);
                if (r < h) {
                    E *dst = T + (int64_t)(i0 + r) * ldt + j0 + c;
                    if (c < w) dst[0] = (E)(R[j][m] & 0xFFFFu);
                    if (c + 1 < w) dst[1] = (E)(R[j][m] >> 16);
                }
            }
    };
    // A operand (entry (row, kk) broadcast) and B operand (row kk lane pairs)
    auto store_Aform = [&](const uint32_t (&R)[TRN][TCN]) {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    uint32_t a0, a1;
                    KD::bcast((R[j][m] >> (16 * h)) & 0xFFFFu, a0, a1);
                    const int kk = 2 * (c0 + 16 * m) + h;
                    sAt0[kk * PB + r0 * TRN + j] = a0;
                    if (KD::AW == 2) sAt1[kk * PB + r0 * TRN + j] = a1;
                }
    };
    auto store_Bform = [&](const uint32_t (&R)[TRN][TCN]) {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m)
                sBp[(r0 + 16 * j) * (PB / 2) + c0 * TCN + m] = R[j][m];
    };

    // ---------------- phase 1: close the diagonal block in registers
    uint32_t X[TRN][TCN];
    load_block(k0, k0, bw, bw, X);

#pragma unroll
    for (int j = 0; j < TRN; ++j) {
        for (int q = 0; q < 16; ++q) {
            const int kk = 16 * j + q;
            if (kk >= bw)
                break;
            const int par = kk & 1;
            if (r0 == q) {
#pragma unroll
                for (int m = 0; m < TCN; ++m)
                    rowbuf[par * (PB / 2) + c0 * TCN + m] = X[j][m];
            }
            if (c0 == 8 * (j & 1) + (q >> 1)) {
                const int sh = 16 * (q & 1);
#pragma unroll
                for (int jj = 0; jj < TRN; ++jj)
                    colbuf[par * PB + r0 * TRN + jj] = (uint16_t)(X[jj][j >> 1] >> sh);
            }
            __syncthreads();
            uint32_t bv[TCN];
#pragma unroll
            for (int m = 0; m < TCN; ++m)
                bv[m] = rowbuf[par * (PB / 2) + c0 * TCN + m];
#pragma unroll
            for (int jj = 0; jj < TRN; ++jj) {
                uint32_t a0, a1;
                KD::bcast(colbuf[par * PB + r0 * TRN + jj], a0, a1);
#pragma unroll
                for (int m = 0; m < TCN; ++m)
                    X[jj][m] = KD::op(X[jj][m], bv[m], a0, a1);
            }
        }
    }

    if (role == 0) {
        store_block(k0, k0, bw, bw, X);
        return;
    }

    // ---------------- phase 2: one panel block, Y := Y ⊕ T_kk ⊗ Y or Y ⊕ Y ⊗ T_kk
    const int i0 = bi * PB, j0 = bj * PB;
    const int h = min(PB, D - i0), w = min(PB, D - j0);
    uint32_t Y[TRN][TCN];
    load_block(i0, j0, h, w, Y);
    if (role == 1) {          // row panel: A = T_kk (closed), B = old Y
        store_Aform(X);
        store_Bform(Y);
    } else {                  // column panel: A = old Y, B = T_kk (closed)
        store_Aform(Y);
        store_Bform(X);
    }
    __syncthreads();
    for (int kk = 0; kk < bw; ++kk) {
        uint32_t bv[TCN], a0[TRN], a1[TRN];
#pragma unroll
        for (int m = 0; m < TCN; ++m)
            bv[m] = sBp[kk * (PB / 2) + c0 * TCN + m];
#pragma unroll
        for (int j = 0; j < TRN; ++j) {
            a0[j] = sAt0[kk * PB + r0 * TRN + j];
            a1[j] = KD::AW == 2 ? sAt1[kk * PB + r0 * TRN + j] : 0u;
        }
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m)
                Y[j][m] = KD::op(Y[j][m], bv[m], a0[j], a1[j]);
    }
    store_block(i0, j0, h, w, Y);
}

// -------------------------------------------------------------------------
// Host launchers
// -------------------------------------------------------------------------
template <class KD, int BM, int BN, int BK, int TM, int TN>
static sr_status launch_mul_cfg(const MulArgs &a, bool vec, cudaStream_t s)
{
    using Cfg = MulCfg<KD, BM, BN, BK, TM, TN>;
    dim3 grid((a.N + BN - 1) / BN, (a.R + BM - 1) / BM);
    if (grid.y > 65535u)
        return fail(SR_EINVAL, "antidist_mul: R too large for the tile grid (%d)", a.R);
    auto kern = vec ? antidist_mul_kernel<KD, BM, BN, BK, TM, TN, true>
                    : antidist_mul_kernel<KD, BM, BN, BK, TM, TN, false>;
    static bool attr_set[2][kMaxDevices] = {};
    const int dev = current_device();
    if (!attr_set[vec][dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr_set[vec][dev] = true;
    }
    kern<<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(a);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_antidist_mul(const MulArgs &a, sr_dtype dt, bool vec, cudaStream_t s)
{
    if (a.R <= 0 || a.N <= 0)
        return SR_OK;
    if (dt == SR_U8)
        return launch_mul_cfg<KindU8, 128, 128, 32, 8, 16>(a, vec, s);
    return launch_mul_cfg<KindU16, 128, 128, 32, 8, 16>(a, vec, s);
}

template <class KD, int PB>
static sr_status launch_panel(void *T, int64_t ldt, int D, int kb, cudaStream_t s)
{
    using Cfg = PanelCfg<KD, PB>;
    const int nb = (D + PB - 1) / PB;
    static bool attr[kMaxDevices] = {};
    const int dev = current_device();
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(antidist_panel_kernel<KD, PB>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr[dev] = true;
    }
    antidist_panel_kernel<KD, PB><<<2 * nb - 1, 256, Cfg::SMEM, s>>>(T, ldt, D, kb);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

template <class KD>
static sr_status closure_impl(void *T, int64_t ldt, int D, bool vec, sr_dtype dt, cudaStream_t s)
{
    constexpr int PB = 64;
    const int nb = (D + PB - 1) / PB;
    using E = typename KD::elem;
    for (int kb = 0; kb < nb; ++kb) {
        const int k0 = kb * PB, bw = std::min(PB, D - k0);
        SR_TRY((launch_panel<KD, PB>(T, ldt, D, kb, s)));
        if (nb > 1) {
            MulArgs a;
            a.A = static_cast<const E *>(T) + k0;
            a.B = static_cast<const E *>(T) + (int64_t)k0 * ldt;
            a.C = T;
            a.lda = a.ldb = a.ldc = ldt;
            a.R = a.N = D - bw;
            a.K = bw;
            a.accumulate = 1;
            a.skip0 = k0;
            a.skipw = bw;
            SR_TRY(launch_antidist_mul(a, dt, vec, s));
        }
    }
    return SR_OK;
}

sr_status launch_antidist_closure(void *T, int64_t ldt, int D, sr_dtype dt, bool vec, cudaStream_t s)
{
    if (dt == SR_U8)
        return closure_impl<KindU8>(T, ldt, D, vec, dt, s);
    return closure_impl<KindU16>(T, ldt, D, vec, dt, s);
}

// -------------------------------------------------------------------------
// Encoding: T = S − w for 0 < w < S, else 0 (Section 3)
// -------------------------------------------------------------------------
template <class E>
__global__ void antidist_encode_kernel(const E *W, int64_t ldw, E *T, int64_t ldt, int R, int C, uint32_t S)
{
    const int64_t n = (int64_t)R * C;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = t / C, c = t % C;
        const uint32_t w = W[r * ldw + c];
        T[r * ldt + c] = (E)((w == 0u || w >= S) ? 0u : S - w);
    }
}

sr_status launch_antidist_encode(const void *W, int64_t ldw, void *T, int64_t ldt, int R, int C,
                                 sr_dtype dt, int num_sms, cudaStream_t s)
{
    const int64_t n = (int64_t)R * C;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
    if (dt == SR_U8)
        antidist_encode_kernel<uint8_t><<<blocks, 256, 0, s>>>(static_cast<const uint8_t *>(W), ldw,
                                                              static_cast<uint8_t *>(T), ldt, R, C, 255u);
    else
        antidist_encode_kernel<uint16_t><<<blocks, 256, 0, s>>>(static_cast<const uint16_t *>(W), ldw,
                                                               static_cast<uint16_t *>(T), ldt, R, C, 65535u);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
