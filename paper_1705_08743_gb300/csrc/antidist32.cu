// u32 anti-distance matrices (S = 2^32 − 1): product kernel and pivot-block closure.
//
// The third entry type of Section 4.  a ⊗ b = max(a + b − S, 0) needs 33 bits, so
// the saturating subtraction that Section 4 builds for 32-bit lanes from a maximum
// and a plain subtraction, x ⊖ y = (x ∨ y) − y, is kept:
//     a ⊗ b = b ⊖ na,  na = S − a = ~a,
// and the subtraction is a wrapping add of −na = a + 1 (mod 2^32), fused with ⊕
// into one DPX add-max:
//     acc = max(max(b, ~a) + (a + 1), acc)            (two ALU instructions per entry)
// max(b, ~a) >= ~a, so the wrapping add gives b − na exactly when b >= na, else 0.
// An absent entry (0) is harmless on either side: a = 0 gives max(b, S) + 1 = 0,
// b = 0 gives na + (a + 1) = 0.  One entry per 32-bit register, so a u32 entry
// costs twice the issue slots of a u16 entry (two lanes per register there).
//
// The closure pipeline (phases 1-3, look-ahead on the side stream) is the one in
// antidist.cu; this file provides its two u32 kernels.

#include <algorithm>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

__device__ __forceinline__ uint32_t op32(uint32_t acc, uint32_t b, uint32_t na, uint32_t pa)
{
    return __viaddmax_u32(max(b, na), pa, acc);
}

__device__ __forceinline__ int remap32(int x, int skip0, int skipw) { return x < skip0 ? x : x + skipw; }

// entries (r, c .. c+3) of a row-major u32 matrix, zero at and beyond column ncol
template <bool VEC>
__device__ __forceinline__ uint4 load4(const uint32_t *base, int64_t ld, int r, int c, int ncol)
{
    const uint32_t *p = base + (int64_t)r * ld + c;
    if (VEC && c + 4 <= ncol)
        return *reinterpret_cast<const uint4 *>(p);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (c < ncol) v.x = p[0];
    if (c + 1 < ncol) v.y = p[1];
    if (c + 2 < ncol) v.z = p[2];
    if (c + 3 < ncol) v.w = p[3];
    return v;
}

// -------------------------------------------------------------------------
// Product kernel (also phases 2 and 3 of the closure)
// -------------------------------------------------------------------------
// One CTA per BM×BN tile of C, k-panels of depth BK double-buffered in shared memory
// (A stored k-major as the two broadcast words ~a and a + 1, B as is).  Thread (tr, tc)
// owns rows (i/4)·4·TR + 4·tr + i%4 and columns (j/4)·4·TC + 4·tc + j%4 of the tile, so
// its A and B operands of one k are 16-byte shared loads.
template <int BM, int BN, int BK, int TM, int TN>
struct Mul32Cfg {
    static constexpr int TR = BM / TM, TC = BN / TN, THREADS = TR * TC;
    static constexpr int A_CHUNKS = BM * BK / 4 / THREADS;
    static constexpr int B_CHUNKS = BK * BN / 4 / THREADS;
    static constexpr size_t SMEM = (size_t)2 * BK * (2 * BM + BN) * sizeof(uint32_t);
    static constexpr int MIN_BLOCKS = THREADS <= 128 ? 3 : 2;      // register cap: no spills
    static_assert(TM % 4 == 0 && TN % 4 == 0 && BK % 4 == 0, "thread tile");
    static_assert(A_CHUNKS * 4 * THREADS == BM * BK && B_CHUNKS * 4 * THREADS == BK * BN, "chunks");
};

template <int BM, int BN, int BK, int TM, int TN, bool VEC>
__global__ void __launch_bounds__(Mul32Cfg<BM, BN, BK, TM, TN>::THREADS, Mul32Cfg<BM, BN, BK, TM, TN>::MIN_BLOCKS)
antidist32_mul_kernel(MulArgs p)
{
    using Cfg = Mul32Cfg<BM, BN, BK, TM, TN>;
    constexpr int TR = Cfg::TR, TC = Cfg::TC, THREADS = Cfg::THREADS;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sAn = smem;                    // [2][BK][BM]  ~a
    uint32_t *sAp = smem + 2 * BK * BM;      // [2][BK][BM]  a + 1
    uint32_t *sB = smem + 4 * BK * BM;       // [2][BK][BN]

    const uint32_t *__restrict__ A = static_cast<const uint32_t *>(p.A);
    const uint32_t *__restrict__ B = static_cast<const uint32_t *>(p.B);
    uint32_t *C = static_cast<uint32_t *>(p.C);

    static_assert(128 % BM == 0 && 128 % BN == 0, "tiles nest in the 128x128 grid of skip_tile");
    const int tile = blockIdx.x;
    const int tid = threadIdx.x, tc = tid % TC, tr = tid / TC;
    const int tiles_n = (p.N + BN - 1) / BN, tiles_m = (p.R + BM - 1) / BM;
    int trow = tile / tiles_n, tcol = tile % tiles_n;
    if (p.group_m > 0) {             // column-major inside groups of group_m tile rows (A's panels reused from L2)
        const int per = p.group_m * tiles_n, g0 = (tile / per) * p.group_m, gm = min(p.group_m, tiles_m - g0);
        trow = g0 + (tile % per) % gm;
        tcol = (tile % per) / gm;
    }
    const int row0 = trow * BM, col0 = tcol * BN;
    if (p.skip_tile >= 0) {          // skip_tile indexes the 128x128 tile grid
        const int tn128 = (p.N + 127) / 128;
        if (row0 / 128 == p.skip_tile / tn128 && col0 / 128 == p.skip_tile % tn128)
            return;
    }
    const int nkt = (p.K + BK - 1) / BK;

    uint4 ra[Cfg::A_CHUNKS], rb[Cfg::B_CHUNKS];
    auto gload = [&](int k0) {
#pragma unroll
        for (int u = 0; u < Cfg::A_CHUNKS; ++u) {
            const int ch = tid + u * THREADS, i = ch % BM, kc = ch / BM;
            const int r = row0 + i;
            ra[u] = r < p.R ? load4<VEC>(A, p.lda, remap32(r, p.rskip0, p.rskipw), k0 + 4 * kc, p.K)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < Cfg::B_CHUNKS; ++u) {
            const int ch = tid + u * THREADS, jc = ch % (BN / 4), kr = ch / (BN / 4);
            const int c = col0 + 4 * jc;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (c < p.N && k0 + kr < p.K) {      // a 4-entry chunk never straddles an excluded range
                const int pc = remap32(c, p.cskip0, p.cskipw);
                v = load4<VEC>(B, p.ldb, k0 + kr, pc, pc + (p.N - c));
            }
            rb[u] = v;
        }
    };
    auto sstore = [&](int buf) {
#pragma unroll
        for (int u = 0; u < Cfg::A_CHUNKS; ++u) {
            const int ch = tid + u * THREADS, i = ch % BM, kc = ch / BM;
            const uint32_t v[4] = {ra[u].x, ra[u].y, ra[u].z, ra[u].w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int k = 4 * kc + t;
                sAn[(buf * BK + k) * BM + i] = ~v[t];
                sAp[(buf * BK + k) * BM + i] = v[t] + 1u;
            }
        }
#pragma unroll
        for (int u = 0; u < Cfg::B_CHUNKS; ++u) {
            const int ch = tid + u * THREADS, jc = ch % (BN / 4), kr = ch / (BN / 4);
            *reinterpret_cast<uint4 *>(sB + (buf * BK + kr) * BN + 4 * jc) = rb[u];
        }
    };

    gload(0);

    uint32_t acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + 4 * tr + (i % 4);
#pragma unroll
        for (int g = 0; g < TN / 4; ++g) {
            const int c = col0 + g * (4 * TC) + 4 * tc;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (p.accumulate && r < p.R && c < p.N) {
                const int pc = remap32(c, p.cskip0, p.cskipw);
                v = load4<VEC>(C, p.ldc, remap32(r, p.rskip0, p.rskipw), pc, pc + (p.N - c));
            }
            acc[i][4 * g] = v.x; acc[i][4 * g + 1] = v.y; acc[i][4 * g + 2] = v.z; acc[i][4 * g + 3] = v.w;
        }
    }

    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nkt; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nkt)
            gload((kt + 1) * BK);
        const uint32_t *anp = sAn + buf * BK * BM + 4 * tr;
        const uint32_t *app = sAp + buf * BK * BM + 4 * tr;
        const uint32_t *bp = sB + buf * BK * BN + 4 * tc;
#pragma unroll 4
        for (int k = 0; k < BK; ++k) {
            uint32_t na[TM], pa[TM], b[TN];
#pragma unroll
            for (int g = 0; g < TM / 4; ++g) {
                const uint4 v = *reinterpret_cast<const uint4 *>(anp + k * BM + g * 4 * TR);
                const uint4 w = *reinterpret_cast<const uint4 *>(app + k * BM + g * 4 * TR);
                na[4 * g] = v.x; na[4 * g + 1] = v.y; na[4 * g + 2] = v.z; na[4 * g + 3] = v.w;
                pa[4 * g] = w.x; pa[4 * g + 1] = w.y; pa[4 * g + 2] = w.z; pa[4 * g + 3] = w.w;
            }
#pragma unroll
            for (int g = 0; g < TN / 4; ++g) {
                const uint4 v = *reinterpret_cast<const uint4 *>(bp + k * BN + g * 4 * TC);
                b[4 * g] = v.x; b[4 * g + 1] = v.y; b[4 * g + 2] = v.z; b[4 * g + 3] = v.w;
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j)
                    acc[i][j] = op32(acc[i][j], b[j], na[i], pa[i]);
        }
        if (kt + 1 < nkt)
            sstore(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + 4 * tr + (i % 4);
        if (r >= p.R)
            continue;
        const int pr = remap32(r, p.rskip0, p.rskipw);
#pragma unroll
        for (int g = 0; g < TN / 4; ++g) {
            const int c = col0 + g * (4 * TC) + 4 * tc;
            if (c >= p.N)
                continue;
            uint32_t *dst = C + (int64_t)pr * p.ldc + remap32(c, p.cskip0, p.cskipw);
            const uint32_t *q = &acc[i][4 * g];
            if (VEC && c + 4 <= p.N) {
                *reinterpret_cast<uint4 *>(dst) = make_uint4(q[0], q[1], q[2], q[3]);
            } else {
                for (int t = 0; t < 4; ++t)
                    if (c + t < p.N) dst[t] = q[t];
            }
        }
    }
}

template <int BM, int BN, int BK, int TM, int TN>
static sr_status launch_mul32_cfg(const MulArgs &a, bool vec, cudaStream_t s)
{
    using Cfg = Mul32Cfg<BM, BN, BK, TM, TN>;
    const int64_t tiles = (int64_t)((a.N + BN - 1) / BN) * ((a.R + BM - 1) / BM);
    if (tiles > 0x7fffffffLL)
        return fail(SR_EINVAL, "antidist_mul: too many tiles (%lld)", (long long)tiles);
    auto kern = vec ? antidist32_mul_kernel<BM, BN, BK, TM, TN, true> : antidist32_mul_kernel<BM, BN, BK, TM, TN, false>;
    static bool attr[2][kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[vec][dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr[vec][dev] = true;
    }
    kern<<<(unsigned)tiles, Cfg::THREADS, Cfg::SMEM, s>>>(a);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_antidist32_mul(const MulArgs &a, bool vec, cudaStream_t s, int tiles)
{
    if (a.R <= 0 || a.N <= 0)
        return SR_OK;
    if (tiles == 1)              // thin panels (closure phase 2)
        return launch_mul32_cfg<64, 64, 16, 4, 4>(a, vec, s);
    return launch_mul32_cfg<128, 64, 8, 8, 8>(a, vec, s);
}

// -------------------------------------------------------------------------
// Phase 1 of the blocked closure: one PB×PB pivot block closed in registers
// -------------------------------------------------------------------------
// One CTA of 256 threads; thread (r0, c0), r0, c0 in [0, 16), holds entries
// (r0 + 16 j, c0 + 16 m) for j, m < PB/16.  Pivot kk = 16 j + q is register row j of
// the threads with r0 == q and register column j of the threads with c0 == q, so every
// register index is a compile-time constant while the loop over q stays rolled.  The
// pivot row and column go through double-buffered shared rows, one barrier per pivot.
// With kprev >= 0 the block first takes its phase-3 update from the previous pivot
// block, T_kk ⊕= T_k,prev ⊗ T_prev,k.
template <int PB>
struct Pivot32Cfg {
    static constexpr int RN = PB / 16;
    static constexpr int LDA = PB + 1;                              // padded: transposed stores
    static constexpr size_t SMEM = ((size_t)PB * LDA + (size_t)PB * PB + 4 * PB) * sizeof(uint32_t);
    static_assert(PB % 16 == 0, "pivot block");
};

template <int PB>
__global__ void __launch_bounds__(256) antidist32_pivot_kernel(uint32_t *T, int64_t ldt, int D, int kb, int kprev)
{
    using Cfg = Pivot32Cfg<PB>;
    constexpr int RN = Cfg::RN, LDA = Cfg::LDA;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA = smem;                      // [PB][LDA]: sA[k][r] = T[block kb row r][block prev col k]
    uint32_t *sB = sA + PB * LDA;             // [PB][PB]:  sB[k][c] = T[block prev row k][block kb col c]
    uint32_t *rowbuf = sB + PB * PB;          // [2][PB]
    uint32_t *colbuf = rowbuf + 2 * PB;       // [2][PB]

    const int tid = threadIdx.x, r0 = tid >> 4, c0 = tid & 15;
    const int k0 = kb * PB, bw = min(PB, D - k0);

    uint32_t X[RN][RN];
#pragma unroll
    for (int j = 0; j < RN; ++j)
#pragma unroll
        for (int m = 0; m < RN; ++m) {
            const int r = r0 + 16 * j, c = c0 + 16 * m;
            X[j][m] = (r < bw && c < bw) ? T[(int64_t)(k0 + r) * ldt + k0 + c] : 0u;
        }

    if (kprev >= 0) {
        const int p0 = kprev * PB, pw = min(PB, D - p0);
        for (int e = tid; e < PB * PB; e += 256) {
            const int r = e / PB, k = e % PB;         // coalesced along the row of T
            sA[k * LDA + r] = (r < bw && k < pw) ? T[(int64_t)(k0 + r) * ldt + p0 + k] : 0u;
            const int kr = e / PB, c = e % PB;
            sB[kr * PB + c] = (kr < pw && c < bw) ? T[(int64_t)(p0 + kr) * ldt + k0 + c] : 0u;
        }
        __syncthreads();
        for (int k = 0; k < pw; ++k) {
            uint32_t b[RN], na[RN], pa[RN];
#pragma unroll
            for (int m = 0; m < RN; ++m) b[m] = sB[k * PB + c0 + 16 * m];
#pragma unroll
            for (int j = 0; j < RN; ++j) {
                const uint32_t a = sA[k * LDA + r0 + 16 * j];
                na[j] = ~a;
                pa[j] = a + 1u;
            }
#pragma unroll
            for (int j = 0; j < RN; ++j)
#pragma unroll
                for (int m = 0; m < RN; ++m) X[j][m] = op32(X[j][m], b[m], na[j], pa[j]);
        }
    }

#pragma unroll
    for (int j = 0; j < RN; ++j) {
        for (int q = 0; q < 16; ++q) {
            const int kk = 16 * j + q;
            if (kk >= bw)
                break;
            const int par = kk & 1;
            if (r0 == q) {
#pragma unroll
                for (int m = 0; m < RN; ++m) rowbuf[par * PB + c0 + 16 * m] = X[j][m];
            }
            if (c0 == q) {
#pragma unroll
                for (int jj = 0; jj < RN; ++jj) colbuf[par * PB + r0 + 16 * jj] = X[jj][j];
            }
            __syncthreads();
            uint32_t b[RN];
#pragma unroll
            for (int m = 0; m < RN; ++m) b[m] = rowbuf[par * PB + c0 + 16 * m];
#pragma unroll
            for (int jj = 0; jj < RN; ++jj) {
                const uint32_t a = colbuf[par * PB + r0 + 16 * jj];
                const uint32_t na = ~a, pa = a + 1u;
#pragma unroll
                for (int m = 0; m < RN; ++m) X[jj][m] = op32(X[jj][m], b[m], na, pa);
            }
        }
    }

#pragma unroll
    for (int j = 0; j < RN; ++j)
#pragma unroll
        for (int m = 0; m < RN; ++m) {
            const int r = r0 + 16 * j, c = c0 + 16 * m;
            if (r < bw && c < bw) T[(int64_t)(k0 + r) * ldt + k0 + c] = X[j][m];
        }
}

sr_status launch_antidist32_pivot(void *T, int64_t ldt, int D, int kb, int kprev, cudaStream_t s)
{
    constexpr int PB = 128;
    using Cfg = Pivot32Cfg<PB>;
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(antidist32_pivot_kernel<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)Cfg::SMEM));
        attr[dev] = true;
    }
    antidist32_pivot_kernel<PB><<<1, 256, Cfg::SMEM, s>>>(static_cast<uint32_t *>(T), ldt, D, kb, kprev);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
