// Boolean product by the method of Four Russians (the speed-up Section 4 names for
// the product; Arlazarov, Dinic, Kronrod and Faradzev, 1970).
//
// K is cut into groups of 8 bits.  For group g the 256 possible byte values x of a
// row of A select 256 ORs of the group's 8 rows of B:
//     T_g[x] = OR over b with bit b of x set of B[8g + b]
// and the product becomes one table read and one OR per (row, group):
//     C_i |= T_g[byte g of A_i].
// So the 8 masked ORs per row and group of the plain word kernel become one lookup;
// the tables cost 256 word-ORs per group and column window, shared by every row of
// the CTA.
//
// CTA: WARPS warps, 32 rows each (BM = 32·WARPS rows) × one window of 32 words of C
// (1024 columns), lane l owning word l of the window for its warp's 32 rows.  With
// 8 warps (BM = 256) two CTAs share an SM, so one CTA's barrier waits overlap the
// other's lookups; building a table then costs as many shared-memory stores as the
// CTA's lookups read (256 entries vs 256 rows), which bounds the method here.  The
// table of group g is T[256][32] words in shared memory, double-buffered: while the
// warps read T_g, they build T_{g+1}, each warp 256/WARPS entries (the low bits of x
// from ORs of the first rows kept in registers, the high bits fixed per warp), one
// barrier per group.  A lookup reads 32 consecutive words (the warp's lanes share the
// row's byte), so table reads are free of bank conflicts.  A word of A (4 groups) is
// loaded by the lane whose index is the row's and broadcast with shuffles.
//
// Excluded row and word ranges (closure phase 3) are remapped as in the masked-OR kernel;
// the result is bit-identical to it: the Boolean product has one value.

#include <algorithm>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

__device__ __forceinline__ uint32_t m4r_word_mask(int w, int nbits)
{
    const int lo = w * 32;
    if (lo + 32 <= nbits) return 0xFFFFFFFFu;
    if (lo >= nbits) return 0u;
    return (1u << (nbits - lo)) - 1u;
}

__device__ __forceinline__ int m4r_remap(int x, int skip0, int skipw) { return x < skip0 ? x : x + skipw; }

__host__ __device__ constexpr int ilog2(int x) { return x <= 1 ? 0 : 1 + ilog2(x / 2); }
constexpr int kM4rWarps = 8;     // warps per CTA (rows per CTA: 32 per warp)

// rows 8g .. 8g+7 of B at word w (0 beyond K or outside the row)
__device__ __forceinline__ void m4r_loadB(uint32_t (&rb)[8], const uint32_t *__restrict__ B, int64_t ldb, int K,
                                          int g, int w, bool wok)
{
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int k = 8 * g + b;
        rb[b] = (wok && k < K) ? __ldg(B + (int64_t)k * ldb + w) : 0u;
    }
}

// this warp's table entries x = EPW·warp + y from the group's 8 rows of B.  Bits LB..7
// of x are fixed by the warp (H); the low LB bits are split into two halves whose
// partial ORs (lo, hi) are formed first, so each entry costs one more OR.
template <int EPW, int LB>
__device__ __forceinline__ void m4r_build(const uint32_t (&rb)[8], uint32_t *Tb, int warp, int lane)
{
    constexpr int LO = LB / 2, HI = LB - LO;
    uint32_t H = 0u;
#pragma unroll
    for (int b = LB; b < 8; ++b)
        H |= rb[b] & (0u - (uint32_t)((warp >> (b - LB)) & 1));
    uint32_t lo[1 << LO], hi[1 << HI];
#pragma unroll
    for (int y = 0; y < (1 << LO); ++y) {
        uint32_t v = 0u;
#pragma unroll
        for (int b = 0; b < LO; ++b)
            if ((y >> b) & 1) v |= rb[b];
        lo[y] = v;
    }
#pragma unroll
    for (int y = 0; y < (1 << HI); ++y) {
        uint32_t v = H;
#pragma unroll
        for (int b = 0; b < HI; ++b)
            if ((y >> b) & 1) v |= rb[LO + b];
        hi[y] = v;
    }
#pragma unroll
    for (int y = 0; y < EPW; ++y)
        Tb[(EPW * warp + y) * 32 + lane] = hi[y >> LO] | lo[y & ((1 << LO) - 1)];
}

template <int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 512 / (WARPS * 32)) bool_m4r_kernel(BoolArgs p)
{
    constexpr int EPW = 256 / WARPS;           // table entries built per warp and group
    constexpr int LB = ilog2(EPW);             // bits of x taken from the in-register partial ORs
    constexpr int TW = 256 * 32;               // words per table
    static_assert((1 << LB) == EPW && LB >= 1 && LB <= 8, "warps per CTA");
    extern __shared__ __align__(16) uint32_t T[];     // [2][256][32]

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int row0 = blockIdx.y * (32 * WARPS) + warp * 32;
    const int w = blockIdx.x * 32 + lane;                         // logical word of B and C
    const bool wok = w < p.ncw;
    const int pw = m4r_remap(w, p.skip0w, p.skipww);              // its physical word
    const int K = p.K, G = (K + 7) / 8, NKW = (K + 31) / 32;
    const uint32_t *__restrict__ Bm = p.B;
    const int64_t ldb = p.ldb;

    uint32_t acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int r = row0 + j;
        acc[j] = (p.accumulate && wok && r < p.R) ? p.C[(int64_t)m4r_remap(r, p.skip0, p.skipw) * p.ldc + pw] : 0u;
    }

    uint32_t nb[8];                              // rows of B of the next table to build
    m4r_loadB(nb, Bm, ldb, K, 0, pw, wok);
    m4r_build<EPW, LB>(nb, T, warp, lane);
    if (G > 1) m4r_loadB(nb, Bm, ldb, K, 1, pw, wok);
    const int rl = row0 + lane;                  // the row whose A words this lane loads
    const int64_t prl = m4r_remap(rl, p.skip0, p.skipw);
    uint32_t anext = (rl < p.R && NKW > 0) ? __ldg(p.A + prl * p.lda) : 0u;
    __syncthreads();

    for (int kw = 0; kw < NKW; ++kw) {
        const uint32_t amine = anext;
        if (kw + 1 < NKW)
            anext = rl < p.R ? __ldg(p.A + prl * p.lda + kw + 1) : 0u;
        uint32_t aw[32];
#pragma unroll
        for (int j = 0; j < 32; ++j)
            aw[j] = __shfl_sync(0xffffffffu, amine, j);
#pragma unroll
        for (int gb = 0; gb < 4; ++gb) {
            const int g = 4 * kw + gb;
            if (g >= G)
                break;                           // uniform across the CTA
            if (g + 1 < G) {
                m4r_build<EPW, LB>(nb, T + ((g + 1) & 1) * TW, warp, lane);
                if (g + 2 < G) m4r_loadB(nb, Bm, ldb, K, g + 2, pw, wok);
            }
            const uint32_t *Tb = T + (g & 1) * TW + lane;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                acc[j] |= Tb[__byte_perm(aw[j], 0u, 0x4440 | gb) * 32];
            __syncthreads();
        }
    }

#pragma unroll
    for (int j = 0; j < 32; ++j) {
        const int r = row0 + j;
        if (wok && r < p.R)
            p.C[(int64_t)m4r_remap(r, p.skip0, p.skipw) * p.ldc + pw] = acc[j] & m4r_word_mask(pw, p.N);
    }
}

template <int WARPS>
static sr_status launch_m4r_cfg(const BoolArgs &a, cudaStream_t s)
{
    constexpr size_t SMEM = (size_t)2 * 256 * 32 * sizeof(uint32_t);
    dim3 grid((a.ncw + 31) / 32, (a.R + 32 * WARPS - 1) / (32 * WARPS));
    if (grid.y > 65535u)
        return fail(SR_EINVAL, "bool_mul: R too large for the tile grid (%d)", a.R);
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(bool_m4r_kernel<WARPS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SMEM));
        attr[dev] = true;
    }
    bool_m4r_kernel<WARPS><<<grid, WARPS * 32, SMEM, s>>>(a);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_mul_m4r(const BoolArgs &a, cudaStream_t s)
{
    if (a.R <= 0 || a.ncw <= 0)
        return SR_OK;
    return launch_m4r_cfg<kM4rWarps>(a, s);
}

}  // namespace sr
