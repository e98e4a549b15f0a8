// Boolean semiring product and closure on bit-packed rows (Section 2; Section 4 matBool).
//
// Entry (i, j) is bit (j mod 32) of 32-bit word floor(j / 32) of row i (a
// 64-bit-word matrix is the same bits, two 32-bit words per 64-bit word).
//
// Product C := (accumulate ? C : 0) ⊕ A ⊗ B: for every k with A_ik = 1, row k
// of B is ORed into row i of C, 32 columns per word operation (the matBool
// listing does the same with 64-bit blocks).  Each CTA owns a BM×BNW-word tile
// of C in registers; k-panels of A (words) and B (rows of words) arrive in
// shared memory by cp.async; per k a thread expands bit k of each of its TM
// rows of A to an all-ones/all-zeros mask and ORs (B word AND mask) into its
// TNW accumulator words.
//
// Closure: the same three-phase blocked Warshall as the anti-distance closure
// (antidist.cu), with PB-bit blocks.

#include <algorithm>

#include "sr_common.cuh"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {

__device__ __forceinline__ int bremap(int x, int skip0, int skipw) { return x < skip0 ? x : x + skipw; }

// valid-bit mask of physical word w of a row with nbits logical bits
__device__ __forceinline__ uint32_t word_mask(int w, int nbits)
{
    const int lo = w * 32;
    if (lo + 32 <= nbits) return 0xFFFFFFFFu;
    if (lo >= nbits) return 0u;
    return (1u << (nbits - lo)) - 1u;
}

__device__ __forceinline__ void cp_async16(void *smem_ptr, const void *gptr, bool valid)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem_ptr);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gptr), "r"(n));
}
__device__ __forceinline__ void cp_async4(void *smem_ptr, const void *gptr, bool valid)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem_ptr);
    const int n = valid ? 4 : 0;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gptr), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// -------------------------------------------------------------------------
// Product kernel (also phase 3 of the closure)
// -------------------------------------------------------------------------
template <int BM, int BNW, int BKW, int TM, int TNW>
struct BoolCfg {
    static constexpr int TR = BM / TM, TC = BNW / TNW, THREADS = TR * TC;
    static constexpr int BKB = BKW * 32;
    static constexpr size_t SMEM = (size_t)2 * (BKW * BM + BKB * BNW) * sizeof(uint32_t);
    // K within one k-tile (closure panels and phase 3): the second B buffer is never used
    static constexpr size_t SMEM_ONE = (size_t)(2 * BKW * BM + BKB * BNW) * sizeof(uint32_t);
    static_assert(TM % 4 == 0 && TNW % 4 == 0, "vector groups");
    static_assert(THREADS % 32 == 0, "warps");
};

template <int BM, int BNW, int BKW, int TM, int TNW, bool VEC>
__global__ void __launch_bounds__(BoolCfg<BM, BNW, BKW, TM, TNW>::THREADS)
bool_mul_kernel(BoolArgs p)
{
    using Cfg = BoolCfg<BM, BNW, BKW, TM, TNW>;
    constexpr int TR = Cfg::TR, TC = Cfg::TC, THREADS = Cfg::THREADS, BKB = Cfg::BKB;
    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA = smem;                         // [2][BKW][BM]  (word kw of each row; transposed)
    uint32_t *sB = smem + 2 * BKW * BM;          // [2][BKB][BNW]

    const int tid = threadIdx.x;
    const int tc = tid % TC, tr = tid / TC;
    const int row0 = blockIdx.y * BM, w0 = blockIdx.x * BNW;
    const int kwords = (p.K + 31) / 32;          // words of A rows holding bits < K

    uint32_t acc[TM][TNW];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + tr * 4 + (i % 4);
#pragma unroll
        for (int u = 0; u < TNW; ++u) {
            const int w = w0 + (u / 4) * (4 * TC) + tc * 4 + (u % 4);
            uint32_t v = 0u;
            if (p.accumulate && p.ksplit == 1 && r < p.R && w < p.ncw)
                v = p.C[(int64_t)bremap(r, p.skip0, p.skipw) * p.ldc + bremap(w, p.skip0w, p.skipww)];
            acc[i][u] = v;
        }
    }

    // A tile: BM rows × BKW words, stored transposed; B tile: BKB rows × BNW words
    auto stage = [&](int kt, int buf) {
        const int kw0 = kt * BKW;
        // A: one thread per (row, word); bits >= K are masked when read
        for (int t = tid; t < BM * BKW; t += THREADS) {
            const int i = t % BM, e = t / BM;
            const int r = row0 + i, kw = kw0 + e;
            const bool ok = r < p.R && kw < kwords;
            const uint32_t *src = p.A + (ok ? (int64_t)bremap(r, p.skip0, p.skipw) * p.lda + kw : 0);
            uint32_t *dst = sA + (buf * BKW + e) * BM + i;
            if (VEC)
                cp_async4(dst, src, ok);
            else
                *dst = ok ? *src : 0u;
        }
        // B: rows k of B, groups of 4 words
        for (int t = tid; t < BKB * (BNW / 4); t += THREADS) {
            const int g = t % (BNW / 4), kr = t / (BNW / 4);
            const int k = kt * BKB + kr;
            const int w = w0 + g * 4;
            uint32_t *dst = sB + (buf * BKB + kr) * BNW + g * 4;
            const bool rowok = k < p.K;
            if (VEC) {
                // the 4-word group never straddles the excluded range (multiples of 4 words)
                const uint32_t *src = p.B + (int64_t)(rowok ? k : 0) * p.ldb + bremap(w < p.ncw ? w : 0, p.skip0w, p.skipww);
                cp_async16(dst, src, rowok && w < p.ncw);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    uint32_t v = 0u;
                    if (rowok && w + e < p.ncw)
                        v = p.B[(int64_t)k * p.ldb + bremap(w + e, p.skip0w, p.skipww)];
                    dst[e] = v;
                }
            }
        }
        if (VEC) cp_async_commit();
    };

    // split-K: CTA z of ksplit takes k-tiles [kt0, kt1) and ORs its partial result into C
    const int nkt_all = (p.K + BKB - 1) / BKB, per = (nkt_all + p.ksplit - 1) / p.ksplit;
    const int kt0 = blockIdx.z * per, nkt = min(nkt_all, kt0 + per);
    if (kt0 < nkt) stage(kt0, 0);
    for (int kt = kt0; kt < nkt; ++kt) {
        const int buf = (kt - kt0) & 1;
        if (VEC) cp_async_wait<0>();
        __syncthreads();
        if (kt + 1 < nkt)
            stage(kt + 1, buf ^ 1);
        const uint32_t *ap = sA + buf * BKW * BM + tr * 4;
        const uint32_t *bp = sB + buf * BKB * BNW + tc * 4;
#pragma unroll 1
        for (int kw = 0; kw < BKW; ++kw) {
            uint32_t a[TM];
#pragma unroll
            for (int g = 0; g < TM / 4; ++g) {
                const uint4 v = *reinterpret_cast<const uint4 *>(ap + kw * BM + g * 4 * TR);
                a[4 * g] = v.x; a[4 * g + 1] = v.y; a[4 * g + 2] = v.z; a[4 * g + 3] = v.w;
            }
            const uint32_t km = word_mask(kt * BKW + kw, p.K);
#pragma unroll
            for (int i = 0; i < TM; ++i)
                a[i] &= km;
#pragma unroll 8
            for (int bit = 0; bit < 32; ++bit) {
                uint32_t b[TNW];
                const uint32_t *brow = bp + (kw * 32 + bit) * BNW;
#pragma unroll
                for (int g = 0; g < TNW / 4; ++g) {
                    const uint4 v = *reinterpret_cast<const uint4 *>(brow + g * 4 * TC);
                    b[4 * g] = v.x; b[4 * g + 1] = v.y; b[4 * g + 2] = v.z; b[4 * g + 3] = v.w;
                }
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    const uint32_t m = (uint32_t)((int32_t)(a[i] << (31 - bit)) >> 31);
#pragma unroll
                    for (int u = 0; u < TNW; ++u)
                        acc[i][u] |= b[u] & m;
                }
            }
        }
        // the next iteration's barrier orders these reads before the next overwrite
        // of this buffer (which is issued only after that barrier)
    }

#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i / 4) * (4 * TR) + tr * 4 + (i % 4);
        if (r >= p.R)
            continue;
        uint32_t *dst = p.C + (int64_t)bremap(r, p.skip0, p.skipw) * p.ldc;
#pragma unroll
        for (int u = 0; u < TNW; ++u) {
            const int w = w0 + (u / 4) * (4 * TC) + tc * 4 + (u % 4);
            if (w < p.ncw) {
                const int pw = bremap(w, p.skip0w, p.skipww);
                const uint32_t m = word_mask(pw, p.N), v = acc[i][u] & m;
                if (p.ksplit == 1) {
                    dst[pw] = v;
                } else {
                    // OR is idempotent: partial products combine in any order.  No CTA sets a
                    // pad bit, so clearing them (z = 0) commutes with the other CTAs' ORs.
                    if (blockIdx.z == 0 && m != 0xffffffffu) atomicAnd(dst + pw, m);
                    if (v) atomicOr(dst + pw, v);
                }
            }
        }
    }
}

// -------------------------------------------------------------------------
// Fused phases 1 + 2 of the Boolean blocked closure: PB rows per block, one
// thread per row holding its PB/32 words.
// -------------------------------------------------------------------------
template <int PB>
__global__ void __launch_bounds__(PB) bool_panel_kernel(uint32_t *T, int64_t ldt, int D, int rw, int kb)
{
    constexpr int PW = PB / 32;
    __shared__ __align__(16) uint32_t sB[PB][PW];
    __shared__ __align__(16) uint32_t rowbuf[2][PW];
    const int i = threadIdx.x;
    const int nb = (D + PB - 1) / PB;
    const int k0 = kb * PB, bw = min(PB, D - k0);
    const int kw0 = k0 / 32;

    int role = 0, bi = kb, bj = kb;
    if (blockIdx.x >= 1 && blockIdx.x < (unsigned)nb) {
        role = 1; bj = (int)blockIdx.x - 1; if (bj >= kb) ++bj;
    } else if (blockIdx.x >= (unsigned)nb) {
        role = 2; bi = (int)blockIdx.x - nb; if (bi >= kb) ++bi;
    }

    // block words: rows [r0, r0+h), words [c0w, c0w + nw) with valid bits up to D
    auto load_row = [&](int r0, int h, int c0w, uint32_t (&R)[PW]) {
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            uint32_t v = 0u;
            if (i < h && c0w + u < rw)
                v = T[(int64_t)(r0 + i) * ldt + c0w + u] & word_mask(c0w + u, D);
            R[u] = v;
        }
    };
    auto store_row = [&](int r0, int h, int c0w, const uint32_t (&R)[PW]) {
        if (i >= h) return;
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if (c0w + u < rw)
                T[(int64_t)(r0 + i) * ldt + c0w + u] = R[u] & word_mask(c0w + u, D);
    };

    // phase 1: Warshall on the diagonal block; pivot kk = 32 w + b
    uint32_t X[PW];
    load_row(k0, bw, kw0, X);
#pragma unroll
    for (int w = 0; w < PW; ++w) {
        for (int b = 0; b < 32; ++b) {
            const int kk = 32 * w + b;
            if (kk >= bw)
                break;
            const int par = kk & 1;
            if (i == kk) {
#pragma unroll
                for (int u = 0; u < PW; ++u) rowbuf[par][u] = X[u];
            }
            __syncthreads();
            const uint32_t m = (uint32_t)((int32_t)(X[w] << (31 - b)) >> 31);
#pragma unroll
            for (int u = 0; u < PW; ++u) X[u] |= rowbuf[par][u] & m;
        }
    }
    if (role == 0) {
        store_row(k0, bw, kw0, X);
        return;
    }

    // phase 2
    const int r0 = bi * PB, h = min(PB, D - r0);
    const int c0w = bj * PW;
    uint32_t Y[PW], Arow[PW];
    load_row(r0, h, c0w, Y);
    if (role == 1) {            // Y := Y ⊕ T_kk ⊗ Y : A row = X (closed pivot block), B = old Y
#pragma unroll
        for (int u = 0; u < PW; ++u) { sB[i][u] = Y[u]; Arow[u] = X[u]; }
    } else {                    // Y := Y ⊕ Y ⊗ T_kk : A row = old Y, B = X
#pragma unroll
        for (int u = 0; u < PW; ++u) { sB[i][u] = X[u]; Arow[u] = Y[u]; }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < PW; ++w) {
        for (int b = 0; b < 32; ++b) {
            const int kk = 32 * w + b;
            if (kk >= bw) break;
            const uint32_t m = (uint32_t)((int32_t)(Arow[w] << (31 - b)) >> 31);
#pragma unroll
            for (int u = 0; u < PW; ++u) Y[u] |= sB[kk][u] & m;
        }
    }
    store_row(r0, h, c0w, Y);
}

// -------------------------------------------------------------------------
// Encoding helpers
// -------------------------------------------------------------------------
// one warp per (row, word): lane l reads column 32 w + l, ballot packs the word
// four bytes -> four bits (byte j nonzero -> bit j)
__device__ __forceinline__ uint32_t pack_nibble(uint32_t x)
{
    const uint32_t m = __vcmpne4(x, 0u) & 0x01010101u;       // bit 8j = [byte j != 0]
    return (m | (m >> 7) | (m >> 14) | (m >> 21)) & 0xFu;
}

// one thread per 32-bit word of M: 32 dense bytes (two 16-byte loads when the row start
// and leading dimension allow) -> 32 bits, LSB first
__global__ void bool_pack_kernel(const uint8_t *dense, int64_t ldd, uint32_t *M, int64_t ldm, int R, int C, int rw,
                                 bool vec)
{
    const int64_t total = (int64_t)R * rw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / rw), w = (int)(t % rw);
        const int c0 = 32 * w;
        const uint8_t *src = dense + (int64_t)r * ldd + c0;
        uint32_t word = 0u;
        if (vec && c0 + 32 <= C) {
            const uint4 a = *reinterpret_cast<const uint4 *>(src), b = *reinterpret_cast<const uint4 *>(src + 16);
            word = pack_nibble(a.x) | pack_nibble(a.y) << 4 | pack_nibble(a.z) << 8 | pack_nibble(a.w) << 12 |
                   pack_nibble(b.x) << 16 | pack_nibble(b.y) << 20 | pack_nibble(b.z) << 24 | pack_nibble(b.w) << 28;
        } else {
            for (int j = 0; j < 32 && c0 + j < C; ++j)
                word |= (src[j] != 0 ? 1u : 0u) << j;
        }
        M[(int64_t)r * ldm + w] = word;
    }
}

// four bits -> four bytes 0/1 (bit j -> byte j)
__device__ __forceinline__ uint32_t unpack_nibble(uint32_t n)
{
    return (n & 1u) | ((n & 2u) << 7) | ((n & 4u) << 14) | ((n & 8u) << 21);
}

// one thread per 32-bit word of M -> 32 dense bytes (two 16-byte stores when aligned)
__global__ void bool_unpack_kernel(const uint32_t *M, int64_t ldm, uint8_t *dense, int64_t ldd, int R, int C, int rw,
                                   bool vec)
{
    const int64_t total = (int64_t)R * rw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / rw), w = (int)(t % rw);
        const int c0 = 32 * w;
        if (c0 >= C) continue;
        const uint32_t word = M[(int64_t)r * ldm + w];
        uint8_t *dst = dense + (int64_t)r * ldd + c0;
        if (vec && c0 + 32 <= C) {
            uint32_t o[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = unpack_nibble((word >> (4 * q)) & 0xFu);
            reinterpret_cast<uint4 *>(dst)[0] = make_uint4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<uint4 *>(dst)[1] = make_uint4(o[4], o[5], o[6], o[7]);
        } else {
            for (int j = 0; j < 32 && c0 + j < C; ++j)
                dst[j] = (uint8_t)((word >> j) & 1u);
        }
    }
}

__global__ void bool_identity_or_kernel(uint32_t *M, int64_t ldm, int D)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < D; i += gridDim.x * blockDim.x)
        M[(int64_t)i * ldm + i / 32] |= 1u << (i % 32);
}

__global__ void copy_rows_kernel(const uint32_t *src, int64_t lds, uint32_t *dst, int64_t ldd, int R, int rw)
{
    const int64_t total = (int64_t)R * rw;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / rw), w = (int)(t % rw);
        dst[(int64_t)r * ldd + w] = src[(int64_t)r * lds + w];
    }
}

// zero the pad bits of every row (bits >= D) so the closure's invariant holds
__global__ void bool_clear_pad_kernel(uint32_t *M, int64_t ldm, int R, int D, int rw)
{
    const int w0 = D / 32;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        for (int w = w0; w < rw; ++w)
            M[(int64_t)r * ldm + w] &= word_mask(w, D);
}

// -------------------------------------------------------------------------
// Host launchers
// -------------------------------------------------------------------------
template <int BM, int BNW, int BKW, int TM, int TNW>
static sr_status launch_bool_cfg(const BoolArgs &a, bool vec, cudaStream_t s)
{
    using Cfg = BoolCfg<BM, BNW, BKW, TM, TNW>;
    dim3 grid((a.ncw + BNW - 1) / BNW, (a.R + BM - 1) / BM, a.ksplit);
    if (grid.y > 65535u)
        return fail(SR_EINVAL, "bool_mul: R too large for the tile grid (%d)", a.R);
    auto kern = vec ? bool_mul_kernel<BM, BNW, BKW, TM, TNW, true> : bool_mul_kernel<BM, BNW, BKW, TM, TNW, false>;
    static bool attr[2][kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[vec][dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        attr[vec][dev] = true;
    }
    kern<<<grid, Cfg::THREADS, a.K <= Cfg::BKB ? Cfg::SMEM_ONE : Cfg::SMEM, s>>>(a);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_mul(const BoolArgs &in, bool vec, cudaStream_t s, int shape)
{
    if (in.R <= 0 || in.ncw <= 0)
        return SR_OK;
    BoolArgs a = in;
    a.ksplit = 1;
    if (shape == 0) {
        // few output tiles (small products): narrower tiles, then split K across CTAs
        const bool plain = a.skipww == 0 && a.skipw == 0;
        if (a.ncw <= 16 && plain) shape = 2;
        const int bm = shape == 2 ? 32 : 128, bnw = shape == 2 ? 16 : 64;
        const int64_t tiles = (int64_t)((a.ncw + bnw - 1) / bnw) * ((a.R + bm - 1) / bm);
        const int nkt = (a.K + 127) / 128, sms = device_sm_count();
        if (plain && tiles < sms && nkt >= 2) {
            a.ksplit = (int)std::min<int64_t>(nkt, (2 * sms + tiles - 1) / tiles);
            if (!a.accumulate)          // partial results are ORed into a zeroed C
                SR_CUDA_CHECK(cudaMemset2DAsync(a.C, (size_t)a.ldc * 4, 0, (size_t)a.ncw * 4, (size_t)a.R, s));
        }
    }
    if (shape == 1)          // panels a few words wide: 128 rows x 4 words per CTA
        return launch_bool_cfg<128, 4, 4, 4, 4>(a, vec, s);
    if (shape == 2)          // panels a few rows high: 32 rows x 16 words per CTA
        return launch_bool_cfg<32, 16, 4, 4, 4>(a, vec, s);
    return launch_bool_cfg<128, 64, 4, 4, 16>(a, vec, s);
}

// Phase 1 of the pipelined Boolean closure: one CTA, one thread per row of the
// PB-bit pivot block.  With kprev >= 0 the block first receives its phase-3
// update from the previous pivot block: X := X ⊕ T[k rows][prev cols] ⊗ T[prev rows][k cols].
template <int PB>
__global__ void __launch_bounds__(PB) bool_pivot_kernel(uint32_t *T, int64_t ldt, int D, int rw, int kb, int kprev)
{
    constexpr int PW = PB / 32;
    __shared__ __align__(16) uint32_t sB[PB][PW];
    __shared__ __align__(16) uint32_t rowbuf[2][PW];
    const int i = threadIdx.x;
    const int k0 = kb * PB, bw = min(PB, D - k0), kw0 = k0 / 32;
    uint32_t X[PW];
#pragma unroll
    for (int u = 0; u < PW; ++u)
        X[u] = (i < bw && kw0 + u < rw) ? T[(int64_t)(k0 + i) * ldt + kw0 + u] & word_mask(kw0 + u, D) : 0u;
    if (kprev >= 0) {
        const int p0 = kprev * PB, pw0 = p0 / 32;       // the previous block is a full block
        uint32_t Arow[PW];
#pragma unroll
        for (int u = 0; u < PW; ++u) {
            Arow[u] = i < bw ? T[(int64_t)(k0 + i) * ldt + pw0 + u] : 0u;
            sB[i][u] = kw0 + u < rw ? T[(int64_t)(p0 + i) * ldt + kw0 + u] & word_mask(kw0 + u, D) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int w = 0; w < PW; ++w)
            for (int b = 0; b < 32; ++b) {
                const uint32_t m = (uint32_t)((int32_t)(Arow[w] << (31 - b)) >> 31);
#pragma unroll
                for (int u = 0; u < PW; ++u) X[u] |= sB[32 * w + b][u] & m;
            }
    }
#pragma unroll
    for (int w = 0; w < PW; ++w) {
        for (int b = 0; b < 32; ++b) {
            const int kk = 32 * w + b;
            if (kk >= bw) break;
            const int par = kk & 1;
            if (i == kk) {
#pragma unroll
                for (int u = 0; u < PW; ++u) rowbuf[par][u] = X[u];
            }
            __syncthreads();
            const uint32_t m = (uint32_t)((int32_t)(X[w] << (31 - b)) >> 31);
#pragma unroll
            for (int u = 0; u < PW; ++u) X[u] |= rowbuf[par][u] & m;
        }
    }
    if (i < bw) {
#pragma unroll
        for (int u = 0; u < PW; ++u)
            if (kw0 + u < rw)
                T[(int64_t)(k0 + i) * ldt + kw0 + u] = X[u] & word_mask(kw0 + u, D);
    }
}

static BoolArgs bool_args(const uint32_t *A, const uint32_t *B, uint32_t *C, int64_t ld, int R, int K, int N, int ncw)
{
    BoolArgs a;
    a.A = A; a.B = B; a.C = C;
    a.lda = a.ldb = a.ldc = ld;
    a.R = R; a.K = K; a.N = N;
    a.ncw = ncw;
    a.accumulate = 1;
    a.skip0 = 0x7fffffff; a.skipw = 0;
    a.skip0w = 0x7fffffff; a.skipww = 0;
    return a;
}

// Pipelined blocked Warshall on bit rows with the same one-block look-ahead as the
// anti-distance closure: per pivot block kb (PB bits = PW words), phase 3 on the main
// stream covers every row and word outside blocks kb and kb+1, while three
// high-priority side streams close block (kb+1, kb+1) (one CTA, after its update from
// pivot kb), apply pivot kb to block row kb+1 and block column kb+1, and then compute
// the row and column panels of kb+1 (monotone OR updates make the in-place read/write
// overlap of a panel product harmless).
constexpr int kM4rPhase3MinRows = 2048;

// Blocked Warshall with 128-bit pivot blocks on the whole D×D matrix of rw words per row
// (pad bits already clear): the one-block look-ahead on the three side streams when they
// exist, otherwise everything on s.
static sr_status bool_closure_blocked(uint32_t *T, int64_t ldt, int D, int rw, bool vec, cudaStream_t s)
{
    constexpr int PB = 128, PW = PB / 32;
    const int nb = (D + PB - 1) / PB;
    auto pivot = [&](int kb, int kprev, cudaStream_t st) -> sr_status {
        bool_pivot_kernel<PB><<<1, PB, 0, st>>>(T, ldt, D, rw, kb, kprev);
        SR_CUDA_CHECK(cudaGetLastError());
        count_launches();
        return SR_OK;
    };
    auto width = [&](int kb) { return std::min(PB, D - kb * PB); };
    // words [kw, end) held by blocks kb .. kb+n-1 (the last block's words run to rw)
    auto word_end = [&](int kb, int n) { return kb + n < nb ? (kb + n) * PW : rw; };
    // phase 2 of block b: its row panel (rows of b, words outside b) ...
    auto row_panel = [&](int b) {
        const int k0 = b * PB, kw = k0 / 32, bw = width(b);
        BoolArgs a = bool_args(T + (int64_t)k0 * ldt + kw, T + (int64_t)k0 * ldt, T + (int64_t)k0 * ldt, ldt,
                               bw, bw, D, rw - (word_end(b, 1) - kw));
        a.skip0w = kw;
        a.skipww = word_end(b, 1) - kw;
        return a;
    };
    // ... and its column panel (rows outside b, the words of b)
    auto col_panel = [&](int b) {
        const int k0 = b * PB, kw = k0 / 32, bw = width(b);
        BoolArgs a = bool_args(T + kw, T + (int64_t)k0 * ldt + kw, T + kw, ldt, D - bw, bw, bw, (bw + 31) / 32);
        a.skip0 = k0;
        a.skipw = bw;
        return a;
    };
    SR_TRY(pivot(0, -1, s));
    if (nb == 1)
        return SR_OK;
    cudaStream_t sp = side_stream(0), sr_ = side_stream(1), sc = side_stream(2);
    if (!sp || !sr_ || !sc) {   // single stream: phase 2, phase 3, next pivot
        for (int kb = 0; kb < nb; ++kb) {
            SR_TRACE_BLOCK("bool_closure.block", kb);
            const int k0 = kb * PB, bw = width(kb), kw = k0 / 32, wn = word_end(kb, 1) - kw;
            SR_TRY(launch_bool_mul(row_panel(kb), vec, s, 2));
            SR_TRY(launch_bool_mul(col_panel(kb), vec, s, 1));
            BoolArgs p3 = bool_args(T + kw, T + (int64_t)k0 * ldt, T, ldt, D - bw, bw, D, rw - wn);
            p3.skip0 = k0; p3.skipw = bw; p3.skip0w = kw; p3.skipww = wn;
            SR_TRY(launch_bool_mul(p3, vec, s));
            if (kb + 1 < nb) SR_TRY(pivot(kb + 1, -1, s));
        }
        return SR_OK;
    }
    std::vector<cudaEvent_t> *ev = nullptr;
    SR_TRY(event_pool(4 * (size_t)nb + 4, ev));
    cudaEvent_t *main_done = ev->data();
    cudaEvent_t *pivot_done = main_done + nb + 1;
    cudaEvent_t *rowp_done = pivot_done + nb + 1;
    cudaEvent_t *colp_done = rowp_done + nb + 1;
    SR_TRY(launch_bool_mul(row_panel(0), vec, s, 2));
    SR_TRY(launch_bool_mul(col_panel(0), vec, s, 1));
    SR_CUDA_CHECK(cudaEventRecord(rowp_done[0], s));
    SR_CUDA_CHECK(cudaEventRecord(colp_done[0], s));
    for (int kb = 0; kb < nb; ++kb) {
        SR_TRACE_BLOCK("bool_closure.block", kb);
        const int k0 = kb * PB, bw = width(kb), kw = k0 / 32;
        const bool next = kb + 1 < nb;
        const int bwn = next ? width(kb + 1) : 0, ex = bw + bwn;          // rows left out
        const int exw = word_end(kb, next ? 2 : 1) - kw;                  // words left out
        if (kb > 0) {
            SR_CUDA_CHECK(cudaStreamWaitEvent(s, rowp_done[kb], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(s, colp_done[kb], 0));
        }
        // phase 3 of kb: rows and words outside blocks kb, kb+1 (Four Russians tables on
        // large matrices)
        BoolArgs p3 = bool_args(T + kw, T + (int64_t)k0 * ldt, T, ldt, D - ex, bw, D, rw - exw);
        p3.skip0 = k0; p3.skipw = ex; p3.skip0w = kw; p3.skipww = exw;
        if (D - ex >= kM4rPhase3MinRows)
            SR_TRY(launch_bool_mul_m4r(p3, s));
        else
            SR_TRY(launch_bool_mul(p3, vec, s));
        if (!next)
            break;
        SR_CUDA_CHECK(cudaEventRecord(main_done[kb], s));
        for (cudaStream_t x : {sp, sr_, sc}) {
            if (kb > 0) SR_CUDA_CHECK(cudaStreamWaitEvent(x, main_done[kb - 1], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(x, rowp_done[kb], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(x, colp_done[kb], 0));
        }
        const int k1 = k0 + bw, kw1 = k1 / 32, wn1 = (bwn + 31) / 32;
        SR_TRY(pivot(kb + 1, kb, sp));
        SR_CUDA_CHECK(cudaEventRecord(pivot_done[kb + 1], sp));
        // block row kb+1 from pivot kb (words outside blocks kb, kb+1), then its panel
        BoolArgs rs = bool_args(T + (int64_t)k1 * ldt + kw, T + (int64_t)k0 * ldt, T + (int64_t)k1 * ldt, ldt,
                                bwn, bw, D, rw - exw);
        rs.skip0w = kw; rs.skipww = exw;
        SR_TRY(launch_bool_mul(rs, vec, sr_, 2));
        SR_CUDA_CHECK(cudaStreamWaitEvent(sr_, pivot_done[kb + 1], 0));
        SR_TRY(launch_bool_mul(row_panel(kb + 1), vec, sr_, 2));
        SR_CUDA_CHECK(cudaEventRecord(rowp_done[kb + 1], sr_));
        // block column kb+1 from pivot kb (rows outside blocks kb, kb+1), then its panel
        BoolArgs cs = bool_args(T + kw, T + (int64_t)k0 * ldt + kw1, T + kw1, ldt, D - ex, bw, bwn, wn1);
        cs.skip0 = k0; cs.skipw = ex;
        SR_TRY(launch_bool_mul(cs, vec, sc, 1));
        SR_CUDA_CHECK(cudaStreamWaitEvent(sc, pivot_done[kb + 1], 0));
        SR_TRY(launch_bool_mul(col_panel(kb + 1), vec, sc, 1));
        SR_CUDA_CHECK(cudaEventRecord(colp_done[kb + 1], sc));
    }
    return SR_OK;
}

static sr_status bool_clear_pad(uint32_t *T, int64_t ldt, int D, int rw, cudaStream_t s)
{
    bool_clear_pad_kernel<<<(D + 255) / 256, 256, 0, s>>>(T, ldt, D, D, rw);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_closure_warshall(uint32_t *T, int64_t ldt, int D, int rw, bool vec, cudaStream_t s)
{
    SR_TRY(bool_clear_pad(T, ldt, D, rw, s));
    return bool_closure_blocked(T, ldt, D, rw, vec, s);
}

// Closure by repeated squaring (Section 2's A ⊗ (I ⊕ A)^(D'-1) identity, D' - 1 rounded up
// to a power of two): M := I ⊕ A, m squarings, then A ⊗ M, copied back into T.  On the
// tensor-core path the squarings stop early, on the device: once a squaring leaves M
// unchanged (M ⊗ M = M) every later one would too, so each squaring runs only if the
// previous one changed M.  One launch before each squaring compares M with the previous
// power, writes that flag and expands M into the product's operands; the product reads the
// flag when it starts (skipped products leave both buffers equal, so the host's buffer
// swap stays right).  The result is the same bits either way.
size_t bool_squaring_workspace(int64_t D, int64_t rw)
{
    const int64_t ldw = (rw + 3) / 4 * 4;
    return 256 + (size_t)(2 * D * ldw * 4) + bool_tc_workspace(D, D, D);
}

sr_status launch_bool_closure_squaring(uint32_t *T, int64_t ldt, int D, int rw, void *ws, size_t ws_bytes, bool tc,
                                       int *status, int spin_limit, cudaStream_t s, int grid_sms)
{
    // flags (256 bytes), then M, M2: D rows of rw 32-bit words each, rows padded to a
    // multiple of 4 words; any workspace beyond them holds the tensor-core operands when
    // it is large enough
    const int64_t ldw = ((int64_t)rw + 3) / 4 * 4;
    const size_t mats = 256 + (size_t)(2 * (int64_t)D * ldw * 4);
    if (mats > ws_bytes)
        return fail(SR_ENOMEM, "bool_closure: squaring needs at least %zu workspace bytes, context has %zu", mats,
                    ws_bytes);
    int *flags = static_cast<int *>(ws);
    uint32_t *M = reinterpret_cast<uint32_t *>(static_cast<char *>(ws) + 256);
    uint32_t *M2 = M + (int64_t)D * ldw;
    SR_TRY(launch_copy_rows(T, ldt, M, ldw, D, rw, s));
    SR_TRY(launch_bool_identity_or(M, ldw, D, s));                       // M = I ⊕ A
    int m = 0;
    while (((int64_t)1 << m) < (D - 1 > 1 ? D - 1 : 1)) ++m;
    void *tcws = static_cast<char *>(ws) + mats;
    const size_t tcbytes = ws_bytes - mats;
    const bool tcpath = tc && bool_tc_workspace(D, D, D) <= tcbytes;
    auto mul32 = [&](const uint32_t *X, int64_t ldx, const uint32_t *Y, int64_t ldy, uint32_t *Z,
                     const int *run_if) -> sr_status {
        BoolArgs a = bool_args(X, Y, Z, ldw, D, D, D, rw);
        a.lda = ldx; a.ldb = ldy;
        a.accumulate = 0;
        if (tcpath)
            return launch_bool_mul_tc(a, tcws, tcbytes, status, spin_limit, s, 0, run_if);
        const bool v = ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) == 0 &&
                       ((ldx & 3) == 0) && ((ldy & 3) == 0);
        return launch_bool_mul(a, v, s);
    };
    if (tcpath)
        SR_CUDA_CHECK(cudaMemsetAsync(flags, 0, 3 * sizeof(int), s));
    for (int it = 0; it < m; ++it) {                                      // M := M ⊗ M
        if (tcpath) {
            // one launch tests whether squaring it-1 changed M and expands M for this product,
            // which runs only if it did (flag it mod 3); two launches a squaring instead of four
            SR_TRY(launch_square_prep(M, M2, ldw, D, rw, tcws, flags, it, s, grid_sms));
            BoolArgs a = bool_args(M, M, M2, ldw, D, D, D, rw);
            a.accumulate = 0;
            const int Kp = (D + 127) / 128 * 128;
            uint8_t *Ae = static_cast<uint8_t *>(tcws);
            SR_TRY(launch_bool_mul_tc_expanded(a, Ae, tc_operand_b(Ae, D, Kp), status, spin_limit, s, 0,
                                               flags + it % 3));
        } else {
            SR_TRY(mul32(M, ldw, M, ldw, M2, nullptr));
        }
        uint32_t *t = M; M = M2; M2 = t;
    }
    SR_TRY(mul32(T, ldt, M, ldw, M2, nullptr));                           // A ⊗ (I ⊕ A)^(2^m)
    return launch_copy_rows(M2, ldw, T, ldt, D, rw, s);
}

// Wide blocks (W = 2048 bits) with phase 3 on the tensor cores.  The tensor-core product
// costs little per K slice but a fixed amount per launch (operand expansion, pipeline
// fill), so deep phase-3 passes pay off (GB300, D = 16384, the earlier one-tile-per-CTA
// kernel alone in passes of K = 128 / 1024 / 2048: 33.8 / 6.4 / 4.4 ms; the persistent
// kernel: 3.6 ms for K = 1024, 2.6 ms for K = 2048; Four Russians tables with K = 128, the
// 128-bit schedule's phase 3, 9.2 ms).  Closure times at D = 16384 with W = 1024 / 2048:
// 6.9 / 6.2 ms (wider blocks: fewer passes but a longer chain of diagonal-block work;
// W = 4096 was slower still with the earlier kernel).  Per block kb:
//   phase 2: the row panel T_kj := T_kj ⊕ T_kk ⊗ T_kj over every word j and the column
//            panel over every row i, side by side on the tensor cores (j = k and i = k
//            change nothing: T_kk ⊗ T_kk <= T_kk once T_kk is closed; the two products
//            overlap only in T_kk, which neither changes);
//   phase 3: T := T ⊕ T_col k ⊗ T_row k over the whole matrix except block row and
//            column kb (the panels, which it would not change; skipping them saves a
//            quarter of its tiles at D = 16384) and the diagonal block kb+1, while a side
//            stream gives block (kb+1, kb+1) its update from kb and closes it by repeated
//            squaring on the tensor cores (phase 1 of kb+1: log2 W + 1 products of W^3; the 128-bit
//            Warshall schedule's 16 dependent pivot blocks took 0.74 ms beside phase 3,
//            longer than phase 3 itself).
// The operands of every tensor-core product are expanded into the workspace before its
// kernel runs, so the in-place products read no entry that they write.  Workspace: the
// main region (phase 3's operands, or the two panels' side by side), then the side
// region (the diagonal update's operands, then the squaring's matrices and operands).
// SMs left to the side stream while phase 3 runs (GB300, D = 16384: 0 / 16 / 32 / 48 SMs
// left give 6.57 / 6.36 / 6.17 / 6.17 ms: the diagonal chain, not phase 3, sets the pace)
constexpr int kWideSideSms = 32;

static size_t wide_main_bytes(int64_t D, int W)
{
    const size_t panel = bool_tc_workspace(W, W, D);
    return (std::max(bool_tc_workspace(D, W, D), 2 * panel) + 255) / 256 * 256;
}

size_t bool_closure_wide_workspace(int64_t D)
{
    constexpr int W = kBoolWideBlock;
    return wide_main_bytes(D, W) + bool_squaring_workspace(W, W / 32 + 2);
}

sr_status launch_bool_closure_wide(uint32_t *T, int64_t ldt, int D, int rw, void *ws, size_t ws_bytes,
                                   int *status, int spin_limit, cudaStream_t s, int side_sms)
{
    if (side_sms < 0) side_sms = kWideSideSms;
    side_sms = std::min(side_sms, device_sm_count() - 1);
    constexpr int W = kBoolWideBlock, WW = W / 32;
    const int nb = (D + W - 1) / W;
    if (bool_closure_wide_workspace(D) > ws_bytes)
        return fail(SR_ENOMEM, "bool_closure: the tensor-core schedule needs %zu workspace bytes",
                    bool_closure_wide_workspace(D));
    auto width = [&](int kb) { return std::min(W, D - kb * W); };
    auto words_of = [&](int kb) { return kb + 1 < nb ? WW : rw - kb * WW; };     // the last block runs to rw
    const size_t main_bytes = wide_main_bytes(D, W), half = main_bytes / 2 / 256 * 256;
    void *ws_col = static_cast<char *>(ws) + half;
    void *ws_side = static_cast<char *>(ws) + main_bytes;
    const size_t side_bytes = ws_bytes - main_bytes;
    // the diagonal blocks after block 0 close beside phase 3: their convergence tests and
    // operand expansions take a grid sized for half the side SMs (GB300, D = 16384: 4.54 ms
    // against 4.68 with a grid for every SM, whose blocks slowed phase 3 down)
    auto close_block = [&](int kb, cudaStream_t st) {
        const int k0 = kb * W;
        return launch_bool_closure_squaring(T + (int64_t)k0 * ldt + k0 / 32, ldt, width(kb), words_of(kb), ws_side,
                                            side_bytes, true, status, spin_limit, st,
                                            kb > 0 && side_sms > 1 ? side_sms / 2 : 0);
    };
    SR_TRY(bool_clear_pad(T, ldt, D, rw, s));
    cudaStream_t sp = side_stream(0), sc = side_stream(1);
    if (!sp) sp = s;
    if (!sc) sc = s;
    std::vector<cudaEvent_t> *ev = nullptr;
    SR_TRY(event_pool(4 * (size_t)nb + 4, ev));
    cudaEvent_t *panels_done = ev->data(), *diag_done = panels_done + nb + 1;
    cudaEvent_t *colp_start = diag_done + nb + 1, *colp_done = colp_start + nb + 1;
    SR_TRY(close_block(0, s));
    for (int kb = 0; kb < nb; ++kb) {
        SR_TRACE_BLOCK("bool_closure.block", kb);
        const int k0 = kb * W, bw = width(kb), kw = k0 / 32, wn = words_of(kb);
        const bool next = kb + 1 < nb;
        SR_CUDA_CHECK(cudaEventRecord(colp_start[kb], s));
        SR_CUDA_CHECK(cudaStreamWaitEvent(sc, colp_start[kb], 0));
        SR_TRY(launch_bool_mul_tc(bool_args(T + kw, T + (int64_t)k0 * ldt + kw, T + kw, ldt, D, bw, bw, wn), ws_col,
                                  main_bytes - half, status, spin_limit, sc));                     // column panel
        SR_CUDA_CHECK(cudaEventRecord(colp_done[kb], sc));
        SR_TRY(launch_bool_mul_tc(bool_args(T + (int64_t)k0 * ldt + kw, T + (int64_t)k0 * ldt, T + (int64_t)k0 * ldt,
                                            ldt, bw, bw, D, rw), ws, half, status, spin_limit, s));   // row panel
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, colp_done[kb], 0));
        const int k1 = k0 + bw, kw1 = k1 / 32;
        if (next) {
            const int bwn = width(kb + 1), wn1 = words_of(kb + 1);
            SR_CUDA_CHECK(cudaEventRecord(panels_done[kb], s));
            SR_CUDA_CHECK(cudaStreamWaitEvent(sp, panels_done[kb], 0));
            // its update from kb on the tensor cores too (operands in the squaring's part of
            // the workspace, which the squaring only takes over after this product)
            SR_TRY(launch_bool_mul_tc(bool_args(T + (int64_t)k1 * ldt + kw, T + (int64_t)k0 * ldt + kw1,
                                                T + (int64_t)k1 * ldt + kw1, ldt, bwn, bw, bwn, wn1),
                                      ws_side, side_bytes, status, spin_limit, sp));
            SR_TRY(close_block(kb + 1, sp));
            SR_CUDA_CHECK(cudaEventRecord(diag_done[kb + 1], sp));
        }
        BoolArgs p3 = bool_args(T + kw, T + (int64_t)k0 * ldt, T, ldt, D, bw, D, rw);
        // block row and column kb are the panels, which phase 3 would leave as they are
        p3.band_r0 = k0; p3.band_rn = bw;
        p3.band_w0 = kw; p3.band_wn = wn;
        if (next) {
            p3.hole_r0 = k1; p3.hole_rn = width(kb + 1);
            p3.hole_w0 = kw1; p3.hole_wn = words_of(kb + 1);
        }
        // beside the diagonal block's squarings, phase 3 leaves side_sms SMs to them
        SR_TRY(launch_bool_mul_tc(p3, ws, main_bytes, status, spin_limit, s,
                                  next ? device_sm_count() - side_sms : 0));
        if (next)
            SR_CUDA_CHECK(cudaStreamWaitEvent(s, diag_done[kb + 1], 0));
    }
    return SR_OK;
}

sr_status launch_bool_pack(const uint8_t *dense, int64_t ldd, uint32_t *M, int64_t ldm, int R, int C, int rw,
                           int num_sms, cudaStream_t s)
{
    const int64_t words = (int64_t)R * rw;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, (int64_t)num_sms * 16));
    const bool vec = (reinterpret_cast<uintptr_t>(dense) & 15) == 0 && (ldd & 15) == 0;
    bool_pack_kernel<<<blocks, 256, 0, s>>>(dense, ldd, M, ldm, R, C, rw, vec);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_unpack(const uint32_t *M, int64_t ldm, uint8_t *dense, int64_t ldd, int R, int C,
                             int num_sms, cudaStream_t s)
{
    const int rw = (C + 31) / 32;
    const int64_t words = (int64_t)R * rw;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, (int64_t)num_sms * 16));
    const bool vec = (reinterpret_cast<uintptr_t>(dense) & 15) == 0 && (ldd & 15) == 0;
    bool_unpack_kernel<<<blocks, 256, 0, s>>>(M, ldm, dense, ldd, R, C, rw, vec);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_identity_or(uint32_t *M, int64_t ldm, int D, cudaStream_t s)
{
    bool_identity_or_kernel<<<(D + 255) / 256, 256, 0, s>>>(M, ldm, D);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_copy_rows(const uint32_t *src, int64_t lds, uint32_t *dst, int64_t ldd, int R, int rw,
                           cudaStream_t s)
{
    const int64_t n = (int64_t)R * rw;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    copy_rows_kernel<<<blocks, 256, 0, s>>>(src, lds, dst, ldd, R, rw);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
