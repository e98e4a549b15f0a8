// Device-side tile routine of the anti-distance product (u8, u16), shared by the
// product/closure kernels (antidist.cu) and the persistent closure kernel
// (closure_persistent.cu).  See antidist.cu for the method.
#pragma once

#include <type_traits>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

__device__ __forceinline__ int remap(int x, int skip0, int skipw) { return x < skip0 ? x : x + skipw; }

// u8 product kernel: accumulators hold acc + 255 in each 16-bit lane and the broadcast
// operand holds a (not a − 255), so max(acc + 255, a + b) = max(acc, a + b − 255) + 255
// with the same single add-max per lane pair and a one-instruction byte broadcast at
// staging.  Lanes stay in [255, 510] (acc >= 0), so adding or removing 255 per lane
// never carries or borrows across lanes.
constexpr uint32_t kShift8 = 0x00FF00FFu;

// -------------------------------------------------------------------------
// 16-byte chunk loads with zero fill outside [0, nrow) × [0, ncol)
// -------------------------------------------------------------------------
// CG: load through L2 only (ld.global.cg).  Kernels that read entries other CTAs of the
// same launch write (the persistent closure) must not see a stale L1 or read-only-cache
// line; the separate launches of the other schedules need no such care.
template <class E, bool VEC, bool CG = false>
__device__ __forceinline__ uint4 load_chunk(const E *base, int64_t ld, int r, int c, int nrow, int ncol)
{
    constexpr int CH = 16 / sizeof(E);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r >= nrow || c >= ncol)
        return v;
    const E *p = base + (int64_t)r * ld + c;
    if (VEC && c + CH <= ncol)
        return CG ? __ldcg(reinterpret_cast<const uint4 *>(p)) : *reinterpret_cast<const uint4 *>(p);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int t = 0; t < CH; ++t)
        if (c + t < ncol)
            w[(t * sizeof(E)) / 4] |= (uint32_t)(CG ? __ldcg(p + t) : p[t]) << (8 * ((t * sizeof(E)) % 4));
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
    static constexpr size_t SMEM = (size_t)2 * BK * (KD::AW * BM + BN / 2) * sizeof(uint32_t)
                                   + (size_t)BM * BN * sizeof(E);                 // prefetched C tile
    static_assert(TM % 4 == 0 && TN % 8 == 0, "thread tile");
    static_assert(BK % CH == 0 && BN % CH == 0, "chunking");
    static_assert(A_CHUNKS * CH * THREADS == BM * BK && B_CHUNKS * CH * THREADS == BK * BN, "chunks");
    static_assert(THREADS % 32 == 0 && BM % 32 == 0, "warps");
    static constexpr int MIN_BLOCKS = TM * TN >= 128 ? 3 : 4;      // register cap for CTAs per SM
};

// Barrier among the threads that compute a tile: the whole CTA (SYNC = 0), or named
// barrier SYNC over the first 128 threads (a CTA that also runs other warps).
template <int SYNC>
__device__ __forceinline__ void tile_sync()
{
    if (SYNC == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, 128;\n" ::"n"(SYNC) : "memory");
}

// Thread-block cluster helpers (distributed shared memory)
__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_size()
{
    uint32_t n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(n));
    return n;
}
// every thread of every CTA of the cluster: writes before it are visible to reads after it
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// the shared::cluster address of the same shared-memory word in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_map(const void *p, uint32_t rank)
{
    uint32_t a;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n"
                 : "=r"(a) : "r"((uint32_t)__cvta_generic_to_shared(p)), "r"(rank));
    return a;
}
// x[0..7] := lanewise max (unsigned 16-bit lanes) of x and the two 16-byte words at
// shared::cluster address a and a + stride; load and max in one block, so that only the
// words in flight add to the registers the accumulators hold
__device__ __forceinline__ void cluster_max8(uint32_t (&x)[8], uint32_t a, uint32_t stride)
{
    asm volatile("{\n"
                 ".reg .b32 t<8>;\n"
                 ".reg .u32 a1;\n"
                 "add.u32 a1, %8, %9;\n"
                 "ld.shared::cluster.v4.u32 {t0, t1, t2, t3}, [%8];\n"
                 "ld.shared::cluster.v4.u32 {t4, t5, t6, t7}, [a1];\n"
                 "max.u16x2 %0, %0, t0;\n"
                 "max.u16x2 %1, %1, t1;\n"
                 "max.u16x2 %2, %2, t2;\n"
                 "max.u16x2 %3, %3, t3;\n"
                 "max.u16x2 %4, %4, t4;\n"
                 "max.u16x2 %5, %5, t5;\n"
                 "max.u16x2 %6, %6, t6;\n"
                 "max.u16x2 %7, %7, t7;\n"
                 "}\n"
                 : "+r"(x[0]), "+r"(x[1]), "+r"(x[2]), "+r"(x[3]), "+r"(x[4]), "+r"(x[5]), "+r"(x[6]), "+r"(x[7])
                 : "r"(a), "r"(stride)
                 : "memory");
}

// Tiles tile0, tile0 + stride, ... below tile_end of the product p (one CTA, or its first 128
// threads with SYNC > 0; shared memory as sized by MulCfg).
//
// SPLIT: the CTAs of a thread-block cluster share one tile, CTA rank r over the slice
// [r·kslice, (r+1)·kslice) of K (kslice a multiple of BK; C joins at rank 0 only).  After
// the k-loop every CTA leaves its accumulators in its own shared memory; rank 0 reads them
// back, taking the lanewise max with the other ranks' through distributed shared memory
// (⊕ = max is associative and commutative, so the slices may merge in any order), and
// alone runs the epilogue.  One tile per CTA, no skipped tiles.
//
// RAGGED: a tile whose valid rows (columns) all lie in its first half skips the other
// half's accumulators in the k-loop (their entries are never stored), so a ragged edge
// tile costs about what a half-size tile would.  The choice is uniform across the CTA and
// made once per k-panel among four copies of the k-loop.
template <class KD, int BM, int BN, int BK, int TM, int TN, bool VEC, bool CG = false, int SYNC = 0,
          bool SPLIT = false, bool RAGGED = false>
__device__ __forceinline__ void mul_tiles(const MulArgs &p, int tile0, int stride, int tile_end = 0x7fffffff,
                                          int kslice = 0)
{
    using Cfg = MulCfg<KD, BM, BN, BK, TM, TN>;
    using E = typename KD::elem;
    constexpr int TR = Cfg::TR, TC = Cfg::TC, THREADS = Cfg::THREADS, CH = Cfg::CH, NP = Cfg::NP;
    constexpr int BN2 = BN / 2;
    constexpr int CROW = BN * (int)sizeof(E) / 16;        // 16-byte chunks per C tile row

    extern __shared__ __align__(16) uint32_t smem[];
    uint32_t *sA0 = smem;                               // [2][BK][BM]  broadcast word 0
    uint32_t *sA1 = smem + 2 * BK * BM;                 // [2][BK][BM]  broadcast word 1 (u16)
    uint32_t *sB = smem + KD::AW * 2 * BK * BM;          // [2][BK][BN/2] lane pairs
    uint4 *sC = reinterpret_cast<uint4 *>(sB + 2 * BK * BN2);   // [BM][CROW] prefetched C tile (raw)

    const E *__restrict__ A = static_cast<const E *>(p.A);
    const E *__restrict__ B = static_cast<const E *>(p.B);
    E *C = static_cast<E *>(p.C);

    const int tid = threadIdx.x;
    const int tc = tid % TC, tr = tid / TC;
    const int tiles_m = (p.R + BM - 1) / BM, tiles_n = (p.N + BN - 1) / BN;
    const int tiles = min(tiles_n * tiles_m, tile_end);
    // tile t -> (tile row, tile column): row-major, or column-major inside groups of group_m
    // tile rows (a wave of CTAs then shares group_m row panels of A and a run of B's column
    // panels in L2, where row-major order streams all of B through L2 once per wave)
    auto tile_rc = [&](int t, int &trow, int &tcol) {
        if (p.group_m <= 0) {
            trow = t / tiles_n;
            tcol = t % tiles_n;
            return;
        }
        const int per = p.group_m * tiles_n, g0 = (t / per) * p.group_m, gm = min(p.group_m, tiles_m - g0);
        const int w = t % per;
        trow = g0 + w % gm;
        tcol = w / gm;
    };
    const uint32_t crank = SPLIT ? cluster_rank() : 0u;
    const int kbeg = SPLIT ? (int)crank * kslice : 0;
    const int kend = SPLIT ? min(p.K, kbeg + kslice) : p.K;
    const bool accum = p.accumulate && crank == 0;
    const int nkt = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;   // an empty slice leaves the identity

    // tiles tile0, tile0 + stride, ... of the row-major tile grid (one per CTA when stride >= tiles)
    // skip_tile names a block of the 128x128 tile grid, which every tile shape here nests in.
    static_assert(128 % BM == 0 && 128 % BN == 0, "tiles nest in the 128x128 grid of skip_tile");
    const int tn128 = (p.N + 127) / 128;
    auto skipped = [&](int t) {
        if (p.skip_tile < 0) return false;
        int trow, tcol;
        tile_rc(t, trow, tcol);
        return (trow * BM) / 128 == p.skip_tile / tn128 && (tcol * BN) / 128 == p.skip_tile % tn128;
    };
    auto advance = [&](int t) {
        t += stride;
        while (t < tiles && skipped(t)) t += stride;
        return t;
    };
    int tile = tile0;
    if (tile < tiles && skipped(tile)) tile = advance(tile);

    // ---- operand staging: global -> registers -> shared
    uint4 ra[Cfg::A_CHUNKS], rb[Cfg::B_CHUNKS];
    auto gload = [&](int row0, int col0, int k0) {
#pragma unroll
        for (int u = 0; u < Cfg::A_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int i = ch % BM, kc = ch / BM;
            const int r = row0 + i;
            ra[u] = r < p.R ? load_chunk<E, VEC, CG>(A, p.lda, remap(r, p.rskip0, p.rskipw), kbeg + k0 + kc * CH,
                                                 0x7fffffff, kend)
                            : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < Cfg::B_CHUNKS; ++u) {
            const int ch = tid + u * THREADS;
            const int jc = ch % (BN / CH), kr = ch / (BN / CH);
            const int c = col0 + jc * CH;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (c < p.N && kbeg + k0 + kr < kend) {   // the chunk never straddles an excluded range
                const int pc = remap(c, p.cskip0, p.cskipw);
                v = load_chunk<E, VEC, CG>(B, p.ldb, kbeg + k0 + kr, pc, kend, pc + (p.N - c));
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
                if (sizeof(E) == 1) {      // raw byte in both lanes (the accumulator carries the −S)
                    a0 = __byte_perm(u4get(ra[u], t / 4), 0u, 0x4040 | (t % 4) | ((t % 4) << 8));
                    a1 = 0u;
                } else {
                    KD::bcast(chunk_elem<E>(ra[u], t), a0, a1);
                }
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
    // C tile -> sC (raw bytes), asynchronously when vector accesses are allowed
    auto cprefetch = [&](int row0, int col0) {
        for (int ch = tid; ch < BM * CROW; ch += THREADS) {
            const int i = ch / CROW, cc = ch % CROW;
            const int r = row0 + i, c = col0 + cc * CH;
            uint4 *dst = sC + ch;
            if (VEC) {
                const bool full = r < p.R && c + CH <= p.N;
                if (full) {
                    const E *src = C + (int64_t)remap(r, p.rskip0, p.rskipw) * p.ldc + remap(c, p.cskip0, p.cskipw);
                    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(dst);
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src));
                    continue;
                }
            }
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (r < p.R && c < p.N) {
                const int pr = remap(r, p.rskip0, p.rskipw), pc = remap(c, p.cskip0, p.cskipw);
                v = load_chunk<E, false, CG>(C, p.ldc, pr, pc, 0x7fffffff, pc + (p.N - c));
            }
            *dst = v;
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    if (tile < tiles) {
        int trow, tcol;
        tile_rc(tile, trow, tcol);
        const int row0 = trow * BM, col0 = tcol * BN;
        if (accum) cprefetch(row0, col0);
        gload(row0, col0, 0);
    }

    for (; tile < tiles; tile = advance(tile)) {
        int trow, tcol, ntr = 0, ntc = 0;
        tile_rc(tile, trow, tcol);
        const int row0 = trow * BM, col0 = tcol * BN;
        const int next = advance(tile);
        if (next < tiles) tile_rc(next, ntr, ntc);
        const int nrow0 = ntr * BM, ncol0 = ntc * BN;

        // C joins the result only in the epilogue (⊕ = max is commutative), so its load,
        // issued before the k-loop, is hidden behind the k-loop
        uint32_t acc[TM][NP];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < NP; ++j) acc[i][j] = sizeof(E) == 1 ? kShift8 : 0u;

        sstore(0);
        tile_sync<SYNC>();
        for (int kt = 0; kt < nkt; ++kt) {
            const int buf = kt & 1;
            if (kt + 1 < nkt)
                gload(row0, col0, (kt + 1) * BK);
            else if (next < tiles)
                gload(nrow0, ncol0, 0);                        // next tile's first k-panel
            const uint32_t *a0p = sA0 + buf * BK * BM + tr * 4;
            const uint32_t *a1p = sA1 + buf * BK * BM + tr * 4;
            const uint32_t *bp = sB + buf * BK * BN2 + tc * 4;
            // thread rows i < TM/2 are the tile's first BM/2 rows (accumulator group g = i / 4
            // holds rows g·4·TR + tr·4 + i % 4), lane pairs j < NP/2 its first BN/2 columns
            auto kpanel = [&](auto half_r, auto half_c) {
                constexpr int TMA = decltype(half_r)::value ? TM / 2 : TM;
                constexpr int NPA = decltype(half_c)::value ? NP / 2 : NP;
#pragma unroll 4
                for (int k = 0; k < BK; ++k) {
                    uint32_t a0[TM], a1[TM], b[NP];
#pragma unroll
                    for (int g = 0; g < TMA / 4; ++g) {
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
                    for (int g = 0; g < NPA / 4; ++g) {
                        const uint4 v = *reinterpret_cast<const uint4 *>(bp + k * BN2 + g * 4 * TC);
                        b[4 * g] = v.x; b[4 * g + 1] = v.y; b[4 * g + 2] = v.z; b[4 * g + 3] = v.w;
                    }
#pragma unroll
                    for (int i = 0; i < TMA; ++i)
#pragma unroll
                        for (int j = 0; j < NPA; ++j)
                            acc[i][j] = KD::op(acc[i][j], b[j], a0[i], a1[i]);
                }
            };
            using F = std::false_type;
            using Tr = std::true_type;
            if constexpr (RAGGED) {
                static_assert(TM % 8 == 0 && NP % 8 == 0, "halves of whole accumulator groups");
                const bool hr = p.R - row0 <= BM / 2, hc = p.N - col0 <= BN / 2;
                if (hr && hc) kpanel(Tr{}, Tr{});
                else if (hr) kpanel(Tr{}, F{});
                else if (hc) kpanel(F{}, Tr{});
                else kpanel(F{}, F{});
            } else {
                kpanel(F{}, F{});
            }
            if (kt + 1 < nkt)
                sstore(buf ^ 1);
            tile_sync<SYNC>();
        }

        if constexpr (SPLIT) {
            // the k-loop's staging is free after its last barrier: the partial goes there,
            // word j of thread t at [j / 4][t] (conflict-free 16-byte rows)
            static_assert(Cfg::SMEM - (size_t)BM * BN * sizeof(E) >= (size_t)TM * NP * 4 * THREADS,
                          "the partial tile fits in the operand staging");
            // (rank 0's too: its accumulators are rebuilt row by row, which keeps the merge
            // within the k-loop's register budget)
            uint4 *part = reinterpret_cast<uint4 *>(smem);
            const uint32_t rank = crank;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int g = 0; g < NP / 4; ++g)
                    part[(i * (NP / 4) + g) * THREADS + tid] =
                        make_uint4(acc[i][4 * g], acc[i][4 * g + 1], acc[i][4 * g + 2], acc[i][4 * g + 3]);
            cluster_sync();
            if (rank == 0) {
                static_assert(NP == 8, "one row of a thread's accumulators is two 16-byte words");
                const uint32_t n = cluster_size();
#pragma unroll
                for (int i = 0; i < TM; ++i) {
                    const uint4 v0 = part[(2 * i) * THREADS + tid], v1 = part[(2 * i + 1) * THREADS + tid];
                    uint32_t x[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
                    for (uint32_t r = 1; r < n; ++r)
                        cluster_max8(x, cluster_map(part + (2 * i) * THREADS + tid, r), (uint32_t)THREADS * 16u);
#pragma unroll
                    for (int u = 0; u < 8; ++u) acc[i][u] = x[u];
                }
            }
            cluster_sync();                        // the other ranks' shared memory outlives the reads
            if (rank != 0)
                continue;
        }

        // ---- epilogue: ⊕ with C (prefetched into sC), store
        if (accum) {
            asm volatile("cp.async.wait_group 0;\n" ::);
            tile_sync<SYNC>();
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int li = (i / 4) * (4 * TR) + tr * 4 + (i % 4);
            const int r = row0 + li;
            if (r >= p.R)
                continue;
            const int pr = remap(r, p.rskip0, p.rskipw);
#pragma unroll
            for (int g = 0; g < NP / 4; ++g) {
                const int lc = g * (8 * TC) + tc * 8;
                const int c = col0 + lc;
                if (c >= p.N)
                    continue;
                E *dst = C + (int64_t)pr * p.ldc + remap(c, p.cskip0, p.cskipw);
                uint32_t q[4];
                if (sizeof(E) == 1) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) q[u] = acc[i][g * 4 + u] - kShift8;
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) q[u] = acc[i][g * 4 + u];
                }
                if (accum) {
                    const uint32_t *crow = reinterpret_cast<const uint32_t *>(sC + li * CROW);
                    if (sizeof(E) == 1) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(crow + lc / 4);
                        q[0] = __vmaxu2(q[0], u8x2_lo(v.x)); q[1] = __vmaxu2(q[1], u8x2_hi(v.x));
                        q[2] = __vmaxu2(q[2], u8x2_lo(v.y)); q[3] = __vmaxu2(q[3], u8x2_hi(v.y));
                    } else {
                        const uint4 v = *reinterpret_cast<const uint4 *>(crow + lc / 2);
                        q[0] = __vmaxu2(q[0], v.x); q[1] = __vmaxu2(q[1], v.y);
                        q[2] = __vmaxu2(q[2], v.z); q[3] = __vmaxu2(q[3], v.w);
                    }
                }
                if (sizeof(E) == 1) {
                    const uint32_t w0 = pack_u8x4(q[0], q[1]);
                    const uint32_t w1 = pack_u8x4(q[2], q[3]);
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
        if (accum) {
            tile_sync<SYNC>();                                   // sC is free again
            if (next < tiles) cprefetch(nrow0, ncol0);         // lands during the next tile's k-loop
        }
    }
}

}  // namespace sr
