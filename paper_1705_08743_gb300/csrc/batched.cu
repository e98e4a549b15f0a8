// Batched anti-distance closure: many independent graphs of uneven size in one
// persistent launch (the Section 2 Warshall / Section 3 Floyd closure, blocked as in
// antidist.cu, applied to every graph of a batch).
//
// Work list.  The host sorts the graphs by cost (D^3, largest first) and forms
// work items: a graph at or above the cooperative threshold is one item closed by
// all NC CTAs of a thread-block cluster together; smaller graphs are grouped NC at
// a time, one per CTA.  Clusters take items in order from a global counter, so the
// largest items start first (longest-processing-time-first scheduling).
//
// Per graph, the CTA (or cluster) runs the three phases for each pivot block of
// PB = 64: the diagonal block is closed in registers by every CTA of the cluster
// (identical results, no exchange needed), panel blocks and then the remaining
// blocks are distributed round-robin over the cluster's CTAs, with a cluster
// barrier (release/acquire) after phase 2 and after phase 3.  All waits are
// hardware barriers; nothing spins on memory.

#include <algorithm>
#include <cmath>
#include <cooperative_groups.h>
#include <cstdio>
#include <map>
#include <string>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "sr_common.cuh"
#include "sr_ctx.h"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace cg = cooperative_groups;

namespace sr {

// Two register layouts of a PB×PB block for 128 threads, thread (r0, c0) with
// r0 = tid / 8 in [0,16) and c0 = tid % 8; both hold rows r0 + 16 j (j < PB/16):
//  - layout S (pivot closure): lane-pair columns c0 + 8 m.  Pivot kk = 16 j + q is
//    row j of threads r0 == q and register column m = j, half q & 1, of threads
//    c0 == q/2, so every register index is a compile-time constant.
//  - layout C (products): lane-pair columns 4 c0 + m, i.e. 8 consecutive entries
//    per row, loaded and stored with one vector access.
// Operands in shared memory: A form sA[kk][r0*TRN + j] (entry (row, kk) broadcast,
// KD::AW words), B form sB[kk][pair] (row kk as lane pairs, natural order).
template <class KD, int PB>
struct BatchTile {
    static constexpr int RS = 16, CS = 8, THREADS = RS * CS;
    static constexpr int TRN = PB / RS, TCN = PB / 2 / CS;
    static_assert(TRN == TCN && TCN == 4, "layouts assume PB = 64");
    using E = typename KD::elem;
    using Regs = uint32_t[TRN][TCN];

    static constexpr int A_WORDS = PB * PB;          // per broadcast word
    static constexpr int B_WORDS = PB * PB / 2;
    static constexpr size_t SMEM =
        (size_t)4 * (2 * KD::AW * A_WORDS + 2 * B_WORDS + 2 * (PB / 2) + PB) + 64;

    // ---- layout S (scalar accesses; used once per pivot block)
    __device__ static void loadS(const E *T, int64_t ldt, int i0, int j0, int h, int w, int r0, int c0, Regs &R)
    {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) {
                const int r = r0 + RS * j, c = 2 * (c0 + CS * m);
                uint32_t v = 0u;
                if (r < h) {
                    const E *src = T + (int64_t)(i0 + r) * ldt + j0 + c;
                    if (c < w) v = (uint32_t)src[0];
                    if (c + 1 < w) v |= (uint32_t)src[1] << 16;
                }
                R[j][m] = v;
            }
    }
    __device__ static void storeS(E *T, int64_t ldt, int i0, int j0, int h, int w, int r0, int c0, const Regs &R)
    {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m) {
                const int r = r0 + RS * j, c = 2 * (c0 + CS * m);
                if (r < h) {
                    E *dst = T + (int64_t)(i0 + r) * ldt + j0 + c;
                    if (c < w) dst[0] = (E)(R[j][m] & 0xFFFFu);
                    if (c + 1 < w) dst[1] = (E)(R[j][m] >> 16);
                }
            }
    }
    // ---- layout C (vector accesses when the row chunk is complete and aligned)
    __device__ static void loadC(const E *T, int64_t ldt, int i0, int j0, int h, int w, int r0, int c0, bool vec,
                                 Regs &R)
    {
        const int c = 8 * c0;
#pragma unroll
        for (int j = 0; j < TRN; ++j) {
            const int r = r0 + RS * j;
            uint32_t q[4] = {0u, 0u, 0u, 0u};
            if (r < h && c < w) {
                const E *src = T + (int64_t)(i0 + r) * ldt + j0 + c;
                if (vec && c + 8 <= w) {
                    if (sizeof(E) == 1) {
                        const uint2 v = *reinterpret_cast<const uint2 *>(src);
                        q[0] = u8x2_lo(v.x); q[1] = u8x2_hi(v.x); q[2] = u8x2_lo(v.y); q[3] = u8x2_hi(v.y);
                    } else {
                        const uint4 v = *reinterpret_cast<const uint4 *>(src);
                        q[0] = v.x; q[1] = v.y; q[2] = v.z; q[3] = v.w;
                    }
                } else {
                    for (int t = 0; t < 8; ++t)
                        if (c + t < w) q[t / 2] |= (uint32_t)src[t] << (16 * (t % 2));
                }
            }
#pragma unroll
            for (int m = 0; m < TCN; ++m) R[j][m] = q[m];
        }
    }
    __device__ static void storeC(E *T, int64_t ldt, int i0, int j0, int h, int w, int r0, int c0, bool vec,
                                  const Regs &R)
    {
        const int c = 8 * c0;
#pragma unroll
        for (int j = 0; j < TRN; ++j) {
            const int r = r0 + RS * j;
            if (r >= h || c >= w) continue;
            E *dst = T + (int64_t)(i0 + r) * ldt + j0 + c;
            if (vec && c + 8 <= w) {
                if (sizeof(E) == 1)
                    *reinterpret_cast<uint2 *>(dst) = make_uint2(pack_u8x4(R[j][0], R[j][1]), pack_u8x4(R[j][2], R[j][3]));
                else
                    *reinterpret_cast<uint4 *>(dst) = make_uint4(R[j][0], R[j][1], R[j][2], R[j][3]);
            } else {
                for (int t = 0; t < 8; ++t)
                    if (c + t < w) dst[t] = (E)((R[j][t / 2] >> (16 * (t % 2))) & 0xFFFFu);
            }
        }
    }
    // ---- operand staging; LAYOUT_S selects which layout R is in
    template <bool LAYOUT_S>
    __device__ static void store_A(uint32_t *sA0, uint32_t *sA1, int r0, int c0, const Regs &R)
    {
#pragma unroll
        for (int j = 0; j < TRN; ++j)
#pragma unroll
            for (int m = 0; m < TCN; ++m)
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    uint32_t a0, a1;
                    KD::bcast((R[j][m] >> (16 * hh)) & 0xFFFFu, a0, a1);
                    const int kk = 2 * (LAYOUT_S ? c0 + CS * m : TCN * c0 + m) + hh;
                    sA0[kk * PB + r0 * TRN + j] = a0;
                    if (KD::AW == 2) sA1[kk * PB + r0 * TRN + j] = a1;
                }
    }
    template <bool LAYOUT_S>
    __device__ static void store_B(uint32_t *sB, int r0, int c0, const Regs &R)
    {
#pragma unroll
        for (int j = 0; j < TRN; ++j) {
            uint32_t *row = sB + (r0 + RS * j) * (PB / 2);
            if (LAYOUT_S) {
#pragma unroll
                for (int m = 0; m < TCN; ++m) row[c0 + CS * m] = R[j][m];
            } else {
                *reinterpret_cast<uint4 *>(row + TCN * c0) = make_uint4(R[j][0], R[j][1], R[j][2], R[j][3]);
            }
        }
    }
    // Y (layout C) := Y ⊕ A ⊗ B over kk < kw
    __device__ static void gemm(Regs &Y, const uint32_t *sA0, const uint32_t *sA1, const uint32_t *sB, int kw,
                                int r0, int c0)
    {
        const uint32_t *ap0 = sA0 + r0 * TRN, *ap1 = sA1 + r0 * TRN, *bp = sB + TCN * c0;
#pragma unroll 2
        for (int kk = 0; kk < kw; ++kk) {
            const uint4 b = *reinterpret_cast<const uint4 *>(bp + kk * (PB / 2));
            const uint4 x0 = *reinterpret_cast<const uint4 *>(ap0 + kk * PB);
            uint4 x1 = make_uint4(0u, 0u, 0u, 0u);
            if (KD::AW == 2) x1 = *reinterpret_cast<const uint4 *>(ap1 + kk * PB);
            const uint32_t bv[4] = {b.x, b.y, b.z, b.w};
            const uint32_t a0[4] = {x0.x, x0.y, x0.z, x0.w};
            const uint32_t a1[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int j = 0; j < TRN; ++j)
#pragma unroll
                for (int m = 0; m < TCN; ++m)
                    Y[j][m] = KD::op(Y[j][m], bv[m], a0[j], a1[j]);
        }
    }
    // Warshall on a block held in registers, layout S (pivots 0..bw-1)
    __device__ static void close(Regs &X, int bw, uint32_t *rowbuf, uint16_t *colbuf, int r0, int c0)
    {
#pragma unroll
        for (int j = 0; j < TRN; ++j) {
            for (int q = 0; q < RS; ++q) {
                const int kk = RS * j + q;
                if (kk >= bw) break;
                const int par = kk & 1;
                if (r0 == q) {
#pragma unroll
                    for (int m = 0; m < TCN; ++m) rowbuf[par * (PB / 2) + c0 * TCN + m] = X[j][m];
                }
                if (c0 == (q >> 1)) {
                    const int sh = 16 * (q & 1);
#pragma unroll
                    for (int jj = 0; jj < TRN; ++jj) colbuf[par * PB + r0 * TRN + jj] = (uint16_t)(X[jj][j] >> sh);
                }
                __syncthreads();
                uint32_t bv[TCN];
#pragma unroll
                for (int m = 0; m < TCN; ++m) bv[m] = rowbuf[par * (PB / 2) + c0 * TCN + m];
#pragma unroll
                for (int jj = 0; jj < TRN; ++jj) {
                    uint32_t a0, a1;
                    KD::bcast(colbuf[par * PB + r0 * TRN + jj], a0, a1);
#pragma unroll
                    for (int m = 0; m < TCN; ++m) X[jj][m] = KD::op(X[jj][m], bv[m], a0, a1);
                }
            }
        }
        __syncthreads();
    }
};

template <int NC>
__device__ __forceinline__ void group_sync()
{
    if (NC > 1) {
        __threadfence();
        cg::this_cluster().sync();
    } else {
        __syncthreads();
    }
}

// Close one graph with the `nc` CTAs of this cluster (rank = this CTA's index).
template <class KD, int PB, int NC>
__device__ void close_graph(const BatchGraph &gr, int rank, int nc, uint32_t *smem)
{
    using BT = BatchTile<KD, PB>;
    using E = typename KD::elem;
    uint32_t *sXA0 = smem;                                  // closed pivot block, A form
    uint32_t *sXA1 = sXA0 + BT::A_WORDS;
    uint32_t *sYA0 = sXA0 + KD::AW * BT::A_WORDS;           // other operand, A form
    uint32_t *sYA1 = sYA0 + BT::A_WORDS;
    uint32_t *sXB = sYA0 + KD::AW * BT::A_WORDS;            // closed pivot block, B form
    uint32_t *sYB = sXB + BT::B_WORDS;                      // other operand, B form
    uint32_t *rowbuf = sYB + BT::B_WORDS;
    uint16_t *colbuf = reinterpret_cast<uint16_t *>(rowbuf + 2 * (PB / 2));

    E *T = static_cast<E *>(gr.T);
    const int64_t ldt = gr.ldt;
    const int D = gr.D;
    const bool vec = gr.pad != 0;                           // rows 16-byte aligned
    const int nb = (D + PB - 1) / PB;
    const int tid = threadIdx.x;
    const int r0 = tid / BT::CS, c0 = tid % BT::CS;

    for (int kb = 0; kb < nb; ++kb) {
        const int k0 = kb * PB, bw = min(PB, D - k0);
        // phase 1 (every CTA of the group computes the same closed block)
        typename BT::Regs X;
        BT::loadS(T, ldt, k0, k0, bw, bw, r0, c0, X);
        BT::close(X, bw, rowbuf, colbuf, r0, c0);
        if (rank == 0)
            BT::storeS(T, ldt, k0, k0, bw, bw, r0, c0, X);
        if (nb == 1)
            break;
        BT::template store_A<true>(sXA0, sXA1, r0, c0, X);
        BT::template store_B<true>(sXB, r0, c0, X);
        __syncthreads();
        // phase 2: panels t = 0 .. 2(nb-1)-1, round-robin over the group
        for (int t = rank; t < 2 * (nb - 1); t += nc) {
            const bool row = t < nb - 1;
            int b = row ? t : t - (nb - 1);
            if (b >= kb) ++b;
            const int i0 = row ? k0 : b * PB, j0 = row ? b * PB : k0;
            const int h = row ? bw : min(PB, D - i0), w = row ? min(PB, D - j0) : bw;
            typename BT::Regs Y;
            BT::loadC(T, ldt, i0, j0, h, w, r0, c0, vec, Y);
            if (row) BT::template store_B<false>(sYB, r0, c0, Y);          // Y ⊕= T_kk ⊗ Y
            else BT::template store_A<false>(sYA0, sYA1, r0, c0, Y);       // Y ⊕= Y ⊗ T_kk
            __syncthreads();
            if (row) BT::gemm(Y, sXA0, sXA1, sYB, bw, r0, c0);
            else BT::gemm(Y, sYA0, sYA1, sXB, bw, r0, c0);
            BT::storeC(T, ldt, i0, j0, h, w, r0, c0, vec, Y);
            __syncthreads();
        }
        group_sync<NC>();
        // phase 3: blocks (i, j), i, j != kb, round-robin over the group, row-major;
        // the next block's operands are loaded into registers while this one computes
        const int n1 = nb - 1, ntile = n1 * n1;
        int t = rank;
        if (t < ntile) {
            auto coords = [&](int tt, int &bi, int &bj) {
                bi = tt / n1; bj = tt % n1;
                if (bi >= kb) ++bi;
                if (bj >= kb) ++bj;
            };
            int bi, bj;
            coords(t, bi, bj);
            typename BT::Regs Cn, Bn, An;
            int cur_i = -1;
            BT::loadC(T, ldt, bi * PB, bj * PB, min(PB, D - bi * PB), min(PB, D - bj * PB), r0, c0, vec, Cn);
            BT::loadC(T, ldt, k0, bj * PB, bw, min(PB, D - bj * PB), r0, c0, vec, Bn);
            BT::loadC(T, ldt, bi * PB, k0, min(PB, D - bi * PB), bw, r0, c0, vec, An);
            for (; t < ntile; t += nc) {
                const int i0 = bi * PB, j0 = bj * PB;
                const int h = min(PB, D - i0), w = min(PB, D - j0);
                if (bi != cur_i) {
                    BT::template store_A<false>(sYA0, sYA1, r0, c0, An);
                    cur_i = bi;
                }
                BT::template store_B<false>(sYB, r0, c0, Bn);
                typename BT::Regs Y;
#pragma unroll
                for (int j = 0; j < BT::TRN; ++j)
#pragma unroll
                    for (int m = 0; m < BT::TCN; ++m) Y[j][m] = Cn[j][m];
                __syncthreads();
                const int tn = t + nc;
                int ni = bi, nj = bj;
                if (tn < ntile) {                                     // prefetch the next block
                    coords(tn, ni, nj);
                    BT::loadC(T, ldt, ni * PB, nj * PB, min(PB, D - ni * PB), min(PB, D - nj * PB), r0, c0, vec, Cn);
                    BT::loadC(T, ldt, k0, nj * PB, bw, min(PB, D - nj * PB), r0, c0, vec, Bn);
                    if (ni != bi)
                        BT::loadC(T, ldt, ni * PB, k0, min(PB, D - ni * PB), bw, r0, c0, vec, An);
                }
                BT::gemm(Y, sYA0, sYA1, sYB, bw, r0, c0);
                BT::storeC(T, ldt, i0, j0, h, w, r0, c0, vec, Y);
                bi = ni; bj = nj;
                __syncthreads();
            }
        }
        group_sync<NC>();
    }
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One thread writes the device clock (ns): the start of a batch launch, or the end of the
// launches before it in the stream.
__global__ void batch_stamp_kernel(uint64_t *at) { *at = global_ns(); }

// done (may be null): done[g] = the device clock when graph g's closure is complete
template <class KD, int PB, int NC>
__global__ void __launch_bounds__(128) batched_closure_kernel(const BatchGraph *graphs, const BatchItem *items,
                                                              int nitems, int *counter, uint64_t *done)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int item_idx;
    int rank = 0;
    if (NC > 1) rank = (int)cg::this_cluster().block_rank();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0)
            item_idx = atomicAdd(counter, 1);
        if (NC > 1) {
            cg::this_cluster().sync();
            if (rank != 0 && threadIdx.x == 0)
                item_idx = *cg::this_cluster().map_shared_rank(&item_idx, 0);
            cg::this_cluster().sync();
        }
        __syncthreads();
        const int it = item_idx;
        __syncthreads();
        if (it >= nitems)
            break;
        const BatchItem item = items[it];
        if (item.coop) {
            close_graph<KD, PB, NC>(graphs[item.g[0]], rank, NC, smem);
            if (done && rank == 0 && threadIdx.x == 0) done[item.g[0]] = global_ns();
        } else {
            if (rank < item.n) {
                close_graph<KD, PB, 1>(graphs[item.g[rank]], 0, 1, smem);
                if (done && threadIdx.x == 0) done[item.g[rank]] = global_ns();
            }
            if (NC > 1) cg::this_cluster().sync();
        }
    }
}

// --------------------------------------------------------------------------- host side
struct BatchPlan {
    int device = 0;
    sr_dtype dtype = SR_U16;
    int n = 0;
    std::vector<BatchGraph> h_graphs;
    std::vector<int> order;          // graph indices by decreasing cost
    // tuning
    int nc = 2;                      // cluster size (1, 2 or 4)
    int coop_threshold = 384;        // graphs with D >= this are cooperative items
    int ctas_per_sm = 2;
    int nitems = 0;
    BatchGraph *d_graphs = nullptr;
    BatchItem *d_items = nullptr;
    int *d_counter = nullptr;
    // grouped schedule (tuning cluster 0): per pivot block kb of 128, the pivot blocks of
    // every graph still open at kb, then all their panels, then all their phase-3 tiles
    struct GroupedStep { int nactive, act_off, npan, pan_off, pan_tiles, np3, p3_off, p3_tiles; };
    std::vector<GroupedStep> gsteps;
    int *d_gactive = nullptr;        // graph indices, concatenated per step
    MulArgs *d_gargs = nullptr;      // products, concatenated per step and kind
    int *d_gstart = nullptr;         // first tile of each product within its launch
    bool gvec = true;                // every graph 16-byte aligned
    // completion stamps (sr_batch_set_timing): [0] launch start, [1 + g] graph g done
    // (persistent kernel), [1 + n + kb] end of pivot step kb (grouped schedule); device clock ns
    uint64_t *d_stamps = nullptr;
    // captured launch
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool use_graph = false;
    double ops = 0;                  // sum of D^3
};

static sr_status build_items(BatchPlan &p)
{
    std::vector<BatchItem> items;
    std::vector<int> small;
    for (int g : p.order) {
        if (p.nc > 1 && p.h_graphs[g].D >= p.coop_threshold) {
            BatchItem it{};
            it.n = 1; it.coop = 1; it.g[0] = g;
            items.push_back(it);
        } else {
            small.push_back(g);
        }
    }
    const size_t per = (size_t)std::max(1, p.nc);         // graphs per item (cluster 0: grouped, unused)
    for (size_t s = 0; s < small.size(); s += per) {
        BatchItem it{};
        it.coop = 0;
        it.n = (int)std::min<size_t>(per, small.size() - s);
        for (int r = 0; r < it.n; ++r) it.g[r] = small[s + r];
        items.push_back(it);
    }
    // items in decreasing cost: cooperative items cost D^3 / nc, groups the max member
    auto cost = [&](const BatchItem &it) {
        double c = 0;
        for (int r = 0; r < it.n; ++r) c = std::max(c, std::pow((double)p.h_graphs[it.g[r]].D, 3.0));
        return it.coop ? c / p.nc : c;
    };
    std::stable_sort(items.begin(), items.end(), [&](const BatchItem &a, const BatchItem &b) { return cost(a) > cost(b); });
    p.nitems = (int)items.size();
    if (p.d_items) { cudaFree(p.d_items); p.d_items = nullptr; }
    SR_CUDA_CHECK(cudaMalloc(&p.d_items, sizeof(BatchItem) * std::max(1, p.nitems)));
    SR_CUDA_CHECK(cudaMemcpy(p.d_items, items.data(), sizeof(BatchItem) * p.nitems, cudaMemcpyHostToDevice));
    return SR_OK;
}

template <class KD, int NC>
static sr_status launch_batched_nc(BatchPlan &p, cudaStream_t s)
{
    constexpr int PB = 64;
    using BT = BatchTile<KD, PB>;
    auto kern = batched_closure_kernel<KD, PB, NC>;
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BT::SMEM));
        if (NC > 1)
            SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr[dev] = true;
    }
    int grid = device_sm_count() * p.ctas_per_sm;
    grid = std::max(NC, grid / NC * NC);
    grid = std::min(grid, std::max(NC, p.nitems * NC));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT::THREADS);
    cfg.dynamicSmemBytes = BT::SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = NC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = NC > 1 ? 1 : 0;
    uint64_t *done = p.d_stamps ? p.d_stamps + 1 : nullptr;
    SR_CUDA_CHECK(cudaLaunchKernelEx(&cfg, kern, (const BatchGraph *)p.d_graphs, (const BatchItem *)p.d_items,
                                     p.nitems, p.d_counter, done));
    count_launches();
    return SR_OK;
}

sr_status launch_batched_closure_flat(sr_dtype dt, const BatchGraph *d_graphs, const BatchItem *d_items, int nitems,
                                      int *d_counter, int ctas_per_sm, cudaStream_t s)
{
    BatchPlan p;
    p.dtype = dt;
    p.nc = 1;
    p.ctas_per_sm = ctas_per_sm;
    p.nitems = nitems;
    p.d_graphs = const_cast<BatchGraph *>(d_graphs);
    p.d_items = const_cast<BatchItem *>(d_items);
    p.d_counter = d_counter;
    SR_CUDA_CHECK(cudaMemsetAsync(d_counter, 0, sizeof(int), s));
    const sr_status st = dt == SR_U8 ? launch_batched_nc<KindU8, 1>(p, s) : launch_batched_nc<KindU16, 1>(p, s);
    p.d_graphs = nullptr; p.d_items = nullptr; p.d_counter = nullptr;   // not owned
    return st;
}

// The grouped schedule's launch lists: blocked Floyd with pivot blocks of 128 run on every
// graph at once, one launch per phase and pivot block (phase 1: one CTA per open graph;
// phase 2: both panels of every graph, 64x64 tiles; phase 3: every other block of every
// graph, 128x128 tiles), graphs in decreasing D so the largest start first in each launch.
static sr_status build_grouped(BatchPlan &p)
{
    if (p.d_gargs || p.d_gactive)
        return SR_OK;
    constexpr int PB = 128;
    const int es = p.dtype == SR_U8 ? 1 : 2;
    int maxnb = 0;
    for (const auto &g : p.h_graphs) maxnb = std::max(maxnb, (g.D + PB - 1) / PB);
    std::vector<int> act, start;
    std::vector<MulArgs> args;
    p.gvec = true;
    for (const auto &g : p.h_graphs) p.gvec = p.gvec && g.pad;
    auto mk = [&](const BatchGraph &g, int64_t a_off, int64_t b_off, int64_t c_off, int R, int K, int N, int rs0,
                  int rsw, int cs0, int csw) {
        MulArgs a;
        char *T = static_cast<char *>(g.T);
        a.A = T + a_off * es; a.B = T + b_off * es; a.C = T + c_off * es;
        a.lda = a.ldb = a.ldc = g.ldt;
        a.R = R; a.K = K; a.N = N;
        a.accumulate = 1;
        a.rskip0 = rs0; a.rskipw = rsw; a.cskip0 = cs0; a.cskipw = csw;
        a.skip_tile = -1;
        return a;
    };
    constexpr int NONE = 0x7fffffff;
    int64_t total_tiles_max = 0;
    for (int kb = 0; kb < maxnb; ++kb) {
        BatchPlan::GroupedStep st{};
        st.act_off = (int)act.size();
        for (int gi : p.order)
            if ((p.h_graphs[gi].D + PB - 1) / PB > kb) act.push_back(gi);
        st.nactive = (int)act.size() - st.act_off;
        for (int kind = 0; kind < 2; ++kind) {            // 0: panels (64x64 tiles), 1: phase 3 (128x128)
            const int off = (int)args.size(), tile = kind == 0 ? 64 : 128;
            int64_t tiles = 0;
            auto add = [&](const MulArgs &a) {
                start.push_back((int)tiles);
                args.push_back(a);
                tiles += (int64_t)((a.R + tile - 1) / tile) * ((a.N + tile - 1) / tile);
            };
            for (int i = st.act_off; i < st.act_off + st.nactive; ++i) {
                const BatchGraph &g = p.h_graphs[act[i]];
                const int D = g.D, k0 = kb * PB, bw = std::min(PB, D - k0);
                const int64_t ld = g.ldt;
                if (D - bw <= 0) continue;                    // a single-block graph: phase 1 only
                if (kind == 0) {
                    add(mk(g, k0 * ld + k0, k0 * ld, k0 * ld, bw, bw, D - bw, NONE, 0, k0, bw));   // row panel
                    add(mk(g, k0, k0 * ld + k0, k0, D - bw, bw, bw, k0, bw, NONE, 0));             // column panel
                } else {
                    add(mk(g, k0, k0 * ld, 0, D - bw, bw, D - bw, k0, bw, k0, bw));                // the rest
                }
            }
            if (tiles > 0x7fffffffLL)
                return fail(SR_EINVAL, "sr_batch: too many tiles in one grouped launch");
            total_tiles_max = std::max(total_tiles_max, tiles);
            if (kind == 0) { st.pan_off = off; st.npan = (int)args.size() - off; st.pan_tiles = (int)tiles; }
            else { st.p3_off = off; st.np3 = (int)args.size() - off; st.p3_tiles = (int)tiles; }
        }
        p.gsteps.push_back(st);
    }
    SR_CUDA_CHECK(cudaMalloc(&p.d_gactive, sizeof(int) * std::max<size_t>(1, act.size())));
    SR_CUDA_CHECK(cudaMalloc(&p.d_gargs, sizeof(MulArgs) * std::max<size_t>(1, args.size())));
    SR_CUDA_CHECK(cudaMalloc(&p.d_gstart, sizeof(int) * std::max<size_t>(1, start.size())));
    if (!act.empty())
        SR_CUDA_CHECK(cudaMemcpy(p.d_gactive, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice));
    if (!args.empty()) {
        SR_CUDA_CHECK(cudaMemcpy(p.d_gargs, args.data(), sizeof(MulArgs) * args.size(), cudaMemcpyHostToDevice));
        SR_CUDA_CHECK(cudaMemcpy(p.d_gstart, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice));
    }
    return SR_OK;
}

static sr_status enqueue_grouped(BatchPlan &p, cudaStream_t s)
{
    SR_TRY(build_grouped(p));
    for (int kb = 0; kb < (int)p.gsteps.size(); ++kb) {
        const BatchPlan::GroupedStep &st = p.gsteps[kb];
        SR_TRY(launch_antidist_pivot_grouped(p.d_graphs, p.d_gactive + st.act_off, st.nactive, kb, p.dtype, s));
        SR_TRY(launch_antidist_mul_grouped(p.d_gargs + st.pan_off, p.d_gstart + st.pan_off, st.npan, st.pan_tiles,
                                           p.dtype, p.gvec, true, s));
        SR_TRY(launch_antidist_mul_grouped(p.d_gargs + st.p3_off, p.d_gstart + st.p3_off, st.np3, st.p3_tiles,
                                           p.dtype, p.gvec, false, s));
        if (p.d_stamps) {                                  // graphs with kb + 1 blocks are done now
            batch_stamp_kernel<<<1, 1, 0, s>>>(p.d_stamps + 1 + p.n + kb);
            SR_CUDA_CHECK(cudaGetLastError());
            count_launches();
        }
    }
    return SR_OK;
}

static sr_status enqueue_batch(BatchPlan &p, cudaStream_t s)
{
    if (p.d_stamps) {
        batch_stamp_kernel<<<1, 1, 0, s>>>(p.d_stamps);
        SR_CUDA_CHECK(cudaGetLastError());
        count_launches();
    }
    if (p.nc == 0)
        return enqueue_grouped(p, s);
    SR_CUDA_CHECK(cudaMemsetAsync(p.d_counter, 0, sizeof(int), s));
    const bool u8 = p.dtype == SR_U8;
    switch (p.nc) {
    case 1: return u8 ? launch_batched_nc<KindU8, 1>(p, s) : launch_batched_nc<KindU16, 1>(p, s);
    case 2: return u8 ? launch_batched_nc<KindU8, 2>(p, s) : launch_batched_nc<KindU16, 2>(p, s);
    default: return u8 ? launch_batched_nc<KindU8, 4>(p, s) : launch_batched_nc<KindU16, 4>(p, s);
    }
}

}  // namespace sr

using namespace sr;

struct sr_batch {
    BatchPlan plan;
};

extern "C" {

sr_status sr_batch_create(sr_ctx *ctx, const sr_desc *d, int n, sr_batch **out)
{
    SR_TRACE("sr_batch_create");
    (void)ctx;
    if (!out || !d || n <= 0)
        return fail(SR_EINVAL, "sr_batch_create: need out, descriptors and n > 0");
    *out = nullptr;
    auto *b = new (std::nothrow) sr_batch();
    if (!b)
        return fail(SR_ENOMEM, "sr_batch_create: host allocation failed");
    BatchPlan &p = b->plan;
    p.n = n;
    p.dtype = (sr_dtype)d[0].dtype;
    for (int i = 0; i < n; ++i) {
        const sr_desc &e = d[i];
        if (e.op != SR_OP_ANTIDIST_CLOSURE || (e.dtype != SR_U8 && e.dtype != SR_U16) || e.dtype != d[0].dtype) {
            delete b;
            return fail(SR_EINVAL, "sr_batch_create: descriptor %d: batches hold anti-distance closures of one dtype", i);
        }
        if (!e.C || e.R <= 0 || e.R > 0x7fffffffLL || e.ldc < e.R) {
            delete b;
            return fail(SR_EINVAL, "sr_batch_create: descriptor %d: bad matrix (C, D = R, ldc >= D)", i);
        }
        BatchGraph g{};
        g.T = e.C;
        g.ldt = e.ldc;
        g.D = (int)e.R;
        const int es = e.dtype == SR_U8 ? 1 : 2;
        g.pad = (aligned16(e.C) && ((e.ldc * es) & 15) == 0) ? 1 : 0;   // vector row accesses allowed
        p.h_graphs.push_back(g);
        p.ops += std::pow((double)g.D, 3.0);
    }
    {   // graphs are closed in place and concurrently: their matrices must not overlap
        const int es = p.dtype == SR_U8 ? 1 : 2;
        std::vector<std::pair<uintptr_t, uintptr_t>> sp;
        for (const auto &g : p.h_graphs) {
            const uintptr_t lo = reinterpret_cast<uintptr_t>(g.T);
            sp.push_back({lo, lo + (uintptr_t)(((int64_t)(g.D - 1) * g.ldt + g.D) * es)});
        }
        std::sort(sp.begin(), sp.end());
        for (size_t i = 1; i < sp.size(); ++i)
            if (sp[i].first < sp[i - 1].second) {
                delete b;
                return fail(SR_EINVAL, "sr_batch_create: two graphs of the batch overlap in memory");
            }
    }
    p.device = current_device();     // after the argument checks, which need no device
    if (p.device < 0) {
        delete b;
        return fail(SR_ECUDA, "sr_batch_create: no current CUDA device with an id below %d", kMaxDevices);
    }
    p.order.resize(n);
    std::iota(p.order.begin(), p.order.end(), 0);
    std::stable_sort(p.order.begin(), p.order.end(),
                     [&](int a, int c) { return p.h_graphs[a].D > p.h_graphs[c].D; });
    cudaError_t e = cudaMalloc(&p.d_graphs, sizeof(BatchGraph) * n);
    if (e == cudaSuccess) e = cudaMemcpy(p.d_graphs, p.h_graphs.data(), sizeof(BatchGraph) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p.d_counter, sizeof(int));
    if (e != cudaSuccess) {
        sr_batch_destroy(b);
        return cuda_fail(e, "sr_batch_create");
    }
    const sr_status st = build_items(p);
    if (st != SR_OK) {
        sr_batch_destroy(b);
        return st;
    }
    *out = b;
    return SR_OK;
}

sr_status sr_batch_set_tuning(sr_batch *b, int cluster, int coop_threshold, int ctas_per_sm)
{
    SR_TRACE("sr_batch_set_tuning");
    if (!b)
        return fail(SR_EINVAL, "sr_batch_set_tuning: NULL batch");
    if ((cluster != 0 && cluster != 1 && cluster != 2 && cluster != 4) || coop_threshold < 1 || ctas_per_sm < 1 ||
        ctas_per_sm > 8)
        return fail(SR_EINVAL, "sr_batch_set_tuning: cluster in {0,1,2,4} (0: grouped launches per pivot block), "
                               "threshold >= 1, 1 <= ctas_per_sm <= 8");
    BatchPlan &p = b->plan;
    p.nc = cluster;
    p.coop_threshold = coop_threshold;
    p.ctas_per_sm = ctas_per_sm;
    if (p.exec) { cudaGraphExecDestroy(p.exec); p.exec = nullptr; }
    if (p.graph) { cudaGraphDestroy(p.graph); p.graph = nullptr; }
    if (cluster == 0)
        SR_TRY(build_grouped(p));            // device arrays now, never during a capture
    return build_items(p);
}

sr_status sr_batch_get_tuning(const sr_batch *b, int *cluster, int *coop_threshold, int *ctas_per_sm)
{
    SR_TRACE("sr_batch_get_tuning");
    if (!b || !cluster || !coop_threshold || !ctas_per_sm)
        return fail(SR_EINVAL, "sr_batch_get_tuning: NULL argument");
    *cluster = b->plan.nc;
    *coop_threshold = b->plan.coop_threshold;
    *ctas_per_sm = b->plan.ctas_per_sm;
    return SR_OK;
}

sr_status sr_batch_launch(sr_batch *b, int use_graph, void *stream)
{
    SR_TRACE("sr_batch_launch");
    if (!b)
        return fail(SR_EINVAL, "sr_batch_launch: NULL batch");
    BatchPlan &p = b->plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!use_graph)
        return enqueue_batch(p, s);
    if (!p.exec) {
        if (p.nc == 0)
            SR_TRY(build_grouped(p));        // allocates: must precede the capture
        // capture counter reset + persistent kernel once, on a private stream
        cudaStream_t cs;
        SR_CUDA_CHECK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        sr_status st = SR_OK;
        if (e == cudaSuccess) st = enqueue_batch(p, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) return cuda_fail(e, "sr_batch_launch: begin capture");
        if (st != SR_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e2 != cudaSuccess) return cuda_fail(e2, "sr_batch_launch: end capture");
        p.graph = g;
        SR_CUDA_CHECK(cudaGraphInstantiate(&p.exec, p.graph, 0));
    }
    SR_CUDA_CHECK(cudaGraphLaunch(p.exec, s));
    count_launches();
    return SR_OK;
}

sr_status sr_batch_set_timing(sr_batch *b, int enable)
{
    SR_TRACE("sr_batch_set_timing");
    if (!b)
        return fail(SR_EINVAL, "sr_batch_set_timing: NULL batch");
    BatchPlan &p = b->plan;
    if ((enable != 0) == (p.d_stamps != nullptr))
        return SR_OK;
    if (p.exec) { cudaGraphExecDestroy(p.exec); p.exec = nullptr; }    // recaptured with or without stamps
    if (p.graph) { cudaGraphDestroy(p.graph); p.graph = nullptr; }
    if (!enable) {
        cudaFree(p.d_stamps);
        p.d_stamps = nullptr;
        return SR_OK;
    }
    int maxnb = 0;
    for (const auto &g : p.h_graphs) maxnb = std::max(maxnb, (g.D + 127) / 128);
    SR_CUDA_CHECK(cudaMalloc(&p.d_stamps, sizeof(uint64_t) * (size_t)(1 + p.n + maxnb)));
    SR_CUDA_CHECK(cudaMemset(p.d_stamps, 0, sizeof(uint64_t) * (size_t)(1 + p.n + maxnb)));
    return SR_OK;
}

sr_status sr_batch_completion_ms(const sr_batch *b, double *ms)
{
    SR_TRACE("sr_batch_completion_ms");
    if (!b || !ms)
        return fail(SR_EINVAL, "sr_batch_completion_ms: NULL batch or output");
    const BatchPlan &p = b->plan;
    if (!p.d_stamps)
        return fail(SR_EINVAL, "sr_batch_completion_ms: timing is off (sr_batch_set_timing)");
    int maxnb = 0;
    for (const auto &g : p.h_graphs) maxnb = std::max(maxnb, (g.D + 127) / 128);
    std::vector<uint64_t> h((size_t)(1 + p.n + maxnb));
    SR_CUDA_CHECK(cudaMemcpy(h.data(), p.d_stamps, sizeof(uint64_t) * h.size(), cudaMemcpyDeviceToHost));
    for (int g = 0; g < p.n; ++g) {
        const uint64_t end = p.nc == 0 ? h[1 + p.n + (p.h_graphs[g].D + 127) / 128 - 1] : h[1 + g];
        ms[g] = end >= h[0] ? (double)(end - h[0]) * 1e-6 : -1.0;
    }
    return SR_OK;
}

sr_status sr_batch_info(const sr_batch *b, int *ngraphs, int *nitems, double *ops)
{
    SR_TRACE("sr_batch_info");
    if (!b)
        return fail(SR_EINVAL, "sr_batch_info: NULL batch");
    if (ngraphs) *ngraphs = b->plan.n;
    if (nitems) *nitems = b->plan.nitems;
    if (ops) *ops = b->plan.ops;
    return SR_OK;
}

void sr_batch_destroy(sr_batch *b)
{
    SR_TRACE("sr_batch_destroy");
    if (!b)
        return;
    BatchPlan &p = b->plan;
    if (p.exec) cudaGraphExecDestroy(p.exec);
    if (p.graph) cudaGraphDestroy(p.graph);
    if (p.d_graphs) cudaFree(p.d_graphs);
    if (p.d_items) cudaFree(p.d_items);
    if (p.d_counter) cudaFree(p.d_counter);
    if (p.d_gactive) cudaFree(p.d_gactive);
    if (p.d_stamps) cudaFree(p.d_stamps);
    if (p.d_gargs) cudaFree(p.d_gargs);
    if (p.d_gstart) cudaFree(p.d_gstart);
    delete b;
}

// Tuning signature: dtype, SM count, and the histogram of D over power-of-two buckets.
static std::string batch_signature(const BatchPlan &p)
{
    int hist[32] = {};
    for (const auto &g : p.h_graphs) {
        int b = 0;
        while ((1 << (b + 1)) <= g.D && b < 31) ++b;
        ++hist[b];
    }
    std::string sig = "batched_closure dtype=" + std::to_string((int)p.dtype) + " sms=" +
                      std::to_string(device_sm_count()) + " hist=";
    for (int b = 0; b < 32; ++b)
        if (hist[b]) sig += std::to_string(b) + ":" + std::to_string(hist[b]) + ",";
    return sig;
}

sr_status sr_batch_autotune(sr_ctx *ctx, sr_batch *b, void *stream, int reps, double *best_ms)
{
    SR_TRACE("sr_batch_autotune");
    if (!b)
        return fail(SR_EINVAL, "sr_batch_autotune: NULL batch");
    BatchPlan &p = b->plan;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const std::string sig = batch_signature(p);
    if (ctx) {
        auto it = ctx->tune.find(sig);
        if (it != ctx->tune.end()) {
            const auto &v = it->second;
            if (best_ms) *best_ms = -1.0;
            return sr_batch_set_tuning(b, v[0], v[1], v[2]);
        }
    }
    reps = std::max(1, reps);
    cudaEvent_t e0, e1;
    SR_CUDA_CHECK(cudaEventCreate(&e0));
    SR_CUDA_CHECK(cudaEventCreate(&e1));
    struct Cand { int nc, thr, cps; };
    std::vector<Cand> cands;
    cands.push_back({0, 1 << 30, 1});                  // grouped launches per pivot block
    for (int cps : {1, 2})
        cands.push_back({1, 1 << 30, cps});
    for (int nc : {2, 4})
        for (int thr : {256, 384, 512, 768})
            for (int cps : {1, 2})
                cands.push_back({nc, thr, cps});
    double best = 1e30;
    Cand bc = cands[0];
    sr_status st = SR_OK;
    for (const Cand &c : cands) {
        // the closure is idempotent: re-running it on closed graphs leaves them unchanged
        if ((st = sr_batch_set_tuning(b, c.nc, c.thr, c.cps)) != SR_OK) break;
        if ((st = enqueue_batch(p, s)) != SR_OK) break;          // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == SR_OK; ++r) st = enqueue_batch(p, s);
        cudaEventRecord(e1, s);
        if (st != SR_OK) break;
        const cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { st = cuda_fail(e, "sr_batch_autotune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms / reps < best) { best = ms / reps; bc = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SR_OK)
        return st;
    if (ctx) {
        ctx->tune[sig] = {bc.nc, bc.thr, bc.cps};
        SR_TRY(tune_persist(ctx));                              // the ctx's tune cache, if any
    }
    if (best_ms) *best_ms = best;
    return sr_batch_set_tuning(b, bc.nc, bc.thr, bc.cps);
}

sr_status sr_batched(sr_ctx *ctx, const sr_desc *d, int n, void *stream)
{
    SR_TRACE("sr_batched");
    sr_batch *b = nullptr;
    SR_TRY(sr_batch_create(ctx, d, n, &b));
    sr_status st = SR_OK;
    if (ctx) {      // apply a tuning found earlier for batches of this shape, if any
        auto it = ctx->tune.find(batch_signature(b->plan));
        if (it != ctx->tune.end()) st = sr_batch_set_tuning(b, it->second[0], it->second[1], it->second[2]);
    }
    if (st == SR_OK) st = sr_batch_launch(b, 0, stream);
    if (st == SR_OK) {
        // the plan's device arrays must outlive the launch
        const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) st = cuda_fail(e, "sr_batched: synchronize");
    }
    sr_batch_destroy(b);
    return st;
}

}  // extern "C"
