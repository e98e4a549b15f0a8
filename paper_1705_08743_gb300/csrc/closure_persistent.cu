// The whole anti-distance closure (u8, u16) in one persistent launch.
//
// Method: Section 2's Warshall loop, generalised by Section 3 to anti-distance
// matrices (Floyd), in the blocked three-phase order with 128-wide pivot blocks:
// for pivot block s, the diagonal block is closed (phase 1), the row and column
// panels take T_sj := T_sj ⊕ T_ss ⊗ T_sj and T_is := T_is ⊕ T_is ⊗ T_ss
// (phase 2), and every other block takes T_ij ⊕= T_is ⊗ T_sj (phase 3).
//
// The stream schedules of closure.cu pay, once per pivot block, for a launch, a
// ramp-up and a partly empty last wave of CTAs.  Here every CTA pulls work items
// from one counter, in a fixed order, until none are left: phase-3 tiles of
// 128×128 entries (on the grid of the matrix without block row and column s),
// panel tiles of the same size, and diagonal blocks.  The tail of one
// pivot block's phase 3 overlaps the next one's, and the next diagonal block and
// panels are computed beside the bulk of the current phase 3.
//
// Ordering.  Every 128×128 block (I, J) carries a version: the number of pivot
// blocks already applied to it.  Each pivot block s updates each block exactly
// once (phase 3 if I ≠ s ≠ J, a panel if one of them is s, phase 1 if both), so
// an item of pivot block s waits until the blocks it writes have version s and
// the panel blocks it reads (T_is, T_sj; T_ss for panels) have version s + 1,
// then raises the versions of what it wrote to s + 1.  Reading an operand that a
// later pivot block has already raised is harmless: every entry always lies
// between its value in the plain Warshall order and the closure, and ⊗ is
// monotone, so a larger operand still gives an entry no larger than the closure.
// The order lists every item after the items it waits for, and items are taken
// only by running CTAs, so the earliest unfinished item can always proceed: no
// CTA waits on a CTA that has not started, and the launch needs no co-residency.
// Every wait is still bounded (the context's spin limit); a wait that gives up
// sets an error flag that stops every CTA and the context's status word
// (sr_stream_status then reports SR_ETIMEOUT).
//
// Loads of T go through L2 only (ld.global.cg / cp.async.cg): the entries were
// written by other CTAs of the same launch.  Versions are published with a
// fence and a release store after the CTA's barrier, and read with acquire
// loads before the barrier that starts the item.

#include <algorithm>

#include "antidist_tile.cuh"
#include "diag128.cuh"
#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {
namespace {

constexpr int PW = 128;         // pivot block width
constexpr int BPT = 1;          // pivot blocks per phase-3 tile side (TT / PW)
constexpr int PBK = 32;         // k-panel depth of the product tiles (deeper panels spill registers)
constexpr int TT = 128;         // phase-3 tile (entries per side)
constexpr int PC_COMPUTE = 128;    // four compute warps
constexpr int PC_THREADS = 160;    // and one control warp
constexpr int BAR_TILE = 1, BAR_READY = 2;   // named barriers (0 is __syncthreads)
// Tries of the control warp's wait for its own compute warps, which always finish: the
// bound only keeps a fault from turning into a hang.
constexpr uint32_t tc_done_limit = 1u << 28;
constexpr int WS_HEADER = 32;   // ints before the version table: [0] item counter, [1] error flag

struct PcArgs {
    void *T;
    int64_t ldt;
    int D, nb;                  // order, number of 64-wide blocks
    int t3m, t3l;               // 128-tiles per side of the phase-3 grid: pivot blocks < nb-1, the last one
    long long p0, lm, items;    // prologue items, items of a full pivot step, all items
    int frac;                   // phase-3 tiles of a step before the next panels, in 1/256 of the rest
    int *ver;                   // nb × nb block versions (zeroed before the launch)
    int *counter;               // next item
    int *err;                   // set when a wait gives up
    int *status;                // context status words ([0] code, [1] where), may be null
    uint32_t limit;             // tries per wait
};

__host__ __device__ __forceinline__ int imin(int x, int y) { return x < y ? x : y; }
__host__ __device__ __forceinline__ int imax(int x, int y) { return x > y ? x : y; }

enum : int { IT_P3 = 0, IT_ROW = 1, IT_COL = 2, IT_DIAG = 3 };

struct Item {
    int type, s, i, j;          // pivot block s; tile coordinates on that block's grid
    int j2;                     // phase 3: a second tile (i, j2) of the same item, or -1
};

__host__ __device__ __forceinline__ int t3_of(const PcArgs &a, int s) { return s == a.nb - 1 ? a.t3l : a.t3m; }
__host__ __device__ __forceinline__ int skip_s(int x, int s) { return x < s ? x : x + 1; }   // grid block -> matrix block

// Tile rows/columns of pivot step s's cross: c0 and c0 + 1 with c0 = min(s / BPT, T - 2)
// (one when T = 1).  They hold the matrix blocks after s (grid indices s, s + 1, ...) where
// the grid has them: block s + 1 feeds the next diagonal block and panels, the blocks after
// it the next step's cross.
__host__ __device__ __forceinline__ int cross_count(int T) { return T >= 2 ? 2 : 1; }
__host__ __device__ __forceinline__ int cross_first(int T, int s) { return T >= 2 ? imin(s / BPT, T - 2) : 0; }

// Items of pivot step s's sequence: the cross (single tiles), the next diagonal block,
// (T - nc) rows of ceil((T - nc) / 2) two-tile items, the next pivot block's 2·Tn panel tiles.
__host__ __device__ __forceinline__ long long seq_len(int T, bool next, int Tn)
{
    const int nc = cross_count(T), Tr = T - nc;
    return (long long)T * T - (long long)Tr * Tr + (next ? 1 : 0) + (long long)Tr * ((Tr + 1) / 2) +
           (next ? 2LL * Tn : 0);
}

// Panel items of pivot block p, m in [0, 2·T): the tiles that hold block p + 1 come first.
__host__ __device__ __forceinline__ Item panel_item(const PcArgs &a, int p, int m)
{
    const int T = t3_of(a, p), c1 = imin(p / BPT, T - 1);
    if (m < 2) return {m == 0 ? IT_ROW : IT_COL, p, c1, c1, -1};
    const int u = (m - 2) >> 1, t = u < c1 ? u : u + 1;
    return {((m - 2) & 1) ? IT_COL : IT_ROW, p, t, t, -1};
}

// Sequence of pivot step s: the cross (first the tile (d, d) that holds block s + 1, then
// rows c0 and c0 + 1, then columns c0 and c0 + 1 in the other rows), the diagonal block
// s + 1, a share of the other phase-3 tiles (two adjacent tiles of a row per item), the
// panels of s + 1, the rest.
__host__ __device__ __forceinline__ Item step_item(const PcArgs &a, int s, long long r)
{
    const int T = t3_of(a, s), c0 = cross_first(T, s), nc = cross_count(T), Tr = T - nc;
    const bool next = s + 1 < a.nb;
    const int P = (Tr + 1) / 2;                            // two-tile items per row outside the cross
    const long long X = (long long)T * T - (long long)Tr * Tr, R = (long long)Tr * P, F = R * a.frac / 256;
    if (r < X) {
        const int d = imin(s / BPT, T - 1);                // the tile that holds block s + 1
        int m = (int)r;
        if (m == 0) return {IT_P3, s, d, d, -1};
        m -= 1;
        if (m < nc * T - 1) {                              // rows c0 .. c0 + nc - 1, (d, d) left out
            const int u = m < (d - c0) * T + d ? m : m + 1;
            return {IT_P3, s, c0 + u / T, u % T, -1};
        }
        m -= nc * T - 1;                                   // columns c0, c0 + 1 in the other rows
        const int x = m % (T - nc);
        return {IT_P3, s, x < c0 ? x : x + nc, c0 + m / (T - nc), -1};
    }
    r -= X;
    if (next) {
        if (r == 0) return {IT_DIAG, s + 1, 0, 0, -1};
        r -= 1;
    }
    long long rest;
    if (r < F) {
        rest = r;
    } else {
        r -= F;
        const long long nd = next ? 2LL * t3_of(a, s + 1) : 0;
        if (r < nd) return panel_item(a, s + 1, (int)r);
        rest = F + (r - nd);
    }
    if (P == 0) return {IT_P3, s, 0, 0, -1};               // no tiles outside the cross (not reached)
    const int ip = (int)(rest / P), jp = 2 * (int)(rest % P);
    const int j1 = jp < c0 ? jp : jp + nc;
    const int j2 = jp + 1 < Tr ? (jp + 1 < c0 ? jp + 1 : jp + 1 + nc) : -1;
    return {IT_P3, s, ip < c0 ? ip : ip + nc, j1, j2};
}

__host__ __device__ __forceinline__ Item decode(const PcArgs &a, long long q)
{
    if (q == 0) return {IT_DIAG, 0, 0, 0, -1};
    if (q < a.p0) return panel_item(a, 0, (int)(q - 1));
    q -= a.p0;
    const long long full = (long long)imax(a.nb - 2, 0) * a.lm;
    if (q < full) return step_item(a, (int)(q / a.lm), q % a.lm);
    q -= full;
    const int s = a.nb - 2;        // the last two steps (nb >= 2)
    const long long Ls = seq_len(a.t3m, true, a.t3l);
    if (q < Ls) return step_item(a, s, q);
    return step_item(a, s + 1, q - Ls);
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int *p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Matrix blocks an item writes (rows × columns, at most 2 × 4).
struct Blocks {
    int r[2], c[4], nr, nc;
};

__host__ __device__ __forceinline__ Blocks written(const PcArgs &a, const Item &it)
{
    Blocks b;
    const int nbc = a.nb - 1;      // blocks on the grid without block s
    b.nr = b.nc = 0;
    auto two = [&](int t, int *dst, int &n) {
        for (int x = BPT * t; x < BPT * t + BPT && x < nbc; ++x) dst[n++] = skip_s(x, it.s);
    };
    if (it.type == IT_DIAG) {
        b.r[0] = b.c[0] = it.s;
        b.nr = b.nc = 1;
    } else if (it.type == IT_P3) {
        two(it.i, b.r, b.nr);
        two(it.j, b.c, b.nc);
        if (it.j2 >= 0) two(it.j2, b.c, b.nc);
    } else if (it.type == IT_ROW) {
        b.r[0] = it.s;
        b.nr = 1;
        two(it.j, b.c, b.nc);
    } else {
        two(it.i, b.r, b.nr);
        b.c[0] = it.s;
        b.nc = 1;
    }
    return b;
}

// Condition k of an item (k < count): the version table entry and the version it needs.
// Written blocks need version s, phase-3 operand panels (T_is, T_sj) and, for panel
// items, the closed diagonal block need s + 1.
__device__ __forceinline__ int conditions(const PcArgs &a, const Item &it, const Blocks &b, int k, const int **ptr)
{
    const int nb = a.nb, s = it.s, nw = b.nr * b.nc;
    if (k < nw) {
        *ptr = a.ver + (int64_t)b.r[k / b.nc] * nb + b.c[k % b.nc];
        return s;
    }
    k -= nw;
    if (it.type == IT_P3) {
        *ptr = k < b.nr ? a.ver + (int64_t)b.r[k] * nb + s : a.ver + (int64_t)s * nb + b.c[k - b.nr];
        return s + 1;
    }
    *ptr = a.ver + (int64_t)s * nb + s;
    return s + 1;
}
__device__ __forceinline__ int condition_count(const Item &it, const Blocks &b)
{
    const int nw = b.nr * b.nc;
    return it.type == IT_P3 ? nw + b.nr + b.nc : it.type == IT_DIAG ? nw : nw + 1;
}

// The control warp, once the compute warps report the item done: its blocks now have
// version s + 1 (one release store per lane; the compute warps' stores come before it
// through their barrier and the release/acquire of the done count in shared memory).
__device__ __forceinline__ void publish_warp(const PcArgs &a, const Item &it, const Blocks &b)
{
    const int lane = threadIdx.x & 31, nw = b.nr * b.nc;
    if (lane < nw) st_release(a.ver + (int64_t)b.r[lane / b.nc] * a.nb + b.c[lane % b.nc], it.s + 1);
}

// ---------------------------------------------------------------- phase 1: one 128×128 block
// (diag128.cuh: the block closed in shared memory by the four compute warps)
using diag::kDiagLdx;
constexpr size_t DIAG_SMEM = diag::kDiagSmem;
static_assert(diag::kDiagW == PW && diag::kDiagThreads == PC_COMPUTE, "one diagonal-block shape");

template <class KD>
__device__ __forceinline__ void close_diag(const PcArgs &a, int s)
{
    extern __shared__ __align__(16) uint32_t smem[];
    diag::close_diag128<KD, BAR_TILE>(static_cast<typename KD::elem *>(a.T), a.ldt, a.D, s * PW, smem);
}

// ---------------------------------------------------------------- phases 2 and 3: product tiles
template <class KD>
__device__ __forceinline__ void run_product(const PcArgs &a, const Item &it)
{
    using E = typename KD::elem;
    E *T = static_cast<E *>(a.T);
    const int s = it.s, k0 = s * PW, bw = min(PW, a.D - k0), Dc = a.D - bw, tn = t3_of(a, s);
    const int64_t ld = a.ldt;
    MulArgs p;
    p.lda = p.ldb = p.ldc = ld;
    p.K = bw;
    p.accumulate = 1;
    p.skip_tile = -1;
    if (it.type == IT_P3) {          // T_ij ⊕= T_is ⊗ T_sj outside block row and column s
        p.A = T + k0; p.B = T + (int64_t)k0 * ld; p.C = T;
        p.R = Dc; p.N = Dc;
        p.rskip0 = k0; p.rskipw = bw; p.cskip0 = k0; p.cskipw = bw;
        const int t1 = it.i * tn + it.j;
        if (it.j2 < 0)
            mul_tiles<KD, TT, TT, PBK, 8, 16, true, true, BAR_TILE>(p, t1, tn * tn, t1 + 1);
        else                          // two tiles of row i; the second's first k-panel loads during the first
            mul_tiles<KD, TT, TT, PBK, 8, 16, true, true, BAR_TILE>(p, t1, it.j2 - it.j, it.i * tn + it.j2 + 1);
    } else if (it.type == IT_ROW) {  // T_sj := T_sj ⊕ T_ss ⊗ T_sj, in place
        p.A = T + (int64_t)k0 * ld + k0; p.B = T + (int64_t)k0 * ld; p.C = T + (int64_t)k0 * ld;
        p.R = bw; p.N = Dc;
        p.rskip0 = 0x7fffffff; p.rskipw = 0; p.cskip0 = k0; p.cskipw = bw;
        mul_tiles<KD, PW, TT, PBK, PW / 16, 16, true, true, BAR_TILE>(p, it.j, tn);
    } else {                          // T_is := T_is ⊕ T_is ⊗ T_ss, in place
        p.A = T + k0; p.B = T + (int64_t)k0 * ld + k0; p.C = T + k0;
        p.R = Dc; p.N = bw;
        p.rskip0 = k0; p.rskipw = bw; p.cskip0 = 0x7fffffff; p.cskipw = 0;
        mul_tiles<KD, TT, PW, PBK, 8, PW / 8, true, true, BAR_TILE>(p, it.i, tn);
    }
}

template <class KD>
struct PcCfg {
    using P3 = MulCfg<KD, TT, TT, PBK, 8, 16>;
    using Row = MulCfg<KD, PW, TT, PBK, PW / 16, 16>;
    using Col = MulCfg<KD, TT, PW, PBK, 8, PW / 8>;
    static constexpr size_t SMEM = std::max({P3::SMEM, Row::SMEM, Col::SMEM, DIAG_SMEM});
    static_assert(P3::THREADS == PC_COMPUTE && Row::THREADS == PC_COMPUTE && Col::THREADS == PC_COMPUTE,
                  "one compute shape for every item");
    static_assert(BPT * PW == TT, "phase-3 tiles hold whole pivot blocks");
    // CTAs per SM the register budget is sized for: u8 two (three would cap a thread at
    // 128 registers and spill the product tile's accumulators), u16 one (its 115 KB of
    // shared memory fit once)
    static constexpr int MIN_BLOCKS = sizeof(typename KD::elem) == 1 ? 2 : 1;
};

__device__ __forceinline__ void bar_arrive160(int id)
{
    asm volatile("bar.arrive %0, 160;\n" ::"r"(id) : "memory");
}
__device__ __forceinline__ void bar_sync160(int id)
{
    asm volatile("bar.sync %0, 160;\n" ::"r"(id) : "memory");
}
__device__ __forceinline__ void st_release_cta(int *p, int v)
{
    asm volatile("st.release.cta.shared::cta.s32 [%0], %1;\n" ::"r"((uint32_t)__cvta_generic_to_shared(p)), "r"(v)
                 : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int *p)
{
    int v;
    asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];\n" : "=r"(v) : "r"((uint32_t)__cvta_generic_to_shared(p))
                 : "memory");
    return v;
}

// Warps 0-3 compute items; warp 4 runs the schedule for them.  While the compute warps
// work on item n - 1, the control warp claims item n, decodes it and waits for its
// conditions; it publishes item n - 1's versions as soon as the compute warps report it
// done (s_done, written after their barrier), whether or not item n is ready yet — so no
// CTA sits on finished work while it waits for another CTA — and hands item n over in a
// shared-memory slot (named barrier READY) once item n - 1 is done.  The compute warps
// never wait on global memory for the schedule.
template <class KD>
__global__ void __launch_bounds__(PC_THREADS, PcCfg<KD>::MIN_BLOCKS)
antidist_closure_persistent_kernel(PcArgs a)
{
    __shared__ Item s_it[2];
    __shared__ int s_end[2];
    __shared__ int s_done;                                 // items the compute warps finished
    const int tid = threadIdx.x;
    if (tid == 0) s_done = 0;
    __syncthreads();
    if (tid < PC_COMPUTE) {
        for (int n = 0;; ++n) {
            bar_sync160(BAR_READY);
            if (s_end[n & 1]) break;
            const Item it = s_it[n & 1];
            if (it.type == IT_DIAG)
                close_diag<KD>(a, it.s);
            else
                run_product<KD>(a, it);
            tile_sync<BAR_TILE>();                         // every compute thread's stores issued
            if (tid == 0) st_release_cta(&s_done, n + 1);
        }
        return;
    }
    const int lane = tid & 31;
    const unsigned full = 0xffffffffu;
    auto claim = [&]() -> long long {
        int q = 0;
        if (lane == 0) q = ld_relaxed(a.err) ? (int)a.items : atomicAdd(a.counter, 1);
        return (long long)__shfl_sync(full, q, 0);
    };
    auto done_count = [&]() { return __shfl_sync(full, lane == 0 ? ld_acquire_cta(&s_done) : 0, 0); };
    Item prev{};
    Blocks pb{};
    bool published = true;                                 // item n - 1's versions are out
    long long q = claim();
    for (int n = 0;; ++n) {
        bool end = q >= a.items;
        Item it{};
        Blocks b{};
        if (!end) {
            it = decode(a, q);
            b = written(a, it);
            // wait for item n's conditions, one per lane; publish item n - 1 once it is done
            const int nc = condition_count(it, b);
            const int *p = nullptr;
            const int need = lane < nc ? conditions(a, it, b, lane, &p) : 0;
            bool ok = lane >= nc;
            for (uint32_t t = 0;; ++t) {
                if (!published && done_count() >= n) {
                    publish_warp(a, prev, pb);
                    published = true;
                }
                if (!ok) ok = ld_acquire(p) >= need;
                if (__all_sync(full, ok)) break;
                if (t >= a.limit || ((t & 15u) == 15u && __any_sync(full, lane == 0 && ld_relaxed(a.err)))) {
                    if (lane == 0) {
                        atomicExch(a.err, 1);
                        if (a.status) {
                            atomicExch(a.status + 1, 3);   // where: the persistent closure
                            atomicExch(a.status, 1);
                        }
                    }
                    end = true;
                    break;
                }
                __nanosleep(t < 32 ? 20 : 200);
            }
        }
        // the compute warps finish item n - 1 (finite work, no waits) before item n is handed over
        for (uint32_t t = 0; done_count() < n && t < tc_done_limit; ++t) __nanosleep(32);
        if (lane == 0) {
            s_it[n & 1] = it;
            s_end[n & 1] = end ? 1 : 0;
        }
        __syncwarp();
        bar_arrive160(BAR_READY);
        if (!published) publish_warp(a, prev, pb);
        if (end) break;
        prev = it;
        pb = b;
        published = false;
        q = claim();
    }
}

// Host-side copies of the order's sizes (the same formulas as the device side).
struct PcShape {
    int nb, t3m, t3l;
    long long p0, lm, items;
};
PcShape pc_shape(int D)
{
    PcShape sh;
    sh.nb = (D + PW - 1) / PW;
    sh.t3m = (D - PW + TT - 1) / TT;
    sh.t3l = (PW * (sh.nb - 1) + TT - 1) / TT;
    sh.p0 = 1 + 2LL * sh.t3m;
    sh.lm = seq_len(sh.t3m, true, sh.t3m);
    sh.items = sh.p0 + (long long)std::max(sh.nb - 2, 0) * sh.lm + seq_len(sh.t3m, true, sh.t3l) +
               seq_len(sh.t3l, false, 0);
    return sh;
}

template <class KD>
sr_status launch_pc(const PcArgs &a, cudaStream_t s)
{
    using Cfg = PcCfg<KD>;
    auto kern = antidist_closure_persistent_kernel<KD>;
    static int per_sm[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!per_sm[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
        int n = 0;
        SR_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, PC_THREADS, Cfg::SMEM));
        per_sm[dev] = std::max(n, 1);
    }
    const long long want = std::min<long long>(a.items, (long long)device_sm_count() * per_sm[dev]);
    kern<<<(unsigned)want, PC_THREADS, Cfg::SMEM, s>>>(a);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace

long long antidist_closure_persistent_order(int64_t D, int frac, int *out, long long cap)
{
    if (D < 2 * PW || D > kPersistentMaxD) return -1;
    const PcShape sh = pc_shape((int)D);
    PcArgs a{};
    a.D = (int)D;
    a.nb = sh.nb;
    a.t3m = sh.t3m;
    a.t3l = sh.t3l;
    a.p0 = sh.p0;
    a.lm = sh.lm;
    a.items = sh.items;
    a.frac = std::min(std::max(frac, 0), 256);
    for (long long q = 0; out && q < std::min(cap, sh.items); ++q) {
        const Item it = decode(a, q);
        int *o = out + 5 * q;
        o[0] = it.type; o[1] = it.s; o[2] = it.i; o[3] = it.j; o[4] = it.j2;
    }
    return sh.items;
}

size_t antidist_closure_persistent_workspace(int64_t D)
{
    if (D < 2 * PW || D > kPersistentMaxD) return 0;
    const int64_t nb = (D + PW - 1) / PW;
    return (size_t)(WS_HEADER + nb * nb) * sizeof(int);
}

sr_status launch_antidist_closure_persistent(void *T, int64_t ldt, int D, sr_dtype dt, void *ws, size_t ws_bytes,
                                             int *status, int spin_limit, int frac, cudaStream_t s)
{
    if (dt != SR_U8 && dt != SR_U16)
        return fail(SR_EINVAL, "antidist_closure (persistent): u8 or u16 only");
    const size_t need = antidist_closure_persistent_workspace(D);
    if (need == 0 || !ws || ws_bytes < need)
        return fail(SR_EINVAL, "antidist_closure (persistent): D = %d needs %zu workspace bytes (have %zu)", D, need,
                    ws_bytes);
    const PcShape sh = pc_shape(D);
    SR_CUDA_CHECK(cudaMemsetAsync(ws, 0, need, s));
    PcArgs a;
    a.T = T;
    a.ldt = ldt;
    a.D = D;
    a.nb = sh.nb;
    a.t3m = sh.t3m;
    a.t3l = sh.t3l;
    a.p0 = sh.p0;
    a.lm = sh.lm;
    a.items = sh.items;
    a.frac = std::min(std::max(frac, 0), 256);
    int *w = static_cast<int *>(ws);
    a.counter = w;
    a.err = w + 1;
    a.ver = w + WS_HEADER;
    a.status = status;
    a.limit = (uint32_t)std::max(0, spin_limit);
    return dt == SR_U8 ? launch_pc<KindU8>(a, s) : launch_pc<KindU16>(a, s);
}

}  // namespace sr
