// Boolean product on the 5th-generation tensor cores: count, then test > 0.
//
// (A ⊗ B)_ij = OR_k (A_ik AND B_kj) equals [Σ_k A_ik·B_kj > 0] over the integers
// (Section 2's ∨/∧ product read as a count).  A and B are expanded from bits to
// fp8 e4m3 bytes (1.0 = 0x38, 0 = 0x00), multiplied by tcgen05.mma (kind::f8f6f4,
// fp32 accumulation in tensor memory), and each fp32 count becomes one bit again.
// Exact: every product is 0 or 1, every partial sum a non-negative integer, and
// rounding a sum of non-negative numbers never reaches 0 from a positive value
// (below 2^24, fp32 holds the counts exactly anyway).
//
// Kernel: persistent, one CTA per SM (8 warps), output tiles of 128×256 (M = 128,
// N = 256 per MMA, K = 32 per MMA).  A producer lane streams 128-byte-deep K slices of A
// (128 rows) and B^T (256 rows) with TMA into a 4-stage shared-memory ring (128-byte
// swizzle); an MMA lane issues the MMAs into one of two tensor-memory accumulators and
// releases each stage with tcgen05.commit; four epilogue warps read their 32 accumulator
// lanes (tcgen05.ld), turn 32 counts into one 32-bit word and OR it into C while the next
// tile accumulates in the other buffer.  Every wait on an mbarrier is bounded; a wait that
// gives up sets a status word and the CTA stops issuing work, waits (bounded) for the
// copies and MMAs it started, frees its tensor memory and returns.

#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "sr_common.cuh"
#include "sr_kernels.h"

namespace sr {

namespace tc {
constexpr int BM = 128, BN = 256, BK = 128;          // BK in bytes = fp8 elements
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK, B_BYTES = BN * BK;
constexpr uint32_t DRAIN_LIMIT = 1u << 24;    // tries per wait for work already started, on the failure path
constexpr int GROUP_M = 16;                  // tile rows per rasterisation group
}  // namespace tc

struct BoolTcArgs {
    uint32_t *C;
    int64_t ldc;          // 32-bit words
    int R, N;             // rows of C; bits per row of C (pad bits written 0)
    int ncw;              // 32-bit words per row of C to write
    int nkb;              // K slices of BK bytes
    int tiles_m, tiles_n; // output tiles (BM rows, BN columns)
    int accumulate;
    int *status;          // nonzero after a bounded wait gave up (may be null)
    uint32_t wait_limit;  // tries per wait before giving up (the context's spin limit)
    int hole_r0, hole_rn, hole_w0, hole_wn;   // tiles inside this block of C are skipped
    int band_r0, band_rn, band_w0, band_wn;   // and tiles inside this row band or word band
    const int *run_if;    // device flag: the product is skipped (C untouched) when it reads 0 (may be null)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the phase with the given parity has completed; false after `limit` tries
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];\n"
                 ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar) : "memory");
}
// shared-memory matrix descriptor: K-major tile with 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32"
                 " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15,"
                 " %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Persistent kernel: one CTA per SM walks its tiles (tile t = blockIdx.x + i·gridDim.x in
// grouped order), the accumulator double-buffered in tensor memory so that the epilogue of
// one tile overlaps the loads and MMAs of the next (GB300, 16384 × 16384 × K: 2.57 ms for
// K = 16384 against 2.77 ms with one CTA per tile; eight passes of K = 2048, the Boolean
// closure's phase-3 shape, 2.56 ms against 4.38 ms).  Warp 0 lane 0 streams K slices
// through the shared-memory ring (across tile boundaries), warp 1 lane 0 issues the MMAs
// into accumulator i & 1 for the CTA's i-th tile and commits it to tfull[i & 1], warp 2
// owns the tensor memory (2 × 256 columns), and warps 4-7 (warp w reads accumulator lanes
// 32·(w mod 4) ..) turn counts into bits, write C and release the accumulator through
// tempty[i & 1].  Every wait is bounded; a role that gives up sets the shared failure flag,
// which the others poll while they wait, and the CTA drains what it started.
namespace tc {
constexpr int P_THREADS = 256, EPI_WARP0 = 4;
constexpr int P_TMEM_COLS = 2 * BN;
constexpr size_t P_SMEM = 1024 + (size_t)STAGES * (A_BYTES + B_BYTES) + 256;
}

__device__ __forceinline__ bool mbar_wait_f(uint32_t bar, uint32_t parity, uint32_t limit, const volatile int *failed)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && *failed) return false;
    }
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// tile t of the grid in grouped order (GROUP_M tile rows per group); false for a hole tile
__device__ __forceinline__ bool tc_tile(const BoolTcArgs &p, int t, int &row0, int &ncol0)
{
    const int per_group = tc::GROUP_M * p.tiles_n;
    const int g = t / per_group, first_m = g * tc::GROUP_M;
    const int gm = min(tc::GROUP_M, p.tiles_m - first_m);
    const int r = t - g * per_group;
    row0 = (first_m + r % gm) * tc::BM;
    ncol0 = (r / gm) * tc::BN;
    if (p.hole_rn > 0 || p.band_rn > 0 || p.band_wn > 0) {
        const int w0 = ncol0 >> 5, r1 = min(row0 + tc::BM, p.R), w1 = min(w0 + tc::BN / 32, p.ncw);
        if (p.hole_rn > 0 && row0 >= p.hole_r0 && r1 <= p.hole_r0 + p.hole_rn && w0 >= p.hole_w0 &&
            w1 <= p.hole_w0 + p.hole_wn)
            return false;
        if (p.band_rn > 0 && row0 >= p.band_r0 && r1 <= p.band_r0 + p.band_rn)
            return false;
        if (p.band_wn > 0 && w0 >= p.band_w0 && w1 <= p.band_w0 + p.band_wn)
            return false;
    }
    return true;
}

__global__ void __launch_bounds__(tc::P_THREADS, 1)
bool_tc_persistent_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, BoolTcArgs p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;                                              // [STAGES][BM][BK]
    uint8_t *sB = smem + tc::STAGES * tc::A_BYTES;                   // [STAGES][BN][BK]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + tc::STAGES * tc::B_BYTES);
    // full[S], empty[S], tfull[2], tempty[2], done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * tc::STAGES + 5);
    __shared__ int failed;
    __shared__ uint32_t loads_per_stage[tc::STAGES];

    if (p.run_if && *p.run_if == 0)     // the whole CTA leaves before it touches a barrier or tensor memory
        return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles = p.tiles_m * p.tiles_n;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + tc::STAGES);
    const uint32_t tfull0 = smem_u32(bars + 2 * tc::STAGES), tempty0 = smem_u32(bars + 2 * tc::STAGES + 2);
    const uint32_t done = smem_u32(bars + 2 * tc::STAGES + 4);
    const volatile int *vfailed = &failed;

    if (tid == 0) {
        failed = 0;
        for (int s = 0; s < tc::STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
            loads_per_stage[s] = 0;
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull0 + 8 * a, 1);
            mbar_init(tempty0 + 8 * a, 4);                      // one arrival per epilogue warp
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tmem_slot)), "r"(tc::P_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = (1u << 4) | ((uint32_t)(tc::BN >> 3) << 17) | ((uint32_t)(tc::BM >> 4) << 24);

    if (warp == 0 && lane == 0) {                               // TMA producer
        uint32_t g = 0;
        for (int t = blockIdx.x; t < tiles && !*vfailed; t += gridDim.x) {
            int row0, ncol0;
            if (!tc_tile(p, t, row0, ncol0)) continue;
            for (int kb = 0; kb < p.nkb; ++kb, ++g) {
                const int s = (int)(g % tc::STAGES);
                if (g >= (uint32_t)tc::STAGES &&
                    !mbar_wait_f(empty0 + 8 * s, ((g / tc::STAGES) - 1) & 1, p.wait_limit, vfailed)) {
                    atomicExch(&failed, 1);
                    break;
                }
                mbar_expect_tx(full0 + 8 * s, tc::A_BYTES + tc::B_BYTES);
                tma_load_2d(smem_u32(sA + s * tc::A_BYTES), &tA, kb * tc::BK, row0, full0 + 8 * s);
                tma_load_2d(smem_u32(sB + s * tc::B_BYTES), &tB, kb * tc::BK, ncol0, full0 + 8 * s);
                ++loads_per_stage[s];
            }
        }
    } else if (warp == 1 && lane == 0) {                        // MMA issuer
        uint32_t g = 0, i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            int row0, ncol0;
            if (!tc_tile(p, t, row0, ncol0)) continue;
            const uint32_t a = i & 1, u = i >> 1;
            if (u >= 1 && !mbar_wait_f(tempty0 + 8 * a, (u - 1) & 1, p.wait_limit, vfailed)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t acc = tmem + a * tc::BN;
            for (int kb = 0; kb < p.nkb; ++kb, ++g) {
                const int s = (int)(g % tc::STAGES);
                if (!mbar_wait_f(full0 + 8 * s, (g / tc::STAGES) & 1, p.wait_limit, vfailed)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = smem_u32(sA + s * tc::A_BYTES), b0 = smem_u32(sB + s * tc::B_BYTES);
#pragma unroll
                for (int k4 = 0; k4 < tc::BK / 32; ++k4)
                    umma_f8(acc, smem_desc(a0 + 32 * k4), smem_desc(b0 + 32 * k4), idesc, (kb | k4) != 0);
                umma_commit(empty0 + 8 * s);
            }
            if (!ok) break;
            umma_commit(tfull0 + 8 * a);
            ++i;
        }
        if (!ok) atomicExch(&failed, 1);
        umma_commit(done);                       // arrives once every MMA issued above has completed
    } else if (warp >= tc::EPI_WARP0) {                         // epilogue
        const int q = warp & 3;                                 // accumulator lanes 32q .. 32q + 31
        uint32_t i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
            int row0, ncol0;
            if (!tc_tile(p, t, row0, ncol0)) continue;
            const uint32_t a = i & 1, u = i >> 1;
            int ok = 0;
            if (lane == 0) ok = mbar_wait_f(tfull0 + 8 * a, u & 1, p.wait_limit, vfailed) ? 1 : 0;
            ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
            if (!ok) {
                if (lane == 0) atomicExch(&failed, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int r = row0 + 32 * q + lane;
#pragma unroll 1
            for (int c = 0; c < tc::BN / 32; ++c) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + a * tc::BN + (uint32_t)(32 * c), v);
                uint32_t word = 0u;
#pragma unroll
                for (int j = 0; j < 32; ++j) word |= (v[j] != 0u ? 1u : 0u) << j;
                const int w = (ncol0 >> 5) + c;
                if (r < p.R && w < p.ncw) {
                    const int lo = w * 32;
                    const uint32_t mask = lo + 32 <= p.N ? 0xFFFFFFFFu : (lo >= p.N ? 0u : (1u << (p.N - lo)) - 1u);
                    uint32_t *dst = p.C + (int64_t)r * p.ldc + w;
                    *dst = ((p.accumulate ? *dst : 0u) | word) & mask;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * a);
            ++i;
        }
    }
    __syncwarp();
    __syncthreads();
    // drain: every TMA copy this CTA started must land before its shared memory is released,
    // and every MMA it issued must finish before its tensor memory is freed
    if (warp == 0 && lane == 0 && failed) {
        for (int s = 0; s < tc::STAGES; ++s)
            if (loads_per_stage[s] > 0) mbar_wait(full0 + 8 * s, (loads_per_stage[s] - 1) & 1, tc::DRAIN_LIMIT);
    }
    if (warp == 1 && lane == 0) mbar_wait(done, 0, tc::DRAIN_LIMIT);
    if (tid == 0 && failed && p.status) atomicExch(p.status, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 2)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tc::P_TMEM_COLS)
                     : "memory");
}

// 32 bits -> 32 e4m3 bytes (1.0 = 0x38, 0 = 0x00), written as two 16-byte stores
__device__ __forceinline__ void expand_word(uint32_t bits, uint8_t *dst)
{
    uint32_t o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        // bit j of the nibble to bit 8j (the multiply's four copies shifted by 0, 7, 14, 21
        // put bit j at 8j, and the mask drops the rest), then each 0x01 byte to e4m3 1.0
        const uint32_t nib = (bits >> (4 * q)) & 0xFu;
        o[q] = ((nib * 0x00204081u) & 0x01010101u) * 0x38u;
    }
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = make_uint4(o[0], o[1], o[2], o[3]);
    d[1] = make_uint4(o[4], o[5], o[6], o[7]);
}

// rows x Kp bytes of A, K-major: item t (one thread) expands word w of row r; zero past K
__device__ __forceinline__ void expand_rows_items(const uint32_t *M, int64_t ldm, int rows, int K, uint8_t *out, int Kp,
                                                  int64_t t0, int64_t stride)
{
    const int64_t total = (int64_t)rows * (Kp / 32);
    for (int64_t t = t0; t < total; t += stride) {
        const int r = (int)(t / (Kp / 32)), w = (int)(t % (Kp / 32));
        const int lo = 32 * w;
        uint32_t bits = lo < K ? M[(int64_t)r * ldm + w] : 0u;
        if (lo + 32 > K) bits &= lo >= K ? 0u : (1u << (K - lo)) - 1u;
        expand_word(bits, out + (int64_t)r * Kp + lo);
    }
}

// 32 x 32 bit transpose across a warp: lane i holds row i (bit j = column j) and gets
// column i (bit j = row j).  Five stages swap the off-diagonal halves of ever smaller
// blocks (16, 8, 4, 2, 1 bits) with the lane s apart, masks selecting the half kept.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane)
{
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int s = 16 >> st;
        const uint32_t m = st == 0 ? 0x0000FFFFu : st == 1 ? 0x00FF00FFu : st == 2 ? 0x0F0F0F0Fu
                         : st == 3 ? 0x33333333u : 0x55555555u;
        const uint32_t p = __shfl_xor_sync(0xFFFFFFFFu, x, s);
        x = (lane & s) ? (x & ~m) | ((p >> s) & m) : (x & m) | ((p & m) << s);
    }
    return x;
}

// transpose + expand: out[n][k] = bit (k, n) of M (K rows of bits), rows n < N, zero past K;
// item t (one warp) transposes the 32 x 32 bits of word w of rows 32kb .. 32kb + 31
__device__ __forceinline__ void expand_cols_items(const uint32_t *M, int64_t ldm, int K, int N, uint8_t *out, int Kp,
                                                  int64_t t0, int64_t stride)
{
    const int lane = threadIdx.x & 31;
    const int nwords = (N + 31) / 32, kblocks = Kp / 32;
    const int64_t total = (int64_t)nwords * kblocks;
    for (int64_t t = t0; t < total; t += stride) {
        const int w = (int)(t / kblocks), kb = (int)(t % kblocks);
        const int k = 32 * kb + lane;
        const uint32_t word = k < K ? M[(int64_t)k * ldm + w] : 0u;   // row k, columns 32w .. 32w+31
        const uint32_t mine = warp_transpose32(word, lane);           // column 32w + lane, rows 32kb..+31
        const int n = 32 * w + lane;
        if (n < N) expand_word(mine, out + (int64_t)n * Kp + 32 * kb);
    }
}

__global__ void expand_rows_kernel(const uint32_t *M, int64_t ldm, int rows, int K, uint8_t *out, int Kp,
                                   const int *run_if)
{
    if (run_if && *run_if == 0) return;
    expand_rows_items(M, ldm, rows, K, out, Kp, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                      (int64_t)gridDim.x * blockDim.x);
}

__global__ void expand_cols_kernel(const uint32_t *M, int64_t ldm, int K, int N, uint8_t *out, int Kp,
                                   const int *run_if)
{
    if (run_if && *run_if == 0) return;
    expand_cols_items(M, ldm, K, N, out, Kp, blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32,
                      (int64_t)gridDim.x * (blockDim.x / 32));
}

// One launch before squaring `it` of the repeated-squaring closure (M is D x D bits, rw
// words a row, row stride ld; M2 holds the previous power): flag[it % 3] := M != M2 (did
// squaring it - 1 change the power?  it = 0: yes); clears flag[(it + 1) % 3] for the next
// launch; and expands M into both operand layouts of M ⊗ M (A rows, B^T rows).  Once a
// squaring left the power unchanged (flag[(it - 1) % 3] = 0) the flag stays 0 and nothing
// is expanded: the later products are skipped.  Blocks [0, nb_cmp) compare, the next
// nb_rows expand rows, the rest transpose-expand.
__global__ void square_prep_kernel(const uint32_t *M, const uint32_t *M2, int64_t ld, int D, int rw, uint8_t *Ae,
                                   uint8_t *Be, int Kp, int *flags, int it, int nb_cmp, int nb_rows)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[(it + 1) % 3] = 0;
    if (it >= 2 && flags[(it + 2) % 3] == 0) return;          // flag[(it - 1) % 3]: already converged
    const int b = blockIdx.x;
    if (b < nb_cmp) {
        if (it == 0) {
            if (b == 0 && threadIdx.x == 0) flags[0] = 1;
            return;
        }
        const int64_t total = (int64_t)D * rw;
        bool diff = false;
        for (int64_t t = b * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)nb_cmp * blockDim.x) {
            const int64_t off = (t / rw) * ld + t % rw;
            diff |= M[off] != M2[off];
        }
        if (__any_sync(0xFFFFFFFFu, diff) && (threadIdx.x & 31) == 0) flags[it % 3] = 1;
    } else if (b < nb_cmp + nb_rows) {
        expand_rows_items(M, ld, D, D, Ae, Kp, (b - nb_cmp) * (int64_t)blockDim.x + threadIdx.x,
                          (int64_t)nb_rows * blockDim.x);
    } else {
        const int nbc = gridDim.x - nb_cmp - nb_rows;
        expand_cols_items(M, ld, D, D, Be, Kp, (b - nb_cmp - nb_rows) * (int64_t)(blockDim.x / 32) + threadIdx.x / 32,
                          (int64_t)nbc * (blockDim.x / 32));
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
    });
    return fn;
}

static bool make_map(CUtensorMap *m, void *base, int rows, int Kp, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp};
    const cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t bool_tc_workspace(int64_t R, int64_t K, int64_t N)
{
    const int64_t Kp = (K + tc::BK - 1) / tc::BK * tc::BK;
    return (size_t)((R + N) * Kp) + 1024;
}

// Tensor-pipe probe (the roofline denominator of the fp8 count path): one CTA per SM,
// lane 0 of warp 1 issues `iters` MMAs (kind::f8f6f4, M = 128, N = 256, K = 32, e4m3
// operands, f32 accumulation — the product kernel's instruction) from shared memory
// holding 0/1 operands into one tensor-memory accumulator, then commits them to an mbarrier; the
// CTA frees its tensor memory once they are done.  (The integer MMA, kind::i8, does not
// exist for sm_103a: ptxas rejects it for that target.)
__global__ void __launch_bounds__(128, 1) tc_peak_f8_kernel(int iters, int *failed)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    // operands like the count path's: e4m3 bytes 1.0 (0x38) or 0, about half of each
    uint32_t *z = reinterpret_cast<uint32_t *>(smem);
    for (int i = tid; i < (tc::A_BYTES + tc::B_BYTES) / 4; i += blockDim.x) {
        const uint32_t h = (uint32_t)i * 0x9E3779B9u;
        z[i] = ((h >> 7) & 0x01010101u) * 0x38u;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");     // the MMAs read through the async proxy
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(&tmem_slot)), "r"(tc::BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    if (tid == 32) {
        const uint32_t idesc = (1u << 4) | ((uint32_t)(tc::BN >> 3) << 17) | ((uint32_t)(tc::BM >> 4) << 24);
        const uint64_t ad = smem_desc(smem_u32(smem)), bd = smem_desc(smem_u32(smem + tc::A_BYTES));
        for (int i = 0; i < iters; ++i) umma_f8(tmem, ad, bd, idesc, i > 0 ? 1u : 0u);
        umma_commit(smem_u32(&bar));
        // the MMAs are finite: this wait ends when they do (its bound only guards a fault)
        if (!mbar_wait(smem_u32(&bar), 0, tc::DRAIN_LIMIT)) atomicExch(failed, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(tc::BN) : "memory");
}

sr_status peak_tc_f8(int iters, cudaStream_t s, double *ms, double *mma_per_s, double *flops)
{
    if (!bool_tc_available())
        return fail(SR_EINVAL, "sr_peak_probe: no tcgen05 tensor cores on this device");
    constexpr size_t SMEM = 1024 + (size_t)tc::A_BYTES + tc::B_BYTES;
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(tc_peak_f8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
        attr[dev] = true;
    }
    const int blocks = device_sm_count();
    int *failed = nullptr;
    SR_CUDA_CHECK(cudaMallocAsync(&failed, sizeof(int), s));
    SR_CUDA_CHECK(cudaMemsetAsync(failed, 0, sizeof(int), s));
    cudaEvent_t e0, e1;
    SR_CUDA_CHECK(cudaEventCreate(&e0));
    SR_CUDA_CHECK(cudaEventCreate(&e1));
    tc_peak_f8_kernel<<<blocks, 128, SMEM, s>>>(std::max(1, iters / 8), failed);     // warm-up
    SR_CUDA_CHECK(cudaEventRecord(e0, s));
    tc_peak_f8_kernel<<<blocks, 128, SMEM, s>>>(iters, failed);
    SR_CUDA_CHECK(cudaEventRecord(e1, s));
    count_launches(2);
    SR_CUDA_CHECK(cudaGetLastError());
    SR_CUDA_CHECK(cudaEventSynchronize(e1));
    float t = 0.f;
    int hf = 0;
    SR_CUDA_CHECK(cudaEventElapsedTime(&t, e0, e1));
    SR_CUDA_CHECK(cudaMemcpyAsync(&hf, failed, sizeof(int), cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(failed, s);
    SR_CUDA_CHECK(cudaStreamSynchronize(s));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (hf)
        return fail(SR_ETIMEOUT, "sr_peak_probe: the tensor-core probe's completion wait gave up");
    const double mmas = (double)iters * blocks;
    *ms = t;
    *mma_per_s = mmas / (t * 1e-3);
    *flops = *mma_per_s * 2.0 * tc::BM * tc::BN * 32;
    return SR_OK;
}

bool bool_tc_available()
{
    int dev = current_device(), major = 0;
    if (dev < 0) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    return major == 10 && encode_fn() != nullptr;
}

sr_status launch_bool_mul_tc(const BoolArgs &a, void *ws, size_t ws_bytes, int *status, int spin_limit,
                             cudaStream_t s, int max_ctas, const int *run_if)
{
    const int Kp = (a.K + tc::BK - 1) / tc::BK * tc::BK;
    if (bool_tc_workspace(a.R, a.K, a.N) > ws_bytes)
        return fail(SR_ENOMEM, "bool_mul (tensor path): workspace too small");
    if (a.skipw != 0 || a.skipww != 0)
        return fail(SR_EINVAL, "bool_mul (tensor path): excluded row or word ranges are not supported");
    if (a.hole_rn > 0) {
        const bool rows_ok = a.hole_r0 % tc::BM == 0 && ((a.hole_r0 + a.hole_rn) % tc::BM == 0 ||
                                                         a.hole_r0 + a.hole_rn >= a.R);
        const bool words_ok = a.hole_w0 % (tc::BN / 32) == 0 &&
                              ((a.hole_w0 + a.hole_wn) % (tc::BN / 32) == 0 || a.hole_w0 + a.hole_wn >= a.ncw);
        if (!rows_ok || !words_ok || a.hole_r0 < 0 || a.hole_w0 < 0 || a.hole_wn <= 0)
            return fail(SR_EINVAL, "bool_mul (tensor path): the untouched block must lie on the 128 x 256 tile grid");
    }
    if (a.band_rn < 0 || a.band_wn < 0 ||
        (a.band_rn > 0 && (a.band_r0 < 0 || a.band_r0 % tc::BM != 0 ||
                           ((a.band_r0 + a.band_rn) % tc::BM != 0 && a.band_r0 + a.band_rn < a.R))) ||
        (a.band_wn > 0 && (a.band_w0 < 0 || a.band_w0 % (tc::BN / 32) != 0 ||
                           ((a.band_w0 + a.band_wn) % (tc::BN / 32) != 0 && a.band_w0 + a.band_wn < a.ncw))))
        return fail(SR_EINVAL, "bool_mul (tensor path): the untouched bands must lie on the 128 x 256 tile grid");
    uint8_t *Ae = static_cast<uint8_t *>(ws);
    uint8_t *Be = tc_operand_b(Ae, a.R, Kp);
    const int sms = device_sm_count();
    {
        const int64_t n = (int64_t)a.R * (Kp / 32);
        expand_rows_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sms * 16)), 256, 0, s>>>(
            a.A, a.lda, a.R, a.K, Ae, Kp, run_if);
        SR_CUDA_CHECK(cudaGetLastError());
        const int64_t nw = (int64_t)((a.N + 31) / 32) * (Kp / 32);
        expand_cols_kernel<<<(int)std::max<int64_t>(1, std::min<int64_t>((nw + 7) / 8, sms * 16)), 256, 0, s>>>(
            a.B, a.ldb, a.K, a.N, Be, Kp, run_if);
        SR_CUDA_CHECK(cudaGetLastError());
        count_launches(2);
    }
    return launch_bool_mul_tc_expanded(a, Ae, Be, status, spin_limit, s, max_ctas, run_if);
}

uint8_t *tc_operand_b(uint8_t *Ae, int64_t R, int Kp)
{
    uint8_t *Be = Ae + R * Kp;
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(Be) + 255) & ~uintptr_t(255));
}

sr_status launch_square_prep(const uint32_t *M, const uint32_t *M2, int64_t ld, int D, int rw, void *ws, int *flags,
                             int it, cudaStream_t s, int grid_sms)
{
    const int Kp = (D + tc::BK - 1) / tc::BK * tc::BK;
    uint8_t *Ae = static_cast<uint8_t *>(ws);
    uint8_t *Be = tc_operand_b(Ae, D, Kp);
    // its loops stride over the grid, so any grid size gives the same result
    const int sms = grid_sms > 0 ? std::min(grid_sms, device_sm_count()) : device_sm_count();
    const int64_t ncmp = (int64_t)D * rw, nrows = (int64_t)D * (Kp / 32), ncols = (int64_t)((D + 31) / 32) * (Kp / 32);
    const int nb_cmp = (int)std::max<int64_t>(1, std::min<int64_t>((ncmp + 255) / 256, sms * 4));
    const int nb_rows = (int)std::max<int64_t>(1, std::min<int64_t>((nrows + 255) / 256, sms * 8));
    const int nb_cols = (int)std::max<int64_t>(1, std::min<int64_t>((ncols + 7) / 8, sms * 8));
    square_prep_kernel<<<nb_cmp + nb_rows + nb_cols, 256, 0, s>>>(M, M2, ld, D, rw, Ae, Be, Kp, flags, it, nb_cmp,
                                                                  nb_rows);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

sr_status launch_bool_mul_tc_expanded(const BoolArgs &a, uint8_t *Ae, uint8_t *Be, int *status, int spin_limit,
                                      cudaStream_t s, int max_ctas, const int *run_if)
{
    const int Kp = (a.K + tc::BK - 1) / tc::BK * tc::BK;
    const int sms = device_sm_count();
    CUtensorMap mA, mB;
    if (!make_map(&mA, Ae, a.R, Kp, tc::BM) || !make_map(&mB, Be, a.N, Kp, tc::BN))
        return fail(SR_ECUDA, "bool_mul (tensor path): cannot encode the tensor maps");
    static bool attr[kMaxDevices] = {};
    SR_DEVICE_SLOT(dev);
    if (!attr[dev]) {
        SR_CUDA_CHECK(cudaFuncSetAttribute(bool_tc_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tc::P_SMEM));
        attr[dev] = true;
    }
    BoolTcArgs p;
    p.C = a.C;
    p.ldc = a.ldc;
    p.R = a.R;
    p.N = a.N;
    p.ncw = a.ncw;
    p.nkb = Kp / tc::BK;
    p.accumulate = a.accumulate;
    p.status = status;
    p.wait_limit = (uint32_t)std::max(0, spin_limit);
    p.hole_r0 = a.hole_r0; p.hole_rn = a.hole_rn; p.hole_w0 = a.hole_w0; p.hole_wn = a.hole_wn;
    p.band_r0 = a.band_r0; p.band_rn = a.band_rn; p.band_w0 = a.band_w0; p.band_wn = a.band_wn;
    p.run_if = run_if;
    p.tiles_n = (a.ncw + tc::BN / 32 - 1) / (tc::BN / 32);
    p.tiles_m = (a.R + tc::BM - 1) / tc::BM;
    const int64_t tiles = (int64_t)p.tiles_m * p.tiles_n;
    if (tiles > 0x7fffffffLL)
        return fail(SR_EINVAL, "bool_mul (tensor path): too many tiles");
    const int64_t grid = std::min<int64_t>(tiles, max_ctas > 0 ? std::min(max_ctas, sms) : sms);
    bool_tc_persistent_kernel<<<(unsigned)grid, tc::P_THREADS, tc::P_SMEM, s>>>(mA, mB, p);
    SR_CUDA_CHECK(cudaGetLastError());
    count_launches();
    return SR_OK;
}

}  // namespace sr
