// Closure schedules for the anti-distance semirings (u8, u16, u32): the three-phase
// blocked form of Warshall's loop (Section 2) and its Floyd generalisation (Section 3),
//   T := A;  for k = 1..D:  T := T ⊕ (T_col k ⊗ T_row k),
// run block by block.  For each k-block of width W:
//   phase 1: T_kk := closure of the diagonal block;
//   phase 2: T_kj := T_kj ⊕ T_kk ⊗ T_kj,  T_ik := T_ik ⊕ T_ik ⊗ T_kk (panels);
//   phase 3: T_ij := T_ij ⊕ T_ik ⊗ T_kj for all other blocks (the product kernel with
//            K = W, panel rows/columns excluded).
// Every pivot order gives the same fixed point, and rows/columns of the pivot block do
// not change in their own step, so the blocked order is exact.
//
// Phase 1 of a 128-wide block runs on one CTA (antidist_pivot_kernel).  A wider block
// (W = 256 or 512: fewer, deeper phase-3 passes) is closed by the same three phases at
// width 128 inside it, on one stream.  Phases 2 and 3 are launches of the product
// kernel.  The look-ahead schedule overlaps the next block's phases 1-2 with the
// current phase 3 on three high-priority side streams.

#include <algorithm>
#include <mutex>
#include <vector>

#include "sr_common.cuh"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {

// Side streams (0..2 high priority, kPeerStream the lowest, as the caller's default
// stream) and a per-thread pool of events for the look-ahead.
cudaStream_t side_stream(int i)
{
    static cudaStream_t st[kMaxDevices][kSideStreams] = {};
    static std::mutex mu;
    const int dev = current_device();
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || i < 0 || i >= kSideStreams)
        return nullptr;
    if (!st[dev][i]) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&st[dev][i], cudaStreamNonBlocking, i == kPeerStream ? lo : hi) != cudaSuccess)
            st[dev][i] = nullptr;
    }
    return st[dev][i];
}

sr_status event_pool(size_t n, std::vector<cudaEvent_t> *&out)
{
    static thread_local std::vector<cudaEvent_t> pool[kMaxDevices];
    SR_DEVICE_SLOT(dev);
    std::vector<cudaEvent_t> &p = pool[dev];
    while (p.size() < n) {
        cudaEvent_t e;
        SR_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p.push_back(e);
    }
    out = &p;
    return SR_OK;
}

namespace {

constexpr int PB = 128;               // pivot-kernel block
constexpr int NONE = 0x7fffffff;      // no excluded range

template <class E>
E *at(void *T, int64_t ldt, int r, int c) { return static_cast<E *>(T) + (int64_t)r * ldt + c; }

// Phase 3 of the k-block [k0, k0+bw) restricted to rows [rbeg, rbeg+R) and columns
// [cbeg, cbeg+N) of the matrix (logical indices), each with one excluded range.
template <class E>
sr_status phase3(void *T, int64_t ldt, int k0, int bw, int rbeg, int R, int rskip0, int rskipw, int cbeg, int N,
                 int cskip0, int cskipw, sr_dtype dt, bool vec, cudaStream_t s, int tiles, int skip_tile = -1)
{
    MulArgs a;
    a.A = at<E>(T, ldt, rbeg, k0);                 // column panel: rows from rbeg, columns of block k
    a.B = at<E>(T, ldt, k0, cbeg);                 // row panel: rows of block k, columns from cbeg
    a.C = at<E>(T, ldt, rbeg, cbeg);
    a.lda = a.ldb = a.ldc = ldt;
    a.R = R;
    a.N = N;
    a.K = bw;
    a.accumulate = 1;
    a.rskip0 = rskip0; a.rskipw = rskipw;
    a.cskip0 = cskip0; a.cskipw = cskipw;
    a.skip_tile = skip_tile;
    return launch_antidist_mul(a, dt, vec, s, tiles);
}

// Phase 2 of the k-block [k0, k0+bw) as an in-place product on many CTAs:
//   row panel    T_kj := T_kj ⊕ T_kk ⊗ T_kj   (B and C are the same panel)
//   column panel T_ik := T_ik ⊕ T_ik ⊗ T_kk   (A and C are the same panel)
// with T_kk already closed.  A CTA may read panel entries another CTA has already
// updated; that is harmless: for any T_kj <= X <= T_kj ⊕ T_kk ⊗ T_kj entrywise,
// T_kj ⊕ T_kk ⊗ X = T_kj ⊕ T_kk ⊗ T_kj, because T_kk ⊗ T_kk <= T_kk (closed) and
// ⊗ distributes over ⊕ and is monotone.  Each entry read is either its old or its
// new value (8/16/32-bit entries are never torn).
template <class E>
sr_status phase2(void *T, int64_t ldt, int D, int k0, int bw, bool row, sr_dtype dt, bool vec, cudaStream_t s,
                 int tiles = 1)
{
    if (D - bw <= 0)
        return SR_OK;
    MulArgs a;
    a.lda = a.ldb = a.ldc = ldt;
    a.K = bw;
    a.accumulate = 1;
    a.skip_tile = -1;
    if (row) {      // rows of block k, all columns but block k
        a.A = at<E>(T, ldt, k0, k0);
        a.B = a.C = at<E>(T, ldt, k0, 0);
        a.R = bw; a.N = D - bw;
        a.rskip0 = NONE; a.rskipw = 0;
        a.cskip0 = k0; a.cskipw = bw;
    } else {        // all rows but block k, columns of block k
        a.A = a.C = at<E>(T, ldt, 0, k0);
        a.B = at<E>(T, ldt, k0, k0);
        a.R = D - bw; a.N = bw;
        a.rskip0 = k0; a.rskipw = bw;
        a.cskip0 = NONE; a.cskipw = 0;
    }
    return launch_antidist_mul(a, dt, vec, s, tiles);
}

// Whole closure of a D×D matrix on one stream, 128-wide blocks: per block kb its two
// panels, then block (kb+1, kb+1)'s update from kb fused with its closure (one CTA),
// then phase 3 of kb over every other block.  Used for the diagonal blocks of a wider
// blocking (D <= 512) and when no side stream exists.
template <class E>
sr_status closure_one_stream(void *T, int64_t ldt, int D, bool vec, sr_dtype dt, cudaStream_t s)
{
    const int nb = (D + PB - 1) / PB;
    SR_TRY(launch_antidist_pivot(T, ldt, D, 0, -1, dt, vec, s));
    for (int kb = 0; kb < nb; ++kb) {
        SR_TRACE_BLOCK("antidist_closure.block", kb);
        const int k0 = kb * PB, bw = std::min(PB, D - k0);
        SR_TRY(phase2<E>(T, ldt, D, k0, bw, true, dt, vec, s));
        SR_TRY(phase2<E>(T, ldt, D, k0, bw, false, dt, vec, s));
        const bool next = kb + 1 < nb;
        if (next)
            SR_TRY(launch_antidist_pivot(T, ldt, D, kb + 1, kb, dt, vec, s));
        // every block outside block row and column kb, except the diagonal block kb+1
        // (logical 128×128 tile (kb, kb) once row and column kb are removed)
        const int tiles_n = (D - bw + PB - 1) / PB;
        if (!next || tiles_n > 1)
            SR_TRY(phase3<E>(T, ldt, k0, bw, 0, D - bw, k0, bw, 0, D - bw, k0, bw, dt, vec, s, 1,
                             next ? kb * tiles_n + kb : -1));
    }
    return SR_OK;
}

// Phase 1 of the W-wide block (k1, k1) of the whole matrix on stream s: its update from
// the previous block [k0, k0+bw) (k0 < 0: none), then its closure.
template <class E>
sr_status close_diagonal(void *T, int64_t ldt, int D, int W, int k1, int bwn, int k0, int bw, bool vec,
                         sr_dtype dt, cudaStream_t s)
{
    if (W == PB)       // the pivot kernel fuses the update
        return launch_antidist_pivot(T, ldt, D, k1 / PB, k0 < 0 ? -1 : k0 / PB, dt, vec, s);
    if (k0 >= 0)
        SR_TRY(phase3<E>(T, ldt, k0, bw, k1, bwn, NONE, 0, k1, bwn, NONE, 0, dt, vec, s, 1));
    return closure_one_stream<E>(at<E>(T, ldt, k1, k1), ldt, bwn, vec, dt, s);
}

// Two-stream schedule (128-wide blocks): per block kb, the two panels of kb side by
// side (row panel on the main stream, column panel on the side stream), then phase 3
// of kb on the main stream over every block outside block row and column kb except
// the diagonal block kb+1, while one CTA on the side stream gives that block its
// update from kb and closes it (phase 1 of kb+1).
template <class E>
sr_status closure_two_streams(void *T, int64_t ldt, int D, bool vec, sr_dtype dt, cudaStream_t s, cudaStream_t s2)
{
    const int nb = (D + PB - 1) / PB;
    std::vector<cudaEvent_t> *ev = nullptr;
    SR_TRY(event_pool(4 * (size_t)nb + 4, ev));
    SR_TRY(launch_antidist_pivot(T, ldt, D, 0, -1, dt, vec, s));
    for (int kb = 0; kb < nb; ++kb) {
        SR_TRACE_BLOCK("antidist_closure.block", kb);
        const int k0 = kb * PB, bw = std::min(PB, D - k0);
        const bool next = kb + 1 < nb;
        cudaEvent_t *e = ev->data() + 4 * kb;
        SR_CUDA_CHECK(cudaEventRecord(e[0], s));                 // pivot kb closed (main order)
        SR_CUDA_CHECK(cudaStreamWaitEvent(s2, e[0], 0));
        SR_TRY(phase2<E>(T, ldt, D, k0, bw, false, dt, vec, s2));
        SR_CUDA_CHECK(cudaEventRecord(e[1], s2));
        SR_TRY(phase2<E>(T, ldt, D, k0, bw, true, dt, vec, s));
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, e[1], 0));          // both panels done
        if (!next) {
            SR_TRY(phase3<E>(T, ldt, k0, bw, 0, D - bw, k0, bw, 0, D - bw, k0, bw, dt, vec, s, 0));
            break;
        }
        SR_CUDA_CHECK(cudaEventRecord(e[2], s));
        SR_CUDA_CHECK(cudaStreamWaitEvent(s2, e[2], 0));
        SR_TRY(launch_antidist_pivot(T, ldt, D, kb + 1, kb, dt, vec, s2));
        SR_CUDA_CHECK(cudaEventRecord(e[3], s2));
        const int tiles_n = (D - bw + PB - 1) / PB;
        SR_TRY(phase3<E>(T, ldt, k0, bw, 0, D - bw, k0, bw, 0, D - bw, k0, bw, dt, vec, s, 0, kb * tiles_n + kb));
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, e[3], 0));
    }
    return SR_OK;
}

// Pipelined three-phase blocked closure with a one-block look-ahead, blocks of width
// W (128, 256 or 512).  The main stream runs phase 3 of block kb on every block outside
// block rows and columns kb and kb+1; meanwhile three high-priority side streams
// prepare block kb+1:
//   P: block (kb+1, kb+1): its update from block kb and its closure (phase 1)
//   R: block kb's update of block row kb+1 (outside blocks kb, kb+1), then, once P is
//      done, the row panel of kb+1 (phase 2)
//   C: the same for block column kb+1
// so phases 1 and 2 of the next block run beside phase 3 of this one instead of after
// it.  The writers are disjoint: main writes outside rows/columns kb, kb+1; R writes
// block row kb+1, C block column kb+1, P the diagonal block; every one of them reads
// only panel kb, the diagonal block after P, and its own row or column.  The side work
// for kb+1 starts once main's phase 3 of kb-1 (the last writer of block row and column
// kb+1) and the panels of kb are done; main's phase 3 of kb+1 waits for both panels.
//
// With a peer stream sb, "main" is two streams: phase 3 of every block is split at a
// tile-row boundary, the upper rows on s and the lower rows on sb.  Each half of pass
// kb+1 needs only the same half of pass kb (its own C tiles) and the panels of kb+1, so
// the two streams run their passes independently, and the drain and launch gap at the
// end of one stream's pass are filled by the other stream's CTAs.  The side work waits
// for both halves.  One half's pass kb+1 may update row or column block kb (outside its
// band) while the other half's pass kb still reads that block as its panel.  The read
// sees old or new entries, and either gives the same fixed point: a new entry is the old
// one ⊕ weights of paths through block kb+1, all of which the closure holds, and ⊗ is
// monotone, so every value stays between the blocked loop's and the closure's.
// Two main streams from this much phase-3 work per pass (128×128 tiles × W / 128 × entry
// bytes).  GB300 closure times, one stream -> two: u8 D = 4608 3.83 -> 3.41 ms, 5120
// 4.90 -> 4.54, 5632 6.27 -> 5.65, 6144 7.82 -> 7.30, 8192 (W = 256) 16.51 -> 16.26; u16
// D = 4096 5.00 -> 4.74.  At u8 D = 4096 (900 tiles a pass, 1.97 waves of 456 CTAs: the
// passes' tails are small already) and below, no change or up to 1.5 % slower.
constexpr int64_t kPeerMinWork = 1000;

template <class E>
sr_status closure_look_ahead(void *T, int64_t ldt, int D, int W, bool vec, sr_dtype dt, cudaStream_t s,
                             cudaStream_t sp, cudaStream_t sr_, cudaStream_t sc, cudaStream_t sb)
{
    const int nb = (D + W - 1) / W;
    auto width = [&](int kb) { return std::min(W, D - kb * W); };
    {   // phase-3 work per pass in 128-deep u8 tiles; below kPeerMinWork one stream
        const int64_t tn = (D - 2 * W + PB - 1) / PB;
        if (tn * tn * (W / PB) * (int64_t)sizeof(E) < kPeerMinWork) sb = nullptr;
    }
    // strips and panels of the next block: 64x64 tiles for 128-wide blocks (enough CTAs
    // for a 128-row panel), 128x128 tiles for wider ones (more work per staged byte;
    // GB300, u8 D = 8192, W = 256: 16.4 ms against 17.0 ms with 64x64 tiles)
    const int side_tiles = W > PB ? 0 : 1;
    std::vector<cudaEvent_t> *ev = nullptr;
    SR_TRY(event_pool(5 * (size_t)nb + 6, ev));
    cudaEvent_t *main_done = ev->data();              // [kb]: main's phase 3 of kb (upper rows with sb)
    cudaEvent_t *pivot_done = main_done + nb + 1;     // [kb]: block (kb, kb) closed
    cudaEvent_t *rowp_done = pivot_done + nb + 1;     // [kb]: row panel of kb
    cudaEvent_t *colp_done = rowp_done + nb + 1;      // [kb]: column panel of kb
    cudaEvent_t *low_done = colp_done + nb + 1;       // [kb]: sb's lower rows of phase 3 of kb; [nb]: join
    // phase 3 of block kb over logical rows [r0, r1) of the D - ex rows outside the band
    // [k0, k0 + ex): the upper part keeps the band's exclusion, the lower part starts at
    // its first physical row and excludes the band only if it still lies below
    auto phase3_rows = [&](int k0, int bw, int ex, int r0, int r1, cudaStream_t st) -> sr_status {
        if (r1 <= r0)
            return SR_OK;
        const int p0 = r0 < k0 ? r0 : r0 + ex;                  // physical first row
        const int rs0 = r0 < k0 ? k0 - r0 : NONE, rsw = r0 < k0 ? ex : 0;
        return phase3<E>(T, ldt, k0, bw, p0, r1 - r0, rs0, rsw, 0, D - ex, k0, ex, dt, vec, st, 0);
    };
    auto phase3_main = [&](int k0, int bw, int ex) -> sr_status {
        const int rows = D - ex;
        if (!sb)
            return phase3_rows(k0, bw, ex, 0, rows, s);
        const int split = ((rows + PB - 1) / PB / 2) * PB;      // a tile-row boundary
        SR_TRY(phase3_rows(k0, bw, ex, 0, split, s));
        return phase3_rows(k0, bw, ex, split, rows, sb);
    };
    SR_TRY(close_diagonal<E>(T, ldt, D, W, 0, width(0), -1, 0, vec, dt, s));
    SR_TRY(phase2<E>(T, ldt, D, 0, width(0), true, dt, vec, s));
    SR_TRY(phase2<E>(T, ldt, D, 0, width(0), false, dt, vec, s));
    SR_CUDA_CHECK(cudaEventRecord(rowp_done[0], s));
    SR_CUDA_CHECK(cudaEventRecord(colp_done[0], s));
    for (int kb = 0; kb < nb; ++kb) {
        SR_TRACE_BLOCK("antidist_closure.block", kb);
        const int k0 = kb * W, bw = width(kb);
        const bool next = kb + 1 < nb;
        const int bwn = next ? width(kb + 1) : 0, ex = bw + bwn;     // rows/columns left out
        // s may be the legacy default stream, whose handle is null: only sb's null means absent
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, rowp_done[kb], 0));
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, colp_done[kb], 0));
        if (sb) {                             // kb = 0: sb forks from s here
            SR_CUDA_CHECK(cudaStreamWaitEvent(sb, rowp_done[kb], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(sb, colp_done[kb], 0));
        }
        SR_TRY(phase3_main(k0, bw, ex));
        if (!next)
            break;
        SR_CUDA_CHECK(cudaEventRecord(main_done[kb], s));
        if (sb) SR_CUDA_CHECK(cudaEventRecord(low_done[kb], sb));
        for (cudaStream_t x : {sp, sr_, sc}) {
            if (kb > 0) SR_CUDA_CHECK(cudaStreamWaitEvent(x, main_done[kb - 1], 0));
            if (kb > 0 && sb) SR_CUDA_CHECK(cudaStreamWaitEvent(x, low_done[kb - 1], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(x, rowp_done[kb], 0));
            SR_CUDA_CHECK(cudaStreamWaitEvent(x, colp_done[kb], 0));
        }
        const int k1 = k0 + bw;
        SR_TRY(close_diagonal<E>(T, ldt, D, W, k1, bwn, k0, bw, vec, dt, sp));
        SR_CUDA_CHECK(cudaEventRecord(pivot_done[kb + 1], sp));
        SR_TRY(phase3<E>(T, ldt, k0, bw, k1, bwn, NONE, 0, 0, D - ex, k0, ex, dt, vec, sr_, side_tiles));
        SR_CUDA_CHECK(cudaStreamWaitEvent(sr_, pivot_done[kb + 1], 0));
        SR_TRY(phase2<E>(T, ldt, D, k1, bwn, true, dt, vec, sr_, side_tiles));
        SR_CUDA_CHECK(cudaEventRecord(rowp_done[kb + 1], sr_));
        SR_TRY(phase3<E>(T, ldt, k0, bw, 0, D - ex, k0, ex, k1, bwn, NONE, 0, dt, vec, sc, side_tiles));
        SR_CUDA_CHECK(cudaStreamWaitEvent(sc, pivot_done[kb + 1], 0));
        SR_TRY(phase2<E>(T, ldt, D, k1, bwn, false, dt, vec, sc, side_tiles));
        SR_CUDA_CHECK(cudaEventRecord(colp_done[kb + 1], sc));
    }
    if (sb) {                                 // join: s waits for sb's last pass
        SR_CUDA_CHECK(cudaEventRecord(low_done[nb], sb));
        SR_CUDA_CHECK(cudaStreamWaitEvent(s, low_done[nb], 0));
    }
    return SR_OK;
}

// Fewer 128-wide blocks than this take the plain two-stream schedule: with little
// phase-3 work per block, the look-ahead's extra launches and events cost more than
// the panels they hide (GB300: two streams 3% faster at D = 3072, the look-ahead 6%
// faster at D = 4096).
constexpr int kLookAheadMinBlocks = 28;

// Block width: wider blocks halve (W = 256) or quarter (W = 512) the phase-3 passes,
// whose launch, staging and tail cost is paid once per pass (GB300, u8, the product
// kernel alone over D = 8192 with K = 128 / 256 / 512 per pass: 17.5 / 16.2 / 15.6 ms),
// but each diagonal block then takes a chain of eight or more launches on the pivot
// stream, which the next phase 3 waits for.  That chain hides behind phase 3 only when
// phase 3 is long (GB300 closure times, u8: D = 4096 2.60 / 3.49 ms at W = 128 / 256,
// D = 6144 7.74 / 7.98, D = 7168 12.2 / 11.7, D = 8192 18.0 / 16.4, D = 10240 at
// W = 128 / 256 / 512 34.6 / 32.0 / 31.0; u16 and u32 at D = 8192 gain 6 % and 3 %).
int auto_width(int D)
{
    if (D >= 9216) return 512;
    if (D >= 7168) return 256;
    return PB;
}

template <class E>
sr_status closure_impl(void *T, int64_t ldt, int D, bool vec, sr_dtype dt, cudaStream_t s, int width)
{
    const int W = width > 0 ? width : auto_width(D);
    cudaStream_t sp = side_stream(0), sr_ = side_stream(1), sc = side_stream(2);
    if (!sp || !sr_ || !sc)
        return closure_one_stream<E>(T, ldt, D, vec, dt, s);
    if (W == PB && (D + PB - 1) / PB < kLookAheadMinBlocks) {
        if (D <= PB)
            return launch_antidist_pivot(T, ldt, D, 0, -1, dt, vec, s);
        return closure_two_streams<E>(T, ldt, D, vec, dt, s, sp);
    }
    return closure_look_ahead<E>(T, ldt, D, W, vec, dt, s, sp, sr_, sc, side_stream(kPeerStream));
}

}  // namespace

sr_status launch_antidist_closure(void *T, int64_t ldt, int D, sr_dtype dt, bool vec, cudaStream_t s, int width)
{
    if (D <= 0)
        return SR_OK;
    if (width != 0 && width != 128 && width != 256 && width != 512)
        return fail(SR_EINVAL, "closure block width must be 0 (automatic), 128, 256 or 512 (got %d)", width);
    if (dt == SR_U8)
        return closure_impl<uint8_t>(T, ldt, D, vec, dt, s, width);
    if (dt == SR_U32)
        return closure_impl<uint32_t>(T, ldt, D, vec, dt, s, width);
    return closure_impl<uint16_t>(T, ldt, D, vec, dt, s, width);
}

}  // namespace sr
