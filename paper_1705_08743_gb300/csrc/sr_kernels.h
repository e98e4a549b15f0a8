// Internal launcher interface between the C ABI (capi.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/semiring.h"

namespace sr {

constexpr int kMaxDevices = 64;
int current_device();          // cudaGetDevice; -1 if that fails or the id is >= kMaxDevices
// Declares `const int var` = the current device id; returns SR_ECUDA from the
// enclosing function when there is no usable device id (per-device tables here
// have kMaxDevices slots, and a clamped id would name another device's entry).
#define SR_DEVICE_SLOT(var)                                                              \
    const int var = ::sr::current_device();                                              \
    if (var < 0)                                                                         \
        return ::sr::fail(SR_ECUDA, "no current CUDA device with an id below %d", ::sr::kMaxDevices)
int device_sm_count();         // SMs of the current device (cached)
void count_launches(int n = 1); // launch counter behind sr_kernel_launches()
// Argument checks shared by the entry points (capi.cu): a dimension in [1, 2^31);
// a non-null matrix of `rows` rows whose leading dimension covers `cols` entries
// (Boolean: words) and whose extent stays below 2^46 units.  SR_EINVAL otherwise.
sr_status check_dim(const char *fn, const char *name, int64_t v);
sr_status check_mat(const char *fn, const char *name, const void *p, int64_t ld, int64_t rows, int64_t cols,
                    sr_dtype t);
// bool_tc.cu: fp8 tensor-pipe probe (tcgen05 kind::f8f6f4, 128x256x32 MMAs); flops = 2·M·N·K per MMA
sr_status peak_tc_f8(int iters, cudaStream_t s, double *ms, double *mma_per_s, double *flops);
// tune.cu: size buckets, keys and lookups of the autotuned choices, the cache file
int64_t tune_bucket(int64_t D);
std::string tune_key(const char *op, sr_dtype t, int64_t D);
bool tune_lookup(const sr_ctx *c, const std::string &key, int *choice);
sr_status tune_load_config(sr_ctx *c, const char *path);   // at sr_create; a missing file is fine
sr_status tune_persist(const sr_ctx *c);                     // rewrite the cache, if the ctx has one
constexpr int kSideStreams = 4;
// per-device streams for look-ahead work (may be null): 0..2 high priority, 3 (kPeerStream)
// default priority, a second main stream beside the caller's
constexpr int kPeerStream = 3;
cudaStream_t side_stream(int i = 0);
sr_status event_pool(size_t n, std::vector<cudaEvent_t> *&out);   // per-thread, per-device events

// Product C := (accumulate ? C : 0) ⊕ A ⊗ B over logical R×K×N.  Rows of A/C
// with logical index >= rskip0 are shifted by rskipw, columns of B/C with logical
// index >= cskip0 by cskipw (the closure's phase 3 excludes pivot blocks this way).
struct MulArgs {
    const void *A;
    const void *B;
    void *C;
    int64_t lda, ldb, ldc;     // elements (anti-distance) or 32-bit words (Boolean)
    int R, K, N;               // logical sizes: anti-distance entries / Boolean bits
    int accumulate;
    int rskip0, rskipw;
    int cskip0, cskipw;
    int skip_tile = -1;        // a tile (row-major index, 128x128 tiles) left untouched, or -1
    int group_m = 0;           // tile order: 0 row-major; g > 0 column-major within groups of g tile rows
    int split = 1;             // a partial last wave of a deep product may split along K (u8/u16)
};

// tiles: 0 = 128x128 CTA tiles (throughput; u32: 128x64), 1 = 64x64 (latency: more CTAs for
//        thin panels and small grids)
sr_status launch_antidist_mul(const MulArgs &a, sr_dtype dt, bool vec, cudaStream_t s, int tiles = 0);
int group_rows(int R, int K, int esize, int bm);   // tile rows per group of a deep product's tile order
// closure_persistent.cu: the whole u8/u16 closure in one persistent launch (64-wide pivot
// blocks, work items in a dependency order, bounded waits on per-block versions).
constexpr int64_t kPersistentMaxD = 32768;
// D from which the persistent schedule is the automatic choice; above kPersistentMaxD: never
// (measured slower than the stream schedules at every size so far)
constexpr int64_t kPersistentAutoMinU8 = kPersistentMaxD + 1, kPersistentAutoMinU16 = kPersistentMaxD + 1;
// closure_fused.cu: u8/u16 closure with one launch per 128-wide pivot block (the next block's
// phases 1-2 as work items of the current phase 3); device workspace for its counters
// (0 if D is out of range), and the launch (16-byte aligned rows; status / spin_limit as for
// the persistent schedule)
size_t closure_fused_workspace(int64_t D);
sr_status launch_antidist_closure_fused(void *T, int64_t ldt, int D, sr_dtype dt, void *ws, size_t ws_bytes,
                                        int *status, int spin_limit, cudaStream_t s);
size_t antidist_closure_persistent_workspace(int64_t D);   // 0: not available for this D
sr_status launch_antidist_closure_persistent(void *T, int64_t ldt, int D, sr_dtype dt, void *ws, size_t ws_bytes,
                                             int *status, int spin_limit, int frac, cudaStream_t s);
// The work order as (type, pivot block, tile row, tile column, second tile column or -1)
// 5-tuples: type 0 phase-3 tiles, 1 row-panel tile, 2 column-panel tile, 3 diagonal block.
// Returns the item count (-1 outside the persistent schedule's range); writes min(cap,
// count) items to out.
long long antidist_closure_persistent_order(int64_t D, int frac, int *out, long long cap);
// closure.cu; width: block width of the blocked closure (0 = automatic, 128, 256, 512)
sr_status launch_antidist_closure(void *T, int64_t ldt, int D, sr_dtype dt, bool vec, cudaStream_t s,
                                  int width = 0);
// one CTA closes the 128-wide diagonal block kb of a D×D matrix, after its update from
// block kprev's panels (kprev < 0: none)
sr_status launch_antidist_pivot(void *T, int64_t ldt, int D, int kb, int kprev, sr_dtype dt, bool vec,
                                cudaStream_t s);
// u32 kernels (antidist32.cu), reached through launch_antidist_mul / launch_antidist_closure
sr_status launch_antidist32_mul(const MulArgs &a, bool vec, cudaStream_t s, int tiles);
sr_status launch_antidist32_pivot(void *T, int64_t ldt, int D, int kb, int kprev, cudaStream_t s);
sr_status launch_antidist_encode(const void *W, int64_t ldw, void *T, int64_t ldt, int R, int C,
                                 sr_dtype dt, int num_sms, cudaStream_t s);

// Boolean kernels work on 32-bit words; a W64 matrix is the same bit layout
// with twice as many 32-bit words per row (little-endian).
struct BoolArgs {
    const uint32_t *A;
    const uint32_t *B;
    uint32_t *C;
    int64_t lda, ldb, ldc;     // 32-bit words
    int R, K, N;               // rows; bits of k; bits per row of C (pad bits of C are written 0)
    int ncw;                   // logical 32-bit words per row of C (and of B) to process
    int accumulate;
    int skip0, skipw;          // excluded row range (rows of A and C)
    int skip0w, skipww;        // excluded word range (words of B and C)
    int ksplit = 1;            // CTAs along K (set by launch_bool_mul; partial results ORed into C)
    // tensor-core path only: a block of C left untouched, rows [hole_r0, hole_r0 + hole_rn) x
    // words [hole_w0, hole_w0 + hole_wn) (hole_rn = 0: none); its edges must fall on the
    // 128-row x 8-word tile grid or at the end of C
    int hole_r0 = 0, hole_rn = 0, hole_w0 = 0, hole_wn = 0;
    // tensor-core path only: a band of rows [band_r0, band_r0 + band_rn) across all words and
    // a band of words [band_w0, band_w0 + band_wn) down all rows, also left untouched (0: none);
    // edges on the same grid as the hole's
    int band_r0 = 0, band_rn = 0, band_w0 = 0, band_wn = 0;
};
// shape: 0 = 128 rows x 64 words per CTA, 1 = 128 x 4 (narrow panels), 2 = 32 x 16 (short panels)
sr_status launch_bool_mul(const BoolArgs &a, bool vec, cudaStream_t s, int shape = 0);
// Tensor-core Boolean product (bool_tc.cu): workspace bytes, availability, launch.
size_t bool_tc_workspace(int64_t R, int64_t K, int64_t N);
bool bool_tc_available();
// spin_limit: tries per bounded wait (0: every wait gives up at once); a wait that gives up
// sets *status and the CTA drains what it started and returns
// max_ctas: at most this many CTAs (one per SM; 0 = every SM), leaving the other SMs to
// work on other streams; run_if: a device flag read when the kernels start, the product
// skipped (C untouched) when it is 0 (null: always run)
sr_status launch_bool_mul_tc(const BoolArgs &a, void *ws, size_t ws_bytes, int *status, int spin_limit,
                             cudaStream_t s, int max_ctas = 0, const int *run_if = nullptr);
// The same product on operands already expanded to e4m3 bytes: Ae (R x Kp, K-major) and Be
// (N x Kp, B transposed), Kp = K rounded up to 128; no excluded ranges or holes.
sr_status launch_bool_mul_tc_expanded(const BoolArgs &a, uint8_t *Ae, uint8_t *Be, int *status, int spin_limit,
                                      cudaStream_t s, int max_ctas = 0, const int *run_if = nullptr);
uint8_t *tc_operand_b(uint8_t *Ae, int64_t R, int Kp);   // where B^T follows A in a tensor-core workspace
// Before squaring `it` of the repeated-squaring closure: one launch that sets flags[it % 3]
// (did squaring it - 1 change M: M != M2; it = 0: 1), clears flags[(it + 1) % 3], and
// expands M into both operands of M ⊗ M at ws (layout of launch_bool_mul_tc's workspace);
// after a squaring that changed nothing the flag stays 0 and nothing is expanded.
// (grid_sms > 0: a grid sized for that many SMs, for a chain that runs beside other work)
sr_status launch_square_prep(const uint32_t *M, const uint32_t *M2, int64_t ld, int D, int rw, void *ws, int *flags,
                             int it, cudaStream_t s, int grid_sms = 0);
// Four Russians (bool_m4r.cu); excluded ranges as in launch_bool_mul, no split K
sr_status launch_bool_mul_m4r(const BoolArgs &a, cudaStream_t s);
sr_status launch_bool_closure_warshall(uint32_t *T, int64_t ldt, int D, int rw, bool vec, cudaStream_t s);
// Closure by repeated squaring, A ⊗ (I ⊕ A)^(2^m): ws holds two D×rw word matrices (rows
// padded to 4 words) and, when tc and room allow, the tensor-core operands of a D^3 product
size_t bool_squaring_workspace(int64_t D, int64_t rw);
sr_status launch_bool_closure_squaring(uint32_t *T, int64_t ldt, int D, int rw, void *ws, size_t ws_bytes, bool tc,
                                       int *status, int spin_limit, cudaStream_t s, int grid_sms = 0);
// Blocked Warshall with kBoolWideBlock-bit blocks and phase 3 on the tensor cores; ws as
// for launch_bool_mul_tc, at least bool_closure_wide_workspace(D) bytes
constexpr int kBoolWideBlock = 2048;
size_t bool_closure_wide_workspace(int64_t D);
sr_status launch_bool_closure_wide(uint32_t *T, int64_t ldt, int D, int rw, void *ws, size_t ws_bytes,
                                   int *status, int spin_limit, cudaStream_t s, int side_sms = -1);
sr_status launch_bool_pack(const uint8_t *dense, int64_t ldd, uint32_t *M, int64_t ldm, int R, int C,
                           int rw, int num_sms, cudaStream_t s);
sr_status launch_bool_unpack(const uint32_t *M, int64_t ldm, uint8_t *dense, int64_t ldd, int R, int C,
                             int num_sms, cudaStream_t s);
sr_status launch_bool_identity_or(uint32_t *M, int64_t ldm, int D, cudaStream_t s);
sr_status launch_copy_rows(const uint32_t *src, int64_t lds, uint32_t *dst, int64_t ldd, int R, int rw,
                           cudaStream_t s);

// Batched closure (batched.cu): graph descriptors and work items on the device.
struct BatchGraph {
    void *T;
    int64_t ldt;
    int D;
    int pad;        // 1: T and every row are 16-byte aligned (vector accesses)
};
struct BatchItem {
    int n;          // graphs in the item (1 for a cooperative item)
    int coop;       // 1: all CTAs of the cluster close g[0] together
    int g[4];
};
// One persistent launch without clusters: item i closes graph items[i].g[0] on one CTA.
// The batched closure's grouped schedule (antidist.cu): many products in one launch, CTA b
// taking tile b - start[i] of product args[i] (thin: 64x64 tiles, else 128x128); block kb
// of graphs[active[0..n)] closed by one CTA each (phase 3 of kb-1 already applied).
sr_status launch_antidist_mul_grouped(const MulArgs *args, const int *start, int n, int tiles, sr_dtype dt,
                                      bool vec, bool thin, cudaStream_t s);
sr_status launch_antidist_pivot_grouped(const BatchGraph *graphs, const int *active, int n, int kb, sr_dtype dt,
                                        cudaStream_t s);
sr_status launch_batched_closure_flat(sr_dtype dt, const BatchGraph *d_graphs, const BatchItem *d_items, int nitems,
                                      int *d_counter, int ctas_per_sm, cudaStream_t s);

// Entrywise operations and the reflexive closure (elementwise.cu).
sr_status launch_entrywise(int op, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                           int R, int N, sr_dtype dt, cudaStream_t s);
sr_status launch_reflexive(void *T, int64_t ldt, int D, sr_dtype dt, cudaStream_t s);

}  // namespace sr
