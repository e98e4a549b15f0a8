/*
 * semiring.h — C ABI of the GB300 semiring library (libsemiring.so).
 *
 * Matrices over the Boolean semiring and over the saturating anti-distance
 * semiring of de Bondt, "Fast algorithms for anti-distance matrices as a
 * generalization of Boolean matrices" (arXiv 1705.08743):
 *
 *   Boolean (Section 2):          entries {0,1},  a ⊕ b = max(a,b),  a ⊗ b = min(a,b)
 *   anti-distance (Sections 3-4): entries {0..S}, a ⊕ b = max(a,b),  a ⊗ b = max(a+b−S, 0)
 *                                 S = 255 (u8), 65535 (u16) or 2^32 − 1 (u32, the three
 *                                 types of Section 4); entry S − d stands
 *                                 for distance d, 0 for "no path / distance >= S".
 *
 * Conventions shared by every call
 *  - Pointers to matrix data are DEVICE pointers owned by the caller (or pinned
 *    host memory the device maps at the same pointer: sr_host_mapped); the
 *    library never frees them.  Matrices are row-major with a leading
 *    dimension ld >= row width, in elements (u8/u16/u32) or in words of the
 *    Boolean word type (32- or 64-bit).
 *  - Boolean matrices are bit-packed: entry (i, j) is bit (j mod w) of word
 *    floor(j / w) of row i (w = 32 or 64), i.e. bit (j & 7) of byte (j >> 3)
 *    on a little-endian machine (Section 4, matBool).  Bits past the logical
 *    width are "pad bits": they are ignored on input and written 0 on output.
 *  - `stream` is a cudaStream_t (0 = legacy default stream).  Calls only
 *    enqueue work and return; results are ordered on `stream`.  A call that
 *    returns SR_OK has launched all its kernels; device-side errors surface at
 *    the next synchronisation (sr_stream_status reports bounded-wait timeouts).
 *  - Vector (16-byte) loads are used when every base pointer is 16-byte
 *    aligned and ld·(bytes per element) is a multiple of 16; any other
 *    alignment is accepted and runs a slower element-wise path.
 *  - Errors: every call returns an sr_status; on failure nothing was enqueued
 *    and sr_last_error() (per calling thread) says why.  No C++ exception
 *    crosses this interface.
 *  - `ctx` may be NULL for calls that need no workspace (products, closures
 *    by the blocked Warshall method, encoding).  Calls that share one ctx and
 *    use its workspace must be ordered on one stream.
 */
#ifndef SEMIRING_H
#define SEMIRING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SR_OK = 0,
    SR_EINVAL = 1,     /* bad argument: size, ld, dtype, overlap, NULL pointer */
    SR_ENOMEM = 2,     /* workspace or serving memory budget too small */
    SR_ECUDA = 3,      /* a CUDA runtime call failed (message has the CUDA error) */
    SR_ETIMEOUT = 4,   /* a bounded device-side or host-side wait gave up */
    SR_EAGAIN = 5,     /* serving: no free slot or memory now; retry later */
    SR_EBUSY = 6,      /* serving: ticket not finished yet */
    SR_ENOTFOUND = 7,  /* serving: unknown or already released ticket */
    SR_ECANCELED = 8   /* serving: the request was cancelled before it ran (sr_cancel) */
} sr_status;

typedef enum {
    SR_BOOL_W32 = 0,   /* Boolean, 32 columns per uint32 word */
    SR_BOOL_W64 = 1,   /* Boolean, 64 columns per uint64 word */
    SR_U8 = 2,         /* anti-distance, S = 255, one uint8 per entry */
    SR_U16 = 3,        /* anti-distance, S = 65535, one uint16 per entry */
    SR_U32 = 4         /* anti-distance, S = 2^32 − 1, one uint32 per entry (Section 4's
                          third type; a + b − S needs 33 bits, so ⊗ is computed as the
                          saturating subtraction b ⊖ (S − a) = max(b, S − a) − (S − a)) */
} sr_dtype;

typedef enum {
    SR_CLOSURE_WARSHALL = 0,   /* three-phase blocked Warshall/Floyd (Section 2) */
    SR_CLOSURE_SQUARING = 1    /* A ⊗ (I ⊕ A)^(2^m), m = ceil(log2(D−1)) (Section 2) */
} sr_closure_method;

typedef enum {
    SR_OP_ANTIDIST_MUL = 0,
    SR_OP_BOOL_MUL = 1,
    SR_OP_ANTIDIST_CLOSURE = 2,
    SR_OP_BOOL_CLOSURE = 3,
    SR_OP_DIST_MUL = 4
} sr_op;

typedef struct sr_ctx sr_ctx;

typedef struct {
    size_t workspace_bytes;    /* device workspace allocated by sr_create (0: none) */
    int spin_limit;            /* iterations before a device-side wait gives up (0: default) */
    const char *tune_cache;    /* JSON file of autotuned choices (NULL: none); sr_create loads it
                                  if it exists, parses, and was written on a GPU of the same name
                                  and SM count (otherwise it starts with no choices), and each new
                                  tuning rewrites it (see sr_autotune_closure) */
    int reserved[4];
} sr_config;

/* ---------------------------------------------------------------- context */

/* Create a context on the current CUDA device; cfg may be NULL (defaults).
 * Allocates cfg->workspace_bytes of device memory once; no later call of the
 * library allocates device memory on this context's behalf except the serving
 * loop (sr_serve_*), which allocates its arena when it starts. */
sr_status sr_create(sr_ctx **out, const sr_config *cfg);
void sr_destroy(sr_ctx *ctx);
/* Message of the last failed call made by this thread ("" if none). */
const char *sr_last_error(void);
/* Library version string. */
const char *sr_version(void);
/* Device workspace bytes for a call on D×D operands (0 for calls that use none): what
 * SR_CLOSURE_SQUARING and dist_mul need, and what lets bool_mul and the Warshall form of
 * bool_closure take their tensor-core paths (they run without it). */
sr_status sr_workspace_query(int op, sr_dtype dtype, int64_t D, int method, size_t *bytes);

/* Options of a context. */
typedef enum {
    SR_OPT_BOOL_TENSOR = 1,  /* Boolean products on the tensor cores (count, then test > 0):
                                0 never, 1 when K >= 1024 (default), 2 whenever possible.
                                Used only with enough ctx workspace (sr_workspace_query). */
    SR_OPT_BOOL_FOUR_RUSSIANS = 2, /* Boolean products off the tensor cores by the method of
                                Four Russians (8-bit groups of K, 256-entry OR tables of
                                rows of B; Section 4 names the method for the product):
                                0 never, 1 for large products (default), 2 always. */
    SR_OPT_SPIN_LIMIT = 3,   /* tries per bounded device-side wait (the tensor-core pipeline's
                                mbarrier waits); a wait that gives up sets the context's status
                                word, which sr_stream_status reports as SR_ETIMEOUT, and the CTA
                                drains the copies and MMAs it started and returns.  0 makes
                                every wait give up at once (fault injection for tests); the
                                default is sr_config.spin_limit. */
    SR_OPT_CLOSURE_BLOCK = 4, /* block width of the anti-distance closure's blocked Warshall/Floyd
                                loop (antidist_closure, dist_closure): 0 automatic (default),
                                128, 256 or 512.  Wider blocks mean fewer, deeper phase-3
                                products; their diagonal blocks are closed at width 128.
                                A width other than 0 also turns the persistent schedule off. */
    SR_OPT_CLOSURE_PERSISTENT = 5, /* u8/u16 anti-distance closure in one persistent launch
                                (128-wide pivot blocks; work items taken in a dependency order,
                                each waiting, bounded by SR_OPT_SPIN_LIMIT, on per-block
                                counters): 0 never, 1 automatic (default; the stream schedule
                                is faster at every size measured so far), 2 whenever
                                possible.  Needs 16-byte aligned rows, 256 <= D <= 32768
                                and a ctx workspace of sr_workspace_query(
                                SR_OP_ANTIDIST_CLOSURE, dtype, D, 0, ..) bytes; without them the
                                stream schedule runs. */
    SR_OPT_CLOSURE_PANEL_SHARE = 6, /* persistent closure: share of each pivot block's phase-3
                                tiles queued before the next pivot block's panels, in 1/256
                                (0..256, default 128) */
    SR_OPT_BOOL_SIDE_SMS = 7, /* Boolean closure on the tensor cores (2048-bit blocks): SMs that
                                phase 3 leaves free for the next diagonal block's update and
                                squarings running beside it (-1: the default, 32) */
    SR_OPT_PRODUCT_SPLIT = 8, /* u8/u16 antidist_mul with K >= 1024: when the last wave of CTAs
                                holds fewer tiles than half the SMs, each of its tiles is
                                shared by a thread-block cluster of 2-4 CTAs over slices of
                                K, merged through distributed shared memory (same result;
                                ⊕ = max is order-free): 0 never, 1 automatic (default) */
    SR_OPT_CLOSURE_FUSED = 9 /* u8/u16 anti-distance closure with one launch per 128-wide pivot
                                block, the next block's phases 1-2 taken as work items beside
                                the current phase 3 (bounded waits as SR_OPT_SPIN_LIMIT):
                                0 never, 1 automatic (default), 2 whenever possible.  Needs
                                16-byte aligned rows and a ctx workspace of
                                sr_workspace_query(SR_OP_ANTIDIST_CLOSURE, ..) bytes;
                                without them the stream schedule runs. */
} sr_option;
sr_status sr_set_option(sr_ctx *ctx, int option, int value);

/* ---------------------------------------------------------------- host buffers */

/* *mapped := 1 if p is pinned host memory (cudaHostAlloc / cudaHostRegister, e.g. a
 * torch pin_memory() tensor) that the current device addresses at the same pointer
 * (unified addressing), else 0 (device memory, pageable or unknown host memory).  Such
 * buffers may be passed as operands, or as the output of a call that never reads it
 * (accumulate = 0): the kernels then read and write host memory over the host link
 * (NVLink-C2C on Grace), with no staging copy.  Pass nothing else that is not device
 * memory.  Errors: SR_EINVAL for a NULL mapped. */
sr_status sr_host_mapped(const void *p, int *mapped);

/* ---------------------------------------------------------------- row-sharded products */

/* Rows [*r0, *r1) of an R-row product for `rank` of `world` processes (one GPU each).
 * The rows of P = A ⊗ B are independent (Section 2 product formula: row i of P needs
 * row i of A and all of B), so a product shards by row blocks of A and C with B
 * replicated and no reduction; each rank then calls antidist_mul / bool_mul on its
 * rows.  Ranges are whole groups of `align` rows (the CTA tile height, 128, keeps every
 * rank's tiles full), as even as possible, disjoint, in rank order, covering [0, R).
 * Host only, no CUDA call. */
sr_status sr_shard_rows(int64_t R, int world, int rank, int64_t align, int64_t *r0, int64_t *r1);

/* ---------------------------------------------------------------- autotuner */

/* Choices the autotuner records (sr_tune_get / sr_tune_set):
 *   SR_OP_ANTIDIST_CLOSURE: 128, 256 or 512 (block width of the stream schedule),
 *                           SR_TUNE_PERSISTENT (the persistent schedule) or SR_TUNE_FUSED
 *                           (one launch per pivot block, SR_OPT_CLOSURE_FUSED);
 *   SR_OP_BOOL_MUL:         SR_TUNE_BOOL_WORDS, SR_TUNE_BOOL_TABLES (Four Russians) or
 *                           SR_TUNE_BOOL_TENSOR;
 *   SR_OP_ANTIDIST_MUL:     128 or 64 (CTA tile side).
 * Choices are kept per (op, dtype, size bucket): buckets are 256, 384, 512, 768, 1024,
 * ... (powers of two and 1.5 times them) and a size uses the smallest bucket >= it. */
enum { SR_TUNE_BOOL_WORDS = 0, SR_TUNE_BOOL_TABLES = 1, SR_TUNE_BOOL_TENSOR = 2, SR_TUNE_PERSISTENT = 1,
       SR_TUNE_FUSED = 2 };

/* Time every schedule of the anti-distance closure (dtype u8/u16/u32) on a scratch
 * matrix of the bucket's order D' >= D (allocated and freed here; D' <= 65536) and record
 * the fastest for the bucket: stream schedules with blocks of 128, 256 and 512, and the
 * persistent and fused-pass schedules (u8/u16) when the ctx workspace holds what they
 * need.  reps timed runs per
 * candidate (best taken) after one untimed run, on `stream` (synchronised).  An existing
 * choice is returned without timing unless force != 0.  antidist_closure and
 * dist_closure then follow the choice while SR_OPT_CLOSURE_BLOCK is 0 and
 * SR_OPT_CLOSURE_PERSISTENT and SR_OPT_CLOSURE_FUSED are 1 (their defaults).  Rewrites
 * the ctx's tune cache.
 * Outputs (may be NULL): the choice and its time in ms. */
sr_status sr_autotune_closure(sr_ctx *ctx, sr_dtype dtype, int64_t D, void *stream, int reps, int force,
                              int *choice, double *best_ms);
/* The same for the D×D×D product: op SR_OP_BOOL_MUL (Boolean dtype; masked-OR words,
 * Four Russians tables, tensor cores when the ctx workspace allows) or
 * SR_OP_ANTIDIST_MUL (u8/u16/u32; 128x128 or 64x64 tiles).  bool_mul / antidist_mul
 * follow the choice for sizes of the bucket (max(R, K, N)) while SR_OPT_BOOL_TENSOR and
 * SR_OPT_BOOL_FOUR_RUSSIANS are 1 (their defaults). */
sr_status sr_autotune_mul(sr_ctx *ctx, int op, sr_dtype dtype, int64_t D, void *stream, int reps, int force,
                          int *choice, double *best_ms);
/* Read or set one recorded choice (SR_ENOTFOUND: none recorded); sr_tune_set rewrites the
 * tune cache. */
sr_status sr_tune_get(const sr_ctx *ctx, int op, sr_dtype dtype, int64_t D, int *choice, double *ms);
sr_status sr_tune_set(sr_ctx *ctx, int op, sr_dtype dtype, int64_t D, int choice);
/* Write every recorded choice (batches included) to a JSON file / merge one written by
 * this library on a GPU of the same name and SM count (SR_EINVAL otherwise). */
sr_status sr_tune_save(const sr_ctx *ctx, const char *path);
sr_status sr_tune_load(sr_ctx *ctx, const char *path);

/* The work order of the persistent anti-distance closure (SR_OPT_CLOSURE_PERSISTENT) for an
 * order-D matrix and panel share `share` (as SR_OPT_CLOSURE_PANEL_SHARE), for tests and
 * tools; host only, no CUDA call.  Writes min(cap, count) items to out (host memory, may be
 * NULL) as 5 ints (type, pivot block s, tile row i, tile column j, second tile column j2
 * or -1) — type 0: 128x128 phase-3 tiles (i, j) and (i, j2) on the grid without block
 * row/column s (Section 2 Warshall step, T_ij ⊕= T_is ⊗ T_sj); 1: a row-panel tile j;
 * 2: a column-panel tile i; 3: the diagonal block s — and returns the item count, or -1
 * if D is outside [256, 32768]. */
long long sr_closure_order(int64_t D, int share, int *out, long long cap);

/* ---------------------------------------------------------------- encoding (Sections 3-4) */

/* T (R×C, dtype SR_U8, SR_U16 or SR_U32) := anti-distance encoding of integer edge
 * lengths W (same element type, same shape): entry = S − w for 0 < w < S,
 * and 0 for w = 0 ("no edge") or w >= S (not distinguished from infinity,
 * Section 3).  W and T may be the same buffer. */
sr_status antidist_encode(sr_ctx *ctx, const void *W, int64_t ldw, void *T, int64_t ldt,
                          int64_t R, int64_t C, sr_dtype dtype, void *stream);

/* M (R×C bits, dtype SR_BOOL_W32/W64) := dense 0/1 bytes (nonzero = 1), pad bits 0. */
sr_status bool_pack(sr_ctx *ctx, const uint8_t *dense, int64_t ldd, void *M, int64_t ldm,
                    int64_t R, int64_t C, sr_dtype dtype, void *stream);
/* dense (R×C bytes) := 0/1 entries of the bit matrix M. */
sr_status bool_unpack(sr_ctx *ctx, const void *M, int64_t ldm, uint8_t *dense, int64_t ldd,
                      int64_t R, int64_t C, sr_dtype dtype, void *stream);

/* ---------------------------------------------------------------- products (Section 2 formula; Section 4 listings) */

/* C := (accumulate ? C : 0) ⊕ A ⊗ B with A R×K, B K×N, C R×N, anti-distance
 * (dtype SR_U8, SR_U16 or SR_U32).  (A ⊗ B)_ij = max over k of max(A_ik + B_kj − S, 0).
 * C must not overlap A or B (the aliased form is the closure).
 * R, K, N >= 1 and < 2^31. */
sr_status antidist_mul(sr_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb,
                       void *C, int64_t ldc, int64_t R, int64_t K, int64_t N,
                       sr_dtype dtype, int accumulate, void *stream);

/* Boolean product of bit matrices: C := (accumulate ? C : 0) ⊕ A ⊗ B,
 * (A ⊗ B)_ij = OR over k of (A_ik AND B_kj).  dtype SR_BOOL_W32 or W64;
 * lda/ldb/ldc in words.  C must not overlap A or B.
 * With a ctx whose workspace holds sr_workspace_query(SR_OP_BOOL_MUL, ..) bytes for
 * max(R, K, N), the product runs on the tensor cores as a count (fp8 0/1 operands,
 * fp32 sums, exact) followed by the test count > 0 (SR_OPT_BOOL_TENSOR); otherwise
 * on 32-bit words, by table lookups (Four Russians, SR_OPT_BOOL_FOUR_RUSSIANS) or by
 * masked ORs (for each k with A_ik = 1, row k of B ORed into row i of C).  Every
 * path gives the same bits. */
sr_status bool_mul(sr_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb,
                   void *C, int64_t ldc, int64_t R, int64_t K, int64_t N,
                   sr_dtype dtype, int accumulate, void *stream);

/* ---------------------------------------------------------------- closures (Section 2 Warshall; Section 3 Floyd) */

/* In place: T (D×D) := A ⊕ A⊗A ⊕ A⊗A⊗A ⊕ ... (non-reflexive closure; T_ii is
 * the best cycle through i).  Anti-distance dtype SR_U8 / SR_U16 / SR_U32; three-phase
 * blocked Warshall/Floyd.  Needs no workspace. */
sr_status antidist_closure(sr_ctx *ctx, void *T, int64_t ldt, int64_t D, sr_dtype dtype,
                           void *stream);

/* In place Boolean transitive closure of the D×D bit matrix T (dtype
 * SR_BOOL_W32/W64).  method SR_CLOSURE_WARSHALL needs no workspace: blocked Warshall
 * with 128-bit pivot blocks.  With a ctx holding sr_workspace_query(SR_OP_BOOL_CLOSURE,
 * .., SR_CLOSURE_WARSHALL) bytes (operands of 2048-deep tensor-core products) and
 * D >= 4096 (any D > 2048 with SR_OPT_BOOL_TENSOR = 2), the loop takes 2048-bit blocks
 * and runs its panels and phase 3 on the tensor cores (count, then test > 0; the same
 * bits).  SR_CLOSURE_SQUARING (A ⊗ (I ⊕ A)^(2^m), m = ceil(log2(D - 1)); Section 2's
 * identity) needs sr_workspace_query() bytes of ctx workspace; on the tensor cores
 * (D >= 1024, or SR_OPT_BOOL_TENSOR = 2) it skips the squarings after the first one that
 * leaves the power unchanged, which gives the same bits. */
sr_status bool_closure(sr_ctx *ctx, void *T, int64_t ldt, int64_t D, sr_dtype dtype,
                       int method, void *stream);

/* ---------------------------------------------------------------- batched closures (many graphs, one launch) */

/* One operation of a batch or a served request.  Closures: C is the D×D matrix
 * closed in place, ldc its leading dimension, R = K = N = D (A, B unused).
 * Products: C := (accumulate ? C : 0) ⊕ A ⊗ B with A R×K, B K×N (lda/ldb/ldc as in
 * the product calls).  All pointers are device pointers owned by the caller. */
typedef struct {
    int op;                /* sr_op */
    int dtype;             /* sr_dtype */
    const void *A;
    const void *B;
    void *C;
    int64_t lda, ldb, ldc;
    int64_t R, K, N;
    int accumulate;
    int method;            /* closures of Boolean matrices: sr_closure_method */
} sr_desc;

typedef struct sr_batch sr_batch;

/* Plan a batch of n independent anti-distance closures (op SR_OP_ANTIDIST_CLOSURE,
 * one dtype for the whole batch, SR_U8 or SR_U16 (SR_U32: SR_EINVAL), matrices must not overlap) for one persistent
 * launch (Section 2 Warshall / Section 3 Floyd on every graph).  Graphs are ordered
 * by cost, largest first; graphs with D >= the cooperative threshold are closed by
 * all CTAs of a thread-block cluster together, smaller ones one per CTA.  Allocates
 * the plan's small device arrays (descriptors, work items, one counter). */
sr_status sr_batch_create(sr_ctx *ctx, const sr_desc *d, int n, sr_batch **out);
/* Enqueue the batch on `stream`.  use_graph != 0: the counter reset and the
 * persistent kernel are captured once into a CUDA graph, replayed on every later call. */
sr_status sr_batch_launch(sr_batch *b, int use_graph, void *stream);
/* Tuning: cluster size (1, 2 or 4), cooperative threshold on D, CTAs per SM.  Cluster 0
 * selects the grouped schedule instead of the persistent kernel: blocked Floyd with
 * pivot blocks of 128 run on every graph at once, three launches per pivot block
 * (phase 1, one CTA per open graph; phase 2, all panels; phase 3, all remaining
 * blocks), captured into the same CUDA graph; the other two values are then unused. */
sr_status sr_batch_set_tuning(sr_batch *b, int cluster, int coop_threshold, int ctas_per_sm);
sr_status sr_batch_get_tuning(const sr_batch *b, int *cluster, int *coop_threshold, int *ctas_per_sm);
/* Autotuner: times the candidate tunings on this batch (closures are idempotent, so
 * re-running them leaves the results unchanged), keeps the fastest, and records it in
 * ctx under the batch's signature (dtype, SM count, histogram of D); a later call with
 * a batch of the same signature reuses it without timing.  Synchronises `stream`.
 * best_ms (may be NULL) receives the best time per launch, or -1 if reused. */
sr_status sr_batch_autotune(sr_ctx *ctx, sr_batch *b, void *stream, int reps, double *best_ms);
sr_status sr_batch_info(const sr_batch *b, int *ngraphs, int *nitems, double *ops);
/* Per-graph completion times.  enable != 0: every later launch writes the device clock
 * (ns) at its start and when each graph is complete — at the end of the graph's own
 * closure in the persistent kernel, at the end of the last pivot step the graph takes
 * part in for the grouped schedule (one more one-thread kernel per step) — into a
 * device array the batch allocates now (8·(1 + n + steps) bytes); 0 frees it.  Either
 * change discards a captured graph, which the next use_graph launch captures again. */
sr_status sr_batch_set_timing(sr_batch *b, int enable);
/* After a timed launch has completed (the caller synchronises its stream): ms[g] =
 * time from the launch's start to graph g's completion, in the order of the batch's
 * descriptors.  Copies the stamps with cudaMemcpy.  SR_EINVAL if timing is off. */
sr_status sr_batch_completion_ms(const sr_batch *b, double *ms);
void sr_batch_destroy(sr_batch *b);
/* One-shot form: plan (using ctx's recorded tuning for this signature, if any),
 * launch, synchronise `stream`, free the plan. */
sr_status sr_batched(sr_ctx *ctx, const sr_desc *d, int n, void *stream);

/* ---------------------------------------------------------------- served request loop */

/* One request of the serving loop.  Matrices are host buffers, dense row-major
 * (leading dimension = row width, in entries or Boolean words), or resident
 * matrices named by a handle.  For overlap and asynchrony the host buffers should
 * be page-locked (cudaHostAlloc, torch pin_memory); pageable buffers still work but
 * serialise the loop.  Inputs must stay valid and outputs untouched until the
 * request is done.
 *  - closures (SR_OP_ANTIDIST_CLOSURE u8/u16/u32, SR_OP_BOOL_CLOSURE W32/W64 with
 *    `method`): D = R; input A (or resident rA); result written to `out`.
 *  - products (SR_OP_ANTIDIST_MUL, SR_OP_BOOL_MUL): A R×K (or rA), B K×N (or rB),
 *    result R×N written to `out` (NULL: no transfer back).
 *  - keep != 0: the result stays resident; sr_result reports its handle. */
typedef struct {
    int op;
    int dtype;
    int64_t R, K, N;
    const void *A;
    const void *B;
    uint64_t rA, rB;
    void *out;
    int keep;
    int method;
} sr_request;

typedef struct {
    size_t arena_bytes;      /* device memory budget for admitted requests and resident matrices (default 1 GiB) */
    int slots;               /* concurrent stream slots: admitted work in flight (default 4) */
    int max_pending;         /* waiting requests before sr_submit answers SR_EAGAIN (default 4096) */
    int batch_max_d;         /* u8/u16 anti-distance closures with D <= this are grouped into one batched launch (512) */
    int batch_max_graphs;    /* graphs per grouped launch (64, at most 1024) */
    int backfill_ms;         /* later requests may overtake the head while it has waited less than this (0) */
} sr_serve_config;

typedef struct {
    int status;              /* SR_OK, or the error that ended this request */
    double latency_ms;       /* submission to completion (host clock) */
    double queue_ms;         /* submission to admission */
    uint64_t resident;       /* handle of the kept result (keep != 0), else 0 */
} sr_result_info;

typedef struct {
    uint64_t submitted, completed, failed, batches, batched_requests, cancelled;
    size_t arena_bytes, arena_in_use, arena_peak_bytes;
    int pending, inflight, residents;
} sr_serve_stats_t;

/* Start the loop on ctx's device: allocates the arena (one cudaMalloc), per-slot
 * streams and staging buffers, and a scheduler thread.  Requests are admitted in
 * submission order as stream slots and arena memory free up (continuous
 * batching); waiting small closures of one dtype join one batched launch.  A request
 * estimated to take a millisecond or more of device time waits while another such
 * request is in flight (two would slow each other down); shorter ones run beside it. */
sr_status sr_serve_start(sr_ctx *ctx, const sr_serve_config *cfg);
/* Stop the loop (waits for admitted work), free its memory; also done by sr_destroy. */
sr_status sr_serve_stop(sr_ctx *ctx);
/* Queue a request; returns its ticket.  SR_EAGAIN: queue full; SR_ENOMEM: larger
 * than the whole arena; SR_EINVAL / SR_ENOTFOUND: bad request / unknown handle. */
sr_status sr_submit(sr_ctx *ctx, const sr_request *req, uint64_t *ticket);
sr_status sr_poll(sr_ctx *ctx, uint64_t ticket, int *done);
/* Block until done or timeout_ms elapsed (SR_ETIMEOUT); returns the request's status. */
sr_status sr_wait(sr_ctx *ctx, uint64_t ticket, int timeout_ms);
sr_status sr_result(sr_ctx *ctx, uint64_t ticket, sr_result_info *info);
/* Withdraw a waiting request: it leaves the queue without running, and sr_wait /
 * sr_result then report SR_ECANCELED for it (its output buffer is not written).
 * SR_EBUSY: already admitted (running requests finish); SR_OK without effect on a
 * finished ticket; SR_ENOTFOUND: unknown ticket.  The ticket still needs sr_release. */
sr_status sr_cancel(sr_ctx *ctx, uint64_t ticket);
/* Forget a finished ticket (a kept result stays resident until sr_resident_free). */
sr_status sr_release(sr_ctx *ctx, uint64_t ticket);
/* Resident matrices (in the arena): upload (blocking), download (synchronises the
 * device first), free. */
sr_status sr_resident_put(sr_ctx *ctx, const void *host, int64_t rows, int64_t cols, sr_dtype dtype,
                          uint64_t *handle);
sr_status sr_resident_get(sr_ctx *ctx, uint64_t handle, void *host);
sr_status sr_resident_free(sr_ctx *ctx, uint64_t handle);
sr_status sr_serve_stats(sr_ctx *ctx, sr_serve_stats_t *out);

/* ---------------------------------------------------------------- allocation-free variant */

/* Size of the library-owned scratch array used by bool_closure_squaring_noalloc. */
#define SR_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Boolean closure by repeated squaring, like bool_closure(..., SR_CLOSURE_SQUARING, ...),
 * but with no workspace argument and no allocation of any kind.  (The paper has no
 * counterpart: this is a deployment variant of the library.)  It is for callers that
 * cannot allocate device memory — code that runs where another allocator already owns
 * the device's memory, plugins held to a fixed memory budget, loops that must not pay
 * for cudaMalloc's implicit synchronisation.  Its scratch is a 16 MiB array inside the
 * library image; once loaded on a GPU it stays there until the process exits.
 *  - Loading: with CUDA's default lazy module loading the array is placed on a device
 *    by the first call on that device (which looks up its address), so that first
 *    call does take 16 MiB of device memory and may synchronise the device.  Make it
 *    (a 1×1 matrix will do) before another allocator claims the device's free
 *    memory, or set CUDA_MODULE_LOADING=EAGER to load it with the CUDA context.
 *  - T, ldt, D, dtype as in bool_closure (same argument checks); D×D problems whose two scratch matrices
 *    (2·D·ceil32(D)/8 bytes, rows padded to 16 bytes) exceed SR_NOALLOC_SCRATCH_BYTES
 *    return SR_EINVAL before anything is queued; every D <= 8192 fits.
 *  - All calls share the one array and leave their data in it; each call overwrites
 *    the scratch it reads, but calls that overlap on the GPU (unordered streams) race.
 *  - The first call on a device looks the array's address up on that device; make that
 *    first call before any stream capture.
 *  - Calls no cudaMalloc/cudaFree or any allocating routine (after the first call on a
 *    device has loaded the array, as above). */
sr_status bool_closure_squaring_noalloc(void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream);

/* ---------------------------------------------------------------- distance form (Section 4 dual; Conclusion) */

/* Distance matrices: entry = length d in {0..S}, S standing for infinity (no
 * path or length >= S).  ∧ = min replaces ∨ and saturating addition replaces ⊗
 * (Section 4: the dual operations; De Morgan: S − (A ⊗ B) = (S − A) + (S − B)).
 *   dist_mul:     C := (accumulate ? C : all-S) ∧ (A + B),
 *                 (A + B)_ij = min over k of min(A_ik + B_kj, S);
 *                 computed as S − antidist_mul(S − A, S − B); needs ctx workspace of
 *                 sr_workspace_query(SR_OP_DIST_MUL, dtype, max(R, K, N), 0) bytes.
 *   dist_closure: in place, T := shortest saturated lengths of paths with >= 1 edge;
 *                 T_ii = shortest cycle through i (the Conclusion's dransclose, minimum
 *                 loop lengths on the diagonal); computed as S − antidist_closure(S − T)
 *                 in place, no workspace.
 * dtype SR_U8, SR_U16 or SR_U32. */
sr_status dist_mul(sr_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                   int64_t R, int64_t K, int64_t N, sr_dtype dtype, int accumulate, void *stream);
sr_status dist_closure(sr_ctx *ctx, void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream);

/* ---------------------------------------------------------------- entrywise (Conclusion table) */

typedef enum {
    SR_EW_AND = 0,     /* a & b = min(a, b)   (Boolean: AND) */
    SR_EW_OR = 1,      /* a | b = max(a, b)   (Boolean: OR)  */
    SR_EW_XOR = 2,     /* a ^ b = |a − b|     (Boolean: XOR) */
    SR_EW_NOT = 3      /* ~a = S − a          (Boolean: NOT; B unused, may be NULL) */
} sr_entrywise_op;

/* C := A op B entrywise, R×N, any dtype (Boolean: words, pad bits written 0).
 * C may be A or B (in place). */
sr_status sr_entrywise(sr_ctx *ctx, int op, const void *A, int64_t lda, const void *B, int64_t ldb, void *C,
                       int64_t ldc, int64_t R, int64_t N, sr_dtype dtype, void *stream);
/* Reflexive closure from the non-reflexive one: T := I ⊕ T (diagonal set to S or to 1). */
sr_status sr_reflexive(sr_ctx *ctx, void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream);

/* ---------------------------------------------------------------- diagnostics */

/* Number of kernel launches this library has made in this process (all devices). */
uint64_t sr_kernel_launches(void);

/* Roofline denominators: micro-benchmark of one inner operation of the
 * kernels, as an issue-bound stream over every SM of the current device
 * (blocks_per_sm CTAs of 256 threads, 128·iters operations per thread).
 * Synchronises `stream`; allocates and frees a few bytes with cudaMallocAsync.
 * Outputs: elapsed ms, instructions/s, semiring operations/s. */
typedef enum {
    SR_PEAK_DPX_S16X2 = 0,   /* max(x + a, acc) on 16-bit lane pairs (u8 product): 2 ops/instr */
    SR_PEAK_U16_PAIR = 1,    /* max(max(x, na) + nga, acc) on lane pairs (u16): 2 ops per 2 instr */
    SR_PEAK_LOP3 = 2,        /* acc |= x & m (Boolean): 32 ops/instr */
    SR_PEAK_IADD = 3,        /* 32-bit integer add (reference) */
    SR_PEAK_U32_PAIR = 4,    /* max(max(x, na) + pa, acc) on one 32-bit entry (u32): 1 op per 2 instr */
    SR_PEAK_TC_F8 = 5        /* tensor cores: tcgen05.mma kind::f8f6f4, M=128 N=256 K=32, e4m3 operands,
                                f32 accumulators (the Boolean count path's instruction), one CTA per SM
                                issuing `iters` MMAs; instr = MMAs, ops = flops (2·M·N·K per MMA).
                                The integer MMA (kind::i8) does not exist for sm_103a. */
} sr_peak_op;
sr_status sr_peak_probe(int op, int iters, int blocks_per_sm, void *stream, double *ms,
                        double *instr_per_s, double *ops_per_s);

/* Reads and clears the context's device status word (bounded waits that gave
 * up), synchronising `stream` first.  SR_OK or SR_ETIMEOUT. */
sr_status sr_stream_status(sr_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SEMIRING_H */
