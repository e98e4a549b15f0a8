// C ABI of the semiring library: argument checks, context, dispatch to kernels.
// Every exported function returns an sr_status and never throws.

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>

#include "sr_common.cuh"
#include "sr_kernels.h"
#include "sr_trace.h"
#include "sr_ctx.h"

namespace sr {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

sr_status fail(sr_status st, const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

sr_status cuda_fail(cudaError_t e, const char *what)
{
    g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SR_ECUDA;
}

static std::atomic<uint64_t> g_launches{0};
void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return -1;
    return (d < 0 || d >= kMaxDevices) ? -1 : d;
}

int device_sm_count()
{
    static int cache[kMaxDevices] = {};
    const int d = current_device();
    if (d < 0) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 1;
        return n;
    }
    if (cache[d] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 1;
        cache[d] = n;
    }
    return cache[d];
}

// ------------------------------------------------------------------ checks
static bool is_anti(sr_dtype t) { return t == SR_U8 || t == SR_U16 || t == SR_U32; }
static bool is_bool(sr_dtype t) { return t == SR_BOOL_W32 || t == SR_BOOL_W64; }
static int esize(sr_dtype t) { return t == SR_U8 ? 1 : t == SR_U16 ? 2 : (t == SR_BOOL_W32 || t == SR_U32) ? 4 : 8; }
// row width in the dtype's own units (entries or words) for a row of n entries
static int64_t row_units(sr_dtype t, int64_t n)
{
    if (t == SR_BOOL_W32) return (n + 31) / 32;
    if (t == SR_BOOL_W64) return (n + 63) / 64;
    return n;
}
static int u32_per_unit(sr_dtype t) { return t == SR_BOOL_W64 ? 2 : 1; }

sr_status check_dim(const char *fn, const char *name, int64_t v)
{
    if (v <= 0 || v > 0x7fffffffLL)
        return fail(SR_EINVAL, "%s: %s = %lld must be in [1, 2^31)", fn, name, (long long)v);
    return SR_OK;
}

sr_status check_mat(const char *fn, const char *name, const void *p, int64_t ld, int64_t rows, int64_t cols,
                    sr_dtype t)
{
    if (!p)
        return fail(SR_EINVAL, "%s: %s is NULL", fn, name);
    const int64_t w = row_units(t, cols);
    if (ld < w)
        return fail(SR_EINVAL, "%s: ld of %s (%lld) is below its row width (%lld)", fn, name, (long long)ld,
                    (long long)w);
    if (ld > (int64_t)1 << 40 || rows * ld > ((int64_t)1 << 46))
        return fail(SR_EINVAL, "%s: %s is too large", fn, name);
    return SR_OK;
}

struct Range {
    uintptr_t lo, hi;
};
static Range span(const void *p, int64_t ld, int64_t rows, int64_t cols, sr_dtype t)
{
    const uintptr_t b = reinterpret_cast<uintptr_t>(p);
    return {b, b + (uintptr_t)(((rows - 1) * ld + row_units(t, cols)) * esize(t))};
}
static bool overlap(Range a, Range b) { return a.lo < b.hi && b.lo < a.hi; }

static bool vec_ok(sr_dtype t, std::initializer_list<std::pair<const void *, int64_t>> mats)
{
    for (auto &m : mats)
        if (!aligned16(m.first) || ((m.second * esize(t)) & 15) != 0)
            return false;
    return true;
}

static cudaStream_t S(void *stream) { return reinterpret_cast<cudaStream_t>(stream); }

void __attribute__((weak)) sr_ctx_shutdown(sr_ctx *) {}

}  // namespace sr

using namespace sr;

// ======================================================================= API
extern "C" {

const char *sr_last_error(void) { return g_err.c_str(); }

sr_status sr_host_mapped(const void *p, int *mapped)
{
    SR_TRACE("sr_host_mapped");
    if (!mapped)
        return fail(SR_EINVAL, "sr_host_mapped: mapped is NULL");
    *mapped = 0;
    if (!p)
        return SR_OK;
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();                 // unregistered host memory: not mapped
        return SR_OK;
    }
    *mapped = a.type == cudaMemoryTypeHost && a.devicePointer == p ? 1 : 0;
    return SR_OK;
}

sr_status sr_shard_rows(int64_t R, int world, int rank, int64_t align, int64_t *r0, int64_t *r1)
{
    if (!r0 || !r1 || R < 0 || world < 1 || rank < 0 || rank >= world || align < 1)
        return fail(SR_EINVAL, "sr_shard_rows: need R >= 0, 0 <= rank < world, align >= 1 and outputs");
    // whole groups of `align` rows, as evenly as possible; the first R mod world groups get one more
    const int64_t groups = (R + align - 1) / align, q = groups / world, rem = groups % world;
    const int64_t g0 = rank * q + std::min<int64_t>(rank, rem), g1 = g0 + q + (rank < rem ? 1 : 0);
    *r0 = std::min(R, g0 * align);
    *r1 = std::min(R, g1 * align);
    return SR_OK;
}

long long sr_closure_order(int64_t D, int share, int *out, long long cap)
{
    return antidist_closure_persistent_order(D, share, out, cap);
}

const char *sr_version(void) { return "semiring-gb300 0.1 (sm_103a)"; }

uint64_t sr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

sr_status sr_create(sr_ctx **out, const sr_config *cfg)
{
    if (!out)
        return fail(SR_EINVAL, "sr_create: out is NULL");
    *out = nullptr;
    sr_ctx *c = new (std::nothrow) sr_ctx();
    if (!c)
        return fail(SR_ENOMEM, "sr_create: host allocation failed");
    c->device = current_device();
    if (c->device < 0) {
        delete c;
        return fail(SR_ECUDA, "sr_create: no current CUDA device with an id below %d", kMaxDevices);
    }
    if (cfg) {
        c->ws_bytes = cfg->workspace_bytes;
        c->spin_limit = cfg->spin_limit > 0 ? cfg->spin_limit : kDefaultSpinLimit;
        const sr_status ts = tune_load_config(c, cfg->tune_cache);
        if (ts != SR_OK) {
            delete c;
            return ts;
        }
    }
    cudaError_t e = cudaMalloc(&c->d_status, sizeof(int) * 4);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "sr_create: cudaMalloc(status)");
    }
    e = cudaMemset(c->d_status, 0, sizeof(int) * 4);
    if (e == cudaSuccess && c->ws_bytes) {
        e = cudaMalloc(&c->ws, c->ws_bytes);
        if (e != cudaSuccess) {
            cudaFree(c->d_status);
            delete c;
            return fail(SR_ENOMEM, "sr_create: cannot allocate %zu workspace bytes (%s)", cfg->workspace_bytes,
                        cudaGetErrorString(e));
        }
    }
    if (e != cudaSuccess) {
        cudaFree(c->d_status);
        delete c;
        return cuda_fail(e, "sr_create");
    }
    *out = c;
    return SR_OK;
}

void sr_destroy(sr_ctx *c)
{
    if (!c)
        return;
    sr_ctx_shutdown(c);
    if (c->ws) cudaFree(c->ws);
    if (c->d_status) cudaFree(c->d_status);
    delete c;
}

sr_status sr_set_option(sr_ctx *c, int option, int value)
{
    if (!c)
        return fail(SR_EINVAL, "sr_set_option: ctx is NULL");
    if (option == SR_OPT_BOOL_TENSOR && value >= 0 && value <= 2) {
        c->bool_tc_mode = value;
        return SR_OK;
    }
    if (option == SR_OPT_BOOL_FOUR_RUSSIANS && value >= 0 && value <= 2) {
        c->bool_m4r_mode = value;
        return SR_OK;
    }
    if (option == SR_OPT_SPIN_LIMIT && value >= 0) {
        c->spin_limit = value;
        return SR_OK;
    }
    if (option == SR_OPT_CLOSURE_BLOCK && (value == 0 || value == 128 || value == 256 || value == 512)) {
        c->closure_width = value;
        return SR_OK;
    }
    if (option == SR_OPT_CLOSURE_PERSISTENT && value >= 0 && value <= 2) {
        c->closure_persistent = value;
        return SR_OK;
    }
    if (option == SR_OPT_CLOSURE_PANEL_SHARE && value >= 0 && value <= 256) {
        c->closure_share = value;
        return SR_OK;
    }
    if (option == SR_OPT_BOOL_SIDE_SMS && value >= -1 && value <= 1024) {
        c->bool_side_sms = value;
        return SR_OK;
    }
    if (option == SR_OPT_CLOSURE_FUSED && value >= 0 && value <= 2) {
        c->closure_fused = value;
        return SR_OK;
    }
    if (option == SR_OPT_PRODUCT_SPLIT && (value == 0 || value == 1)) {
        c->product_split = value;
        return SR_OK;
    }
    return fail(SR_EINVAL, "sr_set_option: unknown option %d or value %d", option, value);
}

sr_status sr_workspace_query(int op, sr_dtype dtype, int64_t D, int method, size_t *bytes)
{
    if (!bytes)
        return fail(SR_EINVAL, "sr_workspace_query: bytes is NULL");
    *bytes = 0;
    SR_TRY(check_dim("sr_workspace_query", "D", D));
    if (op == SR_OP_BOOL_CLOSURE && is_bool(dtype) && method == SR_CLOSURE_WARSHALL && D > kBoolWideBlock)
        *bytes = bool_closure_wide_workspace(D);                           // tensor-core phase 3
    if (op == SR_OP_BOOL_CLOSURE && is_bool(dtype) && method == SR_CLOSURE_SQUARING) {
        *bytes = bool_squaring_workspace(D, row_units(dtype, D) * u32_per_unit(dtype));   // squares + operands
    }
    if (op == SR_OP_BOOL_MUL && is_bool(dtype))
        *bytes = bool_tc_workspace(D, D, D);
    if (op == SR_OP_ANTIDIST_CLOSURE && (dtype == SR_U8 || dtype == SR_U16))   // persistent / fused-pass schedules
        *bytes = std::max(antidist_closure_persistent_workspace(D), closure_fused_workspace(D));
    if (op == SR_OP_DIST_MUL && is_anti(dtype))
        *bytes = (size_t)(2 * D * ((D + 15) / 16 * 16) * esize(dtype) + 1024);
    return SR_OK;
}

sr_status sr_stream_status(sr_ctx *c, void *stream)
{
    SR_TRACE("sr_stream_status");
    if (!c)
        return fail(SR_EINVAL, "sr_stream_status: ctx is NULL");
    SR_CUDA_CHECK(cudaStreamSynchronize(S(stream)));
    int h[4] = {0, 0, 0, 0};
    SR_CUDA_CHECK(cudaMemcpy(h, c->d_status, sizeof h, cudaMemcpyDeviceToHost));
    SR_CUDA_CHECK(cudaMemset(c->d_status, 0, sizeof h));
    if (h[0])
        return fail(SR_ETIMEOUT, "a bounded device-side wait gave up (code %d, where %d)", h[0], h[1]);
    return SR_OK;
}

// ------------------------------------------------------------------ encoding
sr_status antidist_encode(sr_ctx *, const void *W, int64_t ldw, void *T, int64_t ldt, int64_t R, int64_t C,
                          sr_dtype dtype, void *stream)
{
    SR_TRACE("antidist_encode");
    const char *fn = "antidist_encode";
    if (!is_anti(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "C", C));
    SR_TRY(check_mat(fn, "W", W, ldw, R, C, dtype));
    SR_TRY(check_mat(fn, "T", T, ldt, R, C, dtype));
    return launch_antidist_encode(W, ldw, T, ldt, (int)R, (int)C, dtype, device_sm_count(), S(stream));
}

sr_status bool_pack(sr_ctx *, const uint8_t *dense, int64_t ldd, void *M, int64_t ldm, int64_t R, int64_t C,
                    sr_dtype dtype, void *stream)
{
    SR_TRACE("bool_pack");
    const char *fn = "bool_pack";
    if (!is_bool(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_BOOL_W32 or SR_BOOL_W64", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "C", C));
    SR_TRY(check_mat(fn, "dense", dense, ldd, R, C, SR_U8));
    SR_TRY(check_mat(fn, "M", M, ldm, R, C, dtype));
    const int rw = (int)(row_units(dtype, C) * u32_per_unit(dtype));
    return launch_bool_pack(dense, ldd, static_cast<uint32_t *>(M), ldm * u32_per_unit(dtype), (int)R, (int)C, rw,
                            device_sm_count(), S(stream));
}

sr_status bool_unpack(sr_ctx *, const void *M, int64_t ldm, uint8_t *dense, int64_t ldd, int64_t R, int64_t C,
                      sr_dtype dtype, void *stream)
{
    SR_TRACE("bool_unpack");
    const char *fn = "bool_unpack";
    if (!is_bool(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_BOOL_W32 or SR_BOOL_W64", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "C", C));
    SR_TRY(check_mat(fn, "M", M, ldm, R, C, dtype));
    SR_TRY(check_mat(fn, "dense", dense, ldd, R, C, SR_U8));
    return launch_bool_unpack(static_cast<const uint32_t *>(M), ldm * u32_per_unit(dtype), dense, ldd, (int)R,
                              (int)C, device_sm_count(), S(stream));
}

// ------------------------------------------------------------------ products
sr_status antidist_mul(sr_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                       int64_t R, int64_t K, int64_t N, sr_dtype dtype, int accumulate, void *stream)
{
    SR_TRACE("antidist_mul");
    const char *fn = "antidist_mul";
    if (!is_anti(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "K", K));
    SR_TRY(check_dim(fn, "N", N));
    SR_TRY(check_mat(fn, "A", A, lda, R, K, dtype));
    SR_TRY(check_mat(fn, "B", B, ldb, K, N, dtype));
    SR_TRY(check_mat(fn, "C", C, ldc, R, N, dtype));
    const Range rc = span(C, ldc, R, N, dtype);
    if (overlap(rc, span(A, lda, R, K, dtype)) || overlap(rc, span(B, ldb, K, N, dtype)))
        return fail(SR_EINVAL, "%s: C overlaps A or B (use antidist_closure for the in-place form)", fn);
    MulArgs a;
    a.A = A; a.B = B; a.C = C;
    a.lda = lda; a.ldb = ldb; a.ldc = ldc;
    a.R = (int)R; a.K = (int)K; a.N = (int)N;
    a.accumulate = accumulate ? 1 : 0;
    a.rskip0 = a.cskip0 = 0x7fffffff;
    a.rskipw = a.cskipw = 0;
    a.skip_tile = -1;
    a.split = ctx ? ctx->product_split : 1;
    const bool vec = vec_ok(dtype, {{A, lda}, {B, ldb}, {C, ldc}});
    int tile = 128;     // the autotuner's tile side for this size, if it recorded one
    tune_lookup(ctx, tune_key("antidist_mul", dtype, std::max(R, std::max(K, N))), &tile);
    return launch_antidist_mul(a, dtype, vec, S(stream), tile == 64 ? 1 : 0);
}

// tensor-core path when the context allows it and has the workspace
static bool use_tc(const sr_ctx *c, int64_t R, int64_t K, int64_t N, size_t ws_avail)
{
    if (!c || c->bool_tc_mode == 0 || R < 1 || (c->bool_tc_mode == 1 && K < 1024)) return false;
    return bool_tc_workspace(R, K, N) <= ws_avail && bool_tc_available();
}

// Warshall closure with wide blocks and phase 3 on the tensor cores: from D = 4096 by
// default (GB300: 0.83 / 1.37 / 2.00 ms at D = 4096 / 6144 / 8192 against 0.86 / 1.72 /
// 3.07 ms for the 128-bit word schedule), whenever there are two blocks or more with
// SR_OPT_BOOL_TENSOR = 2.
constexpr int64_t kBoolWideMinD = 4096;
static bool use_tc_closure(const sr_ctx *c, int64_t D)
{
    if (!c || c->bool_tc_mode == 0 || D <= kBoolWideBlock || (c->bool_tc_mode == 1 && D < kBoolWideMinD))
        return false;
    return bool_closure_wide_workspace(D) <= c->ws_bytes && bool_tc_available();
}

// Four Russians tables pay off when its 256-row × 32-word CTAs fill the GPU about
// 1.5 times over and K spans many 8-bit groups (GB300: 1.3x the masked-OR kernel at
// 8192^3, 0.64x at 4096^3, where only 64 CTAs exist); smaller products keep the
// masked-OR kernel (with split K).
static bool use_m4r(const sr_ctx *c, int64_t R, int64_t K, int64_t ncw)
{
    const int mode = c ? c->bool_m4r_mode : 1;
    if (mode == 0) return false;
    if (mode == 2) return true;
    const int64_t ctas = ((R + 255) / 256) * ((ncw + 31) / 32);
    return K >= 1024 && 2 * ctas >= 3 * (int64_t)device_sm_count();
}

static sr_status bool_mul_impl(const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                               int64_t R, int64_t K, int64_t N, sr_dtype dtype, int accumulate, cudaStream_t s,
                               sr_ctx *ctx = nullptr, void *ws = nullptr, size_t ws_bytes = 0)
{
    const int u = u32_per_unit(dtype);
    BoolArgs a;
    a.A = static_cast<const uint32_t *>(A);
    a.B = static_cast<const uint32_t *>(B);
    a.C = static_cast<uint32_t *>(C);
    a.lda = lda * u; a.ldb = ldb * u; a.ldc = ldc * u;
    a.R = (int)R; a.K = (int)K; a.N = (int)N;
    a.ncw = (int)(row_units(dtype, N) * u);
    a.accumulate = accumulate ? 1 : 0;
    a.skip0 = 0x7fffffff; a.skipw = 0;
    a.skip0w = 0x7fffffff; a.skipww = 0;
    const bool vec = vec_ok(dtype, {{A, lda}, {B, ldb}, {C, ldc}});
    int tuned = 0;      // a recorded choice applies while both path options are automatic
    if (ctx && ctx->bool_tc_mode == 1 && ctx->bool_m4r_mode == 1 &&
        tune_lookup(ctx, tune_key("bool_mul", dtype, std::max(R, std::max(K, N))), &tuned)) {
        if (tuned == SR_TUNE_BOOL_TENSOR && ws && bool_tc_workspace(R, K, N) <= ws_bytes && bool_tc_available())
            return launch_bool_mul_tc(a, ws, ws_bytes, ctx->d_status, ctx->spin_limit, s);
        if (tuned == SR_TUNE_BOOL_TABLES)
            return launch_bool_mul_m4r(a, s);
        if (tuned == SR_TUNE_BOOL_WORDS)
            return launch_bool_mul(a, vec, s);
    }
    if (use_tc(ctx, R, K, N, ws_bytes))
        return launch_bool_mul_tc(a, ws, ws_bytes, ctx->d_status, ctx->spin_limit, s);
    if (use_m4r(ctx, R, K, a.ncw))
        return launch_bool_mul_m4r(a, s);
    return launch_bool_mul(a, vec, s);
}

sr_status bool_mul(sr_ctx *ctx, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                   int64_t R, int64_t K, int64_t N, sr_dtype dtype, int accumulate, void *stream)
{
    SR_TRACE("bool_mul");
    const char *fn = "bool_mul";
    if (!is_bool(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_BOOL_W32 or SR_BOOL_W64", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "K", K));
    SR_TRY(check_dim(fn, "N", N));
    SR_TRY(check_mat(fn, "A", A, lda, R, K, dtype));
    SR_TRY(check_mat(fn, "B", B, ldb, K, N, dtype));
    SR_TRY(check_mat(fn, "C", C, ldc, R, N, dtype));
    const Range rc = span(C, ldc, R, N, dtype);
    if (overlap(rc, span(A, lda, R, K, dtype)) || overlap(rc, span(B, ldb, K, N, dtype)))
        return fail(SR_EINVAL, "%s: C overlaps A or B (use bool_closure for the in-place form)", fn);
    sr_ctx *c = ctx;
    return bool_mul_impl(A, lda, B, ldb, C, ldc, R, K, N, dtype, accumulate, S(stream), c, c ? c->ws : nullptr,
                         c ? c->ws_bytes : 0);
}

// ------------------------------------------------------------------ closures
// D from which the persistent schedule is the automatic choice (u8, u16)
static int64_t persistent_min_d(sr_dtype t) { return t == SR_U8 ? kPersistentAutoMinU8 : kPersistentAutoMinU16; }

// The anti-distance closure of T in place: the persistent schedule where the context
// allows it and holds its workspace, the stream schedules of closure.cu otherwise.
// the fused-pass schedule, if this call can take it
static bool fused_ok(const sr_ctx *c, int64_t D, sr_dtype dtype, bool vec)
{
    const size_t need = closure_fused_workspace(D);
    return c && vec && (dtype == SR_U8 || dtype == SR_U16) && need > 0 && c->ws && c->ws_bytes >= need;
}

// D from which the fused-pass schedule is the automatic choice (u8, u16)
static bool fused_auto(sr_dtype dtype, int64_t D)
{
    (void)dtype;
    (void)D;
    return false;
}

static sr_status closure_dispatch(sr_ctx *c, void *T, int64_t ldt, int64_t D, sr_dtype dtype, bool vec,
                                  cudaStream_t s)
{
    int tuned = 0;      // a recorded choice applies while the options are automatic
    if (c && c->closure_width == 0 && c->closure_persistent == 1 && c->closure_fused == 1 &&
        tune_lookup(c, tune_key("closure", dtype, D), &tuned)) {
        if (tuned == SR_TUNE_FUSED) {
            if (fused_ok(c, D, dtype, vec))
                return launch_antidist_closure_fused(T, ldt, (int)D, dtype, c->ws, c->ws_bytes, c->d_status,
                                                     c->spin_limit, s);
            return launch_antidist_closure(T, ldt, (int)D, dtype, vec, s, 0);
        }
        if (tuned != SR_TUNE_PERSISTENT)
            return launch_antidist_closure(T, ldt, (int)D, dtype, vec, s, tuned);
        const size_t need = antidist_closure_persistent_workspace(D);
        if (vec && (dtype == SR_U8 || dtype == SR_U16) && need > 0 && c->ws && c->ws_bytes >= need)
            return launch_antidist_closure_persistent(T, ldt, (int)D, dtype, c->ws, c->ws_bytes, c->d_status,
                                                      c->spin_limit, c->closure_share, s);
        return launch_antidist_closure(T, ldt, (int)D, dtype, vec, s, 0);
    }
    if (c && c->closure_width == 0 && c->closure_fused > 0 && (c->closure_fused == 2 || fused_auto(dtype, D)) &&
        fused_ok(c, D, dtype, vec))
        return launch_antidist_closure_fused(T, ldt, (int)D, dtype, c->ws, c->ws_bytes, c->d_status, c->spin_limit, s);
    if (c && vec && c->closure_width == 0 && c->closure_persistent > 0 && (dtype == SR_U8 || dtype == SR_U16) &&
        (c->closure_persistent == 2 || D >= persistent_min_d(dtype))) {
        const size_t need = antidist_closure_persistent_workspace(D);
        if (need > 0 && c->ws && c->ws_bytes >= need)
            return launch_antidist_closure_persistent(T, ldt, (int)D, dtype, c->ws, c->ws_bytes, c->d_status,
                                                      c->spin_limit, c->closure_share, s);
    }
    return launch_antidist_closure(T, ldt, (int)D, dtype, vec, s, c ? c->closure_width : 0);
}

sr_status antidist_closure(sr_ctx *c, void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream)
{
    SR_TRACE("antidist_closure");
    const char *fn = "antidist_closure";
    if (!is_anti(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "D", D));
    SR_TRY(check_mat(fn, "T", T, ldt, D, D, dtype));
    const bool vec = vec_ok(dtype, {{T, ldt}});
    return closure_dispatch(c, T, ldt, D, dtype, vec, S(stream));
}

sr_status bool_closure(sr_ctx *c, void *T, int64_t ldt, int64_t D, sr_dtype dtype, int method, void *stream)
{
    SR_TRACE("bool_closure");
    const char *fn = "bool_closure";
    if (!is_bool(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_BOOL_W32 or SR_BOOL_W64", fn);
    SR_TRY(check_dim(fn, "D", D));
    SR_TRY(check_mat(fn, "T", T, ldt, D, D, dtype));
    const int u = u32_per_unit(dtype);
    const int rw = (int)(row_units(dtype, D) * u);
    const bool vec = vec_ok(dtype, {{T, ldt}});
    uint32_t *T32 = static_cast<uint32_t *>(T);
    if (method == SR_CLOSURE_WARSHALL) {
        if (use_tc_closure(c, D))
            return launch_bool_closure_wide(T32, ldt * u, (int)D, rw, c->ws, c->ws_bytes, c->d_status,
                                            c->spin_limit, S(stream), c->bool_side_sms);
        return launch_bool_closure_warshall(T32, ldt * u, (int)D, rw, vec, S(stream));
    }
    if (method != SR_CLOSURE_SQUARING)
        return fail(SR_EINVAL, "%s: unknown method %d", fn, method);
    if (!c)
        return fail(SR_EINVAL, "%s: the squaring method needs a context with workspace", fn);
    const bool tc = c->bool_tc_mode != 0 && (c->bool_tc_mode == 2 || D >= 1024) && bool_tc_available();
    return launch_bool_closure_squaring(T32, ldt * u, (int)D, rw, c->ws, c->ws_bytes, tc, c->d_status, c->spin_limit,
                                        S(stream));
}

// ------------------------------------------------------------------ distance form
sr_status dist_mul(sr_ctx *c, const void *A, int64_t lda, const void *B, int64_t ldb, void *C, int64_t ldc,
                   int64_t R, int64_t K, int64_t N, sr_dtype dtype, int accumulate, void *stream)
{
    SR_TRACE("dist_mul");
    const char *fn = "dist_mul";
    if (!is_anti(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "K", K));
    SR_TRY(check_dim(fn, "N", N));
    SR_TRY(check_mat(fn, "A", A, lda, R, K, dtype));
    SR_TRY(check_mat(fn, "B", B, ldb, K, N, dtype));
    SR_TRY(check_mat(fn, "C", C, ldc, R, N, dtype));
    const Range rc = span(C, ldc, R, N, dtype);
    if (overlap(rc, span(A, lda, R, K, dtype)) || overlap(rc, span(B, ldb, K, N, dtype)))
        return fail(SR_EINVAL, "%s: C overlaps A or B", fn);
    const int es = esize(dtype);
    const int64_t ka = (K + 15) / 16 * 16, na = (N + 15) / 16 * 16;   // 16-byte aligned rows
    const size_t need = (size_t)((R * ka + K * na) * es) + 512;
    if (!c || !c->ws || c->ws_bytes < need)
        return fail(SR_ENOMEM, "%s: needs a context with %zu workspace bytes", fn, need);
    cudaStream_t s = S(stream);
    char *Ac = static_cast<char *>(c->ws);
    char *Bc = Ac + ((R * ka * es + 255) / 256) * 256;
    // De Morgan (Section 4): A ∧+ B = S − ((S − A) ⊗ (S − B)), and C ∧ X = S − ((S − C) ⊕ (S − X))
    SR_TRY(launch_entrywise(SR_EW_NOT, A, lda, nullptr, 0, Ac, ka, (int)R, (int)K, dtype, s));
    SR_TRY(launch_entrywise(SR_EW_NOT, B, ldb, nullptr, 0, Bc, na, (int)K, (int)N, dtype, s));
    if (accumulate)
        SR_TRY(launch_entrywise(SR_EW_NOT, C, ldc, nullptr, 0, C, ldc, (int)R, (int)N, dtype, s));
    MulArgs a;
    a.A = Ac; a.B = Bc; a.C = C;
    a.lda = ka; a.ldb = na; a.ldc = ldc;
    a.R = (int)R; a.K = (int)K; a.N = (int)N;
    a.accumulate = accumulate ? 1 : 0;
    a.rskip0 = a.cskip0 = 0x7fffffff;
    a.rskipw = a.cskipw = 0;
    a.skip_tile = -1;
    SR_TRY(launch_antidist_mul(a, dtype, vec_ok(dtype, {{Ac, ka}, {Bc, na}, {C, ldc}}), s));
    return launch_entrywise(SR_EW_NOT, C, ldc, nullptr, 0, C, ldc, (int)R, (int)N, dtype, s);
}

sr_status dist_closure(sr_ctx *c, void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream)
{
    SR_TRACE("dist_closure");
    const char *fn = "dist_closure";
    if (!is_anti(dtype))
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "D", D));
    SR_TRY(check_mat(fn, "T", T, ldt, D, D, dtype));
    cudaStream_t s = S(stream);
    // the anti-distance closure of S − T, complemented back (Section 4, De Morgan)
    SR_TRY(launch_entrywise(SR_EW_NOT, T, ldt, nullptr, 0, T, ldt, (int)D, (int)D, dtype, s));
    SR_TRY(closure_dispatch(c, T, ldt, D, dtype, vec_ok(dtype, {{T, ldt}}), s));
    return launch_entrywise(SR_EW_NOT, T, ldt, nullptr, 0, T, ldt, (int)D, (int)D, dtype, s);
}

// ------------------------------------------------------------------ entrywise
sr_status sr_entrywise(sr_ctx *, int op, const void *A, int64_t lda, const void *B, int64_t ldb, void *C,
                       int64_t ldc, int64_t R, int64_t N, sr_dtype dtype, void *stream)
{
    SR_TRACE("sr_entrywise");
    const char *fn = "sr_entrywise";
    if (op < SR_EW_AND || op > SR_EW_NOT)
        return fail(SR_EINVAL, "%s: unknown op %d", fn, op);
    if (!is_anti(dtype) && !is_bool(dtype))
        return fail(SR_EINVAL, "%s: unknown dtype", fn);
    SR_TRY(check_dim(fn, "R", R));
    SR_TRY(check_dim(fn, "N", N));
    SR_TRY(check_mat(fn, "A", A, lda, R, N, dtype));
    if (op != SR_EW_NOT)
        SR_TRY(check_mat(fn, "B", B, ldb, R, N, dtype));
    SR_TRY(check_mat(fn, "C", C, ldc, R, N, dtype));
    return launch_entrywise(op, A, lda, op == SR_EW_NOT ? nullptr : B, ldb, C, ldc, (int)R, (int)N, dtype, S(stream));
}

sr_status sr_reflexive(sr_ctx *, void *T, int64_t ldt, int64_t D, sr_dtype dtype, void *stream)
{
    SR_TRACE("sr_reflexive");
    const char *fn = "sr_reflexive";
    if (!is_anti(dtype) && !is_bool(dtype))
        return fail(SR_EINVAL, "%s: unknown dtype", fn);
    SR_TRY(check_dim(fn, "D", D));
    SR_TRY(check_mat(fn, "T", T, ldt, D, D, dtype));
    return launch_reflexive(T, ldt, (int)D, dtype, S(stream));
}

}  // extern "C"
