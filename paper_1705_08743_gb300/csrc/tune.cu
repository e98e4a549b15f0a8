// Autotuner for the single calls, and the on-disk cache of every tuning.
//
// The kernels' schedule choices depend on the matrix size and on the GPU:
//   closure        block width of the stream schedule (128, 256, 512) or the
//                  persistent schedule (anti-distance closure, Section 2 Warshall /
//                  Section 3 Floyd);
//   bool_mul       masked-OR words, Four Russians tables or the tensor cores (Boolean
//                  product, Section 2 formula; Section 4 names the Four Russians method);
//   antidist_mul   128x128 or 64x64 CTA tiles (anti-distance product, Section 3 ⊗).
// sr_autotune_closure / sr_autotune_mul time the candidates on a scratch matrix of the
// requested order and record the fastest per (op, dtype, D bucket) in the context; the
// single calls then use the recorded choice wherever the caller left the corresponding
// option automatic.  The batched closure's tunings (sr_batch_autotune) live beside them.
// A context created with sr_config.tune_cache loads that JSON file (if it exists and
// was written on a GPU of the same name and SM count) and rewrites it after each new
// tuning, so a later process reuses the choices without timing them again.
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <unistd.h>

#include "sr_common.cuh"
#include "sr_ctx.h"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {

// Size buckets: 256, 384, 512, 768, 1024, ... (powers of two and 1.5 times them); a size
// tunes for the smallest bucket at or above it.
int64_t tune_bucket(int64_t D)
{
    int64_t b = 256;
    while (b < D) b = (b & (b - 1)) == 0 ? b / 2 * 3 : b / 3 * 4;
    return b;
}

static const char *dtype_name(sr_dtype t)
{
    switch (t) {
    case SR_BOOL_W32: return "w32";
    case SR_BOOL_W64: return "w64";
    case SR_U8: return "u8";
    case SR_U16: return "u16";
    default: return "u32";
    }
}

std::string tune_key(const char *op, sr_dtype t, int64_t D)
{
    return std::string(op) + "/" + dtype_name(t) + "/" + std::to_string(tune_bucket(D));
}

bool tune_lookup(const sr_ctx *c, const std::string &key, int *choice)
{
    if (!c) return false;
    auto it = c->tuned.find(key);
    if (it == c->tuned.end()) return false;
    *choice = (int)it->second[0];
    return true;
}

static std::string device_name(int dev)
{
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
    std::string s = p.name;
    for (char &ch : s)
        if (ch == '"' || ch == '\\') ch = '_';
    return s;
}

// {"semiring_tune": 1, "device": "...", "sms": N, "entries": {"key": [a, b, c, ms], ...}}
static sr_status write_cache(const sr_ctx *c, const char *path)
{
    std::string tmp = std::string(path) + ".tmp" + std::to_string((long long)getpid());
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f)
        return fail(SR_EINVAL, "tune cache: cannot write %s (%s)", tmp.c_str(), strerror(errno));
    fprintf(f, "{\n  \"semiring_tune\": 1,\n  \"device\": \"%s\",\n  \"sms\": %d,\n  \"entries\": {",
            device_name(c->device).c_str(), device_sm_count());
    bool first = true;
    for (const auto &e : c->tuned) {
        fprintf(f, "%s\n    \"%s\": [%.0f, %.0f, %.0f, %.6g]", first ? "" : ",", e.first.c_str(), e.second[0],
                e.second[1], e.second[2], e.second[3]);
        first = false;
    }
    for (const auto &e : c->tune) {
        fprintf(f, "%s\n    \"batch/%s\": [%d, %d, %d, 0]", first ? "" : ",", e.first.c_str(), e.second[0],
                e.second[1], e.second[2]);
        first = false;
    }
    fprintf(f, "\n  }\n}\n");
    const bool ok = fflush(f) == 0;
    fclose(f);
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(SR_EINVAL, "tune cache: cannot replace %s", path);
    }
    return SR_OK;
}

// The reader accepts what write_cache writes (whitespace anywhere between tokens).
struct Scan {
    const char *p, *end;
    void ws() { while (p < end && (*p == ' ' || *p == '\n' || *p == '\r' || *p == '\t')) ++p; }
    bool lit(char ch) { ws(); if (p < end && *p == ch) { ++p; return true; } return false; }
    bool str(std::string &out)
    {
        ws();
        if (p >= end || *p != '"') return false;
        const char *q = ++p;
        while (p < end && *p != '"') ++p;
        if (p >= end) return false;
        out.assign(q, p - q);
        ++p;
        return true;
    }
    bool num(double &v)
    {
        ws();
        char *e = nullptr;
        v = strtod(p, &e);
        if (e == p || e > end) return false;
        p = e;
        return true;
    }
};

static sr_status read_cache(sr_ctx *c, const char *path, bool strict)
{
    FILE *f = fopen(path, "r");
    if (!f) {
        if (!strict) return SR_OK;                             // no cache yet (or not readable): start afresh
        return fail(SR_EINVAL, "tune cache: cannot read %s (%s)", path, strerror(errno));
    }
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
    fclose(f);
    Scan s{text.data(), text.data() + text.size()};
    std::string key, device;
    double version = 0, sms = 0;
    bool ok = s.lit('{');
    std::map<std::string, std::array<double, 4>> single;
    std::map<std::string, std::array<int, 3>> batch;
    while (ok && !s.lit('}')) {
        ok = s.str(key) && s.lit(':');
        if (!ok) break;
        if (key == "semiring_tune") ok = s.num(version);
        else if (key == "device") ok = s.str(device);
        else if (key == "sms") ok = s.num(sms);
        else if (key == "entries") {
            ok = s.lit('{');
            while (ok && !s.lit('}')) {
                std::string k;
                std::array<double, 4> v{};
                ok = s.str(k) && s.lit(':') && s.lit('[') && s.num(v[0]) && s.lit(',') && s.num(v[1]) && s.lit(',') &&
                     s.num(v[2]) && s.lit(',') && s.num(v[3]) && s.lit(']');
                if (!ok) break;
                if (k.compare(0, 6, "batch/") == 0)
                    batch[k.substr(6)] = {(int)v[0], (int)v[1], (int)v[2]};
                else
                    single[k] = v;
                s.lit(',');
            }
        } else {
            ok = false;
        }
        s.lit(',');
    }
    if (!ok || version != 1) {
        if (!strict) return SR_OK;                             // at sr_create: an unreadable cache is ignored
        return fail(SR_EINVAL, "tune cache: %s is not a tuning cache this library wrote", path);
    }
    if (device != device_name(c->device) || (int)sms != device_sm_count()) {
        if (strict)
            return fail(SR_EINVAL, "tune cache: %s was tuned on %s with %d SMs", path, device.c_str(), (int)sms);
        return SR_OK;                                          // another GPU's choices: start afresh
    }
    for (auto &e : single) c->tuned[e.first] = e.second;
    for (auto &e : batch) c->tune[e.first] = e.second;
    return SR_OK;
}

sr_status tune_load_config(sr_ctx *c, const char *path)
{
    c->tune_path = path ? path : "";
    return c->tune_path.empty() ? SR_OK : read_cache(c, path, false);
}

sr_status tune_persist(const sr_ctx *c)
{
    return c->tune_path.empty() ? SR_OK : write_cache(c, c->tune_path.c_str());
}

// Time `run` (one enqueue on s): one untimed run, then the best of `reps`; < 0 on failure
// (a launch error, or a bounded wait that gave up, reported in the status word).
template <class F>
static double time_candidate(sr_ctx *c, cudaStream_t s, int reps, F run)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return -1;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1; }
    double best = -1;
    bool ok = run() == SR_OK;
    for (int r = 0; ok && r < reps; ++r) {
        ok = cudaEventRecord(e0, s) == cudaSuccess && run() == SR_OK && cudaEventRecord(e1, s) == cudaSuccess &&
             cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0;
        if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && (best < 0 || ms < best)) best = ms;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) best = -1;
    int st[4] = {0, 0, 0, 0};
    if (cudaMemcpy(st, c->d_status, sizeof st, cudaMemcpyDeviceToHost) == cudaSuccess && st[0]) {
        cudaMemset(c->d_status, 0, sizeof st);
        best = -1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? best : -1;
}

}  // namespace sr

using namespace sr;

extern "C" {

sr_status sr_autotune_closure(sr_ctx *c, sr_dtype dtype, int64_t D, void *stream, int reps, int force, int *choice,
                              double *best_ms)
{
    SR_TRACE("sr_autotune_closure");
    const char *fn = "sr_autotune_closure";
    if (!c)
        return fail(SR_EINVAL, "%s: ctx is NULL", fn);
    if (dtype != SR_U8 && dtype != SR_U16 && dtype != SR_U32)
        return fail(SR_EINVAL, "%s: dtype must be SR_U8, SR_U16 or SR_U32", fn);
    SR_TRY(check_dim(fn, "D", D));
    if (D > 65536)
        return fail(SR_EINVAL, "%s: D = %lld: tuning matrices are limited to 65536", fn, (long long)D);
    const std::string key = tune_key("closure", dtype, D);
    auto have = c->tuned.find(key);
    if (!force && have != c->tuned.end()) {
        if (choice) *choice = (int)have->second[0];
        if (best_ms) *best_ms = have->second[3];
        return SR_OK;
    }
    const int64_t Dt = tune_bucket(D);                           // tune at the bucket's size
    const int es = dtype == SR_U8 ? 1 : dtype == SR_U16 ? 2 : 4;
    const int64_t ld = (Dt * es + 15) / 16 * 16 / es;
    void *T = nullptr;
    SR_CUDA_CHECK(cudaMalloc(&T, (size_t)(Dt * ld * es)));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // timing does not depend on the entries (no kernel skips work): any pattern will do
    cudaError_t e = cudaMemsetAsync(T, 0x5A, (size_t)(Dt * ld * es), s);
    std::vector<std::pair<int, double>> res;
    for (int w : {128, 256, 512}) {
        const double ms = e != cudaSuccess ? -1 : time_candidate(c, s, std::max(1, reps), [&] {
            return launch_antidist_closure(T, ld, (int)Dt, dtype, true, s, w);
        });
        if (ms >= 0) res.push_back({w, ms});
    }
    const size_t need = antidist_closure_persistent_workspace(Dt);
    if (e == cudaSuccess && (dtype == SR_U8 || dtype == SR_U16) && need > 0 && c->ws && c->ws_bytes >= need) {
        const double ms = time_candidate(c, s, std::max(1, reps), [&] {
            return launch_antidist_closure_persistent(T, ld, (int)Dt, dtype, c->ws, c->ws_bytes, c->d_status,
                                                      c->spin_limit, c->closure_share, s);
        });
        if (ms >= 0) res.push_back({SR_TUNE_PERSISTENT, ms});
    }
    const size_t need_f = closure_fused_workspace(Dt);
    if (e == cudaSuccess && (dtype == SR_U8 || dtype == SR_U16) && need_f > 0 && c->ws && c->ws_bytes >= need_f) {
        const double ms = time_candidate(c, s, std::max(1, reps), [&] {
            return launch_antidist_closure_fused(T, ld, (int)Dt, dtype, c->ws, c->ws_bytes, c->d_status,
                                                 c->spin_limit, s);
        });
        if (ms >= 0) res.push_back({SR_TUNE_FUSED, ms});
    }
    cudaFree(T);
    if (e != cudaSuccess) return cuda_fail(e, "sr_autotune_closure: fill");
    if (res.empty())
        return fail(SR_ECUDA, "%s: no candidate schedule ran", fn);
    const auto bestc = *std::min_element(res.begin(), res.end(), [](auto &x, auto &y) { return x.second < y.second; });
    c->tuned[key] = {(double)bestc.first, 0, 0, bestc.second};
    if (choice) *choice = bestc.first;
    if (best_ms) *best_ms = bestc.second;
    return tune_persist(c);
}

sr_status sr_autotune_mul(sr_ctx *c, int op, sr_dtype dtype, int64_t D, void *stream, int reps, int force,
                          int *choice, double *best_ms)
{
    SR_TRACE("sr_autotune_mul");
    const char *fn = "sr_autotune_mul";
    if (!c)
        return fail(SR_EINVAL, "%s: ctx is NULL", fn);
    const bool boolean = op == SR_OP_BOOL_MUL;
    if (boolean ? (dtype != SR_BOOL_W32 && dtype != SR_BOOL_W64)
                : (op != SR_OP_ANTIDIST_MUL || (dtype != SR_U8 && dtype != SR_U16 && dtype != SR_U32)))
        return fail(SR_EINVAL, "%s: op SR_OP_BOOL_MUL with a Boolean dtype or SR_OP_ANTIDIST_MUL with u8/u16/u32", fn);
    SR_TRY(check_dim(fn, "D", D));
    if (D > 65536)
        return fail(SR_EINVAL, "%s: D = %lld: tuning matrices are limited to 65536", fn, (long long)D);
    const std::string key = tune_key(boolean ? "bool_mul" : "antidist_mul", dtype, D);
    auto have = c->tuned.find(key);
    if (!force && have != c->tuned.end()) {
        if (choice) *choice = (int)have->second[0];
        if (best_ms) *best_ms = have->second[3];
        return SR_OK;
    }
    const int64_t Dt = tune_bucket(D);
    // rows of 16-byte multiples: Boolean rows of 32-bit words, anti-distance entries
    const int64_t rowb = boolean ? (Dt + 31) / 32 * 4 : Dt * (dtype == SR_U8 ? 1 : dtype == SR_U16 ? 2 : 4);
    const int64_t ldb = (rowb + 15) / 16 * 16;
    const size_t bytes = (size_t)(Dt * ldb);
    char *M = nullptr;
    SR_CUDA_CHECK(cudaMalloc(&M, 3 * bytes));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(M, 0x5A, 3 * bytes, s);
    std::vector<std::pair<int, double>> res;
    if (e == cudaSuccess && boolean) {
        BoolArgs a;
        a.A = reinterpret_cast<const uint32_t *>(M);
        a.B = reinterpret_cast<const uint32_t *>(M + bytes);
        a.C = reinterpret_cast<uint32_t *>(M + 2 * bytes);
        a.lda = a.ldb = a.ldc = ldb / 4;
        a.R = a.K = a.N = (int)Dt;
        a.ncw = (int)((Dt + 31) / 32);
        a.accumulate = 0;
        a.skip0 = 0x7fffffff; a.skipw = 0;
        a.skip0w = 0x7fffffff; a.skipww = 0;
        double ms = time_candidate(c, s, std::max(1, reps), [&] { return launch_bool_mul(a, true, s); });
        if (ms >= 0) res.push_back({SR_TUNE_BOOL_WORDS, ms});
        ms = time_candidate(c, s, std::max(1, reps), [&] { return launch_bool_mul_m4r(a, s); });
        if (ms >= 0) res.push_back({SR_TUNE_BOOL_TABLES, ms});
        if (bool_tc_available() && c->ws && bool_tc_workspace(Dt, Dt, Dt) <= c->ws_bytes) {
            ms = time_candidate(c, s, std::max(1, reps), [&] {
                return launch_bool_mul_tc(a, c->ws, c->ws_bytes, c->d_status, c->spin_limit, s);
            });
            if (ms >= 0) res.push_back({SR_TUNE_BOOL_TENSOR, ms});
        }
    } else if (e == cudaSuccess) {
        MulArgs a;
        a.A = M; a.B = M + bytes; a.C = M + 2 * bytes;
        const int es = dtype == SR_U8 ? 1 : dtype == SR_U16 ? 2 : 4;
        a.lda = a.ldb = a.ldc = ldb / es;
        a.R = a.K = a.N = (int)Dt;
        a.accumulate = 0;
        a.rskip0 = a.cskip0 = 0x7fffffff;
        a.rskipw = a.cskipw = 0;
        for (int tile : {128, 64}) {
            const double ms = time_candidate(c, s, std::max(1, reps), [&] {
                return launch_antidist_mul(a, dtype, true, s, tile == 64 ? 1 : 0);
            });
            if (ms >= 0) res.push_back({tile, ms});
        }
    }
    cudaFree(M);
    if (e != cudaSuccess) return cuda_fail(e, "sr_autotune_mul: fill");
    if (res.empty())
        return fail(SR_ECUDA, "%s: no candidate ran", fn);
    const auto bestc = *std::min_element(res.begin(), res.end(), [](auto &x, auto &y) { return x.second < y.second; });
    c->tuned[key] = {(double)bestc.first, 0, 0, bestc.second};
    if (choice) *choice = bestc.first;
    if (best_ms) *best_ms = bestc.second;
    return tune_persist(c);
}

sr_status sr_tune_get(const sr_ctx *c, int op, sr_dtype dtype, int64_t D, int *choice, double *ms)
{
    SR_TRACE("sr_tune_get");
    if (!c || !choice)
        return fail(SR_EINVAL, "sr_tune_get: NULL ctx or output");
    const char *name = op == SR_OP_ANTIDIST_CLOSURE ? "closure" : op == SR_OP_BOOL_MUL ? "bool_mul"
                     : op == SR_OP_ANTIDIST_MUL ? "antidist_mul" : nullptr;
    if (!name || D <= 0)
        return fail(SR_EINVAL, "sr_tune_get: op %d or D %lld has no tuning", op, (long long)D);
    auto it = c->tuned.find(tune_key(name, dtype, D));
    if (it == c->tuned.end())
        return fail(SR_ENOTFOUND, "sr_tune_get: no tuning for %s", tune_key(name, dtype, D).c_str());
    *choice = (int)it->second[0];
    if (ms) *ms = it->second[3];
    return SR_OK;
}

sr_status sr_tune_set(sr_ctx *c, int op, sr_dtype dtype, int64_t D, int choice)
{
    SR_TRACE("sr_tune_set");
    if (!c)
        return fail(SR_EINVAL, "sr_tune_set: ctx is NULL");
    const bool anti = dtype == SR_U8 || dtype == SR_U16 || dtype == SR_U32;
    const bool boolean = dtype == SR_BOOL_W32 || dtype == SR_BOOL_W64;
    const bool ok = (op == SR_OP_ANTIDIST_CLOSURE && anti &&
                     (choice == 128 || choice == 256 || choice == 512 || choice == SR_TUNE_PERSISTENT ||
                      (choice == SR_TUNE_FUSED && dtype != SR_U32))) ||
                    (op == SR_OP_BOOL_MUL && boolean && choice >= SR_TUNE_BOOL_WORDS && choice <= SR_TUNE_BOOL_TENSOR) ||
                    (op == SR_OP_ANTIDIST_MUL && anti && (choice == 128 || choice == 64));
    if (!ok || D <= 0)
        return fail(SR_EINVAL, "sr_tune_set: op %d, dtype %d, choice %d or D %lld not valid", op, (int)dtype, choice,
                    (long long)D);
    const char *name = op == SR_OP_ANTIDIST_CLOSURE ? "closure" : op == SR_OP_BOOL_MUL ? "bool_mul" : "antidist_mul";
    c->tuned[tune_key(name, dtype, D)] = {(double)choice, 0, 0, 0};
    return tune_persist(c);
}

sr_status sr_tune_save(const sr_ctx *c, const char *path)
{
    SR_TRACE("sr_tune_save");
    if (!c || !path)
        return fail(SR_EINVAL, "sr_tune_save: NULL ctx or path");
    return write_cache(c, path);
}

sr_status sr_tune_load(sr_ctx *c, const char *path)
{
    SR_TRACE("sr_tune_load");
    if (!c || !path)
        return fail(SR_EINVAL, "sr_tune_load: NULL ctx or path");
    return read_cache(c, path, true);
}

}  // extern "C"
