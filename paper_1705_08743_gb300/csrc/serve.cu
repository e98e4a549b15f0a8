// Served request loop: continuous batching of closure and product requests.
//
// A scheduler thread owns the device side.  Requests (closures and products over
// Boolean, u8 and u16 matrices, any size) wait in a FIFO queue; whenever a stream
// slot and enough device memory are free, the scheduler admits the next requests:
// it carves their buffers out of one device arena, enqueues host->device copies,
// the kernels and device->host copies on the slot's stream, and a host callback
// that marks them done and returns their memory.  Requests that arrive while
// others are on the GPU are admitted as soon as a slot and memory free up, and the
// work of different slots overlaps on the device.  Small anti-distance closures of
// one dtype that are waiting together are admitted as one group and closed in one
// persistent batched launch.  Results may stay resident in the arena (a handle)
// and serve as inputs of later requests without another transfer.
//
// Host side only: the arena is host bookkeeping of offsets into one cudaMalloc
// made at sr_serve_start; completion callbacks make no CUDA calls.  No device code
// waits on anything.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sr_common.cuh"
#include "sr_ctx.h"
#include "sr_kernels.h"
#include "sr_trace.h"

namespace sr {

static double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------------ arena
// First-fit allocator over [0, size) with 256-byte granularity.
class Arena {
  public:
    void reset(size_t size)
    {
        size_ = size;
        free_.clear();
        if (size) free_[0] = size;
        used_ = peak_ = 0;
    }
    bool alloc(size_t n, size_t *off)
    {
        n = (n + 255) / 256 * 256;
        if (n == 0) n = 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const size_t rest = it->second - n, start = it->first + n;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += n;
                peak_ = std::max(peak_, used_);
                sizes_[*off] = n;
                return true;
            }
        }
        return false;
    }
    void release(size_t off)
    {
        auto s = sizes_.find(off);
        if (s == sizes_.end()) return;
        size_t n = s->second;
        sizes_.erase(s);
        used_ -= n;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + n == nx->first) {   // merge with the next free block
            n += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                          // merge with the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += n;
                return;
            }
        }
        free_[off] = n;
    }
    // would n bytes fit after the given extra allocations? (admission check without committing)
    size_t largest_free() const
    {
        size_t m = 0;
        for (auto &f : free_) m = std::max(m, f.second);
        return m;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t peak() const { return peak_; }

  private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
    std::unordered_map<size_t, size_t> sizes_;
};

// ------------------------------------------------------------------ requests
struct Resident {
    size_t off = 0;
    int64_t rows = 0, cols = 0, ld = 0;   // ld in units (entries / words of the dtype)
    sr_dtype dtype = SR_U8;
    size_t bytes = 0;
};

struct Req {
    uint64_t id = 0;
    sr_request r{};
    int status = SR_OK;
    std::string err;
    bool done = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    std::vector<size_t> blocks;            // arena offsets to free at completion
    size_t out_off = 0;                    // result buffer
    int64_t out_ld = 0;
    uint64_t resident = 0;                 // handle of the kept result
};

struct Slot {
    cudaStream_t stream = nullptr;
    bool busy = false;
    bool long_job = false;                 // holds the one long request allowed in flight
    // batched-group staging
    BatchGraph *d_graphs = nullptr;
    BatchItem *d_items = nullptr;
    int *d_counter = nullptr;
    BatchGraph *h_graphs = nullptr;        // pinned
    BatchItem *h_items = nullptr;          // pinned
};

struct ServeState;
struct Completion {
    ServeState *st;
    int slot;
    std::vector<uint64_t> ids;
};

struct ServeState {
    sr_serve_config cfg{};
    int device = 0;
    char *base = nullptr;                  // arena device memory
    Arena arena;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::unordered_map<uint64_t, Resident> residents;
    uint64_t next_id = 1, next_res = 1;
    bool stop = false;
    std::thread th;
    // stats
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, batched_reqs = 0, cancelled = 0;
    int inflight = 0;
    int long_inflight = 0;
};

// Requests expected to keep the GPU busy for a millisecond or more run one at a time:
// two of them sharing the device would each take about twice as long, which is what
// the tail latency is made of; short requests still fill the other slots around them.
// The estimate is the operation count over the kernels' measured rates on GB300.
static bool is_long(const sr_request &r)
{
    const sr_dtype t = (sr_dtype)r.dtype;
    const bool closure = r.op == SR_OP_ANTIDIST_CLOSURE || r.op == SR_OP_BOOL_CLOSURE;
    const double ops = closure ? (double)r.R * r.R * r.R : (double)r.R * r.K * r.N;
    const double rate = t == SR_U8 ? 3.0e13 : t == SR_U16 ? 1.5e13 : t == SR_U32 ? 8.0e12 : 4.0e14;   // ops/s
    return ops / rate >= 1.0e-3;
}

static int es_of(sr_dtype t) { return t == SR_U8 ? 1 : t == SR_U16 ? 2 : (t == SR_BOOL_W32 || t == SR_U32) ? 4 : 8; }
static int64_t units_of(sr_dtype t, int64_t n)
{
    return t == SR_BOOL_W32 ? (n + 31) / 32 : t == SR_BOOL_W64 ? (n + 63) / 64 : n;
}
static int64_t pad_units(sr_dtype t, int64_t u) { const int per = 16 / es_of(t); return (u + per - 1) / per * per; }
// workspace of a word-path squaring closure: its flags and the two squares (no tensor-core operands)
static size_t squaring_bytes(sr_dtype t, int64_t D)
{
    const int64_t rw = units_of(t, D) * (t == SR_BOOL_W64 ? 2 : 1);
    return bool_squaring_workspace(D, rw) - bool_tc_workspace(D, D, D);
}

// device bytes a request needs (buffers it allocates; resident inputs cost nothing)
static size_t request_bytes(const sr_request &r)
{
    const sr_dtype t = (sr_dtype)r.dtype;
    const int es = es_of(t);
    auto mat = [&](int64_t rows, int64_t cols) { return (size_t)(rows * pad_units(t, units_of(t, cols)) * es + 256); };
    size_t n = 0;
    if (r.op == SR_OP_ANTIDIST_CLOSURE || r.op == SR_OP_BOOL_CLOSURE) {
        n += mat(r.R, r.R);
        if (r.op == SR_OP_BOOL_CLOSURE && r.method == SR_CLOSURE_SQUARING)
            n += squaring_bytes(t, r.R) + 256;
    } else {
        if (!r.rA) n += mat(r.R, r.K);
        if (!r.rB) n += mat(r.K, r.N);
        n += mat(r.R, r.N);
    }
    return n;
}

static void CUDART_CB on_complete(void *arg)
{
    std::unique_ptr<Completion> c(static_cast<Completion *>(arg));
    ServeState *st = c->st;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        const double t = now_ms();
        for (uint64_t id : c->ids) {
            auto it = st->reqs.find(id);
            if (it == st->reqs.end()) continue;
            Req &q = *it->second;
            for (size_t off : q.blocks) st->arena.release(off);
            q.blocks.clear();
            q.done = true;
            q.t_done = t;
            ++st->completed;
        }
        st->slots[c->slot].busy = false;
        if (st->slots[c->slot].long_job) {
            st->slots[c->slot].long_job = false;
            --st->long_inflight;
        }
        --st->inflight;
    }
    st->cv_sched.notify_one();
    st->cv_done.notify_all();
}

// A unit of admitted work: one request, or a group of small closures for one
// batched launch.  Built under the lock, enqueued without it.
struct Job {
    int slot = -1;
    bool group = false;
    std::vector<Req *> reqs;
    std::vector<std::vector<size_t>> offs;
    // resident inputs, resolved under the lock (device pointer, leading dimension)
    char *inA = nullptr, *inB = nullptr;
    int64_t ldA = 0, ldB = 0;
};

// Enqueue one request's transfers and kernels on a stream (lock not held).
static sr_status enqueue_request(ServeState &st, Job &job, cudaStream_t s)
{
    Req &q = *job.reqs[0];
    const std::vector<size_t> &offs = job.offs[0];
    const sr_request &r = q.r;
    const sr_dtype t = (sr_dtype)r.dtype;
    const int es = es_of(t);
    const int u32 = t == SR_BOOL_W64 ? 2 : 1;
    auto dptr = [&](size_t off) { return st.base + off; };
    auto h2d = [&](char *dst, int64_t ldd, const void *src, int64_t rows, int64_t cols) -> sr_status {
        const size_t w = (size_t)units_of(t, cols) * es;
        SR_CUDA_CHECK(cudaMemcpy2DAsync(dst, (size_t)ldd * es, src, w, w, (size_t)rows, cudaMemcpyHostToDevice, s));
        return SR_OK;
    };
    auto d2h = [&](void *dst, const char *src, int64_t lds, int64_t rows, int64_t cols) -> sr_status {
        const size_t w = (size_t)units_of(t, cols) * es;
        SR_CUDA_CHECK(cudaMemcpy2DAsync(dst, w, src, (size_t)lds * es, w, (size_t)rows, cudaMemcpyDeviceToHost, s));
        return SR_OK;
    };
    size_t k = 0;
    if (r.op == SR_OP_ANTIDIST_CLOSURE || r.op == SR_OP_BOOL_CLOSURE) {
        const int64_t D = r.R;
        const int64_t ld = pad_units(t, units_of(t, D));
        char *T = dptr(offs[k++]);
        if (job.inA) {
            SR_CUDA_CHECK(cudaMemcpy2DAsync(T, ld * es, job.inA, job.ldA * es, (size_t)units_of(t, D) * es, D,
                                            cudaMemcpyDeviceToDevice, s));
        } else {
            SR_TRY(h2d(T, ld, r.A, D, D));
        }
        if (r.op == SR_OP_ANTIDIST_CLOSURE) {
            SR_TRY(launch_antidist_closure(T, ld, (int)D, t, true, s));
        } else if (r.method == SR_CLOSURE_SQUARING) {
            sr_ctx tmp;                                   // workspace = this request's arena block
            tmp.ws = dptr(offs[k++]);
            tmp.ws_bytes = squaring_bytes(t, D);
            tmp.bool_tc_mode = 0;                         // the block holds the flags and two squares only
            SR_TRY(bool_closure(&tmp, T, ld, D, t, SR_CLOSURE_SQUARING, s));
        } else {
            SR_TRY(launch_bool_closure_warshall(reinterpret_cast<uint32_t *>(T), ld * u32, (int)D,
                                                (int)(units_of(t, D) * u32), true, s));
        }
        if (r.out) SR_TRY(d2h(r.out, T, ld, D, D));
    } else {
        char *A = job.inA, *B = job.inB;
        int64_t lda = job.ldA, ldb = job.ldB;
        if (!A) {
            A = dptr(offs[k++]);
            lda = pad_units(t, units_of(t, r.K));
            SR_TRY(h2d(A, lda, r.A, r.R, r.K));
        }
        if (!B) {
            B = dptr(offs[k++]);
            ldb = pad_units(t, units_of(t, r.N));
            SR_TRY(h2d(B, ldb, r.B, r.K, r.N));
        }
        char *C = dptr(offs[k++]);
        const int64_t ldc = pad_units(t, units_of(t, r.N));
        if (r.op == SR_OP_ANTIDIST_MUL)
            SR_TRY(antidist_mul(nullptr, A, lda, B, ldb, C, ldc, r.R, r.K, r.N, t, 0, s));
        else
            SR_TRY(bool_mul(nullptr, A, lda, B, ldb, C, ldc, r.R, r.K, r.N, t, 0, s));
        if (r.out) SR_TRY(d2h(r.out, C, ldc, r.R, r.N));
    }
    return SR_OK;
}

// Transfers in, one batched closure launch, transfers out (lock not held).
static sr_status enqueue_group(ServeState &st, Job &job, cudaStream_t s)
{
    Slot &sl = st.slots[job.slot];
    const sr_dtype t = (sr_dtype)job.reqs[0]->r.dtype;
    const int es = es_of(t);
    const int n = (int)job.reqs.size();
    for (int g = 0; g < n; ++g) {
        Req &q = *job.reqs[g];
        const int64_t D = q.r.R, ld = pad_units(t, D);
        char *T = st.base + job.offs[g][0];
        const size_t w = (size_t)D * es;
        SR_CUDA_CHECK(cudaMemcpy2DAsync(T, ld * es, q.r.A, w, w, D, cudaMemcpyHostToDevice, s));
        sl.h_graphs[g] = BatchGraph{T, ld, (int)D, 1};
        sl.h_items[g] = BatchItem{1, 0, {g, 0, 0, 0}};
    }
    SR_CUDA_CHECK(cudaMemcpyAsync(sl.d_graphs, sl.h_graphs, sizeof(BatchGraph) * n, cudaMemcpyHostToDevice, s));
    SR_CUDA_CHECK(cudaMemcpyAsync(sl.d_items, sl.h_items, sizeof(BatchItem) * n, cudaMemcpyHostToDevice, s));
    SR_TRY(launch_batched_closure_flat(t, sl.d_graphs, sl.d_items, n, sl.d_counter, 2, s));
    for (int g = 0; g < n; ++g) {
        Req &q = *job.reqs[g];
        if (!q.r.out) continue;
        const int64_t D = q.r.R, ld = pad_units(t, D);
        const size_t w = (size_t)D * es;
        SR_CUDA_CHECK(cudaMemcpy2DAsync(q.r.out, w, st.base + job.offs[g][0], ld * es, w, D,
                                        cudaMemcpyDeviceToHost, s));
    }
    return SR_OK;
}

static std::vector<size_t> buffer_sizes(const sr_request &r)
{
    const sr_dtype t = (sr_dtype)r.dtype;
    const int es = es_of(t);
    auto need = [&](int64_t rows, int64_t cols) { return (size_t)(rows * pad_units(t, units_of(t, cols)) * es); };
    std::vector<size_t> sizes;
    if (r.op == SR_OP_ANTIDIST_CLOSURE || r.op == SR_OP_BOOL_CLOSURE) {
        sizes.push_back(need(r.R, r.R));
        if (r.op == SR_OP_BOOL_CLOSURE && r.method == SR_CLOSURE_SQUARING)
            sizes.push_back(squaring_bytes(t, r.R));
    } else {
        if (!r.rA) sizes.push_back(need(r.R, r.K));
        if (!r.rB) sizes.push_back(need(r.K, r.N));
        sizes.push_back(need(r.R, r.N));
    }
    return sizes;
}

// Pick the next job that fits now (lock held): a free slot, then the head request,
// or with backfill a later one whose buffers fit (a long request also waits while
// another long one is in flight); small closures of the head's dtype waiting behind it
// join its group.  Allocates the buffers; false if nothing fits.
static bool next_job(ServeState &st, Job &job)
{
    int slot = -1;
    for (int i = 0; i < (int)st.slots.size(); ++i)
        if (!st.slots[i].busy) { slot = i; break; }
    if (slot < 0 || st.pending.empty()) return false;
    const double tnow = now_ms();
    const Req &head = *st.reqs[st.pending.front()];
    const bool may_backfill = tnow - head.t_submit < st.cfg.backfill_ms;
    int pick = -1;
    for (int i = 0; i < (int)st.pending.size(); ++i) {
        const Req &q = *st.reqs[st.pending[i]];
        if (request_bytes(q.r) <= st.arena.largest_free() && !(st.long_inflight > 0 && is_long(q.r))) {
            pick = i;
            break;
        }
        if (!may_backfill) break;
    }
    if (pick < 0) return false;
    Req *first = st.reqs[st.pending[pick]].get();
    auto is_small = [&](const Req &q) {
        return q.r.op == SR_OP_ANTIDIST_CLOSURE && (q.r.dtype == SR_U8 || q.r.dtype == SR_U16) &&
               q.r.R <= st.cfg.batch_max_d && !q.r.rA && q.r.dtype == first->r.dtype;
    };
    std::vector<Req *> cand;
    if (is_small(*first)) {
        for (int i = pick; i < (int)st.pending.size() && (int)cand.size() < st.cfg.batch_max_graphs; ++i) {
            Req *q = st.reqs[st.pending[i]].get();
            if (is_small(*q)) cand.push_back(q);
        }
    } else {
        cand.push_back(first);
    }
    job = Job();
    job.slot = slot;
    job.group = is_small(*first);
    for (Req *q : cand) {
        std::vector<size_t> o;
        bool ok = true;
        for (size_t n : buffer_sizes(q->r)) {
            size_t off;
            if (!st.arena.alloc(n, &off)) { ok = false; break; }
            o.push_back(off);
        }
        if (!ok) {
            for (size_t off : o) st.arena.release(off);
            break;
        }
        job.reqs.push_back(q);
        job.offs.push_back(o);
    }
    if (job.reqs.empty()) return false;
    for (size_t g = 0; g < job.reqs.size(); ++g) {
        Req *q = job.reqs[g];
        st.pending.erase(std::find(st.pending.begin(), st.pending.end(), q->id));
        q->t_admit = tnow;
        q->blocks = job.offs[g];
    }
    if (!job.group) {
        const sr_request &r = job.reqs[0]->r;
        if (r.rA) { const Resident &x = st.residents[r.rA]; job.inA = st.base + x.off; job.ldA = x.ld; }
        if (r.rB) { const Resident &x = st.residents[r.rB]; job.inB = st.base + x.off; job.ldB = x.ld; }
    }
    st.slots[slot].busy = true;
    if (!job.group && is_long(job.reqs[0]->r)) {
        st.slots[slot].long_job = true;
        ++st.long_inflight;
    }
    ++st.inflight;
    return true;
}

// After enqueueing (lock held): record failures, register kept results.
static void finish_job(ServeState &st, Job &job, sr_status est, const char *msg)
{
    for (size_t g = 0; g < job.reqs.size(); ++g) {
        Req &q = *job.reqs[g];
        if (est != SR_OK) {
            q.status = est;
            q.err = msg;
            ++st.failed;
            continue;
        }
        if (q.r.keep) {
            const sr_dtype t = (sr_dtype)q.r.dtype;
            const bool prod = q.r.op == SR_OP_ANTIDIST_MUL || q.r.op == SR_OP_BOOL_MUL;
            Resident res;
            res.off = job.offs[g].back();                  // result buffer is the last block
            if (!prod) res.off = job.offs[g][0];
            res.rows = q.r.R;
            res.cols = prod ? q.r.N : q.r.R;
            res.ld = pad_units(t, units_of(t, res.cols));
            res.dtype = t;
            res.bytes = (size_t)(res.rows * res.ld * es_of(t));
            q.resident = st.next_res++;
            st.residents[q.resident] = res;
            q.blocks.erase(std::remove(q.blocks.begin(), q.blocks.end(), res.off), q.blocks.end());
        }
    }
}

static void scheduler(ServeState *st)
{
    cudaSetDevice(st->device);
    std::unique_lock<std::mutex> lk(st->mu);
    while (!st->stop) {
        Job job;
        if (!next_job(*st, job)) {
            // wake on a new request or a completion; re-check periodically for backfill aging
            st->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        cudaStream_t s = st->slots[job.slot].stream;
        lk.unlock();
        sr_status est;
        {
            SR_TRACE(job.group ? "serve: grouped closures" : "serve: request");
            est = job.group ? enqueue_group(*st, job, s) : enqueue_request(*st, job, s);
        }
        const std::string msg = est == SR_OK ? std::string() : std::string(sr_last_error());
        lk.lock();
        finish_job(*st, job, est, msg.c_str());
        if (job.group && est == SR_OK) {
            ++st->batches;
            st->batched_reqs += job.reqs.size();
        }
        auto *c = new Completion{st, job.slot, {}};
        for (Req *q : job.reqs) c->ids.push_back(q->id);
        lk.unlock();
        const cudaError_t e = cudaLaunchHostFunc(s, on_complete, c);
        if (e != cudaSuccess) {            // finish synchronously on this thread
            cudaStreamSynchronize(s);
            on_complete(c);
        }
        lk.lock();
    }
}

static void stop_serving(sr_ctx *c)
{
    ServeState *st = c->serve;
    if (!st) return;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->stop = true;
    }
    st->cv_sched.notify_all();
    if (st->th.joinable()) st->th.join();
    for (auto &sl : st->slots) {
        if (sl.stream) { cudaStreamSynchronize(sl.stream); cudaStreamDestroy(sl.stream); }
        if (sl.d_graphs) cudaFree(sl.d_graphs);
        if (sl.d_items) cudaFree(sl.d_items);
        if (sl.d_counter) cudaFree(sl.d_counter);
        if (sl.h_graphs) cudaFreeHost(sl.h_graphs);
        if (sl.h_items) cudaFreeHost(sl.h_items);
    }
    if (st->base) cudaFree(st->base);
    delete st;
    c->serve = nullptr;
}

void sr_ctx_shutdown(sr_ctx *c) { stop_serving(c); }

}  // namespace sr

using namespace sr;

extern "C" {

sr_status sr_serve_start(sr_ctx *c, const sr_serve_config *cfg)
{
    SR_TRACE("sr_serve_start");
    if (!c)
        return fail(SR_EINVAL, "sr_serve_start: ctx is NULL");
    if (c->serve)
        return fail(SR_EBUSY, "sr_serve_start: already serving");
    sr_serve_config k{};
    if (cfg) k = *cfg;
    if (!k.arena_bytes) k.arena_bytes = (size_t)1 << 30;
    if (k.slots <= 0) k.slots = 4;
    if (k.slots > 64) k.slots = 64;
    if (k.max_pending <= 0) k.max_pending = 4096;
    if (k.batch_max_d <= 0) k.batch_max_d = 512;
    if (k.batch_max_graphs <= 0) k.batch_max_graphs = 64;
    k.batch_max_graphs = std::min(k.batch_max_graphs, 1024);
    if (k.backfill_ms < 0) k.backfill_ms = 0;
    auto *st = new (std::nothrow) ServeState();
    if (!st)
        return fail(SR_ENOMEM, "sr_serve_start: host allocation failed");
    st->cfg = k;
    st->device = current_device();
    if (st->device < 0) {
        delete st;
        return fail(SR_ECUDA, "sr_serve_start: no current CUDA device with an id below %d", kMaxDevices);
    }
    cudaError_t e = cudaMalloc(&st->base, k.arena_bytes);
    if (e != cudaSuccess) {
        delete st;
        return fail(SR_ENOMEM, "sr_serve_start: cannot allocate a %zu-byte arena (%s)", k.arena_bytes,
                    cudaGetErrorString(e));
    }
    st->arena.reset(k.arena_bytes);
    st->slots.resize(k.slots);
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    c->serve = st;
    for (auto &sl : st->slots) {
        e = cudaStreamCreateWithPriority(&sl.stream, cudaStreamNonBlocking, lo);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_graphs, sizeof(BatchGraph) * k.batch_max_graphs);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_items, sizeof(BatchItem) * k.batch_max_graphs);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d_counter, sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_graphs, sizeof(BatchGraph) * k.batch_max_graphs);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.h_items, sizeof(BatchItem) * k.batch_max_graphs);
        if (e != cudaSuccess) {
            stop_serving(c);
            return cuda_fail(e, "sr_serve_start: slot resources");
        }
    }
    st->th = std::thread(scheduler, st);
    return SR_OK;
}

sr_status sr_serve_stop(sr_ctx *c)
{
    SR_TRACE("sr_serve_stop");
    if (!c)
        return fail(SR_EINVAL, "sr_serve_stop: ctx is NULL");
    stop_serving(c);
    return SR_OK;
}

sr_status sr_submit(sr_ctx *c, const sr_request *r, uint64_t *ticket)
{
    SR_TRACE("sr_submit");
    if (!c || !r || !ticket)
        return fail(SR_EINVAL, "sr_submit: NULL argument");
    ServeState *st = c->serve;
    if (!st)
        return fail(SR_EINVAL, "sr_submit: serving is not started (sr_serve_start)");
    const sr_dtype t = (sr_dtype)r->dtype;
    const bool anti = t == SR_U8 || t == SR_U16 || t == SR_U32, boo = t == SR_BOOL_W32 || t == SR_BOOL_W64;
    const bool closure = r->op == SR_OP_ANTIDIST_CLOSURE || r->op == SR_OP_BOOL_CLOSURE;
    if (!((r->op == SR_OP_ANTIDIST_CLOSURE || r->op == SR_OP_ANTIDIST_MUL) ? anti
          : (r->op == SR_OP_BOOL_CLOSURE || r->op == SR_OP_BOOL_MUL) ? boo : false))
        return fail(SR_EINVAL, "sr_submit: op %d does not match dtype %d", r->op, r->dtype);
    if (r->R <= 0 || r->R > 0x7fffffffLL || (!closure && (r->K <= 0 || r->N <= 0 || r->K > 0x7fffffffLL ||
                                                          r->N > 0x7fffffffLL)))
        return fail(SR_EINVAL, "sr_submit: dimensions must be in [1, 2^31)");
    if ((!r->rA && !r->A) || (!closure && !r->rB && !r->B))
        return fail(SR_EINVAL, "sr_submit: missing input (host pointer or resident handle)");
    if (closure && r->op == SR_OP_BOOL_CLOSURE && r->method != SR_CLOSURE_WARSHALL && r->method != SR_CLOSURE_SQUARING)
        return fail(SR_EINVAL, "sr_submit: unknown closure method");
    const size_t need = request_bytes(*r);
    std::lock_guard<std::mutex> lk(st->mu);
    if (need > st->arena.size())
        return fail(SR_ENOMEM, "sr_submit: request needs %zu device bytes, the arena has %zu", need, st->arena.size());
    for (uint64_t h : {r->rA, r->rB})
        if (h && !st->residents.count(h))
            return fail(SR_ENOTFOUND, "sr_submit: unknown resident handle %llu", (unsigned long long)h);
    if ((int)st->pending.size() >= st->cfg.max_pending)
        return fail(SR_EAGAIN, "sr_submit: %d requests already waiting", (int)st->pending.size());
    auto q = std::make_unique<Req>();
    q->id = st->next_id++;
    q->r = *r;
    q->t_submit = now_ms();
    *ticket = q->id;
    st->pending.push_back(q->id);
    st->reqs[q->id] = std::move(q);
    ++st->submitted;
    st->cv_sched.notify_one();
    return SR_OK;
}

sr_status sr_poll(sr_ctx *c, uint64_t ticket, int *done)
{
    if (!c || !c->serve || !done)
        return fail(SR_EINVAL, "sr_poll: not serving or NULL argument");
    ServeState *st = c->serve;
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->reqs.find(ticket);
    if (it == st->reqs.end())
        return fail(SR_ENOTFOUND, "sr_poll: unknown ticket %llu", (unsigned long long)ticket);
    *done = it->second->done ? 1 : 0;
    return SR_OK;
}

sr_status sr_wait(sr_ctx *c, uint64_t ticket, int timeout_ms)
{
    SR_TRACE("sr_wait");
    if (!c || !c->serve)
        return fail(SR_EINVAL, "sr_wait: not serving");
    ServeState *st = c->serve;
    std::unique_lock<std::mutex> lk(st->mu);
    auto it = st->reqs.find(ticket);
    if (it == st->reqs.end())
        return fail(SR_ENOTFOUND, "sr_wait: unknown ticket %llu", (unsigned long long)ticket);
    Req *q = it->second.get();
    const bool ok = st->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)),
                                         [&] { return q->done; });
    if (!ok)
        return fail(SR_ETIMEOUT, "sr_wait: ticket %llu not done after %d ms", (unsigned long long)ticket, timeout_ms);
    if (q->status != SR_OK)
        return fail((sr_status)q->status, "request %llu failed: %s", (unsigned long long)ticket, q->err.c_str());
    return SR_OK;
}

sr_status sr_result(sr_ctx *c, uint64_t ticket, sr_result_info *info)
{
    if (!c || !c->serve || !info)
        return fail(SR_EINVAL, "sr_result: not serving or NULL argument");
    ServeState *st = c->serve;
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->reqs.find(ticket);
    if (it == st->reqs.end())
        return fail(SR_ENOTFOUND, "sr_result: unknown ticket %llu", (unsigned long long)ticket);
    const Req &q = *it->second;
    if (!q.done)
        return fail(SR_EBUSY, "sr_result: ticket %llu not finished", (unsigned long long)ticket);
    info->status = q.status;
    info->latency_ms = q.t_done - q.t_submit;
    info->queue_ms = q.t_admit - q.t_submit;
    info->resident = q.resident;
    return SR_OK;
}

sr_status sr_cancel(sr_ctx *c, uint64_t ticket)
{
    SR_TRACE("sr_cancel");
    if (!c || !c->serve)
        return fail(SR_EINVAL, "sr_cancel: not serving");
    ServeState *st = c->serve;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->reqs.find(ticket);
        if (it == st->reqs.end())
            return fail(SR_ENOTFOUND, "sr_cancel: unknown ticket %llu", (unsigned long long)ticket);
        Req &q = *it->second;
        if (q.done)
            return SR_OK;                                   // finished (or cancelled) already
        auto pos = std::find(st->pending.begin(), st->pending.end(), ticket);
        if (pos == st->pending.end())
            return fail(SR_EBUSY, "sr_cancel: ticket %llu is already running", (unsigned long long)ticket);
        st->pending.erase(pos);                             // never admitted: it holds no memory or slot
        q.status = SR_ECANCELED;
        q.err = "cancelled before admission";
        q.done = true;
        q.t_admit = q.t_done = now_ms();
        ++st->cancelled;
    }
    st->cv_done.notify_all();
    st->cv_sched.notify_one();
    return SR_OK;
}

sr_status sr_release(sr_ctx *c, uint64_t ticket)
{
    if (!c || !c->serve)
        return fail(SR_EINVAL, "sr_release: not serving");
    ServeState *st = c->serve;
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->reqs.find(ticket);
    if (it == st->reqs.end())
        return fail(SR_ENOTFOUND, "sr_release: unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done)
        return fail(SR_EBUSY, "sr_release: ticket %llu not finished", (unsigned long long)ticket);
    st->reqs.erase(it);
    return SR_OK;
}

sr_status sr_resident_put(sr_ctx *c, const void *host, int64_t rows, int64_t cols, sr_dtype dtype, uint64_t *handle)
{
    SR_TRACE("sr_resident_put");
    if (!c || !c->serve || !host || !handle || rows <= 0 || cols <= 0)
        return fail(SR_EINVAL, "sr_resident_put: not serving or bad argument");
    ServeState *st = c->serve;
    const int es = es_of(dtype);
    const int64_t ld = pad_units(dtype, units_of(dtype, cols));
    size_t off;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        if (!st->arena.alloc((size_t)(rows * ld * es), &off))
            return fail(SR_ENOMEM, "sr_resident_put: no room in the arena");
    }
    const size_t w = (size_t)units_of(dtype, cols) * es;
    cudaError_t e = cudaMemcpy2D(st->base + off, ld * es, host, w, w, rows, cudaMemcpyHostToDevice);
    std::lock_guard<std::mutex> lk(st->mu);
    if (e != cudaSuccess) {
        st->arena.release(off);
        return cuda_fail(e, "sr_resident_put");
    }
    Resident r;
    r.off = off; r.rows = rows; r.cols = cols; r.ld = ld; r.dtype = dtype; r.bytes = (size_t)(rows * ld * es);
    *handle = st->next_res++;
    st->residents[*handle] = r;
    return SR_OK;
}

sr_status sr_resident_get(sr_ctx *c, uint64_t handle, void *host)
{
    SR_TRACE("sr_resident_get");
    if (!c || !c->serve || !host)
        return fail(SR_EINVAL, "sr_resident_get: not serving or NULL argument");
    ServeState *st = c->serve;
    Resident r;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        auto it = st->residents.find(handle);
        if (it == st->residents.end())
            return fail(SR_ENOTFOUND, "sr_resident_get: unknown handle %llu", (unsigned long long)handle);
        r = it->second;
    }
    const int es = es_of(r.dtype);
    const size_t w = (size_t)units_of(r.dtype, r.cols) * es;
    // order after the work that produced it: the device is synchronised first
    SR_CUDA_CHECK(cudaDeviceSynchronize());
    SR_CUDA_CHECK(cudaMemcpy2D(host, w, st->base + r.off, r.ld * es, w, r.rows, cudaMemcpyDeviceToHost));
    return SR_OK;
}

sr_status sr_resident_free(sr_ctx *c, uint64_t handle)
{
    if (!c || !c->serve)
        return fail(SR_EINVAL, "sr_resident_free: not serving");
    ServeState *st = c->serve;
    std::lock_guard<std::mutex> lk(st->mu);
    auto it = st->residents.find(handle);
    if (it == st->residents.end())
        return fail(SR_ENOTFOUND, "sr_resident_free: unknown handle %llu", (unsigned long long)handle);
    st->arena.release(it->second.off);
    st->residents.erase(it);
    st->cv_sched.notify_one();
    return SR_OK;
}

sr_status sr_serve_stats(sr_ctx *c, sr_serve_stats_t *out)
{
    if (!c || !c->serve || !out)
        return fail(SR_EINVAL, "sr_serve_stats: not serving or NULL argument");
    ServeState *st = c->serve;
    std::lock_guard<std::mutex> lk(st->mu);
    out->submitted = st->submitted;
    out->completed = st->completed;
    out->failed = st->failed;
    out->batches = st->batches;
    out->batched_requests = st->batched_reqs;
    out->cancelled = st->cancelled;
    out->arena_bytes = st->arena.size();
    out->arena_in_use = st->arena.used();
    out->arena_peak_bytes = st->arena.peak();
    out->pending = (int)st->pending.size();
    out->inflight = st->inflight;
    out->residents = (int)st->residents.size();
    return SR_OK;
}

}  // extern "C"
