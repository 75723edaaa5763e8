// fc_api.cu -- host runtime behind the C ABI of include/fc.h: contexts
// (the loaded database), the batch planner (validation, strategy choice by a
// cost model, work items), plans replayed as CUDA graphs, the host-buffer
// entry points, options and the autotuner.
#include "../../include/fc.h"
#include "fc_internal.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <mutex>
#include <memory>
#include <functional>
#include <condition_variable>
#include <vector>

using namespace fc;

// ------------------------------------------------------------------ errors

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace

int fc::set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(FC_ERR_OOM, "%s: out of device memory", what);
    }
    return fail(FC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define FC_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Device buffer owned by the runtime, or a view of a context pool buffer
// (plans made by the synchronous entry points borrow them, so a call
// allocates nothing once the pool has grown).
struct DBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool owned = true;
    void release()
    {
        if (p && owned) cudaFree(p);
        p = nullptr;
        bytes = 0;
        owned = true;
    }
    cudaError_t ensure(size_t want)
    {
        if (want <= bytes && p) return cudaSuccess;
        release();
        if (want == 0) want = 16;
        cudaError_t e = cudaMalloc(&p, want);
        if (e == cudaSuccess) bytes = want;
        return e;
    }
};

struct Options {
    int32_t strategy = FC_STRAT_AUTO;
    int32_t smem_cells = 24576;       // 96 KiB of tables per CTA
    int32_t threads = 512;
    int32_t ctas_per_sm = 2;
    int32_t hist_copies = 4;
    int64_t min_part_rows = 65536;
    int64_t pair_chunk_rows = 1 << 16;
    int32_t use_graph = 1;
    int64_t wait_limit = 1 << 22;
    int64_t sort_min_cells = 1 << 25;
    // cost model, femtoseconds: bitmap per DFS node per 4096-row chunk;
    // histogram per row and per row-variable; per table cell flushed
    int64_t bitmap_cost = 200000;
    int64_t bitmap_chunk_cost = 0;    // per 4096-row chunk of a bitmap query
    int64_t hist_cost_row = 143;
    int64_t hist_cost_var = 124;
    int64_t flush_cost = 160;
    // register-blocked bitmap path (2-3 variables of arity 2..5): per work
    // unit (cell or state row) per 4096-row chunk
    int64_t small_cost = 12000;
    int32_t bitmap_small = 1;
    int32_t stage_slots = 16;         // bitmap rows a warp stages per chunk
    int32_t bitmap_threads = 256;
    int32_t support_warps = 16;
    int32_t support_sets_per_warp = 4;
    int64_t support_part_words = 8192;
};

}  // namespace

namespace {
// Host worker threads of a context (the planner's per-query work).  run(n, f)
// calls f(0) on the calling thread and f(1..n-1) on workers, and returns when
// all have finished; workers sleep between runs.
class PlanPool {
public:
    ~PlanPool()
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            stop_ = true;
        }
        cv_.notify_all();
        for (auto &t : th_) t.join();
    }
    int size() const { return (int)th_.size() + 1; }
    void start(int workers)
    {
        for (int i = 0; i < workers; ++i) th_.emplace_back([this, i] { loop(i + 1); });
    }
    void run(int n, const std::function<void(int)> &f)
    {
        {
            std::lock_guard<std::mutex> lk(mu_);
            job_ = &f;
            job_n_ = n;
            pending_ = (int)th_.size();
            ++gen_;
        }
        cv_.notify_all();
        f(0);
        std::unique_lock<std::mutex> lk(mu_);
        done_.wait(lk, [&] { return pending_ == 0; });
        job_ = nullptr;
    }

private:
    void loop(int idx)
    {
        uint64_t seen = 0;
        for (;;) {
            std::unique_lock<std::mutex> lk(mu_);
            cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
            if (stop_) return;
            seen = gen_;
            const std::function<void(int)> *f = job_;
            const int n = job_n_;
            lk.unlock();
            if (idx < n) (*f)(idx);
            lk.lock();
            if (--pending_ == 0) done_.notify_one();
        }
    }
    std::vector<std::thread> th_;
    std::mutex mu_;
    std::condition_variable cv_, done_;
    const std::function<void(int)> *job_ = nullptr;
    int job_n_ = 0, pending_ = 0;
    uint64_t gen_ = 0;
    bool stop_ = false;
};
}  // namespace

struct fc_ctx {
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    cudaStream_t stream = nullptr;
    bool transactions = false;  // loaded with fc_load_bits
    int32_t n = 0;
    int64_t m = 0;
    std::vector<int32_t> arity, soff;
    int32_t R = 0;
    int64_t m_pad = 0, words = 0, wstride = 0;
    uint8_t *d_D = nullptr;
    uint64_t *d_bits = nullptr;
    int64_t *d_marg = nullptr;
    int32_t *d_arity = nullptr, *d_soff = nullptr;
    int32_t *d_status = nullptr;
    std::vector<int64_t> marg;
    std::vector<double> entropy;
    Options opt;
    // scratch of the host-buffer entry points
    DBuf io[3];
    DBuf pool[6];        // buffers lent to one-shot plans (descriptors, counters, tables, sort, pairs)
    bool borrow = false; // set while a synchronous entry point builds its plan
    std::vector<uint32_t> mark;
    uint32_t epoch = 0;
    uint64_t generation = 0;  // bumped by every append; plans of older generations refuse to run
    std::vector<fc_plan *> live_plans;  // orphaned (device memory released) if the context goes first
    // pinned staging of plan descriptors: written on the host, copied by DMA;
    // the event marks the end of the last copy out of it
    uint8_t *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    cudaEvent_t h_stage_ev = nullptr;
    std::unique_ptr<PlanPool> pool_threads;  // started by the first large plan
};

namespace {

struct GraphEntry {
    void *o0, *o1, *o2;
    cudaStream_t s;
    cudaGraphExec_t exec;
};

struct SortJob {
    int32_t q;
    int32_t k;
    int32_t key_bits;
    int32_t cells;
    int64_t table_off;
    const QVar *d_vars;
};

enum PlanKind { kPlanCount = 0, kPlanScore = 1, kPlanSupport = 2, kPlanPairs = 3, kPlanFamilies = 4 };

}  // namespace

struct fc_plan {
    fc_ctx *ctx = nullptr;
    int kind = kPlanCount;
    int32_t nq = 0;
    std::vector<int64_t> table_off;  // count plans: caller offsets (nq + 1)
    std::vector<int32_t> strategy;
    int64_t out_cells = 0;
    // count / score
    DBuf desc;           // QHead, QVar, Item, q_list
    DBuf counters;       // next item + tickets
    DBuf scratch_tables; // score plans: tables that live in global memory
    DBuf sort_mem;
    SortScratch sort_sc{};
    std::vector<SortJob> sort_jobs;
    QHead *d_qh = nullptr;
    QVar *d_qv = nullptr;
    Item *d_items = nullptr;
    int32_t *d_qlist = nullptr;
    int32_t n_items = 0, n_qlist = 0, n_counters = 0;
    BTask *d_btasks = nullptr;
    int32_t n_btasks = 0, bm_grid = 0, bm_threads = 0, stage_slots = 0;
    int32_t small_paths = 1;
    bool zero_tables = false;
    int64_t table_buf_cells = 0;  // cells of the buffer the kernel writes
    int score_kind = kNoScore;
    double ess = 1.0;
    int grid = 0, threads = 0, smem_cells = 0;
    size_t smem = 0;
    // support
    SupportParams sp{};
    int sup_grid = 0, sup_threads = 0;
    int64_t n_sub = 0;
    // pairs
    PairsParams pp{};
    DBuf pairs_C, pairs_meta;
    int64_t n_pairs = 0, pair_cells = 0;
    int64_t *d_pair_off = nullptr;
    // families: the joint tables of every variable set (inner count plan) and
    // one job per (child, parents) split
    fc_plan *inner = nullptr;
    DBuf fam_tables, fam_jobs;
    int64_t n_jobs = 0;
    int fam_kind = 0;
    uint64_t generation = 0;  // the context's generation when the plan was built
    size_t upload_bytes = 0;  // host-to-device bytes of the plan's descriptors
    std::vector<GraphEntry> graphs;
};

namespace {

// A plan buffer: its own allocation, or a view of the context's pool slot.
cudaError_t plan_buf(fc_ctx *c, DBuf &b, int slot, size_t bytes)
{
    if (!c->borrow) return b.ensure(bytes);
    cudaError_t e = c->pool[slot].ensure(bytes);
    if (e != cudaSuccess) return e;
    b.p = c->pool[slot].p;
    b.bytes = c->pool[slot].bytes;
    b.owned = false;
    return cudaSuccess;
}

struct BorrowScope {
    fc_ctx *c;
    explicit BorrowScope(fc_ctx *ctx) : c(ctx) { c->borrow = true; }
    ~BorrowScope() { c->borrow = false; }
};

// Pinned host staging of at least `bytes` for plan descriptors, free of any
// copy still reading it; nullptr on failure.
uint8_t *stage_host(fc_ctx *c, size_t bytes)
{
    if (c->h_stage_ev && cudaEventSynchronize(c->h_stage_ev) != cudaSuccess) return nullptr;
    if (bytes > c->h_stage_bytes) {
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        const size_t want = std::max(bytes, c->h_stage_bytes + c->h_stage_bytes / 2);
        if (cudaHostAlloc((void **)&c->h_stage, want, cudaHostAllocDefault) != cudaSuccess) {
            c->h_stage = nullptr;
            return nullptr;
        }
        c->h_stage_bytes = want;
    }
    if (!c->h_stage_ev && cudaEventCreateWithFlags(&c->h_stage_ev, cudaEventDisableTiming) != cudaSuccess)
        return nullptr;
    return c->h_stage;
}

// Copies `bytes` of the staging buffer to dst on the context stream and
// marks the staging buffer busy until the copy ends.
cudaError_t upload_stage(fc_ctx *c, void *dst, size_t bytes)
{
    cudaError_t e = cudaMemcpyAsync(dst, c->h_stage, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->h_stage_ev, c->stream);
    return e;
}

}  // namespace

// ---------------------------------------------------------------- loading

namespace {

int finish_load(fc_ctx *c)
{
    // marginal counts per (variable, state) and entropies (DFS order, Sec. 3.2)
    FC_CUDA(cudaMalloc(&c->d_marg, sizeof(int64_t) * std::max(c->R, 1)), "cudaMalloc marginals");
    FC_CUDA(launch_bit_popcounts(c->d_bits, c->R, c->wstride, c->d_marg, c->stream), "popcounts");
    c->marg.assign(c->R, 0);
    FC_CUDA(cudaMemcpyAsync(c->marg.data(), c->d_marg, sizeof(int64_t) * c->R,
                            cudaMemcpyDeviceToHost, c->stream), "copy marginals");
    FC_CUDA(cudaStreamSynchronize(c->stream), "load");
    c->entropy.assign(c->n, 0.0);
    if (!c->transactions) {
        for (int i = 0; i < c->n; ++i) {
            double h = 0.0;
            for (int s = 0; s < c->arity[i]; ++s) {
                const double p = (double)c->marg[c->soff[i] + s] / (double)c->m;
                if (p > 0.0) h -= p * std::log2(p);
            }
            c->entropy[i] = h;
        }
    }
    c->mark.assign(c->n, 0u);
    return FC_OK;
}

int new_ctx(fc_ctx **out, int32_t n, int64_t m)
{
    fc_ctx *c = new (std::nothrow) fc_ctx();
    if (!c) return fail(FC_ERR_OOM, "host allocation failed");
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    cudaDeviceGetAttribute(&c->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaStreamCreate");
    }
    c->n = n;
    c->m = m;
    c->words = (m + 63) / 64;
    c->wstride = round_up(c->words, kChunkWords);
    *out = c;
    e = cudaMalloc(&c->d_status, 16);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 16, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "status word");
    return FC_OK;
}

}  // namespace

extern "C" int fc_load(fc_ctx **out, const uint8_t *D, int32_t n, int64_t m,
                       const int32_t *arities, int32_t layout, int32_t where)
{
    if (!out || !D || !arities) return fail(FC_ERR_ARG, "fc_load: null argument");
    *out = nullptr;
    if (n < 1 || m < 1) return fail(FC_ERR_ARG, "fc_load: need n >= 1 and m >= 1");
    if (m >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "fc_load: m must be < 2^31");
    if (layout != FC_COL_MAJOR && layout != FC_ROW_MAJOR) return fail(FC_ERR_ARG, "fc_load: bad layout");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_load: bad pointer location");
    for (int i = 0; i < n; ++i)
        if (arities[i] < 1 || arities[i] > 255)
            return fail(FC_ERR_ARG, "fc_load: arity of variable %d is %d, not in 1..255", i, arities[i]);
    fc_ctx *c = nullptr;
    int rc = new_ctx(&c, n, m);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    c->arity.assign(arities, arities + n);
    c->soff.resize(n);
    for (int i = 0; i < n; ++i) {
        c->soff[i] = c->R;
        c->R += arities[i];
    }
    c->m_pad = round_up(m, kChunkRows);
    auto bail = [&](int code) {
        fc_free(c);
        return code;
    };
    cudaError_t e;
    if ((e = cudaMalloc(&c->d_D, (size_t)n * c->m_pad)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc D"));
    if ((e = cudaMemsetAsync(c->d_D, 0, (size_t)n * c->m_pad, c->stream)) != cudaSuccess) return bail(cuda_fail(e, "memset D"));
    const cudaMemcpyKind kind = where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (layout == FC_COL_MAJOR) {
        e = cudaMemcpy2DAsync(c->d_D, c->m_pad, D, m, m, n, kind, c->stream);
        if (e != cudaSuccess) return bail(cuda_fail(e, "copy D"));
    } else {
        uint8_t *tmp = nullptr;
        if ((e = cudaMalloc(&tmp, (size_t)n * m)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc D rows"));
        e = cudaMemcpyAsync(tmp, D, (size_t)n * m, kind, c->stream);
        if (e == cudaSuccess) e = launch_transpose_rows(tmp, m, n, c->d_D, c->m_pad, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e != cudaSuccess) return bail(cuda_fail(e, "transpose D"));
    }
    if ((e = cudaMalloc(&c->d_arity, sizeof(int32_t) * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    if ((e = cudaMalloc(&c->d_soff, sizeof(int32_t) * n)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc"));
    cudaMemcpyAsync(c->d_arity, c->arity.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_soff, c->soff.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream);
    // one row per (variable, state) plus an all-zero row R (states outside an arity)
    const size_t bits_bytes = sizeof(uint64_t) * (size_t)(c->R + 1) * c->wstride;
    if ((e = cudaMalloc(&c->d_bits, bits_bytes)) != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc bitmaps"));
    if ((e = cudaMemsetAsync(c->d_bits, 0, bits_bytes, c->stream)) != cudaSuccess) return bail(cuda_fail(e, "memset bitmaps"));
    int32_t *bad = c->d_status + 1;
    e = launch_pack_bits(c->d_D, c->m_pad, m, n, c->d_arity, c->d_soff, c->d_bits, c->wstride, 255, bad, c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "pack bitmaps"));
    int32_t bad_h = 0;
    e = cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(cuda_fail(e, "load"));
    if (bad_h) return bail(fail(FC_ERR_RANGE, "fc_load: a stored state is >= its variable's arity"));
    cudaMemsetAsync(c->d_status, 0, 16, c->stream);
    rc = finish_load(c);
    if (rc != FC_OK) return bail(rc);
    *out = c;
    return FC_OK;
}

extern "C" int fc_load_bits(fc_ctx **out, const uint64_t *bitmaps, int32_t n_items, int64_t m,
                            int32_t where)
{
    if (!out || !bitmaps) return fail(FC_ERR_ARG, "fc_load_bits: null argument");
    *out = nullptr;
    if (n_items < 1 || m < 1) return fail(FC_ERR_ARG, "fc_load_bits: need n_items >= 1 and m >= 1");
    if (m >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "fc_load_bits: m must be < 2^31");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_load_bits: bad pointer location");
    fc_ctx *c = nullptr;
    int rc = new_ctx(&c, n_items, m);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    c->transactions = true;
    c->arity.assign(n_items, 1);
    c->soff.resize(n_items);
    for (int i = 0; i < n_items; ++i) c->soff[i] = i;
    c->R = n_items;
    const size_t bits_bytes = sizeof(uint64_t) * (size_t)n_items * c->wstride;
    cudaError_t e = cudaMalloc(&c->d_bits, bits_bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_bits, 0, bits_bytes, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(c->d_bits, sizeof(uint64_t) * c->wstride, bitmaps, sizeof(uint64_t) * c->words,
                              sizeof(uint64_t) * c->words, n_items,
                              where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = launch_mask_tail_bits(c->d_bits, n_items, c->wstride, m, c->stream);
    if (e != cudaSuccess) {
        fc_free(c);
        return cuda_fail(e, "fc_load_bits");
    }
    rc = finish_load(c);
    if (rc != FC_OK) {
        fc_free(c);
        return rc;
    }
    *out = c;
    return FC_OK;
}

namespace {
void release_plan(fc_plan *p);
}  // namespace

extern "C" void fc_free(fc_ctx *c)
{
    if (!c) return;
    DevGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    // plans still alive keep their host struct for fc_plan_free but lose
    // their device memory and their context
    for (fc_plan *p : c->live_plans) {
        release_plan(p);
        p->ctx = nullptr;
    }
    c->live_plans.clear();
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->h_stage_ev) cudaEventDestroy(c->h_stage_ev);
    for (auto &b : c->io) b.release();
    for (auto &b : c->pool) b.release();
    cudaFree(c->d_D);
    cudaFree(c->d_bits);
    cudaFree(c->d_marg);
    cudaFree(c->d_arity);
    cudaFree(c->d_soff);
    cudaFree(c->d_status);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ---------------------------------------------------------------- appends
//
// Sec. 6: a database that grows by new instances needs only an update of the
// bitmaps (and the histogram/radix strategies read D as it stands).  Storage
// keeps spare rows: D columns are m_pad bytes apart and bitmap rows wstride
// words apart, both sized for a capacity that grows geometrically, with every
// byte and bit past m zero.

namespace {

int64_t capacity_rows(const fc_ctx *c)
{
    const int64_t bit_rows = c->wstride * 64;
    return c->transactions ? bit_rows : std::min(c->m_pad, bit_rows);
}

// Make room for m_need instances (reallocating and copying when needed).
int grow_storage(fc_ctx *c, int64_t m_need)
{
    if (m_need <= capacity_rows(c)) return FC_OK;
    if (m_need >= ((int64_t)1 << 31)) return fail(FC_ERR_RANGE, "m would reach %lld, must stay < 2^31", (long long)m_need);
    int64_t cap = std::max<int64_t>(m_need, capacity_rows(c) + capacity_rows(c) / 2);
    cap = std::min<int64_t>(round_up(cap, kChunkRows), ((int64_t)1 << 31) - 1);
    cap = std::max(cap, m_need);
    const int64_t new_pad = round_up(cap, kChunkRows);
    const int64_t new_wstride = round_up((new_pad + 63) / 64, kChunkWords);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "append");
    const int64_t rows = c->transactions ? c->R : c->R + 1;
    uint64_t *nb = nullptr;
    const size_t bbytes = sizeof(uint64_t) * (size_t)rows * new_wstride;
    if ((e = cudaMalloc(&nb, bbytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc bitmaps");
    e = cudaMemsetAsync(nb, 0, bbytes, c->stream);
    if (e == cudaSuccess && c->words > 0)
        e = cudaMemcpy2DAsync(nb, sizeof(uint64_t) * new_wstride, c->d_bits, sizeof(uint64_t) * c->wstride,
                              sizeof(uint64_t) * c->words, rows, cudaMemcpyDeviceToDevice, c->stream);
    uint8_t *nd = nullptr;
    if (e == cudaSuccess && !c->transactions) {
        const size_t dbytes = (size_t)c->n * new_pad;
        e = cudaMalloc(&nd, dbytes);
        if (e == cudaSuccess) e = cudaMemsetAsync(nd, 0, dbytes, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(nd, new_pad, c->d_D, c->m_pad, c->m, c->n, cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaFree(nb);
        cudaFree(nd);
        return cuda_fail(e, "grow storage");
    }
    cudaFree(c->d_bits);
    c->d_bits = nb;
    c->wstride = new_wstride;
    if (!c->transactions) {
        cudaFree(c->d_D);
        c->d_D = nd;
        c->m_pad = new_pad;
    }
    return FC_OK;
}

// New instance count, marginals and entropies after an append.
int finish_append(fc_ctx *c, int64_t m_total)
{
    c->m = m_total;
    c->words = (m_total + 63) / 64;
    c->generation += 1;
    cudaError_t e = cudaMemcpyAsync(c->marg.data(), c->d_marg, sizeof(int64_t) * c->R, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "append marginals");
    if (!c->transactions)
        for (int i = 0; i < c->n; ++i) {
            double h = 0.0;
            for (int s = 0; s < c->arity[i]; ++s) {
                const double p = (double)c->marg[c->soff[i] + s] / (double)c->m;
                if (p > 0.0) h -= p * std::log2(p);
            }
            c->entropy[i] = h;
        }
    return FC_OK;
}

}  // namespace

extern "C" int fc_reserve(fc_ctx *c, int64_t m_total)
{
    if (!c) return fail(FC_ERR_ARG, "fc_reserve: null context");
    if (m_total < 0) return fail(FC_ERR_ARG, "fc_reserve: m_total < 0");
    DevGuard g(c->device);
    return grow_storage(c, m_total);
}

extern "C" int fc_append(fc_ctx *c, const uint8_t *D, int64_t m_new, int32_t layout, int32_t where)
{
    if (!c) return fail(FC_ERR_ARG, "fc_append: null context");
    if (c->transactions) return fail(FC_ERR_STATE, "fc_append: a context from fc_load_bits takes fc_append_bits");
    if (m_new < 0) return fail(FC_ERR_ARG, "fc_append: m_new < 0");
    if (m_new == 0) return FC_OK;
    if (!D) return fail(FC_ERR_ARG, "fc_append: null D");
    if (layout != FC_COL_MAJOR && layout != FC_ROW_MAJOR) return fail(FC_ERR_ARG, "fc_append: bad layout");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_append: bad pointer location");
    DevGuard g(c->device);
    const int64_t m0 = c->m, m1 = m0 + m_new;
    int rc = grow_storage(c, m1);
    if (rc != FC_OK) return rc;
    const cudaMemcpyKind kind = where == FC_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e;
    if (layout == FC_COL_MAJOR) {
        e = cudaMemcpy2DAsync(c->d_D + m0, c->m_pad, D, m_new, m_new, c->n, kind, c->stream);
    } else {
        const size_t bytes = (size_t)c->n * m_new;
        e = c->io[2].ensure(bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->io[2].p, D, bytes, kind, c->stream);
        if (e == cudaSuccess)
            e = launch_transpose_rows((const uint8_t *)c->io[2].p, m_new, c->n, c->d_D + m0, c->m_pad, c->stream);
    }
    // states are checked before anything visible changes
    int32_t *bad = c->d_status + 1;
    int32_t bad_h = 0;
    if (e == cudaSuccess) e = launch_check_states(c->d_D, c->m_pad, m0, m1, c->n, c->d_arity, bad, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append");
    if (bad_h) {
        cudaMemsetAsync(bad, 0, sizeof(int32_t), c->stream);
        cudaMemset2DAsync(c->d_D + m0, c->m_pad, 0, m_new, c->n, c->stream);
        cudaStreamSynchronize(c->stream);
        return fail(FC_ERR_RANGE, "fc_append: a state is >= its variable's arity; nothing was appended");
    }
    e = launch_pack_bits(c->d_D, c->m_pad, m1, c->n, c->d_arity, c->d_soff, c->d_bits, c->wstride, 255, bad,
                         c->stream, m0 / 64);
    if (e == cudaSuccess)
        e = launch_state_counts(c->d_D, c->m_pad, m0, m1, c->n, c->d_arity, c->d_soff, c->d_marg, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append bitmaps");
    return finish_append(c, m1);
}

extern "C" int fc_append_bits(fc_ctx *c, const uint64_t *bitmaps, int64_t m_new, int32_t where)
{
    if (!c) return fail(FC_ERR_ARG, "fc_append_bits: null context");
    if (!c->transactions) return fail(FC_ERR_STATE, "fc_append_bits: a categorical context takes fc_append");
    if (m_new < 0) return fail(FC_ERR_ARG, "fc_append_bits: m_new < 0");
    if (m_new == 0) return FC_OK;
    if (!bitmaps) return fail(FC_ERR_ARG, "fc_append_bits: null bitmaps");
    if (where != FC_HOST && where != FC_DEVICE) return fail(FC_ERR_ARG, "fc_append_bits: bad pointer location");
    DevGuard g(c->device);
    const int64_t m0 = c->m, m1 = m0 + m_new;
    int rc = grow_storage(c, m1);
    if (rc != FC_OK) return rc;
    const int64_t n_in = (m_new + 63) / 64;
    const uint64_t *src = bitmaps;
    cudaError_t e = cudaSuccess;
    if (where == FC_HOST) {
        const size_t bytes = sizeof(uint64_t) * (size_t)c->R * n_in;
        e = c->io[2].ensure(bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->io[2].p, bitmaps, bytes, cudaMemcpyHostToDevice, c->stream);
        src = (const uint64_t *)c->io[2].p;
    }
    if (e == cudaSuccess) e = launch_append_bits(c->d_bits, c->wstride, c->R, m0, src, n_in, m_new, c->d_marg, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "fc_append_bits");
    return finish_append(c, m1);
}

extern "C" int64_t fc_info(const fc_ctx *c, int32_t key)
{
    if (!c) return -1;
    switch (key) {
    case 0: return c->n;
    case 1: return c->m;
    case 2: return c->R;
    case 3: return c->device;
    case 4: return capacity_rows(c);
    case 5: return (int64_t)c->generation;
    default: return -1;
    }
}

extern "C" int fc_marginals(const fc_ctx *c, int64_t *out)
{
    if (!c || !out) return fail(FC_ERR_ARG, "fc_marginals: null argument");
    std::memcpy(out, c->marg.data(), sizeof(int64_t) * c->R);
    return FC_OK;
}

// ------------------------------------------------------------------ planner

namespace {

// Validates one variable list and appends its device description: strides in
// the caller's order (last fastest), arity-1 variables dropped (they add no
// digit).  Returns the number of cells or a negative FC_ERR code.
// Validates one query's variables and appends its QVars (arity-1 variables
// dropped, strides of the caller's order, last fastest); returns the cells.
// Reads the context only, so planner threads may call it concurrently (an
// error's message goes to the calling thread's fc_last_error).
int64_t describe(const fc_ctx *c, const int32_t *vars, int32_t k, std::vector<QVar> &qv, int32_t &k_eff)
{
    if (k < 0 || k > c->n) return fail(FC_ERR_ARG, "query has %d variables, n = %d", k, c->n);
    if (k > 0 && !vars) return fail(FC_ERR_ARG, "null variable list");
    int64_t cells = 1;
    for (int t = 0; t < k; ++t) {
        const int v = vars[t];
        if (v < 0 || v >= c->n) return fail(FC_ERR_ARG, "variable %d out of range 0..%d", v, c->n - 1);
        cells *= c->arity[v];
        if (cells > INT32_MAX) return fail(FC_ERR_SIZE, "table over %d variables exceeds 2^31-1 cells", k);
    }
    // duplicates: pairwise for short lists, a sorted copy otherwise
    if (k <= 48) {
        for (int t = 1; t < k; ++t)
            for (int u = 0; u < t; ++u)
                if (vars[u] == vars[t]) return fail(FC_ERR_ARG, "variable %d listed twice in one query", vars[t]);
    } else {
        std::vector<int32_t> sorted(vars, vars + k);
        std::sort(sorted.begin(), sorted.end());
        for (int t = 1; t < k; ++t)
            if (sorted[t] == sorted[t - 1]) return fail(FC_ERR_ARG, "variable %d listed twice in one query", sorted[t]);
    }
    int64_t stride = 1;
    const size_t first = qv.size();
    for (int t = k - 1; t >= 0; --t) {
        const int v = vars[t];
        if (c->arity[v] > 1) qv.push_back(QVar{v, (int32_t)stride, c->arity[v], c->soff[v]});
        stride *= c->arity[v];
    }
    std::reverse(qv.begin() + first, qv.end());
    k_eff = (int32_t)(qv.size() - first);
    return cells;
}

// DFS nodes of the bitmap tree in the given variable order (no pruning).
double dfs_nodes(const QVar *v, int k)
{
    double nodes = 0.0, level = 1.0;
    for (int t = 0; t < k; ++t) {
        level *= v[t].arity;
        nodes += level;
    }
    return nodes;
}

struct QPlan {
    int32_t strategy;
    double cost;  // femtoseconds for the whole query
};

// The bitmap DFS visits variables in ascending entropy (Sec. 3.2); a warp
// stages the state bitmaps of every level but the first.
void entropy_order(const fc_ctx *c, QVar *v, int k)
{
    // stable insertion sort: k is small and this runs once or twice per query
    for (int i = 1; i < k; ++i) {
        const QVar x = v[i];
        const double h = c->entropy[x.var];
        int j = i - 1;
        while (j >= 0 && c->entropy[v[j].var] > h) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = x;
    }
}

// Staged slots of the query in entropy order; the ordered copy goes to o.
// Queries the bitmap kernel counts on its register-blocked path (no tree
// walk): 2 variables, or 3 whose last two in entropy order, of arities 2..5;
// `o` is in entropy order.  Work units per 4096-row chunk: cells plus the
// state rows loaded.
bool small_ok(const QVar *o, int k)
{
    auto ok = [](int r) { return r >= 2 && r <= 5; };
    if (k == 2) return ok(o[0].arity) && ok(o[1].arity);
    if (k == 3) return ok(o[1].arity) && ok(o[2].arity);
    return false;
}

double small_units(const QVar *o, int k)
{
    if (k == 2) return (double)o[0].arity * o[1].arity + o[0].arity + o[1].arity;
    const double rb = o[1].arity, rc = o[2].arity;
    return (double)o[0].arity * (1.0 + rb + rc + rb * rc);
}

bool bitmap_ok(const fc_ctx *c, const QVar *v, int k, QVar *o)
{
    if (k < 1 || k > kMaxBitmapK) return false;
    std::copy(v, v + k, o);
    entropy_order(c, o, k);
    int slots = 0;
    for (int t = 1; t < k; ++t) slots += o[t].arity;
    return slots <= c->opt.stage_slots;
}

// Strategy and cost of one query.  When the bitmap strategy is chosen, the
// variables are left in v in entropy order (the order its kernel walks).
QPlan choose(const fc_ctx *c, QVar *v, int k, int64_t cells, int32_t smem_cells, double chunks)
{
    const Options &o = c->opt;
    const double rows = (double)c->m;
    const double flush = (double)cells * o.flush_cost;
    const bool fits = cells <= smem_cells;
    QVar ord[kMaxBitmapK];
    const bool bm = bitmap_ok(c, v, k, ord);
    const double nodes = bm ? dfs_nodes(ord, k) : 0.0;
    const double hist = rows * (o.hist_cost_row + (double)k * o.hist_cost_var) + flush;
    double bitmap = bm ? chunks * ((double)o.bitmap_chunk_cost + nodes * o.bitmap_cost) + flush : 1e300;
    if (bm && o.bitmap_small && small_ok(ord, k))
        bitmap = chunks * ((double)o.bitmap_chunk_cost + small_units(ord, k) * o.small_cost) + flush;
    const double gatomic = rows * (o.hist_cost_row + (double)k * o.hist_cost_var) * 2.0 + (double)cells * 4.0;
    int32_t s = o.strategy;
    if (k == 0) s = fits ? FC_STRAT_HIST : FC_STRAT_GATOMIC;
    if (k == 1 && fits && (s == FC_STRAT_AUTO || s == FC_STRAT_HIST)) return QPlan{FC_STRAT_MARGINAL, flush};
    if (s == FC_STRAT_BITMAP && !bm) s = FC_STRAT_AUTO;
    if (s == FC_STRAT_HIST && !fits) s = FC_STRAT_AUTO;
    if (s == FC_STRAT_AUTO) {
        if (fits)
            s = bitmap < hist ? FC_STRAT_BITMAP : FC_STRAT_HIST;
        else
            s = cells >= o.sort_min_cells ? FC_STRAT_SORT : FC_STRAT_GATOMIC;
    }
    double cost = s == FC_STRAT_BITMAP ? bitmap : s == FC_STRAT_HIST ? hist : gatomic;
    if (s == FC_STRAT_BITMAP) std::copy(ord, ord + k, v);
    return QPlan{s, cost};
}

// Positions 0..n-1 ordered by decreasing key(i) (a positive cost), ties in
// increasing position: a counting sort on the cost's exponent and top three
// mantissa bits (1/8-octave classes), which is as much order as the
// longest-processing-time-first assignment needs and avoids a comparison
// sort's mispredicted branches on thousands of queries.
template <class Key>
void order_by_cost_desc(size_t n, Key key, std::vector<int32_t> &out)
{
    constexpr int kBits = 14;  // 11 exponent + 3 mantissa bits of a positive double
    std::vector<uint32_t> cls(n);
    std::vector<int32_t> start((1 << kBits) + 1, 0);
    for (size_t i = 0; i < n; ++i) {
        double v = key(i);
        if (!(v > 0.0)) v = 0.0;
        uint64_t b;
        std::memcpy(&b, &v, sizeof b);
        cls[i] = ((1u << kBits) - 1u) - (uint32_t)(b >> (52 - 3));  // descending
        ++start[cls[i] + 1];
    }
    for (int c = 0; c < (1 << kBits); ++c) start[c + 1] += start[c];
    out.resize(n);
    for (size_t i = 0; i < n; ++i) out[start[cls[i]]++] = (int32_t)i;
}

// Builds a count or score plan.  vars lists are read through `get`.
template <class GetVars>
int build_count_plan(fc_ctx *c, int32_t nq, GetVars get, const int64_t *user_off, int score_kind,
                     double ess, fc_plan **out)
{
    if (c->transactions) return fail(FC_ERR_STATE, "context holds transaction bitmaps; use the support calls");
    if (nq < 0) return fail(FC_ERR_ARG, "nq < 0");
    fc_plan *p = new (std::nothrow) fc_plan();
    if (!p) return fail(FC_ERR_OOM, "host allocation failed");
    p->ctx = c;
    p->generation = c->generation;
    c->live_plans.push_back(p);
    p->kind = score_kind == kNoScore ? kPlanCount : kPlanScore;
    p->nq = nq;
    p->score_kind = score_kind;
    p->ess = ess;
    const Options &o = c->opt;
    p->threads = std::max(32, std::min(1024, o.threads / 32 * 32));
    const int max_cells = std::max(1, std::min<int>(o.smem_cells, (c->max_smem_optin - 4096) / 4));
    p->smem_cells = max_cells;

    const double chunks_d = (double)((c->m + kChunkRows - 1) / kChunkRows);
    std::vector<QHead> qh(nq);
    std::vector<QVar> qv;
    std::vector<double> cost(nq);
    p->strategy.resize(nq);
    p->table_off.assign(nq + 1, 0);

    // Per query: validation, QVars and strategy.  Large batches split into
    // contiguous query ranges on host threads (each query's work only reads
    // the context); the ranges' QVars are concatenated in query order.
    struct Range {
        std::vector<QVar> qv;
        int32_t err_q = -1;
        int err_code = 0;
        std::string err_msg;
    };
    int nthreads = 1;
    if (nq >= 4096) nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(fc::host_threads(c), nq / 1024));
    std::vector<Range> ranges(nthreads);
    auto work = [&](int t) {
        Range &R = ranges[t];
        const int32_t q0 = (int32_t)((int64_t)nq * t / nthreads), q1 = (int32_t)((int64_t)nq * (t + 1) / nthreads);
        R.qv.reserve((size_t)(q1 - q0) * 4);
        std::vector<int32_t> buf;
        for (int32_t q = q0; q < q1; ++q) {
            const int32_t *vars;
            int32_t k;
            int32_t child;
            if (!get(q, vars, k, child, buf)) {
                R.err_q = q;
                R.err_code = FC_ERR_ARG;
                R.err_msg = g_err;
                return;
            }
            const size_t first = R.qv.size();
            int32_t k_eff = 0;
            const int64_t cells = describe(c, vars, k, R.qv, k_eff);
            if (cells < 0) {
                R.err_q = q;
                R.err_code = (int)cells;
                R.err_msg = g_err;
                return;
            }
            const QPlan ch = choose(c, R.qv.data() + first, k_eff, cells, max_cells, chunks_d);
            QHead &h = qh[q];
            h.cells = (int32_t)cells;
            h.var_off = (int32_t)first;  // within the range for now
            h.k = (int16_t)k_eff;
            h.strategy = (int16_t)ch.strategy;
            h.nparts = 1;
            h.score_kind = (int16_t)score_kind;
            h.r_child = score_kind == kNoScore ? 1 : c->arity[child];
            h.child_soff = score_kind == kNoScore ? 0 : c->soff[child];
            h.score_slot = q;
            p->strategy[q] = ch.strategy;
            cost[q] = ch.cost;
        }
    };
    fc::run_host_threads(c, nthreads, work);
    for (const Range &R : ranges)
        if (R.err_q >= 0) {  // the first failing range holds the lowest failing query
            fc_plan_free(p);
            return fail(R.err_code, "%s", R.err_msg.c_str());
        }
    {
        size_t total = 0;
        for (const Range &R : ranges) total += R.qv.size();
        qv.reserve(total);
        for (int t = 0; t < nthreads; ++t) {
            const int32_t base = (int32_t)qv.size();
            const int32_t q0 = (int32_t)((int64_t)nq * t / nthreads), q1 = (int32_t)((int64_t)nq * (t + 1) / nthreads);
            for (int32_t q = q0; q < q1; ++q) qh[q].var_off += base;
            qv.insert(qv.end(), ranges[t].qv.begin(), ranges[t].qv.end());
        }
    }

    int64_t scratch = 0;
    for (int32_t q = 0; q < nq; ++q) {
        QHead &h = qh[q];
        const int64_t cells = h.cells;
        if (score_kind == kNoScore) {
            if (user_off) {
                if (user_off[q + 1] - user_off[q] < cells || user_off[q] < 0) {
                    fc_plan_free(p);
                    return fail(FC_ERR_ARG, "table_off of query %d leaves %lld cells, it needs %lld", q,
                                (long long)(user_off[q + 1] - user_off[q]), (long long)cells);
                }
                p->table_off[q] = user_off[q];
            } else {
                p->table_off[q] = scratch;
                scratch += cells;
            }
            h.table_off = p->table_off[q];
        }
        if (user_off) p->table_off[nq] = user_off[nq];
        else p->table_off[nq] = scratch;
    }
    if (score_kind == kNoScore) p->out_cells = p->table_off[nq];

    // work items: split rows when the batch alone cannot fill the GPU
    const size_t smem_bytes = (size_t)max_cells * 4;
    int per_sm = std::max(1, o.ctas_per_sm);
    p->grid = c->num_sms * per_sm;
    p->smem = smem_bytes;
    const int64_t nchunks = (c->m + kChunkRows - 1) / kChunkRows;
    const int64_t max_parts_rows = std::max<int64_t>(1, c->m / std::max<int64_t>(o.min_part_rows, kChunkRows));
    int32_t persistent = 0;
    for (int32_t q = 0; q < nq; ++q)
        if (qh[q].strategy == kHist || qh[q].strategy == kGAtomic) ++persistent;
    // (marginal items hold no rows, so they never split)
    const int64_t target = (int64_t)p->grid * 4;
    int64_t parts = 1;
    if (persistent > 0 && persistent < target)
        parts = std::min<int64_t>({nchunks, max_parts_rows, (target + persistent - 1) / persistent, 32767});
    parts = std::max<int64_t>(1, parts);
    std::vector<Item> items;
    std::vector<int32_t> hq;  // queries that become work items of count_kernel
    std::vector<int32_t> qlist;
    std::vector<std::pair<double, int32_t>> bmo;
    hq.reserve(nq);
    size_t n_items = 0;
    for (int32_t q = 0; q < nq; ++q) {
        QHead &h = qh[q];
        if (h.strategy == kSort) {
            p->sort_jobs.push_back(SortJob{q, h.k, 0, h.cells, 0, nullptr});
            continue;
        }
        if (h.strategy == kBitmap) {
            bmo.push_back({cost[q], q});
            continue;
        }
        const int64_t qparts = h.strategy == kMarginal ? 1 : parts;
        h.nparts = (int16_t)qparts;
        hq.push_back(q);
        n_items += (size_t)qparts;
    }
    // heaviest first by cost per part; a query's parts are consecutive, and
    // within a cost class queries keep their order
    std::vector<int32_t> perm;
    order_by_cost_desc(hq.size(), [&](size_t i) { return cost[hq[i]] / qh[hq[i]].nparts; }, perm);
    items.reserve(n_items);
    for (int32_t i : perm) {
        const int32_t q = hq[i];
        for (int32_t part = 0; part < qh[q].nparts; ++part) items.push_back(Item{q, part});
    }
    p->n_items = (int32_t)items.size();
    // bitmap queries: warp tasks of consecutive 4096-row chunks, heaviest
    // queries first.  A query gets tasks in proportion to its estimated cost
    // (about four tasks' worth of work per warp of the launch), each of at
    // least kMinTaskChunks chunks, so that light queries are not cut into
    // tasks whose fixed costs (dispatch, one reduction and atomic per cell)
    // outweigh their work.
    {
        order_by_cost_desc(bmo.size(), [&](size_t i) { return bmo[i].first; }, perm);
        std::vector<std::pair<double, int32_t>> sorted;
        sorted.reserve(bmo.size());
        for (int32_t i : perm) sorted.push_back(bmo[i]);
        bmo.swap(sorted);
    }
    std::vector<BTask> btasks;
    btasks.reserve(bmo.size() * 4);
    p->bm_threads = std::max(32, std::min(1024, o.bitmap_threads / 32 * 32));
    p->stage_slots = o.stage_slots;
    p->small_paths = o.bitmap_small;
    if (!bmo.empty()) {
        constexpr int64_t kMinTaskChunks = 4;
        p->bm_grid = c->num_sms * bitmap_ctas_per_sm(p->bm_threads, p->stage_slots);
        const int64_t warps = (int64_t)p->bm_grid * (p->bm_threads / 32);
        double total = 0.0;
        for (auto &x : bmo) total += x.first;
        const double unit = std::max(total / (4.0 * (double)warps), 1e-30);
        const int64_t max_tasks = std::max<int64_t>(1, std::min<int64_t>(nchunks / kMinTaskChunks, 32767));
        for (auto &x : bmo) {
            const int32_t q = x.second;
            // a 3-variable register-blocked query splits by the first
            // variable's state as well (one pass over the chunks per state)
            const QVar *ov = qv.data() + qh[q].var_off;
            const int32_t passes = (p->small_paths && qh[q].k == 3 && small_ok(ov, 3)) ? ov[0].arity : 0;
            const double per = x.first / std::max(1, passes);
            const int64_t t = std::max<int64_t>(1, std::min<int64_t>(max_tasks, (int64_t)std::ceil(per / unit)));
            qh[q].nparts = (int16_t)std::min<int64_t>(t * std::max(1, passes), 32767);
            // t balanced chunk ranges: the first nchunks % t get one extra chunk
            const int64_t base = nchunks / t, rem = nchunks % t;
            for (int32_t s0 = passes > 0 ? 0 : -1; s0 < std::max(passes, 0); ++s0) {
                int64_t c0 = 0;
                for (int64_t part = 0; part < t; ++part) {
                    const int64_t c1 = c0 + base + (part < rem ? 1 : 0);
                    btasks.push_back(BTask{q, (int32_t)c0, (int32_t)c1, s0});
                    c0 = c1;
                }
            }
        }
    }
    p->n_btasks = (int32_t)btasks.size();

    // tables that must exist in global memory for score plans
    if (score_kind != kNoScore) {
        for (int32_t q = 0; q < nq; ++q) {
            QHead &h = qh[q];
            const bool global = (h.strategy != kHist && h.strategy != kMarginal) || h.nparts > 1;
            if (global) {
                h.table_off = scratch;
                scratch += h.cells;
            } else {
                h.table_off = 0;
            }
        }
        p->table_buf_cells = scratch;
    } else {
        p->table_buf_cells = p->out_cells;
    }
    for (int32_t q = 0; q < nq; ++q) {
        const QHead &h = qh[q];
        if ((h.strategy != kHist && h.strategy != kMarginal) || h.nparts > 1) p->zero_tables = true;
    }
    for (auto &j : p->sort_jobs) {
        j.table_off = qh[j.q].table_off;
        j.key_bits = j.cells > 1 ? 32 - __builtin_clz((uint32_t)(j.cells - 1)) : 0;
        if (score_kind != kNoScore) qlist.push_back(j.q);
    }
    p->n_qlist = (int32_t)qlist.size();

    // one device allocation for all descriptors
    const size_t b_qh = sizeof(QHead) * std::max(nq, 1);
    const size_t b_qv = sizeof(QVar) * std::max<size_t>(qv.size(), 1);
    const size_t b_it = sizeof(Item) * std::max<size_t>(items.size(), 1);
    const size_t b_ql = sizeof(int32_t) * std::max<size_t>(qlist.size(), 1);
    const size_t b_bq = sizeof(BTask) * std::max<size_t>(btasks.size(), 1);
    const size_t o_qv = round_up(b_qh, 256), o_it = o_qv + round_up(b_qv, 256), o_ql = o_it + round_up(b_it, 256);
    const size_t o_bq = o_ql + round_up(b_ql, 256);
    const size_t total = o_bq + round_up(b_bq, 256);
    uint8_t *host = stage_host(c, total);
    if (!host) {
        fc_plan_free(p);
        return fail(FC_ERR_OOM, "pinned staging of %zu bytes", total);
    }
    std::memcpy(host, qh.data(), sizeof(QHead) * nq);
    std::memcpy(host + o_qv, qv.data(), sizeof(QVar) * qv.size());
    std::memcpy(host + o_it, items.data(), sizeof(Item) * items.size());
    std::memcpy(host + o_ql, qlist.data(), sizeof(int32_t) * qlist.size());
    std::memcpy(host + o_bq, btasks.data(), sizeof(BTask) * btasks.size());
    cudaError_t e = plan_buf(c, p->desc, 0, total);
    if (e == cudaSuccess) e = upload_stage(c, p->desc.p, total);
    p->upload_bytes = total;
    p->n_counters = 2 + nq;
    if (e == cudaSuccess) e = plan_buf(c, p->counters, 1, sizeof(int32_t) * p->n_counters);
    if (e == cudaSuccess && score_kind != kNoScore)
        e = plan_buf(c, p->scratch_tables, 2, sizeof(int32_t) * std::max<int64_t>(p->table_buf_cells, 1));
    if (e == cudaSuccess && !p->sort_jobs.empty()) {
        const int tile = sort_tile_rows();
        const int64_t nb = (c->m + tile - 1) / tile;
        const size_t kb = round_up(sizeof(uint32_t) * c->m, 256);
        e = plan_buf(c, p->sort_mem, 3, 2 * kb + sizeof(uint32_t) * 256 * nb);
        if (e == cudaSuccess) {
            uint8_t *base = (uint8_t *)p->sort_mem.p;
            p->sort_sc.keys_a = (uint32_t *)base;
            p->sort_sc.keys_b = (uint32_t *)(base + kb);
            p->sort_sc.block_hist = (uint32_t *)(base + 2 * kb);
            p->sort_sc.cap_rows = c->m;
            p->sort_sc.cap_blocks = (int32_t)nb;
        }
    }
    // a plan lent to a synchronous call runs on the context stream, after
    // its upload; a plan the caller keeps may run on any stream, so its
    // upload must be complete on return
    if (e == cudaSuccess && !c->borrow) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fc_plan_free(p);
        return cuda_fail(e, "plan upload");
    }
    uint8_t *d = (uint8_t *)p->desc.p;
    p->d_qh = (QHead *)d;
    p->d_qv = (QVar *)(d + o_qv);
    p->d_items = (Item *)(d + o_it);
    p->d_qlist = (int32_t *)(d + o_ql);
    p->d_btasks = (BTask *)(d + o_bq);
    for (auto &j : p->sort_jobs) j.d_vars = p->d_qv + qh[j.q].var_off;
    *out = p;
    return FC_OK;
}

// Enqueues the work of a count/score plan on stream s.
cudaError_t enqueue_count(fc_plan *p, int32_t *tables, float *scores, cudaStream_t s)
{
    fc_ctx *c = p->ctx;
    cudaError_t e = cudaMemsetAsync(p->counters.p, 0, sizeof(int32_t) * p->n_counters, s);
    if (e != cudaSuccess) return e;
    int32_t *tab = p->kind == kPlanScore ? (int32_t *)p->scratch_tables.p : tables;
    if (p->zero_tables && p->table_buf_cells > 0) {
        e = cudaMemsetAsync(tab, 0, sizeof(int32_t) * p->table_buf_cells, s);
        if (e != cudaSuccess) return e;
    }
    if (p->n_items > 0 || p->n_btasks > 0) {
        CountParams P{};
        P.D = c->d_D;
        P.m_pad = c->m_pad;
        P.m = c->m;
        P.bits = c->d_bits;
        P.wstride = c->wstride;
        P.qh = p->d_qh;
        P.qv = p->d_qv;
        P.items = p->d_items;
        P.n_items = p->n_items;
        P.next_item = (int32_t *)p->counters.p;
        P.next_task = (int32_t *)p->counters.p + 1;
        P.tickets = (int32_t *)p->counters.p + 2;
        P.btasks = p->d_btasks;
        P.n_btasks = p->n_btasks;
        P.stage_slots = p->stage_slots;
        P.tables = tab;
        P.scores = scores;
        P.marg = c->d_marg;
        P.ess = p->ess;
        P.write_tables = p->kind == kPlanCount ? 1 : 0;
        P.smem_cells = p->smem_cells;
        P.hist_copies = c->opt.hist_copies;
        P.small_paths = p->small_paths;
        if (p->n_btasks > 0) {
            e = launch_bitmap(P, p->bm_grid, p->bm_threads, s);
            if (e != cudaSuccess) return e;
        }
        if (p->n_items > 0) {
            const int grid = std::min<int64_t>(p->grid, std::max(p->n_items, 1));
            e = launch_count(P, grid, p->threads, p->smem, s);
            if (e != cudaSuccess) return e;
        }
    }
    for (const SortJob &j : p->sort_jobs) {
        e = launch_sort_count(c->d_D, c->m_pad, c->m, j.d_vars, j.k, j.key_bits, tab + j.table_off,
                              j.cells, 0, p->sort_sc, s);
        if (e != cudaSuccess) return e;
    }
    if (p->kind == kPlanScore && p->n_qlist > 0)
        e = launch_score_global(p->d_qh, p->d_qlist, p->n_qlist, tab, scores, c->d_marg, c->m, p->ess, s);
    return e;
}

cudaError_t enqueue_support(fc_plan *p, int32_t *support, int32_t *sub, float *conf, cudaStream_t s);
cudaError_t enqueue_pairs(fc_plan *p, int32_t *pairs, float *mi, cudaStream_t s);

cudaError_t enqueue_families(fc_plan *p, float *scores, cudaStream_t s)
{
    fc_ctx *c = p->ctx;
    cudaError_t e = enqueue_count(p->inner, (int32_t *)p->fam_tables.p, nullptr, s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(p->n_jobs, (int64_t)c->num_sms * 16);
    return launch_family_scores((const FamilyJob *)p->fam_jobs.p, p->n_jobs, (const int32_t *)p->fam_tables.p,
                                c->d_arity, c->d_soff, c->d_marg, c->m, p->fam_kind, p->ess, scores, grid, s);
}

cudaError_t enqueue(fc_plan *p, void *o0, void *o1, void *o2, cudaStream_t s)
{
    switch (p->kind) {
    case kPlanCount: return enqueue_count(p, (int32_t *)o0, nullptr, s);
    case kPlanScore: return enqueue_count(p, nullptr, (float *)o0, s);
    case kPlanSupport: return enqueue_support(p, (int32_t *)o0, (int32_t *)o1, (float *)o2, s);
    case kPlanPairs: return enqueue_pairs(p, (int32_t *)o0, (float *)o1, s);
    case kPlanFamilies: return enqueue_families(p, (float *)o0, s);
    }
    return cudaErrorInvalidValue;
}

int run_plan(fc_plan *p, void *o0, void *o1, void *o2, cudaStream_t s, bool allow_graph)
{
    fc_ctx *c = p->ctx;
    if (!s) s = c->stream;
    if (!(allow_graph && c->opt.use_graph)) {
        cudaError_t e = enqueue(p, o0, o1, o2, s);
        if (e != cudaSuccess) return cuda_fail(e, "plan run");
        return FC_OK;
    }
    for (auto &g : p->graphs)
        if (g.o0 == o0 && g.o1 == o1 && g.o2 == o2 && g.s == s) {
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            return FC_OK;
        }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    cudaError_t e2 = enqueue(p, o0, o1, o2, s);
    e = cudaStreamEndCapture(s, &graph);
    if (e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e2, "plan capture");
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    p->graphs.push_back(GraphEntry{o0, o1, o2, s, exec});
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    return FC_OK;
}

int read_status(fc_ctx *c, cudaStream_t s)
{
    int32_t st[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(st, c->d_status, sizeof st, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "status");
    if (st[0] != kStatusOk) {
        cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), s);
        cudaStreamSynchronize(s);
        return fail(FC_ERR_TIMEOUT, "a bounded device wait ran out (status %d)", st[0]);
    }
    return FC_OK;
}

// Runs a plan on the context stream with runtime-owned device outputs and
// copies them to the caller's host buffers.
int run_to_host(fc_plan *p, void *h0, size_t b0, void *h1, size_t b1, void *h2, size_t b2)
{
    fc_ctx *c = p->ctx;
    void *hs[3] = {h0, h1, h2};
    size_t bs[3] = {b0, b1, b2};
    void *ds[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i) {
        if (!hs[i] || bs[i] == 0) continue;
        cudaError_t e = c->io[i].ensure(bs[i]);
        if (e != cudaSuccess) return cuda_fail(e, "output buffer");
        ds[i] = c->io[i].p;
    }
    int rc = run_plan(p, ds[0], ds[1], ds[2], c->stream, false);
    if (rc != FC_OK) return rc;
    for (int i = 0; i < 3; ++i)
        if (ds[i]) {
            cudaError_t e = cudaMemcpyAsync(hs[i], ds[i], bs[i], cudaMemcpyDeviceToHost, c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "copy outputs");
        }
    return read_status(c, c->stream);
}

}  // namespace

// ------------------------------------------------------------- plan API

extern "C" int fc_plan_count(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                             const int64_t *table_off, fc_plan **out)
{
    if (!c || !out || (nq > 0 && (!var_off || !vars))) return fail(FC_ERR_ARG, "fc_plan_count: null argument");
    *out = nullptr;
    DevGuard g(c->device);
    if (table_off)
        for (int32_t q = 0; q < nq; ++q)
            if (table_off[q + 1] < table_off[q]) return fail(FC_ERR_ARG, "table_off must be non-decreasing");
    auto get = [&](int32_t q, const int32_t *&v, int32_t &k, int32_t &child, std::vector<int32_t> &) {
        const int32_t a = var_off[q], b = var_off[q + 1];
        if (a < 0 || b < a) {
            fail(FC_ERR_ARG, "var_off must be non-decreasing and non-negative");
            return false;
        }
        v = vars + a;
        k = b - a;
        child = -1;
        return true;
    };
    return build_count_plan(c, nq, get, table_off, kNoScore, 1.0, out);
}

extern "C" int fc_plan_score(fc_ctx *c, int32_t nq, const int32_t *child, const int32_t *par_off,
                             const int32_t *parents, int32_t kind, double ess, fc_plan **out)
{
    if (!c || !out || (nq > 0 && (!child || !par_off))) return fail(FC_ERR_ARG, "fc_plan_score: null argument");
    *out = nullptr;
    if (kind < FC_LL || kind > FC_MI) return fail(FC_ERR_ARG, "unknown score kind %d", kind);
    if (kind == FC_BDEU && !(ess > 0.0)) return fail(FC_ERR_ARG, "BDeu needs ess > 0");
    DevGuard g(c->device);
    auto get = [&](int32_t q, const int32_t *&v, int32_t &k, int32_t &ch, std::vector<int32_t> &buf) {
        const int32_t a = par_off[q], b = par_off[q + 1];
        if (a < 0 || b < a || (b > a && !parents)) {
            fail(FC_ERR_ARG, "par_off must be non-decreasing and non-negative");
            return false;
        }
        if (child[q] < 0 || child[q] >= c->n) {
            fail(FC_ERR_ARG, "child %d out of range", child[q]);
            return false;
        }
        buf.assign(parents + a, parents + b);
        buf.push_back(child[q]);
        v = buf.data();
        k = (int32_t)buf.size();
        ch = child[q];
        return true;
    };
    return build_count_plan(c, nq, get, nullptr, kind, ess, out);
}

namespace {
// Kernels one fc_plan_run launches when every output is given (memsets and
// graph bookkeeping excluded).
int64_t plan_launches(const fc_plan *p)
{
    switch (p->kind) {
    case kPlanCount:
    case kPlanScore:
        return (p->n_btasks > 0) + (p->n_items > 0) + (int64_t)p->sort_jobs.size() +
               (p->kind == kPlanScore && p->n_qlist > 0);
    case kPlanSupport: return p->nq > 0 ? (p->sp.full_only ? 1 : 2) : 0;
    case kPlanPairs: return 2;
    case kPlanFamilies: return plan_launches(p->inner) + (p->n_jobs > 0);
    }
    return 0;
}
}  // namespace

extern "C" int64_t fc_plan_size(const fc_plan *p, int32_t key)
{
    if (!p) return -1;
    switch (key) {
    case 0: return p->kind == kPlanPairs ? p->pair_cells : p->out_cells;
    case 1: return p->kind == kPlanScore ? p->nq : p->kind == kPlanPairs ? p->n_pairs
                 : p->kind == kPlanFamilies ? p->n_jobs : 0;
    case 2: return p->kind == kPlanSupport ? p->nq : 0;
    case 3: return p->kind == kPlanSupport ? p->n_sub : 0;
    case 4: return p->nq;
    case 5: return (int64_t)p->upload_bytes;
    case 6: return plan_launches(p);
    default: return -1;
    }
}

extern "C" int fc_plan_table_offsets(const fc_plan *p, int64_t *off)
{
    if (!p || !off) return fail(FC_ERR_ARG, "fc_plan_table_offsets: null argument");
    if (p->kind != kPlanCount) return fail(FC_ERR_STATE, "not a count plan");
    std::memcpy(off, p->table_off.data(), sizeof(int64_t) * (p->nq + 1));
    return FC_OK;
}

extern "C" int fc_plan_strategies(const fc_plan *p, int32_t *s)
{
    if (!p || !s) return fail(FC_ERR_ARG, "fc_plan_strategies: null argument");
    if (p->kind != kPlanCount && p->kind != kPlanScore) return fail(FC_ERR_STATE, "not a count or score plan");
    std::memcpy(s, p->strategy.data(), sizeof(int32_t) * p->nq);
    return FC_OK;
}

extern "C" int fc_plan_run(fc_plan *p, void *o0, void *o1, void *o2, void *stream)
{
    if (!p) return fail(FC_ERR_ARG, "fc_plan_run: null plan");
    if (!p->ctx) return fail(FC_ERR_STATE, "fc_plan_run: the plan's context was freed");
    if (p->generation != p->ctx->generation)
        return fail(FC_ERR_STATE, "fc_plan_run: instances were appended since the plan was built; build a new plan");
    DevGuard g(p->ctx->device);
    if ((p->kind == kPlanCount && p->out_cells > 0 && !o0) || (p->kind == kPlanScore && p->nq > 0 && !o0) ||
        (p->kind == kPlanFamilies && p->n_jobs > 0 && !o0) ||
        (p->kind == kPlanSupport && p->nq > 0 && !o0))
        return fail(FC_ERR_ARG, "fc_plan_run: missing output buffer");
    return run_plan(p, o0, o1, o2, (cudaStream_t)stream, true);
}

namespace {
// Device resources of a plan (its graphs and buffers); the caller has made
// the plan's device current.
void release_plan(fc_plan *p)
{
    cudaStreamSynchronize(p->ctx->stream);
    for (auto &gr : p->graphs) {
        cudaStreamSynchronize(gr.s);
        cudaGraphExecDestroy(gr.exec);
    }
    p->graphs.clear();
    p->desc.release();
    p->counters.release();
    p->scratch_tables.release();
    p->sort_mem.release();
    p->pairs_C.release();
    p->pairs_meta.release();
    p->fam_tables.release();
    p->fam_jobs.release();
}
}  // namespace

extern "C" void fc_plan_free(fc_plan *p)
{
    if (!p) return;
    if (p->ctx) {  // still attached: release here (an orphan was released by fc_free)
        fc_ctx *c = p->ctx;
        DevGuard g(c->device);
        release_plan(p);
        auto &lp = c->live_plans;
        lp.erase(std::remove(lp.begin(), lp.end(), p), lp.end());
    }
    if (p->inner) fc_plan_free(p->inner);
    delete p;
}

extern "C" int fc_sync(fc_ctx *c, void *stream)
{
    if (!c) return fail(FC_ERR_ARG, "fc_sync: null context");
    DevGuard g(c->device);
    if (stream) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    }
    return read_status(c, c->stream);
}

// ------------------------------------------------------- host entry points

extern "C" int fc_count(fc_ctx *c, const int32_t *vars, int32_t k, int32_t *table)
{
    if (!c || !table || (k > 0 && !vars)) return fail(FC_ERR_ARG, "fc_count: null argument");
    int32_t off[2] = {0, k};
    return fc_count_batch(c, 1, off, vars, nullptr, table);
}

extern "C" int fc_count_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                              const int64_t *table_off, int32_t *tables)
{
    if (!c || (nq > 0 && !tables)) return fail(FC_ERR_ARG, "fc_count_batch: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_count(c, nq, var_off, vars, table_off, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, tables, sizeof(int32_t) * p->out_cells, nullptr, 0, nullptr, 0);
    fc_plan_free(p);
    return rc;
}

extern "C" int fc_score_batch(fc_ctx *c, int32_t nq, const int32_t *child, const int32_t *par_off,
                              const int32_t *parents, int32_t kind, double ess, float *scores)
{
    if (!c || (nq > 0 && !scores)) return fail(FC_ERR_ARG, "fc_score_batch: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_score(c, nq, child, par_off, parents, kind, ess, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, scores, sizeof(float) * nq, nullptr, 0, nullptr, 0);
    fc_plan_free(p);
    return rc;
}

extern "C" int fc_count_assignment(fc_ctx *c, const int32_t *vars, const int32_t *states, int32_t k,
                                   int64_t *count)
{
    if (!c || !count || (k > 0 && (!vars || !states))) return fail(FC_ERR_ARG, "fc_count_assignment: null argument");
    if (c->transactions) return fail(FC_ERR_STATE, "context holds transaction bitmaps");
    if (k < 0 || k > c->n) return fail(FC_ERR_ARG, "bad k");
    DevGuard g(c->device);
    std::vector<int32_t> rows;
    for (int t = 0; t < k; ++t) {
        if (vars[t] < 0 || vars[t] >= c->n) return fail(FC_ERR_ARG, "variable %d out of range", vars[t]);
        if (states[t] < 0 || states[t] >= c->arity[vars[t]]) {
            *count = 0;
            return FC_OK;
        }
        rows.push_back(c->soff[vars[t]] + states[t]);
    }
    if (k == 0) {
        *count = c->m;
        return FC_OK;
    }
    cudaError_t e = c->io[0].ensure(sizeof(unsigned long long) + sizeof(int32_t) * k + 64);
    if (e != cudaSuccess) return cuda_fail(e, "scratch");
    unsigned long long *d_cnt = (unsigned long long *)c->io[0].p;
    int32_t *d_rows = (int32_t *)((uint8_t *)c->io[0].p + 64);
    cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), c->stream);
    cudaMemcpyAsync(d_rows, rows.data(), sizeof(int32_t) * k, cudaMemcpyHostToDevice, c->stream);
    e = launch_assignment_count(c->d_bits, c->wstride, d_rows, k, c->words, d_cnt, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "assignment count");
    unsigned long long h = 0;
    e = cudaMemcpyAsync(&h, d_cnt, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "assignment count");
    *count = (int64_t)h;
    return FC_OK;
}

// ----------------------------------------------------------------- support

namespace {

cudaError_t enqueue_support(fc_plan *p, int32_t *support, int32_t *sub, float *conf, cudaStream_t s)
{
    SupportParams P = p->sp;
    P.support = support;
    P.sub_support = sub ? sub : (int32_t *)p->scratch_tables.p;
    P.confidence = P.full_only ? nullptr : conf;
    if (P.full_only) conf = nullptr;
    P.next_item = (int32_t *)p->counters.p;
    cudaError_t e = cudaMemsetAsync(p->counters.p, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    if (P.nparts > 1) {
        if ((e = cudaMemsetAsync(support, 0, sizeof(int32_t) * p->nq, s)) != cudaSuccess) return e;
        if (p->n_sub > 0 && (e = cudaMemsetAsync(P.sub_support, 0, sizeof(int32_t) * p->n_sub, s)) != cudaSuccess)
            return e;
    }
    if (p->nq == 0) return cudaSuccess;
    e = launch_support(P, p->sup_grid, p->sup_threads, 0, s);
    if (e != cudaSuccess) return e;
    if (conf) e = launch_support_confidence(P, s);
    return e;
}

}  // namespace

namespace {
int build_set_plan(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items, int mode,
                   fc_plan **out);
}  // namespace

namespace {
int plan_itemsets(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items, int mode, fc_plan **out);
}  // namespace

extern "C" int fc_plan_support(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items,
                               fc_plan **out)
{
    return plan_itemsets(c, nq, set_off, items, 0, out);
}

extern "C" int fc_plan_support_splits(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items,
                                      fc_plan **out)
{
    return plan_itemsets(c, nq, set_off, items, 2, out);
}

namespace {
// Validated itemset plan: mode 0 = supports with leave-one-out sets, 2 = every
// antecedent split.
int plan_itemsets(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items, int mode, fc_plan **out)
{
    if (!c || !out || (nq > 0 && !set_off)) return fail(FC_ERR_ARG, "fc_plan_support: null argument");
    *out = nullptr;
    if (!c->transactions) return fail(FC_ERR_STATE, "support queries need a context from fc_load_bits");
    if (nq < 0) return fail(FC_ERR_ARG, "nq < 0");
    DevGuard g(c->device);
    if (nq > 0 && set_off[0] != 0) return fail(FC_ERR_ARG, "set_off[0] must be 0");
    const int32_t kmax = mode == 2 ? kMaxSplitK : kMaxK;
    for (int32_t q = 0; q < nq; ++q) {
        const int32_t a = set_off[q], b = set_off[q + 1];
        if (b < a) return fail(FC_ERR_ARG, "set_off must be non-decreasing");
        if (b - a > kmax) return fail(FC_ERR_SIZE, "itemset %d has %d items, at most %d supported", q, b - a, kmax);
        if (b > a && !items) return fail(FC_ERR_ARG, "null items");
        if (++c->epoch == 0) {
            std::fill(c->mark.begin(), c->mark.end(), 0u);
            c->epoch = 1;
        }
        for (int32_t t = a; t < b; ++t) {
            const int32_t it = items[t];
            if (it < 0 || it >= c->n) return fail(FC_ERR_ARG, "item %d out of range", it);
            if (c->mark[it] == c->epoch) return fail(FC_ERR_ARG, "item %d listed twice in itemset %d", it, q);
            c->mark[it] = c->epoch;
        }
    }
    return build_set_plan(c, nq, set_off, items, mode, out);
}
}  // namespace

namespace {

// CTAs of a support-family kernel per SM (cached per device, mode, block size).
int support_ctas_per_sm(int mode, int threads)
{
    static std::mutex mu;
    static int cache[64][3][33];
    int dev = 0;
    cudaGetDevice(&dev);
    const int ti = std::min(32, threads / 32);
    if (dev >= 0 && dev < 64 && mode >= 0 && mode < 3) {
        std::lock_guard<std::mutex> lk(mu);
        if (cache[dev][mode][ti] > 0) return cache[dev][mode][ti];
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, support_kernel_ptr(mode), threads, 0);
    per_sm = std::max(1, per_sm);
    if (dev >= 0 && dev < 64 && mode >= 0 && mode < 3) {
        std::lock_guard<std::mutex> lk(mu);
        cache[dev][mode][ti] = per_sm;
    }
    return per_sm;
}

// A plan over sets of bitmap rows: itemset supports with their leave-one-out
// supports (mode 0), the support of each set alone (mode 1, specific-
// assignment counts), or the supports of every antecedent split (mode 2).
// set_off[0] == 0 and the rows are valid.
int build_set_plan(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items, int mode,
                   fc_plan **out)
{
    const int full_only = mode == 1;
    fc_plan *p = new (std::nothrow) fc_plan();
    if (!p) return fail(FC_ERR_OOM, "host allocation failed");
    p->ctx = c;
    p->generation = c->generation;
    c->live_plans.push_back(p);
    p->kind = kPlanSupport;
    p->nq = nq;
    const int64_t n_sub = nq > 0 ? set_off[nq] : 0;
    p->n_sub = full_only ? 0 : n_sub;
    std::vector<int64_t> split_off;
    if (mode == 2) {
        split_off.assign(nq + 1, 0);
        for (int32_t q = 0; q < nq; ++q) {
            const int k = set_off[q + 1] - set_off[q];
            split_off[q + 1] = split_off[q] + std::max<int64_t>(((int64_t)1 << k) - 2, 0);
        }
        p->n_sub = split_off[nq];
    }
    const Options &o = c->opt;
    // itemsets in decreasing size so that the heavy ones start first
    std::vector<int32_t> order(nq);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return set_off[a + 1] - set_off[a] > set_off[b + 1] - set_off[b];
    });
    const size_t b_off = sizeof(int32_t) * (nq + 1), b_it = sizeof(int32_t) * std::max<int64_t>(n_sub, 1);
    const size_t o_it = round_up(b_off, 256), o_ord = o_it + round_up(b_it, 256);
    const size_t o_spl = o_ord + round_up(sizeof(int32_t) * std::max(nq, 1), 256);
    const size_t total = o_spl + (mode == 2 ? round_up(sizeof(int64_t) * (nq + 1), 256) : 0);
    uint8_t *host = stage_host(c, total);
    if (!host) {
        fc_plan_free(p);
        return fail(FC_ERR_OOM, "pinned staging of %zu bytes", total);
    }
    if (nq > 0) {
        std::memcpy(host, set_off, b_off);
        if (n_sub > 0) std::memcpy(host + o_it, items, sizeof(int32_t) * n_sub);
        std::memcpy(host + o_ord, order.data(), sizeof(int32_t) * nq);
    }
    if (mode == 2) std::memcpy(host + o_spl, split_off.data(), sizeof(int64_t) * (nq + 1));
    cudaError_t e = plan_buf(c, p->desc, 0, total);
    if (e == cudaSuccess) e = upload_stage(c, p->desc.p, total);
    p->upload_bytes = total;
    if (e == cudaSuccess) e = plan_buf(c, p->counters, 1, 16);
    if (e == cudaSuccess) e = plan_buf(c, p->scratch_tables, 2, sizeof(int32_t) * std::max<int64_t>(p->n_sub, 1));
    // a plan lent to a synchronous call runs on the context stream, after
    // its upload; a plan the caller keeps may run on any stream, so its
    // upload must be complete on return
    if (e == cudaSuccess && !c->borrow) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fc_plan_free(p);
        return cuda_fail(e, "plan upload");
    }
    SupportParams &P = p->sp;
    uint8_t *d = (uint8_t *)p->desc.p;
    P.bits = c->d_bits;
    P.wstride = c->wstride;
    P.words = c->words;
    P.set_off = (const int32_t *)d;
    P.items = (const int32_t *)(d + o_it);
    P.order = (const int32_t *)(d + o_ord);
    P.nq = nq;
    P.n_items = c->n;
    p->sup_threads = std::max(1, std::min(32, o.support_warps)) * 32;
    P.sets_per_item = (p->sup_threads / 32) * std::max(1, o.support_sets_per_warp);
    P.m_tail = c->m;
    P.full_only = full_only;
    P.all_splits = mode == 2;
    P.split_off = mode == 2 ? (const int64_t *)(d + o_spl) : nullptr;
    if (full_only) p->sup_threads = std::min(p->sup_threads, 512);
    if (mode == 2) {
        p->sup_threads = std::min(p->sup_threads, 256);
        P.sets_per_item = (p->sup_threads / 32) * std::max(1, o.support_sets_per_warp);
    }
    p->sup_grid = c->num_sms * support_ctas_per_sm(mode, p->sup_threads);
    // word ranges of whole 64-word steps (32 lanes x 2 words): at most
    // support_part_words each, and more of them when the batch has too few
    // itemset groups to give every CTA two work items (a small rule-miner
    // level, a handful of long itemsets)
    const int64_t part_words = std::max<int64_t>(64, round_up(o.support_part_words, 64));
    const int64_t ngroups = std::max<int64_t>(1, ((int64_t)nq + P.sets_per_item - 1) / P.sets_per_item);
    int64_t nparts = std::max<int64_t>(1, (c->words + part_words - 1) / part_words);
    const int64_t want = (2 * (int64_t)p->sup_grid + ngroups - 1) / ngroups;
    nparts = std::max(nparts, std::min(want, std::max<int64_t>(1, (c->words + 63) / 64)));
    P.nparts = (int32_t)std::min<int64_t>(nparts, 1 << 20);
    P.words_per_part = (int32_t)round_up((c->words + P.nparts - 1) / P.nparts, 64);
    *out = p;
    return FC_OK;
}

}  // namespace

extern "C" int fc_plan_assignments(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                                   const int32_t *states, fc_plan **out)
{
    if (!c || !out || (nq > 0 && !var_off)) return fail(FC_ERR_ARG, "fc_plan_assignments: null argument");
    *out = nullptr;
    if (c->transactions) return fail(FC_ERR_STATE, "assignment counts need a categorical context");
    if (nq < 0) return fail(FC_ERR_ARG, "nq < 0");
    DevGuard g(c->device);
    if (nq > 0 && var_off[0] != 0) return fail(FC_ERR_ARG, "var_off[0] must be 0");
    std::vector<int32_t> rows;
    for (int32_t q = 0; q < nq; ++q) {
        const int32_t a = var_off[q], b = var_off[q + 1];
        if (b < a) return fail(FC_ERR_ARG, "var_off must be non-decreasing");
        if (b - a > kMaxK) return fail(FC_ERR_SIZE, "assignment %d has %d conditions, at most %d supported", q, b - a, kMaxK);
        if (b > a && (!vars || !states)) return fail(FC_ERR_ARG, "null vars or states");
        for (int32_t t = a; t < b; ++t) {
            const int32_t v = vars[t];
            if (v < 0 || v >= c->n) return fail(FC_ERR_ARG, "variable %d out of range", v);
            // a state outside the arity matches nothing: the all-zero row R
            rows.push_back(states[t] >= 0 && states[t] < c->arity[v] ? c->soff[v] + states[t] : c->R);
        }
    }
    return build_set_plan(c, nq, var_off, rows.data(), 1, out);
}

int fc::host_threads(fc_ctx *c)
{
    if (!c->pool_threads) {
        const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
        c->pool_threads.reset(new (std::nothrow) PlanPool());
        if (c->pool_threads) c->pool_threads->start(std::max(0, std::min(7, hw - 1)));
    }
    return c->pool_threads ? c->pool_threads->size() : 1;
}

void fc::run_host_threads(fc_ctx *c, int n, const std::function<void(int)> &f)
{
    if (n <= 1 || !c->pool_threads) {
        for (int i = 0; i < std::max(n, 0); ++i) f(i);
        return;
    }
    c->pool_threads->run(std::min(n, c->pool_threads->size()), f);
}

void fc::itemset_universe(const fc_ctx *c, int32_t *n_items, int64_t *m)
{
    *n_items = c->R;
    *m = c->m;
}

void fc::item_groups(const fc_ctx *c, int32_t *group, int64_t *support)
{
    for (int32_t v = 0; v < c->n; ++v)
        for (int32_t s = 0; s < c->arity[v]; ++s) group[c->soff[v] + s] = v;
    std::copy(c->marg.begin(), c->marg.end(), support);
}

int fc::count_itemsets(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *rows, int32_t *counts,
                       ItemsetCountStats *st)
{
    if (nq == 0) return FC_OK;
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = build_set_plan(c, nq, set_off, rows, 1, &p);
    }
    if (rc != FC_OK) return rc;
    const size_t bytes = sizeof(int32_t) * nq;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaError_t e = c->io[0].ensure(bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
    if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], c->stream);
    rc = e != cudaSuccess ? cuda_fail(e, "itemset counts") : run_plan(p, c->io[0].p, nullptr, nullptr, c->stream, false);
    if (rc == FC_OK && (e = cudaEventRecord(ev[1], c->stream)) == cudaSuccess)
        e = cudaMemcpyAsync(counts, c->io[0].p, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (rc == FC_OK && e != cudaSuccess) rc = cuda_fail(e, "itemset counts");
    if (rc == FC_OK) rc = read_status(c, c->stream);
    if (rc == FC_OK && st) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ev[0], ev[1]) == cudaSuccess) st->device_ms += ms;
        st->h2d_bytes += (int64_t)p->upload_bytes;
        st->d2h_bytes += (int64_t)bytes;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    fc_plan_free(p);
    return rc;
}

extern "C" int fc_count_assignment_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                                         const int32_t *states, int64_t *counts)
{
    if (!c || (nq > 0 && !counts)) return fail(FC_ERR_ARG, "fc_count_assignment_batch: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_assignments(c, nq, var_off, vars, states, &p);
    }
    if (rc != FC_OK) return rc;
    std::vector<int32_t> tmp(std::max(nq, 1));
    rc = run_to_host(p, tmp.data(), sizeof(int32_t) * nq, nullptr, 0, nullptr, 0);
    fc_plan_free(p);
    if (rc == FC_OK)
        for (int32_t q = 0; q < nq; ++q) counts[q] = tmp[q];
    return rc;
}

extern "C" int fc_support_splits_batch(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items,
                                       int32_t *support, int32_t *sub_support, float *confidence)
{
    if (!c || (nq > 0 && !support)) return fail(FC_ERR_ARG, "fc_support_splits_batch: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_support_splits(c, nq, set_off, items, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, support, sizeof(int32_t) * nq, sub_support, sizeof(int32_t) * p->n_sub,
                     confidence, sizeof(float) * p->n_sub);
    fc_plan_free(p);
    return rc;
}

extern "C" int fc_support_batch(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items,
                                int32_t *support, int32_t *sub_support, float *confidence)
{
    if (!c || (nq > 0 && !support)) return fail(FC_ERR_ARG, "fc_support_batch: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_support(c, nq, set_off, items, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, support, sizeof(int32_t) * nq, sub_support, sizeof(int32_t) * p->n_sub,
                     confidence, sizeof(float) * p->n_sub);
    fc_plan_free(p);
    return rc;
}

// ------------------------------------------------------------------- pairs

namespace {

cudaError_t enqueue_pairs(fc_plan *p, int32_t *pairs, float *mi, cudaStream_t s)
{
    fc_ctx *c = p->ctx;
    PairsParams P = p->pp;
    P.status = c->d_status;
    cudaError_t e = cudaMemsetAsync(P.C, 0, sizeof(int32_t) * (size_t)P.R_pad * P.R_pad, s);
    if (e != cudaSuccess) return e;
    e = launch_pairs_gemm(P, s);
    if (e != cudaSuccess) return e;
    if (!pairs && !mi) return cudaSuccess;
    return launch_pairs_extract(P.C, P.R_pad, c->n, c->d_arity, c->d_soff, p->d_pair_off, c->m, pairs, mi, s);
}

}  // namespace

extern "C" int64_t fc_pairs_cells(const fc_ctx *c)
{
    if (!c || c->transactions) return -1;
    int64_t cells = 0;
    for (int a = 0; a < c->n; ++a)
        for (int b = a + 1; b < c->n; ++b) cells += (int64_t)c->arity[a] * c->arity[b];
    return cells;
}

extern "C" int fc_plan_pairs(fc_ctx *c, fc_plan **out)
{
    if (!c || !out) return fail(FC_ERR_ARG, "fc_plan_pairs: null argument");
    *out = nullptr;
    if (c->transactions) return fail(FC_ERR_STATE, "all-pairs tables need a categorical context");
    DevGuard g(c->device);
    fc_plan *p = new (std::nothrow) fc_plan();
    if (!p) return fail(FC_ERR_OOM, "host allocation failed");
    p->ctx = c;
    p->generation = c->generation;
    c->live_plans.push_back(p);
    p->kind = kPlanPairs;
    p->nq = 0;
    const int32_t R_pad = (int32_t)round_up(c->R, 256);
    const int64_t npairs = (int64_t)c->n * (c->n - 1) / 2;
    p->n_pairs = npairs;
    std::vector<int64_t> off(npairs + 1, 0);
    int64_t idx = 0;
    for (int a = 0; a < c->n; ++a)
        for (int b = a + 1; b < c->n; ++b, ++idx) off[idx + 1] = off[idx] + (int64_t)c->arity[a] * c->arity[b];
    p->pair_cells = off[npairs];
    cudaError_t e = plan_buf(c, p->pairs_C, 4, sizeof(int32_t) * (size_t)R_pad * R_pad);
    if (e == cudaSuccess) e = plan_buf(c, p->pairs_meta, 5, sizeof(int64_t) * (npairs + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->pairs_meta.p, off.data(), sizeof(int64_t) * (npairs + 1), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fc_plan_free(p);
        return cuda_fail(e, "pairs plan");
    }
    p->d_pair_off = (int64_t *)p->pairs_meta.p;
    PairsParams &P = p->pp;
    P.bits = c->d_bits;
    P.wstride = c->wstride;
    P.words = c->words;
    P.R = c->R;
    P.R_pad = R_pad;
    P.C = (int32_t *)p->pairs_C.p;
    const int64_t chunk_words = std::max<int64_t>(2, c->opt.pair_chunk_rows / 64 / 2 * 2);
    // row splits: enough CTAs to fill the GPU and at most chunk_words per split
    const int32_t tiles = pairs_tile_count(R_pad);
    // one CTA per SM: pick the split count that fills whole waves and gives
    // at least the splits the chunk bound asks for
    const int64_t need = std::max<int64_t>(1, (c->words + chunk_words - 1) / chunk_words);
    const int64_t max_split = std::max<int64_t>(1, (c->words + 1) / 2);
    int64_t ksplit = need;
    for (int64_t waves = 1; waves < 64; ++waves) {
        const int64_t s = waves * c->num_sms / tiles;
        if (s >= need && s * tiles >= waves * c->num_sms - tiles / 2) {
            ksplit = s;
            break;
        }
    }
    ksplit = std::max<int64_t>(1, std::min(ksplit, max_split));
    P.ksplit = (int32_t)ksplit;
    P.chunk_words = (int32_t)chunk_words;
    P.wait_limit = c->opt.wait_limit;
    *out = p;
    return FC_OK;
}

extern "C" int fc_pairs_all(fc_ctx *c, int32_t *pair_tables, float *mi)
{
    if (!c) return fail(FC_ERR_ARG, "fc_pairs_all: null context");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_pairs(c, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, pair_tables, pair_tables ? sizeof(int32_t) * p->pair_cells : 0, mi,
                     mi ? sizeof(float) * p->n_pairs : 0, nullptr, 0);
    fc_plan_free(p);
    return rc;
}

// --------------------------------------------------------- options, errors

namespace {

struct OptDesc {
    const char *key;
    int64_t Options::*p64;
    int32_t Options::*p32;
    int64_t lo, hi;
};

const OptDesc kOpts[] = {
    {"strategy", nullptr, &Options::strategy, -1, 3},
    {"smem_cells", nullptr, &Options::smem_cells, 256, 1 << 20},
    {"threads", nullptr, &Options::threads, 32, 1024},
    {"ctas_per_sm", nullptr, &Options::ctas_per_sm, 1, 32},
    {"hist_copies", nullptr, &Options::hist_copies, 1, 32},
    {"min_part_rows", &Options::min_part_rows, nullptr, kChunkRows, (int64_t)1 << 31},
    {"pair_chunk_rows", &Options::pair_chunk_rows, nullptr, 128, (int64_t)1 << 24},
    {"use_graph", nullptr, &Options::use_graph, 0, 1},
    {"wait_limit", &Options::wait_limit, nullptr, 1, (int64_t)1 << 40},
    {"sort_min_cells", &Options::sort_min_cells, nullptr, 1, (int64_t)1 << 31},
    {"bitmap_cost", &Options::bitmap_cost, nullptr, 0, (int64_t)1 << 40},
    {"bitmap_chunk_cost", &Options::bitmap_chunk_cost, nullptr, 0, (int64_t)1 << 40},
    {"hist_cost_row", &Options::hist_cost_row, nullptr, 0, (int64_t)1 << 40},
    {"hist_cost_var", &Options::hist_cost_var, nullptr, 0, (int64_t)1 << 40},
    {"flush_cost", &Options::flush_cost, nullptr, 0, (int64_t)1 << 40},
    {"small_cost", &Options::small_cost, nullptr, 0, (int64_t)1 << 40},
    {"bitmap_small", nullptr, &Options::bitmap_small, 0, 1},
    {"stage_slots", nullptr, &Options::stage_slots, 1, 64},
    {"bitmap_threads", nullptr, &Options::bitmap_threads, 32, 1024},
    {"support_warps", nullptr, &Options::support_warps, 1, 32},
    {"support_sets_per_warp", nullptr, &Options::support_sets_per_warp, 1, 64},
    {"support_part_words", &Options::support_part_words, nullptr, 64, (int64_t)1 << 40},
};

}  // namespace

extern "C" int fc_set_option(fc_ctx *c, const char *key, int64_t value)
{
    if (!c || !key) return fail(FC_ERR_ARG, "fc_set_option: null argument");
    for (const OptDesc &d : kOpts)
        if (std::strcmp(d.key, key) == 0) {
            if (value < d.lo || value > d.hi)
                return fail(FC_ERR_ARG, "option %s must be in %lld..%lld", key, (long long)d.lo, (long long)d.hi);
            if (d.p64) c->opt.*(d.p64) = value;
            else c->opt.*(d.p32) = (int32_t)value;
            return FC_OK;
        }
    return fail(FC_ERR_ARG, "unknown option %s", key);
}

extern "C" int64_t fc_get_option(const fc_ctx *c, const char *key)
{
    if (!c || !key) return -1;
    for (const OptDesc &d : kOpts)
        if (std::strcmp(d.key, key) == 0) return d.p64 ? c->opt.*(d.p64) : (int64_t)(c->opt.*(d.p32));
    return -1;
}

extern "C" const char *fc_last_error(void) { return g_err.c_str(); }

extern "C" int fc_selftest_wait_timeout(fc_ctx *c, int64_t wait_limit)
{
    if (!c || wait_limit < 1) return fail(FC_ERR_ARG, "fc_selftest_wait_timeout: bad argument");
    DevGuard g(c->device);
    cudaError_t e = launch_wait_selftest(c->d_status, wait_limit, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
    return read_status(c, c->stream);
}

// ---------------------------------------------------------------- autotune

namespace {

uint64_t lcg(uint64_t &s)
{
    s = s * 6364136223846793005ull + 1442695040888963407ull;
    return s >> 33;
}

// Time one plan on the context stream with events (best of `reps`).
double time_plan(fc_plan *p, void *out, int reps)
{
    fc_ctx *c = p->ctx;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double best = 1e30;
    for (int r = 0; r < reps + 1; ++r) {
        cudaEventRecord(a, c->stream);
        run_plan(p, out, nullptr, nullptr, c->stream, false);
        cudaEventRecord(b, c->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (r > 0) best = std::min(best, (double)ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Least squares for y ~ a x0 + b x1 with a, b >= 0.
void fit2(const std::vector<double> &x0, const std::vector<double> &x1, const std::vector<double> &y,
          double &a, double &b)
{
    double s00 = 0, s01 = 0, s11 = 0, t0 = 0, t1 = 0;
    for (size_t i = 0; i < y.size(); ++i) {
        s00 += x0[i] * x0[i];
        s01 += x0[i] * x1[i];
        s11 += x1[i] * x1[i];
        t0 += x0[i] * y[i];
        t1 += x1[i] * y[i];
    }
    const double det = s00 * s11 - s01 * s01;
    if (det > 1e-12 * s00 * s11) {
        a = (t0 * s11 - t1 * s01) / det;
        b = (t1 * s00 - t0 * s01) / det;
    } else {
        a = s00 > 0 ? t0 / s00 : 0;
        b = 0;
    }
    if (a < 0) {
        a = 0;
        b = s11 > 0 ? t1 / s11 : 0;
    } else if (b < 0) {
        b = 0;
        a = s00 > 0 ? t0 / s00 : 0;
    }
}

}  // namespace

// Times, for each query size k, a batch of random queries over the loaded
// variables with each strategy forced, then fits the cost model that
// FC_STRAT_AUTO uses:  histogram = rows (a + b k),  bitmap = chunks (c0 + c1
// nodes), nodes being the DFS tree size of the query in entropy order.
extern "C" int fc_autotune(fc_ctx *c, int32_t budget_ms)
{
    if (!c) return fail(FC_ERR_ARG, "fc_autotune: null context");
    if (c->transactions) return FC_OK;
    DevGuard g(c->device);
    (void)budget_ms;
    const Options saved = c->opt;
    const int kmax = std::min(6, c->n);
    const int nq = std::max(2048, 8 * c->num_sms * std::max(1, saved.ctas_per_sm));
    const double chunks = (double)((c->m + kChunkRows - 1) / kChunkRows);
    const double rows = (double)c->m;
    uint64_t seed = 0x9e3779b97f4a7c15ull;
    std::vector<double> hx0, hx1, hy, bx0, bx1, by;
    std::vector<int32_t> perm(c->n);
    for (int k = 1; k <= kmax; ++k) {
        std::vector<int32_t> off{0}, vars;
        double nodes = 0;
        for (int q = 0; q < nq; ++q) {
            std::iota(perm.begin(), perm.end(), 0);
            int64_t cells = 1;
            int used = 0;
            for (int t = 0; t < c->n && used < k; ++t) {
                const int j = t + (int)(lcg(seed) % (c->n - t));
                std::swap(perm[t], perm[j]);
                if (cells * c->arity[perm[t]] > saved.smem_cells) continue;
                cells *= c->arity[perm[t]];
                vars.push_back(perm[t]);
                ++used;
            }
            off.push_back((int32_t)vars.size());
            std::vector<QVar> qv;
            int32_t ke = 0;
            describe(c, vars.data() + off[q], off[q + 1] - off[q], qv, ke);
            entropy_order(c, qv.data(), ke);
            nodes += dfs_nodes(qv.data(), ke);
        }
        double t[2] = {-1, -1};
        for (int s = 0; s < 2; ++s) {
            c->opt = saved;
            c->opt.strategy = s;
            c->opt.bitmap_small = 0;  // the tree-walk fit; the small path is fitted below
            fc_plan *p = nullptr;
            if (fc_plan_count(c, nq, off.data(), vars.data(), nullptr, &p) != FC_OK) {
                c->opt = saved;
                return FC_ERR_CUDA;
            }
            bool all = true;
            for (int32_t q = 0; q < nq; ++q) all = all && p->strategy[q] == s;
            DBuf out;
            if (out.ensure(sizeof(int32_t) * std::max<int64_t>(p->out_cells, 1)) != cudaSuccess) {
                fc_plan_free(p);
                c->opt = saved;
                return fail(FC_ERR_OOM, "autotune buffer");
            }
            if (all) t[s] = time_plan(p, out.p, 3) * 1e12;  // milliseconds -> femtoseconds
            out.release();
            fc_plan_free(p);
        }
        if (t[1] > 0) {
            hx0.push_back(nq * rows);
            hx1.push_back(nq * rows * k);
            hy.push_back(t[1]);
        }
        if (t[0] > 0) {
            bx0.push_back(nq * chunks);
            bx1.push_back(nodes * chunks);
            by.push_back(t[0]);
        }
    }
    c->opt = saved;
    double a = 0, b = 0;
    if (hy.size() >= 2) {
        fit2(hx0, hx1, hy, a, b);
        c->opt.hist_cost_row = (int64_t)std::max(1.0, a);
        c->opt.hist_cost_var = (int64_t)std::max(1.0, b);
    }
    if (by.size() >= 2) {
        fit2(bx0, bx1, by, a, b);
        c->opt.bitmap_chunk_cost = (int64_t)std::max(0.0, a);
        c->opt.bitmap_cost = (int64_t)std::max(1.0, b);
    }
    // register-blocked path: batches of 2- and 3-variable queries over
    // variables of arity 2..5, timed with the bitmap strategy forced;
    // small_cost = (time - chunk costs) / (chunks x work units)
    std::vector<int32_t> small_vars;
    for (int v = 0; v < c->n; ++v)
        if (c->arity[v] >= 2 && c->arity[v] <= 5) small_vars.push_back(v);
    double num = 0.0, den = 0.0;
    for (int k = 2; k <= 3 && (int)small_vars.size() >= k; ++k) {
        std::vector<int32_t> off{0}, vars;
        double units = 0.0;
        const int ns = (int)small_vars.size();
        std::vector<int32_t> pool(small_vars);
        for (int q = 0; q < nq; ++q) {
            for (int t = 0; t < k; ++t) {
                const int j = t + (int)(lcg(seed) % (ns - t));
                std::swap(pool[t], pool[j]);
                vars.push_back(pool[t]);
            }
            off.push_back((int32_t)vars.size());
            std::vector<QVar> qv;
            int32_t ke = 0;
            describe(c, vars.data() + off[q], k, qv, ke);
            entropy_order(c, qv.data(), ke);
            units += small_units(qv.data(), ke);
        }
        c->opt.strategy = FC_STRAT_BITMAP;
        fc_plan *p = nullptr;
        const int rc = fc_plan_count(c, nq, off.data(), vars.data(), nullptr, &p);
        c->opt.strategy = saved.strategy;
        if (rc != FC_OK) {
            c->opt = saved;
            return rc;
        }
        bool all = true;
        for (int32_t q = 0; q < nq; ++q) all = all && p->strategy[q] == FC_STRAT_BITMAP;
        DBuf out;
        if (out.ensure(sizeof(int32_t) * std::max<int64_t>(p->out_cells, 1)) != cudaSuccess) {
            fc_plan_free(p);
            c->opt = saved;
            return fail(FC_ERR_OOM, "autotune buffer");
        }
        if (all) {
            const double tf = time_plan(p, out.p, 3) * 1e12;
            num += std::max(0.0, tf - (double)nq * chunks * (double)c->opt.bitmap_chunk_cost);
            den += units * chunks;
        }
        out.release();
        fc_plan_free(p);
    }
    if (den > 0.0) c->opt.small_cost = (int64_t)std::max(1.0, num / den);
    return FC_OK;
}

// Tunes the strategy thresholds for one batch: the per-size regression of
// fc_autotune, then the batch itself timed with the bitmap cost scaled by
// 1/4 .. 4 and with the bitmap strategy off; the fastest setting is kept.
extern "C" int fc_autotune_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars)
{
    if (!c || (nq > 0 && (!var_off || !vars))) return fail(FC_ERR_ARG, "fc_autotune_batch: null argument");
    if (c->transactions) return FC_OK;
    int rc = fc_autotune(c, 0);
    if (rc != FC_OK) return rc;
    DevGuard g(c->device);
    const Options base = c->opt;
    const double scales[] = {0.25, 0.5, 1.0, 2.0, 4.0, -1.0};  // -1: bitmap never chosen
    double best_t = 1e30;
    Options best = base;
    for (double sc : scales) {
        c->opt = base;
        c->opt.bitmap_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)std::max(1.0, base.bitmap_cost * sc);
        c->opt.bitmap_chunk_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)(base.bitmap_chunk_cost * sc);
        c->opt.small_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)std::max(1.0, base.small_cost * sc);
        fc_plan *p = nullptr;
        if ((rc = fc_plan_count(c, nq, var_off, vars, nullptr, &p)) != FC_OK) {
            c->opt = base;
            return rc;
        }
        DBuf out;
        if (out.ensure(sizeof(int32_t) * std::max<int64_t>(p->out_cells, 1)) != cudaSuccess) {
            fc_plan_free(p);
            c->opt = base;
            return fail(FC_ERR_OOM, "autotune buffer");
        }
        const double t = time_plan(p, out.p, 3);
        out.release();
        fc_plan_free(p);
        if (t < best_t) {
            best_t = t;
            best = c->opt;
        }
    }
    c->opt = best;
    return FC_OK;
}

// ---------------------------------------------------------------- families
//
// The query stream of parent-set assignment (Sec. 4.2): every child X in a
// variable list and every parent set of at most `max_parents` of the other
// variables.  The family (X, Pa) is the split of the variable set V = Pa + {X}
// with X as the child, so each V is counted once and serves |V| families.

namespace {

int64_t binom(int64_t n, int64_t k)
{
    if (k < 0 || n < 0 || k > n) return 0;
    int64_t r = 1;
    for (int64_t i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// Rank of the ascending combination a[0..k) of {0..N-1} among all
// k-combinations in lexicographic order.
int64_t comb_rank(const int32_t *a, int k, int N)
{
    int64_t r = 0;
    int prev = -1;
    for (int i = 0; i < k; ++i) {
        for (int v = prev + 1; v < a[i]; ++v) r += binom(N - 1 - v, k - 1 - i);
        prev = a[i];
    }
    return r;
}

}  // namespace

extern "C" int64_t fc_families_count(int32_t nv, int32_t max_parents)
{
    if (nv < 1 || max_parents < 0) return -1;
    const int d = std::min(max_parents, nv - 1);
    int64_t per_child = 0;
    for (int s = 0; s <= d; ++s) per_child += binom(nv - 1, s);
    return (int64_t)nv * per_child;
}

extern "C" int fc_plan_families(fc_ctx *c, int32_t nv, const int32_t *vars, int32_t max_parents, int32_t kind,
                                double ess, fc_plan **out)
{
    if (!c || !out || !vars) return fail(FC_ERR_ARG, "fc_plan_families: null argument");
    *out = nullptr;
    if (c->transactions) return fail(FC_ERR_STATE, "family scores need a categorical context");
    if (nv < 1 || nv > c->n || max_parents < 0) return fail(FC_ERR_ARG, "bad nv or max_parents");
    if (kind < FC_LL || kind > FC_MI) return fail(FC_ERR_ARG, "unknown score kind %d", kind);
    if (kind == FC_BDEU && !(ess > 0.0)) return fail(FC_ERR_ARG, "BDeu needs ess > 0");
    const int d = std::min(max_parents, nv - 1);
    if (d + 1 > kMaxFamily) return fail(FC_ERR_SIZE, "at most %d parents per family", kMaxFamily - 1);
    if (++c->epoch == 0) {
        std::fill(c->mark.begin(), c->mark.end(), 0u);
        c->epoch = 1;
    }
    for (int i = 0; i < nv; ++i) {
        if (vars[i] < 0 || vars[i] >= c->n) return fail(FC_ERR_ARG, "variable %d out of range", vars[i]);
        if (c->mark[vars[i]] == c->epoch) return fail(FC_ERR_ARG, "variable %d listed twice", vars[i]);
        c->mark[vars[i]] = c->epoch;
    }
    int64_t nsets = 0;
    for (int s = 1; s <= d + 1; ++s) nsets += binom(nv, s);
    const int64_t njobs = fc_families_count(nv, d);
    if (nsets > INT32_MAX || njobs > INT32_MAX) return fail(FC_ERR_SIZE, "too many variable sets");
    DevGuard g(c->device);
    // every variable set of 1..d+1 variables, ascending positions in `vars`
    std::vector<int32_t> set_pos;  // flattened positions
    std::vector<int32_t> set_off{0};
    std::vector<int32_t> comb(d + 1);
    for (int s = 1; s <= d + 1; ++s) {
        for (int i = 0; i < s; ++i) comb[i] = i;
        for (;;) {
            for (int i = 0; i < s; ++i) set_pos.push_back(comb[i]);
            set_off.push_back((int32_t)set_pos.size());
            int i = s - 1;
            while (i >= 0 && comb[i] == nv - s + i) --i;
            if (i < 0) break;
            ++comb[i];
            for (int j = i + 1; j < s; ++j) comb[j] = comb[j - 1] + 1;
        }
    }
    std::vector<int32_t> set_vars(set_pos.size());
    for (size_t i = 0; i < set_pos.size(); ++i) set_vars[i] = vars[set_pos[i]];
    fc_plan *p = new (std::nothrow) fc_plan();
    if (!p) return fail(FC_ERR_OOM, "host allocation failed");
    p->ctx = c;
    p->generation = c->generation;
    c->live_plans.push_back(p);
    p->kind = kPlanFamilies;
    p->nq = nv;
    p->fam_kind = kind;
    p->ess = ess;
    p->n_jobs = njobs;
    {
        const bool saved = c->borrow;
        c->borrow = false;  // the inner plan owns its buffers for the plan's lifetime
        int rc = fc_plan_count(c, (int32_t)nsets, set_off.data(), set_vars.data(), nullptr, &p->inner);
        c->borrow = saved;
        if (rc != FC_OK) {
            fc_plan_free(p);
            return rc;
        }
    }
    // one job per (variable set, child position); slot = child position in
    // `vars` times the families per child + rank of the parent set
    const int64_t per_child = njobs / nv;
    std::vector<int64_t> level_base(d + 2, 0);
    for (int s = 1; s <= d + 1; ++s) level_base[s] = level_base[s - 1] + binom(nv - 1, s - 1);
    std::vector<FamilyJob> jobs;
    jobs.reserve(njobs);
    std::vector<int32_t> par(d + 1);
    for (int64_t q = 0; q < nsets; ++q) {
        const int32_t a = set_off[q], k = set_off[q + 1] - a;
        for (int cpos = 0; cpos < k; ++cpos) {
            const int32_t child = set_pos[a + cpos];
            int np = 0;
            for (int t = 0; t < k; ++t)
                if (t != cpos) {
                    const int32_t pp = set_pos[a + t];
                    par[np++] = pp < child ? pp : pp - 1;  // position among the other nv - 1 variables
                }
            FamilyJob j{};
            j.table_off = p->inner->table_off[q];
            j.k = (int16_t)k;
            j.child_pos = (int16_t)cpos;
            j.slot = (int32_t)(child * per_child + level_base[np] + comb_rank(par.data(), np, nv - 1));
            for (int t = 0; t < k; ++t) j.vars[t] = set_vars[a + t];
            jobs.push_back(j);
        }
    }
    cudaError_t e = plan_buf(c, p->fam_jobs, 4, sizeof(FamilyJob) * std::max<int64_t>(njobs, 1));
    if (e == cudaSuccess) e = plan_buf(c, p->fam_tables, 5, sizeof(int32_t) * std::max<int64_t>(p->inner->out_cells, 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->fam_jobs.p, jobs.data(), sizeof(FamilyJob) * njobs, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    p->upload_bytes = sizeof(FamilyJob) * njobs + p->inner->upload_bytes;
    if (e != cudaSuccess) {
        fc_plan_free(p);
        return cuda_fail(e, "family plan");
    }
    *out = p;
    return FC_OK;
}

extern "C" int fc_score_families(fc_ctx *c, int32_t nv, const int32_t *vars, int32_t max_parents, int32_t kind,
                                 double ess, float *scores)
{
    if (!c || !scores) return fail(FC_ERR_ARG, "fc_score_families: null argument");
    DevGuard g(c->device);
    fc_plan *p = nullptr;
    int rc;
    {
        BorrowScope b(c);
        rc = fc_plan_families(c, nv, vars, max_parents, kind, ess, &p);
    }
    if (rc != FC_OK) return rc;
    rc = run_to_host(p, scores, sizeof(float) * p->n_jobs, nullptr, 0, nullptr, 0);
    fc_plan_free(p);
    return rc;
}
