// fc_host.h -- host-side internals shared by the runtime translation units:
// contexts (fc_ctx.cu), the count/score planner and plan API (fc_plan.cu),
// itemset plans (fc_sets.cu), the all-pairs plan (fc_pairs_host.cu), options
// and autotuning (fc_tune.cu), family scores (fc_families.cu), and the rule
// miner (fc_rules.cu).
#pragma once

#include "../../include/fc.h"
#include "fc_internal.h"

#include <algorithm>
#include <condition_variable>
#include <cstdarg>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace fc {

// ------------------------------------------------------------------ errors

// Message of the last error on this host thread (fc_last_error).
extern thread_local std::string g_err;
// Records a formatted message for fc_last_error() and returns code.
int fail(int code, const char *fmt, ...);
// FC_ERR_OOM for an allocation failure, FC_ERR_CUDA otherwise.
int cuda_fail(cudaError_t e, const char *what);

#define FC_CUDA(call, what)                                    \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return fc::cuda_fail(e_, what); \
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

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

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
    // launch shape of the mixed count launch; with shape_auto the planner
    // takes 256 threads x 6 CTAs x 8192 cells per SM unless the batch needs
    // the larger table area below (its rule is in the planner)
    int32_t smem_cells = 16384;       // 64 KiB of tables per CTA
    int32_t threads = 512;
    int32_t ctas_per_sm = 2;
    int32_t shape_auto = 1;           // cleared by setting any of the three above
    int32_t hist_copies = 4;
    int64_t min_part_rows = 8192;
    int64_t pair_chunk_rows = 1 << 16;
    int32_t use_graph = 1;
    int64_t wait_limit = 1 << 22;
    int64_t sort_min_cells = 1 << 25;
    int32_t window_max = 16;          // AUTO: most shared-memory windows per table
    int32_t window_cells = 1 << 20;   // cap on the cells of one window
    int32_t window_wide = 1;          // windows in a launch of one 1024-thread CTA per SM
    // cost model, femtoseconds: bitmap per DFS node per 4096-row chunk;
    // histogram per row and per row-variable; per table cell flushed
    int64_t bitmap_cost = 200000;
    int64_t bitmap_chunk_cost = 0;    // per 4096-row chunk of a bitmap query
    int64_t hist_cost_row = 143;
    int64_t hist_cost_var = 124;
    int64_t flush_cost = 160;
    // register-blocked bitmap path (2-3 variables of arity 2..5): per work
    // unit (cell or state row) per 4096-row chunk
    int64_t small_cost = 12000;   // per work unit of a two-variable table
    int64_t small3_cost = 12000;  // per work unit of a three-variable table
    int32_t bitmap_small = 1;
    int32_t stage_slots = 16;         // bitmap rows a warp stages per chunk
    int32_t bitmap_threads = 256;
    int32_t support_warps = 16;
    int32_t support_sets_per_warp = 4;
    int64_t support_part_words = 8192;
    // synchronous count / score calls whose output buffer is page-locked
    // host memory let the kernels store into it directly (no device buffer,
    // no copy) when no output cell is accumulated
    int32_t zero_copy = 1;
    // large count batches whose queries all count in shared memory are
    // planned on the device (fc_dplan.cu)
    int32_t device_plan = 1;
    // the histogram strategy reads the 4-bit copy of the columns when the
    // context holds one (every arity <= 16)
    int32_t codes4 = 1;
};

// Smallest synchronous count batch that is pipelined in parts or planned on
// the device.
constexpr int32_t kDevicePlanMinQueries = 4096;

// Host arrays of the count planner, kept by the context between plan builds
// so that a steady stream of batches allocates (and page-faults) nothing.
struct PlanScratch {
    std::vector<int64_t> base;      // first QVar slot of each query
    std::vector<double> cost;       // cost-model estimate of each query
    std::vector<int32_t> cells;     // table cells of each query
    std::vector<uint32_t> cls;      // cost class of each query (descending order)
    std::vector<uint8_t> passes;    // bitmap queries: first-variable passes (0 = none)
    std::vector<uint8_t> mixed_win; // windowed queries counted in the mixed launch
    std::vector<int32_t> order, start, qlist;
    std::vector<BTask> btasks;
    size_t rest_bytes = 0;          // staging bytes past the QVars in the last plan
};

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
}  // namespace fc

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
    // 1 when the last fc_count_batch was planned on the device (fc_info key 7)
    int32_t last_batch_on_device = 0;
    // the variables' entropies in FP32 on the device (the device planner's
    // cost model), uploaded by the first device-planned batch after a load or
    // an append (entropy_stale)
    float *d_entropy_f = nullptr;
    bool entropy_stale = true;
    // D as 4-bit codes when every arity is at most 16 (else null): the
    // histogram kernel reads half the column bytes
    uint8_t *d_D4 = nullptr;
    uint64_t *d_bits = nullptr;
    int64_t *d_marg = nullptr;
    int32_t *d_arity = nullptr, *d_soff = nullptr;
    int32_t *d_status = nullptr;
    std::vector<int64_t> marg;
    std::vector<double> entropy;
    fc::Options opt;
    // scratch of the host-buffer entry points
    fc::DBuf io[3];
    fc::DBuf marg_delta;     // marginal counts of the instances an append adds (R int64)
    fc::DBuf dplan_buf;      // inputs, descriptors and items of device-planned batches
    std::vector<int64_t> h_marg_delta;
    // buffers lent to one-shot plans (descriptors, counters, tables, sort,
    // pairs), in two banks so that a synchronous call can have a plan
    // running while it builds the next; `bank` selects the one in use
    fc::DBuf pool[2][6];
    fc::DBuf pipe_io[2];     // device outputs of the parts of a pipelined call, per bank
    int bank = 0;
    int32_t q_base = 0;  // index of the plan's first query in the caller's batch (messages)
    bool borrow = false; // set while a synchronous entry point builds its plan
    cudaStream_t out_stream = nullptr;  // device-to-host copies of pipelined calls
    cudaEvent_t part_done[2] = {nullptr, nullptr};   // a bank's part: kernels done
    cudaEvent_t copy_done[2] = {nullptr, nullptr};   // a bank's part: output copied out
    std::vector<uint32_t> mark;
    uint32_t epoch = 0;
    uint64_t generation = 0;  // bumped by every append; plans of older generations refuse to run
    std::vector<fc_plan *> live_plans;  // orphaned (device memory released) if the context goes first
    // pinned staging of plan descriptors, one per bank; `ev` marks the end
    // of the last upload from it
    struct Stage {
        uint8_t *h = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev = nullptr;
    } stage[2];
    std::unique_ptr<fc::PlanPool> pool_threads;  // started by the first large plan
    std::unique_ptr<fc::PlanScratch> plan_scratch;
};

namespace fc {

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

}  // namespace fc

struct fc_plan {
    fc_ctx *ctx = nullptr;
    int kind = fc::kPlanCount;
    int32_t nq = 0;
    std::vector<int64_t> table_off;  // count plans: caller offsets (nq + 1)
    std::vector<int32_t> strategy;
    int64_t out_cells = 0;
    // count / score
    fc::DBuf desc;           // QHead, QVar, Item, q_list
    fc::DBuf counters;       // next item + tickets
    fc::DBuf scratch_tables; // score plans: tables that live in global memory
    fc::DBuf sort_mem;
    fc::SortScratch sort_sc{};
    std::vector<fc::SortJob> sort_jobs;
    fc::QHead *d_qh = nullptr;
    fc::QVar *d_qv = nullptr;
    fc::Item *d_items = nullptr;
    int32_t *d_qlist = nullptr;
    int32_t n_items = 0, n_qlist = 0, n_counters = 0;
    fc::BTask *d_btasks = nullptr;
    int32_t n_btasks = 0, bm_grid = 0, bm_threads = 0, stage_slots = 0;
    int32_t small_paths = 1;
    bool zero_tables = false;
    int64_t table_buf_cells = 0;  // cells of the buffer the kernel writes
    int score_kind = fc::kNoScore;
    double ess = 1.0;
    int grid = 0, threads = 0, smem_cells = 0;
    size_t smem = 0;
    // windowed tables in their own launch (1024 threads, one CTA per SM):
    // items [n_items, n_items + n_witems) of d_items
    int32_t n_witems = 0, wgrid = 0;
    size_t wsmem = 0;
    // support
    fc::SupportParams sp{};
    int sup_grid = 0, sup_threads = 0;
    int64_t n_sub = 0;
    // pairs
    fc::PairsParams pp{};
    fc::DBuf pairs_C, pairs_meta;
    int64_t n_pairs = 0, pair_cells = 0;
    int64_t *d_pair_off = nullptr;
    // families: the joint tables of every variable set (inner count plan) and
    // one job per (child, parents) split
    fc_plan *inner = nullptr;
    fc::DBuf fam_tables, fam_jobs;
    int64_t n_jobs = 0;
    int fam_kind = 0;
    uint64_t generation = 0;  // the context's generation when the plan was built
    size_t upload_bytes = 0;  // host-to-device bytes of the plan's descriptors
    std::vector<fc::GraphEntry> graphs;
};

namespace fc {

// A plan buffer: its own allocation, or a view of the context's pool slot.
inline cudaError_t plan_buf(fc_ctx *c, DBuf &b, int slot, size_t bytes)
{
    if (!c->borrow) return b.ensure(bytes);
    DBuf &lent = c->pool[c->bank][slot];
    cudaError_t e = lent.ensure(bytes);
    if (e != cudaSuccess) return e;
    b.p = lent.p;
    b.bytes = lent.bytes;
    b.owned = false;
    return cudaSuccess;
}

struct BorrowScope {
    fc_ctx *c;
    explicit BorrowScope(fc_ctx *ctx, int bank = 0) : c(ctx)
    {
        c->borrow = true;
        c->bank = bank;
    }
    ~BorrowScope()
    {
        c->borrow = false;
        c->bank = 0;
    }
};

// Pinned host staging (of the current bank) of at least `bytes` for plan
// descriptors, free of any copy still reading it; nullptr on failure
// (fc_ctx.cu).
uint8_t *stage_host(fc_ctx *c, size_t bytes);
// A count batch planned and counted on the device when every query counts in
// shared memory (fc_dplan.cu); *done is clear when the host planner must
// take the batch.
int device_count_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                       const int64_t *table_off, int32_t *tables, bool *done);
// Device address of a page-locked host buffer the kernels can store to, or
// nullptr (fc_plan.cu).
void *device_view(const void *h, size_t bytes);
// Grows the staging buffer to `bytes`, keeping its first `keep` bytes.
uint8_t *stage_grow(fc_ctx *c, size_t bytes, size_t keep);
// Copies `bytes` of the staging buffer to dst on the context stream and marks
// the staging buffer busy until the copy ends (fc_ctx.cu).
cudaError_t upload_stage(fc_ctx *c, void *dst, size_t bytes);

// ------------------------------------------------- planner (fc_plan.cu)

// Validates one query's variables and appends its QVars; returns the cells or
// a negative error code (message in fc_last_error of the calling thread).
int64_t describe(const fc_ctx *c, const int32_t *vars, int32_t k, std::vector<QVar> &qv, int32_t &k_eff);
// Variables in ascending entropy (the bitmap walk's order).
void entropy_order(const fc_ctx *c, QVar *v, int k);
// Nodes of the bitmap tree in the given order (no pruning).
double dfs_nodes(const QVar *v, int k);
// Register-blocked bitmap path: eligibility and work units per chunk.
bool small_ok(const QVar *o, int k);
double small_units(const QVar *o, int k);
// Device resources of a plan (graphs and buffers); the plan's device is current.
void release_plan(fc_plan *p);
cudaError_t enqueue_count(fc_plan *p, int32_t *tables, float *scores, cudaStream_t s);
// Runs a plan on stream s (a graph per (outputs, stream) when allowed).
int run_plan(fc_plan *p, void *o0, void *o1, void *o2, cudaStream_t s, bool allow_graph);
// Reads the context status word (synchronises s); FC_ERR_TIMEOUT if a
// bounded device wait ran out.
int read_status(fc_ctx *c, cudaStream_t s);
// Runs a plan with runtime-owned device outputs and copies them to host buffers.
int run_to_host(fc_plan *p, void *h0, size_t b0, void *h1, size_t b1, void *h2, size_t b2);

// --------------------------------------------------- other plan kinds

// fc_sets.cu: a plan over sets of bitmap rows (mode 0 leave-one-out supports,
// 1 supports alone, 2 every antecedent split) and its enqueue.
int build_set_plan(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *items, int mode,
                   fc_plan **out);
cudaError_t enqueue_support(fc_plan *p, int32_t *support, int32_t *sub, float *conf, cudaStream_t s);
// fc_pairs_host.cu
cudaError_t enqueue_pairs(fc_plan *p, int32_t *pairs, float *mi, cudaStream_t s);
// fc_families.cu
cudaError_t enqueue_families(fc_plan *p, float *scores, cudaStream_t s);

}  // namespace fc
