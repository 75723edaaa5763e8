// fc_dplan.cu -- planning a large count batch on the device.
//
// A synchronous fc_count_batch of thousands of queries spends as long on the
// host planner (validation, per-query descriptors, strategy choice, work
// items in longest-first order) as the GPU spends counting.  When every query
// of a batch is counted in shared memory -- a histogram, a precomputed
// marginal, or windows of the mixed launch (Sec. 3.3's partitions, keyed and
// counted on chip) -- the plan is simple enough to build on the device:
//
//   dplan_describe   one thread per query: validates it, writes its QVars
//                    (strides in the caller's order, arity-1 variables
//                    dropped) and head, picks the strategy with the same cost
//                    model as the host planner, and counts its work items
//                    per cost class;
//   dplan_finish     one CTA: checks the batch-wide conditions of the fast
//                    path (the small launch shape, no row splits), turns the
//                    class counts into positions (longest first) and packs
//                    the table offsets when the caller gave none;
//   dplan_items      one thread per query: writes its items at its class's
//                    next positions;
//
// then the count kernel runs with its item count read from device memory.
// A query the fast path does not handle (one the cost model sends to the
// bitmap strategy, a table beyond the mixed launch's windows, an invalid
// query) leaves the item count at zero, so nothing is counted, and the host
// runs the regular planner, which also produces the error messages.
#include "fc_host.h"

#include <cstddef>
#include <cstring>

namespace fc {

// Result of a device plan, read by the host after the batch ran.
struct DPlanSummary {
    int32_t bad;        // nonzero: a query the fast path does not take (or an invalid one)
    int32_t n_items;    // work items of the count launch (0 when bad)
    int32_t mid;        // tables the planner's large shape would hold whole (8192 < cells <= 16384)
    int32_t hist;       // histogram queries
    int64_t out_cells;  // cells of the packed tables (no caller offsets)
    uint32_t cls_lo_inv;  // span of the cost classes present: ~lo and hi (both zero before
    uint32_t cls_hi;      // planning, an empty span)
};

namespace {

constexpr int kClasses = 1 << 14;  // 1/8-octave cost classes (see cost_class)

struct DPlanParams {
    const int32_t *var_off;   // nq + 1
    const int32_t *vars;      // the lists from var_off[0] on
    int32_t base0;            // var_off[0]
    const int64_t *user_off;  // nq + 1, or null (tables packed in query order)
    const int32_t *arity, *soff;
    const float *entropy;
    int32_t n, nq;
    float rows, chunks;  // the cost model in FP32 (the FP64 pipe is slow)
    // cost model (femtoseconds) and the planner's limits
    float hist_row, hist_var, flush, bitmap_node, bitmap_chunk, small_unit, small_unit3;
    int32_t bitmap_small, stage_slots, force_hist, window_max;
    int32_t small_cells;  // table area of the small launch shape
    int32_t max_cells;    // table area of the large shape
    int32_t min_hist;     // histogram queries needed for one item per query
    int32_t stage_vars;   // 1: dplan_describe stages the variables' tables in shared memory
    QHead *qh;
    QVar *qv;
    Item *items;
    uint32_t *cls;
    int32_t *class_count;  // kClasses
    int32_t *n_items_eff;  // the count launch's item count
    DPlanSummary *sum;
};

// The variables' arity, state offset and entropy, staged in shared memory
// for the CTA (the per-query loops look them up once per variable).
struct VarInfo {
    int32_t arity, soff;
    float entropy;
};

__device__ __forceinline__ uint32_t cost_class_dev(float v)
{
    if (!(v > 0.0f)) v = 0.0f;
    const uint32_t b = __float_as_uint(v);  // exponent and 3 mantissa bits: 1/8-octave classes
    return ((1u << 14) - 1u) - (b >> (23 - 3));
}

// Cost of the bitmap strategy for a query of k <= kMaxBitmapK variables (its
// variables in ascending entropy, as its kernel walks them), or a huge value
// when the bitmap kernel cannot take it.  Mirrors the host planner's model.
__device__ __forceinline__ int arity_of(const DPlanParams &P, const VarInfo *sv, int v)
{
    return P.stage_vars ? sv[v].arity : P.arity[v];
}

__device__ __forceinline__ float entropy_of(const DPlanParams &P, const VarInfo *sv, int v)
{
    return P.stage_vars ? sv[v].entropy : P.entropy[v];
}

__device__ float bitmap_cost(const DPlanParams &P, const VarInfo *sv, const QVar *v, int k)
{
    if (k < 1 || k > kMaxBitmapK) return 3e38f;
    QVar o[kMaxBitmapK];
    for (int t = 0; t < k; ++t) o[t] = v[t];
    for (int i = 1; i < k; ++i) {  // stable insertion sort by entropy
        const QVar x = o[i];
        const float h = entropy_of(P, sv, x.var);
        int j = i - 1;
        while (j >= 0 && entropy_of(P, sv, o[j].var) > h) {
            o[j + 1] = o[j];
            --j;
        }
        o[j + 1] = x;
    }
    int slots = 0;
    for (int t = 1; t < k; ++t) slots += o[t].arity;
    if (slots > P.stage_slots) return 3e38f;
    auto ok = [](int r) { return r >= 2 && r <= 5; };
    const bool small = P.bitmap_small && ((k == 2 && ok(o[0].arity) && ok(o[1].arity)) ||
                                          (k == 3 && ok(o[1].arity) && ok(o[2].arity)));
    if (small) {
        const float units = k == 2 ? (float)(o[0].arity * o[1].arity + o[0].arity + o[1].arity)
                                   : (float)(o[0].arity * (1 + o[1].arity + o[2].arity + o[1].arity * o[2].arity));
        return P.chunks * units * (k == 2 ? P.small_unit : P.small_unit3);
    }
    float nodes = 0.0f, level = 1.0f;
    for (int t = 0; t < k; ++t) {
        level *= o[t].arity;
        nodes += level;
    }
    return P.chunks * (P.bitmap_chunk + nodes * P.bitmap_node);
}

// One query: validation, QVars, head and strategy.  Returns 0 and sets
// *cls / *nwin for a query the fast path takes, else the reason bit for the
// summary (1 invalid, 2 bitmap strategy, 4 beyond the mixed launch's windows).
__device__ int describe_one(const DPlanParams &P, const VarInfo *s_var, int32_t q, uint32_t *cls, int32_t *nwin_out,
                            bool *is_hist, bool *is_mid)
{
    const int32_t a = P.var_off[q], b = P.var_off[q + 1];
    const int32_t k = b - a;
    // the host planner reports every invalid query; here it only stops the fast path
    if (a < P.base0 || b > P.var_off[P.nq] || k < 0 || k > P.n || k > 48) return 1;
    const int32_t *vars = P.vars + (a - P.base0);
    const int64_t base = (int64_t)a - P.base0;
    QVar *out = P.qv + base;
    int64_t cells = 1;
    int k_eff = 0;
    // the cost model reads the QVars back: a copy in registers for short lists
    constexpr int kFast = 8;
    QVar fq[kFast];
    const bool fast = k <= kFast;
    if (fast) {
        // every variable of the list loaded at once (one memory latency, not k)
        int32_t lv[kFast];
#pragma unroll
        for (int t = 0; t < kFast; ++t) lv[t] = t < k ? vars[t] : 0;
        int ar[kFast];
        bool bad = false;
#pragma unroll
        for (int t = 0; t < kFast; ++t) {
            ar[t] = 1;
            if (t < k) {
                bad |= lv[t] < 0 || lv[t] >= P.n;
                if (!bad) ar[t] = arity_of(P, s_var, lv[t]);
#pragma unroll
                for (int u = 0; u < t; ++u) bad |= lv[u] == lv[t];
            }
        }
        if (bad) return 1;
        bool over = false;
#pragma unroll
        for (int t = 0; t < kFast; ++t) {
            cells *= ar[t];
            over |= cells > INT32_MAX;
            if (over) cells = (int64_t)INT32_MAX + 1;  // no int64 overflow on the next product
        }
        if (over) return 1;
        if (P.user_off && (P.user_off[q] < 0 || P.user_off[q + 1] - P.user_off[q] < cells)) return 1;
        // QVars: strides of the caller's order (last fastest), arity-1 variables dropped
#pragma unroll
        for (int t = 0; t < kFast; ++t) k_eff += t < k && ar[t] > 1 ? 1 : 0;
        int64_t stride = 1;
        int w = k_eff;
#pragma unroll
        for (int t = kFast - 1; t >= 0; --t) {
            if (t < k && ar[t] > 1) {
                const QVar x{lv[t], (int32_t)stride, ar[t], P.stage_vars ? s_var[lv[t]].soff : P.soff[lv[t]]};
                --w;
#pragma unroll
                for (int j = 0; j < kFast; ++j)
                    if (j == w) fq[j] = x;
                out[w] = x;
            }
            stride *= ar[t];
        }
    } else {
        for (int t = 0; t < k; ++t) {
            const int v = vars[t];
            if (v < 0 || v >= P.n) return 1;
            cells *= arity_of(P, s_var, v);
            if (cells > INT32_MAX) return 1;
            for (int u = 0; u < t; ++u)
                if (vars[u] == v) return 1;
        }
        if (P.user_off && (P.user_off[q] < 0 || P.user_off[q + 1] - P.user_off[q] < cells)) return 1;
        // QVars: strides of the caller's order (last fastest), arity-1 variables dropped
        int64_t stride = 1;
        for (int t = k - 1; t >= 0; --t)
            if (arity_of(P, s_var, vars[t]) > 1) ++k_eff;
        int w = k_eff;
        for (int t = k - 1; t >= 0; --t) {
            const int v = vars[t];
            const int r = arity_of(P, s_var, v);
            if (r > 1) out[--w] = QVar{v, (int32_t)stride, r, P.stage_vars ? s_var[v].soff : P.soff[v]};
            stride *= r;
        }
    }
    // strategy: the cost model of the host planner, in the small launch
    // shape; only the shared-memory strategies are taken here
    const float hist = P.rows * (P.hist_row + (float)k_eff * P.hist_var) + (float)cells * P.flush;
    int s;
    float cost;
    int32_t nwin = 1;
    if (k_eff == 0) {
        s = kHist;
        cost = hist;
    } else if (k_eff == 1 && cells <= P.max_cells) {
        s = kMarginal;
        cost = (float)cells * P.flush;
    } else if (cells <= P.max_cells) {
        if (!P.force_hist && bitmap_cost(P, s_var, fast ? fq : out, k_eff) + (float)cells * P.flush < hist) return 2;
        if (cells <= P.small_cells) {
            s = kHist;
            cost = hist;
        } else {
            // beyond the small shape's area: windows of it in the same launch
            *is_mid = true;
            nwin = (int32_t)((cells + P.small_cells - 1) / P.small_cells);
            if (nwin > P.window_max) return 4;
            s = kWindow;
            cost = (float)nwin * P.rows * (P.hist_row + (float)k_eff * P.hist_var) * 2.0f + (float)cells * P.flush;
        }
    } else {
        return 4;  // wide windows, global atomics, sort: host planner
    }
    *is_hist = s == kHist;
    QHead h;
    h.table_off = P.user_off ? P.user_off[q] : 0;
    h.cells = (int32_t)cells;
    h.var_off = (int32_t)base;
    h.k = (int16_t)k_eff;
    h.strategy = (int16_t)s;
    h.nparts = (int16_t)nwin;
    h.score_kind = (int16_t)kNoScore;
    h.r_child = 1;
    h.child_soff = 0;
    h.score_slot = q;
    h.nwin = nwin;
    P.qh[q] = h;
    *cls = cost_class_dev(cost / nwin);
    P.cls[q] = *cls;
    *nwin_out = nwin;
    return 0;
}

// A thread per query; the counts a warp adds to the summary go out as one
// atomic per warp.
__global__ void __launch_bounds__(128) dplan_describe(DPlanParams P)
{
    extern __shared__ VarInfo s_var[];
    if (P.stage_vars) {
        for (int v = threadIdx.x; v < P.n; v += blockDim.x) s_var[v] = VarInfo{P.arity[v], P.soff[v], P.entropy[v]};
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;  // cost classes this thread saw
    int bad = 0, n_hist = 0, n_mid = 0;
    for (int32_t q0 = blockIdx.x * blockDim.x; q0 < P.nq; q0 += gridDim.x * blockDim.x) {
        const int32_t q = q0 + threadIdx.x;
        uint32_t cl = 0xFFFFFFFFu;
        int32_t nwin = 0;
        bool is_hist = false, is_mid = false;
        if (q < P.nq) {
            const int why = describe_one(P, s_var, q, &cl, &nwin, &is_hist, &is_mid);
            if (why) {
                bad |= why;
                cl = 0xFFFFFFFFu;
                nwin = 0;
                is_hist = false;
            }
        }
        n_hist += is_hist;
        n_mid += is_mid;
        if (cl != 0xFFFFFFFFu) {
            lo = min(lo, cl);
            hi = max(hi, cl);
            atomicAdd(&P.class_count[cl], nwin);
        }
    }
    // the warp's summary: fast-path refusals, counts, the span of classes
    bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
    n_hist = __reduce_add_sync(0xffffffffu, (unsigned)n_hist);
    n_mid = __reduce_add_sync(0xffffffffu, (unsigned)n_mid);
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (lane == 0) {
        if (bad) atomicOr(&P.sum->bad, bad);
        if (n_hist) atomicAdd(&P.sum->hist, n_hist);
        if (n_mid) atomicAdd(&P.sum->mid, n_mid);
        if (lo <= hi) {
            atomicMax(&P.sum->cls_lo_inv, ~lo);
            atomicMax(&P.sum->cls_hi, hi);
        }
    }
}

// Exclusive prefix sum of x[0..n) in place by one CTA of 1024 threads, in
// coalesced tiles of 1024 (warp shuffles, then the warps' sums), sums in 64
// bits; returns the total to every thread.
template <class T>
__device__ int64_t block_scan(T *x, int64_t n, int64_t *warp_sum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        const int64_t v = i < n ? (int64_t)x[i] : 0;
        int64_t incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int64_t w = lane < (int)(blockDim.x >> 5) ? warp_sum[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += u;
            }
            warp_sum[lane] = w;  // inclusive over the warps
        }
        __syncthreads();
        const int64_t before = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + incl - v;
        if (i < n) x[i] = (T)before;
        carry += warp_sum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    return carry;
}

__global__ void __launch_bounds__(1024) dplan_finish(const DPlanParams P, int64_t *cells_scan)
{
    __shared__ int64_t warp_sum[32];
    __shared__ int s_bad;
    // the small launch shape holds the batch only when few tables would fit
    // the large shape whole, and one item per query fills the GPU only with
    // enough histogram queries (the host planner splits rows otherwise)
    if (threadIdx.x == 0)
        s_bad = P.sum->bad || (int64_t)P.sum->mid * 64 > P.nq || P.sum->hist < P.min_hist ||
                ~P.sum->cls_lo_inv > P.sum->cls_hi;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) {
            P.sum->bad |= 8;
            P.sum->n_items = 0;
            *P.n_items_eff = 0;
        }
        return;
    }
    // positions of the classes' items over the span present: ascending
    // class = descending cost
    const uint32_t lo = ~P.sum->cls_lo_inv, hi = P.sum->cls_hi;
    const int64_t n_items = block_scan<int32_t>(P.class_count + lo, (int64_t)(hi - lo) + 1, warp_sum);
    if (threadIdx.x == 0) {
        P.sum->n_items = (int32_t)n_items;
        *P.n_items_eff = (int32_t)n_items;
    }
    // packed table offsets in query order when the caller gave none
    if (!P.user_off) {
        for (int64_t q = threadIdx.x; q < P.nq; q += blockDim.x) cells_scan[q] = P.qh[q].cells;
        __syncthreads();
        const int64_t total = block_scan<int64_t>(cells_scan, P.nq, warp_sum);
        for (int64_t q = threadIdx.x; q < P.nq; q += blockDim.x) P.qh[q].table_off = cells_scan[q];
        if (threadIdx.x == 0) P.sum->out_cells = total;
    }
}

// Items at their class's next positions; the lanes of a warp with the same
// class take their positions with one atomic (the first such lane adds the
// group's items, the others offset by the items of the lanes before them).
__global__ void dplan_items(const DPlanParams P)
{
    if (*P.n_items_eff == 0) return;
    const int lane = threadIdx.x & 31;
    for (int32_t q0 = blockIdx.x * blockDim.x; q0 < P.nq; q0 += gridDim.x * blockDim.x) {
        const int32_t q = q0 + threadIdx.x;
        const bool live = q < P.nq;
        const uint32_t cl = live ? P.cls[q] : 0xFFFFFFFFu;
        const int32_t nwin = live ? P.qh[q].nwin : 0;
        const unsigned same = __match_any_sync(0xffffffffu, cl);
        const int leader = __ffs(same) - 1;
        // items of the group's lanes before this one, and of the whole group
        int32_t before = 0, group = 0;
        for (unsigned m = same; m; m &= m - 1) {
            const int l = __ffs(m) - 1;
            const int32_t w = __shfl_sync(same, nwin, l);
            if (l < lane) before += w;
            group += w;
        }
        int32_t base = 0;
        if (live && lane == leader) base = atomicAdd(&P.class_count[cl], group);
        base = __shfl_sync(same, base, leader);
        if (live) {
            const int32_t pos = base + before;
            for (int32_t part = 0; part < nwin; ++part) P.items[pos + part] = Item{q, part};
        }
    }
}

// The planner's summary and the status word into the caller's pinned
// return area (one small kernel instead of two copies).
__global__ void dplan_return(const DPlanSummary *sum, const int32_t *status, DPlanSummary *h_sum,
                             int32_t *h_status)
{
    if (threadIdx.x == 0) {
        *h_sum = *sum;
        h_status[0] = status[0];
        h_status[1] = status[1];
    }
}

}  // namespace

// Plans and runs a count batch on the device (see the top of this file).
// Returns FC_OK with *done set when the batch was counted, FC_OK with *done
// clear when the host planner must take it (nothing was written), or an
// error code.
int device_count_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                       const int64_t *table_off, int32_t *tables, bool *done)
{
    *done = false;
    const Options &o = c->opt;
    constexpr int kSmallThreads = 256, kSmallCtas = 6, kSmallCells = 8192;
    if (!o.device_plan || (o.strategy != FC_STRAT_AUTO && o.strategy != FC_STRAT_HIST) || !o.shape_auto ||
        !o.window_wide || c->m >= (1 << 19) || c->transactions || nq < 1)
        return FC_OK;
    const int32_t nvars = var_off[nq] - var_off[0];
    if (var_off[0] < 0 || nvars < 0) return FC_OK;
    const int max_cells = std::max(1, std::min<int>(o.smem_cells, (c->max_smem_optin - 4096) / 4));
    if (max_cells <= kSmallCells) return FC_OK;
    const int grid = c->num_sms * kSmallCtas;

    // The caller's lists go into the pinned staging buffer and up in one
    // copy (reading them in place from page-locked memory measured slower:
    // the describe kernel's chains of dependent loads then cross the link).
    // The staging buffer also receives the summary and the status word at
    // the end.
    const size_t b_off = round_up(sizeof(int32_t) * (nq + 1), 256);
    const size_t b_vars = round_up(sizeof(int32_t) * std::max(nvars, 1), 256);
    const size_t b_user = table_off ? round_up(sizeof(int64_t) * (nq + 1), 256) : 0;
    const size_t in_bytes = b_off + b_vars + b_user;
    static_assert(sizeof(DPlanSummary) + 2 * sizeof(int32_t) <= 256, "return area");
    uint8_t *h = stage_host(c, in_bytes + 256);
    if (!h) return FC_OK;
    if (c->entropy_stale) {  // the FP32 entropies after a load or an append
        if (!c->d_entropy_f && cudaMalloc(&c->d_entropy_f, sizeof(float) * std::max(c->n, 1)) != cudaSuccess) {
            (void)cudaGetLastError();
            c->d_entropy_f = nullptr;
            return FC_OK;  // the host planner takes the batch
        }
        std::vector<float> f(c->entropy.begin(), c->entropy.end());
        cudaError_t e = cudaMemcpy(c->d_entropy_f, f.data(), sizeof(float) * c->n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "upload entropies");
        c->entropy_stale = false;
    }
    DPlanSummary *h_sum = (DPlanSummary *)(h + in_bytes);
    int32_t *h_status = (int32_t *)(h + in_bytes + round_up(sizeof(DPlanSummary), 8));
    std::memcpy(h, var_off, sizeof(int32_t) * (nq + 1));
    std::memcpy(h + b_off, vars + var_off[0], sizeof(int32_t) * nvars);
    if (table_off) std::memcpy(h + b_off + b_vars, table_off, sizeof(int64_t) * (nq + 1));

    // device layout: inputs | heads | QVars | items | classes | packed
    // offsets | class counts | item count | counter | summary (the last four
    // zeroed by one memset)
    const int64_t max_items = (int64_t)nq * std::min(o.window_max, kMaxWindows);
    const size_t o_qh = round_up(in_bytes, 256);
    const size_t o_qv = o_qh + round_up(sizeof(QHead) * nq, 256);
    const size_t o_it = o_qv + round_up(sizeof(QVar) * std::max(nvars, 1), 256);
    const size_t o_cl = o_it + round_up(sizeof(Item) * max_items, 256);
    const size_t o_sc = o_cl + round_up(sizeof(uint32_t) * nq, 256);
    const size_t o_cc = o_sc + round_up(sizeof(int64_t) * nq, 256);
    const size_t o_ct = o_cc + round_up(sizeof(int32_t) * kClasses, 256);  // n_items_eff, next item
    const size_t o_sum = o_ct + 256;
    const size_t total = o_sum + round_up(sizeof(DPlanSummary), 256);
    cudaError_t e = c->dplan_buf.ensure(total);
    if (e != cudaSuccess) return cuda_fail(e, "device plan buffer");
    uint8_t *d = (uint8_t *)c->dplan_buf.p;
    e = cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaEventRecord(c->stage[c->bank].ev, c->stream);
    // class counts, the item counters and the summary start from zero
    if (e == cudaSuccess) e = cudaMemsetAsync(d + o_cc, 0, total - o_cc, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device plan upload");

    DPlanParams P{};
    P.var_off = (const int32_t *)d;
    P.vars = (const int32_t *)(d + b_off);
    P.base0 = var_off[0];
    P.user_off = table_off ? (const int64_t *)(d + b_off + b_vars) : nullptr;
    P.entropy = c->d_entropy_f;
    P.arity = c->d_arity;
    P.soff = c->d_soff;
    P.n = c->n;
    P.nq = nq;
    P.rows = (float)c->m;
    P.chunks = (float)((c->m + kChunkRows - 1) / kChunkRows);
    P.hist_row = (float)o.hist_cost_row;
    P.hist_var = (float)o.hist_cost_var;
    P.flush = (float)o.flush_cost;
    P.bitmap_node = (float)o.bitmap_cost;
    P.bitmap_chunk = (float)o.bitmap_chunk_cost;
    P.small_unit = (float)o.small_cost;
    P.small_unit3 = (float)o.small3_cost;
    P.bitmap_small = o.bitmap_small;
    P.stage_slots = std::max(1, std::min(o.stage_slots, (c->max_smem_optin - 1024) /
                                                            (16 * std::max(32, std::min(256, o.bitmap_threads / 32 * 32)))));
    P.force_hist = o.strategy == FC_STRAT_HIST;
    P.window_max = std::min(o.window_max, kMaxWindows);
    P.small_cells = kSmallCells;
    P.max_cells = max_cells;
    P.min_hist = grid * 4;
    P.qh = (QHead *)(d + o_qh);
    P.qv = (QVar *)(d + o_qv);
    P.items = (Item *)(d + o_it);
    P.cls = (uint32_t *)(d + o_cl);
    P.class_count = (int32_t *)(d + o_cc);
    P.n_items_eff = (int32_t *)(d + o_ct);
    P.sum = (DPlanSummary *)(d + o_sum);
    // small CTAs spread the per-query chains of dependent loads over the SMs;
    // each stages the variables' tables when they fit 32 KiB
    const int threads = 128;
    const int blocks = (int)std::min<int64_t>((nq + threads - 1) / threads, (int64_t)c->num_sms * 8);
    const size_t var_smem = sizeof(VarInfo) * (size_t)c->n;
    P.stage_vars = var_smem <= 32768 ? 1 : 0;
    dplan_describe<<<blocks, threads, P.stage_vars ? var_smem : 0, c->stream>>>(P);
    dplan_finish<<<1, 1024, 0, c->stream>>>(P, (int64_t *)(d + o_sc));
    dplan_items<<<blocks, threads, 0, c->stream>>>(P);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "device plan launch");

    // the count launch in the small shape; its item count comes from the planner
    void *direct = o.zero_copy && table_off ? device_view(tables, sizeof(int32_t) * (size_t)table_off[nq]) : nullptr;
    const size_t out_bytes = table_off ? sizeof(int32_t) * (size_t)table_off[nq] : 0;
    int32_t *dtab = (int32_t *)direct;
    int64_t known_cells = 0;
    if (!dtab) {
        if (!table_off) {
            // the packed size is known only after planning: read the summary first
            e = cudaMemcpyAsync(h_sum, P.sum, sizeof(DPlanSummary), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "device plan summary");
            const DPlanSummary s = *h_sum;
            if (s.bad || s.n_items == 0) return FC_OK;
            known_cells = s.out_cells;
            e = c->io[0].ensure(sizeof(int32_t) * std::max<int64_t>(s.out_cells, 1));
            if (e != cudaSuccess) return cuda_fail(e, "output buffer");
            dtab = (int32_t *)c->io[0].p;
        } else {
            e = c->io[0].ensure(std::max<size_t>(out_bytes, 4));
            if (e != cudaSuccess) return cuda_fail(e, "output buffer");
            dtab = (int32_t *)c->io[0].p;
        }
    }
    CountParams C{};
    C.D = c->d_D;
    C.D4 = c->opt.codes4 ? c->d_D4 : nullptr;
    C.m_pad = c->m_pad;
    C.m = c->m;
    C.bits = c->d_bits;
    C.wstride = c->wstride;
    C.qh = P.qh;
    C.qv = P.qv;
    C.items = P.items;
    C.n_items = INT32_MAX;  // bounded by *n_items_dev
    C.n_items_dev = P.n_items_eff;
    C.next_item = P.n_items_eff + 1;
    C.tables = dtab;
    C.marg = c->d_marg;
    C.ess = 1.0;
    C.write_tables = 1;
    C.smem_cells = kSmallCells;
    C.hist_copies = o.hist_copies;
    C.small_paths = o.bitmap_small;
    e = launch_count(C, grid, kSmallThreads, (size_t)kSmallCells * 4, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "count launch");
    // the outputs (when they are not stored in place), the summary and the
    // status word come back together, after one synchronisation; a batch
    // the fast path refused leaves the caller's buffer to the host planner's run
    if (!direct) {
        const size_t bytes = table_off ? out_bytes : sizeof(int32_t) * (size_t)known_cells;
        if (bytes > 0) e = cudaMemcpyAsync(tables, dtab, bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(e, "copy outputs");
    }
    DPlanSummary *z_sum = (DPlanSummary *)device_view(h_sum, sizeof(DPlanSummary));
    int32_t *z_status = z_sum ? (int32_t *)device_view(h_status, 2 * sizeof(int32_t)) : nullptr;
    if (z_sum && z_status) {
        dplan_return<<<1, 32, 0, c->stream>>>(P.sum, c->d_status, z_sum, z_status);
        e = cudaGetLastError();
    } else {
        e = cudaMemcpyAsync(h_sum, P.sum, sizeof(DPlanSummary), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_status, c->d_status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e == cudaSuccess) e = cudaEventRecord(c->stage[c->bank].ev, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "device plan run");
    const DPlanSummary s = *h_sum;
    if (h_status[0] != kStatusOk) return read_status(c, c->stream);  // reports (and clears) the status
    if (s.bad || s.n_items == 0) return FC_OK;
    *done = true;
    return FC_OK;
}

}  // namespace fc
