// fc_sets.cu -- plans over sets of bitmap rows: itemset supports with their
// leave-one-out supports or every antecedent split (Sec. 4.3), specific
// assignments (end of Sec. 3.3), and the itemset counts the rule miner uses.
#include "fc_host.h"

#include <numeric>

using namespace fc;

// ----------------------------------------------------------------- support

namespace fc {

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
    // the finishing pass fills one-item subsets from the marginals (and the
    // confidences, when asked for)
    if (!P.full_only) e = launch_support_confidence(P, s);
    return e;
}

}  // namespace fc

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

namespace fc {

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
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, support_kernel_ptr(mode, threads), threads, 0);
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
    P.marg = c->d_marg;
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
    // the all-splits kernel keeps 16-bit counts per lane: a work item spans
    // at most 511 steps of 64 words
    if (mode == 2) nparts = std::max<int64_t>(nparts, (c->words + 511 * 64 - 1) / (511 * 64));
    P.nparts = (int32_t)std::min<int64_t>(nparts, 1 << 20);
    P.words_per_part = (int32_t)round_up((c->words + P.nparts - 1) / P.nparts, 64);
    *out = p;
    return FC_OK;
}

}  // namespace fc

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

