// fc_plan.cu -- the count and score planner (validation, strategy choice by
// a cost model, work items in longest-first order, bitmap tasks), plan
// execution as CUDA graphs, the plan API and the host-buffer count and score
// calls.
#include "fc_host.h"

#include <atomic>
#include <cmath>
#include <cstdio>
#include <numeric>

using namespace fc;

// ------------------------------------------------------------------ planner

namespace fc {

// Validates one query's variables and writes its QVars to out (room for k;
// arity-1 variables dropped, strides of the caller's order, last fastest);
// returns the cells.  Reads the context only, so planner threads may call it
// concurrently (an error's message goes to the calling thread's
// fc_last_error).
int64_t describe_into(const fc_ctx *c, const int32_t *vars, int32_t k, QVar *out, int32_t &k_eff)
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
    // strides from the last variable; the kept variables are written from
    // the back of their run and moved to its front
    int64_t stride = 1;
    int32_t n_kept = 0;
    for (int t = k - 1; t >= 0; --t) {
        const int v = vars[t];
        if (c->arity[v] > 1) out[k - 1 - n_kept++] = QVar{v, (int32_t)stride, c->arity[v], c->soff[v]};
        stride *= c->arity[v];
    }
    if (n_kept < k) std::memmove(out, out + (k - n_kept), sizeof(QVar) * n_kept);
    k_eff = n_kept;
    return cells;
}

int64_t describe(const fc_ctx *c, const int32_t *vars, int32_t k, std::vector<QVar> &qv, int32_t &k_eff)
{
    const size_t first = qv.size();
    qv.resize(first + (size_t)std::max(k, 0));
    const int64_t cells = describe_into(c, vars, k, qv.data() + first, k_eff);
    qv.resize(cells < 0 ? first : first + (size_t)k_eff);
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

// Threads per CTA of the bitmap kernel (its launch bound is 256) and the
// state rows a warp stages per chunk (16 bytes per row and thread, within one
// CTA's shared memory).
int bitmap_threads(const fc_ctx *c) { return std::max(32, std::min(256, c->opt.bitmap_threads / 32 * 32)); }
int stage_slots(const fc_ctx *c)
{
    return std::max(1, std::min(c->opt.stage_slots, (c->max_smem_optin - 1024) / (16 * bitmap_threads(c))));
}

bool bitmap_ok(const fc_ctx *c, const QVar *v, int k, QVar *o)
{
    if (k < 1 || k > kMaxBitmapK) return false;
    std::copy(v, v + k, o);
    entropy_order(c, o, k);
    int slots = 0;
    for (int t = 1; t < k; ++t) slots += o[t].arity;
    return slots <= stage_slots(c);
}

// Strategy and cost of one query.  When the bitmap strategy is chosen, the
// variables are left in v in entropy order (the order its kernel walks).
QPlan choose(const fc_ctx *c, QVar *v, int k, int64_t cells, int32_t smem_cells, int32_t win_cells, double chunks)
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
        // the fitted unit cost of the register-blocked path includes its
        // per-chunk overhead (no separate chunk term)
        bitmap = chunks * small_units(ord, k) * (double)(k == 2 ? o.small_cost : o.small3_cost) + flush;
    const double gatomic = rows * (o.hist_cost_row + (double)k * o.hist_cost_var) * 2.0 + (double)cells * 4.0;
    // one pass over the rows per window of the cell range, scalar keys
    const double windows = (double)((cells + win_cells - 1) / win_cells);
    const double window = windows * rows * (o.hist_cost_row + (double)k * o.hist_cost_var) * 2.0 + flush;
    int32_t s = o.strategy;
    if (k == 0) s = fits ? FC_STRAT_HIST : FC_STRAT_GATOMIC;
    if (k == 1 && fits && (s == FC_STRAT_AUTO || s == FC_STRAT_HIST)) return QPlan{FC_STRAT_MARGINAL, flush};
    if (s == FC_STRAT_BITMAP && !bm) s = FC_STRAT_AUTO;
    if (s == FC_STRAT_HIST && !fits) s = FC_STRAT_AUTO;
    if (s == FC_STRAT_WINDOW && windows > kMaxWindows) s = FC_STRAT_AUTO;
    if (s == FC_STRAT_AUTO) {
        if (fits)
            s = bitmap < hist ? FC_STRAT_BITMAP : FC_STRAT_HIST;
        else if (cells >= o.sort_min_cells)
            s = FC_STRAT_SORT;
        else
            s = windows <= std::min<double>(o.window_max, kMaxWindows) ? FC_STRAT_WINDOW : FC_STRAT_GATOMIC;
    }
    double cost = s == FC_STRAT_BITMAP ? bitmap : s == FC_STRAT_HIST ? hist : s == FC_STRAT_WINDOW ? window : gatomic;
    if (s == FC_STRAT_BITMAP) std::copy(ord, ord + k, v);
    return QPlan{s, cost};
}

// Cost class of an estimate for the longest-first orders: its exponent and
// top three mantissa bits (1/8-octave classes), complemented so that classes
// ascend as costs descend.  Fewer than 2^14 classes exist.
inline uint32_t cost_class(double v)
{
    if (!(v > 0.0)) v = 0.0;
    uint64_t b;
    std::memcpy(&b, &v, sizeof b);
    return ((1u << 14) - 1u) - (uint32_t)(b >> (52 - 3));
}

// Queries q with want(q), ordered by ascending cls[q] (descending cost), ties
// in increasing q: a counting sort over the class span [lo, hi] (longest-
// processing-time-first needs no finer order, and it avoids a comparison
// sort's mispredicted branches on thousands of queries).
template <class Want>
void order_by_class(int32_t nq, const std::vector<uint32_t> &cls, uint32_t lo, uint32_t hi, Want want,
                    std::vector<int32_t> &out, std::vector<int32_t> &start)
{
    out.clear();
    if (lo > hi) return;
    const size_t span = (size_t)(hi - lo) + 1;
    start.assign(span + 1, 0);
    int32_t n = 0;
    for (int32_t q = 0; q < nq; ++q)
        if (want(q)) {
            ++start[cls[q] - lo + 1];
            ++n;
        }
    for (size_t c = 0; c < span; ++c) start[c + 1] += start[c];
    out.resize(n);
    for (int32_t q = 0; q < nq; ++q)
        if (want(q)) out[start[cls[q] - lo]++] = q;
}

// Builds a count or score plan.  span(q) gives the length of query q's
// variable list (or -1 after fail() for bad offsets); get(q, ...) the list.
// The query heads and QVars are written straight into the pinned staging
// buffer by the context's host threads, which take the queries in blocks and
// also gather what the serial steps need (totals per strategy, compact
// per-query cells, cost classes), so that those steps read small arrays and
// touch the heads only where a value changes.
template <class Span, class GetVars>
int build_count_plan(fc_ctx *c, int32_t nq, Span span, GetVars get, const int64_t *user_off, int score_kind,
                     double ess, fc_plan **out)
{
    if (c->transactions) return fail(FC_ERR_STATE, "context holds transaction bitmaps; use the support calls");
    if (nq < 0) return fail(FC_ERR_ARG, "nq < 0");
    if (!c->plan_scratch) c->plan_scratch.reset(new (std::nothrow) PlanScratch());
    if (!c->plan_scratch) return fail(FC_ERR_OOM, "host allocation failed");
    PlanScratch &S = *c->plan_scratch;
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
    int threads = std::max(32, std::min(512, o.threads / 32 * 32));
    int ctas_per_sm = std::max(1, o.ctas_per_sm);
    int max_cells = std::max(1, std::min<int>(o.smem_cells, (c->max_smem_optin - 4096) / 4));
    // cells of one window of a windowed table: the whole shared memory of an
    // SM in the wide launch, else the mixed launch's table area
    const bool wide = o.window_wide != 0;
    // the small launch shape (more, smaller CTAs: their per-item barriers and
    // flushes overlap better) when few shared-memory tables need more room
    constexpr int kSmallShapeThreads = 256, kSmallShapeCtas = 6, kSmallShapeCells = 8192;
    const bool auto_shape = o.shape_auto != 0 && wide && max_cells > kSmallShapeCells;
    const int win_cells = std::max(1, std::min<int>(o.window_cells, wide ? (c->max_smem_optin - 4096) / 4 : max_cells));
    const double chunks_d = (double)((c->m + kChunkRows - 1) / kChunkRows);
    constexpr int32_t kThreadedQueries = 2048;  // smaller batches plan on the calling thread

    // each query's QVars get slots of its list's length (arity-1 variables
    // leave the end of a run unused)
    S.base.resize((size_t)nq + 1);
    S.base[0] = 0;
    for (int32_t q = 0; q < nq; ++q) {
        const int32_t k = span(q);
        if (k < 0) {
            fc_plan_free(p);
            return FC_ERR_ARG;
        }
        S.base[q + 1] = S.base[q] + k;
    }
    const int64_t nvars = S.base[nq];
    if (nvars > INT32_MAX) {
        fc_plan_free(p);
        return fail(FC_ERR_SIZE, "batch lists %lld variables", (long long)nvars);
    }

    // staging layout: [heads | QVars | items | score list | bitmap tasks]
    const size_t o_qv = round_up(sizeof(QHead) * std::max(nq, 1), 256);
    const size_t o_rest = o_qv + round_up(sizeof(QVar) * std::max<int64_t>(nvars, 1), 256);
    uint8_t *host = stage_host(c, o_rest + S.rest_bytes);
    if (!host) {
        fc_plan_free(p);
        return fail(FC_ERR_OOM, "pinned staging of %zu bytes", o_rest + S.rest_bytes);
    }
    QHead *qh = reinterpret_cast<QHead *>(host);
    QVar *qv = reinterpret_cast<QVar *>(host + o_qv);
    S.cost.resize(nq);
    S.cells.resize(nq);
    S.cls.resize(nq);
    S.passes.resize(nq);
    p->strategy.resize(nq);
    p->table_off.assign(nq + 1, 0);

    // Per query: validation, QVars, strategy, heads.  Host threads take
    // blocks of queries in order; the lowest failing query is reported
    // (blocks past a failure are skipped, blocks before it all finish).
    constexpr int32_t kBlock = 256;
    int nthreads = 1;
    if (nq >= kThreadedQueries)
        nthreads = (int)std::max<int64_t>(1, std::min<int64_t>(fc::host_threads(c), nq / 512));
    struct Tally {
        int32_t fail_q = INT32_MAX;
        int fail_code = 0;
        std::string fail_msg;
        int64_t n[6] = {0, 0, 0, 0, 0, 0};  // queries per strategy
        int64_t window_items = 0;             // windows of the wide launch's queries
        int64_t mixed_windows = 0;            // windows counted in the mixed launch
        int64_t mid_hist = 0;                 // shared-memory tables beyond the small launch shape
        double hist_cost = 0.0, hist_cost_256 = 0.0;  // histogram work, and that on tables of >= 256 cells
        double bitmap_cost = 0.0;
        uint32_t lo[2] = {UINT32_MAX, UINT32_MAX}, hi[2] = {0, 0};  // class spans: [0] items, [1] bitmap
        std::vector<int32_t> sorts;
    };
    std::vector<Tally> tallies(nthreads);
    std::atomic<int32_t> next_block{0}, first_bad{INT32_MAX};
    auto work = [&](int t) {
        std::vector<int32_t> buf;
        Tally &T = tallies[t];
        auto failed = [&](int32_t q, int code) {
            T.fail_q = q;
            T.fail_code = code;
            T.fail_msg = g_err;
            int32_t cur = first_bad.load(std::memory_order_relaxed);
            while (q < cur && !first_bad.compare_exchange_weak(cur, q, std::memory_order_relaxed)) {
            }
        };
        for (;;) {
            const int32_t q0 = next_block.fetch_add(kBlock, std::memory_order_relaxed);
            if (q0 >= nq || q0 > first_bad.load(std::memory_order_relaxed)) return;
            const int32_t q1 = std::min(nq, q0 + kBlock);
            for (int32_t q = q0; q < q1; ++q) {
                const int32_t *vars;
                int32_t k, child, k_eff = 0;
                int64_t cells = FC_ERR_ARG;
                QVar *qq = qv + S.base[q];
                if (get(q, vars, k, child, buf)) cells = describe_into(c, vars, k, qq, k_eff);
                if (cells < 0) return failed(q, (int)cells);
                int64_t toff = 0;
                if (user_off) {
                    if (user_off[q + 1] - user_off[q] < cells || user_off[q] < 0) {
                        fail(FC_ERR_ARG, "table_off of query %d leaves %lld cells, it needs %lld", q + c->q_base,
                             (long long)(user_off[q + 1] - user_off[q]), (long long)cells);
                        return failed(q, FC_ERR_ARG);
                    }
                    toff = user_off[q];
                    p->table_off[q] = toff;
                }
                const QPlan ch = choose(c, qq, k_eff, cells, max_cells, win_cells, chunks_d);
                const int s = ch.strategy;
                const int32_t nwin = s == kWindow ? (int32_t)((cells + win_cells - 1) / win_cells) : 1;  // <= kMaxWindows
                QHead &h = qh[q];
                h.table_off = toff;
                h.cells = (int32_t)cells;
                h.var_off = (int32_t)S.base[q];
                h.k = (int16_t)k_eff;
                h.strategy = (int16_t)s;
                h.nparts = (int16_t)nwin;  // row splits and bitmap tasks are set later
                h.score_kind = (int16_t)score_kind;
                h.r_child = score_kind == kNoScore ? 1 : c->arity[child];
                h.child_soff = score_kind == kNoScore ? 0 : c->soff[child];
                h.score_slot = q;
                h.nwin = nwin;
                p->strategy[q] = s;
                S.cost[q] = ch.cost;
                S.cells[q] = (int32_t)cells;
                const uint32_t cl = cost_class(ch.cost / nwin);
                S.cls[q] = cl;
                S.passes[q] = (uint8_t)((s == kBitmap && o.bitmap_small && k_eff == 3 && small_ok(qq, 3)) ? qq[0].arity : 0);
                ++T.n[s];
                if (s == kHist && cells > kSmallShapeCells) ++T.mid_hist;
                if (s == kHist) {
                    T.hist_cost += ch.cost;
                    if (cells >= 256) T.hist_cost_256 += ch.cost;
                }
                if (s == kSort) {
                    T.sorts.push_back(q);
                } else {
                    const int g = s == kBitmap ? 1 : 0;
                    T.lo[g] = std::min(T.lo[g], cl);
                    T.hi[g] = std::max(T.hi[g], cl);
                    if (s == kBitmap) T.bitmap_cost += ch.cost;
                    if (s == kWindow) T.window_items += nwin;
                }
            }
        }
    };
    fc::run_host_threads(c, nthreads, work);
    Tally all;
    {
        const Tally *worst = nullptr;
        for (const Tally &T : tallies)
            if (T.fail_q != INT32_MAX && (!worst || T.fail_q < worst->fail_q)) worst = &T;
        if (worst) {
            fc_plan_free(p);
            return fail(worst->fail_code, "%s", worst->fail_msg.c_str());
        }
        for (const Tally &T : tallies) {
            for (int s = 0; s < 6; ++s) all.n[s] += T.n[s];
            all.window_items += T.window_items;
            all.mid_hist += T.mid_hist;
            all.hist_cost += T.hist_cost;
            all.hist_cost_256 += T.hist_cost_256;
            all.bitmap_cost += T.bitmap_cost;
            for (int g = 0; g < 2; ++g) {
                all.lo[g] = std::min(all.lo[g], T.lo[g]);
                all.hi[g] = std::max(all.hi[g], T.hi[g]);
            }
            all.sorts.insert(all.sorts.end(), T.sorts.begin(), T.sorts.end());
        }
        std::sort(all.sorts.begin(), all.sorts.end());
    }

    // launch shape: the small one unless more than 1/64 of the queries are
    // shared-memory tables that it cannot hold, or long row ranges (items of
    // >= 2^19 rows, whose per-item fixed costs the small CTAs save little of)
    // go mostly into tables of >= 256 cells, which get 2-8x more interleaved
    // copies (less atomic contention) in the large shape's table area.  The
    // few tables beyond the small shape's area are planned again with it (as
    // windows of it they stay in the mixed launch).
    const bool long_rows_big_tables = c->m >= (1 << 19) && all.hist_cost_256 > 0.45 * all.hist_cost;
    const bool small_shape = auto_shape && all.mid_hist * 64 <= nq && !long_rows_big_tables;
    if (small_shape) {
        threads = kSmallShapeThreads;
        ctas_per_sm = kSmallShapeCtas;
        max_cells = kSmallShapeCells;
        if (all.mid_hist > 0) S.mixed_win.assign(nq, 0);
        for (int32_t q = 0; q < nq && all.mid_hist > 0; ++q) {
            if (p->strategy[q] != kHist || S.cells[q] <= max_cells) continue;
            --all.mid_hist;
            --all.n[kHist];
            QHead &h = qh[q];
            QVar *qq = qv + h.var_off;
            const QPlan ch = choose(c, qq, h.k, S.cells[q], max_cells, max_cells, chunks_d);
            const int s = ch.strategy;
            const int32_t nwin = s == kWindow ? (int32_t)((S.cells[q] + max_cells - 1) / max_cells) : 1;
            h.strategy = (int16_t)s;
            h.nparts = (int16_t)nwin;
            h.nwin = nwin;
            p->strategy[q] = s;
            S.cost[q] = ch.cost;
            const uint32_t cl = cost_class(ch.cost / nwin);
            S.cls[q] = cl;
            S.passes[q] = (uint8_t)((s == kBitmap && o.bitmap_small && h.k == 3 && small_ok(qq, 3)) ? qq[0].arity : 0);
            ++all.n[s];
            if (s == kSort) {
                all.sorts.insert(std::lower_bound(all.sorts.begin(), all.sorts.end(), q), q);
            } else {
                const int g = s == kBitmap ? 1 : 0;
                all.lo[g] = std::min(all.lo[g], cl);
                all.hi[g] = std::max(all.hi[g], cl);
                if (s == kBitmap) all.bitmap_cost += ch.cost;
                if (s == kWindow) {
                    all.mixed_windows += nwin;
                    S.mixed_win[q] = 1;
                }
            }
        }
    }
    auto mixed_window = [&](int32_t q) { return all.mixed_windows > 0 && S.mixed_win[q]; };
    p->threads = threads;
    p->smem_cells = max_cells;

    // table offsets of count plans: the caller's, else dense in query order
    if (score_kind == kNoScore) {
        if (user_off) {
            p->table_off[nq] = user_off[nq];
        } else {
            int64_t off = 0;
            for (int32_t q = 0; q < nq; ++q) {
                p->table_off[q] = off;
                qh[q].table_off = off;
                off += S.cells[q];
            }
            p->table_off[nq] = off;
        }
        p->out_cells = p->table_off[nq];
    }

    // work items: split rows when the batch alone cannot fill the GPU
    p->grid = c->num_sms * ctas_per_sm;
    p->smem = (size_t)max_cells * 4;
    const int64_t nchunks = (c->m + kChunkRows - 1) / kChunkRows;
    const int64_t max_parts_rows = std::max<int64_t>(1, c->m / std::max<int64_t>(o.min_part_rows, kChunkRows));
    const int64_t persistent = all.n[kHist] + all.n[kGAtomic];
    // (marginal items hold no rows, so they never split)
    const int64_t target = (int64_t)p->grid * 4;
    int64_t parts = 1;
    if (persistent > 0 && persistent < target)
        parts = std::min<int64_t>({nchunks, max_parts_rows, (target + persistent - 1) / persistent, 32767});
    parts = std::max<int64_t>(1, parts);
    // windowed queries split their rows only when their windows alone would
    // leave CTAs idle: a split window adds its nonzero cells to the table
    // with atomics instead of storing every cell once
    p->wgrid = wide ? c->num_sms : p->grid;
    p->wsmem = (size_t)win_cells * 4;
    int64_t wparts = 1;
    if (all.window_items > 0 && all.window_items < p->wgrid)
        wparts = std::min<int64_t>(
            {nchunks, max_parts_rows, (2 * (int64_t)p->wgrid + all.window_items - 1) / all.window_items});
    wparts = std::max<int64_t>(1, wparts);
    int64_t window_parts = all.window_items;  // items of all windowed queries
    if (parts > 1 || wparts > 1) {
        window_parts = 0;
        for (int32_t q = 0; q < nq; ++q) {
            const int s = p->strategy[q];
            if (s == kHist || s == kGAtomic) {
                qh[q].nparts = (int16_t)parts;
            } else if (s == kWindow && !mixed_window(q)) {
                const int32_t nwin = qh[q].nwin;
                qh[q].nparts = (int16_t)(std::max<int64_t>(1, std::min<int64_t>(wparts, 32767 / nwin)) * nwin);
                window_parts += qh[q].nparts;
            }
        }
    }
    const int64_t n_narrow = persistent * parts + all.n[kMarginal] + all.mixed_windows + (wide ? 0 : window_parts);
    p->n_items = (int32_t)n_narrow;
    p->n_witems = (int32_t)(wide ? window_parts : 0);

    // bitmap queries: warp tasks of consecutive 4096-row chunks, heaviest
    // queries first.  A query gets tasks in proportion to its estimated cost
    // (about four tasks' worth of work per warp of the launch), each of at
    // least kMinTaskChunks chunks, so that light queries are not cut into
    // tasks whose fixed costs (dispatch, one reduction and atomic per cell)
    // outweigh their work.
    std::vector<BTask> &btasks = S.btasks;
    btasks.clear();
    p->bm_threads = bitmap_threads(c);
    p->stage_slots = stage_slots(c);
    p->small_paths = o.bitmap_small;
    if (all.n[kBitmap] > 0) {
        constexpr int64_t kMinTaskChunks = 4;
        std::vector<int32_t> &order = S.order;
        order_by_class(nq, S.cls, all.lo[1], all.hi[1], [&](int32_t q) { return p->strategy[q] == kBitmap; },
                       order, S.start);
        p->bm_grid = c->num_sms * bitmap_ctas_per_sm(p->bm_threads, p->stage_slots);
        const int64_t warps = (int64_t)p->bm_grid * (p->bm_threads / 32);
        const double unit = std::max(all.bitmap_cost / (4.0 * (double)warps), 1e-30);
        const int64_t max_tasks = std::max<int64_t>(1, std::min<int64_t>(nchunks / kMinTaskChunks, 32767));
        for (const int32_t q : order) {
            // a 3-variable register-blocked query splits by the first
            // variable's state as well (one pass over the chunks per state);
            // its tasks (the score ticket count) stay below 2^15
            const int32_t passes = S.passes[q];
            const int32_t pmul = std::max(1, passes);
            const double per = S.cost[q] / pmul;
            const int64_t t = std::max<int64_t>(
                1, std::min<int64_t>({max_tasks, 32767 / pmul, (int64_t)std::ceil(per / unit)}));
            qh[q].nparts = (int16_t)(t * pmul);
            // t balanced chunk ranges: the first nchunks % t get one extra chunk
            const int64_t base = nchunks / t, rem = nchunks % t;
            for (int32_t s0 = passes > 0 ? 0 : -1; s0 < passes; ++s0) {
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

    // tables that must exist in global memory for score plans: all but the
    // shared-memory ones of a single item
    if (score_kind != kNoScore) {
        int64_t off = 0;
        for (int32_t q = 0; q < nq; ++q) {
            const int s = p->strategy[q];
            const bool global = s == kMarginal ? false : s == kHist ? parts > 1 : true;
            if (global) {
                qh[q].table_off = off;
                off += S.cells[q];
            }
        }
        p->table_buf_cells = off;
    } else {
        p->table_buf_cells = p->out_cells;
    }
    // tables some item adds to (rather than stores whole) start from zero
    p->zero_tables = all.n[kBitmap] + all.n[kGAtomic] + all.n[kSort] > 0 || (all.n[kHist] > 0 && parts > 1) ||
                     (all.n[kWindow] > 0 && wparts > 1);
    std::vector<int32_t> &qlist = S.qlist;
    qlist.clear();
    for (const int32_t q : all.sorts) {
        const QHead &h = qh[q];
        SortJob j{q, h.k, 0, h.cells, 0, nullptr};
        j.table_off = h.table_off;
        j.key_bits = j.cells > 1 ? 32 - __builtin_clz((uint32_t)(j.cells - 1)) : 0;
        p->sort_jobs.push_back(j);
        if (score_kind != kNoScore) qlist.push_back(q);
    }
    p->n_qlist = (int32_t)qlist.size();

    // the rest of the staging buffer: items straight into it (heaviest
    // first by cost per part, a query's parts consecutive, the windows of
    // the wide launch after the mixed launch's items), then the score list
    // and the bitmap tasks
    const size_t n_all_items = (size_t)(n_narrow + p->n_witems);
    const size_t b_it = sizeof(Item) * std::max<size_t>(n_all_items, 1);
    const size_t b_ql = sizeof(int32_t) * std::max<size_t>(qlist.size(), 1);
    const size_t b_bq = sizeof(BTask) * std::max<size_t>(btasks.size(), 1);
    const size_t o_it = o_rest, o_ql = o_it + round_up(b_it, 256), o_bq = o_ql + round_up(b_ql, 256);
    const size_t total = o_bq + round_up(b_bq, 256);
    S.rest_bytes = total - o_rest;
    host = stage_grow(c, total, o_rest);
    if (!host) {
        fc_plan_free(p);
        return fail(FC_ERR_OOM, "pinned staging of %zu bytes", total);
    }
    qh = reinterpret_cast<QHead *>(host);
    {
        Item *it = reinterpret_cast<Item *>(host + o_it);
        Item *const it_end = it + n_narrow;
        Item *wit = it_end;
        Item *const wit_end = wit + p->n_witems;
        auto item_query = [&](int32_t q) {
            const int s = p->strategy[q];
            return s == kHist || s == kGAtomic || s == kMarginal || s == kWindow;
        };
        std::vector<int32_t> &order = S.order;
        order_by_class(nq, S.cls, all.lo[0], all.hi[0], item_query, order, S.start);
        bool fits = true;  // the counts taken above size both regions exactly
        for (const int32_t q : order) {
            const int s = p->strategy[q];
            const int32_t np = s == kMarginal ? 1 : s == kWindow ? qh[q].nparts : (int32_t)parts;
            const bool to_wide = wide && s == kWindow && !mixed_window(q);
            Item *&dst = to_wide ? wit : it;
            if (dst + np > (to_wide ? wit_end : it_end)) {
                fits = false;
                break;
            }
            for (int32_t part = 0; part < np; ++part) *dst++ = Item{q, part};
        }
        if (!fits || it != it_end || wit != wit_end) {
            fc_plan_free(p);
            return fail(FC_ERR_STATE, "planner: work items do not match their count");
        }
    }
    std::memcpy(host + o_ql, qlist.data(), sizeof(int32_t) * qlist.size());
    std::memcpy(host + o_bq, btasks.data(), sizeof(BTask) * btasks.size());
    cudaError_t e = plan_buf(c, p->desc, 0, total);
    if (e == cudaSuccess) e = upload_stage(c, p->desc.p, total);
    p->upload_bytes = total;
    p->n_counters = 3 + nq;  // next item, next bitmap task, tickets, next wide item
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
    if (p->n_items > 0 || p->n_witems > 0 || p->n_btasks > 0) {
        CountParams P{};
        P.D = c->d_D;
        P.D4 = c->opt.codes4 ? c->d_D4 : nullptr;
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
        if (p->n_witems > 0) {
            CountParams W = P;
            W.items = p->d_items + p->n_items;
            W.n_items = p->n_witems;
            W.next_item = (int32_t *)p->counters.p + 2 + p->nq;
            W.smem_cells = (int32_t)(p->wsmem / 4);
            e = launch_count_wide(W, std::min<int64_t>(p->wgrid, p->n_witems), p->wsmem, s);
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

// Device address of a caller's host output buffer [h, h + bytes) when the
// whole buffer is page-locked host memory the GPU can store to (cudaHostAlloc,
// or cudaHostRegister with mapping; on a GB300 node such stores travel over
// the CPU-GPU link while the kernel runs), else nullptr.
void *device_view(const void *h, size_t bytes)
{
    if (!h || bytes == 0) return nullptr;
    const uint8_t *first = (const uint8_t *)h, *last = first + bytes - 1;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, first) != cudaSuccess || cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if ((const uint8_t *)b.devicePointer - (const uint8_t *)a.devicePointer != (ptrdiff_t)(bytes - 1)) return nullptr;
    return a.devicePointer;
}

// A count or score plan whose kernels only store to the output (no output
// cell is accumulated, so nothing must be zeroed first) can write straight
// into a caller's page-locked host buffer instead of a device buffer that is
// copied afterwards.
bool stores_only(const fc_plan *p)
{
    if (p->kind == kPlanScore || p->kind == kPlanPairs) return true;  // pairs: the extraction kernel stores
    return p->kind == kPlanCount && !p->zero_tables && p->sort_jobs.empty();
}

// Runs a plan on the context stream with runtime-owned device outputs and
// copies them to the caller's host buffers (or, for a plan that only stores
// its outputs, has the kernels write page-locked host buffers directly).
int run_to_host(fc_plan *p, void *h0, size_t b0, void *h1, size_t b1, void *h2, size_t b2)
{
    fc_ctx *c = p->ctx;
    void *hs[3] = {h0, h1, h2};
    size_t bs[3] = {b0, b1, b2};
    void *ds[3] = {nullptr, nullptr, nullptr};
    if (c->opt.zero_copy && stores_only(p)) {
        // every output the caller wants is page-locked: the kernels store into it
        void *dv[3] = {nullptr, nullptr, nullptr};
        bool all = false;
        for (int i = 0; i < 3; ++i) {
            if (!hs[i] || bs[i] == 0) continue;
            dv[i] = device_view(hs[i], bs[i]);
            all = dv[i] != nullptr;
            if (!all) break;
        }
        if (all) {
            int rc = run_plan(p, dv[0], dv[1], dv[2], c->stream, false);
            if (rc != FC_OK) return rc;
            return read_status(c, c->stream);
        }
    }
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

}  // namespace fc

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
    auto span = [&](int32_t q) -> int32_t {
        const int32_t a = var_off[q], b = var_off[q + 1];
        if (a < 0 || b < a) return fail(FC_ERR_ARG, "var_off must be non-decreasing and non-negative"), -1;
        return b - a;
    };
    return build_count_plan(c, nq, span, get, table_off, kNoScore, 1.0, out);
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
    auto span = [&](int32_t q) -> int32_t {
        const int32_t a = par_off[q], b = par_off[q + 1];
        if (a < 0 || b < a || (b > a && !parents))
            return fail(FC_ERR_ARG, "par_off must be non-decreasing and non-negative"), -1;
        if (b - a >= INT32_MAX) return fail(FC_ERR_ARG, "parent list too long"), -1;
        return b - a + 1;
    };
    return build_count_plan(c, nq, span, get, nullptr, kind, ess, out);
}

namespace {
// Kernels one fc_plan_run launches when every output is given (memsets and
// graph bookkeeping excluded).
int64_t plan_launches(const fc_plan *p)
{
    switch (p->kind) {
    case kPlanCount:
    case kPlanScore:
        return (p->n_btasks > 0) + (p->n_items > 0) + (p->n_witems > 0) + (int64_t)p->sort_jobs.size() +
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

namespace fc {
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
}  // namespace fc

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

namespace {

// Batches at least this large run a synchronous call in parts (10,000
// count queries: 0.68 ms per call in two parts, 0.76 ms in three equal ones,
// whose smaller plans use fewer host threads and launch more often).
constexpr int32_t kPipelineQueries = kDevicePlanMinQueries;

// A synchronous call in parts of its batch: each part after the first is
// planned on the host while the previous part's kernels run, and each part's
// output is copied to the host on a second stream while the GPU goes on.
// Parts alternate between two banks of lent buffers; a part's kernels wait
// for the copy-out of the part before it in the same bank.  build(q0, q1,
// &plan, &offset, &bytes) plans queries [q0, q1) and says where its output
// goes in the host buffer.
// The parts end at cuts[i] / 8 of the batch.  A part's kernels hide the
// next part's planning only while they run longer than it plans; a score
// query costs the GPU about four times what it costs the planner, so score
// batches start with a quarter (50,000 queries: 8.45 ms per call against
// 8.85 ms in halves; three parts of 1/8, 2/8 and 5/8 measured the same as
// two), while count batches, which plan about as fast as they count, split
// in halves.
constexpr int kCountCuts[] = {4, 8};
constexpr int kScoreCuts[] = {2, 8};
template <class Build, int kParts>
int run_in_parts(fc_ctx *c, int32_t nq, uint8_t *host, Build build, const int (&cuts)[kParts])
{
    if (!c->out_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&c->out_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            c->out_stream = nullptr;
            return cuda_fail(e, "cudaStreamCreate");
        }
    }
    for (cudaEvent_t *evs : {c->part_done, c->copy_done})
        for (int b = 0; b < 2; ++b)
            if (!evs[b]) {
                cudaError_t e = cudaEventCreateWithFlags(&evs[b], cudaEventDisableTiming);
                if (e != cudaSuccess) {
                    evs[b] = nullptr;
                    return cuda_fail(e, "cudaEventCreate");
                }
            }
    constexpr int parts = kParts;
    fc_plan *plans[parts] = {};
    int rc = FC_OK;
    for (int i = 0; i < parts && rc == FC_OK; ++i) {
        const int bank = i & 1;
        const int32_t q0 = i == 0 ? 0 : (int32_t)((int64_t)nq * cuts[i - 1] / 8);
        const int32_t q1 = (int32_t)((int64_t)nq * cuts[i] / 8);
        size_t off = 0, bytes = 0;
        {
            BorrowScope b(c, bank);
            c->q_base = q0;
            rc = build(q0, q1, &plans[i], &off, &bytes);
            c->q_base = 0;
        }
        if (rc != FC_OK) break;
        // a part whose kernels only store their outputs writes the caller's
        // page-locked buffer directly: no device buffer, no copy
        void *direct = c->opt.zero_copy && stores_only(plans[i]) ? device_view(host + off, bytes) : nullptr;
        if (direct) {
            rc = run_plan(plans[i], direct, nullptr, nullptr, c->stream, false);
            if (rc != FC_OK) break;
            continue;
        }
        cudaError_t e = c->pipe_io[bank].ensure(std::max<size_t>(bytes, 4));
        // the bank's output buffer is free once the earlier part's copy ends
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(c->stream, c->copy_done[bank], 0);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "output buffer");
            break;
        }
        rc = run_plan(plans[i], c->pipe_io[bank].p, nullptr, nullptr, c->stream, false);
        if (rc != FC_OK) break;
        e = cudaEventRecord(c->part_done[bank], c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(c->out_stream, c->part_done[bank], 0);
        if (e == cudaSuccess && bytes > 0)
            e = cudaMemcpyAsync(host + off, c->pipe_io[bank].p, bytes, cudaMemcpyDeviceToHost, c->out_stream);
        if (e == cudaSuccess) e = cudaEventRecord(c->copy_done[bank], c->out_stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy outputs");
    }
    const cudaError_t e = cudaStreamSynchronize(c->out_stream);
    const int status = read_status(c, c->stream);
    for (fc_plan *p : plans)
        if (p) fc_plan_free(p);
    if (rc != FC_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "copy outputs");
    return status;
}

}  // namespace

extern "C" int fc_count_batch(fc_ctx *c, int32_t nq, const int32_t *var_off, const int32_t *vars,
                              const int64_t *table_off, int32_t *tables)
{
    if (!c || (nq > 0 && !tables)) return fail(FC_ERR_ARG, "fc_count_batch: null argument");
    DevGuard g(c->device);
    c->last_batch_on_device = 0;
    if (nq >= kPipelineQueries && var_off && vars && !c->transactions) {
        // planned on the device when every query counts in shared memory
        bool done = false;
        const int rc = device_count_batch(c, nq, var_off, vars, table_off, tables, &done);
        c->last_batch_on_device = rc == FC_OK && done ? 1 : 0;
        if (rc != FC_OK || done) return rc;
        if (table_off && table_off[0] < 0) return fail(FC_ERR_ARG, "table_off must be non-negative");
        std::vector<int64_t> rel;
        int64_t dense = 0;  // cells of the earlier parts when the tables are packed
        auto build = [&](int32_t q0, int32_t q1, fc_plan **p, size_t *off, size_t *bytes) -> int {
            const int64_t *uo = nullptr;
            if (table_off) {
                rel.resize((size_t)(q1 - q0) + 1);
                for (int32_t q = q0; q <= q1; ++q) rel[q - q0] = table_off[q] - table_off[q0];
                uo = rel.data();
            }
            const int rc = fc_plan_count(c, q1 - q0, var_off + q0, vars, uo, p);
            if (rc != FC_OK) return rc;
            const int64_t base = table_off ? table_off[q0] : dense;
            dense += (*p)->out_cells;
            *off = sizeof(int32_t) * (size_t)base;
            *bytes = sizeof(int32_t) * (size_t)(*p)->out_cells;
            return FC_OK;
        };
        return run_in_parts(c, nq, reinterpret_cast<uint8_t *>(tables), build, kCountCuts);
    }
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
    if (nq >= kPipelineQueries && child && par_off && !c->transactions) {
        auto build = [&](int32_t q0, int32_t q1, fc_plan **p, size_t *off, size_t *bytes) -> int {
            const int rc = fc_plan_score(c, q1 - q0, child + q0, par_off + q0, parents, kind, ess, p);
            *off = sizeof(float) * (size_t)q0;
            *bytes = sizeof(float) * (size_t)(q1 - q0);
            return rc;
        };
        return run_in_parts(c, nq, reinterpret_cast<uint8_t *>(scores), build, kScoreCuts);
    }
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

