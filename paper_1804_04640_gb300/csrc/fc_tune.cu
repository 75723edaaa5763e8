// fc_tune.cu -- options of a context, the bounded-wait self test, and the
// autotuners that fit the planner's cost model to this GPU and batch.
#include "fc_host.h"

#include <chrono>
#include <cmath>
#include <numeric>

using namespace fc;

// --------------------------------------------------------- options, errors

namespace {

struct OptDesc {
    const char *key;
    int64_t Options::*p64;
    int32_t Options::*p32;
    int64_t lo, hi;
};

const OptDesc kOpts[] = {
    {"strategy", nullptr, &Options::strategy, -1, 5},
    {"smem_cells", nullptr, &Options::smem_cells, 256, 1 << 20},
    {"threads", nullptr, &Options::threads, 32, 512},
    {"ctas_per_sm", nullptr, &Options::ctas_per_sm, 1, 32},
    {"hist_copies", nullptr, &Options::hist_copies, 1, 32},
    {"min_part_rows", &Options::min_part_rows, nullptr, kChunkRows, (int64_t)1 << 31},
    {"pair_chunk_rows", &Options::pair_chunk_rows, nullptr, 128, (int64_t)1 << 24},
    {"use_graph", nullptr, &Options::use_graph, 0, 1},
    {"wait_limit", &Options::wait_limit, nullptr, 1, (int64_t)1 << 40},
    {"sort_min_cells", &Options::sort_min_cells, nullptr, 1, (int64_t)1 << 31},
    {"window_max", nullptr, &Options::window_max, 0, kMaxWindows},
    {"window_cells", nullptr, &Options::window_cells, 256, 1 << 20},
    {"window_wide", nullptr, &Options::window_wide, 0, 1},
    {"shape_auto", nullptr, &Options::shape_auto, 0, 1},
    {"bitmap_cost", &Options::bitmap_cost, nullptr, 0, (int64_t)1 << 40},
    {"bitmap_chunk_cost", &Options::bitmap_chunk_cost, nullptr, 0, (int64_t)1 << 40},
    {"hist_cost_row", &Options::hist_cost_row, nullptr, 0, (int64_t)1 << 40},
    {"hist_cost_var", &Options::hist_cost_var, nullptr, 0, (int64_t)1 << 40},
    {"flush_cost", &Options::flush_cost, nullptr, 0, (int64_t)1 << 40},
    {"small_cost", &Options::small_cost, nullptr, 0, (int64_t)1 << 40},
    {"small3_cost", &Options::small3_cost, nullptr, 0, (int64_t)1 << 40},
    {"bitmap_small", nullptr, &Options::bitmap_small, 0, 1},
    {"stage_slots", nullptr, &Options::stage_slots, 1, 64},
    {"bitmap_threads", nullptr, &Options::bitmap_threads, 32, 256},
    {"support_warps", nullptr, &Options::support_warps, 1, 32},
    {"support_sets_per_warp", nullptr, &Options::support_sets_per_warp, 1, 64},
    {"support_part_words", &Options::support_part_words, nullptr, 64, (int64_t)1 << 40},
    {"zero_copy", nullptr, &Options::zero_copy, 0, 1},
    {"device_plan", nullptr, &Options::device_plan, 0, 1},
    {"codes4", nullptr, &Options::codes4, 0, 1},
};

}  // namespace

extern "C" int fc_set_option(fc_ctx *c, const char *key, int64_t value)
{
    if (!c || !key) return fail(FC_ERR_ARG, "fc_set_option: null argument");
    for (const OptDesc &d : kOpts)
        if (std::strcmp(d.key, key) == 0) {
            if (value < d.lo || value > d.hi)
                return fail(FC_ERR_ARG, "option %s must be in %lld..%lld", key, (long long)d.lo, (long long)d.hi);
            if (d.p32 == &Options::strategy && value == FC_STRAT_MARGINAL)
                return fail(FC_ERR_ARG, "the marginal strategy is chosen by the planner, never forced");
            if (d.p32 == &Options::threads || d.p32 == &Options::ctas_per_sm || d.p32 == &Options::smem_cells)
                c->opt.shape_auto = 0;  // an explicit launch shape
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
    // small_cost (2 variables) and small3_cost (3) = time / (chunks x work
    // units), fitted apart and with the path's per-chunk overhead folded in
    // (the tree walk's chunk cost, fitted above, does not carry over)
    std::vector<int32_t> small_vars;
    for (int v = 0; v < c->n; ++v)
        if (c->arity[v] >= 2 && c->arity[v] <= 5) small_vars.push_back(v);
    double num[4] = {0, 0, 0, 0}, den[4] = {0, 0, 0, 0};
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
            num[k] += tf;
            den[k] += units * chunks;
        }
        out.release();
        fc_plan_free(p);
    }
    if (den[2] > 0.0) c->opt.small_cost = (int64_t)std::max(1.0, num[2] / den[2]);
    if (den[3] > 0.0) c->opt.small3_cost = (int64_t)std::max(1.0, num[3] / den[3]);
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
    double best_t = 1e30, no_bitmap_t = 1e30;
    Options best = base, no_bitmap = base;
    for (double sc : scales) {
        c->opt = base;
        c->opt.bitmap_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)std::max(1.0, base.bitmap_cost * sc);
        c->opt.bitmap_chunk_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)(base.bitmap_chunk_cost * sc);
        c->opt.small_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)std::max(1.0, base.small_cost * sc);
        c->opt.small3_cost = sc < 0 ? ((int64_t)1 << 50) : (int64_t)std::max(1.0, base.small3_cost * sc);
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
        if (sc < 0) {
            no_bitmap_t = t;
            no_bitmap = c->opt;
        }
    }
    // A synchronous fc_count_batch of such a batch is planned on the device
    // only when no query takes the bitmap strategy, which saves the host
    // planner's ~30 ns per query; a setting with bitmap queries must beat the
    // one without by more than that to be kept.
    const bool device_plannable = base.device_plan && base.strategy == FC_STRAT_AUTO && base.shape_auto &&
                                  base.window_wide && c->m < (1 << 19) && nq >= kDevicePlanMinQueries;
    if (device_plannable && no_bitmap_t - best_t < 3e-5 * (double)nq) best = no_bitmap;
    c->opt = best;
    return FC_OK;
}

