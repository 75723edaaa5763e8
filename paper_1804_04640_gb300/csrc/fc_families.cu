// fc_families.cu -- the parent-set lattice's query stream (Sec. 4.2): every
// variable set counted once, then one family score per (set, child).
#include "fc_host.h"

using namespace fc;

namespace fc {

cudaError_t enqueue_families(fc_plan *p, float *scores, cudaStream_t s)
{
    fc_ctx *c = p->ctx;
    cudaError_t e = enqueue_count(p->inner, (int32_t *)p->fam_tables.p, nullptr, s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(p->n_jobs, (int64_t)c->num_sms * 16);
    return launch_family_scores((const FamilyJob *)p->fam_jobs.p, p->n_jobs, (const int32_t *)p->fam_tables.p,
                                c->d_arity, c->d_soff, c->d_marg, c->m, p->fam_kind, p->ess, scores, grid, s);
}

}  // namespace fc

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

