// fc_pairs_host.cu -- the all-pairs plan: the one-hot tensor-core product
// (fc_pairs.cu) split over row ranges in whole waves, then the pair tables
// and their mutual information.
#include "fc_host.h"

#include <cmath>

using namespace fc;

// ------------------------------------------------------------------- pairs

namespace fc {

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

}  // namespace fc

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

    // regions of C on or above the diagonal (256 x 256, rb-major) and the
    // columns each of their two accumulators needs
    const int nbr = R_pad / 256;
    std::vector<PairsRegion> regs;
    std::vector<double> cost;
    for (int rb = 0; rb < nbr; ++rb) {
        for (int ra = 0; ra <= rb; ++ra) {
            PairsRegion G{};
            G.ra = ra;
            G.rb = rb;
            G.real_b = std::min(256, c->R - rb * 256);
            const int nb = (int)round_up(G.real_b, 16);
            G.n0 = nb;
            if (ra == rb) {
                // rows 128..255 meet only the columns from 128 on
                G.coff1 = 128;
                G.n1 = ra * 256 + 128 < c->R ? nb - 128 : 0;
            } else {
                G.coff1 = 0;
                G.n1 = nb;
            }
            // shared-memory bytes per 128-row stage: each accumulator reads its
            // A half (16 KiB) and n columns of B (128 bytes each); the
            // producers write the B rows and, off the diagonal, both A halves
            double bytes = 0;
            for (const int n : {G.n0, G.n1})
                if (n > 0) bytes += 16384.0 + 128.0 * n;
            bytes += 128.0 * (G.real_b + (ra == rb ? 0 : 256));
            regs.push_back(G);
            cost.push_back(bytes);
        }
    }
    // row splits: one wave of one CTA per SM, each region's share of the SMs
    // in proportion to its traffic, and at least the splits that keep every
    // FP32 partial sum exact (pair_chunk_rows rows each)
    const int64_t chunk_words = std::max<int64_t>(2, c->opt.pair_chunk_rows / 64 / 2 * 2);
    const int64_t need = std::max<int64_t>(1, (c->words + chunk_words - 1) / chunk_words);
    const int64_t max_split = std::max<int64_t>(1, (c->words + 1) / 2);
    double total = 0;
    for (const double x : cost) total += x;
    int64_t cta = 0;
    for (size_t r = 0; r < regs.size(); ++r) {
        int64_t k = (int64_t)std::floor((double)c->num_sms * cost[r] / total);
        k = std::max<int64_t>(1, std::min(std::max(k, need), max_split));
        regs[r].cta0 = (int32_t)cta;
        regs[r].ksplit = (int32_t)k;
        cta += k;
    }
    if (cta > INT32_MAX / 2) {
        fc_plan_free(p);
        return fail(FC_ERR_SIZE, "all-pairs launch of %lld CTAs", (long long)cta);
    }
    const size_t reg_off = round_up(sizeof(int64_t) * (npairs + 1), 256);
    cudaError_t e = plan_buf(c, p->pairs_C, 4, sizeof(int32_t) * (size_t)R_pad * R_pad);
    if (e == cudaSuccess) e = plan_buf(c, p->pairs_meta, 5, reg_off + sizeof(PairsRegion) * regs.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->pairs_meta.p, off.data(), sizeof(int64_t) * (npairs + 1), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((uint8_t *)p->pairs_meta.p + reg_off, regs.data(), sizeof(PairsRegion) * regs.size(),
                            cudaMemcpyHostToDevice, c->stream);
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
    P.nregions = (int32_t)regs.size();
    P.regions = (const PairsRegion *)((uint8_t *)p->pairs_meta.p + reg_off);
    P.grid = (int32_t)cta;
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

