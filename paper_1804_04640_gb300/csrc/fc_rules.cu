// fc_rules.cu -- bottom-up association-rule miner (Sec. 4.3) behind
// fc_mine_rules.  Host code: the level-wise candidate generation over the
// itemset lattice, the frequency filter and the rule extraction.  Each level's
// candidates are counted by one batched device launch of the
// specific-assignment kernel (bitmap AND + popcount, end of Sec. 3.3).
#include "../../include/fc.h"
#include "fc_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

namespace {

// One level of the lattice: n itemsets of k items, stored flat and in
// lexicographic order, with an open-addressing index from itemset to
// position.
struct Level {
    int k = 0;
    std::vector<int32_t> items;  // n * k
    std::vector<int64_t> supp;   // n
    std::vector<int32_t> slots;  // hash slots: -1 or a position
    uint64_t mask = 0;

    int64_t size() const { return (int64_t)supp.size(); }
    const int32_t *at(int64_t i) const { return items.data() + i * k; }

    static uint64_t hash(const int32_t *x, int k)
    {
        uint64_t h = 0x9e3779b97f4a7c15ull ^ (uint64_t)k;
        for (int t = 0; t < k; ++t) {
            h ^= (uint64_t)(uint32_t)x[t];
            h *= 0xff51afd7ed558ccdull;
            h ^= h >> 32;
        }
        return h;
    }

    void build_index()
    {
        size_t cap = 16;
        while (cap < 2 * supp.size() + 1) cap <<= 1;
        slots.assign(cap, -1);
        mask = cap - 1;
        for (int64_t i = 0; i < size(); ++i) {
            uint64_t h = hash(at(i), k) & mask;
            while (slots[h] >= 0) h = (h + 1) & mask;
            slots[h] = (int32_t)i;
        }
    }

    // Position of the itemset x (k items) or -1.
    int64_t find(const int32_t *x) const
    {
        if (slots.empty()) return -1;
        uint64_t h = hash(x, k) & mask;
        while (slots[h] >= 0) {
            const int32_t i = slots[h];
            if (std::memcmp(at(i), x, sizeof(int32_t) * k) == 0) return i;
            h = (h + 1) & mask;
        }
        return -1;
    }
};

int popcount32(uint32_t x)
{
    int c = 0;
    for (; x; x &= x - 1) ++c;
    return c;
}

}  // namespace

struct fc_rules {
    std::vector<int32_t> set_off{0};
    std::vector<int32_t> items;
    std::vector<int64_t> support;
    std::vector<int64_t> rule_set;
    std::vector<uint32_t> rule_mask;
    std::vector<float> rule_conf;
    int64_t candidates = 0, candidate_items = 0;
    int64_t levels = 0;
    fc::ItemsetCountStats io;
};

namespace {

// Level k candidates from the frequent (k-1)-itemsets (k >= 2): two sets that
// share their first k-2 items join into prefix + {x, y} (x < y, different
// groups), kept when every other (k-1)-subset is frequent too.  The order of
// `prev` makes the candidates come out lexicographically sorted.  Prefix
// groups [g0, g1) of prev, indexed by the run starts in `runs`.
void generate_runs(const Level &prev, const std::vector<int32_t> &group, int k, const std::vector<int64_t> &runs,
                   int64_t g0, int64_t g1, std::vector<int32_t> &cand)
{
    const int pk = k - 2;  // shared prefix length
    std::vector<int32_t> T(k), sub(k - 1);
    for (int64_t g = g0; g < g1; ++g) {
        const int64_t i = runs[g], j = runs[g + 1];
        for (int64_t a = i; a < j; ++a) {
            const int32_t x = prev.at(a)[pk];
            for (int64_t b = a + 1; b < j; ++b) {
                const int32_t y = prev.at(b)[pk];
                if (group[x] == group[y]) continue;
                std::memcpy(T.data(), prev.at(a), sizeof(int32_t) * pk);
                T[pk] = x;
                T[pk + 1] = y;
                bool ok = true;
                for (int drop = 0; drop < pk && ok; ++drop) {
                    int w = 0;
                    for (int t = 0; t < k; ++t)
                        if (t != drop) sub[w++] = T[t];
                    ok = prev.find(sub.data()) >= 0;
                }
                if (ok) cand.insert(cand.end(), T.begin(), T.end());
            }
        }
    }
}

// All level-k candidates, the prefix groups split over the context's host
// threads by their pair counts; per-thread lists are joined in group order,
// so the result does not depend on the split.
void generate(fc_ctx *c, const Level &prev, const std::vector<int32_t> &group, int k, std::vector<int32_t> &cand)
{
    cand.clear();
    const int64_t n = prev.size();
    const int pk = k - 2;
    std::vector<int64_t> runs;  // starts of the prefix groups, then n
    double work = 0.0;
    for (int64_t i = 0; i < n;) {
        int64_t j = i + 1;
        while (j < n && std::memcmp(prev.at(i), prev.at(j), sizeof(int32_t) * pk) == 0) ++j;
        runs.push_back(i);
        work += 0.5 * (double)(j - i) * (double)(j - i - 1);
        i = j;
    }
    runs.push_back(n);
    const int64_t ngroups = (int64_t)runs.size() - 1;
    const int nt = work > 4000.0 ? (int)std::min<int64_t>(fc::host_threads(c), ngroups) : 1;
    if (nt <= 1) {
        generate_runs(prev, group, k, runs, 0, ngroups, cand);
        return;
    }
    // split points of roughly equal pair counts
    std::vector<int64_t> cut(nt + 1, ngroups);
    cut[0] = 0;
    double acc = 0.0;
    int t = 1;
    for (int64_t g = 0; g < ngroups && t < nt; ++g) {
        const double sz = (double)(runs[g + 1] - runs[g]);
        acc += 0.5 * sz * (sz - 1.0);
        if (acc >= work * t / nt) cut[t++] = g + 1;
    }
    std::vector<std::vector<int32_t>> part(nt);
    fc::run_host_threads(c, nt, [&](int i) { generate_runs(prev, group, k, runs, cut[i], cut[i + 1], part[i]); });
    size_t total = 0;
    for (auto &v : part) total += v.size();
    cand.reserve(total);
    for (auto &v : part) cand.insert(cand.end(), v.begin(), v.end());
}

// Device counts of `nc` candidates of k items, in batches that keep the
// offsets within int32.
int count_level(fc_ctx *c, const std::vector<int32_t> &cand, int k, int64_t nc, std::vector<int32_t> &counts,
                fc::ItemsetCountStats *st)
{
    counts.resize(nc);
    const int64_t batch = std::max<int64_t>(1, std::min<int64_t>(nc, (int64_t)(INT32_MAX / std::max(k, 1)) / 2));
    std::vector<int32_t> off;
    for (int64_t b0 = 0; b0 < nc; b0 += batch) {
        const int32_t nb = (int32_t)std::min(batch, nc - b0);
        off.resize(nb + 1);
        for (int32_t q = 0; q <= nb; ++q) off[q] = q * k;
        const int rc = fc::count_itemsets(c, nb, off.data(), cand.data() + b0 * k, counts.data() + b0, st);
        if (rc != FC_OK) return rc;
    }
    return FC_OK;
}

}  // namespace

extern "C" int fc_mine_rules(fc_ctx *ctx, double min_support, double min_confidence, int32_t max_size,
                             int32_t all_splits, fc_rules **out)
{
    using fc::set_error;
    if (!ctx || !out) return set_error(FC_ERR_ARG, "fc_mine_rules: null argument");
    *out = nullptr;
    if (!(min_support >= 0.0 && min_support <= 1.0))
        return set_error(FC_ERR_ARG, "min_support must be in [0, 1]");
    if (!(min_confidence >= 0.0) || std::isinf(min_confidence))
        return set_error(FC_ERR_ARG, "min_confidence must be finite and >= 0");
    if (max_size < 1 || max_size > fc::kMaxK || (all_splits && max_size > 16))
        return set_error(FC_ERR_ARG, "max_size %d out of range", max_size);
    fc_rules *R = new (std::nothrow) fc_rules();
    if (!R) return set_error(FC_ERR_OOM, "host allocation failed");

    int32_t n_items = 0;
    int64_t m = 0;
    fc::itemset_universe(ctx, &n_items, &m);
    std::vector<int32_t> group(n_items);
    std::vector<int64_t> single(n_items);
    fc::item_groups(ctx, group.data(), single.data());
    const double thr = min_support * (double)m;

    // level 1: the item bitmaps' popcounts, counted when the context loaded
    std::vector<Level> levels(1);
    levels[0].k = 1;
    for (int32_t i = 0; i < n_items; ++i)
        if ((double)single[i] > thr) {
            levels[0].items.push_back(i);
            levels[0].supp.push_back(single[i]);
        }
    levels[0].build_index();

    std::vector<int32_t> cand, counts;
    for (int k = 2; k <= max_size && levels.back().size() > 0; ++k) {
        generate(ctx, levels.back(), group, k, cand);
        const int64_t nc = (int64_t)cand.size() / k;
        if (nc == 0) break;
        if (nc > INT32_MAX) {
            fc_rules_free(R);
            return set_error(FC_ERR_SIZE, "level %d has %lld candidates", k, (long long)nc);
        }
        const int rc = count_level(ctx, cand, k, nc, counts, &R->io);
        if (rc != FC_OK) {
            fc_rules_free(R);
            return rc;
        }
        R->candidates += nc;
        R->candidate_items += nc * k;
        R->levels += 1;
        Level L;
        L.k = k;
        for (int64_t q = 0; q < nc; ++q)
            if ((double)counts[q] > thr) {
                L.items.insert(L.items.end(), cand.begin() + q * k, cand.begin() + (q + 1) * k);
                L.supp.push_back(counts[q]);
            }
        L.build_index();
        levels.push_back(std::move(L));
    }

    // itemsets, then rules A => S \ A in itemset order and mask order
    std::vector<uint32_t> masks;
    int64_t idx = 0;
    int64_t total_items = 0;
    for (const Level &L : levels) total_items += L.size() * L.k;
    if (total_items > INT32_MAX) {
        fc_rules_free(R);
        return set_error(FC_ERR_SIZE, "%lld items over the frequent itemsets", (long long)total_items);
    }
    for (const Level &L : levels) {
        for (int64_t s = 0; s < L.size(); ++s) {
            R->items.insert(R->items.end(), L.at(s), L.at(s) + L.k);
            R->set_off.push_back((int32_t)R->items.size());
            R->support.push_back(L.supp[s]);
        }
    }
    struct RuleOut {
        std::vector<int64_t> set;
        std::vector<uint32_t> mask;
        std::vector<float> conf;
        bool missing = false;
    };
    for (const Level &L : levels) {
        const int k = L.k;
        if (k < 2) {
            idx += L.size();
            continue;
        }
        // antecedent masks in increasing order: every non-empty proper subset,
        // or the k masks that leave out one item (item k-1 first)
        const uint32_t full = (k == 32) ? 0xffffffffu : ((1u << k) - 1u);
        masks.clear();
        if (all_splits)
            for (uint32_t mk = 1; mk < full; ++mk) masks.push_back(mk);
        else
            for (int t = k - 1; t >= 0; --t) masks.push_back(full ^ (1u << t));
        // itemsets of the level in contiguous ranges on the host threads,
        // each range's rules kept in order and joined in range order
        const int64_t ns = L.size();
        const int nt = ns * (int64_t)masks.size() > 4000 ? (int)std::min<int64_t>(fc::host_threads(ctx), ns) : 1;
        std::vector<RuleOut> outs(nt);
        const int64_t base = idx;
        auto rules_of = [&](int t) {
            RuleOut &o = outs[t];
            std::vector<int32_t> A;
            const int64_t s0 = ns * t / nt, s1 = ns * (t + 1) / nt;
            for (int64_t s = s0; s < s1; ++s) {
                const int32_t *S = L.at(s);
                for (const uint32_t mk : masks) {
                    const int na = popcount32(mk);
                    A.clear();
                    for (int u = 0; u < k; ++u)
                        if (mk >> u & 1u) A.push_back(S[u]);
                    const Level &LA = levels[na - 1];
                    const int64_t ia = LA.find(A.data());
                    if (ia < 0) {  // cannot happen: every subset of a frequent set is frequent
                        o.missing = true;
                        return;
                    }
                    const int64_t sa = LA.supp[ia];
                    if ((double)L.supp[s] > min_confidence * (double)sa) {
                        o.set.push_back(base + s);
                        o.mask.push_back(mk);
                        o.conf.push_back((float)((double)L.supp[s] / (double)sa));
                    }
                }
            }
        };
        fc::run_host_threads(ctx, nt, rules_of);
        for (RuleOut &o : outs) {
            if (o.missing) {
                fc_rules_free(R);
                return set_error(FC_ERR_STATE, "internal: missing subset of a frequent itemset");
            }
            R->rule_set.insert(R->rule_set.end(), o.set.begin(), o.set.end());
            R->rule_mask.insert(R->rule_mask.end(), o.mask.begin(), o.mask.end());
            R->rule_conf.insert(R->rule_conf.end(), o.conf.begin(), o.conf.end());
        }
        idx += ns;
    }
    *out = R;
    return FC_OK;
}

extern "C" int64_t fc_rules_size(const fc_rules *r, int32_t key)
{
    if (!r) return -1;
    switch (key) {
    case 0: return (int64_t)r->support.size();
    case 1: return (int64_t)r->items.size();
    case 2: return (int64_t)r->rule_set.size();
    case 3: return r->candidates;
    case 4: return r->levels;
    case 5: return r->io.h2d_bytes;
    case 6: return r->io.d2h_bytes;
    case 7: return (int64_t)std::llround(r->io.device_ms * 1e6);
    case 8: return r->candidate_items;
    default: return -1;
    }
}

extern "C" int fc_rules_itemsets(const fc_rules *r, int32_t *set_off, int32_t *items, int64_t *support)
{
    if (!r) return fc::set_error(FC_ERR_ARG, "fc_rules_itemsets: null handle");
    if (set_off) std::copy(r->set_off.begin(), r->set_off.end(), set_off);
    if (items) std::copy(r->items.begin(), r->items.end(), items);
    if (support) std::copy(r->support.begin(), r->support.end(), support);
    return FC_OK;
}

extern "C" int fc_rules_list(const fc_rules *r, int64_t *itemset, uint32_t *antecedent, float *confidence)
{
    if (!r) return fc::set_error(FC_ERR_ARG, "fc_rules_list: null handle");
    if (itemset) std::copy(r->rule_set.begin(), r->rule_set.end(), itemset);
    if (antecedent) std::copy(r->rule_mask.begin(), r->rule_mask.end(), antecedent);
    if (confidence) std::copy(r->rule_conf.begin(), r->rule_conf.end(), confidence);
    return FC_OK;
}

extern "C" void fc_rules_free(fc_rules *r) { delete r; }
