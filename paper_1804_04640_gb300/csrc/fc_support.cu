// fc_support.cu -- support and confidence of association rules (Sec. 4.3).
//
// For an itemset S of k items the Bitmap strategy's specific-assignment query
// (end of Sec. 3.3) is the AND of the k item bitmaps followed by a bit count.
// Rules with a single-item consequent, (S without x) => x, also need the k
// leave-one-out supports; with prefix ANDs p_t = a_0 & ... & a_{t-1} and
// suffix ANDs s_t = a_{t+1} & ... & a_{k-1}, the leave-one-out set of item t
// is p_t & s_t, so one pass over the words yields all k + 1 counts.
//
// A warp owns one itemset at a time; its lanes read 64 consecutive 64-bit
// words of every item row (coalesced 16-byte loads per lane) and keep the
// k + 1 counts in registers.  Work items are (word range, group of itemsets),
// issued range-major, so all CTAs sweep the same slice of the item bitmaps at
// the same time and the slice stays in L2 while every itemset passes over it.
#include "fc_internal.h"

namespace fc {
namespace {

constexpr unsigned kFullMask = 0xffffffffu;

// One itemset of K >= 2 items over words [w0, w1) (w0 even): each lane takes
// two consecutive words per step (16-byte loads).  Item rows are zero past m
// and padded with zero words, so reading one word past w1 at the array's end
// adds nothing.  Prefix ANDs p_t = a_0 & .. & a_{t-1} and suffix ANDs
// s_t = a_{t+1} & .. & a_{K-1} give every leave-one-out set as p_t & s_t
// (3K - 5 ANDs per word) and the full set as p_K.
template <int K>
__device__ __forceinline__ void support_set(const SupportParams &P, const int32_t *items,
                                            int64_t w0, int64_t w1, int lane, int32_t *supp,
                                            int32_t *sub, bool atomic)
{
    static_assert(K >= 2, "two or more items");
    const uint64_t *row[K];
#pragma unroll
    for (int t = 0; t < K; ++t) row[t] = P.bits + (int64_t)items[t] * P.wstride;
    unsigned full = 0u;
    unsigned loo[K];
#pragma unroll
    for (int t = 0; t < K; ++t) loo[t] = 0u;
    for (int64_t w = w0 + 2 * lane; w < w1; w += 64) {
        ulonglong2 a[K];
#pragma unroll
        for (int t = 0; t < K; ++t) a[t] = __ldg(reinterpret_cast<const ulonglong2 *>(row[t] + w));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint64_t x[K];
#pragma unroll
            for (int t = 0; t < K; ++t) x[t] = h ? a[t].y : a[t].x;
            uint64_t pre[K + 1];  // pre[t] = AND of x[0..t-1], pre[0] unused
            pre[1] = x[0];
#pragma unroll
            for (int t = 2; t <= K; ++t) pre[t] = pre[t - 1] & x[t - 1];
            full += (unsigned)__popcll(pre[K]);
            // two items: each leave-one-out set is one item, whose count is
            // its marginal (filled in by the finishing kernel)
            if constexpr (K > 2) {
                uint64_t suf = x[K - 1];  // AND of x[t+1..K-1] for t = K-2
                loo[K - 1] += (unsigned)__popcll(pre[K - 1]);
#pragma unroll
                for (int t = K - 2; t >= 1; --t) {
                    loo[t] += (unsigned)__popcll(pre[t] & suf);
                    suf &= x[t];
                }
                loo[0] += (unsigned)__popcll(suf);
            }
        }
    }
    full = __reduce_add_sync(kFullMask, full);
    if constexpr (K > 2) {
#pragma unroll
        for (int t = 0; t < K; ++t) loo[t] = __reduce_add_sync(kFullMask, loo[t]);
    }
    if (lane == 0) {
        if (atomic) {
            if (full) atomicAdd(supp, (int)full);
            if constexpr (K > 2) {
#pragma unroll
                for (int t = 0; t < K; ++t)
                    if (loo[t]) atomicAdd(sub + t, (int)loo[t]);
            }
        } else {
            *supp = (int)full;
            if constexpr (K > 2) {
#pragma unroll
                for (int t = 0; t < K; ++t) sub[t] = (int)loo[t];
            }
        }
    }
}

// supp(S) alone: the AND of K rows and a popcount (specific-assignment
// counts, where no rule confidences are wanted).  Rows are zero past m.
template <int K>
__device__ __forceinline__ void full_set(const SupportParams &P, const int32_t *items, int64_t w0, int64_t w1,
                                         int lane, int32_t *supp, bool atomic)
{
    const uint64_t *row[K];
#pragma unroll
    for (int t = 0; t < K; ++t) row[t] = P.bits + (int64_t)items[t] * P.wstride;
    unsigned full = 0u;
#pragma unroll 1
    for (int64_t w = w0 + 2 * lane; w < w1; w += 64) {
        ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2 *>(row[0] + w));
#pragma unroll
        for (int t = 1; t < K; ++t) {
            const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(row[t] + w));
            x.x &= a.x;
            x.y &= a.y;
        }
        full += (unsigned)(__popcll(x.x) + __popcll(x.y));
    }
    full = __reduce_add_sync(kFullMask, full);
    if (lane == 0) {
        if (atomic) {
            if (full) atomicAdd(supp, (int)full);
        } else {
            *supp = (int)full;
        }
    }
}

__device__ void full_set_any(const SupportParams &P, const int32_t *items, int k, int64_t w0, int64_t w1,
                             int lane, int32_t *supp, bool atomic)
{
    unsigned full = 0u;
    for (int64_t w = w0 + lane; w < w1; w += 32) {
        uint64_t x = __ldg(P.bits + (int64_t)items[0] * P.wstride + w);
        for (int t = 1; t < k; ++t) x &= __ldg(P.bits + (int64_t)items[t] * P.wstride + w);
        full += (unsigned)__popcll(x);
    }
    full = __reduce_add_sync(kFullMask, full);
    if (lane == 0) {
        if (atomic) {
            if (full) atomicAdd(supp, (int)full);
        } else {
            *supp = (int)full;
        }
    }
}

// Itemsets outside the unrolled sizes (0, 1 or more than 6 items): the k + 1
// ANDs recomputed per word, the last word masked to the m transactions.
__device__ void support_set_any(const SupportParams &P, const int32_t *items, int k, int64_t w0,
                                int64_t w1, int lane, int32_t *supp, int32_t *sub, bool atomic)
{
    const int64_t last = P.words - 1;
    const int rem = (int)(P.m_tail & 63);
    const uint64_t tail = rem ? ((1ull << rem) - 1ull) : ~0ull;
    for (int t = -1; t < k; ++t) {
        unsigned cnt = 0u;
        for (int64_t w = w0 + lane; w < w1; w += 32) {
            uint64_t x = w == last ? tail : ~0ull;
            for (int u = 0; u < k; ++u)
                if (u != t) x &= __ldg(P.bits + (int64_t)items[u] * P.wstride + w);
            cnt += (unsigned)__popcll(x);
        }
        cnt = __reduce_add_sync(kFullMask, cnt);
        if (lane == 0) {
            int32_t *dst = t < 0 ? supp : sub + t;
            if (atomic) {
                if (cnt) atomicAdd(dst, (int)cnt);
            } else {
                *dst = (int)cnt;
            }
        }
    }
}

__global__ void __launch_bounds__(1024) support_kernel(const SupportParams P)
{
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t ngroups = ((int64_t)P.nq + P.sets_per_item - 1) / P.sets_per_item;
    const int64_t n_work = ngroups * P.nparts;
    const bool atomic = P.nparts > 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.next_item, 1);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= n_work) break;
        const int64_t part = it / ngroups, group = it % ngroups;
        const int64_t w0 = part * P.words_per_part;
        const int64_t w1 = min(P.words, w0 + P.words_per_part);
        const int64_t g0 = group * P.sets_per_item;
        const int64_t g1 = min((int64_t)P.nq, g0 + P.sets_per_item);
        for (int64_t i = g0 + warp; i < g1; i += nwarps) {
            const int32_t q = P.order[i];
            const int32_t a = P.set_off[q], k = P.set_off[q + 1] - a;
            const int32_t *items = P.items + a;
            int32_t *supp = P.support + q;
            int32_t *sub = P.sub_support + a;
            switch (k) {
            case 2: support_set<2>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 3: support_set<3>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 4: support_set<4>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 5: support_set<5>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 6: support_set<6>(P, items, w0, w1, lane, supp, sub, atomic); break;
            default: support_set_any(P, items, k, w0, w1, lane, supp, sub, atomic); break;
            }
        }
    }
}

// Counts of specific assignments (end of Sec. 3.3): the support-kernel loop
// with supp(S) alone per set of bitmap rows.
__global__ void __launch_bounds__(512, 2) assign_kernel(const SupportParams P)
{
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t ngroups = ((int64_t)P.nq + P.sets_per_item - 1) / P.sets_per_item;
    const int64_t n_work = ngroups * P.nparts;
    const bool atomic = P.nparts > 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.next_item, 1);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= n_work) break;
        const int64_t part = it / ngroups, group = it % ngroups;
        const int64_t w0 = part * P.words_per_part;
        const int64_t w1 = min(P.words, w0 + P.words_per_part);
        const int64_t g0 = group * P.sets_per_item;
        const int64_t g1 = min((int64_t)P.nq, g0 + P.sets_per_item);
        for (int64_t i = g0 + warp; i < g1; i += nwarps) {
            const int32_t q = P.order[i];
            const int32_t a = P.set_off[q], k = P.set_off[q + 1] - a;
            const int32_t *items = P.items + a;
            int32_t *supp = P.support + q;
            switch (k) {
            case 0:  // the empty assignment matches every instance
                if (lane == 0 && (!atomic || part == 0)) {
                    if (atomic)
                        atomicAdd(supp, (int)P.m_tail);
                    else
                        *supp = (int)P.m_tail;
                }
                break;
            case 1: full_set<1>(P, items, w0, w1, lane, supp, atomic); break;
            case 2: full_set<2>(P, items, w0, w1, lane, supp, atomic); break;
            case 3: full_set<3>(P, items, w0, w1, lane, supp, atomic); break;
            case 4: full_set<4>(P, items, w0, w1, lane, supp, atomic); break;
            default: full_set_any(P, items, k, w0, w1, lane, supp, atomic); break;
            }
        }
    }
}

// ---- every split of an itemset into antecedent A and consequent S \ A
//
// supp(A) is needed for all 2^k - 2 non-empty proper subsets A of S.  Per
// word the subsets are walked depth-first (include or skip each item in
// turn), so every subset costs one AND of its parent's word with one item's
// word and one popcount, and the walk keeps only one partial AND per level.
// With k fixed at compile time the walk unrolls completely and the 2^k - 1
// counters (subset masks 1 .. 2^k - 1) sit in registers.

// A one-item subset's support is that item's marginal count, taken when the
// bitmaps were loaded (Sec. 3.3 precomputes single-variable partitions), so
// the walk counts only subsets of two or more items; the finishing kernel
// fills in the one-item entries.

template <int K, int T, int MASK>
struct SubsetWalk {
    // subsets MASK | {some items >= T}; acc is the AND of MASK's words
    static __device__ __forceinline__ void run(const uint64_t (&x)[K], uint64_t acc, unsigned (&cnt)[1 << K])
    {
        if constexpr (T < K) {
            const uint64_t a = MASK == 0 ? x[T] : (acc & x[T]);
            if constexpr (MASK != 0) cnt[MASK | (1 << T)] += (unsigned)__popcll(a);
            SubsetWalk<K, T + 1, MASK | (1 << T)>::run(x, a, cnt);
            SubsetWalk<K, T + 1, MASK>::run(x, acc, cnt);
        }
    }
};

// The walk over both words of a step at once, counting each subset of two
// or more items with a carry-save adder: a per-subset running word `ones`
// takes the step's two AND words, keeps their sum bit and passes the carry
// (weight 2) to the popcount, so a subset costs one 64-bit popcount per two
// words (plus two 3-input logic ops per 32 bits) instead of two.  Pairs of
// items keep plain popcounts (a running word for each would cost more
// registers than it saves).  The counts of subsets 2j and 2j + 1 share one
// register as 16-bit halves: a lane adds at most 128 per step to a pair's
// count and 64 to a larger subset's carries, and the planner gives a work
// item at most 511 steps (511 * 128 < 2^16).  A larger subset's count is
// 2 * carries + popcount(ones) at the end.

template <int K, int T, int MASK>
struct SubsetWalkCsa {
    static __device__ __forceinline__ void run(const uint64_t (&x1)[K], const uint64_t (&x2)[K], uint64_t acc1,
                                               uint64_t acc2, uint64_t (&ones)[1 << K],
                                               unsigned (&cnt)[(1 << K) / 2])
    {
        if constexpr (T < K) {
            const uint64_t a1 = MASK == 0 ? x1[T] : (acc1 & x1[T]);
            const uint64_t a2 = MASK == 0 ? x2[T] : (acc2 & x2[T]);
            if constexpr (MASK != 0 && (MASK & (MASK - 1)) == 0) {
                // two items: plain popcounts (a running word for each of the
                // K(K-1)/2 pairs would cost more registers than it saves)
                constexpr int S = MASK | (1 << T);
                const unsigned c = (unsigned)__popcll(a1) + (unsigned)__popcll(a2);
                cnt[S >> 1] += (S & 1) ? (c << 16) : c;
            } else if constexpr (MASK != 0) {
                constexpr int S = MASK | (1 << T);
                const uint64_t o = ones[S];
                ones[S] = o ^ a1 ^ a2;
                const unsigned c = (unsigned)__popcll((o & a1) | (o & a2) | (a1 & a2));
                cnt[S >> 1] += (S & 1) ? (c << 16) : c;
            }
            SubsetWalkCsa<K, T + 1, MASK | (1 << T)>::run(x1, x2, a1, a2, ones, cnt);
            SubsetWalkCsa<K, T + 1, MASK>::run(x1, x2, acc1, acc2, ones, cnt);
        }
    }
};

template <int K>
__device__ __forceinline__ void splits_set_csa(const SupportParams &P, const int32_t *items, int64_t w0, int64_t w1,
                                               int lane, int32_t *supp, int32_t *sub, bool atomic)
{
    const uint64_t *row[K];
#pragma unroll
    for (int t = 0; t < K; ++t) row[t] = P.bits + (int64_t)items[t] * P.wstride;
    unsigned cnt[(1 << K) / 2];
    uint64_t ones[1 << K];
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) ones[i] = 0ull;
#pragma unroll
    for (int i = 0; i < (1 << K) / 2; ++i) cnt[i] = 0u;
#pragma unroll 1
    for (int64_t w = w0 + 2 * lane; w < w1; w += 64) {
        uint64_t x1[K], x2[K];
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const ulonglong2 a = __ldg(reinterpret_cast<const ulonglong2 *>(row[t] + w));
            x1[t] = a.x;
            x2[t] = a.y;
        }
        SubsetWalkCsa<K, 0, 0>::run(x1, x2, ~0ull, ~0ull, ones, cnt);
    }
    constexpr int kFull = (1 << K) - 1;
#pragma unroll
    for (int i = 1; i <= kFull; ++i) {
        if ((i & (i - 1)) == 0) continue;  // one item: filled from its marginal count
        const unsigned c = (cnt[i >> 1] >> ((i & 1) * 16)) & 0xFFFFu;
        // pairs hold plain counts; larger subsets carries and a running word
        const bool pair = ((i & (i - 1)) & ((i & (i - 1)) - 1)) == 0;
        const unsigned v = __reduce_add_sync(kFullMask, pair ? c : 2u * c + (unsigned)__popcll(ones[i]));
        if (lane == 0) {
            int32_t *dst = i == kFull ? supp : sub + (i - 1);
            if (atomic) {
                if (v) atomicAdd(dst, (int)v);
            } else {
                *dst = (int)v;
            }
        }
    }
}

template <int K>
__device__ __forceinline__ void splits_set(const SupportParams &P, const int32_t *items, int64_t w0, int64_t w1,
                                           int lane, int32_t *supp, int32_t *sub, bool atomic)
{
    const uint64_t *row[K];
#pragma unroll
    for (int t = 0; t < K; ++t) row[t] = P.bits + (int64_t)items[t] * P.wstride;
    unsigned cnt[1 << K];
#pragma unroll
    for (int i = 0; i < (1 << K); ++i) cnt[i] = 0u;
#pragma unroll 1
    for (int64_t w = w0 + 2 * lane; w < w1; w += 64) {
        ulonglong2 a[K];
#pragma unroll
        for (int t = 0; t < K; ++t) a[t] = __ldg(reinterpret_cast<const ulonglong2 *>(row[t] + w));
        uint64_t x[K];
#pragma unroll
        for (int t = 0; t < K; ++t) x[t] = a[t].x;
        SubsetWalk<K, 0, 0>::run(x, ~0ull, cnt);
#pragma unroll
        for (int t = 0; t < K; ++t) x[t] = a[t].y;
        SubsetWalk<K, 0, 0>::run(x, ~0ull, cnt);
    }
    constexpr int kFull = (1 << K) - 1;
#pragma unroll
    for (int i = 1; i <= kFull; ++i) {
        if ((i & (i - 1)) == 0) continue;  // one item: filled from its marginal count
        const unsigned v = __reduce_add_sync(kFullMask, cnt[i]);
        if (lane == 0) {
            int32_t *dst = i == kFull ? supp : sub + (i - 1);
            if (atomic) {
                if (v) atomicAdd(dst, (int)v);
            } else {
                *dst = (int)v;
            }
        }
    }
}

// Any size up to kMaxSplitK (and 0 or 1 items): one pass over the words per
// subset, the last word masked to the m transactions.
__device__ void splits_set_any(const SupportParams &P, const int32_t *items, int k, int64_t w0, int64_t w1,
                               int lane, int32_t *supp, int32_t *sub, bool atomic)
{
    const int64_t last = P.words - 1;
    const int rem = (int)(P.m_tail & 63);
    const uint64_t tail = rem ? ((1ull << rem) - 1ull) : ~0ull;
    const int full = (1 << k) - 1;
    for (int mask = (k == 0 ? 0 : 1); mask <= full; ++mask) {
        unsigned c = 0u;
        for (int64_t w = w0 + lane; w < w1; w += 32) {
            uint64_t x = w == last ? tail : ~0ull;
            for (int t = 0; t < k; ++t)
                if (mask >> t & 1) x &= __ldg(P.bits + (int64_t)items[t] * P.wstride + w);
            c += (unsigned)__popcll(x);
        }
        c = __reduce_add_sync(kFullMask, c);
        if (lane == 0) {
            int32_t *dst = mask == full ? supp : sub + (mask - 1);
            if (atomic) {
                if (c) atomicAdd(dst, (int)c);
            } else {
                *dst = (int)c;
            }
        }
    }
}

// 256 threads x 2 CTAs per SM (the counters of 5-item sets spill a little
// at 128 registers) or 128 threads x 3 CTAs (168 registers, no spills).
template <int kThreads, int kBlocks>
__global__ void __launch_bounds__(kThreads, kBlocks) splits_kernel(const SupportParams P)
{
    __shared__ int s_item;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t ngroups = ((int64_t)P.nq + P.sets_per_item - 1) / P.sets_per_item;
    const int64_t n_work = ngroups * P.nparts;
    const bool atomic = P.nparts > 1;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.next_item, 1);
        __syncthreads();
        const int64_t it = s_item;
        __syncthreads();
        if (it >= n_work) break;
        const int64_t part = it / ngroups, group = it % ngroups;
        const int64_t w0 = part * P.words_per_part;
        const int64_t w1 = min(P.words, w0 + P.words_per_part);
        const int64_t g0 = group * P.sets_per_item;
        const int64_t g1 = min((int64_t)P.nq, g0 + P.sets_per_item);
        for (int64_t i = g0 + warp; i < g1; i += nwarps) {
            const int32_t q = P.order[i];
            const int32_t a = P.set_off[q], k = P.set_off[q + 1] - a;
            const int32_t *items = P.items + a;
            int32_t *supp = P.support + q;
            int32_t *sub = P.sub_support + P.split_off[q];
            switch (k) {
            case 2: splits_set_csa<2>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 3: splits_set_csa<3>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 4: splits_set_csa<4>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 5: splits_set_csa<5>(P, items, w0, w1, lane, supp, sub, atomic); break;
            case 6: splits_set<6>(P, items, w0, w1, lane, supp, sub, atomic); break;
            default: splits_set_any(P, items, k, w0, w1, lane, supp, sub, atomic); break;
            }
        }
    }
}

// Finishing pass of the all-splits mode: the one-item antecedents of the
// unrolled sizes (2..6 items) take their item's marginal count, then
// conf(A => S \ A) = supp(S) / supp(A) for every split, 0 when supp(A) = 0
// (confidences only when asked for).
__global__ void splits_confidence_kernel(const SupportParams P)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P.nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = P.split_off[q], b = P.split_off[q + 1];
        const int32_t i0 = P.set_off[q], k = P.set_off[q + 1] - i0;
        if (k >= 2 && k <= 6) {
            for (int t = 0; t < k; ++t)
                P.sub_support[a + (1 << t) - 1] = (int32_t)P.marg[P.items[i0 + t]];
        }
        if (!P.confidence) continue;
        const float s = (float)P.support[q];
        for (int64_t t = a; t < b; ++t) {
            const int32_t d = P.sub_support[t];
            P.confidence[t] = d > 0 ? __fdiv_rn(s, (float)d) : 0.0f;
        }
    }
}

// Finishing pass of the leave-one-out mode: an itemset of two items has
// one-item leave-one-out sets, whose counts are the items' marginals; then
// conf((S without item t) => item t) = supp(S) / supp(S without item t), 0
// when the denominator is 0 (then supp(S) is 0 as well), when asked for.
__global__ void confidence_kernel(const SupportParams P)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < P.nq;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = P.set_off[q], b = P.set_off[q + 1];
        if (b - a == 2) {
            P.sub_support[a] = (int32_t)P.marg[P.items[a + 1]];
            P.sub_support[a + 1] = (int32_t)P.marg[P.items[a]];
        }
        if (!P.confidence) continue;
        const float s = (float)P.support[q];
        for (int32_t t = a; t < b; ++t) {
            const int32_t d = P.sub_support[t];
            P.confidence[t] = d > 0 ? __fdiv_rn(s, (float)d) : 0.0f;
        }
    }
}

}  // namespace

const void *support_kernel_ptr(int mode, int threads)
{
    return mode == 1 ? (const void *)assign_kernel
         : mode == 2 ? (threads <= 128 ? (const void *)splits_kernel<128, 3> : (const void *)splits_kernel<256, 2>)
                     : (const void *)support_kernel;
}

cudaError_t launch_support(const SupportParams &p, int grid, int threads, size_t smem, cudaStream_t s)
{
    if (p.full_only)
        assign_kernel<<<grid, threads > 512 ? 512 : threads, smem, s>>>(p);
    else if (p.all_splits && threads <= 128)
        splits_kernel<128, 3><<<grid, threads, smem, s>>>(p);
    else if (p.all_splits)
        splits_kernel<256, 2><<<grid, threads > 256 ? 256 : threads, smem, s>>>(p);
    else
        support_kernel<<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_support_confidence(const SupportParams &p, cudaStream_t s)
{
    int64_t blocks = ((int64_t)p.nq + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    if (p.all_splits)
        splits_confidence_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
    else
        confidence_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace fc
