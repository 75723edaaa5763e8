// fc_count.cu -- the batched counting kernels.
//
// A batch of queries with shared context (Sec. 2: every count N_ijk of a
// variable set) runs as two persistent launches, each pulling work from an
// atomic counter so that no CTA or warp ever waits for another:
//
//   bitmap_kernel (Sec. 3.2, Alg. 1), warp-granular tasks (query, chunk
//     range).  A warp owns 4096 instances at a time (two 64-bit words per
//     lane) and walks the tree of state combinations depth first; each node
//     ANDs its parent's partial bitmap with the bitmap of the next variable's
//     state, and a subtree is skipped when that AND is empty in every lane
//     (zero-support pruning).  Variables are visited in ascending entropy
//     (Sec. 3.2).  The state bitmaps of levels 1..k-1, which the tree re-reads
//     once per parent configuration, are staged per lane in shared memory for
//     the chunk; leaves are popcounted, reduced over the warp and added to the
//     table in global memory (L2 atomics).
//
//   count_kernel, CTA-granular items (query, row range) for the strategies
//     that key every instance:
//     kHist    the partitions of Alg. 2-3 identified by their mixed-radix key
//              (the instance's cell index) and counted with shared-memory
//              atomics.  Keys are built two rows per 32-bit register (SWAR):
//              shared-memory tables have fewer than 2^16 cells, so a 16-bit
//              lane never overflows and one multiply-add updates two keys.
//     kGAtomic the same keys, counted straight into the table in global
//              memory (tables too large for shared memory).
//     kWindow  tables too large for shared memory cut into windows of
//              consecutive cells (partitions that share their leading key
//              digits); an item counts one window over its rows in shared
//              memory, skipping keys outside it, and stores the window.  A
//              table costs one pass over the rows per window but no global
//              atomics, and windows run in a launch of one 1024-thread CTA
//              per SM so that a window takes the SM's whole shared memory.
//
// When a query's counts feed a score, the reduction of Sec. 3.1 (Eq. 1,
// Fig. 2) runs in the same launch: from shared memory when one item holds the
// query's whole table, else by the last CTA or warp to finish one of the
// query's pieces (an atomic ticket).
#include "fc_internal.h"

#include <mutex>
#include "fc_score.cuh"

namespace fc {
namespace {

template <bool kGlobal>
__device__ __forceinline__ int32_t tab_ld(const int32_t *t, int64_t i)
{
    if constexpr (kGlobal)
        return __ldcg(t + i);
    else
        return t[i];
}

struct ScoreAcc {
    Kahan k;         // LL / MDL / MI terms; the N ln(N/N_j) part of BDeu (nats)
    Kahan r;         // BDeu: remainder terms R'' (see below)
    double d;        // BDeu: whole remainder terms of large prior counts (a >= 1)
    int32_t nk, nj;  // BDeu: cells and configurations whose R'' omits -lnGamma(a)
};

__device__ __forceinline__ ScoreAcc score_zero() { return ScoreAcc{{0.0f, 0.0f}, {0.0f, 0.0f}, 0.0, 0, 0}; }

// Per-query constants of BDeu (Sec. 3.1/4.2 reading: prior a_j = ess/q per
// parent configuration, a_jk = ess/(r q) per cell).
struct BdeuK {
    float ak, aj;      // a_jk, a_j rounded to float (per-term arithmetic)
    float g1k, g1j;    // lnGamma(1 + a) (small-count branch)
    double akd, ajd;   // exact a (FP64 branch)
    double lgk, lgj;   // lnGamma(a): subtracted once per FP32-branch term, by count
};

// One thread computes the constants; callers broadcast them.
__device__ BdeuK bdeu_consts(int64_t q, int32_t r, double ess)
{
    BdeuK b;
    b.ajd = ess / (double)q;
    b.akd = b.ajd / (double)r;
    b.ak = (float)b.akd;
    b.aj = (float)b.ajd;
    b.g1k = (float)lgamma(1.0 + b.akd);
    b.g1j = (float)lgamma(1.0 + b.ajd);
    b.lgk = lgamma(b.akd);
    b.lgj = lgamma(b.ajd);
    return b;
}

// c_n = lnGamma(n) - n ln n + n for n = 1..7 (index 0 unused).
__constant__ float kBdeuSmall[8] = {0.0f, 1.0f, 0.6137056388801094f, 0.39731031455561583f, 0.2465820247484931f,
                                    0.13086426817744368f, 0.03693492741371607f, -0.0421198313770903f};

// R''(a, n) = lnGamma(a + n) - n ln n + n for a count n >= 1 and a prior a < 1,
// in FP32 without cancellation:
//   n < 8:  lnGamma(1 + a) + c_n + sum_{i=1}^{n-1} log1p(a / i)
//           (Gamma(n + a) = Gamma(1 + a) prod_{i=1}^{n-1} (i + a));
//   n >= 8: n log1p(a/n) + (a - 1/2) ln(n + a) - a + ln(2 pi)/2
//           + 1/(12 z) - 1/(360 z^3), z = n + a (Stirling's series; the next
//           term is below 2.5e-8 for z >= 8).
__device__ __forceinline__ float bdeu_rem(float a, float g1, int64_t n)
{
    if (n < 8) {
        float t = g1 + kBdeuSmall[n];
        for (int i = 1; i < (int)n; ++i) t += log1pf(a / (float)i);
        return t;
    }
    const float nf = (float)n, z = nf + a, iz = 1.0f / z;
    float t = nf * log1pf(a / nf);
    t += (a - 0.5f) * logf(z);
    t += 0.91893853320467274f - a;
    t += iz * (0.083333333333333333f - iz * iz * 0.0027777777777777778f);
    return t;
}

// Parent configuration j of a table laid out parents-major, child-last:
// its r cells start at j * r, one apart.
struct DenseRows {
    int32_t r;
    __device__ __forceinline__ int64_t base(int64_t j) const { return j * r; }
    __device__ __forceinline__ int64_t step() const { return 1; }
};

// Per-thread part of a score over parent configurations j0, j0 + step, ... of
// a complete table; rows.base(j) is the first cell of configuration j and
// rows.step() the distance between its r child cells.
//   LL  = sum N_ijk log2(N_ijk / N_ij) = -(1/ln2) sum N_ijk log1p((N_ij - N_ijk) / N_ijk):
//         every term has the same sign and the integer difference is exact.
//   MDL = -LL + (log2 m / 2)(r - 1) q.
//   BDeu = sum_j [sum_k G(a_jk, N_ijk) - G(a_j, N_ij)], G(a, n) = lnGamma(a+n) - lnGamma(a).
//         Writing G(a, n) = (n ln n - n) + R(a, n), the (n ln n - n) parts of a
//         configuration sum to sum_k N_ijk ln(N_ijk / N_ij) (the -n terms cancel
//         since sum_k N_ijk = N_ij), which takes the LL form above in nats; the
//         remainders R are O(log n) each and are summed in FP32 as
//         R'' = R + lnGamma(a) (bdeu_rem), the lnGamma(a) being added back once
//         per query in FP64 by count.  Priors a >= 1 (tiny tables) take R in
//         FP64 with lgamma.  No FP64 transcendental runs per cell.
//   MI  = (1/ln2) sum_jk p_j p_k [(1 + x_jk) ln(1 + x_jk) - x_jk] over all cells
//         with p_j, p_k > 0, x_jk = (N_jk m - N_j N_k) / (N_j N_k) with an exact
//         int64 numerator; this equals the usual sum because sum p_j p_k x_jk = 0,
//         and every term is >= 0.
template <bool kGlobal, class Rows>
__device__ ScoreAcc score_rows(const int32_t *tab, const Rows &rows, int64_t q, int32_t r, int kind,
                               const int64_t *marg_child, int64_t m, const BdeuK &bk, int64_t j0, int64_t jstep)
{
    ScoreAcc acc = score_zero();
    const int64_t cs = rows.step();
    for (int64_t j = j0; j < q; j += jstep) {
        const int64_t b = rows.base(j);
        int64_t nij = 0;
        for (int k = 0; k < r; ++k) nij += tab_ld<kGlobal>(tab, b + k * cs);
        if (nij == 0) continue;
        if (kind == kLL || kind == kMDL) {
            for (int k = 0; k < r; ++k) {
                const int32_t n = tab_ld<kGlobal>(tab, b + k * cs);
                if (n > 0) kahan_add(acc.k, (float)n * log1pf((float)(nij - n) / (float)n));
            }
        } else if (kind == kBDeu) {
            for (int k = 0; k < r; ++k) {
                const int32_t n = tab_ld<kGlobal>(tab, b + k * cs);
                if (n <= 0) continue;
                kahan_add(acc.k, -(float)n * log1pf((float)(nij - n) / (float)n));
                if (bk.akd < 1.0) {
                    kahan_add(acc.r, bdeu_rem(bk.ak, bk.g1k, n));
                    ++acc.nk;
                } else {
                    acc.d += lgamma(bk.akd + (double)n) - bk.lgk - ((double)n * log((double)n) - (double)n);
                }
            }
            if (bk.ajd < 1.0) {
                kahan_add(acc.r, -bdeu_rem(bk.aj, bk.g1j, nij));
                ++acc.nj;
            } else {
                acc.d -= lgamma(bk.ajd + (double)nij) - bk.lgj - ((double)nij * log((double)nij) - (double)nij);
            }
        } else {  // kMI
            const float pj = (float)nij / (float)m;
            for (int k = 0; k < r; ++k) {
                const int64_t nk = marg_child[k];
                if (nk == 0) continue;
                const int32_t n = tab_ld<kGlobal>(tab, b + k * cs);
                const long long num = (long long)n * m - (long long)nij * nk;
                const float x = (float)num / ((float)nij * (float)nk);
                kahan_add(acc.k, pj * ((float)nk / (float)m) * mi_term(x));
            }
        }
    }
    return acc;
}

__device__ __forceinline__ void acc_merge(ScoreAcc &a, const ScoreAcc &b)
{
    kahan_merge(a.k, b.k);
    kahan_merge(a.r, b.r);
    a.d += b.d;
    a.nk += b.nk;
    a.nj += b.nj;
}

__device__ __forceinline__ void warp_merge(ScoreAcc &acc)
{
    for (int o = 16; o > 0; o >>= 1) {
        ScoreAcc other;
        other.k = Kahan{__shfl_xor_sync(kFull, acc.k.s, o), __shfl_xor_sync(kFull, acc.k.c, o)};
        other.r = Kahan{__shfl_xor_sync(kFull, acc.r.s, o), __shfl_xor_sync(kFull, acc.r.c, o)};
        other.d = __shfl_xor_sync(kFull, acc.d, o);
        other.nk = __shfl_xor_sync(kFull, acc.nk, o);
        other.nj = __shfl_xor_sync(kFull, acc.nj, o);
        acc_merge(acc, other);
    }
}

__device__ float score_finish(const ScoreAcc &t, int kind, int64_t m, int32_t r, int64_t q, const BdeuK &bk)
{
    const float sum = __fsub_rn(t.k.s, t.k.c);
    if (kind == kLL) return -sum * kInvLn2;
    if (kind == kMDL)
        return (float)((double)sum * (double)kInvLn2 + 0.5 * log2((double)m) * (double)(r - 1) * (double)q);
    if (kind == kBDeu)
        return (float)((double)sum + (double)__fsub_rn(t.r.s, t.r.c) + t.d - (double)t.nk * bk.lgk +
                       (double)t.nj * bk.lgj);
    return sum * kInvLn2;
}

// BDeu constants of a (q, r) score computed by thread 0 of the block and
// shared (uniform branch on kind).
__device__ BdeuK block_bdeu_consts(int kind, int64_t q, int32_t r, double ess)
{
    __shared__ BdeuK s_bk;
    BdeuK bk{};
    if (kind == kBDeu) {
        if (threadIdx.x == 0) s_bk = bdeu_consts(q, r, ess);
        __syncthreads();
        bk = s_bk;
        __syncthreads();
    }
    return bk;
}

// The same for one warp (lane 0 computes, the others receive).
__device__ BdeuK warp_bdeu_consts(int kind, int64_t q, int32_t r, double ess)
{
    BdeuK bk{};
    if (kind == kBDeu) {
        if ((threadIdx.x & 31) == 0) bk = bdeu_consts(q, r, ess);
        bk.ak = __shfl_sync(kFull, bk.ak, 0);
        bk.aj = __shfl_sync(kFull, bk.aj, 0);
        bk.g1k = __shfl_sync(kFull, bk.g1k, 0);
        bk.g1j = __shfl_sync(kFull, bk.g1j, 0);
        bk.akd = __shfl_sync(kFull, bk.akd, 0);
        bk.ajd = __shfl_sync(kFull, bk.ajd, 0);
        bk.lgk = __shfl_sync(kFull, bk.lgk, 0);
        bk.lgj = __shfl_sync(kFull, bk.lgj, 0);
    }
    return bk;
}

// Block-wide reduction of per-thread accumulators; thread 0 returns the score.
__device__ float block_finish(ScoreAcc acc, ScoreAcc *red, int kind, int64_t m, int32_t r, int64_t q,
                              const BdeuK &bk)
{
    warp_merge(acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    float out = 0.0f;
    if (threadIdx.x == 0) {
        ScoreAcc t = score_zero();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) acc_merge(t, red[w]);
        out = score_finish(t, kind, m, r, q, bk);
    }
    __syncthreads();
    return out;
}

// Whole block; the result is returned in thread 0.
template <bool kGlobal>
__device__ float block_score(const int32_t *tab, int32_t cells, int32_t r, int kind,
                             const int64_t *marg_child, int64_t m, double ess, ScoreAcc *red)
{
    const int64_t q = cells / r;
    const BdeuK bk = block_bdeu_consts(kind, q, r, ess);
    const ScoreAcc acc = score_rows<kGlobal>(tab, DenseRows{r}, q, r, kind, marg_child, m, bk, threadIdx.x,
                                             blockDim.x);
    return block_finish(acc, red, kind, m, r, q, bk);
}

// One warp; the result is returned in lane 0.
__device__ float warp_score(const int32_t *tab, int32_t cells, int32_t r, int kind,
                            const int64_t *marg_child, int64_t m, double ess)
{
    const int64_t q = cells / r;
    const BdeuK bk = warp_bdeu_consts(kind, q, r, ess);
    ScoreAcc acc = score_rows<true>(tab, DenseRows{r}, q, r, kind, marg_child, m, bk, threadIdx.x & 31, 32);
    warp_merge(acc);
    return score_finish(acc, kind, m, r, q, bk);
}

// ------------------------------------------------------------ bitmap (Alg. 1)

constexpr int kBitmapWarps = 32;  // upper bound on warps per CTA of bitmap_kernel

struct Level {
    const uint64_t *row;     // level 0: first state's bitmap at this chunk (global)
    int32_t arity;
    int32_t stride;
    int32_t slot;            // levels >= 1: first staged slot
};

// One tree node per loop iteration.  acc holds the lane's two words of the
// AND of the states chosen above this level.
template <int K, int L>
struct Dfs {
    static __device__ __forceinline__ void run(const Level *lv, const ulonglong2 *stage, int64_t wstride,
                                               ulonglong2 acc, int cell, int32_t *tab, int lane)
    {
        const Level v = lv[L];
        int s0 = 0;
        if constexpr (L == K - 1 && L > 0) {
            // leaves: the first eight child states unrolled, so their shared-memory
            // loads, popcounts and warp reductions overlap
            unsigned cnt[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                cnt[s] = 0u;
                if (s < v.arity) {
                    const ulonglong2 b = stage[(v.slot + s) * 32 + lane];
                    cnt[s] = (unsigned)(__popcll(acc.x & b.x) + __popcll(acc.y & b.y));
                }
            }
#pragma unroll
            for (int s = 0; s < 8; ++s) {
                if (s < v.arity) {
                    const unsigned c = __reduce_add_sync(kFull, cnt[s]);
                    if (lane == 0 && c) atomicAdd(&tab[cell + s * v.stride], (int)c);
                }
            }
            s0 = 8;
        }
        for (int s = s0; s < v.arity; ++s) {
            ulonglong2 b;
            if constexpr (L == 0)
                b = __ldg(reinterpret_cast<const ulonglong2 *>(v.row + (int64_t)s * wstride));
            else
                b = stage[(v.slot + s) * 32 + lane];
            ulonglong2 x;
            x.x = acc.x & b.x;
            x.y = acc.y & b.y;
            if constexpr (L == K - 1) {
                unsigned cnt = (unsigned)(__popcll(x.x) + __popcll(x.y));
                cnt = __reduce_add_sync(kFull, cnt);
                if (lane == 0 && cnt) atomicAdd(&tab[cell + s * v.stride], (int)cnt);
            } else {
                if (__any_sync(kFull, (x.x | x.y) != 0ull))
                    Dfs<K, L + 1>::run(lv, stage, wstride, x, cell + s * v.stride, tab, lane);
            }
        }
    }
};

template <int K>
__device__ __forceinline__ void bitmap_task(const CountParams &P, const QVar *qv, int64_t c0, int64_t c1,
                                         ulonglong2 *stage, int32_t *tab, int lane)
{
    for (int64_t c = c0; c < c1; ++c) {
        const int64_t w = c * kChunkWords + 2 * lane;
        // level 0 is read in place; levels 1..K-1 are staged per lane
        Level lv[K];
        int slot = 0;
#pragma unroll
        for (int d = 0; d < K; ++d) {
            const QVar v = qv[d];
            const uint64_t *row = P.bits + (int64_t)v.soff * P.wstride + w;
            lv[d] = Level{row, v.arity, v.stride, slot};
            if (d > 0) {
                for (int s = 0; s < v.arity; ++s)
                    stage[(slot + s) * 32 + lane] =
                        __ldg(reinterpret_cast<const ulonglong2 *>(row + (int64_t)s * P.wstride));
                slot += v.arity;
            }
        }
        Dfs<K, 0>::run(lv, stage, P.wstride, make_ulonglong2(~0ull, ~0ull), 0, tab, lane);
        __syncwarp();
    }
}

// Register-blocked bitmap counts for small tables (no tree walk): every
// cell is one AND + popcount of two words per lane per 4096-instance chunk,
// counted in registers over the whole task and reduced across the warp once
// per cell at the end.  Dense small tables gain nothing from zero-support
// pruning, so the walk's per-node control and per-leaf atomics are dropped.
// Two variables of arities RA x RB:
template <int RA, int RB>
__device__ __noinline__ void small2_task(const CountParams &P, const QVar *qv, int64_t c0, int64_t c1,
                                         int32_t *tab, int lane)
{
    const uint64_t *row_a = P.bits + (int64_t)qv[0].soff * P.wstride + 2 * lane;
    const uint64_t *row_b = P.bits + (int64_t)qv[1].soff * P.wstride + 2 * lane;
    unsigned cnt[RA][RB];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) cnt[a][b] = 0u;
    // two chunks per iteration: twice the loads in flight per warp
    constexpr int U = (RA + RB <= 8) ? 2 : 1;
    int64_t c = c0;
    for (; c + U <= c1; c += U) {
        ulonglong2 xa[U][RA], xb[U][RB];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t w = (c + u) * kChunkWords;
#pragma unroll
            for (int a = 0; a < RA; ++a)
                xa[u][a] = __ldg(reinterpret_cast<const ulonglong2 *>(row_a + (int64_t)a * P.wstride + w));
#pragma unroll
            for (int b = 0; b < RB; ++b)
                xb[u][b] = __ldg(reinterpret_cast<const ulonglong2 *>(row_b + (int64_t)b * P.wstride + w));
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int a = 0; a < RA; ++a)
#pragma unroll
                for (int b = 0; b < RB; ++b)
                    cnt[a][b] += (unsigned)(__popcll(xa[u][a].x & xb[u][b].x) + __popcll(xa[u][a].y & xb[u][b].y));
    }
    for (; c < c1; ++c) {
        const int64_t w = c * kChunkWords;
        ulonglong2 xa[RA], xb[RB];
#pragma unroll
        for (int a = 0; a < RA; ++a)
            xa[a] = __ldg(reinterpret_cast<const ulonglong2 *>(row_a + (int64_t)a * P.wstride + w));
#pragma unroll
        for (int b = 0; b < RB; ++b)
            xb[b] = __ldg(reinterpret_cast<const ulonglong2 *>(row_b + (int64_t)b * P.wstride + w));
#pragma unroll
        for (int a = 0; a < RA; ++a)
#pragma unroll
            for (int b = 0; b < RB; ++b)
                cnt[a][b] += (unsigned)(__popcll(xa[a].x & xb[b].x) + __popcll(xa[a].y & xb[b].y));
    }
    const int sa = qv[0].stride, sb = qv[1].stride;
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int b = 0; b < RB; ++b) {
            const unsigned v = __reduce_add_sync(kFull, cnt[a][b]);
            if (lane == 0 && v) atomicAdd(&tab[a * sa + b * sb], (int)v);
        }
}

// Three variables: the first (any arity) is walked state by state, the other
// two (RB x RC) are register-blocked.
template <int RB, int RC>
__device__ __noinline__ void small3_task(const CountParams &P, const QVar *qv, int64_t c0, int64_t c1,
                                         int s0, int32_t *tab, int lane)
{
    const uint64_t *row_a = P.bits + (int64_t)qv[0].soff * P.wstride + 2 * lane;
    const uint64_t *row_b = P.bits + (int64_t)qv[1].soff * P.wstride + 2 * lane;
    const uint64_t *row_c = P.bits + (int64_t)qv[2].soff * P.wstride + 2 * lane;
    const int sa = qv[0].stride, sb = qv[1].stride, sc = qv[2].stride;
    const int a_lo = s0 >= 0 ? s0 : 0, a_hi = s0 >= 0 ? s0 + 1 : qv[0].arity;
    for (int a = a_lo; a < a_hi; ++a) {
        if (P.marg[qv[0].soff + a] == 0) continue;  // a state absent from D
        unsigned cnt[RB][RC];
#pragma unroll
        for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int cc = 0; cc < RC; ++cc) cnt[b][cc] = 0u;
        for (int64_t c = c0; c < c1; ++c) {
            const int64_t w = c * kChunkWords;
            const ulonglong2 xa = __ldg(reinterpret_cast<const ulonglong2 *>(row_a + (int64_t)a * P.wstride + w));
            ulonglong2 xb[RB], xc[RC];
#pragma unroll
            for (int b = 0; b < RB; ++b)
                xb[b] = __ldg(reinterpret_cast<const ulonglong2 *>(row_b + (int64_t)b * P.wstride + w));
#pragma unroll
            for (int cc = 0; cc < RC; ++cc)
                xc[cc] = __ldg(reinterpret_cast<const ulonglong2 *>(row_c + (int64_t)cc * P.wstride + w));
#pragma unroll
            for (int b = 0; b < RB; ++b) {
                const uint64_t px = xa.x & xb[b].x, py = xa.y & xb[b].y;
#pragma unroll
                for (int cc = 0; cc < RC; ++cc)
                    cnt[b][cc] += (unsigned)(__popcll(px & xc[cc].x) + __popcll(py & xc[cc].y));
            }
        }
#pragma unroll
        for (int b = 0; b < RB; ++b)
#pragma unroll
            for (int cc = 0; cc < RC; ++cc) {
                const unsigned v = __reduce_add_sync(kFull, cnt[b][cc]);
                if (lane == 0 && v) atomicAdd(&tab[a * sa + b * sb + cc * sc], (int)v);
            }
    }
}

// Arities the register-blocked paths are compiled for.
constexpr int kSmallLo = 2, kSmallHi = 5;
__device__ __forceinline__ bool small_arity(int r) { return r >= kSmallLo && r <= kSmallHi; }

template <int K>
__device__ bool small_dispatch(const CountParams &P, const QVar *qv_in, int64_t c0, int64_t c1, int s0,
                               int32_t *tab, int lane)
{
    // the two blocked variables are symmetric (each carries its own stride),
    // so they are ordered by arity and only RX <= RY is compiled
    QVar qv[K];
#pragma unroll
    for (int t = 0; t < K; ++t) qv[t] = qv_in[t];
    if (qv[K - 2].arity > qv[K - 1].arity) {
        const QVar tmp = qv[K - 2];
        qv[K - 2] = qv[K - 1];
        qv[K - 1] = tmp;
    }
    const int r1 = qv[K - 2].arity, r2 = qv[K - 1].arity;
    if (!small_arity(r1) || !small_arity(r2)) return false;
#define FC_SMALL_CASE(X, Y)                                                         \
    case (X - kSmallLo) * 4 + (Y - kSmallLo):                                       \
        if constexpr (K == 2) small2_task<X, Y>(P, qv, c0, c1, tab, lane);          \
        else small3_task<X, Y>(P, qv, c0, c1, s0, tab, lane);                       \
        return true;
    switch ((r1 - kSmallLo) * 4 + (r2 - kSmallLo)) {
        FC_SMALL_CASE(2, 2) FC_SMALL_CASE(2, 3) FC_SMALL_CASE(2, 4) FC_SMALL_CASE(2, 5)
        FC_SMALL_CASE(3, 3) FC_SMALL_CASE(3, 4) FC_SMALL_CASE(3, 5)
        FC_SMALL_CASE(4, 4) FC_SMALL_CASE(4, 5)
        FC_SMALL_CASE(5, 5)
    }
#undef FC_SMALL_CASE
    return false;
}

__global__ void __launch_bounds__(256, 2) bitmap_kernel(const CountParams P)
{
    extern __shared__ __align__(16) ulonglong2 stage_all[];
    __shared__ QVar s_qv[kBitmapWarps][kMaxBitmapK];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    ulonglong2 *stage = stage_all + (size_t)warp * P.stage_slots * 32;
    const int64_t n_tasks = P.n_btasks;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(P.next_task, 1);
        t = __shfl_sync(kFull, t, 0);
        if (t >= n_tasks) break;
        const BTask bt = P.btasks[t];
        const int q = bt.q;
        const QHead h = P.qh[q];
        const int k = h.k;
        if (lane < k) s_qv[warp][lane] = P.qv[h.var_off + lane];
        __syncwarp();
        const int64_t c0 = bt.c0, c1 = bt.c1;
        int32_t *tab = P.tables + h.table_off;
        const QVar *qv = s_qv[warp];
        bool done = false;
        if (P.small_paths) {
            if (k == 2) done = small_dispatch<2>(P, qv, c0, c1, -1, tab, lane);
            else if (k == 3) done = small_dispatch<3>(P, qv, c0, c1, bt.s0, tab, lane);
        }
        // a state-split task that did not take the register-blocked path
        // (cannot happen: planner and kernel test the same arities) leaves
        // the whole walk to the task of state 0
        if (!done && bt.s0 > 0) done = true;
        if (!done) switch (k) {
        case 1: bitmap_task<1>(P, qv, c0, c1, stage, tab, lane); break;
        case 2: bitmap_task<2>(P, qv, c0, c1, stage, tab, lane); break;
        case 3: bitmap_task<3>(P, qv, c0, c1, stage, tab, lane); break;
        case 4: bitmap_task<4>(P, qv, c0, c1, stage, tab, lane); break;
        case 5: bitmap_task<5>(P, qv, c0, c1, stage, tab, lane); break;
        case 6: bitmap_task<6>(P, qv, c0, c1, stage, tab, lane); break;
        case 7: bitmap_task<7>(P, qv, c0, c1, stage, tab, lane); break;
        case 8: bitmap_task<8>(P, qv, c0, c1, stage, tab, lane); break;
        default: break;  // the planner never sends other depths here
        }
        if (h.score_kind != kNoScore) {
            __threadfence();
            int last = 0;
            if (lane == 0) last = atomicAdd(&P.tickets[q], 1) == h.nparts - 1;
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                const float s = warp_score(tab, h.cells, h.r_child, h.score_kind, P.marg + h.child_soff,
                                           P.m, P.ess);
                if (lane == 0) P.scores[h.score_slot] = s;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------- mixed-radix key counts

// SWAR keys: 16 rows per thread; register pair (2i, 2i+1) holds rows
// {4i, 4i+2} and {4i+1, 4i+3} in its low and high 16-bit halves.  Valid when
// every key is below 2^16.
__device__ __forceinline__ void key_rows_swar(const CountParams &P, const QVar *vs, int k,
                                              int64_t r0, int64_t r1, int32_t *tab)
{
    const int64_t ngroups = (r1 - r0) >> 4;
    for (int64_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const int64_t p = r0 + (g << 4);
        uint32_t acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = 0u;
        int t = 0;
        for (; t + 2 <= k; t += 2) {  // two columns in flight
            const QVar v0 = vs[t], v1 = vs[t + 1];
            const uint4 x0 = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)v0.var * P.m_pad + p));
            const uint4 x1 = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)v1.var * P.m_pad + p));
            const uint32_t w0[4] = {x0.x, x0.y, x0.z, x0.w}, w1[4] = {x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[2 * i] += (w0[i] & 0x00FF00FFu) * (uint32_t)v0.stride + (w1[i] & 0x00FF00FFu) * (uint32_t)v1.stride;
                acc[2 * i + 1] += ((w0[i] >> 8) & 0x00FF00FFu) * (uint32_t)v0.stride +
                                  ((w1[i] >> 8) & 0x00FF00FFu) * (uint32_t)v1.stride;
            }
        }
        if (t < k) {
            const QVar v0 = vs[t];
            const uint4 x0 = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)v0.var * P.m_pad + p));
            const uint32_t w0[4] = {x0.x, x0.y, x0.z, x0.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[2 * i] += (w0[i] & 0x00FF00FFu) * (uint32_t)v0.stride;
                acc[2 * i + 1] += ((w0[i] >> 8) & 0x00FF00FFu) * (uint32_t)v0.stride;
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            atomicAdd(&tab[acc[j] & 0xFFFFu], 1);
            atomicAdd(&tab[acc[j] >> 16], 1);
        }
    }
    for (int64_t p = r0 + (ngroups << 4) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = 0u;
        for (int t = 0; t < k; ++t)
            key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * (uint32_t)vs[t].stride;
        atomicAdd(&tab[key], 1);
    }
}

// SWAR keys as byte offsets into an interleaved table: L = 2^lshift copies,
// cell c of copy j at word c * L + j, and lane l counts into copy l % L.  The
// copies of one cell sit in consecutive banks, so lanes that hit the same
// cell do not serialise and (for L = 32) every lane owns a bank.  Strides are
// pre-scaled by 4L and each 16-bit lane starts at the lane's copy, so a key
// is one mask or shift away from its atomic's address.  Valid when the
// interleaved table spans at most 64 KiB (cells x L <= 16384).
__device__ __forceinline__ void key_rows_swar_bytes(const CountParams &P, const QVar *vs, int k,
                                                    int64_t r0, int64_t r1, int lshift, int32_t *tab0)
{
    char *smem = reinterpret_cast<char *>(tab0);
    const uint32_t base_bytes = (uint32_t)((threadIdx.x & ((1 << lshift) - 1)) << 2);
    const int sshift = 2 + lshift;
    const uint32_t init = base_bytes | (base_bytes << 16);
    // Warp groups of 1024 rows: lane l of group G reads 16-byte vectors
    // 64 G + l and 64 G + 32 + l, so each load instruction covers 512
    // contiguous bytes of the column.
    const int64_t nfull = (r1 - r0) >> 10;
    const int lane = threadIdx.x & 31;
    for (int64_t u = threadIdx.x; u < (nfull << 5); u += blockDim.x) {
        const int64_t vec = ((u >> 5) << 6) + lane;  // 16-byte vector index in the range
        uint32_t acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = init;
        for (int t = 0; t < k; ++t) {
            const QVar v = vs[t];
            const uint4 *col = reinterpret_cast<const uint4 *>(P.D + (int64_t)v.var * P.m_pad + r0) + vec;
            const uint4 x0 = __ldg(col), x1 = __ldg(col + 32);
            const uint32_t st = (uint32_t)v.stride << sshift;
            const uint32_t w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[2 * i] += __byte_perm(w[i], 0u, 0x4240) * st;
                acc[2 * i + 1] += __byte_perm(w[i], 0u, 0x4341) * st;
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] & 0xFFFFu)), 1);
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] >> 16)), 1);
        }
    }
    for (int64_t p = r0 + (nfull << 10) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = base_bytes;
        for (int t = 0; t < k; ++t)
            key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * ((uint32_t)vs[t].stride << sshift);
        atomicAdd(reinterpret_cast<int *>(smem + key), 1);
    }
}

// key_rows_swar_bytes with the number of variables fixed at compile time:
// column pointers and scaled strides live in registers for the whole item and
// the loop over variables is unrolled.
template <int K>
__device__ __forceinline__ void key_rows_swar_bytes_k(const CountParams &P, const QVar *vs, int64_t r0,
                                                      int64_t r1, int lshift, int32_t *tab0)
{
    char *smem = reinterpret_cast<char *>(tab0);
    const uint32_t base_bytes = (uint32_t)((threadIdx.x & ((1 << lshift) - 1)) << 2);
    const int sshift = 2 + lshift;
    const uint32_t init = base_bytes | (base_bytes << 16);
    const uint4 *col[K];
    uint32_t st[K];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        col[t] = reinterpret_cast<const uint4 *>(P.D + (int64_t)vs[t].var * P.m_pad + r0);
        st[t] = (uint32_t)vs[t].stride << sshift;
    }
    const int64_t nfull = (r1 - r0) >> 10;
    const int lane = threadIdx.x & 31;
    for (int64_t u = threadIdx.x; u < (nfull << 5); u += blockDim.x) {
        const int64_t vec = ((u >> 5) << 6) + lane;
        uint32_t acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = init;
#pragma unroll
        for (int t = 0; t < K; ++t) {
            const uint4 x0 = __ldg(col[t] + vec), x1 = __ldg(col[t] + vec + 32);
            const uint32_t w[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[2 * i] += __byte_perm(w[i], 0u, 0x4240) * st[t];
                acc[2 * i + 1] += __byte_perm(w[i], 0u, 0x4341) * st[t];
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] & 0xFFFFu)), 1);
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] >> 16)), 1);
        }
    }
    for (int64_t p = r0 + (nfull << 10) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = base_bytes;
#pragma unroll
        for (int t = 0; t < K; ++t) key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * st[t];
        atomicAdd(reinterpret_cast<int *>(smem + key), 1);
    }
}

// key_rows_swar_bytes_k on the 4-bit codes (every arity <= 16): a lane's
// 16-byte load brings 32 rows of a column instead of 16, so a warp group of
// 1024 rows is one 512-byte load per column, half the load wavefronts of the
// byte columns.  Word i of a load holds rows 8i .. 8i + 7, row 2b in the low
// nibble of byte b; one mask gives the even rows as bytes, a shift and a mask
// the odd ones.  Consecutive variables are then combined in groups of GS on
// the packed bytes by Horner's rule (g = g * r + s, one IMAD for four rows;
// no carry between bytes while a group has at most 256 joint states), and
// each group enters the 16-bit key lanes once (PRMT + IMAD for two rows) with
// the stride of its last, fastest variable.  The rows past the last whole
// group come from the byte columns.
template <int K, int GS>
__device__ __forceinline__ void key_rows_swar_nib_k(const CountParams &P, const QVar *vs, int64_t r0, int64_t r1,
                                                    int lshift, int32_t *tab0)
{
    constexpr int NG = (K + GS - 1) / GS;
    char *smem = reinterpret_cast<char *>(tab0);
    const uint32_t base_bytes = (uint32_t)((threadIdx.x & ((1 << lshift) - 1)) << 2);
    const int sshift = 2 + lshift;
    const uint32_t init = base_bytes | (base_bytes << 16);
    const int64_t pad4 = P.m_pad / 2;
    const uint4 *col[K];
    uint32_t mul[K];
    uint32_t st[NG];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        col[t] = reinterpret_cast<const uint4 *>(P.D4 + (int64_t)vs[t].var * pad4 + r0 / 2);
        mul[t] = (uint32_t)vs[t].arity;
    }
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) st[gi] = (uint32_t)vs[min(K, (gi + 1) * GS) - 1].stride << sshift;
    const int64_t nfull = (r1 - r0) >> 10;
    const int lane = threadIdx.x & 31;
    for (int64_t u = threadIdx.x; u < (nfull << 5); u += blockDim.x) {
        const int64_t vec = ((u >> 5) << 5) + lane;  // 16-byte vector (32 rows) in the range
        uint32_t acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = init;
#pragma unroll
        for (int gi = 0; gi < NG; ++gi) {
            uint32_t g[8];
#pragma unroll
            for (int t = gi * GS; t < (K < (gi + 1) * GS ? K : (gi + 1) * GS); ++t) {
                const uint4 x = __ldg(col[t] + vec);
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t ev = w[i] & 0x0F0F0F0Fu, od = (w[i] >> 4) & 0x0F0F0F0Fu;
                    g[2 * i] = t == gi * GS ? ev : g[2 * i] * mul[t] + ev;
                    g[2 * i + 1] = t == gi * GS ? od : g[2 * i + 1] * mul[t] + od;
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[2 * i] += __byte_perm(g[i], 0u, 0x4240) * st[gi];
                acc[2 * i + 1] += __byte_perm(g[i], 0u, 0x4341) * st[gi];
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] & 0xFFFFu)), 1);
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] >> 16)), 1);
        }
    }
    for (int64_t p = r0 + (nfull << 10) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = base_bytes;
#pragma unroll
        for (int t = 0; t < K; ++t) key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * ((uint32_t)vs[t].stride << sshift);
        atomicAdd(reinterpret_cast<int *>(smem + key), 1);
    }
}

// key_rows_swar_nib_k for variables of at most 4 states each: consecutive
// variables are first paired on the packed nibbles (a * r + b stays below 16:
// one IMAD for eight rows, no carry between nibbles), each pair is unpacked
// to bytes once, and two pairs combine on the bytes (at most 256 joint
// states) before entering the key lanes, so one PRMT + IMAD per two rows
// carries the digit of up to four variables.
template <int K>
__device__ __forceinline__ void key_rows_swar_nib4_k(const CountParams &P, const QVar *vs, int64_t r0, int64_t r1,
                                                     int lshift, int32_t *tab0)
{
    constexpr int NC = (K + 3) / 4;  // byte digits: runs of up to four variables
    char *smem = reinterpret_cast<char *>(tab0);
    const uint32_t base_bytes = (uint32_t)((threadIdx.x & ((1 << lshift) - 1)) << 2);
    const int sshift = 2 + lshift;
    const uint32_t init = base_bytes | (base_bytes << 16);
    const int64_t pad4 = P.m_pad / 2;
    const uint4 *col[K];
    uint32_t mul[K];
    uint32_t st[NC];
#pragma unroll
    for (int t = 0; t < K; ++t) {
        col[t] = reinterpret_cast<const uint4 *>(P.D4 + (int64_t)vs[t].var * pad4 + r0 / 2);
        mul[t] = (uint32_t)vs[t].arity;
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) st[c] = (uint32_t)vs[min(K, 4 * c + 4) - 1].stride << sshift;
    const int64_t nfull = (r1 - r0) >> 10;
    const int lane = threadIdx.x & 31;
    for (int64_t u = threadIdx.x; u < (nfull << 5); u += blockDim.x) {
        const int64_t vec = ((u >> 5) << 5) + lane;  // 16-byte vector (32 rows) in the range
        uint32_t acc[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[j] = init;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            uint32_t g[8];
#pragma unroll
            for (int t0 = 4 * c; t0 < (K < 4 * c + 4 ? K : 4 * c + 4); t0 += 2) {
                const bool two = t0 + 1 < (K < 4 * c + 4 ? K : 4 * c + 4);
                const uint4 x = __ldg(col[t0] + vec);
                uint32_t w[4] = {x.x, x.y, x.z, x.w};
                uint32_t pr = mul[t0];
                if (two) {
                    const uint4 y = __ldg(col[t0 + 1] + vec);
                    const uint32_t v[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) w[i] = w[i] * mul[t0 + 1] + v[i];
                    pr *= mul[t0 + 1];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const uint32_t ev = w[i] & 0x0F0F0F0Fu, od = (w[i] >> 4) & 0x0F0F0F0Fu;
                    g[2 * i] = t0 == 4 * c ? ev : g[2 * i] * pr + ev;
                    g[2 * i + 1] = t0 == 4 * c ? od : g[2 * i + 1] * pr + od;
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                acc[2 * i] += __byte_perm(g[i], 0u, 0x4240) * st[c];
                acc[2 * i + 1] += __byte_perm(g[i], 0u, 0x4341) * st[c];
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] & 0xFFFFu)), 1);
            atomicAdd(reinterpret_cast<int *>(smem + (acc[j] >> 16)), 1);
        }
    }
    for (int64_t p = r0 + (nfull << 10) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = base_bytes;
#pragma unroll
        for (int t = 0; t < K; ++t) key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * ((uint32_t)vs[t].stride << sshift);
        atomicAdd(reinterpret_cast<int *>(smem + key), 1);
    }
}

__device__ __forceinline__ bool all_arities_at_most_4(const QVar *vs, int k)
{
    for (int t = 0; t < k; ++t)
        if (vs[t].arity > 4) return false;
    return true;
}

// Groups of three when every run of three consecutive variables has at most
// 256 joint states, else of two (always valid for arities <= 16).
__device__ __forceinline__ bool nib_groups_of_three(const QVar *vs, int k)
{
    for (int a = 0; a + 3 <= k; ++a)
        if (vs[a].arity * vs[a + 1].arity * vs[a + 2].arity > 256) return false;
    return true;
}

template <bool kNib>
__device__ __forceinline__ void key_rows_swar_dispatch(const CountParams &P, const QVar *vs, int k, int64_t r0,
                                                       int64_t r1, int lshift, int32_t *tab0)
{
    if constexpr (kNib) {
        if (k >= 2 && k <= 6 && all_arities_at_most_4(vs, k)) {
            switch (k) {
            case 2: key_rows_swar_nib4_k<2>(P, vs, r0, r1, lshift, tab0); return;
            case 3: key_rows_swar_nib4_k<3>(P, vs, r0, r1, lshift, tab0); return;
            case 4: key_rows_swar_nib4_k<4>(P, vs, r0, r1, lshift, tab0); return;
            case 5: key_rows_swar_nib4_k<5>(P, vs, r0, r1, lshift, tab0); return;
            default: key_rows_swar_nib4_k<6>(P, vs, r0, r1, lshift, tab0); return;
            }
        }
        const bool g3 = nib_groups_of_three(vs, k);
        switch (k) {
        case 1: key_rows_swar_nib_k<1, 1>(P, vs, r0, r1, lshift, tab0); return;
        case 2: key_rows_swar_nib_k<2, 2>(P, vs, r0, r1, lshift, tab0); return;
        case 3:
            if (g3) key_rows_swar_nib_k<3, 3>(P, vs, r0, r1, lshift, tab0);
            else key_rows_swar_nib_k<3, 2>(P, vs, r0, r1, lshift, tab0);
            return;
        case 4:
            if (g3) key_rows_swar_nib_k<4, 3>(P, vs, r0, r1, lshift, tab0);
            else key_rows_swar_nib_k<4, 2>(P, vs, r0, r1, lshift, tab0);
            return;
        case 5:
            if (g3) key_rows_swar_nib_k<5, 3>(P, vs, r0, r1, lshift, tab0);
            else key_rows_swar_nib_k<5, 2>(P, vs, r0, r1, lshift, tab0);
            return;
        case 6:
            if (g3) key_rows_swar_nib_k<6, 3>(P, vs, r0, r1, lshift, tab0);
            else key_rows_swar_nib_k<6, 2>(P, vs, r0, r1, lshift, tab0);
            return;
        default: break;
        }
    }
    switch (k) {
    case 1: key_rows_swar_bytes_k<1>(P, vs, r0, r1, lshift, tab0); break;
    case 2: key_rows_swar_bytes_k<2>(P, vs, r0, r1, lshift, tab0); break;
    case 3: key_rows_swar_bytes_k<3>(P, vs, r0, r1, lshift, tab0); break;
    case 4: key_rows_swar_bytes_k<4>(P, vs, r0, r1, lshift, tab0); break;
    case 5: key_rows_swar_bytes_k<5>(P, vs, r0, r1, lshift, tab0); break;
    case 6: key_rows_swar_bytes_k<6>(P, vs, r0, r1, lshift, tab0); break;
    default: key_rows_swar_bytes(P, vs, k, r0, r1, lshift, tab0); break;
    }
}

// Scalar keys (any table size up to 2^31 cells), counted in global memory.
__device__ __forceinline__ void key_rows_global(const CountParams &P, const QVar *vs, int k,
                                                int64_t r0, int64_t r1, int32_t *tab)
{
    const int64_t ngroups = (r1 - r0) >> 4;
    for (int64_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        const int64_t p = r0 + (g << 4);
        uint32_t key[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) key[j] = 0u;
        for (int t = 0; t < k; ++t) {
            const QVar v = vs[t];
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)v.var * P.m_pad + p));
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) key[4 * i + j] += ((w[i] >> (8 * j)) & 0xffu) * (uint32_t)v.stride;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(&tab[key[j]], 1);
    }
    for (int64_t p = r0 + (ngroups << 4) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = 0u;
        for (int t = 0; t < k; ++t)
            key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * (uint32_t)vs[t].stride;
        atomicAdd(&tab[key], 1);
    }
}

// Scalar keys of which only those in the cell window [w0, w0 + wlen) are
// counted, in shared memory.  K > 0 fixes the number of variables at compile
// time (column pointers and strides in registers); K = 0 reads them per group.
template <int K>
__device__ __forceinline__ void key_rows_window(const CountParams &P, const QVar *vs, int kdyn, int64_t r0,
                                                int64_t r1, uint32_t w0, uint32_t wlen, int32_t *win)
{
    constexpr int KR = K > 0 ? K : 1;
    const uint4 *col[KR];
    uint32_t st[KR];
    if constexpr (K > 0) {
#pragma unroll
        for (int t = 0; t < K; ++t) {
            col[t] = reinterpret_cast<const uint4 *>(P.D + (int64_t)vs[t].var * P.m_pad + r0);
            st[t] = (uint32_t)vs[t].stride;
        }
    }
    const int64_t ngroups = (r1 - r0) >> 4;
    for (int64_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        uint32_t key[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) key[j] = 0u - w0;
        if constexpr (K > 0) {
#pragma unroll
            for (int t = 0; t < K; ++t) {
                const uint4 x = __ldg(col[t] + g);
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) key[4 * i + j] += ((w[i] >> (8 * j)) & 0xffu) * st[t];
            }
        } else {
            for (int t = 0; t < kdyn; ++t) {
                const QVar v = vs[t];
                const uint4 x = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)v.var * P.m_pad + r0) + g);
                const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) key[4 * i + j] += ((w[i] >> (8 * j)) & 0xffu) * (uint32_t)v.stride;
            }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (key[j] < wlen) atomicAdd(&win[key[j]], 1);
    }
    for (int64_t p = r0 + (ngroups << 4) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = 0u - w0;
        for (int t = 0; t < kdyn; ++t)
            key += (uint32_t)P.D[(int64_t)vs[t].var * P.m_pad + p] * (uint32_t)vs[t].stride;
        if (key < wlen) atomicAdd(&win[key], 1);
    }
}

// Windowed keys with variables combined in pairs: when r_t r_{t+1} <= 256 the
// pair's joint state s_t r_{t+1} + s_{t+1} fits a byte, so one multiply-add
// per 32-bit word forms it for four rows at once (no carries between bytes)
// and the pair costs one byte extraction per row instead of two.  The pair
// is a digit of the key with the second variable's stride.  Digit d is
// dg[d] = (first variable, second variable, second's arity or 0 when the
// digit has one variable, stride), in shared memory.
template <int D>
__device__ __forceinline__ void key_rows_window_digits(const CountParams &P, const int4 *dg, int64_t r0,
                                                       int64_t r1, uint32_t w0, uint32_t wlen, int32_t *win)
{
    const int64_t ngroups = (r1 - r0) >> 4;
    for (int64_t g = threadIdx.x; g < ngroups; g += blockDim.x) {
        uint32_t key[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) key[j] = 0u - w0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int4 q = dg[d];
            uint4 x = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)q.x * P.m_pad + r0) + g);
            const uint32_t mul = (uint32_t)q.z;
            if (mul) {
                const uint4 y = __ldg(reinterpret_cast<const uint4 *>(P.D + (int64_t)q.y * P.m_pad + r0) + g);
                x.x = x.x * mul + y.x;
                x.y = x.y * mul + y.y;
                x.z = x.z * mul + y.z;
                x.w = x.w * mul + y.w;
            }
            const uint32_t st = (uint32_t)q.w;
            const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) key[4 * i + j] += ((w[i] >> (8 * j)) & 0xffu) * st;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (key[j] < wlen) atomicAdd(&win[key[j]], 1);
    }
    for (int64_t p = r0 + (ngroups << 4) + threadIdx.x; p < r1; p += blockDim.x) {
        uint32_t key = 0u - w0;
        for (int d = 0; d < D; ++d) {
            const int4 q = dg[d];
            uint32_t x = P.D[(int64_t)q.x * P.m_pad + p];
            if (q.z) x = x * (uint32_t)q.z + P.D[(int64_t)q.y * P.m_pad + p];
            key += x * (uint32_t)q.w;
        }
        if (key < wlen) atomicAdd(&win[key], 1);
    }
}

template <bool kDigits>
__device__ __forceinline__ void key_rows_window_dispatch(const CountParams &P, const QVar *vs, int k, int64_t r0,
                                                         int64_t r1, uint32_t w0, uint32_t wlen, int32_t *win)
{
    // digits after pairing neighbours whose joint state fits a byte (every
    // thread derives the same count; thread 0 writes the table)
    __shared__ int4 s_dig[kMaxK];
    int digits = k;
    if constexpr (kDigits)
        for (int t = digits = 0; t < k; ++digits) t += (t + 1 < k && vs[t].arity * vs[t + 1].arity <= 256) ? 2 : 1;
    if (kDigits && k <= 6 && digits < k) {
        if (threadIdx.x == 0) {
            for (int t = 0, d = 0; t < k; ++d) {
                const bool pair = t + 1 < k && vs[t].arity * vs[t + 1].arity <= 256;
                s_dig[d] = make_int4(vs[t].var, pair ? vs[t + 1].var : 0, pair ? vs[t + 1].arity : 0,
                                     vs[pair ? t + 1 : t].stride);
                t += pair ? 2 : 1;
            }
        }
        __syncthreads();
        switch (digits) {
        case 1: key_rows_window_digits<1>(P, s_dig, r0, r1, w0, wlen, win); return;
        case 2: key_rows_window_digits<2>(P, s_dig, r0, r1, w0, wlen, win); return;
        case 3: key_rows_window_digits<3>(P, s_dig, r0, r1, w0, wlen, win); return;
        case 4: key_rows_window_digits<4>(P, s_dig, r0, r1, w0, wlen, win); return;
        default: key_rows_window_digits<5>(P, s_dig, r0, r1, w0, wlen, win); return;
        }
    }
    switch (k) {
    case 2: key_rows_window<2>(P, vs, k, r0, r1, w0, wlen, win); break;
    case 3: key_rows_window<3>(P, vs, k, r0, r1, w0, wlen, win); break;
    case 4: key_rows_window<4>(P, vs, k, r0, r1, w0, wlen, win); break;
    case 5: key_rows_window<5>(P, vs, k, r0, r1, w0, wlen, win); break;
    case 6: key_rows_window<6>(P, vs, k, r0, r1, w0, wlen, win); break;
    default: key_rows_window<0>(P, vs, k, r0, r1, w0, wlen, win); break;
    }
}

// kThreads x kBlocks: 512 x 2 for the mixed launch; 1024 x 1 for windowed
// tables, whose window then takes the whole shared memory of an SM (and
// whose keys pair variables into byte digits, a path kept out of the mixed
// launch's register allocation).  kNib: the mixed launch's histogram keys
// read the 4-bit columns (P.D4 set), a separate instantiation so that each
// key loop gets the registers of its own kernel.
template <int kThreads, int kBlocks, bool kNib = false>
__global__ void __launch_bounds__(kThreads, kBlocks) count_kernel(const CountParams P)
{
    constexpr bool kWide = kThreads == 1024;
    extern __shared__ __align__(16) int32_t smem_tab[];
    __shared__ QVar s_vars[kMaxK];
    __shared__ int s_item;
    __shared__ int s_last;
    __shared__ ScoreAcc s_red[32];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t nchunks = (P.m + kChunkRows - 1) / kChunkRows;
    const int n_items = P.n_items_dev ? *P.n_items_dev : P.n_items;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const Item W = P.items[it];
        const QHead h = P.qh[W.q];
        const int k = h.k;
        if (threadIdx.x < k) s_vars[threadIdx.x] = P.qv[h.var_off + threadIdx.x];
        // a windowed query's items are (row part, window) pairs, windows fastest
        const bool windowed = h.strategy == kWindow;
        const int nwin = windowed ? h.nwin : 1;
        const int rpart = W.part / nwin, rparts = h.nparts / nwin;
        const int64_t c0 = nchunks * rpart / rparts;
        const int64_t c1 = nchunks * (rpart + 1) / rparts;
        const int64_t r0 = c0 * kChunkRows;
        const int64_t r1 = min(P.m, c1 * kChunkRows);
        const bool in_smem = h.strategy == kHist || h.strategy == kMarginal;
        uint32_t w0 = 0, wlen = 0;  // the item's cell window
        if (windowed) {
            const uint32_t wsz = (uint32_t)((h.cells + nwin - 1) / nwin);
            w0 = (uint32_t)(W.part % nwin) * wsz;
            wlen = min(wsz, (uint32_t)h.cells - w0);
            for (uint32_t c = threadIdx.x; c < wlen; c += blockDim.x) smem_tab[c] = 0;
        }
        int copies = 1;   // per-warp copies (large tables, unscaled keys)
        int lshift = -1;  // log2 of the interleaved copies (tables of <= 16384 cells)
        if (h.strategy == kHist && h.cells <= 16384) {
            lshift = 0;
            // L copies plus the folded table must fit: cells (L + 1) <= smem_cells
            while (lshift < 5 && (h.cells << (lshift + 1)) <= 16384 &&
                   (h.cells << (lshift + 1)) + h.cells <= P.smem_cells)
                ++lshift;
            for (int c = threadIdx.x; c < (h.cells << lshift); c += blockDim.x) smem_tab[c] = 0;
        } else if (in_smem) {
            copies = min(P.hist_copies, P.smem_cells / max(h.cells, 1));
            copies = max(1, min(copies, nwarps));
            for (int c = threadIdx.x; c < h.cells * copies; c += blockDim.x) smem_tab[c] = 0;
        }
        __syncthreads();

        if (k == 0) {
            // no variable with more than one state: the single cell counts the rows
            if (threadIdx.x == 0) {
                if (in_smem)
                    smem_tab[0] = (int32_t)(r1 - r0);
                else
                    atomicAdd(&P.tables[h.table_off], (int32_t)(r1 - r0));
            }
        } else if (h.strategy == kMarginal) {
            // one variable: its per-state counts were taken at load time
            const QVar v = s_vars[0];
            for (int s = threadIdx.x; s < v.arity; s += blockDim.x)
                smem_tab[s * v.stride] = (int32_t)P.marg[v.soff + s];
        } else if (windowed) {
            key_rows_window_dispatch<kWide>(P, s_vars, k, r0, r1, w0, wlen, smem_tab);
        } else if constexpr (!kWide) {  // the wide launch holds windows only
            if (lshift >= 0)
                key_rows_swar_dispatch<kNib>(P, s_vars, k, r0, r1, lshift, smem_tab);
            else if (in_smem)
                key_rows_swar(P, s_vars, k, r0, r1, smem_tab + (warp % copies) * h.cells);
            else
                key_rows_global(P, s_vars, k, r0, r1, P.tables + h.table_off);
        }
        __syncthreads();

        // the final table: the interleaved copies are summed into the words that
        // follow them (cells x (L + 1) always fits), lanes reading rotated words
        int32_t *fin = smem_tab;
        if (lshift > 0) {
            const int L = 1 << lshift;
            fin = smem_tab + (h.cells << lshift);
            for (int c = threadIdx.x; c < h.cells; c += blockDim.x) {
                int32_t v = 0;
                for (int j = 0; j < L; ++j) v += smem_tab[(c << lshift) + ((j + c) & (L - 1))];
                fin[c] = v;
            }
            __syncthreads();
        }
        if (in_smem) {
            for (int c = threadIdx.x; c < h.cells; c += blockDim.x) {
                int32_t v = fin[c];
                for (int j = 1; j < copies; ++j) v += fin[j * h.cells + c];
                if (copies > 1) fin[c] = v;
                if (h.nparts == 1) {
                    if (P.write_tables) P.tables[h.table_off + c] = v;
                } else if (v) {
                    atomicAdd(&P.tables[h.table_off + c], v);
                }
            }
            __syncthreads();
        } else if (windowed) {
            // a window over all rows stores its whole cell range (the table
            // lives in global memory for scores too); split rows add
            int32_t *dst = P.tables + h.table_off + w0;
            for (uint32_t c = threadIdx.x; c < wlen; c += blockDim.x) {
                const int32_t v = smem_tab[c];
                if (rparts == 1)
                    dst[c] = v;
                else if (v)
                    atomicAdd(dst + c, v);
            }
        }

        if (h.score_kind != kNoScore) {
            const int64_t *mc = P.marg + h.child_soff;
            if (h.nparts == 1 && in_smem) {
                const float s = block_score<false>(fin, h.cells, h.r_child, h.score_kind, mc, P.m, P.ess, s_red);
                if (threadIdx.x == 0) P.scores[h.score_slot] = s;
            } else {
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) s_last = atomicAdd(&P.tickets[W.q], 1) == h.nparts - 1;
                __syncthreads();
                if (s_last) {
                    __threadfence();
                    const float s = block_score<true>(P.tables + h.table_off, h.cells, h.r_child, h.score_kind,
                                                      mc, P.m, P.ess, s_red);
                    if (threadIdx.x == 0) P.scores[h.score_slot] = s;
                }
            }
        }
        __syncthreads();
    }
}

// The parent configurations of one family inside the joint table of its
// variable set: the parents are every axis but the child's; configuration j
// is decoded over them (last fastest) into a cell offset.
struct FamilyRows {
    int32_t np;
    int32_t ar[kMaxFamily];
    int64_t st[kMaxFamily];
    int64_t cstep;
    // 32-bit division: a joint table has fewer than 2^31 cells (int32 offsets).
    __device__ __forceinline__ int64_t base(int64_t j) const
    {
        uint32_t u = (uint32_t)j;
        int64_t b = 0;
        for (int t = np - 1; t >= 0; --t) {
            const uint32_t a = (uint32_t)ar[t];
            const uint32_t d = u % a;
            u /= a;
            b += (int64_t)d * st[t];
        }
        return b;
    }
    __device__ __forceinline__ int64_t step() const { return cstep; }
};

// One warp per family (child, parents): the score of the child given the
// other variables of a joint table counted once for the whole variable set
// (Sec. 4.2: every family of the parent-set lattice is a (child, rest) split
// of some variable set).
__global__ void family_score_kernel(const FamilyJob *__restrict__ jobs, int64_t njobs,
                                    const int32_t *__restrict__ tables, const int32_t *__restrict__ arity,
                                    const int32_t *__restrict__ soff, const int64_t *__restrict__ marg,
                                    int64_t m, int kind, double ess, float *scores)
{
    // one warp per job: most families' tables have a few hundred cells, so
    // a warp-level reduction replaces the block barriers
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t jb = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); jb < njobs; jb += warps) {
        const FamilyJob job = jobs[jb];
        int32_t ar[kMaxFamily];
        int64_t st[kMaxFamily];
        int64_t stride = 1;
        for (int t = job.k - 1; t >= 0; --t) {
            ar[t] = arity[job.vars[t]];
            st[t] = stride;
            stride *= ar[t];
        }
        FamilyRows rows;
        rows.np = 0;
        int64_t q = 1;
        for (int t = 0; t < job.k; ++t) {
            if (t == job.child_pos) continue;
            rows.ar[rows.np] = ar[t];
            rows.st[rows.np] = st[t];
            ++rows.np;
            q *= ar[t];
        }
        const int32_t rc = ar[job.child_pos];
        rows.cstep = st[job.child_pos];
        const BdeuK bk = warp_bdeu_consts(kind, q, rc, ess);
        ScoreAcc acc = score_rows<true>(tables + job.table_off, rows, q, rc, kind,
                                        marg + soff[job.vars[job.child_pos]], m, bk, lane, 32);
        warp_merge(acc);
        if (lane == 0) scores[job.slot] = score_finish(acc, kind, m, rc, q, bk);
    }
}

__global__ void score_global_kernel(const QHead *__restrict__ qh, const int32_t *__restrict__ q_list,
                                    const int32_t *__restrict__ tables, float *scores,
                                    const int64_t *__restrict__ marg, int64_t m, double ess)
{
    __shared__ ScoreAcc s_red[32];
    const QHead h = qh[q_list[blockIdx.x]];
    const float s = block_score<true>(tables + h.table_off, h.cells, h.r_child, h.score_kind,
                                      marg + h.child_soff, m, ess, s_red);
    if (threadIdx.x == 0) scores[h.score_slot] = s;
}

}  // namespace

const void *bitmap_kernel_ptr() { return (const void *)bitmap_kernel; }

size_t bitmap_smem_bytes(int threads, int stage_slots)
{
    return (size_t)(threads / 32) * stage_slots * 32 * sizeof(ulonglong2);
}

// CTAs of bitmap_kernel one SM holds (the dynamic shared-memory limit of the
// kernel is raised first, or the occupancy query would report none).
// The dynamic shared-memory limit a kernel was last given on each device:
// raising it is a driver call, so it is made only when a launch needs more.
namespace {
std::mutex g_attr_mu;
constexpr int kMaxDevices = 64;
int g_count_smem[kMaxDevices], g_count4_smem[kMaxDevices], g_bitmap_smem[kMaxDevices], g_wide_smem[kMaxDevices];

cudaError_t ensure_smem_attr(const void *fn, int *cache, size_t smem)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (dev >= 0 && dev < kMaxDevices && cache[dev] >= (int)smem) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && dev >= 0 && dev < kMaxDevices) cache[dev] = (int)smem;
    return e;
}

struct OccKey {
    int dev, threads, slots, per_sm;
};
OccKey g_occ[16];
int g_n_occ = 0;
}  // namespace

int bitmap_ctas_per_sm(int threads, int stage_slots)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    {
        std::lock_guard<std::mutex> lock(g_attr_mu);
        for (int i = 0; i < g_n_occ; ++i)
            if (g_occ[i].dev == dev && g_occ[i].threads == threads && g_occ[i].slots == stage_slots)
                return g_occ[i].per_sm;
    }
    const size_t smem = bitmap_smem_bytes(threads, stage_slots);
    if (ensure_smem_attr((const void *)bitmap_kernel, g_bitmap_smem, smem) != cudaSuccess) return 1;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bitmap_kernel, threads, smem) != cudaSuccess)
        return 1;
    per_sm = per_sm > 0 ? per_sm : 1;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_n_occ < 16) g_occ[g_n_occ++] = OccKey{dev, threads, stage_slots, per_sm};
    return per_sm;
}

cudaError_t launch_count(const CountParams &p, int grid, int threads, size_t smem, cudaStream_t s)
{
    if (threads > 512) return cudaErrorInvalidValue;
    if (p.D4) {
        cudaError_t e = ensure_smem_attr((const void *)count_kernel<512, 2, true>, g_count4_smem, smem);
        if (e != cudaSuccess) return e;
        count_kernel<512, 2, true><<<grid, threads, smem, s>>>(p);
        return cudaGetLastError();
    }
    cudaError_t e = ensure_smem_attr((const void *)count_kernel<512, 2>, g_count_smem, smem);
    if (e != cudaSuccess) return e;
    count_kernel<512, 2><<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_count_wide(const CountParams &p, int grid, size_t smem, cudaStream_t s)
{
    cudaError_t e = ensure_smem_attr((const void *)count_kernel<1024, 1>, g_wide_smem, smem);
    if (e != cudaSuccess) return e;
    count_kernel<1024, 1><<<grid, 1024, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_bitmap(const CountParams &p, int grid, int threads, cudaStream_t s)
{
    if (threads > 256) return cudaErrorInvalidValue;  // __launch_bounds__(256, 2)
    const size_t smem = bitmap_smem_bytes(threads, p.stage_slots);
    cudaError_t e = ensure_smem_attr((const void *)bitmap_kernel, g_bitmap_smem, smem);
    if (e != cudaSuccess) return e;
    bitmap_kernel<<<grid, threads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_family_scores(const FamilyJob *jobs, int64_t njobs, const int32_t *tables, const int32_t *arity,
                                 const int32_t *soff, const int64_t *marg, int64_t m, int kind, double ess,
                                 float *scores, int grid, cudaStream_t s)
{
    if (njobs <= 0) return cudaSuccess;
    family_score_kernel<<<grid, 128, 0, s>>>(jobs, njobs, tables, arity, soff, marg, m, kind, ess, scores);
    return cudaGetLastError();
}

cudaError_t launch_score_global(const QHead *qh, const int32_t *q_list, int32_t nlist,
                                const int32_t *tables, float *scores, const int64_t *marg,
                                int64_t m, double ess, cudaStream_t s)
{
    if (nlist <= 0) return cudaSuccess;
    score_global_kernel<<<nlist, 256, 0, s>>>(qh, q_list, tables, scores, marg, m, ess);
    return cudaGetLastError();
}

}  // namespace fc
