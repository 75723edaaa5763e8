// fc_count.cu -- the batched counting kernel.
//
// One persistent launch serves a whole batch of queries with shared context
// (Sec. 2: every count N_ijk of a variable set).  CTAs pull work items
// (query, row range) from an atomic counter; each item is counted with the
// strategy the planner chose for its query:
//
//   kBitmap  Sec. 3.2, Alg. 1.  A warp owns 4096 instances at a time (two
//            64-bit words per lane).  It walks the tree of state combinations
//            depth first; each node ANDs its parent's partial bitmap (kept in
//            registers) with the bitmap of the next variable's state and the
//            subtree is skipped when the AND is empty in every lane (zero
//            support pruning).  Leaves are popcounted, reduced over the warp
//            and added to the table in shared memory.  Variables are visited
//            in ascending entropy (Sec. 3.2).
//   kHist    the partitions of Alg. 2-3 identified by their mixed-radix key:
//            each instance's key (its cell index) is built from 16-byte
//            column loads and counted with a shared-memory atomic; tables
//            are replicated per warp group when shared memory allows.
//   kGAtomic the same keys counted straight into the table in global memory
//            (tables too large for shared memory).
//
// When a query's counts feed a score, the reduction of Sec. 3.1 (Eq. 1, Fig.
// 2) runs in the same launch: from shared memory when one item holds the
// query's whole table, else by the last CTA to finish one of the query's
// items (an atomic ticket; no CTA ever waits for another).
#include "fc_internal.h"
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

// Score of one complete table (parents-major, child-last, r child states),
// computed by the whole block; returns the value in thread 0.
//   LL  = sum N_ijk log2(N_ijk / N_ij) = -(1/ln2) sum N_ijk log1p((N_ij - N_ijk) / N_ijk):
//         every term has the same sign and the integer difference is exact.
//   MDL = -LL + (log2 m / 2)(r - 1) q.
//   BDeu: lgamma differences accumulated in FP64.
//   MI  = (1/ln2) sum_jk p_j p_k [(1 + x_jk) ln(1 + x_jk) - x_jk] over all cells
//         with p_j, p_k > 0, x_jk = (N_jk m - N_j N_k) / (N_j N_k) with an exact
//         int64 numerator; this equals the usual sum because sum p_j p_k x_jk = 0,
//         and every term is >= 0.
template <bool kGlobal>
__device__ float block_score(const int32_t *tab, int32_t cells, int32_t r, int kind,
                             const int64_t *marg_child, int64_t m, double ess, Kahan *red_k,
                             double *red_d)
{
    const int64_t q = cells / r;
    Kahan acc{0.0f, 0.0f};
    double accd = 0.0;
    const double aj = ess / (double)q, ajk = ess / ((double)r * (double)q);
    const double lg_aj = kind == kBDeu ? lgamma(aj) : 0.0;
    const double lg_ajk = kind == kBDeu ? lgamma(ajk) : 0.0;
    for (int64_t j = threadIdx.x; j < q; j += blockDim.x) {
        int64_t nij = 0;
        for (int k = 0; k < r; ++k) nij += tab_ld<kGlobal>(tab, j * r + k);
        if (nij == 0) continue;
        if (kind == kLL || kind == kMDL) {
            for (int k = 0; k < r; ++k) {
                const int32_t n = tab_ld<kGlobal>(tab, j * r + k);
                if (n > 0) kahan_add(acc, (float)n * log1pf((float)(nij - n) / (float)n));
            }
        } else if (kind == kBDeu) {
            accd += lg_aj - lgamma(aj + (double)nij);
            for (int k = 0; k < r; ++k) {
                const int32_t n = tab_ld<kGlobal>(tab, j * r + k);
                if (n > 0) accd += lgamma(ajk + (double)n) - lg_ajk;
            }
        } else {  // kMI
            const float pj = (float)nij / (float)m;
            for (int k = 0; k < r; ++k) {
                const int64_t nk = marg_child[k];
                if (nk == 0) continue;
                const int32_t n = tab_ld<kGlobal>(tab, j * r + k);
                const long long num = (long long)n * m - (long long)nij * nk;
                const float x = (float)num / ((float)nij * (float)nk);
                kahan_add(acc, pj * ((float)nk / (float)m) * mi_term(x));
            }
        }
    }
    // block reduction of (Kahan, double)
    for (int o = 16; o > 0; o >>= 1) {
        Kahan other{__shfl_xor_sync(kFull, acc.s, o), __shfl_xor_sync(kFull, acc.c, o)};
        kahan_merge(acc, other);
        accd += __shfl_xor_sync(kFull, accd, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red_k[warp] = acc;
        red_d[warp] = accd;
    }
    __syncthreads();
    float out = 0.0f;
    if (threadIdx.x == 0) {
        Kahan t{0.0f, 0.0f};
        double td = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            kahan_merge(t, red_k[w]);
            td += red_d[w];
        }
        const float sum = __fsub_rn(t.s, t.c);
        if (kind == kLL)
            out = -sum * kInvLn2;
        else if (kind == kMDL)
            out = (float)((double)sum * (double)kInvLn2 +
                          0.5 * log2((double)m) * (double)(r - 1) * (double)q);
        else if (kind == kBDeu)
            out = (float)td;
        else
            out = sum * kInvLn2;
    }
    __syncthreads();
    return out;
}

// ------------------------------------------------------------ bitmap (Alg. 1)

template <int K, int L>
struct Dfs {
    static __device__ __forceinline__ void run(const uint64_t *__restrict__ bits,
                                               int64_t wstride, const QVar *vs, int64_t w,
                                               ulonglong2 acc, int cell, int32_t *tab, int lane)
    {
        const QVar v = vs[L];
        const uint64_t *row = bits + (int64_t)v.soff * wstride + w;
        for (int s = 0; s < v.arity; ++s) {
            const ulonglong2 b = __ldg(reinterpret_cast<const ulonglong2 *>(row + (int64_t)s * wstride));
            ulonglong2 x;
            x.x = acc.x & b.x;
            x.y = acc.y & b.y;
            if constexpr (L == K - 1) {
                unsigned cnt = (unsigned)(__popcll(x.x) + __popcll(x.y));
                cnt = __reduce_add_sync(kFull, cnt);
                if (lane == 0 && cnt) atomicAdd(&tab[cell + s * v.stride], (int)cnt);
            } else {
                if (__any_sync(kFull, (x.x | x.y) != 0ull))
                    Dfs<K, L + 1>::run(bits, wstride, vs, w, x, cell + s * v.stride, tab, lane);
            }
        }
    }
};

template <int K>
__device__ __forceinline__ void bitmap_chunks(const CountParams &P, const QVar *vs, int64_t c0,
                                              int64_t c1, int32_t *tab)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const ulonglong2 all = make_ulonglong2(~0ull, ~0ull);
    for (int64_t c = c0 + warp; c < c1; c += nwarps) {
        const int64_t w = c * kChunkWords + 2 * lane;
        Dfs<K, 0>::run(P.bits, P.wstride, vs, w, all, 0, tab, lane);
    }
}

__device__ void bitmap_rows(const CountParams &P, const QVar *vs, int k, int64_t c0, int64_t c1,
                            int32_t *tab)
{
    switch (k) {
    case 1: bitmap_chunks<1>(P, vs, c0, c1, tab); break;
    case 2: bitmap_chunks<2>(P, vs, c0, c1, tab); break;
    case 3: bitmap_chunks<3>(P, vs, c0, c1, tab); break;
    case 4: bitmap_chunks<4>(P, vs, c0, c1, tab); break;
    case 5: bitmap_chunks<5>(P, vs, c0, c1, tab); break;
    case 6: bitmap_chunks<6>(P, vs, c0, c1, tab); break;
    case 7: bitmap_chunks<7>(P, vs, c0, c1, tab); break;
    case 8: bitmap_chunks<8>(P, vs, c0, c1, tab); break;
    default: break;  // the planner never sends deeper queries here
    }
}

// ---------------------------------------------------- mixed-radix key counts

__device__ __forceinline__ void add_bytes(uint32_t (&key)[16], const uint4 x, uint32_t st)
{
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) key[4 * i + j] += ((w[i] >> (8 * j)) & 0xffu) * st;
    }
}

// Keys of instances [r0, r1) counted into `tab` (shared or global memory).
// r0 is a multiple of kChunkRows, so every 16-row group is 16-byte aligned.
__device__ __forceinline__ void key_rows(const CountParams &P, const QVar *vs, int k, int64_t r0,
                                         int64_t r1, int32_t *tab)
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
            add_bytes(key, x, (uint32_t)v.stride);
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

// ------------------------------------------------------- the persistent loop

__global__ void __launch_bounds__(1024) count_kernel(const CountParams P)
{
    extern __shared__ __align__(16) int32_t smem_tab[];
    __shared__ QVar s_vars[kMaxK];
    __shared__ int s_item;
    __shared__ int s_last;
    __shared__ Kahan s_red_k[32];
    __shared__ double s_red_d[32];
    const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int64_t nchunks = (P.m + kChunkRows - 1) / kChunkRows;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(P.next_item, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= P.n_items) break;
        const Item W = P.items[it];
        const QHead h = P.qh[W.q];
        const int k = h.k;
        if (threadIdx.x < k) s_vars[threadIdx.x] = P.qv[h.var_off + threadIdx.x];
        const int64_t c0 = nchunks * W.part / h.nparts;
        const int64_t c1 = nchunks * (W.part + 1) / h.nparts;
        const int64_t r0 = c0 * kChunkRows;
        const int64_t r1 = min(P.m, c1 * kChunkRows);
        const bool in_smem = h.strategy == kHist || h.strategy == kBitmap;
        int copies = 1;
        if (h.strategy == kHist) {
            copies = min(P.hist_copies, P.smem_cells / max(h.cells, 1));
            copies = max(1, min(copies, nwarps));
        }
        if (in_smem)
            for (int c = threadIdx.x; c < h.cells * copies; c += blockDim.x) smem_tab[c] = 0;
        __syncthreads();

        if (k == 0) {
            // no variable with more than one state: the single cell counts the rows
            if (threadIdx.x == 0) {
                if (in_smem)
                    smem_tab[0] = (int32_t)(r1 - r0);
                else
                    atomicAdd(&P.tables[h.table_off], (int32_t)(r1 - r0));
            }
        } else if (h.strategy == kHist) {
            key_rows(P, s_vars, k, r0, r1, smem_tab + (warp % copies) * h.cells);
        } else if (h.strategy == kBitmap) {
            bitmap_rows(P, s_vars, k, c0, c1, smem_tab);
        } else {
            key_rows(P, s_vars, k, r0, r1, P.tables + h.table_off);
        }
        __syncthreads();

        if (in_smem) {
            for (int c = threadIdx.x; c < h.cells; c += blockDim.x) {
                int32_t v = smem_tab[c];
                for (int j = 1; j < copies; ++j) v += smem_tab[j * h.cells + c];
                if (copies > 1) smem_tab[c] = v;
                if (h.nparts == 1) {
                    if (P.write_tables) P.tables[h.table_off + c] = v;
                } else if (v) {
                    atomicAdd(&P.tables[h.table_off + c], v);
                }
            }
            __syncthreads();
        }

        if (h.score_kind != kNoScore) {
            const int64_t *mc = P.marg + h.child_soff;
            if (h.nparts == 1 && in_smem) {
                const float s = block_score<false>(smem_tab, h.cells, h.r_child, h.score_kind, mc,
                                                   P.m, P.ess, s_red_k, s_red_d);
                if (threadIdx.x == 0) P.scores[h.score_slot] = s;
            } else {
                __threadfence();
                __syncthreads();
                if (threadIdx.x == 0) s_last = atomicAdd(&P.tickets[W.q], 1) == h.nparts - 1;
                __syncthreads();
                if (s_last) {
                    __threadfence();
                    const float s = block_score<true>(P.tables + h.table_off, h.cells, h.r_child,
                                                      h.score_kind, mc, P.m, P.ess, s_red_k,
                                                      s_red_d);
                    if (threadIdx.x == 0) P.scores[h.score_slot] = s;
                }
            }
        }
        __syncthreads();
    }
}

__global__ void score_global_kernel(const QHead *__restrict__ qh, const int32_t *__restrict__ q_list,
                                    const int32_t *__restrict__ tables, float *scores,
                                    const int64_t *__restrict__ marg, int64_t m, double ess)
{
    __shared__ Kahan s_red_k[32];
    __shared__ double s_red_d[32];
    const QHead h = qh[q_list[blockIdx.x]];
    const float s = block_score<true>(tables + h.table_off, h.cells, h.r_child, h.score_kind,
                                      marg + h.child_soff, m, ess, s_red_k, s_red_d);
    if (threadIdx.x == 0) scores[h.score_slot] = s;
}

}  // namespace

int count_kernel_max_smem() { return 200 * 1024; }

cudaError_t launch_count(const CountParams &p, int grid, int threads, size_t smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    count_kernel<<<grid, threads, smem, s>>>(p);
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
