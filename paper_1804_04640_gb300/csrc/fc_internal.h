// fc_internal.h -- device descriptors and kernel launchers shared by the
// host runtime (fc_host.h and its translation units) and the kernel
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

namespace fc {

constexpr int kMaxK = 32;          // variables of one query in a device descriptor
constexpr int kMaxBitmapK = 8;     // deepest DFS the bitmap kernel is instantiated for
constexpr int kChunkRows = 4096;   // row granule of work items (64 words of 64 bits)
constexpr int kChunkWords = kChunkRows / 64;

enum Strategy : int32_t { kBitmap = 0, kHist = 1, kGAtomic = 2, kSort = 3, kMarginal = 4, kWindow = 5 };
// most cell windows of one kWindow query (its work items stay below 2^15)
constexpr int kMaxWindows = 4096;
enum ScoreKind : int32_t { kNoScore = -1, kLL = 0, kMDL = 1, kBDeu = 2, kMI = 3 };

// Status word values written by kernels (0 = fine).
enum DeviceStatus : int32_t { kStatusOk = 0, kStatusTimeout = 1, kStatusBadState = 2 };

// One query of a count or score batch.
struct QHead {
    int64_t table_off;   // first cell of this query's table in the table buffer
    int32_t cells;       // table cells
    int32_t var_off;     // first entry in the QVar array
    int16_t k;           // variables in the descriptor (arity-1 variables dropped)
    int16_t strategy;    // Strategy
    int16_t nparts;      // work items the query's rows are split into
    int16_t score_kind;  // ScoreKind
    int32_t r_child;     // arity of the child (score queries: child is the last, stride 1)
    int32_t child_soff;  // state offset of the child (marginals for MI)
    int32_t score_slot;  // index into the score output
    int32_t nwin;        // kWindow: cell windows (items = nwin x row parts), else 1
};

// One variable of a query.  stride is the variable's weight in the cell index
// of the table in the caller's variable order; soff is the first bitmap row
// (= sum of the arities of the variables before it).
struct QVar {
    int32_t var;
    int32_t stride;
    int32_t arity;
    int32_t soff;
};

struct Item {
    int32_t q;
    int32_t part;
};

// One warp task of the bitmap strategy: query q over 4096-row chunks
// [c0, c1); s0 >= 0 restricts a 3-variable register-blocked query to state
// s0 of its first variable (-1: every state).
struct BTask {
    int32_t q;
    int32_t c0, c1;
    int32_t s0;
};

struct CountParams {
    const uint8_t *D;        // n columns of m_pad bytes
    int64_t m_pad;
    const uint8_t *D4;       // the same states as 4-bit codes (m_pad / 2 bytes per column), or null
    int64_t m;
    const uint64_t *bits;    // sum(r) rows of wstride words
    int64_t wstride;
    const QHead *qh;
    const QVar *qv;
    const Item *items;
    int32_t n_items;
    const int32_t *n_items_dev;  // if set, the item count is read here (a plan built on the device)
    int32_t *next_item;      // work counter, zero before the launch
    int32_t *tables;         // table buffer (output, or plan scratch for scores)
    int32_t *tickets;        // per query, zero before the launch (nparts > 1 scoring)
    float *scores;
    const int64_t *marg;     // per-state marginal counts
    double ess;
    int32_t write_tables;    // 1: every cell is written (nparts == 1 queries store zeros too)
    int32_t smem_cells;      // int32 cells of dynamic shared memory for tables
    int32_t hist_copies;     // maximum table copies for the histogram strategy
    int32_t small_paths;     // 1: bitmap queries of 2-3 small variables skip the tree walk
    // bitmap strategy: warp-granular tasks (query, chunk range); a query's
    // tasks are consecutive and number qh[q].nparts
    const BTask *btasks;
    int32_t n_btasks;
    int32_t pad2;
    int32_t *next_task;      // warp task counter, zero before the launch
    int32_t stage_slots;     // state bitmaps a warp stages (levels 1..k-1)
};

// Launchers (each defined in the translation unit holding its kernel).
// Bitmap words [first_word, ceil(m / 64)) of every (variable, state) row,
// from the column-major D.  With delta set, delta[row] += the set bits of the
// packed words at positions >= 64 first_word + first_from (the marginal
// counts of appended instances, Sec. 6: a growing database updates the
// bitmaps in place).
cudaError_t launch_pack_bits(const uint8_t *D, int64_t m_pad, int64_t m, int32_t n,
                             const int32_t *d_arity, const int32_t *d_soff, uint64_t *bits,
                             int64_t wstride, int32_t max_arity, int32_t *bad_state,
                             cudaStream_t s, int64_t first_word = 0, int64_t *delta = nullptr,
                             int first_from = 0);
cudaError_t launch_append_bits(uint64_t *bits, int64_t wstride, int32_t n_items, int64_t m_old,
                               const uint64_t *nb, int64_t n_in, int64_t m_new, int64_t *marg, cudaStream_t s);
cudaError_t launch_bit_popcounts(const uint64_t *bits, int64_t rows, int64_t wstride,
                                 int64_t *counts, cudaStream_t s);
cudaError_t launch_transpose_rows(const uint8_t *Drow, int64_t m, int32_t n, uint8_t *Dcol,
                                  int64_t m_pad, cudaStream_t s);
// 4-bit codes of rows [row0, row1) (widened to whole 16-row groups) of the
// n columns of D (all states < 16): column i at D4 + i * m_pad / 2, rows 2b
// and 2b + 1 in the low and high nibble of byte b.
cudaError_t launch_pack_codes4(const uint8_t *D, int64_t m_pad, int32_t n, int64_t row0, int64_t row1,
                               uint8_t *D4, cudaStream_t s);
cudaError_t launch_mask_tail_bits(uint64_t *bits, int64_t rows, int64_t wstride, int64_t m,
                                  cudaStream_t s);

cudaError_t launch_count(const CountParams &p, int grid, int threads, size_t smem, cudaStream_t s);
// count_kernel with 1024 threads and one CTA per SM (windowed tables); smem
// is the window's bytes
cudaError_t launch_count_wide(const CountParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_bitmap(const CountParams &p, int grid, int threads, cudaStream_t s);
size_t bitmap_smem_bytes(int threads, int stage_slots);
int bitmap_ctas_per_sm(int threads, int stage_slots);
const void *bitmap_kernel_ptr();

// Sort + run-length path for one query (large tables).
struct SortScratch {
    uint32_t *keys_a;
    uint32_t *keys_b;
    uint32_t *block_hist;    // 256 x nblocks
    int64_t cap_rows;
    int32_t cap_blocks;
};
int sort_tile_rows();
cudaError_t launch_sort_count(const uint8_t *D, int64_t m_pad, int64_t m, const QVar *d_vars,
                              int32_t k, int32_t key_bits, int32_t *table, int32_t cells,
                              int32_t zero_table, SortScratch sc, cudaStream_t s);

// One family (child, parents) scored from the joint table of its variable
// set: vars in the table's order (last fastest), child at child_pos.
constexpr int kMaxFamily = 8;
struct FamilyJob {
    int64_t table_off;
    int32_t slot;
    int16_t k;
    int16_t child_pos;
    int32_t vars[kMaxFamily];
};
cudaError_t launch_family_scores(const FamilyJob *jobs, int64_t njobs, const int32_t *tables, const int32_t *arity,
                                 const int32_t *soff, const int64_t *marg, int64_t m, int kind, double ess,
                                 float *scores, int grid, cudaStream_t s);

// Scores of queries whose tables are complete in global memory.
cudaError_t launch_score_global(const QHead *qh, const int32_t *q_list, int32_t nlist,
                                const int32_t *tables, float *scores, const int64_t *marg,
                                int64_t m, double ess, cudaStream_t s);

// Specific-assignment count: AND of k bitmap rows, popcount.
cudaError_t launch_assignment_count(const uint64_t *bits, int64_t wstride, const int32_t *d_rows,
                                    int32_t k, int64_t words, unsigned long long *out,
                                    cudaStream_t s);

// Itemset supports (binary transaction bitmaps).
struct SupportParams {
    const uint64_t *bits;    // n_items rows of wstride words
    int64_t wstride;
    int64_t words;           // ceil(m / 64)
    const int32_t *set_off;  // nq + 1
    const int32_t *items;
    const int32_t *order;    // itemsets in processing order (grouped by size)
    int32_t nq;
    int32_t n_items;
    int32_t *support;
    int32_t *sub_support;
    float *confidence;
    int32_t *next_item;      // work counter
    int32_t words_per_part;  // word range of one work item
    int32_t nparts;
    int32_t sets_per_item;   // itemsets one CTA takes per work item
    int32_t full_only;       // 1: only supp(S) (assignment counts), no leave-one-out sets
    int64_t m_tail;          // m: bits at positions >= m are not transactions
    // all-splits mode: sub_support / confidence hold 2^k - 2 entries per
    // itemset from split_off[q], antecedent masks 1 .. 2^k - 2 in order
    const int64_t *split_off;
    int32_t all_splits;
    int32_t pad;
    // marginal count of every item (one-item subsets are not counted by the
    // kernels: the finishing pass copies these)
    const int64_t *marg;
};
constexpr int kMaxSplitK = 16;  // itemset size limit of the all-splits mode
cudaError_t launch_support(const SupportParams &p, int grid, int threads, size_t smem,
                           cudaStream_t s);
cudaError_t launch_support_confidence(const SupportParams &p, cudaStream_t s);
// 0 leave-one-out, 1 full only, 2 all splits (the instantiation that runs
// `threads` threads per CTA)
const void *support_kernel_ptr(int mode, int threads);

// All-pairs one-hot co-occurrence on tcgen05 tensor cores.
//
// One 256 x 256 region of C on or above its diagonal: rows ra*256.. (the A
// operand, two halves of 128 rows, one accumulator each) against columns
// rb*256.. (the B operand).  Only the cells on or above the diagonal of C and
// inside the R x R matrix are needed, so each accumulator multiplies only the
// columns it needs: n0 / n1 columns (multiples of 16, 0 = skipped), the
// second half starting coff1 columns into B (128 on the diagonal, whose
// lower-left quarter lies below the diagonal).  Its rows are split over
// ksplit CTAs from cta0 on.
struct PairsRegion {
    int32_t ra, rb;
    int32_t n0, n1, coff1;
    int32_t real_b;      // B rows inside the R x R matrix (the rest are zero)
    int32_t cta0, ksplit;
};

struct PairsParams {
    const uint64_t *bits;    // R rows of wstride words (one row per (variable, state))
    int64_t wstride;
    int64_t words;           // ceil(m / 64)
    int32_t R;               // sum of arities
    int32_t R_pad;           // padded to the tile size
    int32_t *C;              // R_pad x R_pad int32 co-occurrence (upper tiles), zeroed
    int32_t chunk_words;     // words accumulated in FP32 before the move to int32
    int32_t nregions;
    const PairsRegion *regions;  // device array, cta0 ascending
    int32_t grid;            // CTAs of the launch (sum of the regions' ksplit)
    int32_t *status;
    int64_t wait_limit;
};
cudaError_t launch_pairs_gemm(const PairsParams &p, cudaStream_t s);
cudaError_t launch_pairs_extract(const int32_t *C, int32_t R_pad, int32_t n, const int32_t *d_arity,
                                 const int32_t *d_soff, const int64_t *d_pair_off, int64_t m,
                                 int32_t *pair_tables, float *mi, cudaStream_t s);

cudaError_t launch_wait_selftest(int32_t *status, int64_t wait_limit, cudaStream_t s);

// Records the thread-local message returned by fc_last_error(); returns code.
int set_error(int code, const char *fmt, ...);

}  // namespace fc

// ---- items of a context, for the rule miner (fc_rules.cu)
struct fc_ctx;
namespace fc {
// The context's host worker threads (started on first use): how many can run
// at once (the caller counts as one), and f(0..n-1) run on them, f(0) on the
// caller; returns when all are done.  n must not exceed host_threads(c).
int host_threads(fc_ctx *c);
void run_host_threads(fc_ctx *c, int n, const std::function<void(int)> &f);
// Number of items (bitmap rows) of a context and its instance count m.
void itemset_universe(const fc_ctx *c, int32_t *n_items, int64_t *m);
// For each item: the variable it belongs to (an item of a categorical context
// is one state of a variable; a transaction item is its own group) and its
// support (the popcount of its bitmap).  Arrays of n_items entries.
void item_groups(const fc_ctx *c, int32_t *group, int64_t *support);
// Totals of count_itemsets calls: descriptor bytes uploaded, count bytes read
// back, and device time of the counting launches (CUDA events around them).
struct ItemsetCountStats {
    int64_t h2d_bytes = 0, d2h_bytes = 0;
    double device_ms = 0.0;
};
// Support of each of nq itemsets (lists of item ids in `rows`, CSR offsets
// `set_off` with set_off[0] == 0, ids already validated), counted on the
// device; int32 results in the host array `counts`.  `st` may be NULL.
int count_itemsets(fc_ctx *c, int32_t nq, const int32_t *set_off, const int32_t *rows, int32_t *counts,
                   ItemsetCountStats *st);
}  // namespace fc
