/*
 * fc.h -- C ABI of libfc, exact counting queries over a complete categorical
 * database on one GB300 GPU (sm_103a).
 *
 * The operations follow "Fast Counting in Machine Learning Applications"
 * (Karan, Eichhorn, Hurlburt, Iraci, Zola; UAI 2018):
 *   - database D of n categorical variables X_i with arity r_i and m complete
 *     instances (Sec. 2);
 *   - counting query Count((X_a = x_a) and ...) and queries with shared
 *     context, which produce every count N_ijk of a variable set (Sec. 2, 3.1);
 *   - reduction of the counts by an associative, commutative operator such
 *     as the log-likelihood of Eq. 1 (Sec. 3.1, Fig. 2);
 *   - support and confidence of association rules over binary transaction
 *     data (Sec. 4.3).
 *
 * Conventions (all calls):
 *   - States are stored 0-based, one uint8 per value, so r_i <= 255 (the paper
 *     numbers states 1..r_i).
 *   - A table over the ordered variable list (v_0, ..., v_{k-1}) is a dense
 *     int32 array of prod(r_{v_t}) cells, row-major with the LAST variable
 *     varying fastest: cell((s_0..s_{k-1})) = ((s_0 r_1 + s_1) r_2 + ...) + s_{k-1}.
 *     For a (child, parents) query the list is (parents..., child), so the
 *     q_i parent configurations are rows j and the r_i child states are
 *     columns k: N_ijk = table[j * r_i + k] (Eq. 1's indexing).
 *   - Counts are exact int32; m must be < 2^31.  A table may hold at most
 *     2^31 - 1 cells.
 *   - Unless stated otherwise pointers are HOST pointers, calls are
 *     synchronous and the caller keeps ownership of every buffer it passes.
 *   - Every call returns FC_OK (0) or a negative FC_ERR_* code and then sets a
 *     thread-local message readable with fc_last_error().  On error no output
 *     is written, except the output buffers of batch calls, whose contents
 *     are then unspecified.
 *   - A context is used by one host thread at a time.
 */
#ifndef FC_H
#define FC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FC_OK = 0,
    FC_ERR_ARG = -1,      /* null pointer, bad size, variable out of range, duplicate variable */
    FC_ERR_RANGE = -2,    /* a stored state is >= its arity; m out of range */
    FC_ERR_SIZE = -3,     /* a table or an output is too large */
    FC_ERR_OOM = -4,      /* device or host allocation failed */
    FC_ERR_CUDA = -5,     /* a CUDA runtime call failed */
    FC_ERR_TIMEOUT = -6,  /* a bounded device-side wait ran out; the context stays usable */
    FC_ERR_STATE = -7     /* call does not apply to this context or plan */
};

enum { FC_COL_MAJOR = 0, FC_ROW_MAJOR = 1 };   /* layout of D in fc_load */
enum { FC_HOST = 0, FC_DEVICE = 1 };           /* where an input pointer lives */

/* Score kinds for fc_score_batch.  All scores reduce the stream of non-zero
 * counts (N_ijk, N_ij) of one (child, parents) query (Sec. 3.1).
 *   FC_LL   Eq. 1 with log base 2 (Fig. 2): sum N_ijk log2(N_ijk / N_ij).
 *   FC_MDL  -LL + (log2 m / 2) (r_i - 1) q_i, q_i = prod of parent arities
 *           (Sec. 4.2 names MDL; this is the reading the library implements).
 *   FC_BDEU sum_j [lgamma(a_j) - lgamma(a_j + N_ij)]
 *           + sum_jk [lgamma(a_jk + N_ijk) - lgamma(a_jk)], a_j = ess / q_i,
 *           a_jk = ess / (r_i q_i), natural log, sums over non-zero counts
 *           (Sec. 3.1 and 4.2 name the Dirichlet-prior score).
 *   FC_MI   mutual information in bits between the child and the joint
 *           parent configuration (Sec. 1 names MI). */
enum { FC_LL = 0, FC_MDL = 1, FC_BDEU = 2, FC_MI = 3 };

/* Counting strategies (option "strategy"; FC_STRAT_AUTO lets the planner
 * choose per query). */
enum {
    FC_STRAT_AUTO = -1,
    FC_STRAT_BITMAP = 0,  /* Sec. 3.2, Alg. 1: AND + popcount DFS over per-state bitmaps */
    FC_STRAT_HIST = 1,    /* mixed-radix key per instance into a shared-memory table (Sec. 3.3's partitions as keys) */
    FC_STRAT_GATOMIC = 2, /* mixed-radix key into the output table in global memory */
    FC_STRAT_SORT = 3,    /* mixed-radix key, device radix sort, run-length (Sec. 3.3: partitions are runs of equal keys) */
    FC_STRAT_MARGINAL = 4, /* one variable: the per-state counts precomputed at load (Sec. 3.3, precomputed
                              single-variable partitions); chosen automatically, never forced */
    FC_STRAT_WINDOW = 5   /* tables beyond shared memory: the cell range cut into windows that fit, each
                             counted in shared memory over all instances (Sec. 3.3's partitions grouped by
                             their leading digits) */
};

typedef struct fc_ctx fc_ctx;
typedef struct fc_plan fc_plan;

/* ---------------------------------------------------------------- loading */

/* Load a complete categorical database (Sec. 2) onto the current CUDA device.
 *   D       n * m uint8 states, 0-based.  layout FC_COL_MAJOR: D[i * m + p] is
 *           X_i in instance p (the paper's column D_i); FC_ROW_MAJOR:
 *           D[p * n + i].  `where` says whether D is a host or a device pointer.
 *   arities n int32 values in 1..255 (host).
 * The context copies D (the caller keeps ownership), builds per-variable
 * per-state bitmaps of m bits (Sec. 3.2, Fig. 1a), per-state marginal counts
 * and per-variable entropies (used to order the DFS of Alg. 1).
 * Errors: FC_ERR_ARG (null, n < 1, m < 1, arity outside 1..255),
 * FC_ERR_RANGE (m >= 2^31, or a state >= its arity), FC_ERR_OOM, FC_ERR_CUDA. */
int fc_load(fc_ctx **out, const uint8_t *D, int32_t n, int64_t m, const int32_t *arities,
            int32_t layout, int32_t where);

/* Load binary transaction data for association-rule queries (Sec. 4.3).
 *   bitmaps n_items rows of ceil(m / 64) uint64 words; bit p % 64 of word
 *           p / 64 of row i is set when transaction p holds item i.
 * Bits at positions >= m are ignored.  Only fc_support_batch,
 * fc_plan_support, fc_mine_rules and fc_append_bits apply to such a context.
 * Errors: FC_ERR_ARG, FC_ERR_RANGE (m >= 2^31), FC_ERR_OOM, FC_ERR_CUDA. */
int fc_load_bits(fc_ctx **out, const uint64_t *bitmaps, int32_t n_items, int64_t m, int32_t where);

/* Release a context and all device memory it owns.  Plans made from it and
 * not yet freed lose their device memory and can then only be passed to
 * fc_plan_free (fc_plan_run returns FC_ERR_STATE).  Null is ignored. */
void fc_free(fc_ctx *ctx);

/* Basic facts about a context: key 0 = n (variables or items), 1 = m,
 * 2 = sum of arities, 3 = device ordinal, 4 = instances that fit without
 * reallocating (see fc_reserve), 5 = appends so far, 6 = bits per value of
 * the columns the shared-memory histogram strategy reads (4 with the 4-bit
 * copy of option "codes4", else 8; 0 for a context from fc_load_bits),
 * 7 = 1 when the last fc_count_batch was planned on the device (only its
 * query lists, offsets and the entropies were uploaded), else 0.
 * -1 for a bad key. */
int64_t fc_info(const fc_ctx *ctx, int32_t key);

/* ---------------------------------------------------- growing a database
 *
 * Sec. 6: when the database grows by new instances, the bitmaps take a
 * simple update and the radix/histogram strategies read D as it stands.  An
 * append copies the new instances behind the old ones, repacks only the
 * bitmap words from the old m / 64 on, adds the new instances' state counts
 * to the marginals and refreshes the entropies, so every later query, score
 * and plan sees the m + m_new instances, with results identical to loading
 * the concatenated database at once.
 *
 * Plans built before an append refuse to run (FC_ERR_STATE): build new ones.
 * Storage keeps spare rows and grows by at least half when full (the old
 * contents are copied; the call then synchronises the context's stream);
 * fc_reserve sets the room up front.  The appended instances must not make
 * m reach 2^31 (FC_ERR_RANGE).  Calls on one context must not overlap. */

/* Append m_new instances of a categorical context: D as for fc_load (layout
 * FC_COL_MAJOR = n x m_new, FC_ROW_MAJOR = m_new x n; where FC_HOST or
 * FC_DEVICE; the caller keeps ownership).  A state >= its variable's arity
 * appends nothing and returns FC_ERR_RANGE.  m_new = 0 is a no-op. */
int fc_append(fc_ctx *ctx, const uint8_t *D, int64_t m_new, int32_t layout, int32_t where);

/* Append m_new transactions to a context from fc_load_bits: bitmaps are
 * n_items rows of ceil(m_new / 64) uint64 words, bit p of word w of row i set
 * when new transaction 64 w + p holds item i; bits past m_new are ignored. */
int fc_append_bits(fc_ctx *ctx, const uint64_t *bitmaps, int64_t m_new, int32_t where);

/* Make room for m_total instances (no effect when there is room already). */
int fc_reserve(fc_ctx *ctx, int64_t m_total);

/* Per-state marginal counts: out[state_offset(i) + s] = Count(X_i = s), with
 * state_offset(i) = sum of the arities of X_0..X_{i-1} (host buffer of
 * fc_info(ctx, 2) int64). */
int fc_marginals(const fc_ctx *ctx, int64_t *out);

/* ------------------------------------------------------- counting queries */

/* Full contingency table of one variable list (Sec. 2: all counts of the
 * query with shared context over vars[0..k-1]).
 *   vars   k distinct variable ids (k = 0 gives the single cell m).
 *   table  prod(r_{vars[t]}) int32 cells, layout as described above.
 * Errors: FC_ERR_ARG (bad or duplicate variable), FC_ERR_SIZE, FC_ERR_STATE,
 * FC_ERR_CUDA, FC_ERR_TIMEOUT. */
int fc_count(fc_ctx *ctx, const int32_t *vars, int32_t k, int32_t *table);

/* Count of one assignment, Count((X_vars[0] = states[0]) and ...) (Sec. 2 and
 * the specific-assignment variant at the end of Sec. 3.3).  *count receives
 * the number of instances that match every condition.  A state outside its
 * variable's arity matches nothing (count 0). */
int fc_count_assignment(fc_ctx *ctx, const int32_t *vars, const int32_t *states, int32_t k,
                        int64_t *count);

/* Counts of nq specific assignments in one launch (Sec. 2, Count of one
 * assignment; the single root-to-leaf path of the bitmap DFS, end of
 * Sec. 3.3: the AND of one state bitmap per condition, then a bit count).
 * Assignment q is the conditions (vars[t] = states[t]) for t in
 * var_off[q] .. var_off[q+1) (var_off[0] = 0).  counts: nq int64 (host).  A
 * state outside its arity makes the count 0; no conditions give m; a variable
 * listed twice with two states gives 0. */
int fc_count_assignment_batch(fc_ctx *ctx, int32_t nq, const int32_t *var_off, const int32_t *vars,
                              const int32_t *states, int64_t *counts);

/* Batch of nq tables.  Query q has variables
 * vars[var_off[q] .. var_off[q+1]) and its table starts at cell table_off[q]
 * of `tables`; table_off is non-decreasing with
 * table_off[q+1] - table_off[q] >= cells of query q.  Pass table_off = NULL
 * to pack the tables back to back in query order.  A batch of 4096 queries
 * or more runs in two parts: the second part is planned while the first
 * one's kernels run, and each part's tables are copied back while the GPU
 * goes on (a bad query in the second part is reported after the first part
 * ran); batches whose queries all count in shared memory are planned on the
 * device instead (option "device_plan").  `tables` is best in pinned memory
 * (cudaHostAlloc): the copies can overlap it, and a part whose kernels store
 * every cell of its tables (no cell accumulated; option "zero_copy") writes
 * it directly, with no copy.
 * Cells between tables (when table_off leaves gaps) are unspecified after
 * the call. */
int fc_count_batch(fc_ctx *ctx, int32_t nq, const int32_t *var_off, const int32_t *vars,
                   const int64_t *table_off, int32_t *tables);

/* Scores of nq (child, parents) queries (Sec. 3.1, Eq. 1; kinds above);
 * batches of 4096 or more run in two parts as in fc_count_batch.
 * Query q scores child[q] given parents[par_off[q] .. par_off[q+1]); the
 * child must not be among its parents.  ess is the BDeu equivalent sample
 * size (ignored by the other kinds).  scores: nq float (FP32 result with
 * cancellation-free FP32 terms; BDeu's per-query constants, and its terms
 * for priors of 1 or more, in FP64). */
int fc_score_batch(fc_ctx *ctx, int32_t nq, const int32_t *child, const int32_t *par_off,
                   const int32_t *parents, int32_t kind, double ess, float *scores);

/* Scores of every family of the parent-set lattice over a variable list
 * (Sec. 4.2: for each child X, every parent set Pa of at most max_parents of
 * the other listed variables).  Each variable set V = Pa + {X} is counted
 * once as a joint table and serves all |V| families that split it, so the
 * counting work is that of the distinct variable sets.
 *   vars    nv distinct variable ids; d = min(max_parents, nv - 1) <= 7.
 *   scores  nv * F floats, F = sum_{s=0..d} C(nv-1, s).  The score of child
 *           vars[c] with parents P is at c * F + (number of parent sets
 *           smaller than |P|) + the lexicographic rank of P's positions among
 *           the other nv - 1 variables (in list order).
 * kind and ess as in fc_score_batch.  fc_families_count(nv, max_parents)
 * returns nv * F (or -1 for bad arguments). */
int64_t fc_families_count(int32_t nv, int32_t max_parents);
int fc_score_families(fc_ctx *ctx, int32_t nv, const int32_t *vars, int32_t max_parents, int32_t kind,
                      double ess, float *scores);

/* All pairwise tables and their mutual information (the one-hot
 * co-occurrence product: for variables a < b the table over (a, b) is one
 * block of A^T A, A the m x sum(r) one-hot matrix of D; each table is the
 * Sec. 2 table of the pair).
 *   pair_tables  NULL, or the tables of all pairs a < b in lexicographic order,
 *                packed back to back (r_a * r_b cells each, b fastest).
 *   mi           NULL, or n(n-1)/2 floats, MI in bits of each pair.
 * Errors: FC_ERR_STATE for a transaction context, FC_ERR_SIZE. */
int fc_pairs_all(fc_ctx *ctx, int32_t *pair_tables, float *mi);

/* Number of int32 cells fc_pairs_all writes to pair_tables. */
int64_t fc_pairs_cells(const fc_ctx *ctx);

/* Support and rule confidence of nq itemsets (Sec. 4.3; specific-assignment
 * queries with every item in state 1).  Itemset q is
 * items[set_off[q] .. set_off[q+1]) (distinct items).  Outputs:
 *   support[q]               supp(S), the transactions holding every item;
 *   sub_support[set_off[q]+t] supp(S without its t-th item);
 *   confidence[set_off[q]+t]  supp(S) / supp(S without item t), the confidence
 *                            of (S without item t) => item t; 0 when the
 *                            denominator is 0.
 * sub_support and confidence may be NULL.  Applies to fc_load_bits contexts. */
int fc_support_batch(fc_ctx *ctx, int32_t nq, const int32_t *set_off, const int32_t *items,
                     int32_t *support, int32_t *sub_support, float *confidence);

/* Every split of each itemset into antecedent A and consequent S \ A
 * (Sec. 4.3, rules A => S \ A): for itemset q of k items (k <= 16),
 * sub_support and confidence hold 2^k - 2 entries starting at
 * sum over earlier itemsets of (2^k' - 2) (none for k <= 1), one per
 * antecedent mask 1 .. 2^k - 2 in increasing order (bit t = item t of the
 * itemset's list is in A): sub_support = supp(A), confidence =
 * supp(S) / supp(A) (0 when supp(A) = 0).  support[q] = supp(S).  Host
 * buffers; sub_support and confidence may be NULL.  Applies to fc_load_bits
 * contexts.  Errors as fc_support_batch, FC_ERR_SIZE for k > 16. */
int fc_support_splits_batch(fc_ctx *ctx, int32_t nq, const int32_t *set_off, const int32_t *items,
                            int32_t *support, int32_t *sub_support, float *confidence);

/* ----------------------------------------------- association-rule mining
 *
 * Bottom-up search of the itemset lattice (Sec. 4.3): level 1 is every item,
 * level k every k-itemset whose (k-1)-subsets are all frequent; each level's
 * candidates are counted in one batched device launch (specific-assignment
 * counts, end of Sec. 3.3), the frequent ones kept, and the search stops at
 * max_size items or at an empty level.
 *
 * Items: for a context from fc_load_bits, item i is transaction bitmap i; for
 * a categorical context, item soff(v) + s is the event D[v] == s, where soff(v)
 * is the sum of the arities of variables 0..v-1 (two states of one variable
 * never form an itemset).
 *
 * Thresholds (strict, as the paper states them, decided in double precision):
 *   S is frequent     when supp(S) > min_support * m;
 *   rule A => S \ A   is kept when supp(S) > min_confidence * supp(A),
 * for frequent S of at least 2 items and A a non-empty proper subset of S:
 * every such A when all_splits = 1 (2^k - 2 rules per k-itemset), else only
 * the A that leave one item as consequent (rules Pa(X) => X).
 * min_support in [0, 1], min_confidence >= 0, max_size in [1, 32] (at most 16
 * with all_splits).
 *
 * The result is host memory owned by the returned handle: read it with
 * fc_rules_size / fc_rules_itemsets / fc_rules_list, release it with
 * fc_rules_free.  Errors: FC_ERR_ARG (bad threshold or size), FC_ERR_SIZE
 * (more than 2^31 - 1 candidates on one level), FC_ERR_CUDA, FC_ERR_OOM. */
typedef struct fc_rules fc_rules;
int fc_mine_rules(fc_ctx *ctx, double min_support, double min_confidence, int32_t max_size,
                  int32_t all_splits, fc_rules **out);

/* key 0 = frequent itemsets, 1 = items over all of them, 2 = rules,
 * 3 = candidate itemsets counted on the device, 4 = levels counted on the
 * device, 5 = descriptor bytes copied host to device, 6 = count bytes copied
 * device to host, 7 = nanoseconds of device time in the counting launches
 * (CUDA events around each level's launch), 8 = items over the candidates
 * (bitmap rows the counting launches read).  -1 for a bad key. */
int64_t fc_rules_size(const fc_rules *rules, int32_t key);

/* Frequent itemsets, size by size and lexicographic within a size, each in
 * increasing item order: set_off (count + 1 int32, CSR offsets into items),
 * items (int32) and support (int64).  Host buffers sized by fc_rules_size;
 * any may be NULL. */
int fc_rules_itemsets(const fc_rules *rules, int32_t *set_off, int32_t *items, int64_t *support);

/* Rules in itemset order, then by antecedent mask: itemset (int64 index into
 * the itemset list), antecedent (bit t set when item t of the itemset is in
 * A; the consequent is the rest) and confidence supp(S) / supp(A) (float,
 * the double quotient rounded once).  Host buffers; any may be NULL. */
int fc_rules_list(const fc_rules *rules, int64_t *itemset, uint32_t *antecedent, float *confidence);

void fc_rules_free(fc_rules *rules);

/* ------------------------------------------- plans: device-resident batches
 *
 * A plan validates a batch once, picks a strategy per query, uploads the
 * descriptors and keeps its scratch; fc_plan_run then executes the whole
 * batch as one graph launch on a stream, reading only device memory.  Plans
 * are how a caller keeps inputs and outputs resident in HBM. */

/* Plan of a count batch (arguments as fc_count_batch, table_off may be NULL). */
int fc_plan_count(fc_ctx *ctx, int32_t nq, const int32_t *var_off, const int32_t *vars,
                  const int64_t *table_off, fc_plan **out);

/* Plan of a score batch (arguments as fc_score_batch). */
int fc_plan_score(fc_ctx *ctx, int32_t nq, const int32_t *child, const int32_t *par_off,
                  const int32_t *parents, int32_t kind, double ess, fc_plan **out);

/* Plan of a support batch (arguments as fc_support_batch). */
int fc_plan_support(fc_ctx *ctx, int32_t nq, const int32_t *set_off, const int32_t *items,
                    fc_plan **out);

/* Plan of an all-splits support batch (arguments as fc_support_splits_batch);
 * fc_plan_run takes the outputs of a support plan, fc_plan_size(plan, 3) is
 * the number of split entries. */
int fc_plan_support_splits(fc_ctx *ctx, int32_t nq, const int32_t *set_off, const int32_t *items,
                           fc_plan **out);

/* Plan of an assignment-count batch (arguments as fc_count_assignment_batch);
 * fc_plan_run writes nq int32 counts to out0. */
int fc_plan_assignments(fc_ctx *ctx, int32_t nq, const int32_t *var_off, const int32_t *vars,
                        const int32_t *states, fc_plan **out);

/* Plan of the family scores (arguments as fc_score_families); fc_plan_run
 * writes the nv * F scores to out0 (float, device). */
int fc_plan_families(fc_ctx *ctx, int32_t nv, const int32_t *vars, int32_t max_parents, int32_t kind,
                     double ess, fc_plan **out);

/* Plan of the all-pairs computation (fc_pairs_all). */
int fc_plan_pairs(fc_ctx *ctx, fc_plan **out);

/* Sizes of a plan's outputs: key 0 = int32 cells of the table output (count and
 * pairs plans), 1 = float scores / MI values / family scores, 2 = int32 supports, 3 = entries of
 * sub_support / confidence, 4 = number of queries, 5 = bytes of descriptors the
 * plan copied to the device, 6 = kernels one fc_plan_run launches with every
 * output given.  Returns -1 for a bad key. */
int64_t fc_plan_size(const fc_plan *plan, int32_t key);

/* Table offsets chosen by a count plan (nq + 1 int64, host buffer). */
int fc_plan_table_offsets(const fc_plan *plan, int64_t *table_off);

/* Strategy the plan chose for each query (nq int32, FC_STRAT_* values). */
int fc_plan_strategies(const fc_plan *plan, int32_t *strategy);

/* Run a plan asynchronously on `stream` (a cudaStream_t; NULL = the context's
 * own stream).  Outputs are DEVICE pointers on the context's device:
 *   count plan:   out0 = tables (int32);
 *   score plan:   out0 = scores (float);
 *   pairs plan:   out0 = pair tables (int32, may be NULL), out1 = MI (float, may be NULL);
 *   support plan: out0 = support, out1 = sub_support (may be NULL),
 *                 out2 = confidence (float, may be NULL);
 *   assignment plan: out0 = counts (int32);
 *   families plan: out0 = scores (float).
 * The first run with a given (outputs, stream) captures a CUDA graph; later
 * runs replay it.  Runs of one plan must not overlap in time.  Device-side
 * errors (FC_ERR_TIMEOUT) are reported by fc_sync(). */
int fc_plan_run(fc_plan *plan, void *out0, void *out1, void *out2, void *stream);

/* Release a plan (waits for its runs to finish). */
void fc_plan_free(fc_plan *plan);

/* Wait for the context's stream, and `stream` when not NULL, then report and
 * clear the device status word: FC_OK or FC_ERR_TIMEOUT. */
int fc_sync(fc_ctx *ctx, void *stream);

/* ------------------------------------------------------- options, errors */

/* Set a tuning option; returns FC_ERR_ARG for an unknown key or bad value.
 *   "strategy"          FC_STRAT_* forced for every query (default AUTO;
 *                       FC_STRAT_MARGINAL cannot be forced)
 *   "shape_auto"        1 = the planner picks the count kernel's launch shape
 *                       per batch (default): 256 threads x 8192-cell tables,
 *                       or the three options below when more than 1/64 of the
 *                       batch are shared-memory tables beyond 8192 cells or
 *                       when, with m >= 2^19, most histogram work is on tables
 *                       of 256 cells or more.  Setting any of the three sets
 *                       it to 0.
 *   "smem_cells"        int32 cells of the shared-memory table area per CTA
 *   "threads"           threads per CTA of the count kernel (multiple of 32, <= 512)
 *   "ctas_per_sm"       resident CTAs per SM the count kernel is sized for
 *   "hist_copies"       max copies of a shared-memory table (contention)
 *   "min_part_rows"     smallest row range one work item covers
 *   "pair_chunk_rows"   rows accumulated in FP32 tensor memory before the
 *                       all-pairs kernel moves the counts to int32
 *   "use_graph"         1 = capture plan runs in CUDA graphs (default), 0 = plain launches
 *   "wait_limit"        iteration limit of every device-side wait
 *   "window_max"        most cell windows AUTO gives one query before it
 *                       counts the table in global memory instead
 *   "window_cells"      cap on the cells of one window (default: as many as
 *                       the shared memory of an SM holds)
 *   "window_wide"       1 = windows run in their own launch of one 1024-thread
 *                       CTA per SM (default), 0 = inside the mixed launch
 *   "bitmap_threads"    threads per CTA of the bitmap kernel (<= 256)
 *   "stage_slots"       bitmap rows a warp of the bitmap kernel stages per chunk
 *   "bitmap_small"      1 = register-blocked bitmap path for 2-3 small variables
 *   "sort_min_cells"    tables at least this large take the sort strategy
 *   "bitmap_cost", "bitmap_chunk_cost", "small_cost", "small3_cost", "hist_cost_row",
 *   "hist_cost_var", "flush_cost"
 *                       cost-model coefficients (femtoseconds) used by AUTO
 *   "support_warps", "support_sets_per_warp", "support_part_words"
 *                       launch shape of the itemset-support kernels
 *   "zero_copy"         1 (default) = when the output buffer of fc_count,
 *                       fc_count_batch or fc_score_batch (or every output
 *                       buffer fc_pairs_all is given) is page-locked host
 *                       memory (cudaHostAlloc, or cudaHostRegister with
 *                       mapping) and no output cell is accumulated, the
 *                       kernels store the outputs into it directly instead
 *                       of into a device buffer that is copied afterwards;
 *                       0 = always copy
 *   "device_plan"       1 (default) = an fc_count_batch of 4096 queries or
 *                       more whose queries all count in shared memory (on a
 *                       database of fewer than 2^19 instances) is planned on
 *                       the device (validation, strategy, work order); any
 *                       other batch, or an invalid one, is planned on the
 *                       host, which reports the error; 0 = always the host.
 *   "codes4"            1 (default) = on a database whose arities are all at
 *                       most 16, fc_load keeps a second copy of the columns
 *                       at 4 bits per value (n x m / 2 bytes more device
 *                       memory, skipped when that allocation fails) and the
 *                       shared-memory histogram strategy reads it (half the
 *                       column bytes); 0 = read the byte columns.  Counts
 *                       are the same either way. */
int fc_set_option(fc_ctx *ctx, const char *key, int64_t value);

/* Current value of an option (or -1 for an unknown key). */
int64_t fc_get_option(const fc_ctx *ctx, const char *key);

/* Time each strategy on sample queries over the loaded data and set the
 * cost-model coefficients that FC_STRAT_AUTO uses.  `budget_ms` bounds the
 * time spent (0 = default).  Results are kept in the context. */
int fc_autotune(fc_ctx *ctx, int32_t budget_ms);

/* Tune the strategy thresholds for one count batch (arguments as
 * fc_count_batch): fc_autotune's fit, then the batch itself timed under a few
 * scalings of the bitmap cost (and with the bitmap strategy off); the fastest
 * setting stays in the context for later plans. */
int fc_autotune_batch(fc_ctx *ctx, int32_t nq, const int32_t *var_off, const int32_t *vars);

/* Message of the last error on this host thread ("" if none). */
const char *fc_last_error(void);

/* Run a device wait that nothing will satisfy, bounded by `wait_limit`
 * iterations, and return the status it leaves (FC_ERR_TIMEOUT expected).
 * Exercises the bounded-wait error path without faulting the GPU. */
int fc_selftest_wait_timeout(fc_ctx *ctx, int64_t wait_limit);

/* ------------------------------------------------- throughput probes
 *
 * The paper has no counterpart to this call: it measures the rates of the
 * on-chip units that bound the counting kernels on databases that stay in L2,
 * the denominators of their rooflines (HBM bandwidth bounds none of them
 * there).  Each probe runs one kernel that does nothing but the measured
 * operation, with every lane busy, on the current device:
 *   FC_PROBE_L2_READ      16-byte loads that bypass L1 over a `size`-byte
 *                         buffer (a power of two from 1 MiB to 64 MiB) that
 *                         stays in L2: bytes/s.  The histogram strategy reads
 *                         its columns this way (Sec. 3.3's partition pass).
 *   FC_PROBE_SMEM_ATOMIC  conflict-free atomicAdd(+1) to shared memory, every
 *                         lane of a warp on its own bank: atomics/s.  The
 *                         histogram strategy issues one per instance.
 *   FC_PROBE_AND_POPC     c += popcount(a & b) on 64-bit words held in
 *                         registers: words/s.  The bitmap strategy (Sec. 3.2)
 *                         and itemset supports (Sec. 4.3) do one per word of
 *                         every intersection.
 * `size` is ignored by the last two.  The call allocates a small buffer (and
 * the probe buffer), launches one untimed and five timed kernels on `stream`
 * (NULL = legacy default stream), waits for them and writes the best rate to
 * *rate.  Errors: FC_ERR_ARG (unknown kind, bad size, null rate), FC_ERR_OOM,
 * FC_ERR_CUDA. */
enum { FC_PROBE_L2_READ = 0, FC_PROBE_SMEM_ATOMIC = 1, FC_PROBE_AND_POPC = 2 };
int fc_probe_rate(int32_t kind, int64_t size, double *rate, void *stream);

/* ------------------------------------------------- allocation-free variant
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot let a library allocate device memory: code recording a CUDA graph
 * under a global-mode stream capture (where cudaMalloc is refused), programs
 * whose device memory is owned by their own pool allocator, and
 * latency-critical paths that cannot afford the device synchronisation that
 * cudaMalloc and cudaFree may cause.
 *
 * One contingency table, counted by the sort + run-length strategy
 * (FC_STRAT_SORT), without any context and without allocating.  Its scratch
 * (key buffers and radix-sort histograms) is a fixed 8.25 MiB array compiled
 * into the library, which every GPU that loads the library keeps until the
 * process exits.
 *   D       DEVICE pointer, column-major: state of X_i in instance p at
 *           D[i * ld + p], 0-based.  An instance with a state outside its
 *           variable's arity is not counted.
 *   n, m    variables and instances; m must be at most 2^20 (1,048,576),
 *           larger m returns FC_ERR_SIZE.  ld >= m.
 *   arities n HOST int32 values in 1..255; vars: k HOST int32 distinct ids.
 *   table   DEVICE pointer to prod(r_{vars[t]}) int32 cells, layout as in
 *           fc_count; it is zeroed and then filled on `stream`.
 *   stream  cudaStream_t the work is enqueued on (NULL = the legacy default
 *           stream).  The call returns once the work is enqueued.
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current) and keeps it for the life of
 * the process; make that first call before any stream capture begins, and do
 * not use the call across a cudaDeviceReset (the kept address would be
 * stale).  D may be NULL when m is 0; the table is then all zeros.  All calls share the one scratch array and it
 * keeps the last call's contents, so calls whose work overlaps on the GPU
 * (other streams, other host threads) race and give wrong counts: serialise
 * them.  No call allocates or frees memory.
 * Errors: FC_ERR_ARG, FC_ERR_SIZE, FC_ERR_CUDA. */
int fc_count_sorted_noalloc(const uint8_t *D, int32_t n, int64_t m, int64_t ld,
                            const int32_t *arities, const int32_t *vars, int32_t k,
                            int32_t *table, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FC_H */
