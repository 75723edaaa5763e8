/*
 * fc_oracle.c -- plain, slow, obviously correct CPU oracle for counting
 * queries and the scores computed from their counts.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this code.  The library itself
 * never calls it, and it shares no code, header or table with the CUDA path.
 *
 * Everything here follows the plain definitions of the paper
 * ("Fast Counting in Machine Learning Applications", Karan et al., UAI 2018):
 *   - a database D of n categorical variables, m complete instances (Sec. 2);
 *     this oracle reads its own row-major copy: row p holds the n states of
 *     instance p, states 0-based (the paper numbers them 1..r_i);
 *   - the contingency table of a variable list is built by scanning the
 *     database row by row into a dense lookup table (Sec. 2, the "directly
 *     scan D" approach), with the last listed variable varying fastest;
 *   - scores are aggregations over the stream of non-zero counts N_ijk with
 *     their N_ij (Sec. 2 Eq. 1, Sec. 3.1), computed in double precision.
 *
 * None of the counting strategies of Sec. 3 (bitmaps, radix partitions) are
 * used: their results must equal these plain definitions exactly.
 *
 * Return codes: 0 on success, -1 bad argument, -2 a state outside its arity,
 * -3 the table would be too large.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Number of cells of the table over vars[0..k-1]: prod of arities (Sec. 2,
 * q_i * r_i for a parent set plus child).  Returns -1 on overflow. */
static int64_t orc_cells(const int32_t *arities, int32_t n, const int32_t *vars, int32_t k)
{
    int64_t cells = 1;
    for (int32_t t = 0; t < k; ++t) {
        if (vars[t] < 0 || vars[t] >= n) return -1;
        cells *= arities[vars[t]];
        if (cells > ((int64_t)1 << 40)) return -1;
    }
    return cells;
}

/* Dense contingency table over vars[0..k-1] (Sec. 2): for every instance p,
 * the cell of its joint assignment is incremented.  Cell index of assignment
 * (s_0, ..., s_{k-1}) is ((s_0 * r_1 + s_1) * r_2 + ...) * r_{k-1} + s_{k-1}.
 * table must hold prod(r) int64 cells; it is overwritten. */
int orc_table(const uint8_t *Drow, int64_t m, int32_t n, const int32_t *arities,
              const int32_t *vars, int32_t k, int64_t *table)
{
    if (!Drow || !arities || (k > 0 && !vars) || !table || m < 0 || n <= 0 || k < 0)
        return -1;
    for (int32_t a = 0; a < k; ++a)
        for (int32_t b = a + 1; b < k; ++b)
            if (vars[a] == vars[b]) return -1;
    int64_t cells = orc_cells(arities, n, vars, k);
    if (cells < 0) return -3;
    memset(table, 0, (size_t)cells * sizeof(int64_t));
    for (int64_t p = 0; p < m; ++p) {
        const uint8_t *row = Drow + p * (int64_t)n;
        int64_t idx = 0;
        for (int32_t t = 0; t < k; ++t) {
            int32_t s = row[vars[t]];
            if (s >= arities[vars[t]]) return -2;
            idx = idx * arities[vars[t]] + s;
        }
        table[idx] += 1;
    }
    return 0;
}

/* Count((X_v0 = s0) and (X_v1 = s1) and ...): the size of the support of one
 * assignment (Sec. 2), by checking every instance. */
int64_t orc_count_assignment(const uint8_t *Drow, int64_t m, int32_t n,
                             const int32_t *vars, const int32_t *states, int32_t k)
{
    if (!Drow || m < 0 || n <= 0 || k < 0) return -1;
    int64_t count = 0;
    for (int64_t p = 0; p < m; ++p) {
        const uint8_t *row = Drow + p * (int64_t)n;
        int match = 1;
        for (int32_t t = 0; t < k; ++t) {
            if (vars[t] < 0 || vars[t] >= n) return -1;
            if (row[vars[t]] != states[t]) match = 0;
        }
        count += match;
    }
    return count;
}

/* The tables below are laid out parents-major, child-last: q rows (parent
 * configurations j) of r cells (child states k), so N_ijk = table[j*r + k]
 * and N_ij = sum_k N_ijk (Sec. 2, Eq. 1). */
static int64_t row_total(const int64_t *table, int64_t j, int32_t r)
{
    int64_t s = 0;
    for (int32_t k = 0; k < r; ++k) s += table[j * r + k];
    return s;
}

/* Log-likelihood, Eq. 1 with the base-2 logarithm used by the function object
 * of Fig. 2: sum over non-zero N_ijk of N_ijk * log2(N_ijk / N_ij). */
double orc_ll(const int64_t *table, int64_t q, int32_t r)
{
    double ll = 0.0;
    for (int64_t j = 0; j < q; ++j) {
        int64_t nij = row_total(table, j, r);
        for (int32_t k = 0; k < r; ++k) {
            int64_t nijk = table[j * r + k];
            if (nijk > 0) ll += (double)nijk * log2((double)nijk / (double)nij);
        }
    }
    return ll;
}

/* MDL cost (Sec. 4.2 names MDL after Schwarz; the paper gives no formula).
 * Reading used: -LL + (log2 m / 2) * (r - 1) * q, with q the number of all
 * parent configurations (1 for an empty parent set).  Lower is better. */
double orc_mdl(const int64_t *table, int64_t q, int32_t r, int64_t m)
{
    return -orc_ll(table, q, r) + 0.5 * log2((double)m) * (double)(r - 1) * (double)q;
}

/* BDeu log marginal likelihood (Sec. 3.1 and 4.2 name Dirichlet-prior scores
 * with products of gamma functions; the paper gives no formula).  Reading
 * used, natural logarithm, equivalent sample size ess:
 *   a_j = ess / q, a_jk = ess / (r q),
 *   sum over j with N_ij > 0 of lgamma(a_j) - lgamma(a_j + N_ij)
 * + sum over N_ijk > 0 of lgamma(a_jk + N_ijk) - lgamma(a_jk).
 * Unobserved configurations contribute exactly zero. */
double orc_bdeu(const int64_t *table, int64_t q, int32_t r, double ess)
{
    double aj = ess / (double)q;
    double ajk = ess / ((double)r * (double)q);
    double s = 0.0;
    for (int64_t j = 0; j < q; ++j) {
        int64_t nij = row_total(table, j, r);
        if (nij > 0) s += lgamma(aj) - lgamma(aj + (double)nij);
        for (int32_t k = 0; k < r; ++k) {
            int64_t nijk = table[j * r + k];
            if (nijk > 0) s += lgamma(ajk + (double)nijk) - lgamma(ajk);
        }
    }
    return s;
}

/* Mutual information (Sec. 1 names it for constraint tests; no formula is
 * given).  Reading used, in bits, between the child X (columns) and the joint
 * parent configuration Y (rows):
 *   sum over N_jk > 0 of (N_jk / m) * log2(N_jk * m / (N_j * N_k)). */
double orc_mi(const int64_t *table, int64_t q, int32_t r)
{
    int64_t m = 0;
    for (int64_t c = 0; c < q * r; ++c) m += table[c];
    if (m == 0) return 0.0;
    int64_t *col = (int64_t *)calloc((size_t)r, sizeof(int64_t));
    if (!col) return NAN;
    for (int64_t j = 0; j < q; ++j)
        for (int32_t k = 0; k < r; ++k) col[k] += table[j * r + k];
    double mi = 0.0;
    for (int64_t j = 0; j < q; ++j) {
        int64_t nj = row_total(table, j, r);
        for (int32_t k = 0; k < r; ++k) {
            int64_t njk = table[j * r + k];
            if (njk > 0)
                mi += ((double)njk / (double)m) *
                      log2(((double)njk * (double)m) / ((double)nj * (double)col[k]));
        }
    }
    free(col);
    return mi;
}

/* Transaction p holds item i when bit p % 64 of word p / 64 of item i's bitmap
 * is set (the input format of the transaction data). */
static int holds(const uint64_t *bitmaps, int64_t words, int32_t item, int64_t p)
{
    return (int)((bitmaps[(int64_t)item * words + p / 64] >> (p % 64)) & 1u);
}

/* Support of an itemset (Sec. 4.3): the number of transactions that hold every
 * item of the set, skipping position `skip` of the list (-1 skips nothing). */
static int64_t support_skip(const uint64_t *bitmaps, int64_t words, int64_t m,
                            const int32_t *items, int32_t k, int32_t skip)
{
    int64_t count = 0;
    for (int64_t p = 0; p < m; ++p) {
        int all = 1;
        for (int32_t t = 0; t < k; ++t)
            if (t != skip && !holds(bitmaps, words, items[t], p)) all = 0;
        count += all;
    }
    return count;
}

/* Rules with a single-item consequent (Sec. 4.3: rules Pa => X_i, support =
 * how often Pa and X_i are set together, confidence = how often the rule
 * holds).  For an itemset S of k items: supp[0] = supp(S); for each position t,
 * sub[t] = supp(S without item t) and conf[t] = supp(S) / sub[t], the
 * confidence of (S without item t) => item t, or 0 when sub[t] = 0. */
int orc_support_rules(const uint64_t *bitmaps, int64_t words, int64_t m, int32_t n_items,
                      const int32_t *items, int32_t k, int64_t *supp, int64_t *sub,
                      double *conf)
{
    if (!bitmaps || !items || !supp || k < 0 || m < 0 || words * 64 < m) return -1;
    for (int32_t t = 0; t < k; ++t)
        if (items[t] < 0 || items[t] >= n_items) return -1;
    supp[0] = support_skip(bitmaps, words, m, items, k, -1);
    for (int32_t t = 0; t < k; ++t) {
        sub[t] = support_skip(bitmaps, words, m, items, k, t);
        conf[t] = sub[t] > 0 ? (double)supp[0] / (double)sub[t] : 0.0;
    }
    return 0;
}

/* Every split of an itemset S of k items into a non-empty antecedent A and a
 * non-empty consequent S \ A (Sec. 4.3: rules A => S \ A with support
 * supp(S) and confidence supp(S) / supp(A)).  Antecedents are numbered by
 * their bit mask over the positions of `items` (bit t = item t in A),
 * mask = 1 .. 2^k - 2; for each, sub[mask - 1] = supp(A) counted by scanning
 * the transactions, and conf[mask - 1] = supp(S) / supp(A), 0 when supp(A)
 * = 0.  supp[0] = supp(S).  k <= 20. */
int orc_support_splits(const uint64_t *bitmaps, int64_t words, int64_t m, int32_t n_items,
                       const int32_t *items, int32_t k, int64_t *supp, int64_t *sub, double *conf)
{
    if (!bitmaps || !supp || k < 0 || k > 20 || m < 0 || words * 64 < m || (k > 0 && !items)) return -1;
    for (int32_t t = 0; t < k; ++t)
        if (items[t] < 0 || items[t] >= n_items) return -1;
    supp[0] = support_skip(bitmaps, words, m, items, k, -1);
    const int64_t full = ((int64_t)1 << k) - 1;
    for (int64_t mask = 1; mask < full; ++mask) {
        int64_t count = 0;
        for (int64_t p = 0; p < m; ++p) {
            int all = 1;
            for (int32_t t = 0; t < k && all; ++t)
                if (((mask >> t) & 1) && !holds(bitmaps, words, items[t], p)) all = 0;
            count += all;
        }
        sub[mask - 1] = count;
        conf[mask - 1] = count > 0 ? (double)supp[0] / (double)count : 0.0;
    }
    return 0;
}
