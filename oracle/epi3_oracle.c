/*
 * epi3 CPU oracle -- TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.
 *
 * A plain, slow, obviously correct FP64 statement of what the three-way
 * epistasis scan computes.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header, table
 * or constant with the CUDA library, and the library never calls it.
 *
 * What it follows (arXiv 2201.10956):
 *   - Sec. III: a case-control data set of M SNPs x N samples, genotype values
 *     0/1/2 per (SNP, sample), phenotype 0 = control, 1 = case.  Genotypes are
 *     read SNP-major, geno[m * N + s].
 *   - Sec. III, Fig. 1: the 27 x 2 frequency table of a SNP triplet (X, Y, Z)
 *     counts, per phenotype class, the samples showing each genotype
 *     combination.  Cell index = 9 * gX + 3 * gY + gZ (the gX, gY, gZ loop
 *     order of Algorithms 1 and 2).  Counting here is one sample at a time
 *     from the raw genotype bytes: no bit planes, no NOR trick, no blocking.
 *   - Eq. 1: K2 = sum over cells i of ( sum_{b=1}^{r_i + 1} log b
 *                                       - sum_{j=0,1} sum_{d=1}^{r_ij} log d ).
 *     The inner sums are sums of log over 1..n taken in increasing order; they
 *     are memoised in lf[n] = lf[n-1] + log(n), lf[0] = 0, which performs the
 *     very same additions in the very same order.  Natural log.  The cell
 *     term is evaluated as (lf[r_i + 1] - lf[r_i0]) - lf[r_i1] and the terms
 *     are added to a running sum starting at 0.0 in cell order 0..26.
 *   - Sec. III: the solution is the triplet of lowest K2.  Generalised to the
 *     k best under the total order (K2 ascending, then i, j, k ascending).
 *
 *   - Eq. 1 is stated for any number of interacting SNPs; for two SNPs
 *     (x, y) the table has 3^2 = 9 cells per class, cell = 3 * gX + gY, and
 *     the same K2 in cell order 0..8 (the pairwise, second-order scan).
 *
 * Pins (tests/test_oracle_pins.py): brute-force numpy counting, table
 * invariants, exact K2 from big-integer factorials, hand-worked values,
 * symmetries, degenerate inputs and planted-triplet recovery; the pairwise
 * functions also against the triplet functions on a monomorphic third SNP.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NCELL 27

/* lf[n] for n = 0..n_max: the sum of log(b) for b = 1..n, added in order. */
int oracle_log_factorials(int32_t n_max, double* lf) {
    if (n_max < 0 || !lf) return -1;
    lf[0] = 0.0;
    for (int32_t n = 1; n <= n_max; ++n) lf[n] = lf[n - 1] + log((double)n);
    return 0;
}

/* Frequency table of SNPs (x, y, z) for all samples; ft[c * 27 + cell]. */
static int count_one(const uint8_t* geno, const uint8_t* pheno, int64_t n_samples,
                     int64_t x, int64_t y, int64_t z, int32_t* ft) {
    memset(ft, 0, sizeof(int32_t) * 2 * NCELL);
    const uint8_t* gx = geno + x * n_samples;
    const uint8_t* gy = geno + y * n_samples;
    const uint8_t* gz = geno + z * n_samples;
    for (int64_t s = 0; s < n_samples; ++s) {
        int c = pheno[s];
        int a = gx[s], b = gy[s], d = gz[s];
        if (c > 1 || a > 2 || b > 2 || d > 2) return -1;
        ft[c * NCELL + 9 * a + 3 * b + d] += 1;
    }
    return 0;
}

/* K2 of one 2 x 27 table (Eq. 1) from an lf table that covers every r + 1. */
static double k2_of_table(const int32_t* ft, const double* lf) {
    double k2 = 0.0;
    for (int cell = 0; cell < NCELL; ++cell) {
        int32_t r0 = ft[cell], r1 = ft[NCELL + cell];
        double term = (lf[r0 + r1 + 1] - lf[r0]) - lf[r1];
        k2 = k2 + term;
    }
    return k2;
}

/* Tables of n triplets (any three distinct SNP indices, in the given order).
 * out: [n][2][27] int32.  Returns 0, or -1 on a bad index or value. */
int oracle_tables(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                  int64_t n_samples, int64_t n, const int32_t* trip, int32_t* out) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        int32_t x = trip[3 * t], y = trip[3 * t + 1], z = trip[3 * t + 2];
        if (x < 0 || y < 0 || z < 0 || x >= n_snps || y >= n_snps || z >= n_snps) {
            bad = 1;
            continue;
        }
        if (count_one(geno, pheno, n_samples, x, y, z, out + t * 2 * NCELL)) bad = 1;
    }
    return bad ? -1 : 0;
}

/* K2 of n given tables [n][2][27]; out[n]. */
int oracle_k2(int64_t n, const int32_t* tables, double* out) {
    int64_t rmax = 0;
    for (int64_t t = 0; t < n; ++t)
        for (int cell = 0; cell < NCELL; ++cell) {
            int64_t r0 = tables[t * 2 * NCELL + cell], r1 = tables[t * 2 * NCELL + NCELL + cell];
            if (r0 < 0 || r1 < 0) return -1;
            if (r0 + r1 > rmax) rmax = r0 + r1;
        }
    double* lf = (double*)malloc(sizeof(double) * (size_t)(rmax + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(rmax + 1), lf);
    for (int64_t t = 0; t < n; ++t) out[t] = k2_of_table(tables + t * 2 * NCELL, lf);
    free(lf);
    return 0;
}

/* Table + K2 for n triplets; out_k2[n]. */
int oracle_scores(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                  int64_t n_samples, int64_t n, const int32_t* trip, double* out_k2,
                  int32_t n_threads) {
    double* lf = (double*)malloc(sizeof(double) * (size_t)(n_samples + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(n_samples + 1), lf);
    int bad = 0;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        int32_t ft[2 * NCELL];
        int32_t x = trip[3 * t], y = trip[3 * t + 1], z = trip[3 * t + 2];
        if (x < 0 || y < 0 || z < 0 || x >= n_snps || y >= n_snps || z >= n_snps ||
            count_one(geno, pheno, n_samples, x, y, z, ft)) {
            bad = 1;
            out_k2[t] = NAN;
            continue;
        }
        out_k2[t] = k2_of_table(ft, lf);
    }
    free(lf);
    return bad ? -1 : 0;
}

typedef struct {
    double k2;
    int32_t i, j, k;
} entry;

/* Total order of the answer: K2 ascending, then i, j, k ascending. */
static int before(const entry* a, const entry* b) {
    if (a->k2 != b->k2) return a->k2 < b->k2;
    if (a->i != b->i) return a->i < b->i;
    if (a->j != b->j) return a->j < b->j;
    return a->k < b->k;
}

static int cmp_entry(const void* pa, const void* pb) {
    const entry* a = (const entry*)pa;
    const entry* b = (const entry*)pb;
    if (before(a, b)) return -1;
    if (before(b, a)) return 1;
    return 0;
}

/* Keep the `cap` first entries of a list kept in order (plain insertion). */
static void keep_best(entry* list, int32_t* len, int32_t cap, const entry* e) {
    int32_t n = *len;
    if (n == cap && !before(e, &list[n - 1])) return;
    int32_t pos = (n == cap) ? n - 1 : n;
    while (pos > 0 && before(e, &list[pos - 1])) {
        list[pos] = list[pos - 1];
        --pos;
    }
    list[pos] = *e;
    if (n < cap) *len = n + 1;
}

/* Exhaustive scan over every i < j < k: the top_k triplets by (K2, i, j, k).
 * out_trip [top_k][3], out_k2 [top_k].  n_threads <= 0: OpenMP default.
 * Returns the number of threads used (> 0) or a negative error. */
int oracle_scan_topk(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                     int64_t n_samples, int32_t top_k, int32_t* out_trip, double* out_k2,
                     int32_t n_threads) {
    int64_t m = n_snps;
    if (m < 3 || top_k < 1 || top_k > m * (m - 1) * (m - 2) / 6) return -1;
    double* lf = (double*)malloc(sizeof(double) * (size_t)(n_samples + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(n_samples + 1), lf);
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    entry* lists = (entry*)malloc(sizeof(entry) * (size_t)top_k * nt);
    int32_t* lens = (int32_t*)calloc((size_t)nt, sizeof(int32_t));
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        entry* mine = lists + (size_t)tid * top_k;
#pragma omp for schedule(dynamic, 1)
        for (int32_t i = 0; i < n_snps; ++i)
            for (int32_t j = i + 1; j < n_snps; ++j)
                for (int32_t k = j + 1; k < n_snps; ++k) {
                    int32_t ft[2 * NCELL];
                    if (count_one(geno, pheno, n_samples, i, j, k, ft)) {
                        bad = 1;
                        continue;
                    }
                    entry e = {k2_of_table(ft, lf), i, j, k};
                    keep_best(mine, &lens[tid], top_k, &e);
                }
    }
    int32_t total = 0;
    for (int t = 0; t < nt; ++t) {
        memmove(lists + total, lists + (size_t)t * top_k, sizeof(entry) * lens[t]);
        total += lens[t];
    }
    qsort(lists, (size_t)total, sizeof(entry), cmp_entry);
    for (int32_t r = 0; r < top_k && r < total; ++r) {
        out_trip[3 * r] = lists[r].i;
        out_trip[3 * r + 1] = lists[r].j;
        out_trip[3 * r + 2] = lists[r].k;
        out_k2[r] = lists[r].k2;
    }
    free(lists);
    free(lens);
    free(lf);
    return bad ? -1 : nt;
}

/* ---------------------------------------------------------------- pairs */
#define NPCELL 9

/* Frequency table of SNPs (x, y); ft[c * 9 + 3 * gX + gY]. */
static int count_pair(const uint8_t* geno, const uint8_t* pheno, int64_t n_samples, int64_t x,
                      int64_t y, int32_t* ft) {
    memset(ft, 0, sizeof(int32_t) * 2 * NPCELL);
    const uint8_t* gx = geno + x * n_samples;
    const uint8_t* gy = geno + y * n_samples;
    for (int64_t s = 0; s < n_samples; ++s) {
        int c = pheno[s];
        int a = gx[s], b = gy[s];
        if (c > 1 || a > 2 || b > 2) return -1;
        ft[c * NPCELL + 3 * a + b] += 1;
    }
    return 0;
}

/* K2 of one 2 x 9 table, cell order 0..8, as k2_of_table. */
static double k2_of_pair(const int32_t* ft, const double* lf) {
    double k2 = 0.0;
    for (int cell = 0; cell < NPCELL; ++cell) {
        int32_t r0 = ft[cell], r1 = ft[NPCELL + cell];
        double term = (lf[r0 + r1 + 1] - lf[r0]) - lf[r1];
        k2 = k2 + term;
    }
    return k2;
}

/* Tables of n pairs (two distinct SNP indices, in the given order): out [n][2][9]. */
int oracle_pair_tables(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                       int64_t n_samples, int64_t n, const int32_t* pairs, int32_t* out) {
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        int32_t x = pairs[2 * t], y = pairs[2 * t + 1];
        if (x < 0 || y < 0 || x >= n_snps || y >= n_snps) {
            bad = 1;
            continue;
        }
        if (count_pair(geno, pheno, n_samples, x, y, out + t * 2 * NPCELL)) bad = 1;
    }
    return bad ? -1 : 0;
}

/* Exhaustive pairwise scan over every i < j: the top_k pairs by (K2, i, j).
 * out_pairs [top_k][2], out_k2 [top_k].  Returns threads used (> 0) or a negative error. */
int oracle_scan_pairs_topk(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                           int64_t n_samples, int32_t top_k, int32_t* out_pairs, double* out_k2,
                           int32_t n_threads) {
    int64_t m = n_snps;
    if (m < 2 || top_k < 1 || top_k > m * (m - 1) / 2) return -1;
    double* lf = (double*)malloc(sizeof(double) * (size_t)(n_samples + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(n_samples + 1), lf);
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    entry* lists = (entry*)malloc(sizeof(entry) * (size_t)top_k * nt);
    int32_t* lens = (int32_t*)calloc((size_t)nt, sizeof(int32_t));
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        entry* mine = lists + (size_t)tid * top_k;
#pragma omp for schedule(dynamic, 1)
        for (int32_t i = 0; i < n_snps; ++i)
            for (int32_t j = i + 1; j < n_snps; ++j) {
                int32_t ft[2 * NPCELL];
                if (count_pair(geno, pheno, n_samples, i, j, ft)) {
                    bad = 1;
                    continue;
                }
                entry e = {k2_of_pair(ft, lf), i, j, 0};
                keep_best(mine, &lens[tid], top_k, &e);
            }
    }
    int32_t total = 0;
    for (int t = 0; t < nt; ++t) {
        memmove(lists + total, lists + (size_t)t * top_k, sizeof(entry) * lens[t]);
        total += lens[t];
    }
    qsort(lists, (size_t)total, sizeof(entry), cmp_entry);
    for (int32_t r = 0; r < top_k && r < total; ++r) {
        out_pairs[2 * r] = lists[r].i;
        out_pairs[2 * r + 1] = lists[r].j;
        out_k2[r] = lists[r].k2;
    }
    free(lists);
    free(lens);
    free(lf);
    return bad ? -1 : nt;
}

/* ---------------------------------------------------------------- any order
 * Eq. 1 is stated for an interaction of any number of SNPs.  For `order` SNPs
 * (x_0, ..., x_{order-1}) the table has 3^order cells per class; the cell of a
 * sample is its genotypes read as base-3 digits, the first SNP most significant
 * (cell = 9 gX + 3 gY + gZ for three SNPs, 3 gX + gY for two).  K2 is summed in
 * cell order exactly as for the triplet.  order = 1 .. ORACLE_MAX_ORDER. */
#define ORACLE_MAX_ORDER 6

static int32_t cells_of(int32_t order) {
    int32_t n = 1;
    for (int32_t t = 0; t < order; ++t) n *= 3;
    return n;
}

/* Frequency table of the SNPs snps[0..order); ft[c * 3^order + cell]. */
static int count_order(const uint8_t* geno, const uint8_t* pheno, int64_t n_samples,
                       int32_t order, const int32_t* snps, int32_t* ft) {
    const int32_t ncell = cells_of(order);
    memset(ft, 0, sizeof(int32_t) * 2 * (size_t)ncell);
    for (int64_t s = 0; s < n_samples; ++s) {
        int c = pheno[s];
        if (c > 1) return -1;
        int32_t cell = 0;
        for (int32_t t = 0; t < order; ++t) {
            int g = geno[(int64_t)snps[t] * n_samples + s];
            if (g > 2) return -1;
            cell = 3 * cell + g;
        }
        ft[c * ncell + cell] += 1;
    }
    return 0;
}

/* K2 of one 2 x ncell table, cell order 0..ncell-1, as k2_of_table. */
static double k2_of_cells(const int32_t* ft, int32_t ncell, const double* lf) {
    double k2 = 0.0;
    for (int32_t cell = 0; cell < ncell; ++cell) {
        int32_t r0 = ft[cell], r1 = ft[ncell + cell];
        double term = (lf[r0 + r1 + 1] - lf[r0]) - lf[r1];
        k2 = k2 + term;
    }
    return k2;
}

/* Tables of n SNP sets of the given order (distinct indices, in the given roles):
 * snps [n][order], out [n][2][3^order].  Returns 0, or -1 on a bad order, index or value. */
int oracle_tables_order(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                        int64_t n_samples, int32_t order, int64_t n, const int32_t* snps,
                        int32_t* out) {
    if (order < 1 || order > ORACLE_MAX_ORDER) return -1;
    const int32_t ncell = cells_of(order);
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
    for (int64_t t = 0; t < n; ++t) {
        const int32_t* x = snps + t * order;
        for (int32_t q = 0; q < order; ++q)
            if (x[q] < 0 || x[q] >= n_snps) bad = 1;
        if (bad) continue;
        if (count_order(geno, pheno, n_samples, order, x, out + t * 2 * ncell)) bad = 1;
    }
    return bad ? -1 : 0;
}

/* K2 of n tables [n][2][ncell]; out[n]. */
int oracle_k2_cells(int64_t n, int32_t ncell, const int32_t* tables, double* out) {
    int64_t rmax = 0;
    for (int64_t t = 0; t < n; ++t)
        for (int32_t cell = 0; cell < ncell; ++cell) {
            int64_t r0 = tables[t * 2 * ncell + cell], r1 = tables[t * 2 * ncell + ncell + cell];
            if (r0 < 0 || r1 < 0) return -1;
            if (r0 + r1 > rmax) rmax = r0 + r1;
        }
    double* lf = (double*)malloc(sizeof(double) * (size_t)(rmax + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(rmax + 1), lf);
    for (int64_t t = 0; t < n; ++t) out[t] = k2_of_cells(tables + t * 2 * ncell, ncell, lf);
    free(lf);
    return 0;
}

typedef struct {
    double k2;
    int32_t x[ORACLE_MAX_ORDER];
} entry_o;

/* Total order: K2 ascending, then the SNP indices lexicographically. */
static int before_o(const entry_o* a, const entry_o* b, int32_t order) {
    if (a->k2 != b->k2) return a->k2 < b->k2;
    for (int32_t t = 0; t < order; ++t)
        if (a->x[t] != b->x[t]) return a->x[t] < b->x[t];
    return 0;
}

static void keep_best_o(entry_o* list, int32_t* len, int32_t cap, const entry_o* e, int32_t order) {
    int32_t n = *len;
    if (n == cap && !before_o(e, &list[n - 1], order)) return;
    int32_t pos = (n == cap) ? n - 1 : n;
    while (pos > 0 && before_o(e, &list[pos - 1], order)) {
        list[pos] = list[pos - 1];
        --pos;
    }
    list[pos] = *e;
    if (n < cap) *len = n + 1;
}

/* Exhaustive scan over every SNP set x_0 < x_1 < ... < x_{order-1}: the top_k sets by
 * (K2, x_0, x_1, ...).  out_snps [top_k][order], out_k2 [top_k].  Returns the number of
 * threads used (> 0) or a negative error. */
int oracle_scan_order_topk(const uint8_t* geno, const uint8_t* pheno, int32_t n_snps,
                           int64_t n_samples, int32_t order, int32_t top_k, int32_t* out_snps,
                           double* out_k2, int32_t n_threads) {
    if (order < 1 || order > ORACLE_MAX_ORDER || n_snps < order || top_k < 1) return -1;
    double total_sets = 1.0;
    for (int32_t t = 0; t < order; ++t) total_sets = total_sets * (double)(n_snps - t) / (double)(t + 1);
    if ((double)top_k > total_sets + 0.5) return -1;
    const int32_t ncell = cells_of(order);
    double* lf = (double*)malloc(sizeof(double) * (size_t)(n_samples + 2));
    if (!lf) return -2;
    oracle_log_factorials((int32_t)(n_samples + 1), lf);
    int nt = 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
    nt = omp_get_max_threads();
#endif
    entry_o* lists = (entry_o*)malloc(sizeof(entry_o) * (size_t)top_k * nt);
    int32_t* lens = (int32_t*)calloc((size_t)nt, sizeof(int32_t));
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        entry_o* mine = lists + (size_t)tid * top_k;
        int32_t* ft = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)ncell);
#pragma omp for schedule(dynamic, 1)
        for (int32_t first = 0; first < n_snps; ++first) {
            /* every increasing completion x_1 < ... < x_{order-1} of x_0 = first */
            int32_t x[ORACLE_MAX_ORDER];
            x[0] = first;
            int32_t depth = 1;
            if (order > 1) x[1] = first;
            while (depth > 0) {
                if (depth == order) {
                    if (count_order(geno, pheno, n_samples, order, x, ft)) {
                        bad = 1;
                    } else {
                        entry_o e;
                        e.k2 = k2_of_cells(ft, ncell, lf);
                        for (int32_t t = 0; t < order; ++t) e.x[t] = x[t];
                        keep_best_o(mine, &lens[tid], top_k, &e, order);
                    }
                    --depth;
                    continue;
                }
                /* next candidate at position depth (depth >= 1 here) */
                ++x[depth];
                if (x[depth] > n_snps - (order - depth)) {
                    --depth;
                    continue;
                }
                ++depth;
                if (depth < order) x[depth] = x[depth - 1];
            }
        }
        free(ft);
    }
    int32_t total = 0;
    for (int t = 0; t < nt; ++t) {
        memmove(lists + total, lists + (size_t)t * top_k, sizeof(entry_o) * lens[t]);
        total += lens[t];
    }
    /* plain insertion sort of the merged lists (at most top_k * threads entries) */
    for (int32_t a = 1; a < total; ++a) {
        entry_o e = lists[a];
        int32_t p = a;
        while (p > 0 && before_o(&e, &lists[p - 1], order)) {
            lists[p] = lists[p - 1];
            --p;
        }
        lists[p] = e;
    }
    for (int32_t r = 0; r < top_k && r < total; ++r) {
        for (int32_t t = 0; t < order; ++t) out_snps[r * order + t] = lists[r].x[t];
        out_k2[r] = lists[r].k2;
    }
    free(lists);
    free(lens);
    free(lf);
    return bad ? -1 : nt;
}
