/* Row-parallel generator of planted-partition graphs.
 *
 * Input generation only: this file holds none of the community integration
 * arithmetic.  Both the oracle and the CUDA path take the graphs it builds.
 *
 * Node ids are in block order: community c occupies [off[c], off[c+1]), the
 * nodes from off[m] to n belong to no community.  An unordered pair {i, j} of
 * one community is linked iff
 *
 *     mix(seed + (min(i,j) * n + max(i,j) + 1) * 0x9E3779B97F4A7C15) < thr,
 *
 * with mix the SplitMix64 output function (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) and
 * thr = floor(p_in * 2^64) (every pair when `all` is set, for p_in = 1): a
 * Bernoulli(p_in) draw per pair that any row can evaluate on its own,
 * symmetric by construction.  Inter-community links are
 * given as a symmetric CSR (inter_rowptr, inter_col, columns ascending and
 * outside the row's community); each output row is the inter links below the
 * community's range, then the present intra links, then the inter links above
 * it, so rows come out sorted.
 */
#include <stdint.h>

static inline uint64_t syn_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline int syn_linked(uint64_t seed, uint64_t thr, int all, uint64_t n, uint64_t i, uint64_t j) {
    if (all) return 1;
    const uint64_t lo = i < j ? i : j, hi = i < j ? j : i;
    return syn_mix(seed + (lo * n + hi + 1) * 0x9E3779B97F4A7C15ULL) < thr;
}

/* The hash of one pair key, for the numpy cross-check of this file. */
uint64_t syn_pair_hash(uint64_t seed, uint64_t key) {
    return syn_mix(seed + (key + 1) * 0x9E3779B97F4A7C15ULL);
}

static int64_t syn_block_of(int64_t m, const int64_t *off, int64_t i) {
    if (m == 0 || i >= off[m]) return -1;
    int64_t a = 0, b = m;
    while (b - a > 1) {
        const int64_t mid = (a + b) / 2;
        if (off[mid] <= i) a = mid; else b = mid;
    }
    return a;
}

/* Pass 1: rowptr[0..n] of the output (rowptr[0] = 0); returns nnz. */
int64_t syn_hash_sbm_rowptr(int64_t n, int64_t m, const int64_t *off, uint64_t seed, uint64_t thr,
                            int all, const int64_t *inter_rowptr, int64_t *rowptr) {
    rowptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = syn_block_of(m, off, i);
        int64_t cnt = inter_rowptr[i + 1] - inter_rowptr[i];
        if (c >= 0)
            for (int64_t j = off[c]; j < off[c + 1]; ++j)
                cnt += (j != i) && syn_linked(seed, thr, all, (uint64_t)n, (uint64_t)i, (uint64_t)j);
        rowptr[i + 1] = cnt;
    }
    for (int64_t i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
    return rowptr[n];
}

/* Pass 2: the column indices, rows ascending. */
void syn_hash_sbm_fill(int64_t n, int64_t m, const int64_t *off, uint64_t seed, uint64_t thr, int all,
                       const int64_t *inter_rowptr, const int32_t *inter_col, const int64_t *rowptr,
                       int32_t *col) {
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = syn_block_of(m, off, i);
        const int64_t lo = c >= 0 ? off[c] : 0, hi = c >= 0 ? off[c + 1] : 0;
        int64_t w = rowptr[i], e = inter_rowptr[i];
        const int64_t e_end = inter_rowptr[i + 1];
        while (e < e_end && inter_col[e] < lo) col[w++] = inter_col[e++];
        for (int64_t j = lo; j < hi; ++j)
            if (j != i && syn_linked(seed, thr, all, (uint64_t)n, (uint64_t)i, (uint64_t)j)) col[w++] = (int32_t)j;
        while (e < e_end) col[w++] = inter_col[e++];
    }
}
