// Host-only parts of libcia shared by the planner and community detection:
// the thread-local error text behind cia_last_error() and the validation of
// an input graph (no CUDA calls, so that this file also builds without the
// CUDA runtime).
#include <algorithm>
#include <cstdint>
#include <string>
#include <vector>

#include "cia_internal.h"

namespace cia {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

static cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

// SplitMix64 output function (Steele, Lea and Flood 2014) of a link key.
static inline uint64_t link_hash(uint64_t key) {
    uint64_t z = (key + 1) * 0x9E3779B97F4A7C15ULL + 0x2203166570ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Validate the CSR: bounds, ordering and self loops row by row, then
// symmetry.  A streaming pass first sums, modulo 2^64, a 64-bit hash of the
// unordered pair {i, j} over the entries above the diagonal and over those
// below it: for a symmetric matrix the two multisets of pairs are equal, so
// the sums agree (and so do the counts), and the check is done in one read of
// the columns.  Otherwise (or in the 2^-64-scale event of colliding sums of
// an asymmetric input, which then passes) the exact pass runs: every entry
// (i, j) above the diagonal must have its mirror (j, i), found by binary
// search in the sorted row j, and the entries below the diagonal must be
// exactly as many (the mirrors are distinct entries, so then every entry
// below the diagonal is some mirror).  Rows run in parallel; the smallest
// offending row is reported.
cia_status validate_graph(const cia_graph *g) {
    const int64_t n = g->n;
    if (g->rowptr[0] != 0) return fail(CIA_ERR_INVALID_GRAPH, "rowptr[0] != 0");
    for (int64_t i = 0; i < n; ++i)
        if (g->rowptr[i + 1] < g->rowptr[i])
            return fail(CIA_ERR_INVALID_GRAPH, "rowptr decreases at row " + std::to_string(i));
    int64_t bad_row = -1;
    std::string why;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
        int32_t prev = -1;
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            int32_t j = g->col[e];
            const char *w = nullptr;
            if (j < 0 || j >= n) w = "column out of range";
            else if (j == i) w = "self loop";
            else if (j <= prev) w = "columns not strictly increasing";
            if (w) {
#pragma omp critical
                {
                    if (bad_row < 0 || i < bad_row) { bad_row = i; why = w; }
                }
                break;
            }
            prev = j;
        }
    }
    if (bad_row >= 0) return fail(CIA_ERR_INVALID_GRAPH, why + " in row " + std::to_string(bad_row));
    {
        uint64_t up = 0, down = 0;
        int64_t n_up = 0, n_down = 0;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : up, down, n_up, n_down)
        for (int64_t i = 0; i < n; ++i) {
            for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
                const int64_t j = g->col[e];
                if (j > i) {
                    up += link_hash((uint64_t)i * (uint64_t)n + (uint64_t)j);
                    ++n_up;
                } else {
                    down += link_hash((uint64_t)j * (uint64_t)n + (uint64_t)i);
                    ++n_down;
                }
            }
        }
        if (up == down && n_up == n_down) return CIA_OK;
    }
    int64_t above = 0, below = 0, bad_i = -1, bad_j = -1;
#pragma omp parallel for schedule(dynamic, 4096) reduction(+ : above, below)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            const int64_t j = g->col[e];
            if (j < i) {
                ++below;
                continue;
            }
            ++above;
            const int32_t *lo = g->col + g->rowptr[j], *hi = g->col + g->rowptr[j + 1];
            const int32_t *f = std::lower_bound(lo, hi, (int32_t)i);
            if (f == hi || *f != i) {
#pragma omp critical
                {
                    if (bad_i < 0 || i < bad_i) { bad_i = i; bad_j = j; }
                }
            }
        }
    }
    if (bad_i >= 0)
        return fail(CIA_ERR_INVALID_GRAPH, "asymmetric: link " + std::to_string(bad_i) + "->" +
                                               std::to_string(bad_j) + " has no reverse");
    if (above != below) {
        // an entry below the diagonal without its mirror: the smallest such row
        for (int64_t j = 0; j < n; ++j)
            for (int64_t e = g->rowptr[j]; e < g->rowptr[j + 1]; ++e) {
                const int64_t i = g->col[e];
                if (i >= j) break;
                const int32_t *lo = g->col + g->rowptr[i], *hi = g->col + g->rowptr[i + 1];
                const int32_t *f = std::lower_bound(lo, hi, (int32_t)j);
                if (f == hi || *f != j)
                    return fail(CIA_ERR_INVALID_GRAPH, "asymmetric: link " + std::to_string(j) + "->" +
                                                           std::to_string(i) + " has no reverse");
            }
    }
    return CIA_OK;
}

}  // namespace cia

extern "C" const char *cia_last_error(void) { return cia::g_last_error.c_str(); }
