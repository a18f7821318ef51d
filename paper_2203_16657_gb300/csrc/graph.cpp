// Host-only parts of libcia shared by the planner and community detection:
// the thread-local error text behind cia_last_error() and the validation of
// an input graph (no CUDA calls, so that this file also builds without the
// CUDA runtime).
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

// Validate the CSR: bounds, ordering, self loops, then symmetry in O(nnz):
// rows are visited in increasing order, so the entries (j, i) with i < j of
// row j are met in increasing i; a cursor per row checks they appear exactly
// in that order, and at the end every entry below the diagonal was matched.
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
    std::vector<int64_t> cursor(g->rowptr, g->rowptr + n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
            int64_t j = g->col[e];
            if (j <= i) continue;
            int64_t &cj = cursor[j];
            if (cj >= g->rowptr[j + 1] || g->col[cj] != i)
                return fail(CIA_ERR_INVALID_GRAPH, "asymmetric: link " + std::to_string(i) + "->" +
                                                       std::to_string(j) + " has no reverse");
            ++cj;
        }
    }
    for (int64_t j = 0; j < n; ++j) {
        int64_t c = cursor[j];
        if (c < g->rowptr[j + 1] && g->col[c] < j)
            return fail(CIA_ERR_INVALID_GRAPH, "asymmetric: link " + std::to_string(j) + "->" +
                                                   std::to_string(g->col[c]) + " has no reverse");
    }
    return CIA_OK;
}

}  // namespace cia

extern "C" const char *cia_last_error(void) { return cia::g_last_error.c_str(); }
