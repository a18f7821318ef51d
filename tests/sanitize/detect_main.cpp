// Drives the host-only community detection and graph validation of libcia
// (detect.cpp, graph.cpp) on small graphs, for a build with the address and
// undefined-behaviour sanitizers.  Exit status 0 when every check holds.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "cia.h"

namespace {

struct Csr {
    std::vector<int64_t> rowptr;
    std::vector<int32_t> col;
};

// Symmetric CSR from an adjacency predicate over i < j.
template <typename F>
Csr build(int64_t n, F linked) {
    std::vector<std::vector<int32_t>> adj(n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (linked(i, j)) {
                adj[i].push_back((int32_t)j);
                adj[j].push_back((int32_t)i);
            }
    Csr c;
    c.rowptr.push_back(0);
    for (int64_t i = 0; i < n; ++i) {
        std::vector<int32_t> &r = adj[i];
        std::vector<int32_t> sorted(r);
        for (size_t a = 1; a < sorted.size(); ++a)   // insertion sort, small rows
            for (size_t b = a; b > 0 && sorted[b - 1] > sorted[b]; --b) std::swap(sorted[b - 1], sorted[b]);
        c.col.insert(c.col.end(), sorted.begin(), sorted.end());
        c.rowptr.push_back((int64_t)c.col.size());
    }
    return c;
}

uint64_t mix(uint64_t x) {
    x += 0x9e3779b97f4a7c15ull;
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
    return x ^ (x >> 31);
}

int failures = 0;

void check(bool ok, const char *what) {
    if (!ok) {
        std::printf("FAILED: %s (%s)\n", what, cia_last_error());
        ++failures;
    }
}

void detect(const Csr &c, int64_t n, double gamma, double mu, int min_size, const char *what) {
    cia_graph g{n, c.rowptr.data(), c.col.data()};
    cia_detect_options opt;
    cia_detect_options_default(&opt);
    opt.gamma = gamma;
    opt.community_cost = mu;
    opt.min_size = min_size;
    opt.seed = 7;
    std::vector<int32_t> labels(n > 0 ? n : 1, -2);
    cia_detect_report rep;
    check(cia_detect_communities(&g, &opt, labels.data(), &rep) == CIA_OK, what);
    int32_t top = -1;
    int64_t unl = 0;
    for (int64_t i = 0; i < n; ++i) {
        check(labels[i] >= -1, what);
        if (labels[i] > top) top = labels[i];
        unl += labels[i] < 0;
    }
    check(rep.communities == top + 1 && rep.unlabelled == unl, what);
    check(rep.nnz_missing >= 0 && rep.nnz_inter >= 0 && rep.nnz_inter <= c.rowptr[n], what);
}

}  // namespace

int main() {
    const int64_t n = 300;
    // planted blocks of 20..60 nodes, p_in 0.8, sparse extra links
    std::vector<int32_t> block(n);
    for (int64_t i = 0, b = 0, left = 0; i < n; ++i) {
        if (left == 0) {
            left = 20 + (int64_t)(mix(b) % 41);
            ++b;
        }
        block[i] = (int32_t)b;
        --left;
    }
    const Csr sbm = build(n, [&](int64_t i, int64_t j) {
        const double u = (double)(mix(i * 1000003 + j) >> 11) / 9007199254740992.0;
        return block[i] == block[j] ? u < 0.8 : u < 0.01;
    });
    detect(sbm, n, 1.0, 0.0, 2, "planted blocks");
    detect(sbm, n, 4.0, 0.0, 1, "high resolution");
    detect(sbm, n, 1.0, 50.0, 3, "community cost");
    const Csr complete = build(40, [](int64_t, int64_t) { return true; });
    detect(complete, 40, 0.5, 0.0, 2, "complete graph");
    const Csr empty = build(25, [](int64_t, int64_t) { return false; });
    detect(empty, 25, 1.0, 0.0, 2, "no links");
    const Csr star = build(30, [](int64_t i, int64_t) { return i == 0; });
    detect(star, 30, 1.0, 0.0, 1, "star");
    const Csr one = build(1, [](int64_t, int64_t) { return false; });
    detect(one, 1, 1.0, 0.0, 1, "single node");

    // invalid graphs are rejected before any work
    std::vector<int32_t> labels(4);
    cia_detect_options opt;
    cia_detect_options_default(&opt);
    const int64_t rp_asym[] = {0, 1, 1, 1, 1};
    const int32_t col_asym[] = {1};
    cia_graph g_asym{4, rp_asym, col_asym};
    check(cia_detect_communities(&g_asym, &opt, labels.data(), nullptr) == CIA_ERR_INVALID_GRAPH, "asymmetric");
    const int64_t rp_loop[] = {0, 1, 1, 1, 1};
    const int32_t col_loop[] = {0};
    cia_graph g_loop{4, rp_loop, col_loop};
    check(cia_detect_communities(&g_loop, &opt, labels.data(), nullptr) == CIA_ERR_INVALID_GRAPH, "self loop");
    const int64_t rp_range[] = {0, 1, 1, 1, 1};
    const int32_t col_range[] = {9};
    cia_graph g_range{4, rp_range, col_range};
    check(cia_detect_communities(&g_range, &opt, labels.data(), nullptr) == CIA_ERR_INVALID_GRAPH, "out of range");
    opt.gamma = -1.0;
    check(cia_detect_communities(&g_range, &opt, labels.data(), nullptr) == CIA_ERR_INVALID_ARG, "bad gamma");

    std::printf("%s\n", failures ? "FAILED" : "OK");
    return failures ? 1 : 0;
}
