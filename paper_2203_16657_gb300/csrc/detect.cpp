// Community detection for step P1 (Sec. "Community Detection (P1)"): a
// partition that makes S sparse, by minimising the Potts Hamiltonian with the
// Erdos-Renyi null model (the objective of rber_pots, the paper's choice),
//   H = -sum_{m != l} (a_ml - gamma p) delta(c_m, c_l) + mu M
//     = -e_in + gamma p sum_c s_c (s_c - 1) + mu M,
// e_in the directed links inside communities, s_c the community sizes,
// p = nnz(A) / (N (N - 1)), M the number of communities and mu an extra cost
// per community (the paper's remark that the E1 work grows with the number
// of communities).  Louvain scheme: local moving of single (weighted) nodes,
// aggregation of the communities into weighted nodes, repeat; then one more
// local-moving pass over the original nodes, so that the result is a local
// minimum under single-node moves.  Host code, deterministic for a seed.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <string>
#include <vector>

#include "cia_internal.h"

namespace cia {
namespace {

// A level of the Louvain hierarchy seen as weighted nodes (size = original
// nodes inside) and weighted directed links without self loops (w = links
// between the two groups of original nodes, counted once per direction): the
// input graph itself (unit sizes and weights, its int32 columns), or an
// aggregated level (Owned).
struct View {
    int64_t n = 0;
    const int64_t *rowptr = nullptr;
    const int32_t *col32 = nullptr;   // input graph
    const int64_t *col64 = nullptr;   // aggregated level
    const double *w = nullptr;        // null: unit weights
    const double *size = nullptr;     // null: unit sizes
    int64_t nbr(int64_t e) const { return col32 ? (int64_t)col32[e] : col64[e]; }
    double weight(int64_t e) const { return w ? w[e] : 1.0; }
    double sz(int64_t i) const { return size ? size[i] : 1.0; }
};

struct Owned {
    std::vector<int64_t> rowptr, col;
    std::vector<double> w, size;
    View view() const {
        View v;
        v.n = (int64_t)size.size();
        v.rowptr = rowptr.data();
        v.col64 = col.data();
        v.w = w.data();
        v.size = size.data();
        return v;
    }
};

struct Objective {
    double gp;   // gamma p
    double mu;   // cost per community
};

// SplitMix64 (Steele, Lea and Flood 2014) for the visiting order.
uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Local moving on one level, starting from `comm` (ids in [0, n)); returns
// the moves made.  Moving node i (size s_i) from community A to B lowers H by
//   gain = 2 [k_iB - gp s_i S_B] - 2 [k_iA - gp s_i (S_A - s_i)] + mu [A empties] - mu [B is new],
// k_iC the link weight from i into C (without i itself), S_C the sizes.  The
// candidates are the communities of i's neighbours and a new community; the
// best strictly positive gain wins, the first found among equals.
int64_t local_moving(const View &L, const Objective &ob, std::vector<int64_t> &comm, uint64_t &rng) {
    const int64_t n = L.n;
    std::vector<double> csize(n, 0.0);
    for (int64_t i = 0; i < n; ++i) csize[comm[i]] += L.sz(i);
    std::vector<int64_t> empties;
    for (int64_t c = n - 1; c >= 0; --c)
        if (csize[c] == 0.0) empties.push_back(c);
    std::vector<double> kto(n, 0.0);
    std::vector<char> seen(n, 0);
    std::vector<int64_t> touched;
    std::vector<int64_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    for (int64_t i = n - 1; i > 0; --i) std::swap(order[i], order[(int64_t)(splitmix64(rng) % (uint64_t)(i + 1))]);
    int64_t moves = 0;
    for (int sweep = 0; sweep < 64; ++sweep) {
        int64_t moved = 0;
        for (int64_t i : order) {
            const int64_t a = comm[i];
            const double si = L.sz(i);
            touched.clear();
            for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e) {
                const int64_t c = comm[L.nbr(e)];
                if (!seen[c]) {
                    seen[c] = 1;
                    touched.push_back(c);
                }
                kto[c] += L.weight(e);
            }
            const bool alone = csize[a] == si;
            const double stay = 2.0 * (kto[a] - ob.gp * si * (csize[a] - si)) - (alone ? ob.mu : 0.0);
            int64_t best = a;
            double best_gain = 1e-9;   // strictly positive decreases of H only
            for (int64_t c : touched) {
                if (c == a) continue;
                const double gain = 2.0 * (kto[c] - ob.gp * si * csize[c]) - stay;
                if (gain > best_gain) {
                    best = c;
                    best_gain = gain;
                }
            }
            // a new community of its own (an empty id exists whenever i is not alone)
            if (!alone && !empties.empty() && -stay - ob.mu > best_gain) best = -1;
            for (int64_t c : touched) {
                kto[c] = 0.0;
                seen[c] = 0;
            }
            if (best != a) {
                if (best < 0) {
                    best = empties.back();
                    empties.pop_back();
                }
                csize[a] -= si;
                csize[best] += si;
                if (csize[a] == 0.0) empties.push_back(a);
                comm[i] = best;
                ++moved;
            }
        }
        moves += moved;
        if (!moved) break;
    }
    return moves;
}

// Renumber communities 0..M-1 in order of first appearance; returns M.
int64_t renumber(std::vector<int64_t> &comm) {
    std::vector<int64_t> id(comm.size(), -1);
    int64_t m = 0;
    for (auto &c : comm) {
        if (id[c] < 0) id[c] = m++;
        c = id[c];
    }
    return m;
}

// The communities of L as the nodes of the next level.
Owned aggregate(const View &L, const std::vector<int64_t> &comm, int64_t M) {
    Owned A;
    A.size.assign(M, 0.0);
    for (int64_t i = 0; i < L.n; ++i) A.size[comm[i]] += L.sz(i);
    std::vector<std::vector<int64_t>> members(M);
    for (int64_t i = 0; i < L.n; ++i) members[comm[i]].push_back(i);
    A.rowptr.assign(M + 1, 0);
    std::vector<double> acc(M, 0.0);
    std::vector<char> seen(M, 0);
    std::vector<int64_t> touched;
    for (int64_t c = 0; c < M; ++c) {
        touched.clear();
        for (int64_t i : members[c])
            for (int64_t e = L.rowptr[i]; e < L.rowptr[i + 1]; ++e) {
                const int64_t d = comm[L.nbr(e)];
                if (d == c) continue;   // internal links do not move
                if (!seen[d]) {
                    seen[d] = 1;
                    touched.push_back(d);
                }
                acc[d] += L.weight(e);
            }
        std::sort(touched.begin(), touched.end());
        for (int64_t d : touched) {
            A.col.push_back(d);
            A.w.push_back(acc[d]);
            acc[d] = 0.0;
            seen[d] = 0;
        }
        A.rowptr[c + 1] = (int64_t)A.col.size();
    }
    return A;
}

cia_status bad(const std::string &msg) {
    set_error(msg);
    return CIA_ERR_INVALID_ARG;
}

}  // namespace
}  // namespace cia

using namespace cia;

extern "C" void cia_detect_options_default(cia_detect_options *opt) {
    if (!opt) return;
    opt->gamma = 1.0;
    opt->community_cost = 0.0;
    opt->min_size = 2;
    opt->max_levels = 8;
    opt->seed = 0;
}

extern "C" cia_status cia_detect_communities(const cia_graph *g, const cia_detect_options *opt, int32_t *labels,
                                             cia_detect_report *report) {
    clear_error();
    if (!g || !opt || !labels) return bad("graph, options or labels is NULL");
    if (!(opt->gamma > 0.0) || !std::isfinite(opt->gamma)) return bad("gamma must be positive and finite");
    if (!(opt->community_cost >= 0.0) || !std::isfinite(opt->community_cost))
        return bad("community_cost must be >= 0 and finite");
    if (opt->min_size < 1) return bad("min_size must be >= 1");
    if (opt->max_levels < 1) return bad("max_levels must be >= 1");
    cia_status st = validate_graph(g);
    if (st != CIA_OK) return st;
    const int64_t n = g->n;
    const int64_t nnz = g->rowptr[n];
    const Objective ob{opt->gamma * (n > 1 ? (double)nnz / ((double)n * (double)(n - 1)) : 0.0), opt->community_cost};

    View base;
    base.n = n;
    base.rowptr = g->rowptr;
    base.col32 = g->col;

    uint64_t rng = opt->seed;
    std::vector<int64_t> node_comm(n);            // community of every original node
    std::iota(node_comm.begin(), node_comm.end(), 0);
    Owned agg;   // the current aggregated level
    View L = base;
    int levels = 0;
    int64_t moves = 0;
    for (; levels < opt->max_levels; ++levels) {
        std::vector<int64_t> comm(L.n);
        std::iota(comm.begin(), comm.end(), 0);
        const int64_t mv = local_moving(L, ob, comm, rng);
        moves += mv;
        if (mv == 0) break;
        const int64_t M = renumber(comm);
        for (auto &c : node_comm) c = comm[c];
        if (M == L.n) break;
        agg = aggregate(L, comm, M);
        L = agg.view();
    }
    // a last pass over the original nodes: a local minimum under single moves
    moves += local_moving(base, ob, node_comm, rng);
    const int64_t M = renumber(node_comm);

    // H, then the labels with small communities as -1
    std::vector<int64_t> csize(M, 0);
    for (int64_t i = 0; i < n; ++i) ++csize[node_comm[i]];
    int64_t e_in = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) e_in += node_comm[g->col[e]] == node_comm[i];
    double pairs = 0.0;
    for (int64_t c = 0; c < M; ++c) pairs += (double)csize[c] * (double)(csize[c] - 1);
    const double H = -(double)e_in + ob.gp * pairs + ob.mu * (double)M;

    std::vector<int64_t> out_id(M, -1);
    int64_t mout = 0, unl = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t c = node_comm[i];
        if (csize[c] < opt->min_size) {
            labels[i] = -1;
            ++unl;
            continue;
        }
        if (out_id[c] < 0) out_id[c] = mout++;
        labels[i] = (int32_t)out_id[c];
    }
    if (report) {
        // entries of S for the returned labels (unlabelled nodes: all links extra)
        int64_t inside = 0;
        double miss_pairs = 0.0;
        for (int64_t i = 0; i < n; ++i)
            for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e)
                inside += labels[i] >= 0 && labels[g->col[e]] == labels[i];
        for (int64_t c = 0; c < M; ++c)
            if (csize[c] >= opt->min_size) miss_pairs += (double)csize[c] * (double)(csize[c] - 1);
        report->communities = mout;
        report->unlabelled = unl;
        report->nnz_missing = (int64_t)miss_pairs - inside;
        report->nnz_inter = nnz - inside;
        report->hamiltonian = H;
        report->levels = levels;
        report->moves = moves;
    }
    return CIA_OK;
}
