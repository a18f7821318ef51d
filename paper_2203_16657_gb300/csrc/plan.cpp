// Host planner of libcia: step P1 of the CIA (Sec. 3.1 and App. A.1).
//
// Given the symmetric 0/1 adjacency A (CSR) and community labels, the plan
//  - validates A (symmetric, no self loops, sorted unique in-range columns),
//  - builds the permutation kappa sorting nodes by (label, original id) with
//    unlabelled nodes (label -1, "no community") last, so that B = P A P^T has
//    the communities as consecutive diagonal blocks,
//  - records the block sizes lambda_c as offsets (the dense part D is never
//    stored, Sec. 3.1),
//  - splits the sparse remainder S = B - D into its -1 entries (links missing
//    inside a block; the diagonal is handled analytically by the kernels) and
//    its +1 entries (links between blocks), each as a CSR over permuted ids,
//  - cuts every community into work tiles of at most tile_nodes nodes,
//  - uploads everything and allocates the device work buffers.
// The planner is offline and untimed; it runs row-parallel with OpenMP.
#include <omp.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "cia_basis.h"
#include "cia_internal.h"

namespace cia {

// Raise a kernel's dynamic shared-memory limit to `smem` on `device` (once
// per kernel, device and size): the default limit covers dynamic plus static
// shared memory up to 48 KiB, so a kernel with static buffers can need the
// attribute below 48 KiB of dynamic memory as well.
cudaError_t ensure_dynamic_smem(const void *kernel, int device, size_t smem) {
    if (smem == 0) return cudaSuccess;
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, size_t> done;
    std::lock_guard<std::mutex> lock(mu);
    size_t &have = done[{kernel, device}];
    if (smem <= have) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) have = smem;
    return e;
}

cia_status cuda_fail(cudaError_t e, const char *what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? CIA_ERR_OOM : CIA_ERR_CUDA;
}

static cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

// Device copy of src (count elements; zero-filled when src is NULL), owned by
// the plan; `tile` marks buffers that belong to the current tiling.
template <typename T>
static cia_status upload(cia_plan *pl, T **dst, const T *src, size_t count, bool tile = false) {
    size_t bytes = std::max<size_t>(count * sizeof(T), 256);
    void *p = nullptr;
    CIA_CUDA_TRY(cudaMalloc(&p, bytes));
    (tile ? pl->tile_allocs : pl->allocations).push_back(p);
    pl->device_bytes += (int64_t)bytes;
    if (tile) pl->tile_bytes += (int64_t)bytes;
    if (src && count) CIA_CUDA_TRY(cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
    else CIA_CUDA_TRY(cudaMemset(p, 0, bytes));
    *dst = (T *)p;
    return CIA_OK;
}

static cia_status alloc_bytes(cia_plan *pl, void **dst, size_t bytes) {
    return upload<unsigned char>(pl, (unsigned char **)dst, nullptr, bytes);
}

// Ensemble instance of an original node id (0 for a single network).
static int64_t instance_of_node(const cia_plan *pl, int64_t id) {
    if (pl->B <= 1) return 0;
    return (int64_t)(std::upper_bound(pl->inst_off.begin(), pl->inst_off.end(), id) - pl->inst_off.begin()) - 1;
}

// One instance of a streamed ensemble plan, split, kept until the plan is
// finished: rows in the instance's permuted order (its labelled nodes, then
// its free ones).
struct StagedInstance {
    int64_t n = 0, n_lab = 0, M = 0, nnz = 0, max_comm = 0;
    std::vector<int32_t> perm;       // [n] permuted -> original id within the instance
    std::vector<int64_t> off;        // [M + 1] community offsets within the instance
    std::vector<int64_t> miss_cnt;   // [n_lab] missing links per labelled row
    std::vector<uint16_t> miss;      // community-local indices, rows in order
    std::vector<int64_t> inter_cnt;  // [n] inter links per row
    std::vector<int64_t> inter;      // targets: >= 0 the ensemble's permuted id of a labelled
                                     // node; < 0: -1 - (index among all free nodes so far)
    std::vector<double> omega;       // [n] natural frequencies, permuted (empty: zero)
};

struct BatchStaging {
    cia_options opt{};
    std::vector<StagedInstance> inst;
    int64_t lab_total = 0, free_total = 0, comm_total = 0, n_total = 0;
};

static void free_all(cia_plan *pl) {
    delete pl->batch_stage;
    pl->batch_stage = nullptr;
    invalidate_graphs(pl);
    if (pl->capture_stream) cudaStreamDestroy(pl->capture_stream);
    pl->capture_stream = nullptr;
    for (int i = 0; i < 4; ++i) {
        if (pl->gc_side[i]) cudaStreamDestroy(pl->gc_side[i]);
        if (pl->gc_join[i]) cudaEventDestroy(pl->gc_join[i]);
        pl->gc_side[i] = nullptr;
        pl->gc_join[i] = nullptr;
    }
    if (pl->gc_fork) cudaEventDestroy(pl->gc_fork);
    pl->gc_fork = nullptr;
    for (void *p : pl->allocations) cudaFree(p);
    pl->allocations.clear();
    for (void *p : pl->tile_allocs) cudaFree(p);
    pl->tile_allocs.clear();
    for (cudaEvent_t e : pl->prof_ev) cudaEventDestroy(e);
    pl->prof_ev.clear();
    if (pl->d.r_tmp_host) cudaFreeHost(pl->d.r_tmp_host);
    pl->d.r_tmp = pl->d.r_tmp_host = nullptr;
    pl->d.r_cap = 0;
    if (pl->d.err_flag_host) cudaFreeHost(pl->d.err_flag_host);
    pl->d.err_flag_host = nullptr;
    pl->d.err_flag = nullptr;
}

}  // namespace cia

using namespace cia;

extern "C" const char *cia_status_string(cia_status s) {
    switch (s) {
        case CIA_OK: return "CIA_OK";
        case CIA_ERR_INVALID_ARG: return "CIA_ERR_INVALID_ARG";
        case CIA_ERR_INVALID_GRAPH: return "CIA_ERR_INVALID_GRAPH";
        case CIA_ERR_UNSUPPORTED: return "CIA_ERR_UNSUPPORTED";
        case CIA_ERR_CUDA: return "CIA_ERR_CUDA";
        case CIA_ERR_TIMEOUT: return "CIA_ERR_TIMEOUT";
        case CIA_ERR_FALLBACK: return "CIA_ERR_FALLBACK";
        case CIA_ERR_NUMERIC: return "CIA_ERR_NUMERIC";
        case CIA_ERR_OOM: return "CIA_ERR_OOM";
    }
    return "CIA_ERR_UNKNOWN";
}


// Longest missing-link chunk of one lane: longer lists are split into
// chunks ("virtual rows") whose partial sums Phase B adds in a fixed order.
static const int64_t kChunk = 64;
// Most chunks per tile (shared-memory partial sums of one consumer group).
static const int64_t kMaxChunks = 512;

// Scratch of the missing-link scheduler (one per planning thread).
struct MissScheduler {
    std::vector<int32_t> bucket[32][16];   // greedy: remaining entries of each lane by bank group
    std::vector<int32_t> lane_at;          // colouring: [lane][colour] entry, -1 = free
    std::vector<int32_t> grp_at;           // colouring: [bank group][colour] lane, -1 = free
    std::vector<int32_t> path;             // colouring: (lane, group, colour) triples of a swap path
    std::vector<int32_t> later;            // colouring: (lane, entry) pairs whose bank group is full
    std::vector<uint16_t> out;             // [position][32] scheduled entries of one slice
};

// Extra 8-entry vectors per slice that the conflict-free schedule may add
// beyond the longest lane's list (padding entries read the zero slots).
#ifndef CIA_SCHED_EXTRA_VECTORS
#define CIA_SCHED_EXTRA_VECTORS 0
#endif

// Set of colours (positions) < 128.
struct ColourSet {
    uint64_t w[2] = {0, 0};
    void fill(int64_t n) {
        w[0] = n >= 64 ? ~0ull : ((1ull << n) - 1);
        w[1] = n >= 128 ? ~0ull : n > 64 ? ((1ull << (n - 64)) - 1) : 0ull;
    }
    bool has(int64_t c) const { return (w[c >> 6] >> (c & 63)) & 1ull; }
    void set(int64_t c) { w[c >> 6] |= 1ull << (c & 63); }
    void clear(int64_t c) { w[c >> 6] &= ~(1ull << (c & 63)); }
    int64_t first() const { return w[0] ? __builtin_ctzll(w[0]) : w[1] ? 64 + __builtin_ctzll(w[1]) : -1; }
};

// Greedy order of one group of G lanes (fallback): at each position the
// lanes with fewer remaining entries pick first, each taking an unused bank
// group from its largest bucket.
static void greedy_group(const uint16_t *const ent[], const int64_t len[], int G, int64_t ncol, int32_t *lane_at,
                         MissScheduler &sc) {
    int remaining[16];
    for (int u = 0; u < G; ++u) {
        for (auto &bk : sc.bucket[u]) bk.clear();
        for (int64_t e = 0; e < len[u]; ++e) sc.bucket[u][ent[u][e] & (G - 1)].push_back(ent[u][e]);
        remaining[u] = (int)len[u];
    }
    for (int64_t p = 0; p < ncol; ++p) {
        int order[16];
        for (int q = 0; q < G; ++q) order[q] = q;
        std::stable_sort(order, order + G, [&](int x, int y) { return remaining[x] < remaining[y]; });
        unsigned used = 0;
        for (int q = 0; q < G; ++q) {
            const int u = order[q];
            lane_at[(size_t)u * ncol + p] = -1;
            if (remaining[u] == 0) continue;
            int best = -1;
            for (int pass = 0; pass < 2 && best < 0; ++pass)
                for (int c = 0; c < G; ++c) {
                    if (sc.bucket[u][c].empty() || (pass == 0 && (used >> c & 1u))) continue;
                    if (best < 0 || sc.bucket[u][c].size() > sc.bucket[u][best].size()) best = c;
                }
            lane_at[(size_t)u * ncol + p] = sc.bucket[u][best].back();
            sc.bucket[u][best].pop_back();
            --remaining[u];
            used |= 1u << best;
        }
    }
}

// Edge colouring of one group of G lanes (see schedule_slice); false if a
// swap path ran longer than the graph allows (the caller then falls back).
static bool colour_group(const uint16_t *const ent[], const int64_t len[], int G, int64_t ncol, MissScheduler &sc) {
    int32_t *LA = sc.lane_at.data();   // [u * ncol + c]
    int32_t *GA = sc.grp_at.data();    // [g * ncol + c]
    std::fill(LA, LA + (size_t)G * ncol, -1);
    std::fill(GA, GA + (size_t)G * ncol, -1);
    ColourSet lane_free[16], grp_free[16];
    for (int v = 0; v < G; ++v) {
        lane_free[v].fill(ncol);
        grp_free[v].fill(ncol);
    }
    sc.later.clear();
    const int64_t max_steps = 2 * (int64_t)G * ncol + 2;
    for (int u = 0; u < G; ++u) {
        for (int64_t k = 0; k < len[u]; ++k) {
            const int32_t e = ent[u][k];
            const int g = e & (G - 1);
            const int64_t ca = lane_free[u].first();   // exists: len <= ncol
            const int64_t cb = grp_free[g].first();
            if (cb < 0) {                              // bank group full: placed after the colouring
                sc.later.insert(sc.later.end(), {u, e});
                continue;
            }
            int64_t c = ca;
            if (!grp_free[g].has(ca)) {
                if (lane_free[u].has(cb)) {
                    c = cb;
                } else {
                    // swap ca <-> cb along the alternating path from g that starts with ca
                    sc.path.clear();
                    int node = g;
                    bool at_group = true;
                    int64_t col = ca;
                    for (int64_t step = 0;; ++step) {
                        if (step > max_steps) return false;
                        if (at_group) {
                            const int32_t lu = GA[(size_t)node * ncol + col];
                            if (lu < 0) break;
                            sc.path.insert(sc.path.end(), {lu, node, (int32_t)col});
                            node = lu;
                        } else {
                            const int32_t ee = LA[(size_t)node * ncol + col];
                            if (ee < 0) break;
                            sc.path.insert(sc.path.end(), {node, ee & (G - 1), (int32_t)col});
                            node = ee & (G - 1);
                        }
                        at_group = !at_group;
                        col = col == ca ? cb : ca;
                    }
                    const size_t np = sc.path.size() / 3;
                    std::vector<int32_t> moved(np);
                    for (size_t i = 0; i < np; ++i) {
                        const int32_t lu = sc.path[3 * i], gg = sc.path[3 * i + 1], cc = sc.path[3 * i + 2];
                        moved[i] = LA[(size_t)lu * ncol + cc];
                        LA[(size_t)lu * ncol + cc] = -1;
                        GA[(size_t)gg * ncol + cc] = -1;
                    }
                    for (size_t i = 0; i < np; ++i) {
                        const int32_t lu = sc.path[3 * i], gg = sc.path[3 * i + 1], cc = sc.path[3 * i + 2];
                        const int64_t nc = cc == ca ? cb : ca;
                        LA[(size_t)lu * ncol + nc] = moved[i];
                        GA[(size_t)gg * ncol + nc] = lu;
                    }
                    for (size_t i = 0; i < np; ++i) {
                        const int32_t lu = sc.path[3 * i], gg = sc.path[3 * i + 1];
                        for (const int64_t cc : {ca, cb}) {
                            if (LA[(size_t)lu * ncol + cc] < 0) lane_free[lu].set(cc); else lane_free[lu].clear(cc);
                            if (GA[(size_t)gg * ncol + cc] < 0) grp_free[gg].set(cc); else grp_free[gg].clear(cc);
                        }
                    }
                }
            }
            LA[(size_t)u * ncol + c] = e;
            GA[(size_t)g * ncol + c] = u;
            lane_free[u].clear(c);
            grp_free[g].clear(c);
        }
    }
    // entries of full bank groups: any free position of their lane (a conflict)
    for (size_t i = 0; i < sc.later.size(); i += 2) {
        const int u = sc.later[i];
        const int64_t c = lane_free[u].first();
        LA[(size_t)u * ncol + c] = sc.later[i + 1];
        lane_free[u].clear(c);
    }
    return true;
}

// Order the missing-link entries of one slice (32 lanes, lane l sums
// ent[l][0..len[l])) into positions: at position p every lane reads one
// entry (or a padding entry), and the kernels issue one shared-memory gather
// per position for the whole warp.  A warp's 8-byte loads are served per
// half-warp (G = 16 lanes, 16 bank groups of 8 bytes: the community-local
// index mod 16), 16-byte loads per quarter-warp (G = 8); a position is free
// of bank conflicts when the live lanes of each group of G lanes use distinct
// bank groups.  For each group of G lanes this is an edge colouring of the
// bipartite multigraph lanes x bank groups (one edge per entry, colours =
// positions): with as many colours as the largest degree (the longest list,
// or the most entries of the G lanes in one bank group) a colouring exists
// (Koenig's theorem); it is built edge by edge, swapping the two colours
// along an alternating path when no colour is free at both ends.  Positions
// are capped at the longest list rounded up to 8 plus CIA_SCHED_EXTRA_VECTORS
// vectors; entries of a bank group that then has no free position are placed
// last, at free positions of their lanes (conflicts).  Padding entries take
// distinct unused bank groups: sentinel + 1 + j, j in [0, G), all of them zero
// slots after the community window, when `spread` allows (else the sentinel
// itself).  Returns the number of positions (a multiple of 8);
// sc.out[p * 32 + lane].
static int64_t schedule_slice(const uint16_t *const ent[32], const int64_t len[32], int G, uint16_t sentinel,
                              bool spread, MissScheduler &sc) {
    int64_t maxlen = 0;
    for (int lane = 0; lane < 32; ++lane) maxlen = std::max(maxlen, len[lane]);
    const int64_t npos_min = (maxlen + 7) / 8 * 8;
    int64_t delta = maxlen;
    for (int q = 0; q < 32 / G; ++q) {
        int64_t load[16] = {0};
        for (int u = 0; u < G; ++u)
            for (int64_t e = 0; e < len[q * G + u]; ++e) ++load[ent[q * G + u][e] & (G - 1)];
        for (int g = 0; g < G; ++g) delta = std::max(delta, load[g]);
    }
    const int64_t ncol = std::min<int64_t>((delta + 7) / 8 * 8, npos_min + 8 * CIA_SCHED_EXTRA_VECTORS);
    sc.out.assign((size_t)ncol * 32, sentinel);
    if (ncol == 0) return 0;
    sc.lane_at.resize((size_t)G * ncol);
    sc.grp_at.resize((size_t)G * ncol);
    for (int q = 0; q < 32 / G; ++q) {
        // the colour sets hold 128 positions: longer lists take the greedy order
        if (ncol > 128 || !colour_group(ent + q * G, len + q * G, G, ncol, sc))
            greedy_group(ent + q * G, len + q * G, G, ncol, sc.lane_at.data(), sc);
        const int32_t *LA = sc.lane_at.data();
        // padding entries: distinct bank groups unused at their position
        for (int64_t p = 0; p < ncol; ++p) {
            unsigned used = 0;
            for (int u = 0; u < G; ++u)
                if (LA[(size_t)u * ncol + p] >= 0) used |= 1u << (LA[(size_t)u * ncol + p] & (G - 1));
            int g = 0;
            for (int u = 0; u < G; ++u) {
                const int32_t e = LA[(size_t)u * ncol + p];
                uint16_t v;
                if (e >= 0) {
                    v = (uint16_t)e;
                } else if (spread) {
                    while (g < G && (used >> g & 1u)) ++g;
                    const int gg = g < G ? g : (sentinel & (G - 1));
                    v = (uint16_t)(sentinel + 1 + ((gg - sentinel - 1) & (G - 1)));
                    if (g < G) used |= 1u << g;
                } else {
                    v = sentinel;
                }
                sc.out[(size_t)p * 32 + q * G + u] = v;
            }
        }
    }
    return ncol;
}

// One tile's blob (see cia::DeviceBuffers): slice descriptors, row maps, the
// row -> chunk table, missing vectors over chunks, inter vectors over rows.
struct TileBlob {
    std::vector<unsigned char> bytes;
    int32_t nsl = 0;
    uint32_t vtab_off = 0, mvec_off = 0, ivec_off = 0;
};

static int64_t chunks_of(int64_t entries) { return std::max<int64_t>(1, (entries + kChunk - 1) / kChunk); }

static void build_tile_blob(int64_t f, int64_t cnt, uint16_t msent, bool spread, int32_t inter_sent,
                            int bank_lanes, const std::vector<int64_t> &miss_cnt, const std::vector<int64_t> &miss_off,
                            const std::vector<uint16_t> &miss_local, const std::vector<int64_t> &inter_cnt,
                            const std::vector<int64_t> &inter_off, const std::vector<int32_t> &inter_col,
                            TileBlob &tb, MissScheduler &sc) {
    // chunks: row r's missing list in v_r nearly equal contiguous pieces,
    // numbered vbase_r .. vbase_r + v_r - 1
    struct Chunk { int32_t row, vidx; int64_t e0, len; };
    std::vector<Chunk> ch;
    std::vector<uint32_t> vtab(cnt);
    for (int64_t r = 0; r < cnt; ++r) {
        const int64_t E = miss_cnt[f + r], v = chunks_of(E);
        vtab[r] = (uint32_t)ch.size() | ((uint32_t)v << 16);
        int64_t e = 0;
        for (int64_t c = 0; c < v; ++c) {
            const int64_t len = E / v + (c < E % v ? 1 : 0);
            ch.push_back({(int32_t)r, (int32_t)ch.size(), e, len});
            e += len;
        }
    }
    const int64_t V = (int64_t)ch.size();
    std::vector<int32_t> mo(V), io(cnt);
    for (int64_t q = 0; q < V; ++q) mo[q] = (int32_t)q;
    for (int64_t r = 0; r < cnt; ++r) io[r] = (int32_t)r;
    std::stable_sort(mo.begin(), mo.end(), [&](int32_t x, int32_t y) { return ch[x].len > ch[y].len; });
    std::stable_sort(io.begin(), io.end(), [&](int32_t x, int32_t y) { return inter_cnt[f + x] > inter_cnt[f + y]; });
    const int64_t nsm = (V + 31) / 32, nsi = (cnt + 31) / 32, nsl = std::max(nsm, nsi);
    // schedule every slice's missing entries first: the schedule fixes its vector count
    std::vector<int64_t> nvm(nsl, 0), nvi(nsl, 0);
    std::vector<std::vector<uint16_t>> sched(nsl);
    int64_t mv = 0, iv = 0;
    for (int64_t s = 0; s < nsl; ++s) {
        const uint16_t *ent[32];
        int64_t len[32];
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t ms = 32 * s + lane;
            const Chunk *c = ms < V ? &ch[mo[ms]] : nullptr;
            ent[lane] = c ? miss_local.data() + miss_off[f + c->row] + c->e0 : nullptr;
            len[lane] = c ? c->len : 0;
        }
        nvm[s] = s < nsm ? schedule_slice(ent, len, bank_lanes, msent, spread, sc) / 8 : 0;
        sched[s].swap(sc.out);
        if (s < nsi) nvi[s] = (inter_cnt[f + io[32 * s]] + 3) / 4;
        mv += 32 * nvm[s];
        iv += 32 * nvi[s];
    }
    tb.nsl = (int32_t)nsl;
    tb.vtab_off = (uint32_t)(144 * nsl);
    tb.mvec_off = tb.vtab_off + (uint32_t)((4 * cnt + 15) & ~(int64_t)15);
    tb.ivec_off = tb.mvec_off + (uint32_t)(16 * mv);
    tb.bytes.assign(tb.ivec_off + 16 * iv, 0);
    uint32_t *desc = reinterpret_cast<uint32_t *>(tb.bytes.data());
    uint32_t *rows = reinterpret_cast<uint32_t *>(tb.bytes.data() + 16 * nsl);
    std::memcpy(tb.bytes.data() + tb.vtab_off, vtab.data(), 4 * cnt);
    uint16_t *mvec = reinterpret_cast<uint16_t *>(tb.bytes.data() + tb.mvec_off);
    int32_t *ivec = reinterpret_cast<int32_t *>(tb.bytes.data() + tb.ivec_off);
    mv = iv = 0;
    for (int64_t s = 0; s < nsl; ++s) {
        desc[4 * s + 0] = (uint32_t)mv;
        desc[4 * s + 1] = (uint32_t)nvm[s];
        desc[4 * s + 2] = (uint32_t)iv;
        desc[4 * s + 3] = (uint32_t)nvi[s];
        for (int lane = 0; lane < 32; ++lane) {
            const int64_t ms = 32 * s + lane;
            const bool mlive = ms < V, ilive = ms < cnt;
            const int32_t ir = ilive ? io[ms] : -1;
            rows[32 * s + lane] = (uint32_t)(mlive ? ch[mo[ms]].vidx : 0xffff) | ((uint32_t)(ilive ? ir : 0xffff) << 16);
            for (int64_t j = 0; j < nvi[s]; ++j)
                for (int h = 0; h < 4; ++h) {
                    const int64_t e = 4 * j + h;
                    const bool has = ilive && e < inter_cnt[f + ir];
                    ivec[4 * (iv + 32 * j + lane) + h] = has ? inter_col[inter_off[f + ir] + e] : inter_sent;
                }
            // position p of the schedule is entry h = p % 8 of vector j = p / 8
            for (int64_t p = 0; p < 8 * nvm[s]; ++p)
                mvec[8 * (mv + 32 * (p / 8) + lane) + (p % 8)] = sched[s][(size_t)p * 32 + lane];
        }
        mv += 32 * nvm[s];
        iv += 32 * nvi[s];
    }
}

// Segmented blob of one tile for the persistent ring kernel: every row's
// missing list is cut into v near-equal chunks (v = ceil(len / 64), at most 32)
// that occupy v consecutive lanes of one slice, so that a warp can add a row's
// chunk sums itself; rows (longest first) fill slices of 32 lanes in order, a
// row that does not fit the current slice opening the next.  Lane map word:
// row within the tile | v << 16 | lane offset within the row << 22
// (0xffffffff: no row); the inter-community list of a row sits on its first
// lane.  Layout: [slice descriptors: nsl x uint4 (miss offset, miss vectors,
// inter offset, inter vectors)][lane maps: nsl x 32 x u32][missing vectors:
// 8 x u16][inter vectors: 4 x i32].
#ifndef CIA_SEG_CHUNK
#define CIA_SEG_CHUNK 64
#endif
static constexpr int64_t kSegChunk = CIA_SEG_CHUNK;

static int64_t seg_lanes(int64_t entries) {
    return std::min<int64_t>(32, std::max<int64_t>(1, (entries + kSegChunk - 1) / kSegChunk));
}

static void build_tile_blob_seg(int64_t f, int64_t cnt, uint16_t msent, bool spread, int32_t inter_sent,
                                int bank_lanes, const std::vector<int64_t> &miss_cnt,
                                const std::vector<int64_t> &miss_off, const std::vector<uint16_t> &miss_local,
                                const std::vector<int64_t> &inter_cnt, const std::vector<int64_t> &inter_off,
                                const std::vector<int32_t> &inter_col, TileBlob &tb, MissScheduler &sc) {
    std::vector<int32_t> order(cnt);
    for (int64_t r = 0; r < cnt; ++r) order[r] = (int32_t)r;
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return miss_cnt[f + x] > miss_cnt[f + y]; });
    // slices: per lane (row, chunk index, first entry, length)
    struct Lane { int32_t row = -1, part = 0, v = 0; int64_t e0 = 0, len = 0; };
    std::vector<std::array<Lane, 32>> sl;
    int used = 32;
    for (int32_t r : order) {
        const int64_t E = miss_cnt[f + r], v = seg_lanes(E);
        if (used + v > 32) {
            sl.emplace_back();
            used = 0;
        }
        int64_t e = 0;
        for (int64_t c = 0; c < v; ++c) {
            const int64_t len = E / v + (c < E % v ? 1 : 0);
            sl.back()[used + c] = Lane{r, (int32_t)c, (int32_t)v, e, len};
            e += len;
        }
        used += (int)v;
    }
    const int64_t nsl = (int64_t)sl.size();
    std::vector<int64_t> nvm(nsl, 0), nvi(nsl, 0);
    std::vector<std::vector<uint16_t>> sched(nsl);
    int64_t mv = 0, iv = 0;
    for (int64_t s = 0; s < nsl; ++s) {
        const uint16_t *ent[32];
        int64_t len[32];
        int64_t imax = 0;
        for (int lane = 0; lane < 32; ++lane) {
            const Lane &L = sl[s][lane];
            ent[lane] = L.row >= 0 ? miss_local.data() + miss_off[f + L.row] + L.e0 : nullptr;
            len[lane] = L.row >= 0 ? L.len : 0;
            if (L.row >= 0 && L.part == 0) imax = std::max<int64_t>(imax, inter_cnt[f + L.row]);
        }
        nvm[s] = schedule_slice(ent, len, bank_lanes, msent, spread, sc) / 8;
        sched[s].swap(sc.out);
        nvi[s] = (imax + 3) / 4;
        mv += 32 * nvm[s];
        iv += 32 * nvi[s];
    }
    tb.nsl = (int32_t)nsl;
    tb.vtab_off = 0;
    tb.mvec_off = (uint32_t)(144 * nsl);
    tb.ivec_off = tb.mvec_off + (uint32_t)(16 * mv);
    tb.bytes.assign(tb.ivec_off + 16 * iv, 0);
    uint32_t *desc = reinterpret_cast<uint32_t *>(tb.bytes.data());
    uint32_t *rows = reinterpret_cast<uint32_t *>(tb.bytes.data() + 16 * nsl);
    uint16_t *mvec = reinterpret_cast<uint16_t *>(tb.bytes.data() + tb.mvec_off);
    int32_t *ivec = reinterpret_cast<int32_t *>(tb.bytes.data() + tb.ivec_off);
    mv = iv = 0;
    for (int64_t s = 0; s < nsl; ++s) {
        desc[4 * s + 0] = (uint32_t)mv;
        desc[4 * s + 1] = (uint32_t)nvm[s];
        desc[4 * s + 2] = (uint32_t)iv;
        desc[4 * s + 3] = (uint32_t)nvi[s];
        for (int lane = 0; lane < 32; ++lane) {
            const Lane &L = sl[s][lane];
            rows[32 * s + lane] = L.row < 0 ? 0xffffffffu
                                            : (uint32_t)L.row | ((uint32_t)L.v << 16) | ((uint32_t)L.part << 22);
            const bool head = L.row >= 0 && L.part == 0;
            for (int64_t j = 0; j < nvi[s]; ++j)
                for (int h = 0; h < 4; ++h) {
                    const int64_t e = 4 * j + h;
                    const bool has = head && e < inter_cnt[f + L.row];
                    ivec[4 * (iv + 32 * j + lane) + h] = has ? inter_col[inter_off[f + L.row] + e] : inter_sent;
                }
            for (int64_t p = 0; p < 8 * nvm[s]; ++p)
                mvec[8 * (mv + 32 * (p / 8) + lane) + (p % 8)] = sched[s][(size_t)p * 32 + lane];
        }
        mv += 32 * nvm[s];
        iv += 32 * nvi[s];
    }
}

// Options and model of a plan (no graph yet); has_omega: natural
// frequencies are given.
static cia_status configure(const cia_coupling *cp, const cia_options *opt, bool has_omega, cia_plan *pl) {
    pl->precision = opt ? opt->precision : CIA_FP64;
    if (pl->precision != CIA_FP64 && pl->precision != CIA_FP32)
        return fail(CIA_ERR_INVALID_ARG, "unknown precision");
    pl->has_direct = opt ? (opt->build_direct != 0) : 0;
    pl->tile_nodes = (opt && opt->tile_nodes) ? opt->tile_nodes : 256;
    if (pl->tile_nodes < 32 || pl->tile_nodes > 1024 || pl->tile_nodes % 32)
        return fail(CIA_ERR_INVALID_ARG, "tile_nodes must be a multiple of 32 in [32, 1024]");
    pl->tile_index_bytes = (opt && opt->tile_index_bytes) ? opt->tile_index_bytes : 65536;
    if (pl->tile_index_bytes < 256 || pl->tile_index_bytes % 16)
        return fail(CIA_ERR_INVALID_ARG, "tile_index_bytes must be a multiple of 16, at least 256");
    pl->staging = opt ? opt->staging : 0;
    if (pl->staging < 0 || pl->staging > 4) return fail(CIA_ERR_INVALID_ARG, "staging must be 0, 1, 2, 3 or 4");
    pl->use_graphs = opt ? opt->use_graphs : 0;
    if (pl->use_graphs != 0 && pl->use_graphs != 1) return fail(CIA_ERR_INVALID_ARG, "use_graphs must be 0 or 1");
    if (cp->model != CIA_MODEL_KURAMOTO && cp->model != CIA_MODEL_KURAMOTO_HO &&
        cp->model != CIA_MODEL_CUCKER_SMALE && cp->model != CIA_MODEL_POLYNOMIAL &&
        cp->model != CIA_MODEL_POLYNOMIAL_GENERAL && cp->model != CIA_MODEL_FOURIER_GENERAL)
        return fail(CIA_ERR_UNSUPPORTED, "unknown model");
    if (cp->model == CIA_MODEL_POLYNOMIAL || cp->model == CIA_MODEL_POLYNOMIAL_GENERAL ||
        cp->model == CIA_MODEL_FOURIER_GENERAL) {
        const bool general = cp->model == CIA_MODEL_POLYNOMIAL_GENERAL;
        const bool fourier = cp->model == CIA_MODEL_FOURIER_GENERAL;
        if (pl->precision != CIA_FP64)
            return fail(CIA_ERR_UNSUPPORTED, "the polynomial and Fourier couplings run in FP64 (precision CIA_FP64)");
        if (has_omega) return fail(CIA_ERR_INVALID_ARG, "omega must be NULL for the polynomial and Fourier couplings");
        if (!fourier && (cp->p < 0 || cp->p > CIA_MAX_POLY))
            return fail(CIA_ERR_INVALID_ARG, "p must be in [0, CIA_MAX_POLY]");
        if (fourier && (cp->p < 1 || cp->p > CIA_MAX_HARMONICS))
            return fail(CIA_ERR_INVALID_ARG, "p must be in [1, CIA_MAX_HARMONICS]");
        if (!std::isfinite(cp->K)) return fail(CIA_ERR_NUMERIC, "K is not finite");
        constexpr int S = CIA_MAX_POLY + 1, SH = CIA_MAX_HARMONICS + 1;
        for (int k = 0; k < S; ++k) {
            if ((!general && !fourier && !std::isfinite(cp->poly_c[k])) || !std::isfinite(cp->dV[k]))
                return fail(CIA_ERR_NUMERIC, "a polynomial coefficient is not finite");
            for (int b = 0; general && b < S; ++b)
                if (!std::isfinite(cp->poly_g[k * S + b]))
                    return fail(CIA_ERR_NUMERIC, "a polynomial coefficient is not finite");
        }
        if (fourier) {
            if (!std::isfinite(cp->fourier_L) || !(cp->fourier_L > 0.0))
                return fail(CIA_ERR_INVALID_ARG, "fourier_L must be positive and finite");
            for (int q = 0; q < 4; ++q)
                for (int i = 0; i < SH * SH; ++i)
                    if (!std::isfinite(cp->fourier_c[q][i]))
                        return fail(CIA_ERR_NUMERIC, "a Fourier coefficient is not finite");
        }
        if (pl->tile_nodes > 256)
            return fail(CIA_ERR_INVALID_ARG, "tile_nodes must be <= 256 for the polynomial and Fourier couplings");
        pl->model = CIA_MODEL_POLYNOMIAL;   // one kernel family for the three
        pl->poly_general = general;
        pl->gc_basis = fourier ? 1 : 0;
        pl->p = 1;
        pl->poly_p = fourier ? cp->p : std::max(cp->p, 1);   // degree 1..4 (coefficients above p are zero)
        pl->gc_k = fourier ? 2 * cp->p + 1 : pl->poly_p + 1;
        for (int k = 0; k < S; ++k) {
            pl->poly_c[k] = !general && !fourier && k <= cp->p ? cp->poly_c[k] : 0.0;
            pl->poly_dv[k] = cp->dV[k];
            for (int b = 0; b < S; ++b)
                pl->poly_g[k * S + b] = general && k <= cp->p && b <= cp->p ? cp->poly_g[k * S + b] : 0.0;
        }
        // g(u, y) = sum_{k,j} E_kj phi_k(u) phi_j(y)
        constexpr int F = CIA_GC_MAX_FEATURES;
        std::fill(pl->gc_e, pl->gc_e + F * F, 0.0);
        if (fourier) {
            // phi = (1, cos wu, sin wu, cos 2wu, ...): cos(a w u) is feature 2a - 1
            // (the constant for a = 0), sin(a w u) feature 2a; sin 0 = 0 drops out
            pl->gc_w = 3.14159265358979323846 / cp->fourier_L;
            auto ci = [](int a) { return a == 0 ? 0 : 2 * a - 1; };
            auto si = [](int a) { return 2 * a; };
            for (int a = 0; a <= cp->p; ++a)
                for (int b = 0; b <= cp->p; ++b) {
                    const int i = a * SH + b;
                    pl->gc_e[ci(a) * F + ci(b)] += cp->fourier_c[0][i];
                    if (b) pl->gc_e[ci(a) * F + si(b)] += cp->fourier_c[1][i];
                    if (a) pl->gc_e[si(a) * F + ci(b)] += cp->fourier_c[2][i];
                    if (a && b) pl->gc_e[si(a) * F + si(b)] += cp->fourier_c[3][i];
                }
        } else {
            // G itself, or h(u - y) = sum_a c_a (u - y)^a regrouped by the power of u:
            // E_kj = c_{k+j} binom(k+j, k) (-1)^j
            for (int k = 0; k < S; ++k)
                for (int j = 0; j < S; ++j) {
                    if (general) {
                        pl->gc_e[k * F + j] = pl->poly_g[k * S + j];
                    } else if (k + j < S) {
                        double binom = 1.0;
                        for (int q = 1; q <= k; ++q) binom = binom * (double)(j + q) / (double)q;
                        pl->gc_e[k * F + j] = pl->poly_c[k + j] * binom * ((j & 1) ? -1.0 : 1.0);
                    }
                }
        }
        pl->K = cp->K;
    } else if (cp->model == CIA_MODEL_CUCKER_SMALE) {
        if (pl->precision != CIA_FP32)
            return fail(CIA_ERR_UNSUPPORTED, "the Cucker-Smale model runs in FP32 (precision CIA_FP32)");
        if (has_omega) return fail(CIA_ERR_INVALID_ARG, "omega must be NULL for the Cucker-Smale model");
        if (!std::isfinite(cp->K) || !std::isfinite(cp->sigma) || !std::isfinite(cp->beta))
            return fail(CIA_ERR_NUMERIC, "K, sigma or beta is not finite");
        if (!(cp->sigma > 0.0)) return fail(CIA_ERR_INVALID_ARG, "sigma must be positive");
        if (!(opt && opt->tile_nodes)) pl->tile_nodes = 128;
        if (pl->tile_nodes > 128)
            return fail(CIA_ERR_INVALID_ARG, "tile_nodes must be <= 128 for the Cucker-Smale model");
        pl->model = cp->model;
        pl->state_dim = 4;
        pl->p = 1;
        pl->K = cp->K;
        pl->cs_sigma = cp->sigma;
        pl->cs_beta = cp->beta;
        pl->staging = 1;   // the TMA-pipelined stage kernel is the Kuramoto one
    } else {
    if (cp->p < 1 || cp->p > CIA_MAX_HARMONICS)
        return fail(CIA_ERR_INVALID_ARG, "p must be in [1, CIA_MAX_HARMONICS]");
    pl->model = cp->model;
    pl->triadic = cp->model == CIA_MODEL_KURAMOTO_HO;
    // the higher-order model needs the second-harmonic moments Z_2: carry at
    // least two harmonics (extra ones with zero coefficients)
    pl->p = pl->triadic ? std::max(cp->p, 2) : cp->p;
    pl->K = cp->K;
    pl->K2 = pl->triadic ? cp->K2 : 0.0;
    if (!std::isfinite(cp->K)) return fail(CIA_ERR_NUMERIC, "K is not finite");
    if (pl->triadic && !std::isfinite(cp->K2)) return fail(CIA_ERR_NUMERIC, "K2 is not finite");
    for (int k = 0; k < cp->p; ++k) {
        if (!std::isfinite(cp->d_sin[k]) || !std::isfinite(cp->d_cos[k]))
            return fail(CIA_ERR_NUMERIC, "coupling coefficient is not finite");
        pl->d_sin[k] = cp->d_sin[k];
        pl->d_cos[k] = cp->d_cos[k];
    }
    for (int k = cp->p; k < CIA_MAX_HARMONICS; ++k) pl->d_sin[k] = pl->d_cos[k] = 0.0;
    }
    return CIA_OK;
}

// Validation of A, kappa and the split of S into the host lists kept by the
// plan (pl->hs) and, with the direct method, its padded permuted CSR.
static cia_status split_graph(const cia_graph *g, const int32_t *community, cia_plan *pl,
                              std::vector<int64_t> &full_rp, std::vector<int32_t> &full_col) {
    const int64_t n = g->n;
    // ---- validate A
    cia_status st = validate_graph(g);
    if (st != CIA_OK) return st;
    pl->n = n;
    pl->nnz_graph = g->rowptr[n];
    pl->ph_stride = (n + 2) & ~(int64_t)1;

    // ---- labels, kappa (stable counting sort by label, unlabelled last)
    int64_t M = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (community[i] < -1)
            return fail(CIA_ERR_INVALID_ARG, "community label below -1 at node " + std::to_string(i));
        M = std::max<int64_t>(M, (int64_t)community[i] + 1);
    }
    pl->M = M;
    std::vector<int64_t> cnt(M + 2, 0);
    for (int64_t i = 0; i < n; ++i) cnt[(community[i] < 0 ? M : community[i]) + 1]++;
    for (int64_t c = 0; c <= M; ++c) cnt[c + 1] += cnt[c];
    pl->off.assign(cnt.begin(), cnt.begin() + M + 1);
    pl->n_free = n - pl->off[M];
    pl->perm.assign(n, 0);
    {
        std::vector<int64_t> pos(cnt.begin(), cnt.end() - 1);
        for (int64_t i = 0; i < n; ++i) pl->perm[pos[community[i] < 0 ? M : community[i]]++] = (int32_t)i;
    }
    std::vector<int32_t> iperm(n);
    for (int64_t m = 0; m < n; ++m) iperm[pl->perm[m]] = (int32_t)m;
    pl->max_comm = 0;
    for (int64_t c = 0; c < M; ++c) pl->max_comm = std::max(pl->max_comm, pl->off[c + 1] - pl->off[c]);
    pl->miss_idx_bytes = pl->max_comm <= 65535 ? 2 : 4;
    auto &hs = pl->hs;
    hs.comm_of.assign(n, -1);
    auto &comm_of = hs.comm_of;
    for (int64_t c = 0; c < M; ++c)
        for (int64_t m = pl->off[c]; m < pl->off[c + 1]; ++m) comm_of[m] = (int32_t)c;

    // ---- pass 1: per-row counts of missing and inter links
    hs.miss_cnt.assign(n, 0);
    hs.inter_cnt.assign(n, 0);
    auto &miss_cnt = hs.miss_cnt;
    auto &inter_cnt = hs.inter_cnt;
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t m = 0; m < n; ++m) {
        int32_t i = pl->perm[m];
        int32_t c = comm_of[m];
        int64_t inside = 0, deg = g->rowptr[i + 1] - g->rowptr[i];
        if (c >= 0) {
            int64_t lo = pl->off[c], hi = pl->off[c + 1];
            for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
                int64_t pm = iperm[g->col[e]];
                inside += (pm >= lo && pm < hi);
            }
            miss_cnt[m] = (hi - lo - 1) - inside;
        }
        inter_cnt[m] = deg - inside;
    }
    auto pad4 = [](int64_t x) { return (x + 3) & ~(int64_t)3; };
    hs.miss_off.assign(n + 1, 0);
    hs.inter_off.assign(n + 1, 0);
    auto &miss_off = hs.miss_off;
    auto &inter_off = hs.inter_off;
    full_rp.clear();
    for (int64_t m = 0; m < n; ++m) {
        miss_off[m + 1] = miss_off[m] + miss_cnt[m];
        inter_off[m + 1] = inter_off[m] + inter_cnt[m];
    }
    pl->nnz_missing = miss_off[n];
    pl->nnz_inter = inter_off[n];
    if (pl->has_direct) {
        full_rp.assign(n + 1, 0);
        for (int64_t m = 0; m < n; ++m) {
            int32_t i = pl->perm[m];
            full_rp[m + 1] = full_rp[m] + pad4(g->rowptr[i + 1] - g->rowptr[i]);
        }
    }

    // ---- pass 2: the lists themselves (missing as community-local indices),
    // ascending within each row
    hs.miss_local.assign(pl->miss_idx_bytes == 2 ? miss_off[n] : 0, 0);
    hs.inter_col.assign(inter_off[n], 0);
    auto &miss_local = hs.miss_local;
    auto &inter_col = hs.inter_col;
    full_col.assign(pl->has_direct ? full_rp[n] : 0, 0);
#pragma omp parallel
    {
        std::vector<unsigned char> mark(pl->max_comm + 1, 0);
        std::vector<int32_t> outside;
#pragma omp for schedule(dynamic, 1024)
        for (int64_t m = 0; m < n; ++m) {
            int32_t i = pl->perm[m];
            int32_t c = comm_of[m];
            int64_t lo = c >= 0 ? pl->off[c] : 0, hi = c >= 0 ? pl->off[c + 1] : 0;
            outside.clear();
            for (int64_t e = g->rowptr[i]; e < g->rowptr[i + 1]; ++e) {
                int64_t pm = iperm[g->col[e]];
                if (c >= 0 && pm >= lo && pm < hi) mark[pm - lo] = 1;
                else outside.push_back((int32_t)pm);
            }
            std::sort(outside.begin(), outside.end());
            std::copy(outside.begin(), outside.end(), inter_col.begin() + inter_off[m]);
            int64_t w = miss_off[m];
            int64_t f = pl->has_direct ? full_rp[m] : 0;
            size_t oi = 0;
            if (c >= 0) {
                for (int64_t u = 0; u < hi - lo; ++u) {
                    if (mark[u]) {
                        if (pl->has_direct) {
                            while (oi < outside.size() && outside[oi] < lo + u) full_col[f++] = outside[oi++];
                            full_col[f++] = (int32_t)(lo + u);
                        }
                        mark[u] = 0;
                    } else if (lo + u != m) {
                        if (pl->miss_idx_bytes == 2) miss_local[w++] = (uint16_t)u;
                    }
                }
            }
            if (pl->has_direct) {
                while (oi < outside.size()) full_col[f++] = outside[oi++];
                while (f < full_rp[m + 1]) full_col[f++] = (int32_t)n;
            }
        }
    }

    return CIA_OK;
}

// Every device buffer of a plan that does not depend on the tiling, after
// its split; omega_perm: natural frequencies in permuted order (NULL: zero).
static cia_status upload_split(cia_plan *pl, const cia_options *opt, const double *omega_perm,
                               const std::vector<int64_t> &full_rp, const std::vector<int32_t> &full_col) {
    const int64_t n = pl->n, M = pl->M;
    const auto &comm_of = pl->hs.comm_of;
    // ---- default threads per row of the direct method (16-byte vectors;
    // about two vectors per thread)
    const int gs = opt ? opt->group_size : 0;
    if (gs != 0 && gs != 4 && gs != 8 && gs != 16 && gs != 32)
        return fail(CIA_ERR_INVALID_ARG, "group_size must be 0, 4, 8, 16 or 32");
    pl->group_size = 32;
    if (pl->has_direct) {
        double mean_vec_direct = (double)(full_rp[n] / 4) / (double)std::max<int64_t>(1, n);
        int gd = 4;
        while (gd < 32 && 2.0 * gd < mean_vec_direct) gd *= 2;
        pl->group_size_direct = gs ? gs : gd;
    }

    // ---- upload
    CIA_CUDA_TRY(cudaGetDevice(&pl->device));
    auto &d = pl->d;
#define UP(dst, src, cnt)                                  \
    do {                                                   \
        cia_status _s = upload(pl, &(dst), (src), (cnt));  \
        if (_s != CIA_OK) return _s;                       \
    } while (0)
    UP(d.perm, pl->perm.data(), (size_t)n);
    UP(d.off, pl->off.data(), (size_t)M + 1);
    if (pl->has_direct) {
        UP(d.full_rowptr, full_rp.data(), full_rp.size());
        UP(d.full_col, full_col.data(), full_col.size());
    }
    const size_t rb = pl->precision == CIA_FP64 ? sizeof(double) : sizeof(float);
    {
        std::vector<unsigned char> om(n * rb, 0);
        for (int64_t m = 0; m < n; ++m) {
            double w = omega_perm ? omega_perm[m] : 0.0;
            if (rb == sizeof(double)) std::memcpy(&om[m * rb], &w, rb);
            else {
                float wf = (float)w;
                std::memcpy(&om[m * rb], &wf, rb);
            }
        }
        unsigned char *po = nullptr;
        UP(po, om.data(), om.size());
        d.omega = po;
    }
    cia_status s2;
    CIA_CUDA_TRY(cudaDeviceGetAttribute(&pl->n_sms, cudaDevAttrMultiProcessorCount, pl->device));
    CIA_CUDA_TRY(cudaDeviceGetAttribute(&pl->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
    CIA_CUDA_TRY(cudaDeviceGetAttribute(&pl->smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, pl->device));
    if ((s2 = upload<double>(pl, &d.rhs_tmp, nullptr, (size_t)n * pl->state_dim)) != CIA_OK) return s2;
    if ((s2 = upload<double>(pl, &d.x_tmp, nullptr, (size_t)n * pl->state_dim)) != CIA_OK) return s2;
    // the error flag lives in mapped pinned host memory: kernels that give up a
    // bounded wait set it through its device alias, cia_sync reads it after
    // synchronising without a copy
    if (!d.err_flag_host) {
        CIA_CUDA_TRY(cudaHostAlloc((void **)&d.err_flag_host, sizeof(int), cudaHostAllocMapped));
        *d.err_flag_host = 0;
        CIA_CUDA_TRY(cudaHostGetDevicePointer((void **)&d.err_flag, d.err_flag_host, 0));
    }
    if ((s2 = upload<int64_t>(pl, &d.r_counter, nullptr, 1)) != CIA_OK) return s2;
    if (pl->B > 1) UP(d.inst_off, pl->inst_off.data(), pl->inst_off.size());
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        for (int b = 0; b < 2; ++b)
            if ((s2 = alloc_bytes(pl, (void **)&d.cs_y[b], (size_t)(n + 1) * sizeof(float4))) != CIA_OK) return s2;
        if ((s2 = upload<double>(pl, &d.cs_master, nullptr, (size_t)n * 4)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, (void **)&d.cs_acc, (size_t)n * sizeof(float4))) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, &d.cs_feat, (size_t)n * CIA_BASIS_RANK * 2)) != CIA_OK) return s2;
        if ((s2 = upload<float>(pl, &d.cs_params, nullptr, CIA_BASIS_PARAMS)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, (void **)&d.cs_cen, (size_t)std::max<int64_t>(M, 1) * sizeof(float2))) != CIA_OK)
            return s2;
        if ((s2 = alloc_bytes(pl, (void **)&d.cs_shift, (size_t)std::max<int64_t>(M, 1) * sizeof(float2))) != CIA_OK)
            return s2;
        // nodes of the learned-basis check: evenly spaced over the community nodes
        const int64_t nc = pl->off[M];
        pl->cs_check_count = std::min<int64_t>(512, nc);
        std::vector<int32_t> cn(pl->cs_check_count), cc(pl->cs_check_count);
        for (int64_t k = 0; k < pl->cs_check_count; ++k) {
            cn[k] = (int32_t)((2 * k + 1) * nc / (2 * pl->cs_check_count));
            cc[k] = comm_of[cn[k]];
        }
        UP(d.cs_check_nodes, cn.data(), cn.size());
        UP(d.cs_check_comm, cc.data(), cc.size());
        if ((s2 = upload<double>(pl, &d.cs_check_out, nullptr, (size_t)std::max<int64_t>(1, pl->cs_check_count) * 2)) !=
            CIA_OK)
            return s2;
    }
    if (pl->model == CIA_MODEL_POLYNOMIAL) {
        if ((s2 = upload<double>(pl, &d.theta, nullptr, n)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, &d.acc, n * sizeof(double))) != CIA_OK) return s2;
        for (int b = 0; b < 2; ++b)
            if ((s2 = upload<double>(pl, &d.gc_y[b], nullptr, (size_t)n + 1)) != CIA_OK) return s2;
        if (pl->gc_basis == 1)
            for (int b = 0; b < 2; ++b)
                if ((s2 = upload<double>(pl, &d.gc_f[b], nullptr, (size_t)n * (pl->gc_k - 1))) != CIA_OK) return s2;
    } else if (pl->model != CIA_MODEL_CUCKER_SMALE) {
        if ((s2 = upload<double>(pl, &d.theta, nullptr, n)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, &d.acc, n * rb)) != CIA_OK) return s2;
        for (int b = 0; b < 2; ++b)
            if ((s2 = alloc_bytes(pl, &d.ph[b], (size_t)pl->p * pl->ph_stride * 2 * rb)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, &d.wdt_half, n * rb)) != CIA_OK) return s2;
        if ((s2 = alloc_bytes(pl, &d.wdt_full, n * rb)) != CIA_OK) return s2;
        if ((s2 = upload<double>(pl, &d.wdt_full64, nullptr, n)) != CIA_OK) return s2;
        if (pl->triadic && pl->has_direct && (s2 = alloc_bytes(pl, &d.tri, n * rb)) != CIA_OK) return s2;
    }
#undef UP
    return CIA_OK;
}

// Phase 1 of planning: options, model, validation, kappa and the split of S
// into the host lists kept by the plan (pl->hs), the direct method's CSR and
// every device buffer that does not depend on the tiling.
static cia_status build_split(const cia_graph *g, const int32_t *community, const double *omega,
                              const cia_coupling *cp, const cia_options *opt, cia_plan *pl) {
    cia_status st = configure(cp, opt, omega != nullptr, pl);
    if (st != CIA_OK) return st;
    const int64_t n = g->n;
    if (omega)
        for (int64_t i = 0; i < n; ++i)
            if (!std::isfinite(omega[i]))
                return fail(CIA_ERR_NUMERIC, "omega[" + std::to_string(i) + "] is not finite");
    std::vector<int64_t> full_rp;
    std::vector<int32_t> full_col;
    if ((st = split_graph(g, community, pl, full_rp, full_col)) != CIA_OK) return st;
    std::vector<double> om;
    if (omega) {
        om.resize(n);
        for (int64_t m = 0; m < n; ++m) om[m] = omega[pl->perm[m]];
    }
    return upload_split(pl, opt, omega ? om.data() : nullptr, full_rp, full_col);
}

// Phase 2 of planning: cut the communities into work tiles, build the
// sliced-ELL blobs and every device buffer whose size depends on the tiling.
// Runs again (after freeing the previous tiling) when the tiling changes.
static cia_status build_tiles(cia_plan *pl) {
    const int64_t n = pl->n, M = pl->M;
    auto &hs = pl->hs;
    const auto &miss_cnt = hs.miss_cnt;
    const auto &miss_off = hs.miss_off;
    const auto &miss_local = hs.miss_local;
    const auto &inter_cnt = hs.inter_cnt;
    const auto &inter_off = hs.inter_off;
    const auto &inter_col = hs.inter_col;
    for (void *p : pl->tile_allocs) cudaFree(p);
    pl->device_bytes -= pl->tile_bytes;
    pl->tile_allocs.clear();
    pl->tile_bytes = 0;
    pl->staging = pl->staging_req;
    pl->n_ctas = 0;
    pl->max_cta_tiles = pl->max_cta_runs = 0;
    invalidate_graphs(pl);
    auto pad4 = [](int64_t x) { return (x + 3) & ~(int64_t)3; };
    auto pad8 = [](int64_t x) { return (x + 7) & ~(int64_t)7; };
    // ---- tiles: runs of consecutive rows of one community, cut at tile_nodes
    // rows or when the rows' sparse indices (padded to 16-byte vectors) would
    // exceed tile_index_bytes; a single longer row forms a tile of its own
    std::vector<int32_t> tile_comm, tile_first, tile_count, comm_tile_begin(M + 1, 0);
    // the persistent per-tile kernel (staging 4) holds a tile's community
    // window and its blob in one shared-memory buffer of tile_index_bytes: the
    // window of a large community leaves less room for the tile's indices
    const bool budget_window = pl->staging_req == 4;
    auto cut = [&](int32_t c, int64_t b, int64_t e) {
        int64_t limit = pl->tile_index_bytes;
        if (budget_window)
            limit = std::max<int64_t>(2048, limit - stream_tile_buf_bytes(pl, c >= 0 ? pl->off[c + 1] - pl->off[c] : 0, 0));
        int64_t s = b;
        while (s < e) {
            int64_t rows = 0, bytes = 0, r = s;
            int64_t chunks = 0;
            while (r < e && rows < pl->tile_nodes) {
                // index vectors, plus (staging 4) the row's share of the blob's tables
                int64_t rb = pad8(miss_cnt[r]) * 2 + pad4(inter_cnt[r]) * 4 + (budget_window ? 9 : 0);
                int64_t rc = budget_window ? seg_lanes(miss_cnt[r]) : chunks_of(miss_cnt[r]);
                if (rows > 0 && (bytes + rb > limit || chunks + rc > kMaxChunks)) break;
                bytes += rb;
                chunks += rc;
                ++rows;
                ++r;
            }
            tile_comm.push_back(c);
            tile_first.push_back((int32_t)s);
            tile_count.push_back((int32_t)rows);
            s = r;
        }
    };
    for (int64_t c = 0; c < M; ++c) {
        comm_tile_begin[c] = (int32_t)tile_comm.size();
        cut((int32_t)c, pl->off[c], pl->off[c + 1]);
    }
    comm_tile_begin[M] = (int32_t)tile_comm.size();
    // nodes without a community: never a tile across two instances of a batch
    {
        int64_t s = pl->off[M];
        while (s < n) {
            const int64_t inst = instance_of_node(pl, pl->perm[s]);
            int64_t e = s + 1;
            while (e < n && instance_of_node(pl, pl->perm[e]) == inst) ++e;
            cut(-1, s, e);
            s = e;
        }
    }
    const int64_t T = (int64_t)tile_comm.size();
    pl->n_tiles = T;

    // ---- sliced ELL per tile, one blob per tile (only with 16-bit
    // community-local indices; larger communities have no CIA layout)
    std::vector<TileDesc> tdesc(T);
    std::vector<unsigned char> blob;
    pl->max_tile_idx_bytes = 0;
    std::vector<int64_t> tile_bytes(T, 0);
    pl->blob_segmented = false;
    // the persistent ring kernel (staging 4) reads rows' chunks from consecutive
    // lanes; when its ring does not fit, the chunk layout of the other kernels
    // is built instead
    for (int attempt = 0; attempt < 2 && pl->miss_idx_bytes == 2; ++attempt) {
        // (the ring kernel needs tiles of at most 256 rows and spread padding)
        const bool segmented = attempt == 0 && pl->staging_req == 4 && pl->tile_nodes <= 256 &&
                               pl->max_comm + kPadSlots <= 65535;
        pl->max_tile_idx_bytes = 0;
        std::vector<TileBlob> tbs(T);
#pragma omp parallel
        {
            MissScheduler sched;
#pragma omp for schedule(dynamic, 8)
            for (int64_t t = 0; t < T; ++t) {
                const int32_t c = tile_comm[t];
                const int64_t lam = c >= 0 ? pl->off[c + 1] - pl->off[c] : 0;
                const uint16_t msent = (uint16_t)lam;
                // bank groups of the gathered element: 16-byte elements (Cucker--Smale
                // states, FP64 phasors, the general couplings' node-major windows of
                // two or more fixed-point features) are served per quarter-warp,
                // 8-byte ones per half-warp
                const bool wide = pl->model == CIA_MODEL_CUCKER_SMALE ||
                                  (pl->model != CIA_MODEL_POLYNOMIAL && pl->precision == CIA_FP64) ||
                                  (pl->model == CIA_MODEL_POLYNOMIAL && pl->gc_k >= 3);
                const int bank_lanes = wide ? 8 : 16;
                // padding entries lambda + 1 .. lambda + 16 (zero slots after the window)
                const bool spread = lam + kPadSlots <= 65535;
                if (segmented)
                    build_tile_blob_seg(tile_first[t], tile_count[t], msent, spread, (int32_t)n, bank_lanes, miss_cnt,
                                        miss_off, miss_local, inter_cnt, inter_off, inter_col, tbs[t], sched);
                else
                    build_tile_blob(tile_first[t], tile_count[t], msent, spread, (int32_t)n, bank_lanes, miss_cnt,
                                    miss_off, miss_local, inter_cnt, inter_off, inter_col, tbs[t], sched);
            }
        }
        std::vector<int64_t> blob_off(T + 1, 0);
        for (int64_t t = 0; t < T; ++t) blob_off[t + 1] = blob_off[t] + (int64_t)tbs[t].bytes.size();
        blob.assign(blob_off[T], 0);
        const int64_t per16 = pl->precision == CIA_FP64 ? 1 : 2;
        pl->n_slices = 0;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t t = 0; t < T; ++t) {
            std::memcpy(blob.data() + blob_off[t], tbs[t].bytes.data(), tbs[t].bytes.size());
            tile_bytes[t] = (int64_t)tbs[t].bytes.size();
            std::vector<unsigned char>().swap(tbs[t].bytes);
            TileDesc &d = tdesc[t];
            d.comm = tile_comm[t];
            d.first = tile_first[t];
            d.count = tile_count[t];
            d.nsl = tbs[t].nsl;
            d.blob_bytes = (uint32_t)tile_bytes[t];
            d.mvec_off = tbs[t].mvec_off;
            d.ivec_off = tbs[t].ivec_off;
            d.lam = d.comm >= 0 ? (uint32_t)(pl->off[d.comm + 1] - pl->off[d.comm]) : 0u;
            d.blob_off = blob_off[t];
            d.lo = d.comm >= 0 ? pl->off[d.comm] : 0;
            d.run = -1;
            d.pbuf = 0;
            d.shift = (int32_t)(d.lo - (d.lo & ~(per16 - 1)));
            d.vtab_off = tbs[t].vtab_off;
        }
        pl->max_tile_buf = 0;
        for (int64_t t = 0; t < T; ++t) {
            pl->max_tile_idx_bytes = std::max<int64_t>(pl->max_tile_idx_bytes, tile_bytes[t]);
            pl->max_tile_buf = std::max<int64_t>(
                pl->max_tile_buf,
                stream_tile_buf_bytes(pl, tile_comm[t] >= 0 ? pl->off[tile_comm[t] + 1] - pl->off[tile_comm[t]] : 0,
                                      tile_bytes[t]));
            pl->n_slices += tbs[t].nsl;
        }
        pl->blob_bytes = blob_off[T];
        pl->blob_segmented = segmented;
        bool slices_fit = true;
        for (int64_t t = 0; t < T && segmented; ++t) slices_fit = slices_fit && tdesc[t].nsl <= kRingMaxSlices;
        if (!segmented || (slices_fit && ring_slots_that_fit(pl) >= 2)) break;
    }

    // ---- upload
    auto &d = pl->d;
#define UPT(dst, src, cnt)                                       \
    do {                                                         \
        cia_status _s = upload(pl, &(dst), (src), (cnt), true);  \
        if (_s != CIA_OK) return _s;                             \
    } while (0)
    UPT(d.tile_comm, tile_comm.data(), tile_comm.size());
    UPT(d.tile_first, tile_first.data(), tile_first.size());
    UPT(d.tile_count, tile_count.data(), tile_count.size());
    UPT(d.comm_tile_begin, comm_tile_begin.data(), comm_tile_begin.size());
    UPT(d.blob, blob.data(), blob.size());
    cia_status s2;
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        for (int b = 0; b < 2; ++b)
            if ((s2 = upload<double>(pl, &d.cs_part[b], nullptr, (size_t)T * 3 * CIA_BASIS_RANK, true)) != CIA_OK)
                return s2;
        pl->cs_feat_valid = false;
    } else if (pl->model == CIA_MODEL_POLYNOMIAL) {
        for (int b = 0; b < 2; ++b)
            if ((s2 = upload<double>(pl, &d.gc_part[b], nullptr, (size_t)T * pl->gc_k, true)) != CIA_OK)
                return s2;
    } else {
        for (int b = 0; b < 2; ++b)
            if ((s2 = upload<double>(pl, &d.part[b], nullptr, (size_t)T * pl->p * 2, true)) != CIA_OK) return s2;
        // community observables written by the ring kernel (staging 4) for the next stage
        for (int b = 0; b < 2; ++b)
            if ((s2 = upload<double>(pl, &d.zsum[b], nullptr, (size_t)std::max<int64_t>(M, 1) * pl->p * 2, true)) !=
                CIA_OK)
                return s2;
        if ((s2 = upload<int>(pl, &d.comm_done, nullptr, (size_t)std::max<int64_t>(M, 1), true)) != CIA_OK) return s2;
    }
    // ensembles: K / N_i per tile and each instance's tile ranges
    if (pl->B > 1) {
        const size_t rb = pl->precision == CIA_FP64 ? sizeof(double) : sizeof(float);
        std::vector<unsigned char> kn(T * rb);
        std::vector<int32_t> itab(4 * pl->B, 0);
        for (int64_t i = 0; i < pl->B; ++i) {
            itab[4 * i + 0] = comm_tile_begin[pl->inst_comm_off[i]];
            itab[4 * i + 1] = comm_tile_begin[pl->inst_comm_off[i + 1]];
            itab[4 * i + 2] = itab[4 * i + 3] = (int32_t)T;
        }
        for (int64_t t = 0; t < T; ++t) {
            const int64_t inst = instance_of_node(pl, pl->perm[tile_first[t]]);
            const double v = pl->K / (double)(pl->inst_off[inst + 1] - pl->inst_off[inst]);
            if (rb == sizeof(double)) std::memcpy(&kn[t * rb], &v, rb);
            else {
                const float f = (float)v;
                std::memcpy(&kn[t * rb], &f, rb);
            }
            if (tile_comm[t] < 0) {
                if (itab[4 * inst + 2] == (int32_t)T) itab[4 * inst + 2] = (int32_t)t;
                itab[4 * inst + 3] = (int32_t)t + 1;
            }
        }
        for (int64_t i = 0; i < pl->B; ++i)
            if (itab[4 * i + 2] == (int32_t)T) itab[4 * i + 2] = itab[4 * i + 3] = 0;
        unsigned char *pk = nullptr;
        UPT(pk, kn.data(), kn.size());
        d.tile_kn = pk;
        UPT(d.inst_tiles, itab.data(), itab.size());
    }
    if (pl->model == CIA_MODEL_POLYNOMIAL) {
        // its own one-CTA-per-tile kernel: community window in shared memory
        // (auto, window, pipeline) or plain loads (plain); the window launches
        // take the tiles by community size, largest first, so that each run
        // of tiles gets a window sized to its largest community
        pl->staging = pl->staging == 1 ? 1 : 2;
        std::vector<int32_t> order(T);
        for (int64_t t = 0; t < T; ++t) order[t] = (int32_t)t;
        auto lam_of = [&](int32_t t) { return tdesc[t].comm >= 0 ? (int64_t)tdesc[t].lam : (int64_t)0; };
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return lam_of(x) > lam_of(y); });
        pl->gc_tile_lam.resize(T);
        for (int64_t i = 0; i < T; ++i) pl->gc_tile_lam[i] = lam_of(order[i]);
        UPT(d.gc_tiles, order.data(), order.size());
        // the runs' launches fork from the caller's stream and join it again
        // (created here, outside any graph capture)
        if (!pl->gc_fork) {
            CIA_CUDA_TRY(cudaEventCreateWithFlags(&pl->gc_fork, cudaEventDisableTiming));
            for (int i = 0; i < 4; ++i) {
                CIA_CUDA_TRY(cudaStreamCreateWithFlags(&pl->gc_side[i], cudaStreamNonBlocking));
                CIA_CUDA_TRY(cudaEventCreateWithFlags(&pl->gc_join[i], cudaEventDisableTiming));
            }
        }
    }
    if (pl->model == CIA_MODEL_CUCKER_SMALE || pl->model == CIA_MODEL_POLYNOMIAL) {
        UPT(d.tile_desc, tdesc.data(), tdesc.size());
        CIA_CUDA_TRY(cudaDeviceSynchronize());
        return CIA_OK;
    }
    // The persistent TMA pipeline needs at most 256 nodes per tile (one
    // consumer thread per node) and, in shared memory, the CTA's tile
    // descriptors and observables plus a ring of at least two tile buffers
    // and two community phasor windows; otherwise the kernels use plain loads.
    // kernel choice: 0 (auto) takes the window kernel; the window and the
    // pipelined kernel need 16-bit community-local indices, at most 256 rows
    // per tile and shared memory for their buffers, else plain loads
    pl->ring_stages = 0;
    if (pl->staging == 0) pl->staging = 2;
    if (pl->staging != 1 && (pl->miss_idx_bytes != 2 || pl->tile_nodes > 256)) pl->staging = 1;
    if (pl->staging == 2) {
        int optin = 0;
        CIA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
        if (window_smem_bytes(pl) > (size_t)optin - 1024) pl->staging = 1;
    }
    if (pl->staging == 4) {
        pl->ring_slots = pl->blob_segmented ? ring_slots_that_fit(pl) : 0;
        if (pl->ring_slots < 2) pl->staging = 1;
    }
    if (pl->staging == 3) {
        // contiguous tile ranges, one per SM, balanced by the bytes each tile
        // moves (index vectors, per-node state, community phasor windows)
        int sms = 0;
        CIA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl->device));
        const int64_t cb = (pl->precision == CIA_FP64 ? 16 : 8) * (int64_t)pl->p;
        std::vector<double> cost(T);
        double total = 0.0;
        for (int64_t t = 0; t < T; ++t) {
            const bool first_of_run = t == 0 || tile_comm[t] != tile_comm[t - 1];
            const int64_t lam = tile_comm[t] >= 0 ? pl->off[tile_comm[t] + 1] - pl->off[tile_comm[t]] : 0;
            cost[t] = (double)tile_bytes[t] + 48.0 * tile_count[t] + (first_of_run ? (double)(cb * lam) : 0.0) + 256.0;
            total += cost[t];
        }
        const int nc = (int)std::max<int64_t>(1, std::min<int64_t>(sms, T));
        std::vector<int32_t> ctb(nc + 1, 0);
        double acc = 0.0;
        int64_t t = 0;
        for (int c = 0; c < nc; ++c) {
            ctb[c] = (int32_t)t;
            const double target = total * (double)(c + 1) / nc;
            while (t < T && (acc + 0.5 * cost[t] <= target || c == nc - 1)) acc += cost[t++];
        }
        ctb[nc] = (int32_t)T;
        std::vector<int32_t> runs(nc, 0);
        for (int c = 0; c < nc; ++c)
            for (int64_t u = ctb[c]; u < ctb[c + 1]; ++u)
                if (tile_comm[u] >= 0 && (u == ctb[c] || tile_comm[u] != tile_comm[u - 1])) ++runs[c];
        pl->n_ctas = nc;
        pl->max_cta_tiles = 0;
        pl->max_cta_runs = 1;
        for (int c = 0; c < nc; ++c) pl->max_cta_runs = std::max<int64_t>(pl->max_cta_runs, runs[c]);
        for (int c = 0; c < nc; ++c) {
            pl->max_cta_tiles = std::max<int64_t>(pl->max_cta_tiles, ctb[c + 1] - ctb[c]);
            int r = -1;
            for (int64_t u = ctb[c]; u < ctb[c + 1]; ++u) {
                if (tile_comm[u] >= 0 && (u == ctb[c] || tile_comm[u] != tile_comm[u - 1])) ++r;
                tdesc[u].run = tile_comm[u] >= 0 ? r : -1;
                tdesc[u].pbuf = tile_comm[u] >= 0 ? (r & 1) : 0;
            }
        }
        UPT(d.cta_tile_begin, ctb.data(), ctb.size());
        UPT(d.cta_runs, runs.data(), runs.size());
    }
    if (pl->staging == 3) {
        int optin = 0;
        CIA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
        // a multiple of the two consumer groups, so that each ring buffer is
        // only ever consumed by one group (its waits can then never see a
        // barrier two phases ahead)
        for (int st = 4; st >= 2 && pl->ring_stages == 0; st -= 2)
            if (pipeline_smem_bytes(pl, st) <= (size_t)optin - 1024) pl->ring_stages = st;
        if (pl->ring_stages == 0) pl->staging = 1;
    }
    {
        // launch order of the one-CTA-per-tile kernels: the costliest tiles
        // first, so that the last CTAs to start are short (greedy longest-
        // processing-time scheduling by the hardware's CTA dispatcher)
        std::vector<int32_t> order(T);
        for (int64_t t = 0; t < T; ++t) order[t] = (int32_t)t;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return tile_bytes[x] + 48 * (int64_t)tile_count[x] > tile_bytes[y] + 48 * (int64_t)tile_count[y];
        });
        UPT(d.tile_order, order.data(), order.size());
    }
    UPT(d.tile_desc, tdesc.data(), tdesc.size());
#undef UPT
    CIA_CUDA_TRY(cudaDeviceSynchronize());
    return CIA_OK;
}

static cia_status build_plan(const cia_graph *g, const int32_t *community, const double *omega,
                             const cia_coupling *cp, const cia_options *opt, cia_plan *pl) {
    cia_status st = build_split(g, community, omega, cp, opt, pl);
    if (st != CIA_OK) return st;
    pl->staging_req = pl->staging;
    return build_tiles(pl);
}

extern "C" cia_status cia_plan_create(const cia_graph *g, const int32_t *community,
                                      const double *omega, const cia_coupling *coupling,
                                      const cia_options *opt, cia_plan_t **out) {
    clear_error();
    if (!out) return fail(CIA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g || !coupling || !community) return fail(CIA_ERR_INVALID_ARG, "graph, community or coupling is NULL");
    if (g->n < 1 || g->n > (int64_t)INT32_MAX - 1) return fail(CIA_ERR_INVALID_ARG, "n out of range");
    if (!g->rowptr || (!g->col && g->rowptr[g->n] > 0))
        return fail(CIA_ERR_INVALID_ARG, "rowptr or col is NULL");
    cia_plan *pl = new (std::nothrow) cia_plan();
    if (!pl) return fail(CIA_ERR_OOM, "host allocation of the plan failed");
    cia_status st;
    try {
        st = build_plan(g, community, omega, coupling, opt, pl);
    } catch (const std::bad_alloc &) {
        st = fail(CIA_ERR_OOM, "host allocation failed while planning");
    } catch (const std::exception &e) {
        st = fail(CIA_ERR_INVALID_ARG, std::string("planning failed: ") + e.what());
    }
    if (st != CIA_OK) {
        free_all(pl);
        delete pl;
        return st;
    }
    *out = pl;
    return CIA_OK;
}

extern "C" cia_status cia_plan_create_batch(int64_t B, const cia_graph *graphs, const int32_t *const *communities,
                                            const double *const *omegas, const cia_coupling *coupling,
                                            const cia_options *opt, cia_plan_t **out) {
    clear_error();
    if (!out) return fail(CIA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (B < 1 || !graphs || !communities || !coupling)
        return fail(CIA_ERR_INVALID_ARG, "need B >= 1 and non-NULL graphs, communities and coupling");
    if (coupling->model != CIA_MODEL_KURAMOTO)
        return fail(CIA_ERR_UNSUPPORTED, "ensembles support the Kuramoto model only");
    cia_plan *pl = new (std::nothrow) cia_plan();
    if (!pl) return fail(CIA_ERR_OOM, "host allocation of the plan failed");
    cia_status st = CIA_OK;
    try {
        // the disjoint union: node ids and community labels offset per instance
        pl->B = B;
        pl->inst_off.assign(B + 1, 0);
        pl->inst_comm_off.assign(B + 1, 0);
        int64_t nnz = 0;
        for (int64_t i = 0; i < B && st == CIA_OK; ++i) {
            const cia_graph &g = graphs[i];
            if (g.n < 1 || !g.rowptr || (!g.col && g.rowptr[g.n] > 0) || !communities[i])
                st = fail(CIA_ERR_INVALID_ARG, "instance " + std::to_string(i) + ": empty graph or NULL array");
            else {
                int32_t mx = -1;
                for (int64_t v = 0; v < g.n; ++v) mx = std::max(mx, communities[i][v]);
                pl->inst_off[i + 1] = pl->inst_off[i] + g.n;
                pl->inst_comm_off[i + 1] = pl->inst_comm_off[i] + (int64_t)mx + 1;
                nnz += g.rowptr[g.n];
            }
        }
        if (st == CIA_OK && (pl->inst_off[B] > (int64_t)INT32_MAX - 1 || pl->inst_comm_off[B] > (int64_t)INT32_MAX))
            st = fail(CIA_ERR_INVALID_ARG, "the ensemble has too many nodes or communities");
        if (st == CIA_OK) {
            const int64_t n = pl->inst_off[B];
            std::vector<int64_t> rowptr(n + 1, 0);
            std::vector<int32_t> col(nnz), lab(n);
            std::vector<double> om(n, 0.0);
            int64_t w = 0;
            for (int64_t i = 0; i < B; ++i) {
                const cia_graph &g = graphs[i];
                const int64_t o = pl->inst_off[i];
                for (int64_t v = 0; v < g.n; ++v) {
                    for (int64_t e = g.rowptr[v]; e < g.rowptr[v + 1]; ++e) {
                        const int32_t c = g.col[e];
                        // out-of-range columns stay out of range of the instance (checked below)
                        col[w++] = (c < 0 || c >= g.n) ? -1 : (int32_t)(c + o);
                    }
                    rowptr[o + v + 1] = w;
                    const int32_t l = communities[i][v];
                    lab[o + v] = l < 0 ? l : (int32_t)(l + pl->inst_comm_off[i]);
                    if (omegas && omegas[i]) om[o + v] = omegas[i][v];
                }
            }
            cia_graph u{n, rowptr.data(), col.data()};
            st = build_plan(&u, lab.data(), om.data(), coupling, opt, pl);
        }
    } catch (const std::bad_alloc &) {
        st = fail(CIA_ERR_OOM, "host allocation failed while planning");
    } catch (const std::exception &e) {
        st = fail(CIA_ERR_INVALID_ARG, std::string("planning failed: ") + e.what());
    }
    if (st != CIA_OK) {
        free_all(pl);
        delete pl;
        return st;
    }
    *out = pl;
    return CIA_OK;
}

// ---- streamed ensemble plans ------------------------------------------------

extern "C" cia_status cia_plan_batch_begin(const cia_coupling *coupling, const cia_options *opt, cia_plan_t **out) {
    clear_error();
    if (!out) return fail(CIA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!coupling) return fail(CIA_ERR_INVALID_ARG, "coupling is NULL");
    if (coupling->model != CIA_MODEL_KURAMOTO) return fail(CIA_ERR_UNSUPPORTED, "ensembles support the Kuramoto model only");
    if (opt && opt->build_direct)
        return fail(CIA_ERR_UNSUPPORTED, "a streamed ensemble plan has no direct method: plan a sample of the "
                                         "instances with cia_plan_create_batch for it");
    cia_plan *pl = new (std::nothrow) cia_plan();
    if (!pl) return fail(CIA_ERR_OOM, "host allocation of the plan failed");
    cia_status st = CIA_OK;
    try {
        st = configure(coupling, opt, true, pl);
        if (st == CIA_OK) {
            pl->batch_stage = new BatchStaging();
            if (opt) pl->batch_stage->opt = *opt;
            pl->B = 0;
            pl->inst_off.assign(1, 0);
            pl->inst_comm_off.assign(1, 0);
        }
    } catch (const std::bad_alloc &) {
        st = fail(CIA_ERR_OOM, "host allocation failed while planning");
    }
    if (st != CIA_OK) {
        free_all(pl);
        delete pl;
        return st;
    }
    *out = pl;
    return CIA_OK;
}

extern "C" cia_status cia_plan_batch_add(cia_plan_t *pl, const cia_graph *g, const int32_t *community,
                                         const double *omega) {
    clear_error();
    if (!pl || !pl->batch_stage) return fail(CIA_ERR_INVALID_ARG, "not a streamed ensemble plan being built");
    BatchStaging &bs = *pl->batch_stage;
    const int64_t i = (int64_t)bs.inst.size();
    const std::string who = "instance " + std::to_string(i) + ": ";
    if (!g || g->n < 1 || !g->rowptr || (!g->col && g->rowptr[g->n] > 0) || !community)
        return fail(CIA_ERR_INVALID_ARG, who + "empty graph or NULL array");
    if (bs.n_total + g->n > (int64_t)INT32_MAX - 1)
        return fail(CIA_ERR_INVALID_ARG, who + "the ensemble has too many nodes");
    if (omega)
        for (int64_t v = 0; v < g->n; ++v)
            if (!std::isfinite(omega[v]))
                return fail(CIA_ERR_NUMERIC, who + "omega[" + std::to_string(v) + "] is not finite");
    try {
        // split the instance on its own (the direct method's CSR is not built)
        cia_plan tmp;
        tmp.has_direct = 0;
        std::vector<int64_t> rp;
        std::vector<int32_t> col;
        cia_status st = split_graph(g, community, &tmp, rp, col);
        if (st != CIA_OK) return fail(st, who + cia_last_error());
        if (tmp.max_comm > 65535)
            return fail(CIA_ERR_UNSUPPORTED, who + "a community above 65535 nodes has no CIA layout");
        StagedInstance si;
        si.n = g->n;
        si.M = tmp.M;
        si.n_lab = tmp.off[tmp.M];
        si.nnz = tmp.nnz_graph;
        si.max_comm = tmp.max_comm;
        si.perm = std::move(tmp.perm);
        si.off = std::move(tmp.off);
        si.miss_cnt.assign(tmp.hs.miss_cnt.begin(), tmp.hs.miss_cnt.begin() + si.n_lab);
        si.miss = std::move(tmp.hs.miss_local);
        si.inter_cnt = std::move(tmp.hs.inter_cnt);
        // the ensemble's permuted order: every instance's labelled nodes, then
        // every instance's free nodes, both in instance order
        const auto &ic = tmp.hs.inter_col;
        si.inter.resize(ic.size());
        for (size_t e = 0; e < ic.size(); ++e) {
            const int64_t q = ic[e];
            si.inter[e] = q < si.n_lab ? bs.lab_total + q : -1 - (bs.free_total + (q - si.n_lab));
        }
        if (omega) {
            si.omega.resize(si.n);
            for (int64_t m = 0; m < si.n; ++m) si.omega[m] = omega[si.perm[m]];
        }
        bs.lab_total += si.n_lab;
        bs.free_total += si.n - si.n_lab;
        bs.comm_total += si.M;
        bs.n_total += si.n;
        pl->inst_off.push_back(bs.n_total);
        pl->inst_comm_off.push_back(bs.comm_total);
        bs.inst.push_back(std::move(si));
    } catch (const std::bad_alloc &) {
        return fail(CIA_ERR_OOM, who + "host allocation failed while planning");
    }
    pl->B = (int64_t)bs.inst.size();
    return CIA_OK;
}

extern "C" cia_status cia_plan_batch_finish(cia_plan_t *pl) {
    clear_error();
    if (!pl || !pl->batch_stage) return fail(CIA_ERR_INVALID_ARG, "not a streamed ensemble plan being built");
    BatchStaging &bs = *pl->batch_stage;
    const int64_t B = (int64_t)bs.inst.size();
    if (B < 1) return fail(CIA_ERR_INVALID_ARG, "no instance was added");
    cia_status st = CIA_OK;
    try {
        const int64_t n = bs.n_total, M = bs.comm_total, L = bs.lab_total;
        pl->n = n;
        pl->M = M;
        pl->n_free = bs.free_total;
        pl->ph_stride = (n + 2) & ~(int64_t)1;
        pl->miss_idx_bytes = 2;
        pl->max_comm = 0;
        pl->nnz_graph = 0;
        auto &hs = pl->hs;
        pl->perm.assign(n, 0);
        pl->off.assign(M + 1, 0);
        hs.comm_of.assign(n, -1);
        hs.miss_cnt.assign(n, 0);
        hs.inter_cnt.assign(n, 0);
        std::vector<double> om(n, 0.0);
        bool any_omega = false;
        // row of the ensemble for row m of instance i
        std::vector<int64_t> lab_base(B), free_base(B);
        for (int64_t i = 0, lb = 0, fb = L; i < B; ++i) {
            lab_base[i] = lb;
            free_base[i] = fb;
            lb += bs.inst[i].n_lab;
            fb += bs.inst[i].n - bs.inst[i].n_lab;
        }
#pragma omp parallel for schedule(dynamic, 1) reduction(|| : any_omega)
        for (int64_t i = 0; i < B; ++i) {
            const StagedInstance &si = bs.inst[i];
            const int64_t o = pl->inst_off[i], c0 = pl->inst_comm_off[i];
            for (int64_t m = 0; m < si.n; ++m) {
                const int64_t r = m < si.n_lab ? lab_base[i] + m : free_base[i] + (m - si.n_lab);
                pl->perm[r] = (int32_t)(o + si.perm[m]);
                hs.inter_cnt[r] = si.inter_cnt[m];
                if (!si.omega.empty()) om[r] = si.omega[m];
            }
            for (int64_t c = 0; c < si.M; ++c) {
                pl->off[c0 + c] = lab_base[i] + si.off[c];
                for (int64_t m = si.off[c]; m < si.off[c + 1]; ++m) hs.comm_of[lab_base[i] + m] = (int32_t)(c0 + c);
            }
            for (int64_t m = 0; m < si.n_lab; ++m) hs.miss_cnt[lab_base[i] + m] = si.miss_cnt[m];
            any_omega = any_omega || !si.omega.empty();
        }
        pl->off[M] = L;
        hs.miss_off.assign(n + 1, 0);
        hs.inter_off.assign(n + 1, 0);
        for (int64_t m = 0; m < n; ++m) {
            hs.miss_off[m + 1] = hs.miss_off[m] + hs.miss_cnt[m];
            hs.inter_off[m + 1] = hs.inter_off[m] + hs.inter_cnt[m];
        }
        pl->nnz_missing = hs.miss_off[n];
        pl->nnz_inter = hs.inter_off[n];
        // the lists, instance by instance, releasing each staged copy
        hs.miss_local.resize(pl->nnz_missing);
        hs.inter_col.resize(pl->nnz_inter);
        for (int64_t i = 0; i < B; ++i) {
            StagedInstance &si = bs.inst[i];
            std::copy(si.miss.begin(), si.miss.end(), hs.miss_local.begin() + hs.miss_off[lab_base[i]]);
            // labelled rows' inter links, then free rows'
            int64_t split = 0;
            for (int64_t m = 0; m < si.n_lab; ++m) split += si.inter_cnt[m];
            auto decode = [&](int64_t v) { return (int32_t)(v >= 0 ? v : L + (-1 - v)); };
            int32_t *dl = hs.inter_col.data() + hs.inter_off[lab_base[i]];
            for (int64_t e = 0; e < split; ++e) dl[e] = decode(si.inter[e]);
            if (si.n > si.n_lab) {
                int32_t *df = hs.inter_col.data() + hs.inter_off[free_base[i]];
                for (int64_t e = split; e < (int64_t)si.inter.size(); ++e) df[e - split] = decode(si.inter[e]);
            }
            pl->max_comm = std::max(pl->max_comm, si.max_comm);
            pl->nnz_graph += si.nnz;
            si = StagedInstance();
        }
        const cia_options opt = bs.opt;
        delete pl->batch_stage;
        pl->batch_stage = nullptr;
        std::vector<int64_t> no_rp;
        std::vector<int32_t> no_col;
        st = upload_split(pl, &opt, any_omega ? om.data() : nullptr, no_rp, no_col);
        if (st == CIA_OK) {
            pl->staging_req = pl->staging;
            st = build_tiles(pl);
        }
    } catch (const std::bad_alloc &) {
        st = fail(CIA_ERR_OOM, "host allocation failed while planning");
    }
    return st;
}

extern "C" cia_status cia_plan_retile(cia_plan_t *pl, int tile_nodes, int tile_index_bytes, int staging) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    const int tn = tile_nodes ? tile_nodes : (pl->model == CIA_MODEL_CUCKER_SMALE ? 128 : 256);
    if (tn < 32 || tn > 1024 || tn % 32 || (pl->model == CIA_MODEL_CUCKER_SMALE && tn > 128) ||
        (pl->model == CIA_MODEL_POLYNOMIAL && tn > 256))
        return fail(CIA_ERR_INVALID_ARG, "tile_nodes must be a multiple of 32 in [32, 1024] (<= 128 for Cucker-Smale)");
    const int tib = tile_index_bytes ? tile_index_bytes : 65536;
    if (tib < 256 || tib % 16) return fail(CIA_ERR_INVALID_ARG, "tile_index_bytes must be a multiple of 16, at least 256");
    if (staging < 0 || staging > 4) return fail(CIA_ERR_INVALID_ARG, "staging must be 0, 1, 2, 3 or 4");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(CIA_ERR_INVALID_ARG, "plan belongs to another device");
    CIA_CUDA_TRY(cudaDeviceSynchronize());
    pl->tile_nodes = tn;
    pl->tile_index_bytes = tib;
    pl->staging_req = pl->model == CIA_MODEL_CUCKER_SMALE ? 1 : staging;
    cia_status st;
    try {
        st = build_tiles(pl);
    } catch (const std::bad_alloc &) {
        st = fail(CIA_ERR_OOM, "host allocation failed while re-tiling");
    }
    pl->needs_load = true;
    return st;
}

extern "C" cia_status cia_plan_destroy(cia_plan_t *plan) {
    clear_error();
    if (!plan) return CIA_OK;
    free_all(plan);
    delete plan;
    return CIA_OK;
}

extern "C" cia_status cia_plan_get_info(const cia_plan_t *pl, cia_plan_info *info) {
    clear_error();
    if (!pl || !info) return fail(CIA_ERR_INVALID_ARG, "plan or info is NULL");
    info->ring_slots = pl->staging == 4 ? pl->ring_slots : 0;
    info->n = pl->n;
    info->M = pl->M;
    info->n_free = pl->n_free;
    info->max_community = pl->max_comm;
    info->nnz_graph = pl->nnz_graph;
    info->nnz_missing = pl->nnz_missing;
    info->nnz_inter = pl->nnz_inter;
    info->n_tiles = pl->n_tiles;
    info->device_bytes = pl->device_bytes;
    info->precision = pl->precision;
    info->group_size = pl->group_size;
    info->tile_nodes = pl->tile_nodes;
    info->missing_index_bytes = pl->miss_idx_bytes;
    info->staging = pl->staging;
    info->group_size_direct = pl->group_size_direct;
    info->max_tile_index_bytes = pl->max_tile_idx_bytes;
    info->model = pl->gc_basis == 1 ? CIA_MODEL_FOURIER_GENERAL
                  : pl->poly_general  ? CIA_MODEL_POLYNOMIAL_GENERAL
                                      : pl->model;
    info->state_dim = pl->state_dim;
    info->instances = pl->B;
    return CIA_OK;
}

extern "C" cia_status cia_plan_get_permutation(const cia_plan_t *pl, int32_t *perm, int64_t *offsets) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    if (perm) std::memcpy(perm, pl->perm.data(), pl->perm.size() * sizeof(int32_t));
    if (offsets) std::memcpy(offsets, pl->off.data(), pl->off.size() * sizeof(int64_t));
    return CIA_OK;
}

extern "C" cia_status cia_plan_get_split(const cia_plan_t *pl, int64_t *miss_rowptr, int32_t *miss_col,
                                         int64_t *inter_rowptr, int32_t *inter_col) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    if (pl->miss_idx_bytes != 2)
        return fail(CIA_ERR_UNSUPPORTED, "communities above 65535 nodes have no CIA layout");
    const int64_t n = pl->n, T = pl->n_tiles;
    // decode the device's sliced-ELL blobs back into plain CSRs
    std::vector<TileDesc> td(T);
    std::vector<unsigned char> blob(pl->blob_bytes);
    CIA_CUDA_TRY(cudaMemcpy(td.data(), pl->d.tile_desc, T * sizeof(TileDesc), cudaMemcpyDeviceToHost));
    if (pl->blob_bytes)
        CIA_CUDA_TRY(cudaMemcpy(blob.data(), pl->d.blob, pl->blob_bytes, cudaMemcpyDeviceToHost));
    std::vector<std::vector<int32_t>> mrow(n), irow(n);
    for (int64_t t = 0; t < T; ++t) {
        const TileDesc &d = td[t];
        const unsigned char *b = blob.data() + d.blob_off;
        const uint32_t *desc = reinterpret_cast<const uint32_t *>(b);
        const uint32_t *rows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
        const uint32_t *vtab = reinterpret_cast<const uint32_t *>(b + d.vtab_off);
        std::vector<int32_t> chunk_row;          // chunk -> tile row
        if (!pl->blob_segmented)
            for (int32_t r = 0; r < d.count; ++r)
                for (uint32_t c = 0; c < (vtab[r] >> 16); ++c) chunk_row.push_back(r);
        const uint16_t *sm = reinterpret_cast<const uint16_t *>(b + d.mvec_off);
        const int32_t *si = reinterpret_cast<const int32_t *>(b + d.ivec_off);
        for (int64_t sl = 0; sl < d.nsl; ++sl) {
            const uint32_t moff = desc[4 * sl], nvm = desc[4 * sl + 1], ioff = desc[4 * sl + 2], nvi = desc[4 * sl + 3];
            for (int lane = 0; lane < 32; ++lane) {
                const uint32_t rr = rows[32 * sl + lane];
                if (pl->blob_segmented) {
                    // lane map: row | lanes of the row << 16 | lane within the row << 22
                    if (rr == 0xffffffffu) continue;
                    const int32_t row = (int32_t)(rr & 0xffffu);
                    for (uint32_t j = 0; j < nvm; ++j)
                        for (int h = 0; h < 8; ++h) {
                            const uint16_t v = sm[8 * (moff + 32 * j + lane) + h];
                            if (v < d.lam) mrow[d.first + row].push_back((int32_t)(d.lo + v));
                        }
                    for (uint32_t j = 0; j < nvi; ++j)
                        for (int h = 0; h < 4; ++h) {
                            const int32_t v = si[4 * (ioff + 32 * j + lane) + h];
                            if (v != n) irow[d.first + row].push_back(v);
                        }
                    continue;
                }
                const uint32_t mr = rr & 0xffffu, ir = rr >> 16;
                if (mr != 0xffffu)
                    for (uint32_t j = 0; j < nvm; ++j)
                        for (int h = 0; h < 8; ++h) {
                            const uint16_t v = sm[8 * (moff + 32 * j + lane) + h];
                            if (v < d.lam) mrow[d.first + chunk_row[mr]].push_back((int32_t)(d.lo + v));   // >= lam: padding
                        }
                if (ir != 0xffffu)
                    for (uint32_t j = 0; j < nvi; ++j)
                        for (int h = 0; h < 4; ++h) {
                            const int32_t v = si[4 * (ioff + 32 * j + lane) + h];
                            if (v != n) irow[d.first + ir].push_back(v);
                        }
            }
        }
    }
    int64_t wm = 0, wi = 0;
    if (miss_rowptr) miss_rowptr[0] = 0;
    if (inter_rowptr) inter_rowptr[0] = 0;
    for (int64_t m = 0; m < n; ++m) {
        std::sort(mrow[m].begin(), mrow[m].end());   // device order is bank-scheduled
        for (int32_t v : mrow[m]) {
            if (miss_col) miss_col[wm] = v;
            ++wm;
        }
        for (int32_t v : irow[m]) {
            if (inter_col) inter_col[wi] = v;
            ++wi;
        }
        if (miss_rowptr) miss_rowptr[m + 1] = wm;
        if (inter_rowptr) inter_rowptr[m + 1] = wi;
    }
    return CIA_OK;
}
