/*
 * cia.h -- C ABI of the GB300 community integration algorithm (CIA) library.
 *
 * The library evaluates the right-hand side of a network ODE
 *
 *     x_m' = f_m(x_m) + (1/N) sum_l a_ml g(x_l, x_m),   m = 1..N
 *
 * (eq. GeneralNetworkSystem, Sec. 2 of Boehle, Thalhammer, Kuehn, "Community
 * Integration Algorithms (CIAs) for Dynamical Systems on Networks",
 * arXiv 2203.16657) with the CIA of Sec. 3: community observables stand in for
 * the dense diagonal blocks D of the permuted adjacency B = P A P^T = D + S,
 * and the sparse remainder S (missing links inside a block, extra links
 * between blocks) is summed directly.  A direct O(|E|) CSR evaluation of the
 * same sum is provided for comparison.
 *
 * Conventions shared by every entry point:
 *  - Every call returns a cia_status; nothing aborts, throws or exits.  The
 *    text of the last error of the calling thread is cia_last_error().
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the device that was current when the plan was made.
 *  - State at the boundary is always FP64 in the ORIGINAL node numbering of
 *    the graph, d values per node (d = 1 for the Kuramoto models: theta_m;
 *    d = 4 for Cucker--Smale: s_x, s_y, v_x, v_y, node-major).  The compute
 *    precision inside is the plan's (cia_options).
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device work is asynchronous on that stream; an asynchronous CUDA error
 *    surfaces as CIA_ERR_CUDA from a later call on the same plan.
 *  - The caller owns every buffer it passes; the plan owns the device copies
 *    of the network structure and its work buffers until cia_plan_destroy.
 *  - A plan is not thread-safe: calls on one plan must not overlap.
 */
#ifndef CIA_H
#define CIA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CIA_OK = 0,
    CIA_ERR_INVALID_ARG = 1,    /* null pointer, bad size or option */
    CIA_ERR_INVALID_GRAPH = 2,  /* asymmetric, self loop, unsorted/duplicate or out-of-range column */
    CIA_ERR_UNSUPPORTED = 3,    /* valid request the library does not implement */
    CIA_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the CUDA error) */
    CIA_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    CIA_ERR_FALLBACK = 6,       /* informational: a learned basis failed its check, direct was used */
    CIA_ERR_NUMERIC = 7,        /* NaN or Inf in an input */
    CIA_ERR_OOM = 8             /* device or host allocation failed */
} cia_status;

typedef enum {
    CIA_MODEL_KURAMOTO = 0,     /* phase oscillators, h = sum_k d_sin[k] sin kx + d_cos[k] cos kx (App. A.4) */
    CIA_MODEL_KURAMOTO_HO = 1,  /* the same plus a triadic term on complete community hyperedges (App. A.7) */
    CIA_MODEL_CUCKER_SMALE = 2, /* 2-D flocking agents (App. A.6), state (s_x, s_y, v_x, v_y) per node */
    CIA_MODEL_POLYNOMIAL = 3,   /* polynomial difference coupling with a potential (App. A.3, A.5) */
    CIA_MODEL_POLYNOMIAL_GENERAL = 4, /* general polynomial coupling g(x_l, x_m) with a potential (App. A.3) */
    CIA_MODEL_FOURIER_GENERAL = 5     /* general real 2-D Fourier coupling g(x_l, x_m) with a potential (App. A.3) */
} cia_model;

typedef enum {
    CIA_FP64 = 0,               /* state, observables and sums in FP64 */
    CIA_FP32 = 1                /* stage state, observables and sums in FP32; FP64 time accumulation */
} cia_precision;

typedef enum {
    CIA_METHOD_CIA = 0,         /* community observables + sparse corrections (Sec. 3.2, E1 + E2) */
    CIA_METHOD_DIRECT = 1       /* direct O(|E|) sum over the CSR neighbours */
} cia_method;

#define CIA_MAX_HARMONICS 4
#define CIA_MAX_POLY 4

/* Undirected, unweighted graph without self loops as a symmetric CSR (host).
 * Columns of each row must be strictly increasing.  A is 0/1 (Sec. 2). */
typedef struct {
    int64_t n;                  /* number of nodes N >= 1 */
    const int64_t *rowptr;      /* host, n + 1 entries, rowptr[0] = 0 */
    const int32_t *col;         /* host, rowptr[n] entries in [0, n) */
} cia_graph;

/* The model: f_m and g.  For CIA_MODEL_KURAMOTO,
 *   f_m(theta) = omega_m,  g(x_l, x_m) = K h(x_l - x_m),
 *   h(x) = sum_{k=1..p} d_sin[k-1] sin(kx) + d_cos[k-1] cos(kx)
 * (the higher-harmonics Kuramoto model, App. A.4; p = 1, d_sin = {1},
 * d_cos = {0} is the classical model).
 * CIA_MODEL_KURAMOTO_HO adds, for every node m of a community c, the triadic
 * term of the higher-order Kuramoto model (App. A.7, eq. HOKuramoto with
 * lambda = (1, 1, -2)) over the community's complete 2-simplices:
 *   (K2/N^2) sum_{j != k; j, k in c, both != m} sin(theta_j + theta_k - 2 theta_m);
 * nodes in no community get no triadic term.  The CIA evaluates it from the
 * community moments Z_1, Z_2 (eq. HOKuramoto_fastRHS with the tuples that
 * repeat an index removed); the direct method sums the pairs one by one.
 * CIA_MODEL_CUCKER_SMALE (App. A.6, eq. Cucker_Smale, n = 2): per node the
 * state is x_m = (s_m, v_m), position and velocity in R^2, and
 *   s_m' = v_m,   v_m' = (1/N) sum_l a_ml eta(||s_l - s_m||^2) (v_l - v_m),
 *   eta(y) = K (sigma^2 + y)^-beta.
 * Its CIA needs a separable basis of eta (step P2): a learned feature map set
 * with cia_plan_set_basis (include/cia_basis.h).  The links of S (missing and
 * inter-community) are summed with the exact eta.  FP32 only; p, d_sin,
 * d_cos and K2 are ignored.
 * CIA_MODEL_POLYNOMIAL (eq. GeneralNetworkPolyDifference, App. A.3, with the
 * potential of the Desai-Zwanzig model, eq. DesaiZwanzig, App. A.5):
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml h(x_l - x_m),
 *   h(x) = sum_{a=0..p} poly_c[a] x^a,   V'(x) = sum_{j=0..4} dV[j] x^j,
 * p in [0, CIA_MAX_POLY].  The CIA uses the community moments
 * W_ck = sum_{l in c} x_l^k, k <= p (eq. PolyMoments) and the binomial
 * expansion of h (eq. PolyDifferenceRHSfast); the links of S are summed with
 * h itself.  Desai-Zwanzig: p = 1, poly_c = (0, 1).  FP64 only; omega must be
 * NULL.
 * CIA_MODEL_POLYNOMIAL_GENERAL (eq. GeneralNetworkPoly with eq. PolyApprox,
 * App. A.3): the same with a general polynomial coupling
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),
 *   g(u, y) = sum_{a=0..p} sum_{b=0..p} poly_g[a * (CIA_MAX_POLY + 1) + b] u^a y^b
 * (u is the neighbour's state; entries with a or b above p are ignored).  The
 * CIA evaluates the dense term sum_{a,b} poly_g[a][b] W_ca x_m^b (eq. PolyRHS)
 * from the same moments; the links of S are summed with g itself.  poly_c is
 * ignored.  FP64 only; omega must be NULL.
 * CIA_MODEL_FOURIER_GENERAL (eq. GeneralNetworkFourier with the real series
 * of eq. FourierRealExpansion, App. A.3): the same with
 *   g(u, y) = sum_{a,b=0..p} C11[a][b] cos(a w u) cos(b w y) + C12[a][b] cos(a w u) sin(b w y)
 *                          + C21[a][b] sin(a w u) cos(b w y) + C22[a][b] sin(a w u) sin(b w y),
 * w = pi / fourier_L, C11 = fourier_c[0], C12 = fourier_c[1], C21 = fourier_c[2],
 * C22 = fourier_c[3], each row-major with CIA_MAX_HARMONICS + 1 columns;
 * p in [1, CIA_MAX_HARMONICS] (entries with a or b above p are ignored).  The
 * CIA keeps the real generalised order parameters sum_{l in c} cos(a w x_l),
 * sum_{l in c} sin(a w x_l) per community (eq. RealOP); the links of S are
 * summed with g itself.  FP64 only; omega must be NULL. */
typedef struct {
    int model;                  /* cia_model */
    int p;                      /* Kuramoto and Fourier models: harmonics, 1..CIA_MAX_HARMONICS;
                                   polynomial models: degree, 0..CIA_MAX_POLY */
    double d_sin[CIA_MAX_HARMONICS];
    double d_cos[CIA_MAX_HARMONICS];
    double K;                   /* coupling constant multiplying (1/N) sum */
    double K2;                  /* triadic coupling (CIA_MODEL_KURAMOTO_HO), multiplies (1/N^2) sum */
    double sigma, beta;         /* Cucker--Smale weight eta(y) = K (sigma^2 + y)^-beta, sigma > 0 */
    double poly_c[CIA_MAX_POLY + 1];   /* polynomial model: coefficients of h, degree p */
    double dV[CIA_MAX_POLY + 1];       /* polynomial models: coefficients of V' */
    double poly_g[(CIA_MAX_POLY + 1) * (CIA_MAX_POLY + 1)]; /* general polynomial model: g[a][b], row-major */
    double fourier_L;                  /* general Fourier model: half period, > 0 */
    double fourier_c[4][(CIA_MAX_HARMONICS + 1) * (CIA_MAX_HARMONICS + 1)]; /* C11, C12, C21, C22 */
} cia_coupling;

typedef struct {
    int precision;              /* cia_precision */
    int build_direct;           /* nonzero: also keep the full CSR on the device (CIA_METHOD_DIRECT) */
    int tile_nodes;             /* nodes per work tile, 0 = default (256; 128 for Cucker--Smale);
                                   a multiple of 32, <= 1024 (<= 128 for Cucker--Smale) */
    int group_size;             /* threads per row of the direct method's CSR sums: 0 = default,
                                   else 4, 8, 16 or 32 (the CIA sums use one thread per row) */
    int tile_index_bytes;       /* sparse-index bytes per tile, 0 = default (65536); a multiple of 16.
                                   A tile is cut at tile_nodes rows or at this many index bytes. */
    int staging;                /* CIA stage kernel: 0 = auto (2 when it fits); 1 = plain loads,
                                   one CTA per tile; 2 = one CTA per tile with the community's
                                   phasors copied (TMA) into shared memory; 3 = persistent
                                   warp-specialised CTAs with TMA copies of each tile's indices
                                   and community phasors; 4 = persistent CTAs, each tile's
                                   community phasors and indices copied (TMA) into one
                                   shared-memory buffer of at most tile_index_bytes (the window
                                   of a large community leaves less room for indices, so its
                                   tiles are shorter), the next tile's copy overlapping the
                                   current tile's node phase.  2, 3 and 4 fall back to 1 when
                                   their buffers do not fit.  Polynomial and Fourier couplings: 1 =
                                   the community's features from global memory, 0, 2, 3 and 4 = in
                                   shared memory as 64-bit fixed point: tiles are sorted by
                                   community size and each stage launches one kernel per run of
                                   tiles that fit 4, 3, 2 or 1 CTAs per SM (window sized to the
                                   run's largest community), concurrently on streams forked from
                                   the caller's and joined to it; tiles of a community that no
                                   window holds read its features from global memory. */
    int use_graphs;             /* 0 = auto: cia_advance replays one captured CUDA graph per RK4
                                   step when it advances >= 2 steps, or from the first step when
                                   an earlier call captured the graph of the same method, state
                                   slot, dt and r_out (not while profiling); 1 = plain launches
                                   only */
} cia_options;

typedef struct cia_plan cia_plan_t;

/* Sizes of a plan (all counts, no pointers). */
typedef struct {
    int64_t n;                  /* nodes */
    int64_t M;                  /* communities (labels 0..M-1) */
    int64_t n_free;             /* nodes with label -1 (no community) */
    int64_t max_community;      /* largest lambda_c */
    int64_t nnz_graph;          /* entries of the input CSR (2 |E|) */
    int64_t nnz_missing;        /* missing links inside blocks, off-diagonal, both directions */
    int64_t nnz_inter;          /* links between different blocks (or touching free nodes), both directions */
    int64_t n_tiles;            /* work tiles of the CIA kernels */
    int64_t device_bytes;       /* device memory held by the plan */
    int precision;
    int group_size;
    int tile_nodes;
    int missing_index_bytes;    /* 2 (16-bit community-local index) or 4 */
    int staging;                /* the kernel in use: 1, 2, 3 or 4 as in cia_options */
    int group_size_direct;      /* threads per row of the direct method */
    int64_t max_tile_index_bytes; /* largest sparse-index footprint of a tile */
    int model;                  /* cia_model */
    int state_dim;              /* d: FP64 values per node at the boundary */
    int64_t instances;          /* independent networks (1 unless cia_plan_create_batch) */
    int ring_slots;             /* staging 4: tile buffers of the ring in shared memory (else 0) */
} cia_plan_info;

/* ---- status -------------------------------------------------------------- */

/* Static string naming a status code. */
const char *cia_status_string(cia_status s);

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next library call on this thread. */
const char *cia_last_error(void);

/* ---- planning: step P1 (Sec. 3.1, App. A.1), offline and untimed --------- */

/* Community detection for step P1 (Sec. "Community Detection (P1)"): labels
 * that make S sparse, by minimising the Potts Hamiltonian with the
 * Erdos-Renyi null model (the rber_pots objective the paper recommends)
 *   H = -sum_{m != l} (a_ml - gamma p) delta(c_m, c_l) + mu M,
 * p = 2|E| / (N (N - 1)) the link density, M the number of communities and
 * mu = community_cost an extra charge per community: the paper notes that
 * the E1 work grows with the number of communities, so that fewer, larger
 * communities can pay off, more so for a high expansion order.  With
 * gamma p = 1/2 and mu = 0, H = nnz(S)/2 - |E|: H then counts the entries of
 * S exactly.  Optimisation: local moving of single nodes to the neighbouring
 * community with the largest decrease of H, in a seeded random order, then
 * aggregation of the communities into weighted nodes and again (the Louvain
 * scheme), then a last local-moving pass over the original nodes, so that
 * no single-node move lowers H.  Host code (offline, like the rest of P1).
 * labels: host, g->n entries, written: 0..M-1 in order of first appearance,
 * -1 for nodes in communities smaller than min_size (no community, Sec. 3.1). */
typedef struct {
    double gamma;               /* resolution, > 0; 1 = the paper's choice */
    double community_cost;      /* mu >= 0, in units of directed entries of a_ml */
    int min_size;               /* >= 1; smaller communities come back as -1 */
    int max_levels;             /* aggregation levels, >= 1 */
    uint64_t seed;              /* visiting order */
} cia_detect_options;

typedef struct {
    int64_t communities;        /* labelled communities returned (M) */
    int64_t unlabelled;         /* nodes returned as -1 */
    int64_t nnz_missing;        /* -1 entries of S for the returned labels (directed, no diagonal) */
    int64_t nnz_inter;          /* +1 entries of S for the returned labels (directed) */
    double hamiltonian;         /* H of the optimised partition (before the min_size relabelling) */
    int levels;                 /* aggregation levels run */
    int64_t moves;              /* single-node moves made, all levels */
} cia_detect_report;

/* Defaults: gamma 1, community_cost 0, min_size 2, max_levels 8, seed 0. */
void cia_detect_options_default(cia_detect_options *opt);

/* CIA_ERR_INVALID_GRAPH as cia_plan_create; CIA_ERR_INVALID_ARG for bad
 * options or NULL pointers.  report may be NULL. */
cia_status cia_detect_communities(const cia_graph *g, const cia_detect_options *opt, int32_t *labels,
                                  cia_detect_report *report);

/* Step P1's trade-off between the number of communities and the CIA's cost
 * per stage, chosen by measuring this library's own kernels (Sec. "Community
 * Detection (P1)": fewer, larger communities can pay off, more so for a high
 * expansion order p).  Three partitions are detected and planned with
 * `coupling` and `opt` (Kuramoto models), and each is timed for `steps` RK4
 * steps (after two warm-up steps) from the state x (host, g->n doubles,
 * original order) with step dt: 0 = the fewest entries of S (gamma p = 1/2,
 * mu = 0), 1 = a
 * coarser probe (a charge of one average block's directed pairs per
 * community), 2 = the partition minimising the modelled stage time
 *   T = c_tile tiles + c_byte (bytes of nodes, missing links, inter links),
 * with c_tile and c_byte fitted to the timings of 0 and 1 (p enters through
 * the gathered phasor bytes and the measured costs): gamma p =
 * c_miss / (c_miss + c_inter) and mu = c_tile / (c_miss + c_inter) make the
 * detector's Hamiltonian that model.  labels (host, g->n) receives the
 * fastest of the three as measured, so the choice never loses to mu = 0.
 * The device work allocates (plans, one state buffer) and synchronises. */
typedef struct {
    int64_t communities[3];      /* of partitions 0 (mu = 0), 1 (probe), 2 (modelled optimum) */
    int64_t tiles[3];            /* work tiles of their plans */
    int64_t nnz_s[3];            /* entries of S (missing + inter, directed) */
    double ms_per_step[3];       /* measured device time of one RK4 step */
    double per_tile_us;          /* fitted cost of one tile per stage */
    double per_byte_ps;          /* fitted cost of one byte per stage */
    double gamma, community_cost;   /* detection options of partition 2 */
    double probe_community_cost; /* mu of partition 1 */
    int chosen;                  /* the partition in labels: 0, 1 or 2 */
} cia_partition_report;

cia_status cia_choose_partition(const cia_graph *g, const double *omega, const cia_coupling *coupling,
                                const cia_options *opt, const double *x, double dt, int64_t steps,
                                int32_t *labels, cia_partition_report *report);

/* Build a plan for graph g with the given community labels.
 *
 * community: host, g->n entries; community[i] in [0, M) names the block of
 *   node i, -1 puts node i in no community (allowed "for numerical reasons",
 *   Sec. 3.1): all its links are then treated as sparse extra links.
 *   Labels need not be contiguous in i; M = max label + 1 (empty labels allowed).
 * omega: host, g->n natural frequencies f_m = omega_m (NULL = all zero).
 *   With CIA_FP32 they are rounded to FP32.  Must be NULL for Cucker--Smale.
 * The plan computes the permutation kappa that sorts nodes by (label, id)
 * with unlabelled nodes last, the community offsets, and the two halves of S:
 *   missing links inside each block (the -1 entries of S without the
 *   diagonal, which is handled analytically) and extra links (+1 entries).
 * Validation: symmetric, no self loops, columns sorted, unique and in range;
 * violations return CIA_ERR_INVALID_GRAPH and no plan.  NaN/Inf in omega or
 * the coupling returns CIA_ERR_NUMERIC.
 * On success *out owns device memory until cia_plan_destroy(*out). */
cia_status cia_plan_create(const cia_graph *g, const int32_t *community, const double *omega,
                           const cia_coupling *coupling, const cia_options *opt,
                           cia_plan_t **out);

/* An ensemble of B independent networks in one plan, so that every RK4
 * stage of all of them is one launch.  Instance i has its own graph
 * graphs[i], labels communities[i] and frequencies omegas[i] (omegas or
 * omegas[i] may be NULL = zero), and its own normalisation K / N_i.  The
 * state of the ensemble concatenates the instances in order (instance i
 * occupies [sum_{j<i} N_j, sum_{j<=i} N_j)); cia_integrate / cia_advance then
 * fill r_out with nsteps x B order parameters, r_out[j * B + i] for instance
 * i after step j + 1.  Kuramoto model (CIA_MODEL_KURAMOTO) only. */
cia_status cia_plan_create_batch(int64_t B, const cia_graph *graphs, const int32_t *const *communities,
                                 const double *const *omegas, const cia_coupling *coupling,
                                 const cia_options *opt, cia_plan_t **out);

/* The same ensemble plan built one instance at a time, so that the caller
 * never holds every instance's graph at once (an ensemble of thousands of
 * networks can have tens of billions of CSR entries).  cia_plan_batch_begin
 * takes the coupling (CIA_MODEL_KURAMOTO) and options (build_direct must be
 * 0: CIA_ERR_UNSUPPORTED otherwise; plan a sample of instances with
 * cia_plan_create_batch for the direct method); cia_plan_batch_add validates
 * and splits one instance (step P1, Sec. 3.1) -- g, community and omega
 * (nullable) as for cia_plan_create, copied, so the caller may free them when
 * it returns; every community of an added instance must have at most 65535
 * nodes (CIA_ERR_UNSUPPORTED).  cia_plan_batch_finish lays the instances out
 * on the device exactly as cia_plan_create_batch would for the same
 * instances in the same order; the plan can then be used like any other.  A
 * failed add leaves the plan as it was; a failed finish leaves a plan that
 * only cia_plan_destroy accepts. */
cia_status cia_plan_batch_begin(const cia_coupling *coupling, const cia_options *opt, cia_plan_t **out);
cia_status cia_plan_batch_add(cia_plan_t *plan, const cia_graph *g, const int32_t *community, const double *omega);
cia_status cia_plan_batch_finish(cia_plan_t *plan);

/* Rank-one link weights for the polynomial models (Sec. "Rank One Coupling",
 * eq. rank1system, on the plan's graph): every link's coupling is scaled by
 * alpha_m beta_l,
 *   x_m' = -V'(x_m) + (K/N) sum_l a_ml alpha_m beta_l g(x_l, x_m).
 * The CIA then uses the weighted moments sum_{l in c} beta_l x_l^a
 * (eq. rank1precompute) and scales the coupling by alpha_m (eq. rank1fast).
 * alpha, beta: host, n doubles each in the original node order, copied; NULL
 * stands for all ones; both NULL removes the weights.  Call cia_state_load
 * again before cia_advance.  CIA_ERR_UNSUPPORTED for other models,
 * CIA_ERR_NUMERIC for a weight that is not finite. */
cia_status cia_plan_set_weights(cia_plan_t *plan, const double *alpha, const double *beta);

/* Cut the plan's communities into tiles again with other tile parameters
 * (the same meaning and limits as in cia_options; 0 = default); the split of
 * S is reused.  The resident state's observables are recomputed on the next
 * cia_state_load, so call it again before cia_advance. */
cia_status cia_plan_retile(cia_plan_t *plan, int tile_nodes, int tile_index_bytes, int staging);

typedef struct {
    int candidates;             /* tilings timed */
    int tile_nodes, tile_index_bytes, staging;   /* the fastest, now the plan's tiling */
    double best_ms_per_step;    /* its device time per RK4 step */
    double worst_ms_per_step;   /* the slowest candidate's */
} cia_tune_report;

/* Autotuner: time `steps` RK4 steps of the CIA (after two warm-up steps) for
 * each candidate tiling -- the window kernel (staging 2) with 256-row tiles
 * and tile_index_bytes 32768, 65536 or 98304, with 128-row tiles and 32768 or
 * with 64-row tiles and 16384,
 * the pipelined (3) and the plain (1) kernel with 256-row tiles and 32768, the
 * ring kernel (4) with 256-row tiles and 49152 or 65536;
 * for Cucker--Smale, 64- or 128-row tiles with 16384 or 32768 -- starting
 * from the state x (device, n x d doubles, original order), and keep the
 * fastest.
 * Leaves x's state resident (cia_state_load).  Synchronises the stream. */
cia_status cia_plan_autotune(cia_plan_t *plan, const double *x, double dt, int64_t steps,
                             cia_tune_report *report, void *stream);

/* Release everything the plan owns (NULL is a no-op). */
cia_status cia_plan_destroy(cia_plan_t *plan);

/* Fill *info with the plan's sizes. */
cia_status cia_plan_get_info(const cia_plan_t *plan, cia_plan_info *info);

/* Bookkeeping of step P1, copied to host arrays the caller allocated:
 *   perm:   n entries, perm[m] = original id of permuted node m (kappa)
 *   offsets: M + 1 entries, community c = permuted ids [offsets[c], offsets[c+1])
 * Either pointer may be NULL. */
cia_status cia_plan_get_permutation(const cia_plan_t *plan, int32_t *perm, int64_t *offsets);

/* The sparse remainder S as two CSRs over PERMUTED ids (host arrays the
 * caller allocated with sizes from cia_plan_info):
 *   miss_rowptr[n+1], miss_col[nnz_missing]: the -1 entries of S except the
 *     diagonal, columns ascending, as permuted global ids;
 *   inter_rowptr[n+1], inter_col[nnz_inter]: the +1 entries, ascending.
 * Any pointer may be NULL. */
cia_status cia_plan_get_split(const cia_plan_t *plan, int64_t *miss_rowptr, int32_t *miss_col,
                              int64_t *inter_rowptr, int32_t *inter_col);

/* ---- evaluation: steps E1 + E2 (Sec. 3.2) --------------------------------- */

/* One right-hand-side evaluation dxdt = H(x) with the CIA:
 * (E1) per-community observables Z_{c,k} = sum_{l in c} e^{i k x_l} and the
 * dense term from them (eq. FastHdense), (E2) the sparse sum over S, plus f.
 * x, dxdt: device, n x d doubles each, original node order; they may not alias.
 * Cucker--Smale: needs a basis (cia_plan_set_basis); the dense term is
 *   sum_r phi_r(s_m) (H_cr - U_cr v_m) with U_c = (1/N) sum_{l in c} phi(s_l),
 *   H_c = (1/N) sum_{l in c} phi(s_l) v_l (eqs. Cucker_Smale_orderParams and
 *   Cucker_Smale_fast_RHS), positions relative to the community centroid.
 * With CIA_FP32 the state is rounded to FP32 and all sums run in FP32
 * (per-community observables with FP64 accumulation across tiles). */
cia_status cia_rhs(cia_plan_t *plan, const double *x, double *dxdt, void *stream);

/* Same result by the direct sum over all CSR neighbours (needs
 * opt.build_direct).  Same layout and precision rules as cia_rhs. */
cia_status cia_rhs_direct(cia_plan_t *plan, const double *x, double *dxdt, void *stream);

/* Advance x by nsteps classical RK4 steps of size dt (the paper allows any
 * Runge-Kutta method, Sec. 3), evaluating every stage with `method`.
 * x: device, n x d doubles, original order, in/out; Kuramoto phases are
 *   returned wrapped to [-pi, pi].  Time accumulation theta += dt sum_s b_s k_s is FP64 in both
 *   precisions; stage states are in the plan's precision.
 * r_out: device, nsteps doubles or NULL; r_out[j] = |(1/N) sum_l e^{i x_l}|
 *   after step j+1 (the Kuramoto order parameter, eq. KuramotoFirstOP);
 *   nsteps x B values for an ensemble (cia_plan_create_batch); must be NULL
 *   for Cucker--Smale and for the polynomial and Fourier couplings.
 * nsteps = 0 only round-trips x through the wrap.
 * Cucker--Smale with method CIA and an error check set (cia_plan_set_check):
 * if a check fails, the remaining steps use the direct method and the call
 * returns CIA_ERR_FALLBACK after completing them (x is valid). */
cia_status cia_integrate(cia_plan_t *plan, int method, double *x, double dt, int64_t nsteps,
                         double *r_out, void *stream);

/* cia_integrate with HOST buffers: copies x (n x d doubles) to the device, runs,
 * copies x back and, if r_out_host is not NULL, writes nsteps x instances order
 * parameters there (step-major, as cia_integrate's r_out), then synchronises
 * the stream.  Pinned host memory makes the copies asynchronous.  The order
 * parameters are staged in mapped pinned host memory that the plan keeps
 * (grown on demand). */
cia_status cia_integrate_host(cia_plan_t *plan, int method, double *x_host, double dt,
                              int64_t nsteps, double *r_out_host, void *stream);

/* ---- resident state: the pieces cia_integrate is made of ------------------ */

/* Load x (device, n x d doubles, original order) into the plan's resident
 * FP64 master state (permuted; Kuramoto phases wrapped to [-pi, pi]) and
 * compute the observables of that state.  Until the next load the plan owns
 * the state. */
cia_status cia_state_load(cia_plan_t *plan, const double *x, void *stream);

/* Copy the resident master state to x (device, n x d doubles, original order). */
cia_status cia_state_store(cia_plan_t *plan, double *x, void *stream);

/* Advance the resident state by nsteps RK4 steps of size dt (see
 * cia_integrate for method and r_out).  One step is four stage launches; the
 * state never leaves the device. */
cia_status cia_advance(cia_plan_t *plan, int method, double dt, int64_t nsteps, double *r_out,
                       void *stream);

/* ---- profiling: CUDA events around every stage launch ---------------------- */

typedef struct {
    int64_t stage_launches;     /* stage kernels launched while profiling */
    double stage_ms;            /* summed device time of those launches */
    int64_t other_launches;     /* other kernels of the plan (observables, order parameter, I/O) */
} cia_profile;

/* Start recording: up to `capacity` stage launches get a CUDA event pair on
 * the launching stream (capacity <= 0 stops recording).  Recording adds two
 * event records per launch. */
cia_status cia_profile_begin(cia_plan_t *plan, int64_t capacity);

/* Stop recording, wait for the recorded events and return the totals. */
cia_status cia_profile_end(cia_plan_t *plan, cia_profile *out);

/* Wait for the plan's work on `stream` and report any asynchronous error.
 * Returns CIA_ERR_TIMEOUT (and clears the flag) if a device-side wait of the
 * plan's kernels gave up since the last cia_sync; results of that work are
 * then invalid. */
cia_status cia_sync(cia_plan_t *plan, void *stream);

/* Failure-detection self-test: launch, on `stream`, a kernel that waits on an
 * mbarrier nothing arrives on, with a bound of limit_ns nanoseconds (1e3 ..
 * 1e9).  The wait gives up, sets the plan's error flag and the kernel
 * returns; the next cia_sync reports CIA_ERR_TIMEOUT and clears the flag.
 * The CUDA context and the plan stay usable. */
cia_status cia_selftest_bounded_wait(cia_plan_t *plan, int64_t limit_ns, void *stream);

/* ---- right-hand side without device allocation --------------------------- */

/* The FP64 Kuramoto CIA right-hand side of cia_rhs, for callers that may not
 * have the library allocate device memory (a host application that owns the
 * device-memory budget through its own pool allocator, or a latency-critical
 * loop where cudaMalloc, which may synchronise the device, is not allowed).
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scratch
 * (phasors and community observables) is one fixed 5 MiB array in device
 * memory.  A device reserves that array when the library's module is loaded
 * there -- at the latest at the first call on that device (under CUDA's
 * default lazy module loading), earlier if modules are loaded eagerly -- and
 * keeps it until the process exits.
 * The paper has no counterpart of this entry point.
 *
 * Everything is in PERMUTED node order (communities contiguous, unlabelled
 * nodes last), as a plan reports it:
 *   offsets: device, M + 1 entries (cia_plan_get_permutation);
 *   miss_rowptr/miss_col, inter_rowptr/inter_col: device CSRs of the missing
 *     and inter-community links over permuted ids (cia_plan_get_split);
 *     the column arrays may be NULL when they have no entries;
 *   x, omega, dxdt: device, n doubles (omega may be NULL = 0);
 *   coupling: host, CIA_MODEL_KURAMOTO with p harmonics.
 * Limit: p * (n + M) <= 327680 (n and M each at most 327680), otherwise
 * CIA_ERR_INVALID_ARG and nothing runs.
 * The first call on a device (and the first after a device reset, which gives
 * the device a new context) resolves the scratch array's device address with
 * that device current, which may load the module; make that first call
 * before any stream capture.
 * All calls share the scratch array: calls that can overlap on the GPU (e.g.
 * on unordered streams) race with each other. */
cia_status cia_rhs_kuramoto_static(int64_t n, int64_t M, const int64_t *offsets,
                                   const int64_t *miss_rowptr, const int32_t *miss_col,
                                   const int64_t *inter_rowptr, const int32_t *inter_col,
                                   const double *x, const double *omega,
                                   const cia_coupling *coupling, double *dxdt, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CIA_H */
