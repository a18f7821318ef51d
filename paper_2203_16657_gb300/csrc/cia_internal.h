// Internal declarations of libcia: the plan object and the kernel launchers.
// Not part of the public ABI (include/cia.h is).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "cia.h"

// Features per node of the general separable couplings (general_coupling.cu):
// 1, cos, sin of up to CIA_MAX_HARMONICS harmonics.
#define CIA_GC_MAX_FEATURES (2 * CIA_MAX_HARMONICS + 1)

namespace cia {

// Thread-local error text behind cia_last_error().
void set_error(const std::string &msg);
void clear_error();
cia_status cuda_fail(cudaError_t e, const char *what);

#define CIA_CUDA_TRY(expr)                                                  \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) return ::cia::cuda_fail(_e, #expr);          \
    } while (0)

// Padding entries of the missing-link vectors are lambda_c + 1 .. lambda_c +
// kPadSlots (each a distinct shared-memory bank group, so that padding never
// conflicts with a live gather), or lambda_c itself for communities too large
// for that range in 16 bits; kernels that stage the community in shared
// memory keep the entries lambda_c .. lambda_c + kPadSlots after it zero (entry
// lambda_c is a guard that a copy rounded up to 16 bytes may overwrite before
// the ring kernel reads the window), the others skip any index >= lambda_c.
constexpr int kPadSlots = 16;

// Most slices of one tile that the persistent ring kernel's slot header holds
// (their phasor sums are added in slice order into the tile partial).
constexpr int kRingMaxSlices = 32;

// Descriptor of one work tile (64 bytes, read by every CIA kernel).
struct alignas(16) TileDesc {
    int32_t comm, first, count, nsl;      // community (-1: unlabelled), first node, nodes, slices
    uint32_t blob_bytes, mvec_off, ivec_off, lam;   // blob size; byte offsets of its vector sections
    int64_t blob_off;                     // byte offset of the blob
    int64_t lo;                           // first node of the community
    int32_t run, pbuf, shift;             // community run inside the CTA's tile range, its buffer,
                                          // lo - (lo rounded down to 16 bytes of phasors)
    uint32_t vtab_off;                    // byte offset of the row -> chunk table
};
static_assert(sizeof(TileDesc) == 64, "tile descriptor is 64 bytes");

// Device layout of one plan.  All node-indexed arrays are in PERMUTED order
// (communities contiguous, unlabelled nodes last).
struct DeviceBuffers {
    // step P1 bookkeeping
    int32_t *perm = nullptr;            // [n] permuted -> original id
    int64_t *off = nullptr;             // [M+1]
    // work tiles: a tile is a run of consecutive nodes of one community
    int32_t *tile_comm = nullptr;       // [T] community id, -1 for unlabelled nodes
    int32_t *tile_first = nullptr;      // [T] first permuted node
    int32_t *tile_count = nullptr;      // [T] nodes in the tile
    int32_t *comm_tile_begin = nullptr; // [M+1] tiles of community c: [begin[c], begin[c+1])
    // S, split in its two signs, as sliced ELL: a slice is 32 rows of a tile
    // (one per lane), rows ordered by decreasing list length; missing lists
    // hold 16-bit community-local indices (padding lambda_c .. lambda_c + 15), inter lists
    // 32-bit permuted ids (sentinel n); vector j of lane r sits at
    // slice_offset + 32 j + r.  Each tile is one contiguous blob:
    //   [slice descriptors: nsl x uint4 (miss offset, miss vectors, inter offset, inter vectors)]
    //   [row maps: nsl x 32 x u32 (lane -> missing chunk | inter row << 16, 0xffff = none)]
    //   [row -> chunk table: count x u32 (first chunk | chunks << 16), padded to 16 bytes]
    //   [missing vectors over chunks: 8 x u16][inter vectors over rows: 4 x i32]
    // A missing list longer than 64 entries is split into chunks whose
    // partial sums are added per row in chunk order.
    cia::TileDesc *tile_desc = nullptr; // [T]
    int32_t *tile_order = nullptr;      // [T] launch order of the per-tile kernels (costliest first)
    int32_t *gc_tiles = nullptr;        // [T] general couplings: tiles by community size, largest first
    unsigned char *blob = nullptr;      // [sum of blob bytes]
    int32_t *cta_tile_begin = nullptr;  // [n_ctas+1] tile range of each persistent CTA
    int32_t *cta_runs = nullptr;        // [n_ctas] community runs (maximal same-community tile runs) per CTA
    // full permuted CSR for the direct method (optional), rows padded to
    // whole 4 x i32 vectors with the sentinel n
    int64_t *full_rowptr = nullptr;     // [n+1]
    int32_t *full_col = nullptr;        // [padded nnz]
    // model
    void *omega = nullptr;              // [n] compute precision
    // work buffers
    double *theta = nullptr;            // [n] FP64 master state
    void *acc = nullptr;                // [n] sum_s b_s C_s, compute precision
    void *ph[2] = {nullptr, nullptr};   // [p][n] complex phasors e^{i k y}, compute precision
    double *part[2] = {nullptr, nullptr}; // [T][p] complex tile sums (FP64)
    double *zsum[2] = {nullptr, nullptr}; // [M][p] complex community observables Z_c (FP64; ring kernel)
    int *comm_done = nullptr;           // [M] tiles of the community finished in the running launch
    void *wdt_half = nullptr;           // [n] wrap(dt omega / 2), compute precision
    void *wdt_full = nullptr;           // [n] wrap(dt omega), compute precision
    double *wdt_full64 = nullptr;       // [n] wrap(dt omega), FP64
    double *rhs_tmp = nullptr;          // [n] staging for host-buffer calls
    void *tri = nullptr;                // [n] triadic term by the direct method (higher-order model)
    double *x_tmp = nullptr;            // [n] staging for host-buffer calls
    int *err_flag = nullptr;            // set by a kernel whose bounded wait gave up (device alias
                                        // of err_flag_host)
    int *err_flag_host = nullptr;       // the flag in mapped pinned host memory, read by cia_sync
    double *r_tmp = nullptr;            // [r_cap] staging for order parameters (device alias
                                        // of r_tmp_host)
    double *r_tmp_host = nullptr;       // the same in mapped pinned host memory
    int64_t r_cap = 0;
    // Cucker--Smale (4 state values per node)
    float4 *cs_y[2] = {nullptr, nullptr};     // [n] FP32 stage states (s_x, s_y, v_x, v_y)
    double *cs_master = nullptr;              // [n][4] FP64 master state
    float4 *cs_acc = nullptr;                 // [n] sum_s b_s k_s
    void *cs_feat = nullptr;                  // [n][64] BF16 features of the current stage state
    double *cs_part[2] = {nullptr, nullptr};  // [T][192] tile sums of phi, phi v_x, phi v_y
    float *cs_params = nullptr;               // basis parameters (FP32 master copy)
    void *cs_wimage = nullptr;                // the basis weights in their shared-memory layout (BF16 W2)
    int32_t *cs_check_nodes = nullptr;        // [check_count] sampled community nodes
    int32_t *cs_check_comm = nullptr;         // their communities
    double *cs_check_out = nullptr;           // [check_count][2] error, reference
    float2 *cs_cen = nullptr;                 // [M] community centroids (pair sampling)
    float2 *cs_shift = nullptr;               // [M] shift of phi's input during one RK4 step
    // general couplings (FP64 stage states and tile feature sums)
    double *gc_y[2] = {nullptr, nullptr};     // [n+1] stage states
    double *gc_part[2] = {nullptr, nullptr};  // [T][K] sums of the (beta-weighted) features per tile
    double *gc_alpha = nullptr, *gc_beta = nullptr;  // [n] rank-one link weights (permuted)
    double *gc_f[2] = {nullptr, nullptr};     // Fourier basis: [n][K-1] features of gc_y
    // ensembles of independent networks
    void *tile_kn = nullptr;                  // [T] K / N_i of the tile's instance, compute precision
    int32_t *inst_tiles = nullptr;            // [B][4] community tiles [0,1), free tiles [2,3) of instance i
    int64_t *inst_off = nullptr;              // [B+1] node offsets of the instances
    int64_t *r_counter = nullptr;             // step index of the next order-parameter row
};

struct BatchStaging;   // instances of a streamed ensemble plan before cia_plan_batch_finish

// The split of S kept on the host after planning (re-tiling reuses it).
struct HostSplit {
    std::vector<int32_t> comm_of;              // [n] community of permuted node m, -1 if none
    std::vector<int64_t> miss_cnt, miss_off;   // per row: missing links, offsets into miss_local
    std::vector<uint16_t> miss_local;          // community-local indices, ascending per row (only
                                               // when every community has at most 65535 nodes)
    std::vector<int64_t> inter_cnt, inter_off; // per row: inter links, offsets into inter_col
    std::vector<int32_t> inter_col;            // permuted ids, ascending per row
};

}  // namespace cia

struct cia_plan {
    int device = 0;
    int64_t n = 0, M = 0, n_free = 0, max_comm = 0;
    int64_t nnz_graph = 0, nnz_missing = 0, nnz_inter = 0, n_tiles = 0;
    int64_t device_bytes = 0;
    int precision = CIA_FP64;
    int model = CIA_MODEL_KURAMOTO;
    int p = 1;
    double d_sin[CIA_MAX_HARMONICS] = {0};
    double d_cos[CIA_MAX_HARMONICS] = {0};
    double K = 0.0;
    double K2 = 0.0;                    // triadic coupling (higher-order model)
    bool triadic = false;               // higher-order model: Z_1 and Z_2 are carried (p >= 2)
    int tile_nodes = 256;
    int group_size = 8;                 // threads per row, CIA sparse sums
    int group_size_direct = 32;         // threads per row, direct sums
    int miss_idx_bytes = 2;
    int has_direct = 0;
    int64_t ph_stride = 0;              // phasor entries per harmonic: n + 1 rounded up to even
    int tile_index_bytes = 24576;
    int64_t max_tile_idx_bytes = 0;     // largest index footprint of one tile (bytes)
    int64_t max_tile_buf = 0;           // largest window + blob of one tile (persistent ring kernel)
    int ring_slots = 0;                 // ring slots of the persistent ring kernel (staging 4)
    bool blob_segmented = false;        // blobs in the ring kernel's layout (rows on consecutive lanes)
    int64_t n_slices = 0, blob_bytes = 0, max_cta_tiles = 0, max_cta_runs = 0;
    int n_ctas = 0;                     // persistent grid of the pipelined CIA kernel (one per SM)
    int ring_stages = 0;                // tile buffers of its TMA ring
    int staging = 2;                    // kernel: 1 = plain loads, 2 = per-tile CTAs with the community
                                        // window in shared memory, 3 = persistent TMA pipeline
    double dt_cached = 0.0;             // dt the wdt_* buffers were computed for
    bool wdt_valid = false;
    std::vector<int32_t> perm;          // host copy of kappa
    std::vector<int64_t> off;           // host copy of the offsets
    cia::DeviceBuffers d;
    std::vector<void *> allocations;    // everything to cudaFree
    // profiling (cia_profile_begin / cia_profile_end)
    bool prof_on = false;
    int64_t prof_cap = 0, prof_used = 0, prof_other = 0;
    std::vector<cudaEvent_t> prof_ev;   // 2 per recorded launch
    int state_slot = 0;                 // phasor/partial slot holding the resident state
    int n_sms = 0;
    cia::HostSplit hs;
    std::vector<void *> tile_allocs;    // device buffers of the current tiling
    int64_t tile_bytes = 0;
    int staging_req = 0;                // staging the caller asked for (the tiling may downgrade it)
    int use_graphs = 0;                 // 0: one CUDA graph per RK4 step when advancing >= 2 steps
    // ensembles of independent networks (cia_plan_create_batch)
    int64_t B = 1;
    std::vector<int64_t> inst_off;      // [B+1] node offsets (original ids)
    std::vector<int64_t> inst_comm_off; // [B+1] community offsets
    cia::BatchStaging *batch_stage = nullptr;   // streamed ensemble plan being built
    // CUDA graph of one RK4 step (cached by method, dt, slot and order-parameter output)
    cudaGraphExec_t graph_exec = nullptr;
    int graph_method = -1, graph_slot = -1;
    bool graph_r = false;
    double graph_dt = 0.0;
    double *graph_r_out = nullptr;
    cudaStream_t capture_stream = nullptr;
    bool needs_load = false;            // the tiling changed since the last cia_state_load
    // Cucker--Smale
    int state_dim = 1;                  // FP64 values per node at the boundary
    double cs_sigma = 1.0, cs_beta = 0.0;
    // general couplings (polynomial and Fourier; model CIA_MODEL_POLYNOMIAL internally)
    int poly_p = 0;                     // polynomial degree (1..4), or harmonics (Fourier)
    int smem_optin = 0;                 // opt-in shared memory per block of the device
    int smem_per_sm = 0;                // shared memory per SM of the device
    std::vector<int64_t> gc_tile_lam;   // community size of each tile in gc_tiles' order
    cudaStream_t gc_side[4] = {};       // general couplings: streams of the concurrent window launches
    cudaEvent_t gc_fork = nullptr, gc_join[4] = {};
    double poly_c[CIA_MAX_POLY + 1] = {0};  // difference form: h
    double poly_dv[CIA_MAX_POLY + 1] = {0}; // V'
    bool poly_general = false;          // g(x_l, x_m) instead of h(x_l - x_m)
    bool gc_weighted = false;           // rank-one link weights alpha_m beta_l
    int gc_basis = 0;                   // general couplings: 0 polynomial, 1 real Fourier features
    int gc_k = 2;                       // features per node incl. the constant
    double gc_w = 0.0;                  // Fourier basis: pi / L
    double gc_e[CIA_GC_MAX_FEATURES * CIA_GC_MAX_FEATURES] = {0};  // g = sum E_kj phi_k(u) phi_j(y)
    double poly_g[(CIA_MAX_POLY + 1) * (CIA_MAX_POLY + 1)] = {0};
    bool cs_has_basis = false;          // a basis was set (cia_plan_set_basis)
    bool cs_feat_valid = false;         // features/partials match the resident state
    int64_t cs_check_count = 0;
    int64_t check_every = 0;            // steps between learned-basis checks (0 = off)
    double check_bound = 0.0;
    int64_t checks = 0;
    double check_last = 0.0, check_max = 0.0;
    bool fell_back = false;
    int64_t fallback_step = -1;
};

namespace cia {

// Kernel launchers (kuramoto.cu).  All return cudaGetLastError() of the launch.
struct Method {
    enum { CIA = 0, DIRECT = 1 };
};

cudaError_t launch_phasors_from_x(cia_plan *pl, const double *x, bool write_master, int ph_slot,
                                  cudaStream_t s);
cudaError_t launch_rhs(cia_plan *pl, int method, int ph_slot, double *dxdt, cudaStream_t s);
cudaError_t launch_omega_constants(cia_plan *pl, double dt, cudaStream_t s);
cudaError_t launch_rk4_stage(cia_plan *pl, int method, int stage, int ph_in_slot, double dt,
                             cudaStream_t s);
cudaError_t launch_scatter_master(cia_plan *pl, double *x, cudaStream_t s);
size_t stage_smem_bytes(const cia_plan *pl, int method);
size_t pipeline_smem_bytes(const cia_plan *pl, int stages);
size_t stream_smem_bytes(const cia_plan *pl);
int ring_slots_that_fit(const cia_plan *pl);
int64_t stream_tile_buf_bytes(const cia_plan *pl, int64_t lam, int64_t blob_bytes);
size_t window_smem_bytes(const cia_plan *pl);

// Drop the cached CUDA graph of an RK4 step (api.cu).
void invalidate_graphs(cia_plan *pl);

// Checks a graph as cia_plan_create does (plan.cpp); sets the error message.
cia_status validate_graph(const cia_graph *g);

// Raises `kernel`'s dynamic shared-memory limit on `device` to at least
// `smem` bytes when that is above the default 48 KB; remembers the largest
// value set per (kernel, device), so a repeated launch costs one lookup.
cudaError_t ensure_dynamic_smem(const void *kernel, int device, size_t smem);
// Order parameters of every instance of the state in slot `slot`:
// r_base[counter * B + i], then ++counter (kuramoto.cu).
cudaError_t launch_order_parameters(cia_plan *pl, int slot, double *r_base, cudaStream_t s);

// Cucker--Smale launchers (cucker_smale.cu).
cudaError_t cs_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s);
cudaError_t cs_launch_features(cia_plan *pl, int slot, cudaStream_t s);
cudaError_t cs_launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s);
cudaError_t cs_launch_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s);
cudaError_t cs_launch_store(cia_plan *pl, double *x, cudaStream_t s);
cudaError_t cs_launch_check(cia_plan *pl, int slot, cudaStream_t s);
cudaError_t cs_launch_sample(cia_plan *pl, int slot, int64_t count, uint64_t seed, float *pairs, cudaStream_t s);
size_t cs_stage_smem_bytes(const cia_plan *pl);
// Pack the plan's basis parameters into the shared-memory image that every
// feature-evaluating CTA copies (after cia_plan_set_basis).
cudaError_t cs_pack_weights(cia_plan *pl, cudaStream_t s);

// General-coupling launchers (general_coupling.cu): the polynomial models and the
// real 2-D Fourier model, all kept under model CIA_MODEL_POLYNOMIAL internally.
cudaError_t gc_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s);
cudaError_t gc_launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s);
cudaError_t gc_launch_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s);

}  // namespace cia
