// Device kernels of the polynomial couplings with a potential, FP64:
//   difference form (eq. GeneralNetworkPolyDifference, App. A.3; Desai-Zwanzig,
//   App. A.5):  x_m' = -V'(x_m) + (K/N) sum_l a_ml h(x_l - x_m),
//               h(x) = sum_{a=0..p} c_a x^a;
//   general form (eq. GeneralNetworkPoly, eq. PolyApprox):
//               x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),
//               g(u, y) = sum_{a,b=0..p} G_ab u^a y^b;
//   V'(x) = sum_{j=0..4} v_j x^j.
//
// CIA (steps E1 + E2) for m in community c with moments W_ck = sum_{l in c} x_l^k:
//   difference: sum_{l in c} h(x_l - x_m) = sum_a c_a sum_{k=0..a} binom(a, k)
//   W_ck (-x_m)^{a-k} (eq. PolyDifferenceRHSfast without the 1/N);
//   general: sum_{l in c} g(x_l, x_m) = sum_a W_ca e_a(x_m) with
//   e_a(y) = sum_b G_ab y^b (eq. PolyRHS without the 1/N);
//   then minus the diagonal l = m (a_mm = 0), minus the coupling over the
//   missing links, plus the coupling over the inter-community links.
//
// One CTA (256 threads) per tile and launch: (0) the community's moments from
// the previous launch's tile sums and its states in shared memory, (A) the
// sparse sums over the tile's sliced-ELL blob (missing links from shared
// memory), (B) one thread per node: dense term, RK4 stage update and the
// tile's sums of the powers of the next stage state.  The direct method's
// kernel has the same epilogue, so either method leaves valid moments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cia_internal.h"

namespace cia {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxChunks = 512;
constexpr int kTileMax = 256;
constexpr int kMaxP = CIA_MAX_POLY;

enum PolyMode { kRhs = 0, kStage = 1, kFinal = 2 };

struct PolyParams {
    int64_t n;
    int p;                       // degree of h
    double c[kMaxP + 1];         // h
    double v[kMaxP + 1];         // V'
    double g[kMaxP + 1][kMaxP + 1];  // general form: G_ab, zero above degree p
    double k_over_n;
    int group;                   // threads per row of the direct kernel
    int win_cap;                 // shared-memory window capacity (nodes); 0 = read the
                                 // community's states from global memory
    const TileDesc *tile_desc;
    const unsigned char *blob;
    const int32_t *comm_tile_begin;
    const int64_t *full_rowptr;
    const int32_t *full_col;
    const double *y_in;          // [n] stage state (permuted)
    double *y_out;               // [n] next stage state
    const double *part_in;       // [tiles][p+1] sums of y_in^k
    double *part_out;            // [tiles][p+1] sums of y_out^k
    double *acc, *theta;         // RK4 accumulator, FP64 master
    const int32_t *perm;
    double *rhs_out;             // kRhs: original order
    double c_next_dt, b_s, dt;
    int first_stage;
};

__device__ __forceinline__ double horner(const double *c, int p, double x) {
    double s = 0.0;
    for (int a = p; a >= 0; --a) s = fma(s, x, c[a]);
    return s;
}

// The coupling of one node y against its neighbours u: h(u - y) (difference
// form) or g(u, y) = sum_a e_a(y) u^a (general form, e_a precomputed per node).
// Coefficients above degree p are zero, so the full-degree Horner chain gives
// the degree-p value exactly.
template <bool GEN>
struct Coupling {
    double e[kMaxP + 1];
    double y;
    __device__ __forceinline__ Coupling(const PolyParams &a, double y_) : y(y_) {
        if (GEN) {
#pragma unroll
            for (int al = 0; al <= kMaxP; ++al) {
                double s = 0.0;
#pragma unroll
                for (int b = kMaxP; b >= 0; --b) s = fma(s, y_, a.g[al][b]);
                e[al] = s;
            }
        }
    }
    __device__ __forceinline__ double operator()(const PolyParams &a, double u) const {
        double s = 0.0;
        if (GEN) {
#pragma unroll
            for (int al = kMaxP; al >= 0; --al) s = fma(s, u, e[al]);
        } else {
            const double d = u - y;
#pragma unroll
            for (int al = kMaxP; al >= 0; --al) s = fma(s, d, a.c[al]);
        }
        return s;
    }
};

// RK4 stage update from the derivative k; returns the next stage state.
template <int MODE>
__device__ __forceinline__ double rk4_update(const PolyParams &a, int64_t m, double k) {
    if (MODE == kRhs) {
        a.rhs_out[a.perm[m]] = k;
        return 0.0;
    }
    const double s = (a.first_stage ? 0.0 : a.acc[m]) + a.b_s * k;
    double y;
    if (MODE == kStage) {
        a.acc[m] = s;
        y = a.theta[m] + a.c_next_dt * k;
    } else {
        y = a.theta[m] + a.dt * s;   // FP64 time accumulation x += dt sum_s b_s k_s
        a.theta[m] = y;
    }
    a.y_out[m] = y;
    return y;
}

// Sums over the tile of y^k, k = 0..p (each thread contributes its node's
// value, nothing when it has no node), in a fixed order, to part_out[tile].
__device__ __forceinline__ void tile_power_sums(int p, double *part_out, int tile, bool live, double y,
                                                double (*red)[kMaxP + 1]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double pw[kMaxP + 1];
    double q = 1.0;
#pragma unroll
    for (int k = 0; k <= kMaxP; ++k) {
        pw[k] = live ? q : 0.0;
        q *= y;
    }
#pragma unroll
    for (int k = 0; k <= kMaxP; ++k)
        for (int o = 16; o > 0; o >>= 1) pw[k] += __shfl_xor_sync(0xffffffffu, pw[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k <= kMaxP; ++k) red[warp][k] = pw[k];
    __syncthreads();
    if (threadIdx.x <= p) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        part_out[(int64_t)tile * (p + 1) + threadIdx.x] = s;
    }
}

// Dense term of node state x: the community sum of the coupling from the
// moments W, without the diagonal term (h(0) = c_0, or g(x, x)).
template <bool GEN>
__device__ __forceinline__ double dense_from_moments(const PolyParams &a, const double *W, double x) {
    if (GEN) {
        const Coupling<true> cx(a, x);
        double dense = 0.0;
#pragma unroll
        for (int al = 0; al <= kMaxP; ++al)
            if (al <= a.p) dense = fma(W[al], cx.e[al], dense);
        return dense - cx(a, x);
    }
    double dense = 0.0;
    for (int al = 0; al <= a.p; ++al) {
        double inner = 0.0, binom = 1.0, negx = 1.0;
        // sum_{k=0..al} binom(al, k) W_k (-x)^{al-k}, accumulated from k = al down
        for (int k = al; k >= 0; --k) {
            inner = fma(binom * W[k], negx, inner);
            negx *= -x;
            binom = binom * (double)k / (double)(al - k + 1);
        }
        dense = fma(a.c[al], inner, dense);
    }
    return dense - a.c[0];
}

template <int MODE, bool GEN>
__global__ void __launch_bounds__(kThreads) poly_stage_kernel(const PolyParams a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double yrow[kTileMax];
    __shared__ double W[kMaxP + 1];
    __shared__ double red[kWarps][kMaxP + 1];
    double *win = reinterpret_cast<double *>(smem_raw);            // [win_cap] community states
    double *sWm = win + a.win_cap;                                  // [kMaxChunks] missing-chunk sums
    double *sWi = sWm + kMaxChunks;                                 // [kTileMax] inter sums per row
    uint16_t *chunk_row = reinterpret_cast<uint16_t *>(sWi + kTileMax);
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool comm = d.comm >= 0;
    const int lam = comm ? (int)d.lam : 0;
    const int count = d.count;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned char *b = a.blob + d.blob_off;
    const uint32_t *vtab = reinterpret_cast<const uint32_t *>(b + d.vtab_off);
    const double *cw = a.win_cap ? win : a.y_in + d.lo;
    // (0) window, own rows, moments (FP64 over the community's tiles), chunk table
    if (a.win_cap)
        for (int i = threadIdx.x; i < lam; i += kThreads) win[i] = a.y_in[d.lo + i];
    if (threadIdx.x < count) {
        yrow[threadIdx.x] = a.y_in[d.first + threadIdx.x];
        const uint32_t vt = __ldg(vtab + threadIdx.x);
        for (uint32_t c = vt & 0xffffu; c < (vt & 0xffffu) + (vt >> 16); ++c) chunk_row[c] = (uint16_t)threadIdx.x;
    }
    if (comm && warp == 0) {
        const int u0 = a.comm_tile_begin[d.comm], u1 = a.comm_tile_begin[d.comm + 1];
        for (int k = 0; k <= a.p; ++k) {
            double s = 0.0;
            for (int u = u0 + lane; u < u1; u += 32) s += a.part_in[(int64_t)u * (a.p + 1) + k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) W[k] = s;
        }
    }
    __syncthreads();
    // (A) sparse sums: warp per slice, lane per missing chunk and inter row
    const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
    const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
    const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
    const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);
    for (int s = warp; s < d.nsl; s += kWarps) {
        const uint4 sd = __ldg(sdesc + s);
        const uint32_t rows = __ldg(srows + s * 32 + lane);
        const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
        double ms = 0.0, is = 0.0;
        {
            const Coupling<GEN> cp(a, yrow[mrow != 0xffffu ? chunk_row[mrow] : 0]);
            const uint4 *mv = mvec + sd.x + lane;
            for (uint32_t j = 0; j < sd.y; ++j) {
                const uint4 q = __ldg(mv + 32 * j);
                const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int l0 = (int)(w4[e] & 0xffffu), l1 = (int)(w4[e] >> 16);
                    if (l0 < lam) ms += cp(a, cw[l0]);
                    if (l1 < lam) ms += cp(a, cw[l1]);
                }
            }
        }
        {
            const Coupling<GEN> cp(a, yrow[irow != 0xffffu ? irow : 0]);
            const int4 *iv = ivec + sd.z + lane;
            for (uint32_t j = 0; j < sd.w; ++j) {
                const int4 q = __ldg(iv + 32 * j);
                const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (l4[e] < a.n) is += cp(a, __ldg(a.y_in + l4[e]));
            }
        }
        if (mrow != 0xffffu) sWm[mrow] = ms;
        if (irow != 0xffffu) sWi[irow] = is;
    }
    __syncthreads();
    // (B) thread per node
    const bool live = threadIdx.x < count;
    double ynext = 0.0;
    if (live) {
        const int r = threadIdx.x;
        const int64_t m = d.first + r;
        const double x = yrow[r];
        double sparse = sWi[r];
        const uint32_t vt = __ldg(vtab + r);
        for (uint32_t c = vt & 0xffffu; c < (vt & 0xffffu) + (vt >> 16); ++c) sparse -= sWm[c];
        const double dense = comm ? dense_from_moments<GEN>(a, W, x) : 0.0;
        const double k = -horner(a.v, kMaxP, x) + a.k_over_n * (dense + sparse);
        ynext = rk4_update<MODE>(a, m, k);
    }
    if (MODE == kRhs) return;
    tile_power_sums(a.p, a.part_out, t, live, ynext, red);
}

// Direct method, one CTA per tile: `group` threads per row sum h(x_l - x_m)
// over the row's CSR neighbours (rows padded to 4-entry vectors with the
// sentinel n), then the same update and power sums as the CIA.
template <int MODE, bool GEN>
__global__ void __launch_bounds__(kThreads) poly_direct_kernel(const PolyParams a) {
    __shared__ double sW[kTileMax];
    __shared__ double red[kWarps][kMaxP + 1];
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const int G = a.group, gl = threadIdx.x % G, grp = threadIdx.x / G, ngrp = kThreads / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int4 *col4 = reinterpret_cast<const int4 *>(a.full_col);
    for (int r = grp; r < d.count; r += ngrp) {
        const int64_t m = d.first + r;
        const Coupling<GEN> cp(a, a.y_in[m]);
        double s = 0.0;
        for (int64_t v = a.full_rowptr[m] / 4 + gl; v < a.full_rowptr[m + 1] / 4; v += G) {
            const int4 q = __ldg(col4 + v);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (l4[e] < a.n) s += cp(a, __ldg(a.y_in + l4[e]));
        }
        for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (gl == 0) sW[r] = s;
    }
    __syncthreads();
    const bool live = threadIdx.x < d.count;
    double ynext = 0.0;
    if (live) {
        const int64_t m = d.first + threadIdx.x;
        const double x = a.y_in[m];
        const double k = -horner(a.v, kMaxP, x) + a.k_over_n * sW[threadIdx.x];
        ynext = rk4_update<MODE>(a, m, k);
    }
    if (MODE == kRhs) return;
    tile_power_sums(a.p, a.part_out, t, live, ynext, red);
}

// State load: x (original order) -> master (optional) and stage state,
// with the tile sums of its powers.  One CTA per tile.
__global__ void __launch_bounds__(kThreads) poly_load_kernel(const PolyParams a, const double *x, double *master) {
    __shared__ double red[kWarps][kMaxP + 1];
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool live = threadIdx.x < d.count;
    double y = 0.0;
    if (live) {
        const int64_t m = d.first + threadIdx.x;
        y = x[a.perm[m]];
        if (master) master[m] = y;
        a.y_out[m] = y;
    }
    tile_power_sums(a.p, a.part_out, t, live, y, red);
}

size_t window_cap(const cia_plan *pl) { return (size_t)((pl->max_comm + 1) & ~(int64_t)1); }
constexpr size_t kTables = kMaxChunks * 8 + kTileMax * 8 + kMaxChunks * 2;

// The largest community fits the shared-memory window (the kernel's static
// shared memory is under 4 KB).
bool window_fits(const cia_plan *pl) {
    return window_cap(pl) * 8 + kTables + 4096 <= (size_t)pl->smem_optin;
}

size_t stage_smem(const cia_plan *pl) { return (pl->staging == 2 ? window_cap(pl) * 8 : 0) + kTables; }

PolyParams base_params(const cia_plan *pl, int slot) {
    PolyParams a{};
    const auto &d = pl->d;
    a.n = pl->n;
    a.p = pl->poly_p;
    for (int k = 0; k <= kMaxP; ++k) {
        a.c[k] = k <= pl->poly_p ? pl->poly_c[k] : 0.0;
        a.v[k] = pl->poly_dv[k];
        for (int b = 0; b <= kMaxP; ++b) a.g[k][b] = pl->poly_g[k * (kMaxP + 1) + b];
    }
    a.k_over_n = pl->K / (double)pl->n;
    a.group = pl->group_size_direct;
    a.win_cap = pl->staging == 2 ? (int)window_cap(pl) : 0;
    a.tile_desc = d.tile_desc;
    a.blob = d.blob;
    a.comm_tile_begin = d.comm_tile_begin;
    a.full_rowptr = d.full_rowptr;
    a.full_col = d.full_col;
    a.y_in = d.pl_y[slot];
    a.y_out = d.pl_y[slot ^ 1];
    a.part_in = d.pl_part[slot];
    a.part_out = d.pl_part[slot ^ 1];
    a.acc = d.theta == nullptr ? nullptr : static_cast<double *>(d.acc);
    a.theta = d.theta;
    a.perm = d.perm;
    return a;
}


// One launch of `kernel`, one tile per CTA; ID tells the instantiations apart
// so that each kernel keeps its own configured shared-memory limit.
template <int ID>
cudaError_t launch(void (*kernel)(PolyParams), const cia_plan *pl, size_t smem, const PolyParams &a,
                   cudaStream_t s) {
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = smem;
    }
    void *args[] = {const_cast<PolyParams *>(&a)};
    return cudaLaunchKernel((const void *)kernel, dim3((unsigned)pl->n_tiles), dim3(kThreads), args, smem, s);
}

template <int MODE, bool GEN>
cudaError_t launch_form(const cia_plan *pl, int method, const PolyParams &a, cudaStream_t s) {
    constexpr int id = 2 * MODE + (GEN ? 1 : 0);
    if (method == Method::DIRECT) return launch<id + 6>(poly_direct_kernel<MODE, GEN>, pl, 0, a, s);
    return launch<id>(poly_stage_kernel<MODE, GEN>, pl, stage_smem(pl), a, s);
}

template <int MODE>
cudaError_t launch_mode(const cia_plan *pl, int method, const PolyParams &a, cudaStream_t s) {
    return pl->poly_general ? launch_form<MODE, true>(pl, method, a, s) : launch_form<MODE, false>(pl, method, a, s);
}

}  // namespace

bool poly_window_fits(const cia_plan *pl) { return window_fits(pl); }

cudaError_t poly_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    // the load writes the state and its power sums into slot `slot`
    PolyParams a = base_params(pl, slot ^ 1);
    poly_load_kernel<<<(unsigned)pl->n_tiles, kThreads, 0, s>>>(a, x, write_master ? pl->d.theta : nullptr);
    return cudaGetLastError();
}

cudaError_t poly_launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s) {
    PolyParams a = base_params(pl, slot);
    a.rhs_out = dxdt;
    return launch_mode<kRhs>(pl, method, a, s);
}

cudaError_t poly_launch_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s) {
    static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    static const double c_next[4] = {0.5, 0.5, 1.0, 0.0};
    PolyParams a = base_params(pl, slot);
    a.b_s = b[stage - 1];
    a.c_next_dt = c_next[stage - 1] * dt;
    a.dt = dt;
    a.first_stage = stage == 1;
    return stage == 4 ? launch_mode<kFinal>(pl, method, a, s) : launch_mode<kStage>(pl, method, a, s);
}

}  // namespace cia
