// Device kernels of the polynomial couplings with a potential, FP64:
//   difference form (eq. GeneralNetworkPolyDifference, App. A.3; Desai-Zwanzig,
//   App. A.5):  x_m' = -V'(x_m) + (K/N) sum_l a_ml h(x_l - x_m),
//               h(x) = sum_{a=0..p} c_a x^a;
//   general form (eq. GeneralNetworkPoly, eq. PolyApprox):
//               x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),
//               g(u, y) = sum_{a,b=0..p} G_ab u^a y^b;
//   V'(x) = sum_{j=0..4} v_j x^j.
//
// Both forms are sums of the neighbours' powers: sum_l a_ml g(x_l, x_m) =
// sum_a T_a(m) e_a(x_m) with T_a(m) = sum_l a_ml x_l^a and e_a(y) = sum_b E_ab y^b,
// where E = G for the general form (eq. PolyRHS) and E_ab = c_{a+b} binom(a+b, a)
// (-1)^b for the difference form (eq. PolyDifferenceRHSfast, its sum over a
// regrouped by the power of the moment).  The CIA splits T_a(m) as in steps
// E1 + E2: the community moment W_ca = sum_{l in c} x_l^a (eq. PolyMoments,
// without the 1/N), minus the diagonal x_m^a (a_mm = 0), minus the power sums
// over the missing links, plus those over the inter-community links.  Every
// link therefore costs p - 1 multiplications and p additions in FP64 (one
// addition for Desai-Zwanzig), not an evaluation of g.
//
// FP64 additions are scarce on this GPU (a few per clock and SM), so the
// missing-link sums, the bulk of the work, are exact integer sums: the tile's
// window holds each power of the community's states as a 64-bit fixed-point
// number, u^a = M 2^E_a with |M| < 2^55 and E_a set by the community's largest
// |u^a|, so that a chunk of at most 64 links sums without overflow.  The
// rounding to the grid 2^E_a (at most 2^-56 of the largest value) is below the
// rounding error of an FP64 sum of the same values.
//
// One CTA (256 threads) per tile and launch: (0) the community's moments from
// the previous launch's tile sums and the powers of its states in shared
// memory, (A) the sparse power sums over the tile's sliced-ELL blob,
// (B) one thread per node: T_a, the coupling, RK4 stage update and the tile's
// sums of the powers of the next stage state.  The direct method's kernel
// evaluates g link by link and has the same epilogue, so either method leaves
// valid moments.
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
    double c[kMaxP + 1];             // difference form: h, zero above degree p
    double e[kMaxP + 1][kMaxP + 1];  // E_ab (both forms), zero above degree p
    double v[kMaxP + 1];             // V'
    double k_over_n;
    int group;                       // threads per row of the direct kernel
    int win_cap;                     // shared-memory window capacity (nodes); 0 = read the
                                     // community's states from global memory
    const TileDesc *tile_desc;
    const unsigned char *blob;
    const int32_t *comm_tile_begin;
    const int64_t *full_rowptr;
    const int32_t *full_col;
    const double *y_in;              // [n] stage state (permuted)
    double *y_out;                   // [n] next stage state
    const double *part_in;           // [tiles][P+1] sums of y_in^a
    double *part_out;                // [tiles][P+1] sums of y_out^a
    double *acc, *theta;             // RK4 accumulator, FP64 master
    const int32_t *perm;
    double *rhs_out;                 // kRhs: original order
    const double *alpha, *beta;      // rank-one link weights (permuted), or both null
    double c_next_dt, b_s, dt;
    int first_stage;
};

template <int P>
__device__ __forceinline__ double horner(const double *c, double x) {
    double s = c[P];
#pragma unroll
    for (int a = P - 1; a >= 0; --a) s = fma(s, x, c[a]);
    return s;
}

// e_a(y) = sum_b E_ab y^b, a = 0..P.
template <int P>
__device__ __forceinline__ void coefficients(const PolyParams &a, double y, double (&e)[P + 1]) {
#pragma unroll
    for (int al = 0; al <= P; ++al) e[al] = horner<P>(a.e[al], y);
}

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

// Sums over the tile of w y^a, a = 0..P (w = the node's beta, or 1; each thread
// contributes its node's value, nothing when it has no node), in a fixed
// order, to part_out[tile].
template <int P>
__device__ __forceinline__ void tile_power_sums(double *part_out, int tile, bool live, double y, double wnode,
                                                double (*red)[kMaxP + 1]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double pw[P + 1];
    double q = wnode;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
        pw[k] = live ? q : 0.0;
        q *= y;
    }
#pragma unroll
    for (int k = 0; k <= P; ++k)
        for (int o = 16; o > 0; o >>= 1) pw[k] += __shfl_xor_sync(0xffffffffu, pw[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k <= P; ++k) red[warp][k] = pw[k];
    __syncthreads();
    if (threadIdx.x <= P) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        part_out[(int64_t)tile * (P + 1) + threadIdx.x] = s;
    }
}

// The tile's sums of w y^a, a = 0..P (w = the node's beta, or 1), through shared memory: every thread
// stores its powers in scratch ([P+1][kThreads] doubles, free at this point),
// then warp a adds row a in a fixed order.  Fewer FP64 additions than a
// shuffle tree in every warp.
template <int P>
__device__ __forceinline__ void tile_power_sums_smem(double *part_out, int tile, bool live, double y,
                                                     double wnode, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();   // scratch was read before
    double q = wnode;
#pragma unroll
    for (int k = 0; k <= P; ++k) {
        scratch[k * kThreads + threadIdx.x] = live ? q : 0.0;
        q *= y;
    }
    __syncthreads();
    if (warp <= P) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < kThreads / 32; ++j) s += scratch[warp * kThreads + j * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) part_out[(int64_t)tile * (P + 1) + warp] = s;
    }
}

// Round u 2^sh to the nearest integer (ties away from zero) with integer
// operations only; the caller picks sh so that |u| 2^sh < 2^55.
__device__ __forceinline__ long long to_fixed(double u, int sh) {
    const long long bits = __double_as_longlong(u);
    const int e = (int)((bits >> 52) & 0x7ff);
    const long long mant = (bits & 0xfffffffffffffLL) | (e ? (1LL << 52) : 0LL);
    const int k = min((e ? e : 1) - 1075 + sh, 2);   // u 2^sh = mant 2^k
    long long m;
    if (k >= 0) m = mant << k;
    else if (k < -62) m = 0;
    else m = (mant + (1LL << (-k - 1))) >> (-k);
    return bits < 0 ? -m : m;
}

// Adds u^1..u^P to s[0..P-1].
template <int P>
__device__ __forceinline__ void add_powers(double (&s)[P], double u) {
    double q = u;
#pragma unroll
    for (int al = 0; al < P; ++al) {
        s[al] += q;
        if (al + 1 < P) q *= u;
    }
}

// WT: rank-one weighted links (eq. rank1system): every power sum carries the
// neighbour's beta_l (the moments become eq. rank1precompute's weighted
// sums, the degree a weighted degree) and the coupling is scaled by alpha_m
// (eq. rank1fast).  Window rows: powers 1..P (unweighted; the degree is an
// integer count) or 0..P times beta (weighted).
template <int MODE, int P, bool WT>
__global__ void __launch_bounds__(kThreads) poly_stage_kernel(const PolyParams a) {
    constexpr int NR = P + (WT ? 1 : 0);   // window rows / sparse sums per link
    constexpr int A0 = WT ? 0 : 1;         // power of row 0
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double W[kMaxP + 1];
    __shared__ double red[kWarps][kMaxP + 1];
    static_assert(NR * kMaxChunks >= (P + 1) * kThreads, "the tile sums reuse the chunk table");
    double *win = reinterpret_cast<double *>(smem_raw);        // [NR][win_cap] powers of the community's states
    double *sWm = win + (size_t)NR * a.win_cap;                 // [NR][kMaxChunks] missing-chunk power sums
    double *sWi = sWm + NR * kMaxChunks;                        // [NR][kTileMax] inter power sums per row
    int *smc = reinterpret_cast<int *>(sWi + NR * kTileMax);    // [kMaxChunks] missing links per chunk
    int *sic = smc + kMaxChunks;                                // [kTileMax] inter links per row
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool comm = d.comm >= 0;
    const int lam = comm ? (int)d.lam : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned char *b = a.blob + d.blob_off;
    const int cap = a.win_cap;
    const double *cy = a.y_in + d.lo;
    const double *cb = WT ? a.beta + d.lo : nullptr;
    long long *wfix = reinterpret_cast<long long *>(win);   // the window after conversion
    double unit[NR];                                         // 2^E_a
    // the terms of one link l: beta_l^[WT] x_l^a for the NR powers
    auto terms = [&](double u, double wl, double (&q)[NR]) {
        double v = WT ? wl : u;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            q[r] = v;
            if (r + 1 < NR) v *= u;
        }
    };
    // (0) window of powers and their largest magnitudes, moments (FP64 over
    // the community's tiles)
    if (cap) {
        // largest |term| as the integer order of the magnitude's bits
        unsigned long long mx[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) mx[r] = 0ull;
        for (int i = threadIdx.x; i < lam; i += kThreads) {
            double q[NR];
            terms(cy[i], WT ? cb[i] : 1.0, q);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                win[r * cap + i] = q[r];
                mx[r] = max(mx[r], (unsigned long long)__double_as_longlong(q[r]) & 0x7fffffffffffffffull);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            for (int o = 16; o > 0; o >>= 1) mx[r] = max(mx[r], __shfl_xor_sync(0xffffffffu, mx[r], o));
            if (lane == 0) red[warp][r] = __longlong_as_double((long long)mx[r]);
        }
    }
    if (comm && warp == 0) {
        const int u0 = a.comm_tile_begin[d.comm], u1 = a.comm_tile_begin[d.comm + 1];
#pragma unroll
        for (int k = 0; k <= P; ++k) {
            double s = 0.0;
            for (int u = u0 + lane; u < u1; u += 32) s += a.part_in[(int64_t)u * (P + 1) + k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) W[k] = s;
        }
    }
    __syncthreads();
    if (cap) {
        // E_a from the community's largest |term| (the same in every thread),
        // then each thread converts the entries it wrote
        int sh[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            unsigned long long m = 0ull;
            for (int w = 0; w < kWarps; ++w) m = max(m, (unsigned long long)__double_as_longlong(red[w][r]));
            const int em = (int)(m >> 52);
            const int ex = (em ? em : 1) - 1022;   // largest |term| < 2^ex
            sh[r] = min(55 - ex, 1000);            // |term| 2^sh < 2^55
            unit[r] = ldexp(1.0, -sh[r]);
        }
        for (int i = threadIdx.x; i < lam; i += kThreads)
#pragma unroll
            for (int r = 0; r < NR; ++r) wfix[r * cap + i] = to_fixed(win[r * cap + i], sh[r]);
        __syncthreads();
    }
    // (A) sparse power sums: warp per slice, lane per missing chunk and inter row
    const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
    const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
    const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
    const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);
    for (int s = warp; s < d.nsl; s += kWarps) {
        const uint4 sd = __ldg(sdesc + s);
        const uint32_t rows = __ldg(srows + s * 32 + lane);
        const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
        double ms[NR], is[NR];
        long long mfix[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            ms[r] = is[r] = 0.0;
            mfix[r] = 0;
        }
        int mc = 0, ic = 0;
        const uint4 *mv = mvec + sd.x + lane;
        for (uint32_t j = 0; j < sd.y; ++j) {
            const uint4 q = __ldg(mv + 32 * j);
            const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int l = (int)(h ? w4[e] >> 16 : w4[e] & 0xffffu);
                    if (l < lam) {
                        ++mc;
                        if (cap) {
#pragma unroll
                            for (int r = 0; r < NR; ++r) mfix[r] += wfix[r * cap + l];
                        } else {
                            double tq[NR];
                            terms(cy[l], WT ? cb[l] : 1.0, tq);
#pragma unroll
                            for (int r = 0; r < NR; ++r) ms[r] += tq[r];
                        }
                    }
                }
            }
        }
        const int4 *iv = ivec + sd.z + lane;
        for (uint32_t j = 0; j < sd.w; ++j) {
            const int4 q = __ldg(iv + 32 * j);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (l4[e] < a.n) {
                    ++ic;
                    double tq[NR];
                    terms(__ldg(a.y_in + l4[e]), WT ? __ldg(a.beta + l4[e]) : 1.0, tq);
#pragma unroll
                    for (int r = 0; r < NR; ++r) is[r] += tq[r];
                }
        }
        if (mrow != 0xffffu) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
                sWm[r * kMaxChunks + mrow] = cap ? (double)mfix[r] * unit[r] : ms[r];
            smc[mrow] = mc;
        }
        if (irow != 0xffffu) {
#pragma unroll
            for (int r = 0; r < NR; ++r) sWi[r * kTileMax + irow] = is[r];
            sic[irow] = ic;
        }
    }
    __syncthreads();
    // (B) thread per node: T_a = W_a - diagonal - missing + inter, then
    // alpha_m^[WT] sum_a T_a e_a(x)
    const bool live = threadIdx.x < d.count;
    double ynext = 0.0, wnode = 0.0;
    if (live) {
        const int r0 = threadIdx.x;
        const int64_t m = d.first + r0;
        const double x = a.y_in[m];
        wnode = WT ? a.beta[m] : 1.0;
        double T[P + 1];
        int deg = sic[r0];
#pragma unroll
        for (int r = 0; r < NR; ++r) T[r + A0] = sWi[r * kTileMax + r0];
        const uint32_t vt = __ldg(reinterpret_cast<const uint32_t *>(b + d.vtab_off) + r0);
        for (uint32_t c = vt & 0xffffu; c < (vt & 0xffffu) + (vt >> 16); ++c) {
            deg -= smc[c];
#pragma unroll
            for (int r = 0; r < NR; ++r) T[r + A0] -= sWm[r * kMaxChunks + c];
        }
        if (!WT) T[0] = (double)deg;
        if (comm) {
            double q = wnode;   // the diagonal term beta_m^[WT] x_m^a
#pragma unroll
            for (int al = 0; al <= P; ++al) {
                T[al] += W[al] - q;
                q *= x;
            }
        }
        double e[P + 1];
        coefficients<P>(a, x, e);
        double coup = 0.0;
#pragma unroll
        for (int al = 0; al <= P; ++al) coup = fma(T[al], e[al], coup);
        if (WT) coup *= a.alpha[m];
        const double k = -horner<kMaxP>(a.v, x) + a.k_over_n * coup;
        ynext = rk4_update<MODE>(a, m, k);
    }
    if (MODE == kRhs) return;
    tile_power_sums_smem<P>(a.part_out, t, live, ynext, wnode, sWm);
}

// Direct method, one CTA per tile: `group` threads per row evaluate the
// coupling link by link over the row's CSR neighbours (rows padded to 4-entry
// vectors with the sentinel n): h(x_l - x_m), or g(x_l, x_m) = sum_a e_a(x_m)
// x_l^a, times beta_l and finally alpha_m when the links are weighted; then
// the same update and power sums as the CIA.
template <int MODE, bool GEN, int P>
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
        const double y = a.y_in[m];
        double e[P + 1];
        if (GEN) coefficients<P>(a, y, e);
        double s = 0.0;
        for (int64_t v = a.full_rowptr[m] / 4 + gl; v < a.full_rowptr[m + 1] / 4; v += G) {
            const int4 q = __ldg(col4 + v);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (l4[k] < a.n) {
                    const double u = __ldg(a.y_in + l4[k]);
                    const double gl_ = GEN ? horner<P>(e, u) : horner<P>(a.c, u - y);
                    s += a.beta ? __ldg(a.beta + l4[k]) * gl_ : gl_;
                }
        }
        for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (gl == 0) sW[r] = s;
    }
    __syncthreads();
    const bool live = threadIdx.x < d.count;
    double ynext = 0.0, wnode = 0.0;
    if (live) {
        const int64_t m = d.first + threadIdx.x;
        const double x = a.y_in[m];
        const double coup = a.alpha ? a.alpha[m] * sW[threadIdx.x] : sW[threadIdx.x];
        const double k = -horner<kMaxP>(a.v, x) + a.k_over_n * coup;
        ynext = rk4_update<MODE>(a, m, k);
        wnode = a.beta ? a.beta[m] : 1.0;
    }
    if (MODE == kRhs) return;
    tile_power_sums<P>(a.part_out, t, live, ynext, wnode, red);
}

// State load: x (original order) -> master (optional) and stage state,
// with the tile sums of its powers.  One CTA per tile.
template <int P>
__global__ void __launch_bounds__(kThreads) poly_load_kernel(const PolyParams a, const double *x, double *master) {
    __shared__ double red[kWarps][kMaxP + 1];
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool live = threadIdx.x < d.count;
    double y = 0.0, wnode = 0.0;
    if (live) {
        const int64_t m = d.first + threadIdx.x;
        y = x[a.perm[m]];
        if (master) master[m] = y;
        a.y_out[m] = y;
        wnode = a.beta ? a.beta[m] : 1.0;
    }
    tile_power_sums<P>(a.part_out, t, live, y, wnode, red);
}

size_t window_cap(const cia_plan *pl) { return (size_t)((pl->max_comm + 1) & ~(int64_t)1); }

// Rows of the window and of the sparse sums: powers 1..P, or 0..P when weighted.
int rows(const cia_plan *pl) { return pl->poly_p + (pl->poly_weighted ? 1 : 0); }

size_t tables_bytes(int nr) { return (size_t)nr * (kMaxChunks + kTileMax) * 8 + (kMaxChunks + kTileMax) * 4; }

// The powers of the largest community's states fit the shared-memory window
// (the kernel's static shared memory is under 4 KB).
bool window_fits(const cia_plan *pl) {
    return window_cap(pl) * 8 * rows(pl) + tables_bytes(rows(pl)) + 4096 <= (size_t)pl->smem_optin;
}

size_t stage_smem(const cia_plan *pl) {
    return (pl->staging == 2 ? window_cap(pl) * 8 * rows(pl) : 0) + tables_bytes(rows(pl));
}

PolyParams base_params(const cia_plan *pl, int slot) {
    PolyParams a{};
    const auto &d = pl->d;
    constexpr int S = kMaxP + 1;
    a.n = pl->n;
    for (int k = 0; k < S; ++k) {
        a.c[k] = pl->poly_c[k];
        a.v[k] = pl->poly_dv[k];
    }
    // E_ab: G itself, or the regrouped binomial expansion of h
    for (int al = 0; al < S; ++al)
        for (int b = 0; b < S; ++b) {
            if (pl->poly_general) {
                a.e[al][b] = pl->poly_g[al * S + b];
            } else if (al + b < S) {
                double binom = 1.0;   // binom(al + b, al)
                for (int j = 1; j <= al; ++j) binom = binom * (double)(b + j) / (double)j;
                a.e[al][b] = pl->poly_c[al + b] * binom * ((b & 1) ? -1.0 : 1.0);
            }
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
    a.acc = static_cast<double *>(d.acc);
    a.theta = d.theta;
    a.perm = d.perm;
    a.alpha = pl->poly_weighted ? d.pl_alpha : nullptr;
    a.beta = pl->poly_weighted ? d.pl_beta : nullptr;
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

template <int MODE, int P>
cudaError_t launch_degree(const cia_plan *pl, int method, const PolyParams &a, cudaStream_t s) {
    constexpr int id = 3 * (P - 1) + MODE;   // stage kernels 0..23, direct kernels 24..47
    if (method == Method::DIRECT)
        return pl->poly_general ? launch<24 + 2 * id>(poly_direct_kernel<MODE, true, P>, pl, 0, a, s)
                                : launch<25 + 2 * id>(poly_direct_kernel<MODE, false, P>, pl, 0, a, s);
    return pl->poly_weighted ? launch<12 + id>(poly_stage_kernel<MODE, P, true>, pl, stage_smem(pl), a, s)
                             : launch<id>(poly_stage_kernel<MODE, P, false>, pl, stage_smem(pl), a, s);
}

template <int MODE>
cudaError_t launch_mode(const cia_plan *pl, int method, const PolyParams &a, cudaStream_t s) {
    switch (pl->poly_p) {
        case 1: return launch_degree<MODE, 1>(pl, method, a, s);
        case 2: return launch_degree<MODE, 2>(pl, method, a, s);
        case 3: return launch_degree<MODE, 3>(pl, method, a, s);
        default: return launch_degree<MODE, 4>(pl, method, a, s);
    }
}

}  // namespace

bool poly_window_fits(const cia_plan *pl) { return window_fits(pl); }

cudaError_t poly_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    // the load writes the state and its power sums into slot `slot`
    PolyParams a = base_params(pl, slot ^ 1);
    double *master = write_master ? pl->d.theta : nullptr;
    const unsigned grid = (unsigned)pl->n_tiles;
    switch (pl->poly_p) {
        case 1: poly_load_kernel<1><<<grid, kThreads, 0, s>>>(a, x, master); break;
        case 2: poly_load_kernel<2><<<grid, kThreads, 0, s>>>(a, x, master); break;
        case 3: poly_load_kernel<3><<<grid, kThreads, 0, s>>>(a, x, master); break;
        default: poly_load_kernel<4><<<grid, kThreads, 0, s>>>(a, x, master); break;
    }
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
