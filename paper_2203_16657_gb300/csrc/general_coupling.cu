// Device kernels of the general separable couplings with a potential, FP64:
//   x_m' = -V'(x_m) + (K/N) sum_l a_ml g(x_l, x_m),   V'(x) = sum_{j=0..4} v_j x^j,
// where g is a finite sum of products of features of its two arguments,
//   g(u, y) = sum_{k,j} E_kj phi_k(u) phi_j(y),   phi_0 = 1.
// Polynomial basis (App. A.3): phi_k(u) = u^k, k <= p (eq. PolyApprox; E = G
// for the general form, eq. PolyRHS; E_kj = c_{k+j} binom(k+j, k) (-1)^j for
// the difference form h(u - y), eq. PolyDifferenceRHSfast with its sum over
// a regrouped by the power of the moment; Desai-Zwanzig, App. A.5, is h = u).
// Fourier basis (eq. FourierRealExpansion): phi = (1, cos wu, sin wu, ...,
// cos pwu, sin pwu), w = pi / L, E holding C11, C12, C21, C22.
//
// Every link then contributes its neighbour's feature vector: sum_l a_ml
// g(x_l, x_m) = sum_k T_k(m) e_k(x_m) with T_k(m) = sum_l a_ml phi_k(x_l) and
// e_k(y) = sum_j E_kj phi_j(y).  The CIA splits T_k(m) as in steps E1 + E2:
// the community moment W_ck = sum_{l in c} phi_k(x_l) (eq. PolyMoments /
// eq. RealOP, without the 1/N), minus the diagonal phi_k(x_m) (a_mm = 0),
// minus the sums over the missing links, plus those over the inter-community
// links; T_0 is the degree.  Rank-one link weights alpha_m beta_l
// (eq. rank1system; polynomial basis) put beta_l into every sum (the moments
// of eq. rank1precompute) and alpha_m on the coupling (eq. rank1fast).
//
// FP64 additions are scarce on this GPU (a few per clock and SM), so the
// missing-link sums, the bulk of the work, are exact integer sums: the tile's
// window holds each feature of the community's states as a 64-bit fixed-point
// number, phi = M 2^E with |M| < 2^55 and E set by the community's largest
// |phi|, so that a chunk of at most 64 links sums without overflow.  The
// rounding to the grid 2^E (at most 2^-56 of the largest value) is below the
// rounding error of an FP64 sum of the same values.  Fourier features are
// computed once per node and stage (one sincos and the angle-addition
// recurrence) and stored; polynomial features are computed where needed.
//
// The window of a community of lambda nodes takes 8 lambda bytes per feature
// row, so one large community would set every CTA's shared memory.  The
// plan therefore sorts the tiles by community size; each stage launches one
// kernel per run of tiles that fit the same number of resident CTAs per SM
// (4, 3, 2, 1, with a window sized to the run's largest community; tiles of a
// community that fits no window read its features from global memory), and
// these launches run concurrently on forked streams.
//
// One CTA (256 threads) per tile: (0) the community's moments from
// the previous launch's tile sums and its features in shared memory, (A) the
// sparse feature sums over the tile's sliced-ELL blob, (B) one thread per
// node: T_k, the coupling, RK4 stage update, the next state's features and the
// tile's feature sums.  The direct method's kernel evaluates g link by link
// and has the same epilogue, so either method leaves valid moments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "cia_internal.h"

namespace cia {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxChunks = 512;
constexpr int kTileMax = 256;
constexpr int kMaxP = CIA_MAX_POLY;
constexpr int kMaxK = CIA_GC_MAX_FEATURES;   // features incl. phi_0

enum Mode { kRhs = 0, kStage = 1, kFinal = 2 };
enum Basis { kPoly = 0, kFourier = 1 };

struct GcParams {
    int64_t n;
    double c[kMaxP + 1];         // polynomial difference form: h (direct method)
    double e[kMaxK][kMaxK];      // E_kj
    double v[kMaxP + 1];         // V'
    double w;                    // Fourier basis: pi / L
    double k_over_n;
    int group;                   // threads per row of the direct kernel
    int win_cap;                 // shared-memory window capacity (nodes); 0 = read the
                                 // community's features from global memory
    int diff;                    // direct method: h(u - y) instead of the separable form
    const TileDesc *tile_desc;
    const int32_t *tile_list;    // the launch's tiles (window launches), or null: tile = CTA
    const unsigned char *blob;
    const int32_t *comm_tile_begin;
    const int64_t *full_rowptr;
    const int32_t *full_col;
    const double *y_in;          // [n] stage state (permuted)
    double *y_out;               // [n] next stage state
    const double *f_in;          // Fourier basis: [n][K-1] features of y_in
    double *f_out;               // [n][K-1] features of y_out
    const double *part_in;       // [tiles][K] feature sums of y_in
    double *part_out;            // [tiles][K] feature sums of y_out
    double *acc, *theta;         // RK4 accumulator, FP64 master
    const int32_t *perm;
    double *rhs_out;             // kRhs: original order
    const double *alpha, *beta;  // rank-one link weights (permuted), or both null
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

// phi_0..phi_{K-1} of u: powers, or (1, cos wu, sin wu, cos 2wu, ...) by one
// sincos and the angle-addition recurrence.
template <int B, int K>
__device__ __forceinline__ void features(const GcParams &a, double u, double (&f)[K]) {
    f[0] = 1.0;
    if (B == kPoly) {
#pragma unroll
        for (int k = 1; k < K; ++k) f[k] = f[k - 1] * u;
    } else {
        double s1, c1;
        sincos(a.w * u, &s1, &c1);
        if (K > 1) f[1] = c1;
        if (K > 2) f[2] = s1;
#pragma unroll
        for (int k = 3; k + 1 < K; k += 2) {
            f[k] = f[k - 2] * c1 - f[k - 1] * s1;       // cos((j+1)wu)
            f[k + 1] = f[k - 1] * c1 + f[k - 2] * s1;   // sin((j+1)wu)
        }
    }
}

// The stored features 1..K-1 of node l (Fourier basis) or computed from its
// state (polynomial basis), times beta_l when weighted.
template <int B, int K>
__device__ __forceinline__ void node_features(const GcParams &a, int64_t l, double (&f)[K]) {
    if (B == kPoly) {
        features<B, K>(a, __ldg(a.y_in + l), f);
    } else {
        f[0] = 1.0;
#pragma unroll
        for (int k = 1; k < K; ++k) f[k] = __ldg(a.f_in + l * (K - 1) + (k - 1));
    }
}

// e_k(y) = sum_j E_kj phi_j(y).
template <int K>
__device__ __forceinline__ void coefficients(const GcParams &a, const double (&ph)[K], double (&e)[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < K; ++j) s = fma(a.e[k][j], ph[j], s);
        e[k] = s;
    }
}

// RK4 stage update from the derivative k; returns the next stage state.
template <int MODE>
__device__ __forceinline__ double rk4_update(const GcParams &a, int64_t m, double k) {
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

// Features of the next state: stored (Fourier basis) and summed over the
// tile, weighted by the node's beta, in a fixed order through shared memory:
// every thread stores its values in scratch ([K][kThreads] doubles, free at
// this point), then warp k adds row k.
template <int B, int K>
__device__ __forceinline__ void next_features(const GcParams &a, int tile, int64_t m, bool live, double y,
                                              double wnode, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double f[K];
    features<B, K>(a, y, f);
    if (B == kFourier && live)
#pragma unroll
        for (int k = 1; k < K; ++k) a.f_out[m * (K - 1) + (k - 1)] = f[k];
    __syncthreads();   // scratch was read before
#pragma unroll
    for (int k = 0; k < K; ++k) scratch[k * kThreads + threadIdx.x] = live ? wnode * f[k] : 0.0;
    __syncthreads();
    for (int k = warp; k < K; k += kWarps) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < kThreads / 32; ++j) s += scratch[k * kThreads + j * 32 + lane];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) a.part_out[(int64_t)tile * K + k] = s;
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

// WT: rank-one weighted links; the rows of the window and of the sparse sums
// are the features 1..K-1 (unweighted; the degree is an integer count) or
// 0..K-1 times beta (weighted).
template <int MODE, int B, int K, bool WT>
__global__ void __launch_bounds__(kThreads) gc_stage_kernel(const GcParams a) {
    constexpr int NR = K - 1 + (WT ? 1 : 0);   // window rows / sparse sums per link
    constexpr int NRP = NR == 1 ? 1 : (NR + 1) & ~1;   // a node's window entries (even from 2 on)
    constexpr int A0 = WT ? 0 : 1;             // feature of row 0
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double W[kMaxK];
    __shared__ double red[kWarps][kMaxK];
    static_assert(NR * kMaxChunks >= K * kThreads, "the tile sums reuse the chunk table");
    double *win = reinterpret_cast<double *>(smem_raw);        // [win_cap][NRP] features of the community
    double *sWm = win + (size_t)NRP * a.win_cap;                // [NR][kMaxChunks] missing-chunk sums
    double *sWi = sWm + NR * kMaxChunks;                        // [NR][kTileMax] inter sums per row
    int *smc = reinterpret_cast<int *>(sWi + NR * kTileMax);    // [kMaxChunks] missing links per chunk
    int *sic = smc + kMaxChunks;                                // [kTileMax] inter links per row
    const int t = a.tile_list ? a.tile_list[blockIdx.x] : (int)blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool comm = d.comm >= 0;
    const int lam = comm ? (int)d.lam : 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned char *b = a.blob + d.blob_off;
    const int cap = a.win_cap;
    long long *wfix = reinterpret_cast<long long *>(win);   // the window after conversion
    // Node-major window: node l's entries are contiguous, so that a link reads
    // them with NRP / 2 16-byte loads.  With four entries the two halves of
    // node l swap places when bit 2 of l is set: load h of eight lanes then
    // touches 16-byte units 2l + (h ^ bit2(l)), distinct for distinct l mod 8
    // (the planner orders each quarter-warp's links by l mod 8).
    auto wslot = [](int l, int r) {
        if constexpr (NRP == 4) return 4 * l + ((((r >> 1) ^ (l >> 2)) & 1) << 1) + (r & 1);
        else return NRP * l + r;
    };
    double unit[NR];                                         // 2^E per row
    // the NR terms of node l: beta_l^[WT] phi_k(x_l), from its state (powers)
    // or its stored features
    const double *yv = a.y_in, *fv = a.f_in, *bv = a.beta;
    auto terms = [yv, fv, bv](int64_t l, double (&q)[NR]) {
        if constexpr (B == kPoly) {
            const double u = __ldg(yv + l);
            double v = WT ? __ldg(bv + l) : u;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                q[r] = v;
                if (r + 1 < NR) v *= u;
            }
        } else {
#pragma unroll
            for (int r = 0; r < NR; ++r) q[r] = __ldg(fv + l * (K - 1) + r);
        }
    };
    // (0) window of features and their largest magnitudes, moments (FP64 over
    // the community's tiles)
    if (cap) {
        // largest |term| as the integer order of the magnitude's bits
        unsigned long long mx[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) mx[r] = 0ull;
        for (int i = threadIdx.x; i < lam; i += kThreads) {
            double q[NR];
            terms(d.lo + i, q);
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                win[wslot(i, r)] = q[r];
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
        for (int k = 0; k < K; ++k) {
            double s = 0.0;
            for (int u = u0 + lane; u < u1; u += 32) s += a.part_in[(int64_t)u * K + k];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) W[k] = s;
        }
    }
    __syncthreads();
    if (cap) {
        // E from the community's largest |term| (the same in every thread),
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
            for (int r = 0; r < NRP; ++r) wfix[wslot(i, r)] = r < NR ? to_fixed(win[wslot(i, r)], sh[r < NR ? r : 0]) : 0;
        __syncthreads();
    }
    // (A) sparse feature sums: warp per slice, lane per missing chunk and inter row
    const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
    const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
    const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
    const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);
    for (int s = warp; s < d.nsl; s += kWarps) {
        const uint4 sd = __ldg(sdesc + s);
        const uint32_t rows = __ldg(srows + s * 32 + lane);
        const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
        double ms[NR], is[NR];
        long long mfix[NRP];   // entry NR of an odd NR sums the zero padding
#pragma unroll
        for (int r = 0; r < NR; ++r) ms[r] = is[r] = 0.0;
#pragma unroll
        for (int r = 0; r < NRP; ++r) mfix[r] = 0;
        int mc = 0, ic = 0;
        const uint4 *mv = mvec + sd.x + lane;
        // one loop per source of the community's features (the fixed-point
        // window or global memory), so that neither carries the other's work
        auto missing = [&](auto windowed) {
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
                            if constexpr (decltype(windowed)::value) {
                                if constexpr (NRP == 1) {
                                    mfix[0] += wfix[l];
                                } else {
                                    const longlong2 *wp = reinterpret_cast<const longlong2 *>(wfix) + (size_t)l * (NRP / 2);
#pragma unroll
                                    for (int hh = 0; hh < NRP / 2; ++hh) {
                                        const longlong2 v = wp[NRP == 4 ? (hh ^ ((l >> 2) & 1)) : hh];
                                        mfix[2 * hh] += v.x;
                                        mfix[2 * hh + 1] += v.y;
                                    }
                                }
                            } else {
                                double tq[NR];
                                terms(d.lo + l, tq);
#pragma unroll
                                for (int r = 0; r < NR; ++r) ms[r] += tq[r];
                            }
                        }
                    }
                }
            }
        };
        if (cap) missing(std::true_type{});
        else missing(std::false_type{});
        const int4 *iv = ivec + sd.z + lane;
        for (uint32_t j = 0; j < sd.w; ++j) {
            const int4 q = __ldg(iv + 32 * j);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (l4[e] < a.n) {
                    ++ic;
                    double tq[NR];
                    terms(l4[e], tq);
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
    // (B) thread per node: T_k = W_k - diagonal - missing + inter, then
    // alpha_m^[WT] sum_k T_k e_k(x)
    const bool live = threadIdx.x < d.count;
    const int64_t m = d.first + threadIdx.x;
    double ynext = 0.0, wnode = 0.0;
    if (live) {
        const int r0 = threadIdx.x;
        double T[K];
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
        double ph[K];
        node_features<B, K>(a, m, ph);
        wnode = WT ? a.beta[m] : 1.0;
        if (comm)
#pragma unroll
            for (int k = 0; k < K; ++k) T[k] += W[k] - (WT ? wnode * ph[k] : ph[k]);   // the diagonal term
        double e[K];
        coefficients<K>(a, ph, e);
        double coup = 0.0;
#pragma unroll
        for (int k = 0; k < K; ++k) coup = fma(T[k], e[k], coup);
        if (WT) coup *= a.alpha[m];
        const double x = a.y_in[m];
        const double kd = -horner<kMaxP>(a.v, x) + a.k_over_n * coup;
        ynext = rk4_update<MODE>(a, m, kd);
    }
    if (MODE == kRhs) return;
    next_features<B, K>(a, t, m, live, ynext, wnode, sWm);
}

// Direct method, one CTA per tile: `group` threads per row evaluate the
// coupling link by link over the row's CSR neighbours (rows padded to 4-entry
// vectors with the sentinel n): h(x_l - x_m) for the polynomial difference
// form (DIFF), else sum_k e_k(x_m) phi_k(x_l); times beta_l and finally
// alpha_m when the links are weighted; then the same update and feature sums
// as the CIA.
template <int MODE, int B, int K, bool DIFF>
__global__ void __launch_bounds__(kThreads) gc_direct_kernel(const GcParams a) {
    __shared__ double sW[K * kThreads];   // row sums, then the tile's feature sums
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const int G = a.group, gl = threadIdx.x % G, grp = threadIdx.x / G, ngrp = kThreads / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int4 *col4 = reinterpret_cast<const int4 *>(a.full_col);
    const double *yv = a.y_in, *bv = a.beta;
    const int64_t n = a.n;
    for (int r = grp; r < d.count; r += ngrp) {
        const int64_t m = d.first + r;
        const double y = yv[m];
        double e[K];
        if constexpr (!DIFF) {
            double ph[K];
            node_features<B, K>(a, m, ph);
            coefficients<K>(a, ph, e);
        }
        const int64_t v0 = a.full_rowptr[m] / 4 + gl, v1 = a.full_rowptr[m + 1] / 4;
        // one loop per weighting, so that the unweighted one carries no weight loads
        auto row_sum = [&](auto weighted) {
            double s = 0.0;
            for (int64_t v = v0; v < v1; v += G) {
                const int4 q = __ldg(col4 + v);
                const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (l4[k] < n) {
                        double gv;
                        if constexpr (DIFF) {
                            gv = horner<K - 1>(a.c, __ldg(yv + l4[k]) - y);
                        } else if constexpr (B == kPoly) {
                            gv = horner<K - 1>(e, __ldg(yv + l4[k]));   // sum_k e_k u^k
                        } else {
                            double f[K];
                            node_features<B, K>(a, l4[k], f);
                            gv = 0.0;
#pragma unroll
                            for (int j = 0; j < K; ++j) gv = fma(e[j], f[j], gv);
                        }
                        if constexpr (decltype(weighted)::value) gv *= __ldg(bv + l4[k]);
                        s += gv;
                    }
            }
            return s;
        };
        double s = bv ? row_sum(std::true_type{}) : row_sum(std::false_type{});
        for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (gl == 0) sW[r] = s;
    }
    __syncthreads();
    const bool live = threadIdx.x < d.count;
    const int64_t m = d.first + threadIdx.x;
    double ynext = 0.0, wnode = 0.0;
    if (live) {
        const double x = yv[m];
        const double coup = a.alpha ? a.alpha[m] * sW[threadIdx.x] : sW[threadIdx.x];
        const double kd = -horner<kMaxP>(a.v, x) + a.k_over_n * coup;
        ynext = rk4_update<MODE>(a, m, kd);
        wnode = bv ? bv[m] : 1.0;
    }
    if (MODE == kRhs) return;
    next_features<B, K>(a, t, m, live, ynext, wnode, sW);
}

// State load: x (original order) -> master (optional) and stage state,
// its features and their tile sums.  One CTA per tile.
template <int B, int K>
__global__ void __launch_bounds__(kThreads) gc_load_kernel(const GcParams a, const double *x, double *master) {
    __shared__ double scratch[K * kThreads];
    const int t = blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const bool live = threadIdx.x < d.count;
    const int64_t m = d.first + threadIdx.x;
    double y = 0.0, wnode = 0.0;
    if (live) {
        y = x[a.perm[m]];
        if (master) master[m] = y;
        a.y_out[m] = y;
        wnode = a.beta ? a.beta[m] : 1.0;
    }
    next_features<B, K>(a, t, m, live, y, wnode, scratch);
}

// Rows of the window and of the sparse sums: features 1..K-1, or 0..K-1 when weighted.
int rows(const cia_plan *pl) { return pl->gc_k - 1 + (pl->gc_weighted ? 1 : 0); }

// Window entries per node (the node-major window pads an odd row count from 3 on).
int window_entries(const cia_plan *pl) { return rows(pl) == 1 ? 1 : (rows(pl) + 1) & ~1; }

size_t tables_bytes(int nr) { return (size_t)nr * (kMaxChunks + kTileMax) * 8 + (kMaxChunks + kTileMax) * 4; }

constexpr size_t kStaticReserve = 4096;   // the stage kernel's static shared memory (under 1 KB) and margin

// The largest window (nodes, even) with which `per_sm` CTAs of the stage
// kernel fit one SM; 0 if not even the tables do.
int64_t window_cap_for(const cia_plan *pl, int per_sm) {
    const size_t sm = pl->smem_per_sm > 0 ? (size_t)pl->smem_per_sm : (size_t)pl->smem_optin;
    size_t per_cta = sm / (size_t)per_sm;
    per_cta = per_cta > 1024 ? per_cta - 1024 : 0;   // the runtime reserves 1 KB per CTA
    per_cta = std::min(per_cta, (size_t)pl->smem_optin);
    const size_t fixed = tables_bytes(rows(pl)) + kStaticReserve;
    if (per_cta <= fixed) return 0;
    return (int64_t)((per_cta - fixed) / (8 * (size_t)window_entries(pl))) & ~(int64_t)1;
}

// A window launch over a run of tiles: their community windows need at most
// `cap` nodes (0: the run reads features from global memory).
struct Run {
    int64_t begin, end, cap;
};

// Runs of the size-sorted tile list: each tile goes to the launch with the
// most resident CTAs per SM (4, 3, 2, 1) whose window holds its community;
// tiles of communities no window holds read from global memory.
std::vector<Run> window_runs(const cia_plan *pl) {
    std::vector<Run> runs;
    const auto &lam = pl->gc_tile_lam;
    const int64_t T = (int64_t)lam.size();
    int64_t caps[5];
    for (int k = 1; k <= 4; ++k) caps[k] = window_cap_for(pl, k);
    auto level = [&](int64_t l) {
        for (int k = 4; k >= 1; --k)
            if (l <= caps[k]) return k;
        return 0;
    };
    for (int64_t i = 0; i < T;) {
        const int k = level(lam[i]);
        int64_t j = i + 1;
        while (j < T && level(lam[j]) == k) ++j;
        runs.push_back({i, j, k == 0 ? 0 : (lam[i] + 1) & ~(int64_t)1});
        i = j;
    }
    return runs;
}

size_t stage_smem(const cia_plan *pl, int64_t cap) {
    return (size_t)cap * 8 * window_entries(pl) + tables_bytes(rows(pl));
}

GcParams base_params(const cia_plan *pl, int slot) {
    GcParams a{};
    const auto &d = pl->d;
    a.n = pl->n;
    for (int k = 0; k <= kMaxP; ++k) {
        a.c[k] = pl->poly_c[k];
        a.v[k] = pl->poly_dv[k];
    }
    for (int k = 0; k < kMaxK; ++k)
        for (int j = 0; j < kMaxK; ++j) a.e[k][j] = pl->gc_e[k * kMaxK + j];
    a.w = pl->gc_w;
    a.diff = pl->gc_basis == kPoly && !pl->poly_general;
    a.k_over_n = pl->K / (double)pl->n;
    a.group = pl->group_size_direct;
    a.win_cap = 0;
    a.tile_desc = d.tile_desc;
    a.tile_list = nullptr;
    a.blob = d.blob;
    a.comm_tile_begin = d.comm_tile_begin;
    a.full_rowptr = d.full_rowptr;
    a.full_col = d.full_col;
    a.y_in = d.gc_y[slot];
    a.y_out = d.gc_y[slot ^ 1];
    a.f_in = d.gc_f[slot];
    a.f_out = d.gc_f[slot ^ 1];
    a.part_in = d.gc_part[slot];
    a.part_out = d.gc_part[slot ^ 1];
    a.acc = static_cast<double *>(d.acc);
    a.theta = d.theta;
    a.perm = d.perm;
    a.alpha = pl->gc_weighted ? d.gc_alpha : nullptr;
    a.beta = pl->gc_weighted ? d.gc_beta : nullptr;
    return a;
}

// One launch of `kernel`, one tile per CTA.
cudaError_t launch(void (*kernel)(GcParams), const cia_plan *pl, size_t smem, const GcParams &a, cudaStream_t s) {
    cudaError_t e = ensure_dynamic_smem((const void *)kernel, pl->device, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<GcParams *>(&a)};
    return cudaLaunchKernel((const void *)kernel, dim3((unsigned)pl->n_tiles), dim3(kThreads), args, smem, s);
}

// The CIA stage kernel: one launch over all tiles with plain loads (staging
// 1), or one launch per run of the size-sorted tiles, each with a window for
// its largest community (staging 2).  The runs' tiles are disjoint, so their
// launches run concurrently: the first on the caller's stream, the others on
// side streams that fork from it and join it again, so that CTAs of every
// run share the SMs instead of each run's last wave idling them.
cudaError_t launch_cia(void (*kernel)(GcParams), const cia_plan *pl, const GcParams &a0, cudaStream_t s) {
    if (pl->staging != 2) return launch(kernel, pl, stage_smem(pl, 0), a0, s);
    const std::vector<Run> runs = window_runs(pl);
    if (runs.size() > 5) return cudaErrorInvalidValue;   // at most one run per level (0, 1, 2, 3, 4)
    cudaError_t e = cudaSuccess;
    if (runs.size() > 1 && (e = cudaEventRecord(pl->gc_fork, s)) != cudaSuccess) return e;
    for (size_t i = 0; i < runs.size(); ++i) {
        const Run &run = runs[i];
        cudaStream_t rs = i == 0 ? s : pl->gc_side[i - 1];
        if (i > 0 && (e = cudaStreamWaitEvent(rs, pl->gc_fork, 0)) != cudaSuccess) return e;
        GcParams a = a0;
        a.win_cap = (int)run.cap;
        a.tile_list = pl->d.gc_tiles + run.begin;
        const size_t smem = stage_smem(pl, run.cap);
        if ((e = ensure_dynamic_smem((const void *)kernel, pl->device, smem)) != cudaSuccess) return e;
        void *args[] = {&a};
        e = cudaLaunchKernel((const void *)kernel, dim3((unsigned)(run.end - run.begin)), dim3(kThreads), args, smem, rs);
        if (e != cudaSuccess) return e;
        if (i > 0) {
            if ((e = cudaEventRecord(pl->gc_join[i - 1], rs)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, pl->gc_join[i - 1], 0)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

template <int MODE, int B, int K>
cudaError_t launch_shape(const cia_plan *pl, int method, const GcParams &a, cudaStream_t s) {
    if (method == Method::DIRECT) {
        if constexpr (B == kPoly)
            if (a.diff) return launch(gc_direct_kernel<MODE, B, K, true>, pl, 0, a, s);
        return launch(gc_direct_kernel<MODE, B, K, false>, pl, 0, a, s);
    }
    if constexpr (B == kPoly)
        if (pl->gc_weighted) return launch_cia(gc_stage_kernel<MODE, B, K, true>, pl, a, s);
    return launch_cia(gc_stage_kernel<MODE, B, K, false>, pl, a, s);
}

template <int MODE>
cudaError_t launch_mode(const cia_plan *pl, int method, const GcParams &a, cudaStream_t s) {
    if (pl->gc_basis == kFourier) {
        switch (pl->gc_k) {
            case 3: return launch_shape<MODE, kFourier, 3>(pl, method, a, s);
            case 5: return launch_shape<MODE, kFourier, 5>(pl, method, a, s);
            case 7: return launch_shape<MODE, kFourier, 7>(pl, method, a, s);
            default: return launch_shape<MODE, kFourier, 9>(pl, method, a, s);
        }
    }
    switch (pl->gc_k) {
        case 2: return launch_shape<MODE, kPoly, 2>(pl, method, a, s);
        case 3: return launch_shape<MODE, kPoly, 3>(pl, method, a, s);
        case 4: return launch_shape<MODE, kPoly, 4>(pl, method, a, s);
        default: return launch_shape<MODE, kPoly, 5>(pl, method, a, s);
    }
}

template <int B, int K>
void launch_load(const cia_plan *pl, const GcParams &a, const double *x, double *master, cudaStream_t s) {
    gc_load_kernel<B, K><<<(unsigned)pl->n_tiles, kThreads, 0, s>>>(a, x, master);
}

}  // namespace


cudaError_t gc_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    // the load writes the state, its features and their sums into slot `slot`
    GcParams a = base_params(pl, slot ^ 1);
    double *master = write_master ? pl->d.theta : nullptr;
    if (pl->gc_basis == kFourier) {
        switch (pl->gc_k) {
            case 3: launch_load<kFourier, 3>(pl, a, x, master, s); break;
            case 5: launch_load<kFourier, 5>(pl, a, x, master, s); break;
            case 7: launch_load<kFourier, 7>(pl, a, x, master, s); break;
            default: launch_load<kFourier, 9>(pl, a, x, master, s); break;
        }
    } else {
        switch (pl->gc_k) {
            case 2: launch_load<kPoly, 2>(pl, a, x, master, s); break;
            case 3: launch_load<kPoly, 3>(pl, a, x, master, s); break;
            case 4: launch_load<kPoly, 4>(pl, a, x, master, s); break;
            default: launch_load<kPoly, 5>(pl, a, x, master, s); break;
        }
    }
    return cudaGetLastError();
}

cudaError_t gc_launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s) {
    GcParams a = base_params(pl, slot);
    a.rhs_out = dxdt;
    return launch_mode<kRhs>(pl, method, a, s);
}

cudaError_t gc_launch_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s) {
    static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    static const double c_next[4] = {0.5, 0.5, 1.0, 0.0};
    GcParams a = base_params(pl, slot);
    a.b_s = b[stage - 1];
    a.c_next_dt = c_next[stage - 1] * dt;
    a.dt = dt;
    a.first_stage = stage == 1;
    return stage == 4 ? launch_mode<kFinal>(pl, method, a, s) : launch_mode<kStage>(pl, method, a, s);
}

}  // namespace cia
