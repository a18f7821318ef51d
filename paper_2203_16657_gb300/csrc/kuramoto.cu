// Device kernels of the Kuramoto CIA hot path (sm_103a).
//
// Model (App. A.4): theta_m' = omega_m + (K/N) sum_l a_ml h(theta_l - theta_m),
//   h(x) = sum_{k=1..p} d_sin_k sin(kx) + d_cos_k cos(kx).
// With phasors u_{l,k} = e^{i k theta_l} the pair sum separates (Sec. 3.2):
//   sum_l a_ml h(theta_l - theta_m)
//     = sum_k d_sin_k Im(W_mk conj(u_mk)) + d_cos_k Re(W_mk conj(u_mk)),
//   W_mk = sum_l a_ml u_lk.
// CIA (steps E1 + E2): for m in community c,
//   W_mk = Z_ck - u_mk - sum_{l in miss(m)} u_lk + sum_{l in inter(m)} u_lk,
// where Z_ck = sum_{l in c} u_lk is the community observable
// (eq. PrecomputeQuantities up to the 1/N factor), u_mk removes the diagonal
// of the block (a_mm = 0), miss(m) are the -1 entries of S and inter(m) the +1
// entries.  The direct method sums W_mk over all CSR neighbours.
//
// One launch per RK4 stage.  A CTA owns a tile of consecutive nodes of one
// community: it (1) reduces the community's tile partial sums into Z_c,
// (2) stages the community's phasors in shared memory so that the missing-link
// gathers are shared-memory reads, (3) evaluates the coupling C_m of each node
// of the tile with `group` threads per row, (4) applies the RK4 stage update,
// computes the phasors of the next stage state and (5) writes its tile's
// partial sums of those phasors, which the next launch reduces into Z.
#include <cuda_runtime.h>

#include <cstdint>

#include "cia_internal.h"
#include "sync.cuh"

namespace cia {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
#ifndef CIA_WINDOW_VECTORS_P2
#define CIA_WINDOW_VECTORS_P2 1    // the same for two harmonics (higher-order model)
#endif
#ifndef CIA_WINDOW_INTER_VECTORS
#define CIA_WINDOW_INTER_VECTORS 2 // inter-link index vectors of a slice whose gathers fly together (<= 4)
#endif
#ifndef CIA_WINDOW_LATE_INPUTS
#define CIA_WINDOW_LATE_INPUTS 1   // window kernel: load Phase B's node inputs after Phase A
#endif
#ifndef CIA_WINDOW_MIN_BLOCKS
#define CIA_WINDOW_MIN_BLOCKS 4    // resident CTAs per SM the window kernel's registers are sized for
#endif
#ifndef CIA_WINDOW_DYNAMIC
#define CIA_WINDOW_DYNAMIC 1       // warps take the window kernel's slices from a shared counter
#endif
#ifndef CIA_WINDOW_VECTORS
#define CIA_WINDOW_VECTORS 2       // missing-index vectors of a chunk loaded before any is used (<= 8)
#endif
constexpr int kMaxChunks = 512;    // missing-list chunks per tile (partial sums in shared memory)

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ float2 mk2(float a, float b) { return make_float2(a, b); }
// Component-wise sum of two complex numbers: one packed FP32 add (two
// IEEE round-to-nearest additions in one instruction) or two FP64 adds.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(*reinterpret_cast<uint64_t *>(&a)), "l"(*reinterpret_cast<uint64_t *>(&b)));
    return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 mk2(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ void sincos_t(float y, float *s, float *c) { sincosf(y, s, c); }
__device__ __forceinline__ void sincos_t(double y, double *s, double *c) { sincos(y, s, c); }

// Representative of y in R / 2 pi Z within [-pi, pi] (FP64).
__device__ __forceinline__ double wrap_pi(double y) {
    const double two_pi = 6.283185307179586476925286766559;
    const double inv_two_pi = 0.15915494309189533576888376337251;
    return y - two_pi * rint(y * inv_two_pi);
}

// Phasors e^{i k y}, k = 1..P, by repeated multiplication of e^{i y}.
template <typename T, int P>
__device__ __forceinline__ void phasors(T y, typename Vec2<T>::type (&u)[P]) {
    T s, c;
    sincos_t(y, &s, &c);
    u[0] = mk2(c, s);
#pragma unroll
    for (int k = 1; k < P; ++k)
        u[k] = mk2(u[k - 1].x * c - u[k - 1].y * s, u[k - 1].x * s + u[k - 1].y * c);
}

// Triadic term of the higher-order model (App. A.7, lambda = (1, 1, -2)) on
// the complete community hyperedges, from the community moments: with
// w1 = Z_1 - u_1 and w2 = Z_2 - u_2 (the node itself removed), the ordered
// pairs j != k of the other members sum to w1^2 - w2, so the term is
// Im((w1^2 - w2) conj(u_2)).
template <typename T>
__device__ __forceinline__ T triadic_from_moments(T z1r, T z1i, T z2r, T z2i, T u1r, T u1i, T u2r, T u2i) {
    const T w1r = z1r - u1r, w1i = z1i - u1i;
    const T qr = w1r * w1r - w1i * w1i - (z2r - u2r);
    const T qi = T(2) * w1r * w1i - (z2i - u2i);
    return qi * u2r - qr * u2i;
}


enum Mode { kRhs = 0, kStage = 1, kFinal = 2 };

// Bytes of the per-run observable array, rounded up to 128 so that the
// shared-memory regions after it stay aligned for bulk copies.
__host__ __device__ constexpr size_t zrun_bytes(int64_t runs, int p, size_t complex_bytes) {
    return ((size_t)runs * (size_t)p * complex_bytes + 127) & ~(size_t)127;
}

// Shared-memory phasor entries per harmonic for TMA staging: lambda_max, the
// guard and kPadSlots zero entries after it, and up to one entry before it
// from rounding the window to 16 bytes.
int64_t tma_ph_region(const cia_plan *pl) { return (pl->max_comm + kPadSlots + 3) & ~(int64_t)1; }

template <typename T>
struct StageParams {
    using C = typename Vec2<T>::type;
    int64_t n;
    int64_t ph_stride;         // phasor entries per harmonic (>= n + 1; slot n is a zero phasor)
    int group;                 // threads per row of the direct method: 4, 8, 16 or 32
    int tile_nodes;
    T d_sin[CIA_MAX_HARMONICS], d_cos[CIA_MAX_HARMONICS];
    T k_over_n;                // K / N
    const T *tile_kn;          // ensembles: K / N_i per tile (NULL: k_over_n everywhere)
    T k2_over_n2;              // K2 / N^2 (higher-order model; 0 otherwise)
    const T *tri;              // direct method, higher-order model: triadic term per node
    const int64_t *off;
    const int32_t *tile_comm, *tile_first, *tile_count, *comm_tile_begin;
    // CIA: sliced-ELL sparse remainder, one blob per tile
    const TileDesc *tile_desc;
    const int32_t *tile_order;  // launch order of the per-tile kernels (NULL: tile = block)
    const unsigned char *blob;
    // direct: padded full CSR
    const int64_t *sp_rowptr;
    const int32_t *sp_col;
    const C *ph_in;            // [P][ph_stride] phasors of the stage state
    C *ph_out;                 // [P][ph_stride] phasors of the next stage state
    const double *part_in;     // [tiles][P] complex tile sums of ph_in
    double *part_out;          // [tiles][P] complex tile sums of ph_out
    const double *z_in;        // ring kernel: [M][P] community observables of ph_in
    double *z_out;             // ring kernel: [M][P] community observables of ph_out
    int *comm_done;            // ring kernel: [M] tiles finished per community (reset by the last)
    // kRhs
    const T *omega;
    const int32_t *perm;
    double *rhs_out;
    // kStage / kFinal
    T *acc;                    // sum_s b_s C_s
    double *theta;             // FP64 master
    const T *wdt_next;         // wrap(c_{s+1} dt omega)
    const double *wdt64;       // wrap(dt omega) (kFinal)
    T c_next_dt;               // c_{s+1} dt
    T b_s;                     // RK4 weight of this stage
    double dt;
    int first_stage;
    // TMA staging
    int64_t n_tiles;           // tiles of the plan (persistent kernels)
    int tile_buf;              // persistent per-tile kernel: bytes of its window + blob buffer
    int ph_region;             // shared-memory phasor entries per harmonic
    int idx_cap;               // shared-memory index buffer bytes
    int *err_flag;             // set when a bounded wait gives up
    int stages;                // ring buffers of the pipelined kernel
    int max_cta_tiles;         // most tiles of one persistent CTA
    int max_cta_runs;          // most community runs of one persistent CTA
    const int32_t *cta_tile_begin;
    const int32_t *cta_runs;   // community runs in each CTA's tile range
};

// Sum of per-thread values over the block, returned to thread 0..2P-1 as
// doubles: each warp reduces by a shuffle tree, then thread j adds the warps.
template <typename T, int P>
__device__ __forceinline__ void block_tile_sum(T (&re)[P], T (&im)[P], double (*red)[2 * P],
                                               double *dst) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re[k] += __shfl_xor_sync(0xffffffffu, re[k], o);
            im[k] += __shfl_xor_sync(0xffffffffu, im[k], o);
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            red[warp][2 * k] = (double)re[k];
            red[warp][2 * k + 1] = (double)im[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * P) {
        double s = 0.0;
        for (int w = 0; w < kWarps; ++w) s += red[w][threadIdx.x];
        dst[threadIdx.x] = s;
    }
}

// Phase B, one thread per node of the tile: coupling from the sparse sums
// sW (plus the dense term Z - u_m for community nodes), RK4 stage update,
// phasors of the next stage state and the tile's partial sums of them.
// own(k, m) returns u_{m,k}.
template <typename T, int P, int MODE, typename Own>
__device__ __forceinline__ void finalize_tile(const StageParams<T> &a, int t, int first, int count,
                                              bool dense, const typename Vec2<T>::type *zc,
                                              const typename Vec2<T>::type *sW, double (*red)[2 * P],
                                              Own own) {
    using C = typename Vec2<T>::type;
    const int64_t stride = a.ph_stride;
    T sre[P], sim[P];
#pragma unroll
    for (int k = 0; k < P; ++k) sre[k] = sim[k] = T(0);
    for (int r = threadIdx.x; r < count; r += kThreads) {
        const int64_t m = first + r;
        T coup = T(0);
        C uk[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const C u = own(k, m);
            uk[k] = u;
            const C wv = sW[k * a.tile_nodes + r];
            T zr = wv.x, zi = wv.y;
            if (dense) {
                // (E1.2) dense term: the whole block minus its diagonal (a_mm = 0)
                zr += zc[k].x - u.x;
                zi += zc[k].y - u.y;
            }
            // W conj(u_m): real part -> cosine harmonics, imaginary part -> sine
            const T re = zr * u.x + zi * u.y;
            const T im = zi * u.x - zr * u.y;
            coup += a.d_sin[k] * im + a.d_cos[k] * re;
        }
        coup *= a.tile_kn ? a.tile_kn[t] : a.k_over_n;
        if (P >= 2 && dense && a.k2_over_n2 != T(0))
            coup += a.k2_over_n2 * triadic_from_moments<T>(zc[0].x, zc[0].y, zc[P >= 2 ? 1 : 0].x, zc[P >= 2 ? 1 : 0].y,
                                                           uk[0].x, uk[0].y, uk[P >= 2 ? 1 : 0].x, uk[P >= 2 ? 1 : 0].y);
        if (a.tri) coup += a.tri[m];
        if (MODE == kRhs) {
            a.rhs_out[a.perm[m]] = (double)a.omega[m] + (double)coup;
        } else {
            const T accv = (a.first_stage ? T(0) : a.acc[m]) + a.b_s * coup;
            T y;
            if (MODE == kStage) {
                a.acc[m] = accv;
                y = (T)a.theta[m] + a.wdt_next[m] + a.c_next_dt * coup;
            } else {
                // FP64 time accumulation: theta += dt omega + dt sum_s b_s C_s
                const double th = wrap_pi(a.theta[m] + a.wdt64[m] + a.dt * (double)accv);
                a.theta[m] = th;
                y = (T)th;
            }
            C u[P];
            phasors<T, P>(y, u);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                a.ph_out[k * stride + m] = u[k];
                sre[k] += u[k].x;
                sim[k] += u[k].y;
            }
        }
    }
    if (MODE == kRhs) return;
    block_tile_sum<T, P>(sre, sim, red, a.part_out + (size_t)t * P * 2);
}

// (E1.1) community observable Z_ck = sum over the community's tiles of their
// partial sums, by warp 0: lane j adds tiles j, j + 32, ... in FP64, then a
// fixed shuffle tree combines the lanes (deterministic order).
template <typename T, int P>
__device__ __forceinline__ void community_observable(const StageParams<T> &a, int comm,
                                                     typename Vec2<T>::type *zc) {
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    const int u0 = a.comm_tile_begin[comm], u1 = a.comm_tile_begin[comm + 1];
    double re[P], im[P];
#pragma unroll
    for (int k = 0; k < P; ++k) re[k] = im[k] = 0.0;
    for (int u = u0 + lane; u < u1; u += 32) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(a.part_in) + (int64_t)u * P + k);
            re[k] += v.x;
            im[k] += v.y;
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re[k] += __shfl_xor_sync(0xffffffffu, re[k], o);
            im[k] += __shfl_xor_sync(0xffffffffu, im[k], o);
        }
        if (lane == 0) zc[k] = mk2((T)re[k], (T)im[k]);
    }
}

// CIA stage with plain loads, one CTA per tile (fallback when the pipelined
// kernel's shared-memory ring does not fit).  Phase A: one warp per slice,
// one lane per row, no cross-lane reduction -- first the missing links (-1
// entries of S, gathered from the community's phasors), then the
// inter-community links (+1 entries).  Phase B: one thread per node.
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(kThreads) cia_stage_kernel(const StageParams<T> a) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ C zc[P];
    __shared__ double red[kWarps][2 * P];

    const int t = a.tile_order ? a.tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const int64_t stride = a.ph_stride;
    const bool dense = d.comm >= 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lam = (int)d.lam;
    if (dense) community_observable<T, P>(a, d.comm, zc);
    C *sWm = reinterpret_cast<C *>(smem_raw);           // [P][kMaxChunks] chunk sums
    C *sWi = sWm + P * kMaxChunks;                      // [P][tile_nodes] inter sums
    const C *cph = a.ph_in + d.lo;
    const unsigned char *b = a.blob + d.blob_off;
    const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
    const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
    const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
    const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);

    for (int s = warp; s < d.nsl; s += kWarps) {
        const uint4 sd = __ldg(sdesc + s);
        const uint32_t rows = __ldg(srows + s * 32 + lane);
        const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
        T mre[P], mim[P], ire[P], iim[P];
#pragma unroll
        for (int k = 0; k < P; ++k) mre[k] = mim[k] = ire[k] = iim[k] = T(0);
        const uint4 *mv = mvec + sd.x + lane;
#pragma unroll 2
        for (uint32_t j = 0; j < sd.y; ++j) {
            const uint4 q = __ldg(mv + 32 * j);
            const unsigned w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int l0 = (int)(w4[h] & 0xffffu), l1 = (int)(w4[h] >> 16);
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const C v0 = l0 < lam ? __ldg(cph + k * stride + l0) : mk2(T(0), T(0));
                    const C v1 = l1 < lam ? __ldg(cph + k * stride + l1) : mk2(T(0), T(0));
                    mre[k] -= v0.x + v1.x;
                    mim[k] -= v0.y + v1.y;
                }
            }
        }
        const int4 *iv = ivec + sd.z + lane;
#pragma unroll 2
        for (uint32_t j = 0; j < sd.w; ++j) {
            const int4 q = __ldg(iv + 32 * j);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const C u = __ldg(a.ph_in + k * stride + l4[h]);
                    ire[k] += u.x;
                    iim[k] += u.y;
                }
            }
        }
        if (mrow != 0xffffu) {
#pragma unroll
            for (int k = 0; k < P; ++k) sWm[k * kMaxChunks + mrow] = mk2(mre[k], mim[k]);
        }
        if (irow != 0xffffu) {
#pragma unroll
            for (int k = 0; k < P; ++k) sWi[k * a.tile_nodes + irow] = mk2(ire[k], iim[k]);
        }
    }
    __syncthreads();
    // per row: its chunk sums in chunk order plus its inter sum, then Phase B
    const uint32_t *vtab = reinterpret_cast<const uint32_t *>(b + d.vtab_off);
    for (int r = threadIdx.x; r < d.count; r += kThreads) {
        const uint32_t vt = __ldg(vtab + r);
        const int c0 = (int)(vt & 0xffffu), nc = (int)(vt >> 16);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            C w = sWi[k * a.tile_nodes + r];
            for (int c = c0; c < c0 + nc; ++c) {
                const C v = sWm[k * kMaxChunks + c];
                w.x += v.x;
                w.y += v.y;
            }
            sWi[k * a.tile_nodes + r] = w;
        }
    }
    __syncthreads();
    finalize_tile<T, P, MODE>(a, t, d.first, d.count, dense, zc, sWi, red,
                              [&](int k, int64_t m) { return __ldg(a.ph_in + k * stride + m); });
}

// CIA stage with the community window in shared memory, one CTA per tile.
// Thread 0 copies the phasors of the tile's community (lo - shift ..
// lo + lambda, rounded to 16 bytes) into shared memory with one bulk (TMA)
// copy per harmonic; meanwhile warp 0 reduces the community observable and
// every thread loads its node's inputs.  The entry after the community is set
// to zero, so the padding index lambda of the missing lists reads a zero
// phasor without a test.  Phase A (warp per slice, lane per row) then reads
// the missing links from shared memory and the inter-community links from
// global memory; Phase B is one thread per node.  Many CTAs share an SM, so
// the hardware interleaves tiles at different phases.
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(kThreads, CIA_WINDOW_MIN_BLOCKS) cia_window_kernel(const StageParams<T> a) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ C zc[P];
    __shared__ double red[kWarps][2 * P];
    __shared__ uint64_t wbar;
    __shared__ int s_next;            // next slice to take (dynamic assignment)

    const int t = a.tile_order ? a.tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileDesc d = a.tile_desc[t];
    const int64_t stride = a.ph_stride;
    const bool dense = d.comm >= 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // bring the tile's index blob into L2 while the window, the observable
    // and the node inputs are fetched: Phase A then reads it at L2 latency
    if (threadIdx.x == 32) bulk_prefetch_l2(a.blob + d.blob_off, d.blob_bytes);
    C *win = reinterpret_cast<C *>(smem_raw);                       // [P][ph_region]
    C *sWm = win + (size_t)P * a.ph_region;                         // [P][kMaxChunks]
    C *sWi = sWm + P * kMaxChunks;                                  // [P][tile_nodes]
    const C *cw = win + d.shift;                                    // cw[k * ph_region + l], l in [0, lambda]
    if (threadIdx.x == 0) s_next = kWarps;
    if (dense && threadIdx.x == 0) {
        mbar_init(&wbar, 1);
        const uint32_t bytes = (uint32_t)(((size_t)(d.shift + d.lam) * sizeof(C) + 15) & ~(size_t)15);
        mbar_arrive_expect_tx(&wbar, bytes * P);
        for (int k = 0; k < P; ++k)
            bulk_g2s(win + (size_t)k * a.ph_region, a.ph_in + k * stride + (d.lo - d.shift), bytes, &wbar);
    }
    if (dense) community_observable<T, P>(a, d.comm, zc);
    // node inputs of Phase B: loaded while the copy is in flight, or (with
    // CIA_WINDOW_LATE_INPUTS) brought into L2 now and loaded after Phase A,
    // which keeps them out of Phase A's registers
    const int r = threadIdx.x;
    const int64_t m = d.first + r;
    const bool live = r < d.count;
    double theta_m = 0.0, wdt64_m = 0.0;
    T acc_m = T(0), wdt_m = T(0), omega_m = T(0);
    int32_t perm_m = 0;
    const unsigned char *b = a.blob + d.blob_off;
    uint32_t vt = 0u;
    auto load_inputs = [&]() {
        if (MODE == kRhs) {
            omega_m = a.omega[m];
            perm_m = a.perm[m];
        } else {
            theta_m = a.theta[m];
            if (!a.first_stage) acc_m = a.acc[m];
            if (MODE == kStage) wdt_m = a.wdt_next[m];
            else wdt64_m = a.wdt64[m];
        }
        vt = __ldg(reinterpret_cast<const uint32_t *>(b + d.vtab_off) + r);
    };
#if CIA_WINDOW_LATE_INPUTS
    if (live && MODE != kRhs) {
        prefetch_l2(a.theta + m);
        if (!a.first_stage) prefetch_l2(a.acc + m);
        if (MODE == kStage) prefetch_l2(a.wdt_next + m);
        else prefetch_l2(a.wdt64 + m);
    }
#else
    if (live) load_inputs();
#endif
    const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
    const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
    const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
    const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);
    __syncthreads();   // the barrier's initialisation is visible to every waiter
    bool ok = true;
    if (dense) {
        ok = mbar_wait_bounded(&wbar, 0, kWaitLimitNs);
        if (!ok && threadIdx.x == 0) atomicExch(a.err_flag, 1);
    }
    if (__syncthreads_or(!ok)) {
        // the copy may still land: wait for it once more before the CTA's
        // shared memory is released
        if (dense) mbar_wait_bounded(&wbar, 0, kWaitLimitNs);
        return;
    }
    // the padding entries lambda .. lambda + kPadSlots read zero phasors
    if (dense && threadIdx.x < P * (kPadSlots + 1))
        win[(size_t)(threadIdx.x / (kPadSlots + 1)) * a.ph_region + d.shift + d.lam + threadIdx.x % (kPadSlots + 1)] =
            mk2(T(0), T(0));
    __syncthreads();

#if CIA_WINDOW_DYNAMIC
    // slices are taken in order (longest first) by whichever warp is free
    for (int s = warp;; ) {
        if (s >= d.nsl) break;
#else
    for (int s = warp; s < d.nsl; s += kWarps) {
#endif
        const uint4 sd = __ldg(sdesc + s);
        const uint32_t rows = __ldg(srows + s * 32 + lane);
        const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
        C macc[P], iacc[P];   // sum over the missing links (subtracted at the end), over the inter links
#pragma unroll
        for (int k = 0; k < P; ++k) macc[k] = iacc[k] = mk2(T(0), T(0));
        const int4 *iv = ivec + sd.z + lane;
        const uint4 *mv = mvec + sd.x + lane;
        // every load of the slice's first index vectors is issued before any
        // of them is used: inter-community vectors, then the first missing
        // vectors; the inter gathers (global memory, longest latency) follow,
        // and the missing links (shared memory) are summed while they fly
        constexpr uint32_t kPre = (P == 1 && sizeof(T) == 4) ? CIA_WINDOW_INTER_VECTORS : 1;
        constexpr uint32_t kMv = sizeof(T) != 4 ? 1 : P == 1 ? CIA_WINDOW_VECTORS : P == 2 ? CIA_WINDOW_VECTORS_P2 : 1;   // vectors loaded ahead
        int4 qi[kPre];
        uint4 qm[kMv];
#pragma unroll
        for (uint32_t j = 0; j < kPre; ++j)
            if (j < sd.w) qi[j] = __ldg(iv + 32 * j);
#pragma unroll
        for (uint32_t j = 0; j < kMv; ++j)
            if (j < sd.y) qm[j] = __ldg(mv + 32 * j);
        C pre[kPre][4][P];
        for (uint32_t j0 = 0; j0 < sd.w || j0 == 0; j0 += kPre) {
            if (j0 > 0) {
#pragma unroll
                for (uint32_t j = 0; j < kPre; ++j)
                    if (j0 + j < sd.w) qi[j] = __ldg(iv + 32 * (j0 + j));
            }
#pragma unroll
            for (uint32_t j = 0; j < kPre; ++j) {
                if (j0 + j < sd.w) {
                    const int l4[4] = {qi[j].x, qi[j].y, qi[j].z, qi[j].w};
#pragma unroll
                    for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                        for (int k = 0; k < P; ++k) pre[j][hh][k] = __ldg(a.ph_in + k * stride + l4[hh]);
                }
            }
            if (j0 == 0) {
                for (uint32_t m0 = 0; m0 < sd.y; m0 += kMv) {
                    if (m0 > 0) {
#pragma unroll
                        for (uint32_t j = 0; j < kMv; ++j)
                            if (m0 + j < sd.y) qm[j] = __ldg(mv + 32 * (m0 + j));
                    }
#pragma unroll
                    for (uint32_t j = 0; j < kMv; ++j) {
                        if (m0 + j < sd.y) {
                            const uint32_t w4[4] = {qm[j].x, qm[j].y, qm[j].z, qm[j].w};
#pragma unroll
                            for (int hh = 0; hh < 4; ++hh) {
                                const int l0 = (int)(w4[hh] & 0xffffu), l1 = (int)(w4[hh] >> 16);
#pragma unroll
                                for (int k = 0; k < P; ++k)
                                    macc[k] = add2(macc[k], add2(cw[k * a.ph_region + l0], cw[k * a.ph_region + l1]));
                            }
                        }
                    }
                }
            }
#pragma unroll
            for (uint32_t j = 0; j < kPre; ++j) {
                if (j0 + j < sd.w) {
#pragma unroll
                    for (int k = 0; k < P; ++k)
                        iacc[k] = add2(iacc[k], add2(add2(pre[j][0][k], pre[j][1][k]), add2(pre[j][2][k], pre[j][3][k])));
                }
            }
        }
        if (mrow != 0xffffu) {
#pragma unroll
            for (int k = 0; k < P; ++k) sWm[k * kMaxChunks + mrow] = mk2(-macc[k].x, -macc[k].y);
        }
        if (irow != 0xffffu) {
#pragma unroll
            for (int k = 0; k < P; ++k) sWi[k * a.tile_nodes + irow] = iacc[k];
        }
#if CIA_WINDOW_DYNAMIC
        int nx = 0;
        if (lane == 0) nx = atomicAdd(&s_next, 1);
        s = __shfl_sync(0xffffffffu, nx, 0);
#endif
    }
    __syncthreads();
    // Phase B, thread per node
    T sre[P], sim[P];
#pragma unroll
    for (int k = 0; k < P; ++k) sre[k] = sim[k] = T(0);
#if CIA_WINDOW_LATE_INPUTS
    if (live) load_inputs();
#endif
    if (live) {
        T coup = T(0);
        C uk[P];
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const C u = dense ? cw[k * a.ph_region + (int)(m - d.lo)] : __ldg(a.ph_in + k * stride + m);
            uk[k] = u;
            C w = sWi[k * a.tile_nodes + r];
            for (int c = (int)(vt & 0xffffu); c < (int)(vt & 0xffffu) + (int)(vt >> 16); ++c) {
                const C v = sWm[k * kMaxChunks + c];
                w.x += v.x;
                w.y += v.y;
            }
            T zr = w.x, zi = w.y;
            if (dense) {
                // (E1.2) dense term: the whole block minus its diagonal (a_mm = 0)
                zr += zc[k].x - u.x;
                zi += zc[k].y - u.y;
            }
            const T re = zr * u.x + zi * u.y;
            const T im = zi * u.x - zr * u.y;
            coup += a.d_sin[k] * im + a.d_cos[k] * re;
        }
        coup *= a.tile_kn ? a.tile_kn[t] : a.k_over_n;
        if (P >= 2 && dense && a.k2_over_n2 != T(0))
            coup += a.k2_over_n2 * triadic_from_moments<T>(zc[0].x, zc[0].y, zc[P >= 2 ? 1 : 0].x,
                                                           zc[P >= 2 ? 1 : 0].y, uk[0].x, uk[0].y,
                                                           uk[P >= 2 ? 1 : 0].x, uk[P >= 2 ? 1 : 0].y);
        if (a.tri) coup += a.tri[m];
        if (MODE == kRhs) {
            a.rhs_out[perm_m] = (double)omega_m + (double)coup;
        } else {
            const T accv = acc_m + a.b_s * coup;
            T y;
            if (MODE == kStage) {
                a.acc[m] = accv;
                y = (T)theta_m + wdt_m + a.c_next_dt * coup;
            } else {
                // FP64 time accumulation: theta += dt omega + dt sum_s b_s C_s
                const double th = wrap_pi(theta_m + wdt64_m + a.dt * (double)accv);
                a.theta[m] = th;
                y = (T)th;
            }
            C u[P];
            phasors<T, P>(y, u);
#pragma unroll
            for (int k = 0; k < P; ++k) {
                a.ph_out[k * stride + m] = u[k];
                sre[k] = u[k].x;
                sim[k] = u[k].y;
            }
        }
    }
    if (MODE == kRhs) return;
    block_tile_sum<T, P>(sre, sim, red, a.part_out + (size_t)t * P * 2);
}

// Z_c = sum of community c's tile partials in FP64, by one warp: lane j adds
// tiles j, j + 32, ..., then a fixed xor tree (the order of
// community_observable); every lane ends with the sums.  part is read
// through L2, so that partials other CTAs wrote in this launch are seen.
template <int P>
__device__ __forceinline__ void community_sum_fp64(const int32_t *comm_tile_begin, const double *part, int c, int lane,
                                                   double (&re)[P], double (&im)[P]) {
    const int u0 = comm_tile_begin[c], u1 = comm_tile_begin[c + 1];
#pragma unroll
    for (int k = 0; k < P; ++k) re[k] = im[k] = 0.0;
    for (int u = u0 + lane; u < u1; u += 32) {
#pragma unroll
        for (int k = 0; k < P; ++k) {
            const double2 v = __ldcg(reinterpret_cast<const double2 *>(part) + (int64_t)u * P + k);
            re[k] += v.x;
            im[k] += v.y;
        }
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re[k] += __shfl_xor_sync(0xffffffffu, re[k], o);
            im[k] += __shfl_xor_sync(0xffffffffu, im[k], o);
        }
    }
}

// (E1.1) Z_c of every community from the tile partials of a loaded state
// (one warp per community), and the ring kernel's per-community counters
// reset, before its first stage.
template <int P>
__global__ void community_sums_kernel(int64_t M, const int32_t *comm_tile_begin, const double *part, double *z,
                                      int *comm_done) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    if (c >= M) return;
    double re[P], im[P];
    community_sum_fp64<P>(comm_tile_begin, part, (int)c, lane, re, im);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < P; ++k) reinterpret_cast<double2 *>(z)[c * P + k] = make_double2(re[k], im[k]);
        comm_done[c] = 0;
    }
}

// ---- persistent CIA stage with a ring of per-tile buffers (staging 4) -------
//
// One CTA per SM.  The last warp is the producer: for each of the CTA's
// tiles (round k of CTA c takes launch rank k G + c for even k, k G + G - 1 - c
// for odd k: the costliest-first order dealt out in a snake) it waits for a
// free ring slot, copies the tile's descriptor into the slot's header, issues
// bulk (TMA) copies of the community's phasor window (every harmonic) and of
// the tile's index blob into the slot, writes the window's zero padding, sums
// the community observable Z_c from the previous stage's tile partials and
// then arrives on the slot's `full` barrier.  The other warps consume: they
// take the slices of successive tiles round-robin (slice g of the running
// count goes to warp g mod W), so no warp waits for another within a tile.
// A slice holds whole rows: a row's missing list is cut into v chunks on v
// consecutive lanes, the lanes' sums are combined by a segmented shuffle tree,
// and the row's first lane applies the coupling, the RK4 stage update and the
// next phasors (Phase B).  Each warp records its slice's phasor sums in the
// slot header; the warp that completes a tile adds them in slice order into
// the tile partial and every warp arrives on the slot's `empty` barrier.
#ifndef CIA_RING_WARPS
#define CIA_RING_WARPS 16           // consumer warps per CTA
#endif
constexpr int kRingWarps = CIA_RING_WARPS;
constexpr int kRingThreads = 32 * (kRingWarps + 1);
constexpr int kRingMaxSlots = 6;

template <typename T, int P>
struct RingHeader {
    using C = typename Vec2<T>::type;
    TileDesc d;
    C zc[P];
    int tile;
    int done;                                 // slices finished (the completing warp resets it)
    double part[kRingMaxSlices][2 * P];       // per slice: sum of the next phasors
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

template <typename T, int P>
__device__ __forceinline__ uint32_t ring_window_stride(const TileDesc &d) {
    // bytes per harmonic: shift + lambda phasors, the guard entry and the
    // kPadSlots zero entries, 16-byte rounded
    using C = typename Vec2<T>::type;
    return d.comm >= 0 ? (uint32_t)(((size_t)(d.shift + d.lam + 1 + kPadSlots) * sizeof(C) + 15) & ~(size_t)15) : 0u;
}

template <typename T, int P, int MODE>
__global__ void __launch_bounds__(kRingThreads, 1) cia_ring_kernel(const StageParams<T> a) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kRingMaxSlots], empty_bar[kRingMaxSlots];
    __shared__ __align__(16) RingHeader<T, P> hdr[kRingMaxSlots];
    __shared__ volatile int s_abort;

    const int S = a.stages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x;
    const int64_t stride = a.ph_stride;
    auto tile_at = [&](int k) -> int {
        const int64_t rank = (int64_t)k * G + ((k & 1) ? G - 1 - (int)blockIdx.x : (int)blockIdx.x);
        return rank < a.n_tiles ? a.tile_order[rank] : -1;
    };
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full_bar[q], 1);
            mbar_init(&empty_bar[q], kRingWarps);
            hdr[q].done = 0;
        }
        s_abort = 0;
    }
    __syncthreads();

    if (warp == kRingWarps) {
        // ------------------------------------------------------------ producer
        // lane 0 fetches the next tile's descriptor and community observable
        // before it waits for that tile's slot, so the loads overlap the wait
        int issued = 0;
        int t_next = tile_at(0);
        TileDesc d_next;
        C z_next[P];
        auto fetch = [&](int t) {
            d_next = a.tile_desc[t];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
                const double2 zz = d_next.comm >= 0
                                       ? reinterpret_cast<const double2 *>(a.z_in)[(int64_t)d_next.comm * P + kk]
                                       : make_double2(0.0, 0.0);
                z_next[kk] = mk2((T)zz.x, (T)zz.y);
            }
        };
        if (lane == 0 && t_next >= 0) fetch(t_next);
        for (int k = 0; t_next >= 0; ++k) {
            const int t = t_next;
            const int q = k % S;
            int ok = 1;
            if (lane == 0) {
                if (s_abort) ok = 0;
                else if (k >= S) ok = mbar_wait_bounded(&empty_bar[q], (uint32_t)((k / S - 1) & 1), kWaitLimitNs);
                if (!ok && !s_abort) {
                    atomicExch(a.err_flag, 1);
                    s_abort = 1;
                }
                if (ok) {
                    hdr[q].d = d_next;
                    hdr[q].tile = t;
#pragma unroll
                    for (int kk = 0; kk < P; ++kk) hdr[q].zc[kk] = z_next[kk];
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            __syncwarp();
            const TileDesc &d = hdr[q].d;
            unsigned char *buf = smem_raw + (size_t)q * a.tile_buf;
            const uint32_t wreg = ring_window_stride<T, P>(d);
            // the window rounded up to 16 bytes (the guard entry lambda may take
            // the next community's first phasor) and the blob
            const uint32_t wtma = d.comm >= 0 ? (uint32_t)(((size_t)(d.shift + d.lam) * sizeof(C) + 15) & ~(size_t)15) : 0u;
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_expect_tx(&full_bar[q], wtma * P + d.blob_bytes);
                if (wtma)
                    for (int kk = 0; kk < P; ++kk)
                        bulk_g2s(buf + (size_t)kk * wreg, a.ph_in + kk * stride + (d.lo - d.shift), wtma, &full_bar[q]);
                if (d.blob_bytes) bulk_g2s(buf + (size_t)P * wreg, a.blob + d.blob_off, d.blob_bytes, &full_bar[q]);
            }
            ++issued;
            // the padding entries lambda + 1 .. lambda + kPadSlots (zero), beyond the copy
            if (d.comm >= 0)
                for (int i = lane; i < P * kPadSlots; i += 32)
                    reinterpret_cast<C *>(buf + (size_t)(i / kPadSlots) * wreg)[d.shift + d.lam + 1 + i % kPadSlots] =
                        mk2(T(0), T(0));
            __threadfence_block();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_bar[q]);                 // release: header and padding
            t_next = tile_at(k + 1);
            if (lane == 0 && t_next >= 0) fetch(t_next);
        }
        // every copy issued has landed before the CTA can retire
        if (lane == 0)
            for (int k = issued > S ? issued - S : 0; k < issued; ++k)
                mbar_wait_bounded(&full_bar[k % S], (uint32_t)((k / S) & 1), kWaitLimitNs);
        return;
    }

    // -------------------------------------------------------------- consumers
    // this CTA's tiles: the rounds whose launch rank exists (no memory access)
    int ntiles = 0;
    while ((int64_t)ntiles * G + ((ntiles & 1) ? G - 1 - (int)blockIdx.x : (int)blockIdx.x) < a.n_tiles) ++ntiles;
    int64_t base = 0;   // slices of the tiles before this one
    for (int k = 0; k < ntiles; ++k) {
        const int q = k % S;
        bool ok = mbar_wait_bounded(&full_bar[q], (uint32_t)((k / S) & 1), kWaitLimitNs);
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err_flag, 1);
                s_abort = 1;
            }
            return;
        }
        const RingHeader<T, P> &h = hdr[q];
        const int t = h.tile;
        const int nsl = h.d.nsl, count = h.d.count;
        const bool dense = h.d.comm >= 0;
        const int64_t first = h.d.first, lo = h.d.lo;
        const unsigned char *buf = smem_raw + (size_t)q * a.tile_buf;
        const uint32_t wreg = ring_window_stride<T, P>(h.d);
        const int wstride = (int)(wreg / sizeof(C));
        const C *cw = reinterpret_cast<const C *>(buf) + h.d.shift;        // cw[k * wstride + l]
        const unsigned char *b = buf + (size_t)P * wreg;
        const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
        const uint32_t *lmap = reinterpret_cast<const uint32_t *>(b + 16 * nsl);
        const uint4 *mvec = reinterpret_cast<const uint4 *>(b + h.d.mvec_off);
        const int4 *ivec = reinterpret_cast<const int4 *>(b + h.d.ivec_off);
        const T kn = a.tile_kn ? a.tile_kn[t] : a.k_over_n;
        (void)count;
        int mine = 0;
        for (int sl = (int)(((int64_t)warp - base) % kRingWarps + kRingWarps) % kRingWarps; sl < nsl;
             sl += kRingWarps) {
            ++mine;
            const uint32_t mw = lmap[sl * 32 + lane];
            const bool live = mw != 0xffffffffu;
            const int r = (int)(mw & 0xffffu), v = (int)((mw >> 16) & 63u), off = (int)((mw >> 22) & 31u);
            const bool head = live && off == 0;
            const int64_t m = first + r;
            // node inputs of the row (first lane), loaded while the gathers run
            double theta_m = 0.0, wdt64_m = 0.0;
            T acc_m = T(0), wdt_m = T(0), omega_m = T(0);
            int32_t perm_m = 0;
            C um[P];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) um[kk] = mk2(T(0), T(0));
            if (head) {
                if (MODE == kRhs) {
                    omega_m = a.omega[m];
                    perm_m = a.perm[m];
                } else {
                    theta_m = a.theta[m];
                    if (!a.first_stage) acc_m = a.acc[m];
                    if (MODE == kStage) wdt_m = a.wdt_next[m];
                    else wdt64_m = a.wdt64[m];
                }
#pragma unroll
                for (int kk = 0; kk < P; ++kk)
                    um[kk] = dense ? cw[kk * wstride + (int)(m - lo)] : __ldg(a.ph_in + kk * stride + m);
            }
            // Phase A: inter-community gathers (global) issued first, missing
            // links from the shared-memory window while they fly
            const uint4 sdv = sdesc[sl];
            C macc[P], iacc[P];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) macc[kk] = iacc[kk] = mk2(T(0), T(0));
            const int4 *iv = ivec + sdv.z + lane;
            const uint4 *mv = mvec + sdv.x + lane;
            constexpr uint32_t kPre = (P == 1 && sizeof(T) == 4) ? CIA_WINDOW_INTER_VECTORS : 1;
            for (uint32_t j0 = 0; j0 < sdv.w || j0 == 0; j0 += kPre) {
                C pre[kPre][4][P];
#pragma unroll
                for (uint32_t qq = 0; qq < kPre; ++qq) {
                    if (j0 + qq < sdv.w) {
                        const int4 iq = iv[32 * (j0 + qq)];
                        const int l4[4] = {iq.x, iq.y, iq.z, iq.w};
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                            for (int kk = 0; kk < P; ++kk) pre[qq][hh][kk] = __ldg(a.ph_in + kk * stride + l4[hh]);
                    }
                }
                if (j0 == 0) {
#pragma unroll 2
                    for (uint32_t jj = 0; jj < sdv.y; ++jj) {
                        const uint4 mq = mv[32 * jj];
                        const uint32_t w4[4] = {mq.x, mq.y, mq.z, mq.w};
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh) {
                            const int l0 = (int)(w4[hh] & 0xffffu), l1 = (int)(w4[hh] >> 16);
#pragma unroll
                            for (int kk = 0; kk < P; ++kk)
                                macc[kk] = add2(macc[kk], add2(cw[kk * wstride + l0], cw[kk * wstride + l1]));
                        }
                    }
                }
#pragma unroll
                for (uint32_t qq = 0; qq < kPre; ++qq) {
                    if (j0 + qq < sdv.w) {
#pragma unroll
                        for (int kk = 0; kk < P; ++kk)
                            iacc[kk] = add2(iacc[kk], add2(add2(pre[qq][0][kk], pre[qq][1][kk]),
                                                           add2(pre[qq][2][kk], pre[qq][3][kk])));
                    }
                }
            }
            // a row's chunk sums: segmented tree over its v lanes (the first lane
            // ends with lanes [0, v) of the row, in a fixed order)
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const bool take = live && off + o < v;
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
                    const T xr = __shfl_down_sync(0xffffffffu, macc[kk].x, o);
                    const T xi = __shfl_down_sync(0xffffffffu, macc[kk].y, o);
                    if (take) macc[kk] = mk2(macc[kk].x + xr, macc[kk].y + xi);
                }
            }
            // Phase B, first lane of each row
            T sre[P], sim[P];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) sre[kk] = sim[kk] = T(0);
            if (head) {
                T coup = T(0);
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
                    const C u = um[kk];
                    T zr = iacc[kk].x - macc[kk].x, zi = iacc[kk].y - macc[kk].y;
                    if (dense) {
                        // (E1.2) dense term: the whole block minus its diagonal (a_mm = 0)
                        zr += h.zc[kk].x - u.x;
                        zi += h.zc[kk].y - u.y;
                    }
                    const T re = zr * u.x + zi * u.y;
                    const T im = zi * u.x - zr * u.y;
                    coup += a.d_sin[kk] * im + a.d_cos[kk] * re;
                }
                coup *= kn;
                if (P >= 2 && dense && a.k2_over_n2 != T(0))
                    coup += a.k2_over_n2 * triadic_from_moments<T>(h.zc[0].x, h.zc[0].y, h.zc[P >= 2 ? 1 : 0].x,
                                                                   h.zc[P >= 2 ? 1 : 0].y, um[0].x, um[0].y,
                                                                   um[P >= 2 ? 1 : 0].x, um[P >= 2 ? 1 : 0].y);
                if (a.tri) coup += a.tri[m];
                if (MODE == kRhs) {
                    a.rhs_out[perm_m] = (double)omega_m + (double)coup;
                } else {
                    const T accv = acc_m + a.b_s * coup;
                    T y;
                    if (MODE == kStage) {
                        a.acc[m] = accv;
                        y = (T)theta_m + wdt_m + a.c_next_dt * coup;
                    } else {
                        // FP64 time accumulation: theta += dt omega + dt sum_s b_s C_s
                        const double th = wrap_pi(theta_m + wdt64_m + a.dt * (double)accv);
                        a.theta[m] = th;
                        y = (T)th;
                    }
                    C u[P];
                    phasors<T, P>(y, u);
#pragma unroll
                    for (int kk = 0; kk < P; ++kk) {
                        a.ph_out[kk * stride + m] = u[kk];
                        sre[kk] = u[kk].x;
                        sim[kk] = u[kk].y;
                    }
                }
            }
            if (MODE != kRhs) {
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        sre[kk] += __shfl_xor_sync(0xffffffffu, sre[kk], o);
                        sim[kk] += __shfl_xor_sync(0xffffffffu, sim[kk], o);
                    }
                }
                if (lane < P) {
                    hdr[q].part[sl][2 * lane] = (double)sre[lane];
                    hdr[q].part[sl][2 * lane + 1] = (double)sim[lane];
                }
            }
        }
        base += nsl;
        // the warp that finishes the tile's last slice writes its partial sums
        int last = 0;
        if (MODE != kRhs) {
            if (lane == 0 && mine > 0) {
                __threadfence_block();
                last = atomicAdd(&hdr[q].done, mine) + mine == nsl;
            }
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence_block();
                if (lane < 2 * P) {
                    double sum = 0.0;
                    for (int sl = 0; sl < nsl; ++sl) sum += hdr[q].part[sl][lane];
                    a.part_out[(size_t)t * P * 2 + lane] = sum;
                }
                // the partial is visible device-wide before the community counter moves
                __threadfence();
                if (lane == 0) hdr[q].done = 0;
            }
        }
        const int comm = h.d.comm;
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty_bar[q]);                    // the slot is free again
        if (last && comm >= 0) {
            // the community's last tile: its observable for the next stage from
            // every tile partial, in the fixed order of the other kernels
            int fin = 0;
            if (lane == 0)
                fin = atomicAdd(a.comm_done + comm, 1) + 1 == a.comm_tile_begin[comm + 1] - a.comm_tile_begin[comm];
            if (__shfl_sync(0xffffffffu, fin, 0)) {
                __threadfence();
                double re[P], im[P];
                community_sum_fp64<P>(a.comm_tile_begin, a.part_out, comm, lane, re, im);
                if (lane == 0) {
#pragma unroll
                    for (int kk = 0; kk < P; ++kk)
                        reinterpret_cast<double2 *>(a.z_out)[(int64_t)comm * P + kk] = make_double2(re[kk], im[kk]);
                    a.comm_done[comm] = 0;
                }
            }
        }
    }
}

// ---- persistent, warp-specialised CIA stage (the main path) ----------------
//
// One CTA per SM walks a contiguous range of tiles.  The last warp is the
// producer: its lane 0 copies, with TMA bulk copies, each tile's sliced-ELL
// index vectors into a ring of `stages` shared-memory buffers (mbarrier
// full/empty pairs) and the phasors of each new community into one of two
// community buffers (pfull/pempty), running ahead of the consumers.  Two
// consumer groups of eight warps take alternate tiles (ping-pong), so one
// group's latency-bound phase overlaps the other's.  Per tile a group runs
// Phase A (warp per slice, lane per row: inter-community gathers issued
// first, then the shared-memory gathers of the missing links; separate sum
// arrays, so no barrier between them) and Phase B (thread per node).  Every
// wait is bounded; a wait that gives up sets the plan's error flag and all
// warps leave once the copies already issued have landed.

constexpr int kConsumerWarps = 8;                 // per group
constexpr int kConsumers = 32 * kConsumerWarps;   // threads per group = max tile rows
constexpr int kGroups = 2;
constexpr int kPipeThreads = kGroups * kConsumers + 32;
constexpr int kMaxStages = 4;


template <typename T, int P, int MODE>
__global__ void __launch_bounds__(kPipeThreads, 1) cia_pipeline_kernel(const StageParams<T> a) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages];
    __shared__ __align__(8) uint64_t pfull_bar[2], pempty_bar[2], desc_bar;
    __shared__ __align__(8) uint64_t swfull_bar[2], swempty_bar[2];   // gather -> node hand-off
    __shared__ __align__(8) uint64_t zready_bar;   // observables of all runs written
    __shared__ double red[kConsumerWarps][2 * P];
    __shared__ volatile int s_prod_abort, s_cons_abort;

    const int S = a.stages;
    const int tb = a.cta_tile_begin[blockIdx.x], te = a.cta_tile_begin[blockIdx.x + 1];
    // shared memory: tile descriptors | ring of tile blobs | 2 community windows | W sums
    TileDesc *sdesc = reinterpret_cast<TileDesc *>(smem_raw);               // [max_cta_tiles]
    C *zrun = reinterpret_cast<C *>(sdesc + a.max_cta_tiles);               // [max_cta_runs][P]
    // the ring is the destination of bulk copies: keep it 128-byte aligned
    unsigned char *ring = reinterpret_cast<unsigned char *>(zrun) + zrun_bytes(a.max_cta_runs, P, sizeof(C));
    C *pbuf = reinterpret_cast<C *>(ring + (size_t)S * a.idx_cap);         // [2][P][ph_region]
    C *sWall = pbuf + 2 * P * a.ph_region;                                 // [groups][2][P][kConsumers]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = a.ph_stride;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], kConsumerWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&pfull_bar[b], 1);
            mbar_init(&pempty_bar[b], kConsumerWarps);
            mbar_init(&swfull_bar[b], kConsumerWarps);
            mbar_init(&swempty_bar[b], kConsumerWarps);
        }
        mbar_init(&desc_bar, 1);
        mbar_init(&zready_bar, 1);
        s_prod_abort = 0;
        s_cons_abort = 0;
        // this CTA's tile descriptors, one bulk copy
        const uint32_t dbytes = (uint32_t)((te - tb) * sizeof(TileDesc));
        mbar_arrive_expect_tx(&desc_bar, dbytes);
        if (dbytes) bulk_g2s(sdesc, a.tile_desc + tb, dbytes, &desc_bar);
    }
    __syncthreads();
    {
        bool fail = false;
        if (threadIdx.x == 0) {
            fail = !mbar_wait_bounded(&desc_bar, 0, kWaitLimitNs);
            if (fail) {
                atomicExch(a.err_flag, 1);
                mbar_wait_bounded(&desc_bar, 0, kWaitLimitNs / 2);
            }
        }
        if (__syncthreads_or(fail)) return;
    }

    if (warp == kGroups * kConsumerWarps) {
        // ------------------------------------------------------------ producer
        // lane 0 waits and issues the copies.  The whole warp reduces the
        // community observables of every run of this CTA and posts them on
        // zready before the producer's first wait that can block: consumers
        // need them to finish a tile, and that wait may need a finished tile.
        int issued = 0, last_pload = -1;
        bool zdone = false;
        auto post_observables = [&]() {
            // (E1.1) lane j adds tiles j, j + 32, ... in FP64, then a fixed
            // shuffle tree (deterministic order)
            for (int q = 0; q < te - tb; ++q) {
                const TileDesc &dq = sdesc[q];
                if (dq.comm < 0 || (q > 0 && sdesc[q - 1].run == dq.run)) continue;
                const int u0 = a.comm_tile_begin[dq.comm], u1 = a.comm_tile_begin[dq.comm + 1];
                double re[P], im[P];
#pragma unroll
                for (int kk = 0; kk < P; ++kk) re[kk] = im[kk] = 0.0;
                for (int u = u0 + lane; u < u1; u += 32) {
#pragma unroll
                    for (int kk = 0; kk < P; ++kk) {
                        const double2 v = __ldg(reinterpret_cast<const double2 *>(a.part_in) + (int64_t)u * P + kk);
                        re[kk] += v.x;
                        im[kk] += v.y;
                    }
                }
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        re[kk] += __shfl_xor_sync(0xffffffffu, re[kk], o);
                        im[kk] += __shfl_xor_sync(0xffffffffu, im[kk], o);
                    }
                    if (lane == 0) zrun[(size_t)dq.run * P + kk] = mk2((T)re[kk], (T)im[kk]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&zready_bar);     // all observables written (release)
            zdone = true;
        };
        for (int i = tb; i < te; ++i) {
            const int li = i - tb, s = li % S, k = li / S;
            const TileDesc &d = sdesc[li];
            const bool dense = d.comm >= 0;
            const bool new_run = dense && (li == 0 || sdesc[li - 1].run != d.run);
            if (!zdone && (k >= 1 || (new_run && d.run >= 2))) post_observables();
            int ok = 1;
            if (lane == 0) {
                if (s_cons_abort) ok = 0;
                else if (k >= 1) ok = mbar_wait_bounded(&empty_bar[s], (k - 1) & 1, kWaitLimitNs);
                if (!ok && !s_cons_abort) {
                    atomicExch(a.err_flag, 1);
                    s_prod_abort = 1;
                }
            }
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            if (new_run) {
                const int run = d.run, b = run & 1;
                if (lane == 0) {
                    // every group releases run - 2 of this buffer before it is reused
                    if (run >= 2) ok = mbar_wait_bounded(&pempty_bar[b], ((run >> 1) - 1) & 1, kWaitLimitNs);
                    if (!ok) {
                        atomicExch(a.err_flag, 1);
                        s_prod_abort = 1;
                    } else {
                        constexpr int64_t per16 = 16 / (int64_t)sizeof(C);
                        const int64_t pstart = d.lo - d.shift;
                        const int64_t pend = (d.lo + d.lam + 1 + per16 - 1) & ~(per16 - 1);
                        const uint32_t pbytes = (uint32_t)((pend - pstart) * (int64_t)sizeof(C));
                        mbar_arrive_expect_tx(&pfull_bar[b], P * pbytes);
                        for (int kk = 0; kk < P; ++kk)
                            bulk_g2s(pbuf + (b * P + kk) * a.ph_region, a.ph_in + kk * stride + pstart, pbytes,
                                     &pfull_bar[b]);
                    }
                }
                if (!__shfl_sync(0xffffffffu, ok, 0)) break;
                last_pload = run;
            }
            if (lane == 0) {
                unsigned char *slot = ring + (size_t)s * a.idx_cap;
                mbar_arrive_expect_tx(&full_bar[s], d.blob_bytes);
                if (d.blob_bytes) bulk_g2s(slot, a.blob + d.blob_off, d.blob_bytes, &full_bar[s]);
            }
            ++issued;
        }
        if (!zdone && !s_prod_abort && !s_cons_abort) post_observables();
        // let every copy this warp issued land before the CTA can retire
        if (lane == 0) {
            for (int li = (issued > S ? issued - S : 0); li < issued; ++li)
                mbar_wait_bounded(&full_bar[li % S], (li / S) & 1, kWaitLimitNs);
            for (int r = (last_pload > 0 ? last_pload - 1 : 0); r <= last_pload; ++r)
                mbar_wait_bounded(&pfull_bar[r & 1], (r >> 1) & 1, kWaitLimitNs);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int grp = warp / kConsumerWarps;                 // 0: gather warps, 1: node warps
    const int gw = warp % kConsumerWarps;                  // warp within the group
    const int gt = threadIdx.x - grp * kConsumers;         // thread within the group
    auto gsync_or = [&](bool pred) {
        uint32_t r;
        asm volatile(
            "{\n\t.reg .pred p, q;\n\t"
            "setp.ne.u32 p, %1, 0;\n\t"
            "bar.red.or.pred q, %2, %3, p;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(r)
            : "r"((uint32_t)pred), "r"(1 + grp), "r"(kConsumers)
            : "memory");
        return r != 0;
    };
    auto gsync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(kConsumers) : "memory"); };
    // hand-off buffers, two of each: chunk sums, inter sums, row -> chunk tables
    auto sWm_of = [&](int b) { return sWall + (size_t)b * P * (kMaxChunks + kConsumers); };   // [P][kMaxChunks]
    auto sWi_of = [&](int b) { return sWm_of(b) + P * kMaxChunks; };                           // [P][kConsumers]
    uint32_t *sWv = reinterpret_cast<uint32_t *>(sWall + 2 * (size_t)P * (kMaxChunks + kConsumers));   // [2][kConsumers]

    if (grp == 0) {
        // ------------------------------------------------- gather warps (Phase A)
        for (int i = tb; i < te; ++i) {
            const int li = i - tb, s = li % S, k = li / S, b = li & 1, u = li >> 1;
            const unsigned char *slot = ring + (size_t)s * a.idx_cap;
            const TileDesc h = sdesc[li];
            const bool dense = h.comm >= 0;
            bool fail = false;
            if (gt == 0) {
                fail = s_prod_abort || !mbar_wait_bounded(&full_bar[s], k & 1, kWaitLimitNs);
                if (!fail && dense) {
                    fail = !mbar_wait_bounded(&pfull_bar[h.pbuf], (h.run >> 1) & 1, kWaitLimitNs);
                    // the slots after the community are where padding entries point: zero them
                    if (!fail)
                        for (int kk = 0; kk < P; ++kk)
                            for (int j = 0; j <= kPadSlots; ++j)
                                pbuf[(h.pbuf * P + kk) * a.ph_region + h.shift + h.lam + j] = mk2(T(0), T(0));
                }
                if (!fail && u >= 1) fail = !mbar_wait_bounded(&swempty_bar[b], (u - 1) & 1, kWaitLimitNs);
                if (fail) {
                    atomicExch(a.err_flag, 1);
                    s_cons_abort = 1;
                }
            }
            if (gsync_or(fail)) break;
            const C *cph = pbuf + (size_t)h.pbuf * P * a.ph_region + h.shift;   // cph[k * ph_region + l]
            const uint4 *sdsl = reinterpret_cast<const uint4 *>(slot);
            const uint32_t *srows = reinterpret_cast<const uint32_t *>(slot + 16 * h.nsl);
            const uint4 *mvec = reinterpret_cast<const uint4 *>(slot + h.mvec_off);
            const int4 *ivec = reinterpret_cast<const int4 *>(slot + h.ivec_off);
            C *sWm = sWm_of(b), *sWi = sWi_of(b);
            // per slice: inter-community gathers (global) issued first, then the
            // missing links from the community window (shared)
            for (int sl = gw; sl < h.nsl; sl += kConsumerWarps) {
                const uint4 d = sdsl[sl];
                const uint32_t rows = srows[sl * 32 + lane];
                const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
                T ire[P], iim[P], mre[P], mim[P];
#pragma unroll
                for (int kk = 0; kk < P; ++kk) ire[kk] = iim[kk] = mre[kk] = mim[kk] = T(0);
                const int4 *iv = ivec + d.z + lane;
                constexpr uint32_t kPre = (P == 1 && sizeof(T) == 4) ? 4 : 1;   // vectors gathered ahead
                C pre[kPre][4][P];
                const uint32_t npre = d.w < kPre ? d.w : kPre;
#pragma unroll
                for (uint32_t j = 0; j < kPre; ++j) {
                    if (j < npre) {
                        const int4 q = iv[32 * j];
                        const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                            for (int kk = 0; kk < P; ++kk) pre[j][hh][kk] = __ldg(a.ph_in + kk * stride + l4[hh]);
                    }
                }
                const uint4 *mv = mvec + d.x + lane;
#pragma unroll 2
                for (uint32_t j = 0; j < d.y; ++j) {
                    const uint4 q = mv[32 * j];
                    const unsigned w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int hh = 0; hh < 4; ++hh) {
                        const int l0 = (int)(w4[hh] & 0xffffu), l1 = (int)(w4[hh] >> 16);
#pragma unroll
                        for (int kk = 0; kk < P; ++kk) {
                            const C v0 = cph[kk * a.ph_region + l0];
                            const C v1 = cph[kk * a.ph_region + l1];
                            mre[kk] -= v0.x + v1.x;
                            mim[kk] -= v0.y + v1.y;
                        }
                    }
                }
#pragma unroll
                for (uint32_t j = 0; j < kPre; ++j) {
                    if (j < npre) {
#pragma unroll
                        for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                            for (int kk = 0; kk < P; ++kk) {
                                ire[kk] += pre[j][hh][kk].x;
                                iim[kk] += pre[j][hh][kk].y;
                            }
                    }
                }
                // longer inter lists: further batches of kPre vectors, loads first
                for (uint32_t j0 = kPre; j0 < d.w; j0 += kPre) {
#pragma unroll
                    for (uint32_t j = 0; j < kPre; ++j) {
                        if (j0 + j < d.w) {
                            const int4 q = iv[32 * (j0 + j)];
                            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                            for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                                for (int kk = 0; kk < P; ++kk) pre[j][hh][kk] = __ldg(a.ph_in + kk * stride + l4[hh]);
                        }
                    }
#pragma unroll
                    for (uint32_t j = 0; j < kPre; ++j) {
                        if (j0 + j < d.w) {
#pragma unroll
                            for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                                for (int kk = 0; kk < P; ++kk) {
                                    ire[kk] += pre[j][hh][kk].x;
                                    iim[kk] += pre[j][hh][kk].y;
                                }
                        }
                    }
                }
                if (mrow != 0xffffu) {
#pragma unroll
                    for (int kk = 0; kk < P; ++kk) sWm[kk * kMaxChunks + mrow] = mk2(mre[kk], mim[kk]);
                }
                if (irow != 0xffffu) {
#pragma unroll
                    for (int kk = 0; kk < P; ++kk) sWi[kk * kConsumers + irow] = mk2(ire[kk], iim[kk]);
                }
            }
            // the row -> chunk table travels with the sums (the ring buffer is
            // released below)
            if (gt < h.count) sWv[b * kConsumers + gt] = reinterpret_cast<const uint32_t *>(slot + h.vtab_off)[gt];
            gsync();
            if (lane == 0) {
                mbar_arrive(&empty_bar[s]);                   // the ring buffer is free again
                mbar_arrive(&swfull_bar[b]);                  // the sums of tile i are ready (release)
            }
        }
        return;
    }

    // ------------------------------------------------------- node warps (Phase B)
    // release of a community buffer: once per run, in run order, as soon as
    // these warps have finished their last tile of the run (known from the
    // tile descriptors, never from the producer, which may itself be waiting
    // for the release).  A run is released only after its own phasor load
    // has landed: that load was issued after the producer saw the release of
    // run - 2, so a buffer's pempty barrier never runs two phases ahead of
    // its waiter.
    int released = -1;
    const int nruns = a.cta_runs[blockIdx.x];
    auto release_through = [&](int run_upto) {
        for (int r = released + 1; r <= run_upto; ++r) {
            if (lane == 0 && !s_cons_abort && !s_prod_abort) {
                if (mbar_wait_bounded(&pfull_bar[r & 1], (r >> 1) & 1, kWaitLimitNs)) {
                    mbar_arrive(&pempty_bar[r & 1]);
                } else {
                    atomicExch(a.err_flag, 1);
                    s_cons_abort = 1;
                }
            }
        }
        if (run_upto > released) released = run_upto;
    };
    bool zwaited = false;
    for (int i = tb; i < te; ++i) {
        const int li = i - tb, b = li & 1, u = li >> 1;
        const TileDesc h = sdesc[li];
        const bool dense = h.comm >= 0;
        // this thread's node inputs, loaded while the gather warps work
        const int r = gt;
        const int64_t m = h.first + r;
        const bool live = r < h.count;
        double theta_m = 0.0, wdt64_m = 0.0;
        T acc_m = T(0), wdt_m = T(0), omega_m = T(0);
        int32_t perm_m = 0;
        if (live) {
            if (MODE == kRhs) {
                omega_m = a.omega[m];
                perm_m = a.perm[m];
            } else {
                theta_m = a.theta[m];
                if (!a.first_stage) acc_m = a.acc[m];
                if (MODE == kStage) wdt_m = a.wdt_next[m];
                else wdt64_m = a.wdt64[m];
            }
        }
        bool fail = false;
        if (gt == 0) {
            fail = !mbar_wait_bounded(&swfull_bar[b], u & 1, kWaitLimitNs);
            if (!fail && !zwaited) fail = !mbar_wait_bounded(&zready_bar, 0, kWaitLimitNs);
            if (fail) {
                atomicExch(a.err_flag, 1);
                s_cons_abort = 1;
            }
        }
        if (gsync_or(fail)) break;
        zwaited = true;
        const C *cph = pbuf + (size_t)h.pbuf * P * a.ph_region + h.shift;
        const C *sWm = sWm_of(b), *sWi = sWi_of(b);
        T sre[P], sim[P];
#pragma unroll
        for (int kk = 0; kk < P; ++kk) sre[kk] = sim[kk] = T(0);
        if (live) {
            const uint32_t vt = sWv[b * kConsumers + r];
            T coup = T(0);
            C uk[P];
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
                const C uu = dense ? cph[kk * a.ph_region + (int)(m - h.lo)] : __ldg(a.ph_in + kk * stride + m);
                uk[kk] = uu;
                const C wi = sWi[kk * kConsumers + r];
                T zr = wi.x, zi = wi.y;
                for (int c = (int)(vt & 0xffffu); c < (int)(vt & 0xffffu) + (int)(vt >> 16); ++c) {
                    const C wm = sWm[kk * kMaxChunks + c];
                    zr += wm.x;
                    zi += wm.y;
                }
                if (dense) {
                    // (E1.2) dense term: the whole block minus its diagonal (a_mm = 0)
                    zr += zrun[(size_t)h.run * P + kk].x - uu.x;
                    zi += zrun[(size_t)h.run * P + kk].y - uu.y;
                }
                // W conj(u_m): real part -> cosine harmonics, imaginary part -> sine
                const T re = zr * uu.x + zi * uu.y;
                const T im = zi * uu.x - zr * uu.y;
                coup += a.d_sin[kk] * im + a.d_cos[kk] * re;
            }
            coup *= a.tile_kn ? a.tile_kn[i] : a.k_over_n;
            if (P >= 2 && dense && a.k2_over_n2 != T(0)) {
                const C z1 = zrun[(size_t)h.run * P], z2 = zrun[(size_t)h.run * P + (P >= 2 ? 1 : 0)];
                coup += a.k2_over_n2 * triadic_from_moments<T>(z1.x, z1.y, z2.x, z2.y, uk[0].x, uk[0].y,
                                                               uk[P >= 2 ? 1 : 0].x, uk[P >= 2 ? 1 : 0].y);
            }
            if (MODE == kRhs) {
                a.rhs_out[perm_m] = (double)omega_m + (double)coup;
            } else {
                const T accv = acc_m + a.b_s * coup;
                T y;
                if (MODE == kStage) {
                    a.acc[m] = accv;
                    y = (T)theta_m + wdt_m + a.c_next_dt * coup;
                } else {
                    // FP64 time accumulation: theta += dt omega + dt sum_s b_s C_s
                    const double th = wrap_pi(theta_m + wdt64_m + a.dt * (double)accv);
                    a.theta[m] = th;
                    y = (T)th;
                }
                C uo[P];
                phasors<T, P>(y, uo);
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
                    a.ph_out[kk * stride + m] = uo[kk];
                    sre[kk] = uo[kk].x;
                    sim[kk] = uo[kk].y;
                }
            }
        }
        if (MODE != kRhs) {
#pragma unroll
            for (int kk = 0; kk < P; ++kk) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    sre[kk] += __shfl_xor_sync(0xffffffffu, sre[kk], o);
                    sim[kk] += __shfl_xor_sync(0xffffffffu, sim[kk], o);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int kk = 0; kk < P; ++kk) {
                    red[gw][2 * kk] = (double)sre[kk];
                    red[gw][2 * kk + 1] = (double)sim[kk];
                }
            }
        }
        gsync();                                             // node phase of tile i done
        if (lane == 0) mbar_arrive(&swempty_bar[b]);         // its sums are consumed
        if (MODE != kRhs && gt < 2 * P) {
            double sum = 0.0;
            for (int w = 0; w < kConsumerWarps; ++w) sum += red[w][gt];
            a.part_out[(size_t)i * P * 2 + gt] = sum;
        }
        // release every run before the run of the next tile
        {
            const int ni = i + 1;
            release_through((!dense || ni >= te || sdesc[ni - tb].comm < 0) ? nruns - 1 : sdesc[ni - tb].run - 1);
        }
    }
    release_through(nruns - 1);
}

// Direct method: every CSR neighbour gathered from global memory, `group`
// threads per row over 16-byte index vectors, then Phase B (no dense term).
template <typename T, int P, int MODE>
__global__ void __launch_bounds__(kThreads) direct_stage_kernel(const StageParams<T> a) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[kWarps][2 * P];
    const int t = blockIdx.x;
    const int first = a.tile_first[t];
    const int count = a.tile_count[t];
    const int64_t stride = a.ph_stride;
    C *sW = reinterpret_cast<C *>(smem_raw);            // [P][tile_nodes]
    const int G = a.group;
    const int lane = threadIdx.x & (G - 1);
    const int grp = threadIdx.x / G;
    const int ngrp = kThreads / G;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    for (int r = grp; r < count; r += ngrp) {
        const int64_t m = first + r;
        T wre[P], wim[P];
#pragma unroll
        for (int k = 0; k < P; ++k) wre[k] = wim[k] = T(0);
        const int4 *sv = reinterpret_cast<const int4 *>(a.sp_col + a.sp_rowptr[m]);
        const int nv = (int)((a.sp_rowptr[m + 1] - a.sp_rowptr[m]) >> 2);
#pragma unroll 2
        for (int v = lane; v < nv; v += G) {
            const int4 q = __ldg(sv + v);
            const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
#pragma unroll
                for (int k = 0; k < P; ++k) {
                    const C u = __ldg(a.ph_in + k * stride + l4[h]);
                    wre[k] += u.x;
                    wim[k] += u.y;
                }
            }
        }
        for (int o = G >> 1; o > 0; o >>= 1) {
#pragma unroll
            for (int k = 0; k < P; ++k) {
                wre[k] += __shfl_xor_sync(gmask, wre[k], o);
                wim[k] += __shfl_xor_sync(gmask, wim[k], o);
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < P; ++k) sW[k * a.tile_nodes + r] = mk2(wre[k], wim[k]);
        }
    }
    __syncthreads();
    finalize_tile<T, P, MODE>(a, t, first, count, false, (const C *)nullptr, sW, red,
                              [&](int k, int64_t m) { return __ldg(a.ph_in + k * stride + m); });
}

// Phasors (and tile sums) of a state given in original order; optionally
// stores the wrapped FP64 master in permuted order.
template <typename T, int P>
__global__ void __launch_bounds__(kThreads)
phasor_kernel(int64_t n, int64_t stride, const int32_t *perm, const int32_t *tile_first,
              const int32_t *tile_count, const double *x, double *theta, typename Vec2<T>::type *ph_out,
              double *part_out) {
    using C = typename Vec2<T>::type;
    __shared__ double red[kWarps][2 * P];
    const int t = blockIdx.x;
    const int first = tile_first[t], count = tile_count[t];
    T sre[P], sim[P];
#pragma unroll
    for (int k = 0; k < P; ++k) sre[k] = sim[k] = T(0);
    for (int r = threadIdx.x; r < count; r += kThreads) {
        const int64_t m = first + r;
        const double y = wrap_pi(x[perm[m]]);
        if (theta) theta[m] = y;
        C u[P];
        phasors<T, P>((T)y, u);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            ph_out[k * stride + m] = u[k];
            sre[k] += u[k].x;
            sim[k] += u[k].y;
        }
    }
    block_tile_sum<T, P>(sre, sim, red, part_out + (size_t)t * P * 2);
}

// Per-node constants of one time step: wrap(dt omega / 2), wrap(dt omega).
template <typename T>
__global__ void omega_constants_kernel(int64_t n, const T *omega, double dt, T *wh, T *wf, double *wf64) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const double w = (double)omega[m];
        const double h = wrap_pi(0.5 * dt * w), f = wrap_pi(dt * w);
        wh[m] = (T)h;
        wf[m] = (T)f;
        wf64[m] = f;
    }
}

// Order parameter of every instance, r_i = |sum over the instance's tiles of
// the first-harmonic tile sums| / N_i (eq. KuramotoFirstOP), written to
// r_base[c * B + i] with c = *counter, which is then incremented: the same
// launch, captured once in a CUDA graph, fills consecutive rows.  One block;
// warp w handles instances w, w + 32, ...
template <int P>
__global__ void __launch_bounds__(1024) order_parameters_kernel(int64_t B, const int32_t *inst_tiles,
                                                                const int64_t *inst_off, const double *part,
                                                                double *r_base, int64_t *counter) {
    __shared__ int64_t row;
    if (threadIdx.x == 0) row = *counter;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t i = warp; i < B; i += nw) {
        double re = 0.0, im = 0.0;
        for (int rng = 0; rng < 2; ++rng)
            for (int t = inst_tiles[4 * i + 2 * rng] + lane; t < inst_tiles[4 * i + 2 * rng + 1]; t += 32) {
                re += part[(int64_t)t * P * 2];
                im += part[(int64_t)t * P * 2 + 1];
            }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) r_base[row * B + i] = sqrt(re * re + im * im) / (double)(inst_off[i + 1] - inst_off[i]);
    }
    __syncthreads();
    if (threadIdx.x == 0) *counter = row + 1;
}

// r = |sum over all tiles of the first-harmonic tile sums| / N, written to
// r_base[*counter], then ++*counter.
template <int P>
__global__ void order_parameter_kernel(int64_t n, int64_t tiles, const double *part, double *r_base,
                                       int64_t *counter) {
    __shared__ double sre[kThreads], sim[kThreads];
    double re = 0.0, im = 0.0;
    for (int64_t t = threadIdx.x; t < tiles; t += kThreads) {
        re += part[t * P * 2];
        im += part[t * P * 2 + 1];
    }
    sre[threadIdx.x] = re;
    sim[threadIdx.x] = im;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sre[threadIdx.x] += sre[threadIdx.x + s];
            sim[threadIdx.x] += sim[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t row = *counter;
        r_base[row] = sqrt(sre[0] * sre[0] + sim[0] * sim[0]) / (double)n;
        *counter = row + 1;
    }
}

__global__ void scatter_master_kernel(int64_t n, const int32_t *perm, const double *theta, double *x) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x)
        x[perm[m]] = theta[m];
}

// Direct evaluation of the triadic term (higher-order model): for node m of
// community c, the plain double sum over ordered pairs of distinct other
// members, S_m = sum_{j != m} sum_{k != m, j} u_j u_k, then
// tri_m = (K2/N^2) Im(S_m conj(u_m)^2).  O(lambda^2) per node.  One block per
// tile; the community's phasors are staged in shared memory; each inner sum
// over k is accumulated in T, the sum over j in FP64.
template <typename T>
__global__ void __launch_bounds__(kThreads)
triadic_direct_kernel(const int32_t *tile_comm, const int32_t *tile_first, const int32_t *tile_count,
                      const int64_t *off, const typename Vec2<T>::type *u, T k2_over_n2, T *tri) {
    using C = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *cu = reinterpret_cast<C *>(smem_raw);
    const int t = blockIdx.x;
    const int comm = tile_comm[t], first = tile_first[t], count = tile_count[t];
    if (comm < 0) {
        for (int r = threadIdx.x; r < count; r += kThreads) tri[first + r] = T(0);
        return;
    }
    const int64_t lo = off[comm];
    const int lam = (int)(off[comm + 1] - lo);
    for (int i = threadIdx.x; i < lam; i += kThreads) cu[i] = u[lo + i];
    __syncthreads();
    for (int r = threadIdx.x; r < count; r += kThreads) {
        const int mloc = (int)(first + r - lo);
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < lam; ++j) {
            if (j == mloc) continue;
            T ir = T(0), ii = T(0);
            for (int k = 0; k < lam; ++k) {
                if (k == mloc || k == j) continue;
                ir += cu[k].x;
                ii += cu[k].y;
            }
            // u_j times the sum of u_k
            sr += (double)(cu[j].x * ir - cu[j].y * ii);
            si += (double)(cu[j].x * ii + cu[j].y * ir);
        }
        const C um = cu[mloc];
        const T c2r = um.x * um.x - um.y * um.y, c2i = T(2) * um.x * um.y;   // u_m^2
        // Im(S conj(u_m^2)) = si c2r - sr c2i
        tri[first + r] = k2_over_n2 * (T)(si * (double)c2r - sr * (double)c2i);
    }
}

template <typename T>
StageParams<T> base_params(cia_plan *pl, int method) {
    StageParams<T> a{};
    a.n = pl->n;
    a.ph_stride = pl->ph_stride;
    a.group = pl->group_size_direct;
    a.tile_nodes = pl->tile_nodes;
    for (int k = 0; k < CIA_MAX_HARMONICS; ++k) {
        a.d_sin[k] = (T)pl->d_sin[k];
        a.d_cos[k] = (T)pl->d_cos[k];
    }
    a.k_over_n = (T)(pl->K / (double)pl->n);
    a.tile_kn = (const T *)pl->d.tile_kn;
    a.tile_order = pl->d.tile_order;
    a.k2_over_n2 = (T)(pl->K2 / ((double)pl->n * (double)pl->n));
    a.tri = (method == Method::DIRECT && pl->triadic) ? (const T *)pl->d.tri : nullptr;
    a.off = pl->d.off;
    a.tile_comm = pl->d.tile_comm;
    a.tile_first = pl->d.tile_first;
    a.tile_count = pl->d.tile_count;
    a.comm_tile_begin = pl->d.comm_tile_begin;
    a.tile_desc = pl->d.tile_desc;
    a.blob = pl->d.blob;
    a.sp_rowptr = pl->d.full_rowptr;
    a.sp_col = pl->d.full_col;
    a.omega = (const T *)pl->d.omega;
    a.perm = pl->d.perm;
    a.acc = (T *)pl->d.acc;
    a.theta = pl->d.theta;
    a.wdt64 = pl->d.wdt_full64;
    a.n_tiles = pl->n_tiles;
    a.comm_done = pl->d.comm_done;
    a.tile_buf = (int)((pl->max_tile_buf + 127) & ~(int64_t)127);
    a.ph_region = (int)tma_ph_region(pl);
    a.idx_cap = (int)((pl->max_tile_idx_bytes + 15) & ~(int64_t)15);
    a.err_flag = pl->d.err_flag;
    a.stages = pl->ring_stages;
    a.max_cta_tiles = (int)pl->max_cta_tiles;
    a.max_cta_runs = (int)pl->max_cta_runs;
    a.cta_tile_begin = pl->d.cta_tile_begin;
    a.cta_runs = pl->d.cta_runs;
    (void)method;
    return a;
}

template <typename K>
cudaError_t launch_kernel(K kernel, const cia_plan *pl, int64_t blocks, size_t smem, const void *params,
                          cudaStream_t s) {
    cudaError_t e = ensure_dynamic_smem((const void *)kernel, pl->device, smem);
    if (e != cudaSuccess) return e;
    void *args[] = {const_cast<void *>(params)};
    return cudaLaunchKernel((const void *)kernel, dim3((unsigned)blocks), dim3(kThreads), args, smem, s);
}

template <typename T, int P, int MODE>
cudaError_t launch_cia_t(const cia_plan *pl, const StageParams<T> &a, cudaStream_t s) {
    if (pl->staging == 3) {
        auto kernel = cia_pipeline_kernel<T, P, MODE>;
        const size_t smem = pipeline_smem_bytes(pl, pl->ring_stages);
        cudaError_t e = ensure_dynamic_smem((const void *)kernel, pl->device, smem);
        if (e != cudaSuccess) return e;
        void *args[] = {const_cast<StageParams<T> *>(&a)};
        return cudaLaunchKernel((const void *)kernel, dim3((unsigned)pl->n_ctas), dim3(kPipeThreads), args, smem, s);
    }
    if (pl->staging == 2)
        return launch_kernel(cia_window_kernel<T, P, MODE>, pl, pl->n_tiles, window_smem_bytes(pl), &a, s);
    if (pl->staging == 4) {
        auto kernel = cia_ring_kernel<T, P, MODE>;
        const size_t smem = (size_t)pl->ring_slots * (size_t)a.tile_buf;
        cudaError_t e = ensure_dynamic_smem((const void *)kernel, pl->device, smem);
        if (e != cudaSuccess) return e;
        StageParams<T> r = a;
        r.stages = pl->ring_slots;
        void *args[] = {&r};
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(pl->n_tiles, pl->n_sms));
        return cudaLaunchKernel((const void *)kernel, dim3((unsigned)grid), dim3(kRingThreads), args, smem, s);
    }
    return launch_kernel(cia_stage_kernel<T, P, MODE>, pl, pl->n_tiles, stage_smem_bytes(pl, Method::CIA), &a, s);
}

template <typename T, int P, int MODE>
cudaError_t launch_direct_t(const cia_plan *pl, const StageParams<T> &a, cudaStream_t s) {
    return launch_kernel(direct_stage_kernel<T, P, MODE>, pl, pl->n_tiles, stage_smem_bytes(pl, Method::DIRECT),
                         &a, s);
}

template <typename T, int MODE>
cudaError_t dispatch_stage(cia_plan *pl, int method, const StageParams<T> &a, cudaStream_t s) {
    const bool direct = method == Method::DIRECT;
    if (direct && pl->triadic) {
        // the direct method's triadic term, pair by pair, before the stage
        using C = typename Vec2<T>::type;
        auto kernel = triadic_direct_kernel<T>;
        const size_t smem = sizeof(C) * (size_t)std::max<int64_t>(1, pl->max_comm);
        cudaError_t e0 = ensure_dynamic_smem((const void *)kernel, pl->device, smem);
        if (e0 != cudaSuccess) return e0;
        kernel<<<(unsigned)pl->n_tiles, kThreads, smem, s>>>(pl->d.tile_comm, pl->d.tile_first, pl->d.tile_count,
                                                            pl->d.off, a.ph_in, a.k2_over_n2, (T *)pl->d.tri);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
#define CIA_CASE(P)                                                                   \
    case P:                                                                           \
        return direct ? launch_direct_t<T, P, MODE>(pl, a, s) : launch_cia_t<T, P, MODE>(pl, a, s);
    switch (pl->p) {
        CIA_CASE(1)
        CIA_CASE(2)
        CIA_CASE(3)
        CIA_CASE(4)
    }
#undef CIA_CASE
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t phasors_t(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    using C = typename Vec2<T>::type;
    double *theta = write_master ? pl->d.theta : nullptr;
    C *ph = (C *)pl->d.ph[slot];
    double *part = pl->d.part[slot];
    const unsigned g = (unsigned)pl->n_tiles;
    switch (pl->p) {
        case 1: phasor_kernel<T, 1><<<g, kThreads, 0, s>>>(pl->n, pl->ph_stride, pl->d.perm, pl->d.tile_first, pl->d.tile_count, x, theta, ph, part); break;
        case 2: phasor_kernel<T, 2><<<g, kThreads, 0, s>>>(pl->n, pl->ph_stride, pl->d.perm, pl->d.tile_first, pl->d.tile_count, x, theta, ph, part); break;
        case 3: phasor_kernel<T, 3><<<g, kThreads, 0, s>>>(pl->n, pl->ph_stride, pl->d.perm, pl->d.tile_first, pl->d.tile_count, x, theta, ph, part); break;
        case 4: phasor_kernel<T, 4><<<g, kThreads, 0, s>>>(pl->n, pl->ph_stride, pl->d.perm, pl->d.tile_first, pl->d.tile_count, x, theta, ph, part); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || pl->staging != 4 || pl->M == 0) return e;
    // the ring kernel reads the community observables, not the tile partials
    const unsigned blocks = (unsigned)((pl->M * 32 + 255) / 256);
    switch (pl->p) {
        case 1: community_sums_kernel<1><<<blocks, 256, 0, s>>>(pl->M, pl->d.comm_tile_begin, part, pl->d.zsum[slot], pl->d.comm_done); break;
        case 2: community_sums_kernel<2><<<blocks, 256, 0, s>>>(pl->M, pl->d.comm_tile_begin, part, pl->d.zsum[slot], pl->d.comm_done); break;
        case 3: community_sums_kernel<3><<<blocks, 256, 0, s>>>(pl->M, pl->d.comm_tile_begin, part, pl->d.zsum[slot], pl->d.comm_done); break;
        default: community_sums_kernel<4><<<blocks, 256, 0, s>>>(pl->M, pl->d.comm_tile_begin, part, pl->d.zsum[slot], pl->d.comm_done); break;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t rhs_t(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s) {
    using C = typename Vec2<T>::type;
    StageParams<T> a = base_params<T>(pl, method);
    a.ph_in = (const C *)pl->d.ph[slot];
    a.part_in = pl->d.part[slot];
    a.z_in = pl->d.zsum[slot];
    a.rhs_out = dxdt;
    return dispatch_stage<T, kRhs>(pl, method, a, s);
}

template <typename T>
cudaError_t stage_t(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s) {
    using C = typename Vec2<T>::type;
    // classical RK4: nodes c = (0, 1/2, 1/2, 1), weights b = (1/6, 1/3, 1/3, 1/6)
    static const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    static const double c_next[4] = {0.5, 0.5, 1.0, 0.0};
    StageParams<T> a = base_params<T>(pl, method);
    a.ph_in = (const C *)pl->d.ph[slot];
    a.ph_out = (C *)pl->d.ph[slot ^ 1];
    a.part_in = pl->d.part[slot];
    a.part_out = pl->d.part[slot ^ 1];
    a.z_in = pl->d.zsum[slot];
    a.z_out = pl->d.zsum[slot ^ 1];
    a.b_s = (T)b[stage - 1];
    a.c_next_dt = (T)(c_next[stage - 1] * dt);
    a.wdt_next = (const T *)(stage == 3 ? pl->d.wdt_full : pl->d.wdt_half);
    a.dt = dt;
    a.first_stage = stage == 1;
    return stage == 4 ? dispatch_stage<T, kFinal>(pl, method, a, s) : dispatch_stage<T, kStage>(pl, method, a, s);
}

}  // namespace

// Dynamic shared memory of the plain-load CIA kernel and of the direct
// kernel: the W sums of one tile.
size_t stage_smem_bytes(const cia_plan *pl, int method) {
    const size_t cb = (pl->precision == CIA_FP64 ? 16 : 8) * (size_t)pl->p;
    return method == Method::DIRECT ? cb * (size_t)pl->tile_nodes : cb * (size_t)(kMaxChunks + pl->tile_nodes);
}

// Dynamic shared memory of the window kernel: the community phasor window
// of every harmonic, chunk sums and inter sums.
size_t window_smem_bytes(const cia_plan *pl) {
    const size_t cb = (pl->precision == CIA_FP64 ? 16 : 8) * (size_t)pl->p;
    return cb * ((size_t)tma_ph_region(pl) + kMaxChunks + (size_t)pl->tile_nodes);
}

// Ring slots of the persistent ring kernel that fit the device's shared
// memory (each holds the largest tile's window and blob), at most
// kRingMaxSlots; the kernel needs two.
template <typename T, int P>
size_t ring_static_smem() {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, cia_ring_kernel<T, P, kStage>) != cudaSuccess) {
        cudaGetLastError();
        return sizeof(RingHeader<T, CIA_MAX_HARMONICS>) * kRingMaxSlots + 1024;
    }
    return fa.sharedSizeBytes;
}

int ring_slots_that_fit(const cia_plan *pl) {
    const size_t slot = (size_t)((pl->max_tile_buf + 127) & ~(int64_t)127);
    size_t stat = 0;
    switch (pl->p) {
        case 1: stat = pl->precision == CIA_FP64 ? ring_static_smem<double, 1>() : ring_static_smem<float, 1>(); break;
        case 2: stat = pl->precision == CIA_FP64 ? ring_static_smem<double, 2>() : ring_static_smem<float, 2>(); break;
        case 3: stat = pl->precision == CIA_FP64 ? ring_static_smem<double, 3>() : ring_static_smem<float, 3>(); break;
        default: stat = pl->precision == CIA_FP64 ? ring_static_smem<double, 4>() : ring_static_smem<float, 4>(); break;
    }
    if ((size_t)pl->smem_optin < stat + 1024 + 2 * slot) return 0;
    const size_t avail = (size_t)pl->smem_optin - stat - 1024;
    return (int)std::min<size_t>(kRingMaxSlots, slot ? avail / slot : kRingMaxSlots);
}

// Dynamic shared memory of the persistent ring kernel with its slots.
size_t stream_smem_bytes(const cia_plan *pl) {
    return (size_t)std::max(pl->ring_slots, 2) * (size_t)((pl->max_tile_buf + 127) & ~(int64_t)127);
}

// Bytes of the per-tile buffer of the persistent per-tile kernel for a tile
// of a community of lam nodes (lam = 0: free nodes) with a blob of the given
// size; the window rounding is the device's with the larger shift.
int64_t stream_tile_buf_bytes(const cia_plan *pl, int64_t lam, int64_t blob_bytes) {
    const int64_t cb = pl->precision == CIA_FP64 ? 16 : 8;
    const int64_t shift = pl->precision == CIA_FP64 ? 0 : 1;
    const int64_t wreg = lam > 0 ? ((shift + lam + 1 + kPadSlots) * cb + 15) & ~(int64_t)15 : 0;
    return (int64_t)pl->p * wreg + blob_bytes;
}

// Dynamic shared memory of the pipelined CIA kernel: a ring of tile buffers
// (64-byte header + index vectors), two community phasor windows, W sums.
size_t pipeline_smem_bytes(const cia_plan *pl, int stages) {
    const size_t cb = (pl->precision == CIA_FP64 ? 16 : 8) * (size_t)pl->p;
    const size_t idx_cap = (size_t)((pl->max_tile_idx_bytes + 15) & ~(int64_t)15);
    return (size_t)pl->max_cta_tiles * sizeof(TileDesc) +
           zrun_bytes(pl->max_cta_runs, 1, cb) + (size_t)stages * idx_cap +
           2 * cb * (size_t)tma_ph_region(pl) + 2 * cb * (size_t)(kMaxChunks + kConsumers) +
           2 * sizeof(uint32_t) * (size_t)kConsumers;
}

cudaError_t launch_phasors_from_x(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    return pl->precision == CIA_FP64 ? phasors_t<double>(pl, x, write_master, slot, s)
                                     : phasors_t<float>(pl, x, write_master, slot, s);
}

cudaError_t launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s) {
    return pl->precision == CIA_FP64 ? rhs_t<double>(pl, method, slot, dxdt, s)
                                     : rhs_t<float>(pl, method, slot, dxdt, s);
}

cudaError_t launch_rk4_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s) {
    return pl->precision == CIA_FP64 ? stage_t<double>(pl, method, stage, slot, dt, s)
                                     : stage_t<float>(pl, method, stage, slot, dt, s);
}

cudaError_t launch_omega_constants(cia_plan *pl, double dt, cudaStream_t s) {
    const unsigned blocks = (unsigned)std::min<int64_t>((pl->n + 255) / 256, 152 * 8);
    if (pl->precision == CIA_FP64)
        omega_constants_kernel<double><<<blocks, 256, 0, s>>>(pl->n, (const double *)pl->d.omega, dt,
                                                             (double *)pl->d.wdt_half, (double *)pl->d.wdt_full,
                                                             pl->d.wdt_full64);
    else
        omega_constants_kernel<float><<<blocks, 256, 0, s>>>(pl->n, (const float *)pl->d.omega, dt,
                                                            (float *)pl->d.wdt_half, (float *)pl->d.wdt_full,
                                                            pl->d.wdt_full64);
    return cudaGetLastError();
}

cudaError_t launch_order_parameters(cia_plan *pl, int slot, double *r_base, cudaStream_t s) {
    const double *part = pl->d.part[slot];
    int64_t *ctr = pl->d.r_counter;
    if (pl->B > 1) {
        const int64_t *io = pl->d.inst_off;
        const int32_t *it = pl->d.inst_tiles;
        switch (pl->p) {
            case 1: order_parameters_kernel<1><<<1, 1024, 0, s>>>(pl->B, it, io, part, r_base, ctr); break;
            case 2: order_parameters_kernel<2><<<1, 1024, 0, s>>>(pl->B, it, io, part, r_base, ctr); break;
            case 3: order_parameters_kernel<3><<<1, 1024, 0, s>>>(pl->B, it, io, part, r_base, ctr); break;
            default: order_parameters_kernel<4><<<1, 1024, 0, s>>>(pl->B, it, io, part, r_base, ctr); break;
        }
        return cudaGetLastError();
    }
    switch (pl->p) {
        case 1: order_parameter_kernel<1><<<1, kThreads, 0, s>>>(pl->n, pl->n_tiles, part, r_base, ctr); break;
        case 2: order_parameter_kernel<2><<<1, kThreads, 0, s>>>(pl->n, pl->n_tiles, part, r_base, ctr); break;
        case 3: order_parameter_kernel<3><<<1, kThreads, 0, s>>>(pl->n, pl->n_tiles, part, r_base, ctr); break;
        default: order_parameter_kernel<4><<<1, kThreads, 0, s>>>(pl->n, pl->n_tiles, part, r_base, ctr); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_master(cia_plan *pl, double *x, cudaStream_t s) {
    const unsigned blocks = (unsigned)std::min<int64_t>((pl->n + 255) / 256, 152 * 8);
    scatter_master_kernel<<<blocks, 256, 0, s>>>(pl->n, pl->d.perm, pl->d.theta, x);
    return cudaGetLastError();
}

}  // namespace cia
