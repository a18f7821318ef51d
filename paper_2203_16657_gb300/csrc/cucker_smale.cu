// Device kernels of the Cucker--Smale model (App. A.6, eq. Cucker_Smale with
// n = 2): per node m the state is (s_m, v_m) in R^2 x R^2 and
//   s_m' = v_m,   v_m' = (1/N) sum_l a_ml eta(||s_l - s_m||^2) (v_l - v_m),
//   eta(y) = K (sigma^2 + y)^-beta.
//
// CIA with a separable basis eta(||s_l - s_m||^2) ~ phi(s_l) . phi(s_m)
// (step P2; phi is the learned feature map of mlp_tile.cuh, evaluated on
// positions relative to the community centroid, a shift that leaves every
// difference s_l - s_m unchanged):
//   (E1.1) U_c = (1/N) sum_{l in c} phi(l),  H_c = (1/N) sum_{l in c} phi(l) v_l
//          (eq. Cucker_Smale_orderParams, per community, both components of v)
//   (E1.2) dense_m = sum_r phi_r(m) (H_cr - U_cr v_m)   (eq. Cucker_Smale_fast_RHS)
//   (E2)   sparse_m = (1/N) [sum_{l in inter(m)} - sum_{l in miss(m)}]
//                     eta(||s_l - s_m||^2) (v_l - v_m)   with the exact eta.
// The diagonal l = m of the dense block contributes phi(m).phi(m) (v_m - v_m)
// = 0, so it needs no correction.
//
// CTAs of 256 threads walk tiles of at most 128 nodes of one community:
//  - the feature launch (kLoad) stages the community's positions to get its
//    centroid c and evaluates phi(s - c) on the tile (layer 2 on the tensor
//    cores), storing the BF16 features, the tile's partial sums of phi,
//    phi v_x, phi v_y, and c as the community's shift;
//  - the stage launch (0) reduces the community's tile partial sums into
//    U_c, H_c and stages the community's state in shared memory, (A) sums the
//    sparse links (missing links from shared memory, inter-community links
//    from global memory) in the sliced-ELL layout of the plan, (B) adds the
//    dense term from each node's stored features and applies the RK4 stage
//    update and, in stages 1-3, (C) evaluates the features and moment partial
//    sums of the next stage state it has just written, with the recorded
//    shift.
// One RK4 step is thus four stage launches and one feature launch (after
// stage 4, for the new state).  All four stages of a step evaluate phi with
// the centroid of the step's initial state as the shift; any shift common to
// a community leaves every difference s_l - s_m unchanged, and this one moves
// the inputs by O(dt |v|) from the stage state's own centroid.  The right-hand
// side at a state that starts a step (cia_rhs, the sampled check, the state
// after a resume) uses that state's own centroid.  The features are rounded
// to BF16 once and the same values enter the moments and the dense term, so
// the approximate pair weight is exactly symmetric.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "cia_internal.h"
#include "mlp_tile.cuh"

namespace cia {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTileMax = 128;          // rows of a tile = MMA M
constexpr int kMaxChunks = 512;        // missing-list chunks per tile (plan limit)
constexpr int kPart = 3 * CIA_BASIS_RANK;   // U, H_x, H_y per tile
constexpr int kRank = CIA_BASIS_RANK;
constexpr int kFw = kRank / 2;               // 32-bit words (BF16 pairs) of a feature-tile row
constexpr size_t kFeatTileBytes = (size_t)kTileMax * kFw * 4;   // phase C feature tile
constexpr size_t kRedBytes = 4 * (size_t)3 * kRank * 4;        // phase C moment partials [4][kPart]

enum CsMode { kRhs = 0, kStage = 1, kFinal = 2, kLoad = 3 };

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr size_t kWeightsBytes = align_up(sizeof(mlp::Weights), 1024);
static_assert(sizeof(mlp::Weights) % 16 == 0, "the weights travel by one bulk copy");

struct CsParams {
    int64_t n;
    int n_tiles;
    int group;                 // threads per row of the direct method
    float inv_n;               // 1 / N
    double inv_n64;
    float K, sigma2, neg_beta; // eta(y) = K (sigma2 + y)^neg_beta
    const TileDesc *tile_desc;
    const int32_t *tile_order;
    const unsigned char *blob;
    const int32_t *comm_tile_begin;
    const int64_t *full_rowptr;
    const int32_t *full_col;
    const float4 *y_in;        // [n] stage state (s_x, s_y, v_x, v_y), permuted
    float4 *y_out;             // [n] next stage state
    const double *part_in;     // [tiles][kPart] moment partial sums of y_in's features
    float2 *shift;             // [M] shift of phi's input: written by the feature launch,
                               // read by the fused stage launches of the same RK4 step
    double *part_out;          // [tiles][kPart] of y_out's features
    __nv_bfloat16 *feat;       // [n][kRank] features of y_in on entry, of y_out on exit
    const float *params;       // basis parameters (FP32 master)
    const mlp::Weights *wimage;  // the same in their shared-memory layout (W2 in BF16), copied by TMA
    float4 *acc;               // [n] sum_s b_s k_s
    double *master;            // [n][4] FP64 master state
    const int32_t *perm;
    double *rhs_out;           // kRhs: [N][4] in original order
    float c_next_dt, b_s;
    double dt;
    int first_stage;
    uint32_t win_bytes;        // shared-memory bytes of the community state window
    int *err_flag;
};

// eta(||s_l - s_m||^2) (v_l - v_m) added to (sx, sy).
__device__ __forceinline__ void pair_term(const CsParams &a, float4 own, float4 y, float &sx, float &sy) {
    const float dx = y.x - own.x, dy = y.y - own.y;
    const float w = a.K * __powf(fmaf(dx, dx, fmaf(dy, dy, a.sigma2)), a.neg_beta);
    sx = fmaf(w, y.z - own.z, sx);
    sy = fmaf(w, y.w - own.w, sy);
}

__device__ __forceinline__ float bf16_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// RK4 stage update of node m from its derivative k (all modes but kLoad);
// returns the next stage state.
template <int MODE>
__device__ __forceinline__ float4 rk4_update(const CsParams &a, int64_t m, float4 own, float4 k) {
    if (MODE == kRhs) {
        double *o = a.rhs_out + 4 * (int64_t)a.perm[m];
        o[0] = k.x;
        o[1] = k.y;
        o[2] = k.z;
        o[3] = k.w;
        return own;
    }
    float4 s = a.first_stage ? make_float4(0.f, 0.f, 0.f, 0.f) : a.acc[m];
    s.x = fmaf(a.b_s, k.x, s.x);
    s.y = fmaf(a.b_s, k.y, s.y);
    s.z = fmaf(a.b_s, k.z, s.z);
    s.w = fmaf(a.b_s, k.w, s.w);
    double2 *mp = reinterpret_cast<double2 *>(a.master + 4 * m);
    double2 m0 = mp[0], m1 = mp[1];
    float4 y;
    if (MODE == kStage) {
        a.acc[m] = s;
        y = make_float4((float)m0.x + a.c_next_dt * k.x, (float)m0.y + a.c_next_dt * k.y,
                        (float)m1.x + a.c_next_dt * k.z, (float)m1.y + a.c_next_dt * k.w);
    } else {
        // FP64 time accumulation: x += dt sum_s b_s k_s
        m0.x += a.dt * (double)s.x;
        m0.y += a.dt * (double)s.y;
        m1.x += a.dt * (double)s.z;
        m1.y += a.dt * (double)s.w;
        mp[0] = m0;
        mp[1] = m1;
        y = make_float4((float)m0.x, (float)m0.y, (float)m1.x, (float)m1.y);
    }
    a.y_out[m] = y;
    return y;
}

#ifndef CIA_CS_FUSED
#define CIA_CS_FUSED 1        // stages 1-3 evaluate the next state's features in their epilogue
#endif
#ifndef CIA_CS_MIN_BLOCKS
#define CIA_CS_MIN_BLOCKS 4   // resident CTAs per SM the stage launches' registers are sized for
#endif

template <int MODE>
__global__ void __launch_bounds__(kThreads, CIA_CS_MIN_BLOCKS) cs_stage_kernel(const CsParams a) {
    constexpr bool kFused = CIA_CS_FUSED && MODE == kStage;   // features of the next stage state
    constexpr bool kFeatures = MODE == kLoad || kFused;      // phi and its moment partial sums
    constexpr bool kSums = MODE != kLoad;                    // the right-hand side and the stage update
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint64_t wbar;                  // the weights' bulk copy
    __shared__ uint32_t tslot;
    __shared__ float4 yrow[kTileMax];          // stage state of the tile's rows, then the next one
    __shared__ float mom[kPart];               // U_c, H_cx, H_cy (with the 1/N)
    __shared__ float cred[kWarps][2];
    __shared__ float2 cen;
    __shared__ int s_next;                     // next slice of the tile to take

    mlp::Weights &w = *reinterpret_cast<mlp::Weights *>(smem);
    unsigned char *region = smem + (kFeatures ? kWeightsBytes : 0);
    float4 *win = reinterpret_cast<float4 *>(region);                  // community window (phases 0-B)
    float2 *sWm = reinterpret_cast<float2 *>(region + a.win_bytes);     // missing-chunk sums
    float2 *sWi = sWm + kMaxChunks;                                    // inter sums per row
    uint16_t *chunk_row = reinterpret_cast<uint16_t *>(sWi + kTileMax);
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(region);      // phase C: layer-2 operand
    // phase C: the tile's BF16 features, row r's word j (features 2j, 2j + 1)
    // at r * kFw + (j ^ (r & 31)), so that a warp's rows or a warp's
    // features hit distinct banks; then the moment partials
    uint32_t *F = reinterpret_cast<uint32_t *>(region);
    float(*red)[kPart] = reinterpret_cast<float(*)[kPart]>(region + kFeatTileBytes);

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, r = t & 127, h = t >> 7;
    uint32_t tmem = 0;
    if (kFeatures) {
        if (warp == 0) umma::tmem_alloc(&tslot, 64);
        if (t == 0) {
            mbar_init(&bar, 1);
            // the weights arrive by one bulk copy while the tile's sums run
            mbar_init(&wbar, 1);
            mbar_arrive_expect_tx(&wbar, (uint32_t)sizeof(mlp::Weights));
            bulk_g2s(&w, a.wimage, (uint32_t)sizeof(mlp::Weights), &wbar);
        }
        umma::fence_before_sync();
    }
    __syncthreads();
    if (kFeatures) {
        umma::fence_after_sync();
        tmem = tslot;
    }
    uint32_t phase = 0;
    bool ok = true, have_w = false;

    for (int k = blockIdx.x; k < a.n_tiles; k += gridDim.x) {
        const int tile = a.tile_order ? a.tile_order[k] : k;   // costliest tiles first
        const TileDesc d = a.tile_desc[tile];
        const bool comm = d.comm >= 0;
        if (MODE == kLoad && !comm) continue;   // nodes without a community have no dense term
        const int lam = comm ? (int)d.lam : 0;
        const int count = d.count;
        const unsigned char *b = a.blob + d.blob_off;
        const uint32_t *vtab = reinterpret_cast<const uint32_t *>(b + d.vtab_off);
        // (0) community window, own rows, moments, chunk -> row table
        for (int i = t; i < lam; i += kThreads) win[i] = a.y_in[d.lo + i];
        if (t < count) yrow[t] = a.y_in[d.first + t];
        if (t == 0) s_next = kWarps;   // the previous tile's slices ended at its last barrier
        if (kFused && comm && t == 0) cen = a.shift[d.comm];
        if (kSums) {
            if (comm && t < kPart) {
                double s = 0.0;
                for (int u = a.comm_tile_begin[d.comm]; u < a.comm_tile_begin[d.comm + 1]; ++u)
                    s += a.part_in[(int64_t)u * kPart + t];
                mom[t] = (float)(s * a.inv_n64);
            }
            if (t < count) {
                const uint32_t vt = __ldg(vtab + t);
                for (uint32_t c = vt & 0xffffu; c < (vt & 0xffffu) + (vt >> 16); ++c) chunk_row[c] = (uint16_t)t;
            }
        }
        __syncthreads();
        if (MODE == kLoad && comm) {
            // centroid of the community's positions in this state (the shift
            // of phi's input); a fixed reduction order, identical in every
            // tile of the community
            float sx = 0.f, sy = 0.f;
            for (int i = t; i < lam; i += kThreads) {
                sx += win[i].x;
                sy += win[i].y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
                sy += __shfl_xor_sync(0xffffffffu, sy, o);
            }
            if (lane == 0) {
                cred[warp][0] = sx;
                cred[warp][1] = sy;
            }
        }
        if (kSums) {
            // (A) sparse sums: warp per slice, lane per row (missing chunk and
            // inter row); slices are taken in order by whichever warp is free.
            // A slice's first inter vector, its gathers and its first two
            // missing vectors are issued before any is used, and each missing
            // vector is loaded two iterations ahead of its use
            const uint4 *sdesc = reinterpret_cast<const uint4 *>(b);
            const uint32_t *srows = reinterpret_cast<const uint32_t *>(b + 16 * d.nsl);
            const uint4 *mvec = reinterpret_cast<const uint4 *>(b + d.mvec_off);
            const int4 *ivec = reinterpret_cast<const int4 *>(b + d.ivec_off);
            for (int s = warp;;) {
                if (s >= d.nsl) break;
                const uint4 sd = __ldg(sdesc + s);
                const uint32_t rows = __ldg(srows + s * 32 + lane);
                const uint32_t mrow = rows & 0xffffu, irow = rows >> 16;
                const int4 *iv = ivec + sd.z + lane;
                const uint4 *mv = mvec + sd.x + lane;
                const int4 none = make_int4(a.n, a.n, a.n, a.n);
                int4 qi = sd.w > 0 ? __ldg(iv) : none;
                uint4 q0 = make_uint4(0u, 0u, 0u, 0u), q1 = q0;
                if (sd.y > 0) q0 = __ldg(mv);
                if (sd.y > 1) q1 = __ldg(mv + 32);
                float4 g[4];
                {
                    const int l4[4] = {qi.x, qi.y, qi.z, qi.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) g[e] = l4[e] < a.n ? __ldg(a.y_in + l4[e]) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                float mx = 0.f, my = 0.f, ix = 0.f, iy = 0.f;
                {
                    const float4 own = yrow[mrow != 0xffffu ? chunk_row[mrow] : 0];
                    for (uint32_t j = 0; j < sd.y; ++j) {
                        const uint4 q = q0;
                        q0 = q1;
                        if (j + 2 < sd.y) q1 = __ldg(mv + 32 * (j + 2));
                        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int l0 = (int)(w4[e] & 0xffffu), l1 = (int)(w4[e] >> 16);
                            if (l0 < lam) pair_term(a, own, win[l0], mx, my);
                            if (l1 < lam) pair_term(a, own, win[l1], mx, my);
                        }
                    }
                }
                {
                    const float4 own = yrow[irow != 0xffffu ? irow : 0];
                    for (uint32_t j = 0; j < sd.w; ++j) {
                        if (j > 0) {
                            qi = __ldg(iv + 32 * j);
                            const int l4[4] = {qi.x, qi.y, qi.z, qi.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                g[e] = l4[e] < a.n ? __ldg(a.y_in + l4[e]) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                        const int l4[4] = {qi.x, qi.y, qi.z, qi.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (l4[e] < a.n) pair_term(a, own, g[e], ix, iy);
                    }
                }
                if (mrow != 0xffffu) sWm[mrow] = make_float2(mx, my);
                if (irow != 0xffffu) sWi[irow] = make_float2(ix, iy);
                int nx = 0;
                if (lane == 0) nx = atomicAdd(&s_next, 1);
                s = __shfl_sync(0xffffffffu, nx, 0);
            }
            __syncthreads();
            // (B) dense term, derivative, RK4 update: thread per row
            if (t < count) {
                const int64_t m = d.first + t;
                const float4 own = yrow[t];
                float sx = sWi[t].x, sy = sWi[t].y;
                const uint32_t vt = __ldg(vtab + t);
                for (uint32_t c = vt & 0xffffu; c < (vt & 0xffffu) + (vt >> 16); ++c) {
                    sx -= sWm[c].x;
                    sy -= sWm[c].y;
                }
                float ax = a.inv_n * sx, ay = a.inv_n * sy;
                if (comm) {
                    const uint4 *fp = reinterpret_cast<const uint4 *>(a.feat + m * kRank);
                    float dx = 0.f, dy = 0.f;
#pragma unroll
                    for (int q = 0; q < kRank / 8; ++q) {
                        const uint4 v = fp[q];
                        const uint32_t u4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int rr = 8 * q + 2 * e;
                            const float f0 = bf16_lo(u4[e]), f1 = bf16_hi(u4[e]);
                            dx = fmaf(f0, fmaf(-mom[rr], own.z, mom[kRank + rr]), dx);
                            dy = fmaf(f0, fmaf(-mom[rr], own.w, mom[2 * kRank + rr]), dy);
                            dx = fmaf(f1, fmaf(-mom[rr + 1], own.z, mom[kRank + rr + 1]), dx);
                            dy = fmaf(f1, fmaf(-mom[rr + 1], own.w, mom[2 * kRank + rr + 1]), dy);
                        }
                    }
                    ax += dx;
                    ay += dy;
                }
                yrow[t] = rk4_update<MODE>(a, m, own, make_float4(own.z, own.w, ax, ay));
            }
        }
        __syncthreads();
        if (kFeatures && comm) {
            if (MODE == kLoad && t == 0) {
                float sx = 0.f, sy = 0.f;
                for (int i = 0; i < kWarps; ++i) {
                    sx += cred[i][0];
                    sy += cred[i][1];
                }
                cen = make_float2(sx / (float)lam, sy / (float)lam);
                // the shift of the fused stages that follow, recorded by the
                // community's first tile (every tile computes the same value)
                if (tile == a.comm_tile_begin[d.comm]) a.shift[d.comm] = cen;
            }
            if (!have_w) {
                have_w = true;
                if (__syncthreads_or(!mbar_wait_bounded(&wbar, 0, kWaitLimitNs))) {
                    ok = false;
                    break;
                }
            }
            __syncthreads();
            // (C) features of this state (feature launch) or of the next
            // stage state (fused stage launch) and their tile partial sums
            const bool valid = r < count;
            const float4 yn = valid ? yrow[r] : make_float4(0.f, 0.f, 0.f, 0.f);
            mlp::hidden_to_smem(w, yn.x - cen.x, yn.y - cen.y, r, h, valid, A);
            umma::fence_smem_to_async();
            umma::fence_before_sync();
            __syncthreads();
            if (t == 0) mlp::issue_layer2(A, w, tmem, &bar);
            const bool got = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
            phase ^= 1u;
            umma::fence_after_sync();
            float f[32];
            mlp::load_features(tmem, w, h, f);
            uint32_t pk[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                __nv_bfloat162 v = __floats2bfloat162_rn(f[2 * e], f[2 * e + 1]);
                pk[e] = *reinterpret_cast<uint32_t *>(&v);
                F[r * kFw + ((16 * h + e) ^ (r & 31))] = pk[e];
            }
            if (valid) {
                uint4 *dst = reinterpret_cast<uint4 *>(a.feat + (d.first + r) * kRank + 32 * h);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
            }
            umma::fence_before_sync();
            __syncthreads();
            {
                const int fr = t & 63, q4 = t >> 6;
                float su = 0.f, hx = 0.f, hy = 0.f;
                const int i1 = min(32 * q4 + 32, count);
                for (int i = 32 * q4; i < i1; ++i) {
                    const uint32_t wv = F[i * kFw + ((fr >> 1) ^ (i & 31))];
                    const float v = (fr & 1) ? bf16_hi(wv) : bf16_lo(wv);
                    su += v;
                    hx = fmaf(v, yrow[i].z, hx);
                    hy = fmaf(v, yrow[i].w, hy);
                }
                red[q4][fr] = su;
                red[q4][kRank + fr] = hx;
                red[q4][2 * kRank + fr] = hy;
            }
            __syncthreads();
            if (t < kPart)
                a.part_out[(int64_t)tile * kPart + t] =
                    ((double)red[0][t] + (double)red[1][t]) + ((double)red[2][t] + (double)red[3][t]);
        }
        __syncthreads();
    }
    if (kFeatures) {
        if (!ok) {
            if (t == 0) atomicExch(a.err_flag, 1);
            mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        }
        // the weights' copy must have landed before the CTA's shared memory is released
        if (!have_w || !ok) mbar_wait_bounded(&wbar, 0, kWaitLimitNs);
        umma::fence_before_sync();
        __syncthreads();
        if (warp == 0) umma::tmem_dealloc(tmem, 64);
    }
}

// Direct method: `group` threads per row sum the exact pair terms over the
// row's CSR neighbours (padded to 4-entry vectors with the sentinel n).
template <int MODE>
__global__ void __launch_bounds__(kThreads) cs_direct_kernel(const CsParams a) {
    const int G = a.group, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per_warp = 32 / G;
    const int4 *col4 = reinterpret_cast<const int4 *>(a.full_col);
    for (int64_t base = ((int64_t)blockIdx.x * kWarps + warp) * per_warp; base < a.n;
         base += (int64_t)gridDim.x * kWarps * per_warp) {
        const int64_t m = base + lane / G;
        const int gl = lane % G;
        const bool valid = m < a.n;
        float sx = 0.f, sy = 0.f;
        float4 own = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            own = a.y_in[m];
            const int64_t v0 = a.full_rowptr[m] / 4, v1 = a.full_rowptr[m + 1] / 4;
            for (int64_t v = v0 + gl; v < v1; v += G) {
                const int4 q = __ldg(col4 + v);
                const int l4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (l4[e] < a.n) pair_term(a, own, __ldg(a.y_in + l4[e]), sx, sy);
            }
        }
        for (int o = G / 2; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (valid && gl == 0)
            rk4_update<MODE>(a, m, own, make_float4(own.z, own.w, a.inv_n * sx, a.inv_n * sy));
    }
}

// x (original order, [N][4] doubles) -> FP64 master (optional) and FP32 state, permuted.
__global__ void cs_load_kernel(int64_t n, const int32_t *perm, const double *x, double *master, float4 *y) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const double2 *src = reinterpret_cast<const double2 *>(x + 4 * (int64_t)perm[m]);
        const double2 p = src[0], v = src[1];
        if (master) {
            double2 *dst = reinterpret_cast<double2 *>(master + 4 * m);
            dst[0] = p;
            dst[1] = v;
        }
        y[m] = make_float4((float)p.x, (float)p.y, (float)v.x, (float)v.y);
    }
}

__global__ void cs_store_kernel(int64_t n, const int32_t *perm, const double *master, double *x) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const double2 *src = reinterpret_cast<const double2 *>(master + 4 * m);
        double2 *dst = reinterpret_cast<double2 *>(x + 4 * (int64_t)perm[m]);
        dst[0] = src[0];
        dst[1] = src[1];
    }
}

// Sampled check of the learned basis at the current stage state, one block
// per sampled node m of community c:
//   err_m = max over both components of |dense_m - (1/N) sum_{l in c, l != m} eta (v_l - v_m)|,
//   ref_m = max over both components of |(1/N) sum_{l in N(m)} eta (v_l - v_m)|.
// The CIA value of v_m' differs from the direct one by exactly the first
// difference (the sparse corrections are exact), the second is the direct
// value itself.
__global__ void __launch_bounds__(kThreads) cs_check_kernel(const CsParams a, const int32_t *nodes,
                                                            const int32_t *node_comm, const int64_t *off,
                                                            double *out) {
    __shared__ float mom[kPart];
    __shared__ double red[kWarps][4];
    const int k = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t m = nodes[k];
    const int c = node_comm[k];
    const int64_t lo = off[c], hi = off[c + 1];
    if (t < kPart) {
        double s = 0.0;
        for (int u = a.comm_tile_begin[c]; u < a.comm_tile_begin[c + 1]; ++u) s += a.part_in[(int64_t)u * kPart + t];
        mom[t] = (float)(s * a.inv_n64);
    }
    const float4 own = a.y_in[m];
    float bx = 0.f, by = 0.f, ex = 0.f, ey = 0.f;
    for (int64_t l = lo + t; l < hi; l += kThreads)
        if (l != m) pair_term(a, own, a.y_in[l], bx, by);
    const int4 *col4 = reinterpret_cast<const int4 *>(a.full_col);
    for (int64_t v = a.full_rowptr[m] / 4 + t; v < a.full_rowptr[m + 1] / 4; v += kThreads) {
        const int4 q = col4[v];
        const int l4[4] = {q.x, q.y, q.z, q.w};
        for (int e = 0; e < 4; ++e)
            if (l4[e] < a.n) pair_term(a, own, a.y_in[l4[e]], ex, ey);
    }
    double v4[4] = {bx, by, ex, ey};
    for (int i = 0; i < 4; ++i)
        for (int o = 16; o > 0; o >>= 1) v4[i] += __shfl_xor_sync(0xffffffffu, v4[i], o);
    if (lane == 0)
        for (int i = 0; i < 4; ++i) red[warp][i] = v4[i];
    __syncthreads();
    if (warp == 0) {
        // dense term from the stored features: lane handles features lane, lane + 32
        float dx = 0.f, dy = 0.f;
        for (int rr = lane; rr < kRank; rr += 32) {
            const float f = __bfloat162float(a.feat[m * kRank + rr]);
            dx = fmaf(f, fmaf(-mom[rr], own.z, mom[kRank + rr]), dx);
            dy = fmaf(f, fmaf(-mom[rr], own.w, mom[2 * kRank + rr]), dy);
        }
        for (int o = 16; o > 0; o >>= 1) {
            dx += __shfl_xor_sync(0xffffffffu, dx, o);
            dy += __shfl_xor_sync(0xffffffffu, dy, o);
        }
        if (lane == 0) {
            double s[4] = {0.0, 0.0, 0.0, 0.0};
            for (int i = 0; i < kWarps; ++i)
                for (int j = 0; j < 4; ++j) s[j] += red[i][j];
            const double errx = fabs((double)dx - a.inv_n64 * s[0]), erry = fabs((double)dy - a.inv_n64 * s[1]);
            out[2 * k] = fmax(errx, erry);
            out[2 * k + 1] = a.inv_n64 * fmax(fabs(s[2]), fabs(s[3]));
        }
    }
}

// Centroid of each community's positions in the FP32 state (one block per community).
__global__ void __launch_bounds__(kThreads) cs_centroid_kernel(const int64_t *off, const float4 *y, float2 *cen) {
    __shared__ float red[kWarps][2];
    const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t lo = off[c], hi = off[c + 1];
    float sx = 0.f, sy = 0.f;
    for (int64_t l = lo + t; l < hi; l += kThreads) {
        sx += y[l].x;
        sy += y[l].y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        red[warp][0] = sx;
        red[warp][1] = sy;
    }
    __syncthreads();
    if (t == 0) {
        float a = 0.f, b = 0.f;
        for (int i = 0; i < kWarps; ++i) {
            a += red[i][0];
            b += red[i][1];
        }
        const float lam = (float)(hi - lo);
        cen[c] = hi > lo ? make_float2(a / lam, b / lam) : make_float2(0.f, 0.f);
    }
}

// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014) applied to a counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Pair q: node i uniform over the community nodes, partner l uniform over the
// other nodes of i's community; positions relative to the community centroid;
// target eta(||s_i - s_l||^2).  Output [count][5] floats.
__global__ void cs_sample_kernel(int64_t count, uint64_t seed, int64_t M, const int64_t *off, const float4 *y,
                                 const float2 *cen, float K, float sigma2, float neg_beta, float *pairs) {
    const int64_t ncomm = off[M];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = splitmix64(seed + 2 * (uint64_t)q), r1 = splitmix64(seed + 2 * (uint64_t)q + 1);
        const int64_t i = (int64_t)(r0 % (uint64_t)ncomm);
        int64_t lo = 0, hi = M;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) / 2;
            if (off[mid] <= i) lo = mid;
            else hi = mid;
        }
        const int64_t a0 = off[lo], lam = off[lo + 1] - a0;
        int64_t l = i;
        if (lam > 1) {
            l = a0 + (int64_t)(r1 % (uint64_t)(lam - 1));
            if (l >= i) ++l;
        }
        const float4 yi = y[i], yl = y[l];
        const float2 c = cen[lo];
        const float dx = yl.x - yi.x, dy = yl.y - yi.y;
        float *o = pairs + 5 * q;
        o[0] = yi.x - c.x;
        o[1] = yi.y - c.y;
        o[2] = yl.x - c.x;
        o[3] = yl.y - c.y;
        o[4] = K * __powf(fmaf(dx, dx, fmaf(dy, dy, sigma2)), neg_beta);
    }
}

CsParams base_params(const cia_plan *pl, int slot) {
    CsParams a{};
    const auto &d = pl->d;
    a.n = pl->n;
    a.n_tiles = (int)pl->n_tiles;
    a.group = pl->group_size_direct;
    a.inv_n = (float)(1.0 / (double)pl->n);
    a.inv_n64 = 1.0 / (double)pl->n;
    a.K = (float)pl->K;
    a.sigma2 = (float)(pl->cs_sigma * pl->cs_sigma);
    a.neg_beta = (float)(-pl->cs_beta);
    a.tile_desc = d.tile_desc;
    a.tile_order = d.tile_order;
    a.blob = d.blob;
    a.comm_tile_begin = d.comm_tile_begin;
    a.full_rowptr = d.full_rowptr;
    a.full_col = d.full_col;
    a.y_in = d.cs_y[slot];
    a.y_out = d.cs_y[slot ^ 1];
    a.part_in = d.cs_part[slot];
    a.part_out = d.cs_part[slot ^ 1];
    a.shift = d.cs_shift;
    a.feat = static_cast<__nv_bfloat16 *>(d.cs_feat);
    a.params = d.cs_params;
    a.wimage = static_cast<const mlp::Weights *>(d.cs_wimage);
    a.acc = d.cs_acc;
    a.master = d.cs_master;
    a.perm = d.perm;
    a.win_bytes = (uint32_t)align_up((size_t)pl->max_comm * sizeof(float4), 16);
    a.err_flag = d.err_flag;
    return a;
}

// Dynamic shared memory of a launch: the weights (feature launch and fused
// stages), then one region holding the community window and the sparse-sum
// tables (stage launches) and, reused, the layer-2 operand or the feature tile.
size_t stage_smem(const cia_plan *pl, bool features, bool sums) {
    const size_t win = align_up((size_t)pl->max_comm * sizeof(float4), 16);
    const size_t tables = sums ? kMaxChunks * sizeof(float2) + kTileMax * sizeof(float2) + kMaxChunks * 2 : 0;
    const size_t mlp = features ? std::max((size_t)kTileMax * CIA_BASIS_HIDDEN * 2, kFeatTileBytes + kRedBytes) : 0;
    return (features ? kWeightsBytes : 0) + std::max(win + tables, mlp);
}

template <int MODE>
constexpr bool fused_stage() { return CIA_CS_FUSED && MODE == kStage; }

template <int MODE>
cudaError_t launch_stage_t(const cia_plan *pl, const CsParams &a, cudaStream_t s) {
    constexpr bool features = MODE == kLoad || fused_stage<MODE>();
    const size_t smem = stage_smem(pl, features, MODE != kLoad);
    cudaError_t e = ensure_dynamic_smem((const void *)cs_stage_kernel<MODE>, pl->device, smem);
    if (e != cudaSuccess) return e;
    // one CTA per tile (each loads the weights and, when it evaluates
    // features, allocates tensor memory for its tile); the hardware starts
    // the next tile wherever a slot frees up
    const int64_t grid = pl->n_tiles;
    void *args[] = {const_cast<CsParams *>(&a)};
    return cudaLaunchKernel((const void *)cs_stage_kernel<MODE>, dim3((unsigned)std::max<int64_t>(grid, 1)),
                            dim3(kThreads), args, smem, s);
}

template <int MODE>
cudaError_t launch_direct_t(const cia_plan *pl, const CsParams &a, cudaStream_t s) {
    const int64_t rows_per_block = (int64_t)kWarps * (32 / a.group);
    const int64_t grid = std::min<int64_t>((pl->n + rows_per_block - 1) / rows_per_block, (int64_t)pl->n_sms * 16);
    cs_direct_kernel<MODE><<<(unsigned)std::max<int64_t>(grid, 1), kThreads, 0, s>>>(a);
    return cudaGetLastError();
}

unsigned grid_1d(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

}  // namespace

// The weights' shared-memory image in global memory, packed once per basis.
__global__ void __launch_bounds__(kThreads) cs_pack_weights_kernel(const float *params, mlp::Weights *out) {
    mlp::load_weights(params, *out);
}

cudaError_t cs_pack_weights(cia_plan *pl, cudaStream_t s) {
    if (!pl->d.cs_wimage) {
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, sizeof(mlp::Weights));
        if (e != cudaSuccess) return e;
        pl->allocations.push_back(p);
        pl->device_bytes += (int64_t)sizeof(mlp::Weights);
        pl->d.cs_wimage = p;
    }
    cs_pack_weights_kernel<<<1, kThreads, 0, s>>>(pl->d.cs_params, static_cast<mlp::Weights *>(pl->d.cs_wimage));
    return cudaGetLastError();
}

size_t cs_stage_smem_bytes(const cia_plan *pl) {
    return std::max({stage_smem(pl, false, true), stage_smem(pl, true, false), stage_smem(pl, true, true)});
}

cudaError_t cs_launch_load(cia_plan *pl, const double *x, bool write_master, int slot, cudaStream_t s) {
    cs_load_kernel<<<grid_1d(pl->n), 256, 0, s>>>(pl->n, pl->d.perm, x, write_master ? pl->d.cs_master : nullptr,
                                                  pl->d.cs_y[slot]);
    return cudaGetLastError();
}

cudaError_t cs_launch_features(cia_plan *pl, int slot, cudaStream_t s) {
    // features and moment partial sums of y[slot] itself (no stage update)
    CsParams a = base_params(pl, slot);
    a.part_out = pl->d.cs_part[slot];
    return launch_stage_t<kLoad>(pl, a, s);
}

cudaError_t cs_launch_rhs(cia_plan *pl, int method, int slot, double *dxdt, cudaStream_t s) {
    CsParams a = base_params(pl, slot);
    a.rhs_out = dxdt;
    return method == Method::DIRECT ? launch_direct_t<kRhs>(pl, a, s) : launch_stage_t<kRhs>(pl, a, s);
}

cudaError_t cs_launch_stage(cia_plan *pl, int method, int stage, int slot, double dt, cudaStream_t s) {
    static const float b[4] = {1.0f / 6.0f, 1.0f / 3.0f, 1.0f / 3.0f, 1.0f / 6.0f};
    static const double c_next[4] = {0.5, 0.5, 1.0, 0.0};
    CsParams a = base_params(pl, slot);
    a.b_s = b[stage - 1];
    a.c_next_dt = (float)(c_next[stage - 1] * dt);
    a.dt = dt;
    a.first_stage = stage == 1;
    if (method == Method::DIRECT)
        return stage == 4 ? launch_direct_t<kFinal>(pl, a, s) : launch_direct_t<kStage>(pl, a, s);
    cudaError_t e = stage == 4 ? launch_stage_t<kFinal>(pl, a, s) : launch_stage_t<kStage>(pl, a, s);
    if (e != cudaSuccess) return e;
    // the fused stages 1-3 wrote the next stage state's features (with the
    // shift of this RK4 step); after stage 4 the feature launch evaluates
    // them with the new state's own centroid, the shift of the next step
    if (stage < 4 && fused_stage<kStage>()) return cudaSuccess;
    return cs_launch_features(pl, slot ^ 1, s);
}

cudaError_t cs_launch_store(cia_plan *pl, double *x, cudaStream_t s) {
    cs_store_kernel<<<grid_1d(pl->n), 256, 0, s>>>(pl->n, pl->d.perm, pl->d.cs_master, x);
    return cudaGetLastError();
}

cudaError_t cs_launch_check(cia_plan *pl, int slot, cudaStream_t s) {
    CsParams a = base_params(pl, slot);
    cs_check_kernel<<<(unsigned)pl->cs_check_count, kThreads, 0, s>>>(a, pl->d.cs_check_nodes, pl->d.cs_check_comm,
                                                                      pl->d.off, pl->d.cs_check_out);
    return cudaGetLastError();
}

cudaError_t cs_launch_sample(cia_plan *pl, int slot, int64_t count, uint64_t seed, float *pairs, cudaStream_t s) {
    cs_centroid_kernel<<<(unsigned)pl->M, kThreads, 0, s>>>(pl->d.off, pl->d.cs_y[slot], pl->d.cs_cen);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cs_sample_kernel<<<grid_1d(count), 256, 0, s>>>(count, seed, pl->M, pl->d.off, pl->d.cs_y[slot], pl->d.cs_cen,
                                                    (float)pl->K, (float)(pl->cs_sigma * pl->cs_sigma),
                                                    (float)(-pl->cs_beta), pairs);
    return cudaGetLastError();
}

}  // namespace cia
