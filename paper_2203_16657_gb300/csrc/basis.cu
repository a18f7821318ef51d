// Learned separable basis of the Cucker--Smale weight (include/cia_basis.h):
// tensor-core forward, pair-loss backward, gradient reduction and Adam.
//
// Forward (per tile of 128 inputs): layer 1 on the FP32 cores, BF16
// activations A (K-major, shared memory), layer 2 D = A W2^T as tcgen05 MMAs
// (BF16 operands, FP32 accumulator in tensor memory).
//
// Backward of L = (1/B) sum_b (phi(a_b) . phi(c_b) - t_b)^2 (per tile of 64
// pairs = 128 inputs: rows 0..63 hold a_b, rows 64..127 hold c_b):
//   e_b = phi(a_b) . phi(c_b) - t_b,  g_b = 2 e_b / B
//   dPhi(a_b) = g_b phi(c_b),  dPhi(c_b) = g_b phi(a_b)
//   dA1   = dPhi W2                 (MMA: 128 x 128 x 64)
//   dW2^T += A1^T dPhi              (MMA: 128 x 64 x 128, accumulated in tensor
//                                    memory over all tiles of the CTA)
//   dZ1   = dA1 * cos(Z1)           (FP32 cores; the activation is sin)
//   dW1, db1, db2: column sums over the tile rows (FP32 cores)
// Each CTA writes its partial gradient; a second kernel adds the partials in
// CTA order (deterministic).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "cia_basis.h"
#include "cia_internal.h"
#include "mlp_tile.cuh"

struct cia_basis {
    int device = 0;
    int n_sms = 0;
    float *params = nullptr;        // [kParams] FP32 master
    float *adam_m = nullptr, *adam_v = nullptr;
    int64_t adam_t = 0;             // Adam steps taken
    float *grad = nullptr;          // [kParams] scratch of cia_basis_fit
    float *partial = nullptr;       // [n_sms][kParams] per-CTA partial gradients
    double *loss_part = nullptr;    // [n_sms]
    double *fit_loss = nullptr;     // [2]: first batch loss, running sum of the epoch
    int *err_flag = nullptr;
};

namespace cia {
namespace {

using mlp::kHidden;
using mlp::kParams;
using mlp::kRank;
using mlp::kThreads;
using mlp::kTileRows;

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---- forward ---------------------------------------------------------------

constexpr size_t kFwdWeights = 0;
constexpr size_t kFwdA = align_up(sizeof(mlp::Weights), 1024);
constexpr size_t kFwdSmem = kFwdA + (size_t)kTileRows * kHidden * 2;

__global__ void __launch_bounds__(kThreads) basis_features_kernel(const float *__restrict__ params,
                                                                  const float *__restrict__ x, int64_t count,
                                                                  float *__restrict__ phi, int *err_flag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    mlp::Weights &w = *reinterpret_cast<mlp::Weights *>(smem + kFwdWeights);
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(smem + kFwdA);
    const int t = threadIdx.x, r = t & 127, h = t >> 7;

    mlp::load_weights(params, w);
    if (t < 32) umma::tmem_alloc(&tslot, 64);
    if (t == 0) mbar_init(&bar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;

    const int64_t tiles = (count + kTileRows - 1) / kTileRows;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row = tile * kTileRows + r;
        const bool valid = row < count;
        float x0 = 0.f, x1 = 0.f;
        if (valid) {
            const float2 v = __ldg(reinterpret_cast<const float2 *>(x) + row);
            x0 = v.x;
            x1 = v.y;
        }
        mlp::hidden_to_smem(w, x0, x1, r, h, valid, A);
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
        if (valid) {
            float4 *dst = reinterpret_cast<float4 *>(phi + row * kRank + 32 * h);
#pragma unroll
            for (int e = 0; e < 8; ++e) dst[e] = make_float4(f[4 * e], f[4 * e + 1], f[4 * e + 2], f[4 * e + 3]);
        }
        umma::fence_before_sync();
        __syncthreads();
    }
    if (!ok) {
        if (t == 0) atomicExch(err_flag, 1);
        // the MMA may still be running: give it one more bounded wait before
        // the tensor memory is released
        mbar_wait_bounded(&bar, phase, kWaitLimitNs);
    }
    umma::fence_before_sync();
    __syncthreads();
    if (t < 32) umma::tmem_dealloc(tmem, 64);
}

// ---- backward of the pair loss -----------------------------------------------

constexpr size_t kBwdWeights = 0;
constexpr size_t kBwdW2T = align_up(sizeof(mlp::Weights), 1024);          // [128 j][64 r] K-major
constexpr size_t kBwdA1 = kBwdW2T + (size_t)kHidden * kRank * 2;           // [128 i][128 j]
constexpr size_t kBwdA1T = kBwdA1 + (size_t)kTileRows * kHidden * 2;       // [128 j][128 i]
constexpr size_t kBwdGA = kBwdA1T + (size_t)kHidden * kTileRows * 2;       // [128 i][64 r]
constexpr size_t kBwdGT = kBwdGA + (size_t)kTileRows * kRank * 2;          // [64 r][128 i]
constexpr size_t kBwdS = kBwdGT + (size_t)kRank * kTileRows * 2;           // FP32 scratch [128][128]
constexpr size_t kBwdX = kBwdS + (size_t)kTileRows * kHidden * 4;          // float2 [128]
constexpr size_t kBwdT = kBwdX + (size_t)kTileRows * 8;                    // float [64]
constexpr size_t kBwdRed = kBwdT + 64 * 4;                                 // float [3][256]
constexpr size_t kBwdSmem = kBwdRed + 3 * kThreads * 4;
static_assert(kBwdSmem <= 227 * 1024 - 64, "backward tile fits one CTA");

constexpr uint32_t kIdescDA1 = umma::idesc_bf16_f32(kTileRows, kHidden);   // 128 x 128, K = 64
constexpr uint32_t kIdescDW2 = umma::idesc_bf16_f32(kHidden, kRank);       // 128 x 64, K = 128
constexpr uint32_t kTmemCols = 256;    // [0,64) Phi, [64,192) dA1, [192,256) dW2^T

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void st_bf16(unsigned char *base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
}

__global__ void __launch_bounds__(kThreads, 1) basis_pair_grad_kernel(const float *__restrict__ params,
                                                                      const float *__restrict__ pairs, int64_t count,
                                                                      float *__restrict__ partial,
                                                                      double *__restrict__ loss_part, int *err_flag) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ double lred[kThreads / 32];
    mlp::Weights &w = *reinterpret_cast<mlp::Weights *>(smem + kBwdWeights);
    unsigned char *W2T = smem + kBwdW2T;
    unsigned char *A1 = smem + kBwdA1;
    unsigned char *A1T = smem + kBwdA1T;
    unsigned char *GA = smem + kBwdGA;
    unsigned char *GT = smem + kBwdGT;
    float *S = reinterpret_cast<float *>(smem + kBwdS);
    float2 *X = reinterpret_cast<float2 *>(smem + kBwdX);
    float *T = reinterpret_cast<float *>(smem + kBwdT);
    float *red = reinterpret_cast<float *>(smem + kBwdRed);
    const int t = threadIdx.x, r = t & 127, h = t >> 7;

    mlp::load_weights(params, w);
    // W2 as the B operand of dA1 = dPhi W2: rows j, K = r
    for (int i = t; i < kHidden * (kRank / 8); i += kThreads) {
        const int j = i / (kRank / 8), r0 = (i % (kRank / 8)) * 8;
        uint32_t q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
            q[e] = pack_bf16(params[mlp::kOffW2 + (r0 + 2 * e) * kHidden + j],
                             params[mlp::kOffW2 + (r0 + 2 * e + 1) * kHidden + j]);
        *reinterpret_cast<uint4 *>(W2T + umma::kmajor_offset(j, r0, kRank)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
    if (t < 32) umma::tmem_alloc(&tslot, kTmemCols);
    if (t == 0) mbar_init(&bar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t lane_base = (uint32_t)(32 * ((t >> 5) & 3)) << 16;

    const float inv_count = 1.0f / (float)count;
    const int64_t tiles = (count + 63) / 64;
    uint32_t phase = 0;
    bool ok = true, any = false;
    float gw0 = 0.f, gw1 = 0.f, gb1 = 0.f, gb2 = 0.f;   // this thread's share of dW1, db1, db2
    double lsum = 0.0;

    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t pair0 = tile * 64;
        // (a) inputs and layer 1
        const int pb = r & 63;
        const bool valid = pair0 + pb < count;
        float x0 = 0.f, x1 = 0.f;
        if (valid) {
            const float *q = pairs + (pair0 + pb) * 5 + (r < 64 ? 0 : 2);
            x0 = __ldg(q);
            x1 = __ldg(q + 1);
        }
        if (h == 0) X[r] = make_float2(x0, x1);
        if (h == 0 && r < 64) T[r] = valid ? __ldg(pairs + (pair0 + pb) * 5 + 4) : 0.f;
        for (int q8 = 0; q8 < 8; ++q8) {
            const int j0 = 64 * h + 8 * q8;
            float a[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int j = j0 + e;
                a[e] = valid ? mlp::bf16r(mlp::act(fmaf(w.W1[j].x, x0, fmaf(w.W1[j].y, x1, w.b1[j])))) : 0.f;
                st_bf16(A1T, umma::kmajor_offset(j, r, kTileRows), a[e]);
            }
            *reinterpret_cast<uint4 *>(A1 + umma::kmajor_offset(r, j0, kHidden)) =
                make_uint4(pack_bf16(a[0], a[1]), pack_bf16(a[2], a[3]), pack_bf16(a[4], a[5]), pack_bf16(a[6], a[7]));
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        // (b) Phi = A1 W2^T
        if (t == 0) mlp::issue_layer2(reinterpret_cast<const __nv_bfloat16 *>(A1), w, tmem, &bar);
        bool got = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        umma::fence_after_sync();
        {
            float f[32];
            mlp::load_features(tmem, w, h, f);
#pragma unroll
            for (int e = 0; e < 32; ++e) S[r * kRank + 32 * h + e] = f[e];
        }
        umma::fence_before_sync();
        __syncthreads();
        // (c) pair residuals and dPhi: thread t handles pair b = t >> 2, features 16 (t & 3) ..
        {
            const int b = t >> 2, q = t & 3;
            float fa[16], fc[16], dot = 0.f;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                fa[e] = S[b * kRank + 16 * q + e];
                fc[e] = S[(b + 64) * kRank + 16 * q + e];
                dot = fmaf(fa[e], fc[e], dot);
            }
            dot += __shfl_xor_sync(0xffffffffu, dot, 1);
            dot += __shfl_xor_sync(0xffffffffu, dot, 2);
            const float e_b = (pair0 + b < count) ? dot - T[b] : 0.f;
            if (q == 0) lsum += (double)e_b * (double)e_b;
            const float g = 2.0f * e_b * inv_count;
            float da[16], dc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                da[e] = g * fc[e];
                dc[e] = g * fa[e];
                S[b * kRank + 16 * q + e] = da[e];
                S[(b + 64) * kRank + 16 * q + e] = dc[e];
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                *reinterpret_cast<uint4 *>(GA + umma::kmajor_offset(b, 16 * q + 8 * hh, kRank)) =
                    make_uint4(pack_bf16(da[8 * hh], da[8 * hh + 1]), pack_bf16(da[8 * hh + 2], da[8 * hh + 3]),
                               pack_bf16(da[8 * hh + 4], da[8 * hh + 5]), pack_bf16(da[8 * hh + 6], da[8 * hh + 7]));
                *reinterpret_cast<uint4 *>(GA + umma::kmajor_offset(b + 64, 16 * q + 8 * hh, kRank)) =
                    make_uint4(pack_bf16(dc[8 * hh], dc[8 * hh + 1]), pack_bf16(dc[8 * hh + 2], dc[8 * hh + 3]),
                               pack_bf16(dc[8 * hh + 4], dc[8 * hh + 5]), pack_bf16(dc[8 * hh + 6], dc[8 * hh + 7]));
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                st_bf16(GT, umma::kmajor_offset(16 * q + e, b, kTileRows), da[e]);
                st_bf16(GT, umma::kmajor_offset(16 * q + e, b + 64, kTileRows), dc[e]);
            }
        }
        umma::fence_smem_to_async();
        umma::fence_before_sync();
        __syncthreads();
        // (d) dA1 = dPhi W2 and dW2^T += A1^T dPhi
        if (t == 0) {
            umma::fence_after_sync();
#pragma unroll
            for (int kk = 0; kk < kRank / 16; ++kk)
                umma::mma_bf16(tmem + 64, umma::smem_desc(GA + 256 * kk, 128, 128 * (kRank / 8)),
                               umma::smem_desc(W2T + 256 * kk, 128, 128 * (kRank / 8)), kIdescDA1, kk > 0);
#pragma unroll
            for (int kk = 0; kk < kTileRows / 16; ++kk)
                umma::mma_bf16(tmem + 192, umma::smem_desc(A1T + 256 * kk, 128, 128 * (kTileRows / 8)),
                               umma::smem_desc(GT + 256 * kk, 128, 128 * (kTileRows / 8)), kIdescDW2,
                               any || kk > 0);
            umma::mma_commit(&bar);
        }
        any = true;
        // db2 while the tensor core works: column r2 = t & 63 over rows 32 (t >> 6) ..
        {
            const int r2 = t & 63, q4 = t >> 6;
            for (int i = 32 * q4; i < 32 * q4 + 32; ++i) gb2 += S[i * kRank + r2];
        }
        got = mbar_wait_bounded(&bar, phase, kWaitLimitNs);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        phase ^= 1u;
        umma::fence_after_sync();
        // (e) dZ1 = dA1 * sin'(Z1) into the scratch, row r, units [64h, 64h + 64)
        for (int c = 0; c < 4; ++c) {
            float v[16];
            umma::tmem_ld16(tmem + lane_base + (uint32_t)(64 + 64 * h + 16 * c), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int j = 64 * h + 16 * c + e;
                const float z = fmaf(w.W1[j].x, x0, fmaf(w.W1[j].y, x1, w.b1[j]));
                S[r * kHidden + j] = v[e] * mlp::act_grad(z);
            }
        }
        umma::fence_before_sync();
        __syncthreads();
        // (f) dW1, db1: unit j = t & 127 over rows 64 (t >> 7) ..
        {
            const int j = t & 127, q2 = t >> 7;
            for (int i = 64 * q2; i < 64 * q2 + 64; ++i) {
                const float d = S[i * kHidden + j];
                const float2 xi = X[i];
                gw0 = fmaf(d, xi.x, gw0);
                gw1 = fmaf(d, xi.y, gw1);
                gb1 += d;
            }
        }
        __syncthreads();
    }

    if (!ok) {
        if (t == 0) atomicExch(err_flag, 1);
        mbar_wait_bounded(&bar, phase, kWaitLimitNs);
    }
    // partial gradient of this CTA
    float *out = partial + (size_t)blockIdx.x * kParams;
    red[t] = gw0;
    red[kThreads + t] = gw1;
    red[2 * kThreads + t] = gb1;
    __syncthreads();
    if (t < kHidden) {
        out[mlp::kOffW1 + 2 * t] = red[t] + red[t + 128];
        out[mlp::kOffW1 + 2 * t + 1] = red[kThreads + t] + red[kThreads + t + 128];
        out[mlp::kOffB1 + t] = red[2 * kThreads + t] + red[2 * kThreads + t + 128];
    }
    __syncthreads();
    red[t] = gb2;
    __syncthreads();
    if (t < kRank) out[mlp::kOffB2 + t] = red[t] + red[t + 64] + red[t + 128] + red[t + 192];
    // dW2[r][j] = D[j][r]: thread (j = r, h) holds columns [32h, 32h + 32)
    if (any && ok) {
        umma::fence_after_sync();
        float v[16];
        for (int c = 0; c < 2; ++c) {
            umma::tmem_ld16(tmem + lane_base + (uint32_t)(192 + 32 * h + 16 * c), v);
#pragma unroll
            for (int e = 0; e < 16; ++e) out[mlp::kOffW2 + (32 * h + 16 * c + e) * kHidden + r] = v[e];
        }
    } else {
        for (int c = 0; c < 32; ++c) out[mlp::kOffW2 + (32 * h + c) * kHidden + r] = 0.f;
    }
    // loss partial
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0) lred[t >> 5] = lsum;
    umma::fence_before_sync();
    __syncthreads();
    if (t == 0) {
        double s = 0.0;
        for (int i = 0; i < kThreads / 32; ++i) s += lred[i];
        loss_part[blockIdx.x] = s;
    }
    if (t < 32) umma::tmem_dealloc(tmem, kTmemCols);
}

// grad = sum of the CTA partials in CTA order; loss = (sum of loss partials) / count.
// fit_loss, if given: [0] receives the loss when first_step, [1] accumulates it.
__global__ void basis_reduce_kernel(const float *__restrict__ partial, int nparts, const double *__restrict__ loss_part,
                                    int64_t count, float *__restrict__ grad, double *loss, double *fit_loss,
                                    int first_step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kParams) {
        float s = 0.f;
        for (int c = 0; c < nparts; ++c) s += partial[(size_t)c * kParams + i];
        grad[i] = s;
    }
    if (i == 0) {
        double s = 0.0;
        for (int c = 0; c < nparts; ++c) s += loss_part[c];
        s /= (double)count;
        if (loss) *loss = s;
        if (fit_loss) {
            if (first_step) fit_loss[0] = s;
            fit_loss[1] += s;
        }
    }
}

// Adam (Kingma & Ba, Algorithm 1) with bias correction; t is the 1-based step.
__global__ void basis_adam_kernel(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                                  const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1,
                                  float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kParams) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

cia_status check_basis(const cia_basis *b) {
    if (!b) return fail(CIA_ERR_INVALID_ARG, "basis is NULL");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != b->device) return fail(CIA_ERR_INVALID_ARG, "basis belongs to another device");
    return CIA_OK;
}

cia_status launch_pair_grad(cia_basis *b, const float *pairs, int64_t count, float *grad, double *loss,
                            double *fit_loss, bool first_step, cudaStream_t s) {
    const int64_t tiles = (count + 63) / 64;
    const int grid = (int)std::min<int64_t>(tiles, b->n_sms);
    basis_pair_grad_kernel<<<grid, kThreads, kBwdSmem, s>>>(b->params, pairs, count, b->partial, b->loss_part,
                                                           b->err_flag);
    CIA_CUDA_TRY(cudaGetLastError());
    basis_reduce_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(b->partial, grid, b->loss_part, count, grad, loss,
                                                             fit_loss, first_step ? 1 : 0);
    CIA_CUDA_TRY(cudaGetLastError());
    return CIA_OK;
}

cia_status adam(cia_basis *b, const float *grad, const cia_adam_options *o, cudaStream_t s) {
    b->adam_t += 1;
    const double c1 = 1.0 - std::pow(o->beta1, (double)b->adam_t);
    const double c2 = 1.0 - std::pow(o->beta2, (double)b->adam_t);
    basis_adam_kernel<<<(kParams + 255) / 256, 256, 0, s>>>(b->params, b->adam_m, b->adam_v, grad, (float)o->lr,
                                                           (float)o->beta1, (float)o->beta2, (float)o->eps,
                                                           (float)c1, (float)c2);
    CIA_CUDA_TRY(cudaGetLastError());
    return CIA_OK;
}

cia_status check_adam(const cia_adam_options *o) {
    if (!o) return fail(CIA_ERR_INVALID_ARG, "Adam options are NULL");
    if (!(o->lr > 0.0) || !(o->beta1 >= 0.0 && o->beta1 < 1.0) || !(o->beta2 >= 0.0 && o->beta2 < 1.0) ||
        !(o->eps > 0.0))
        return fail(CIA_ERR_INVALID_ARG, "Adam needs lr > 0, 0 <= beta1, beta2 < 1 and eps > 0");
    return CIA_OK;
}

void free_basis(cia_basis *b) {
    if (!b) return;
    for (void *p : {(void *)b->params, (void *)b->adam_m, (void *)b->adam_v, (void *)b->grad, (void *)b->partial,
                    (void *)b->loss_part, (void *)b->fit_loss, (void *)b->err_flag})
        if (p) cudaFree(p);
    delete b;
}

}  // namespace
}  // namespace cia

using namespace cia;

namespace {

// SplitMix64 (Steele, Lea and Flood 2014): seeded doubles in [0, 1).
struct SplitMix {
    uint64_t s;
    double uniform() {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    }
};

}  // namespace

extern "C" cia_status cia_basis_params_fourier(double K, double sigma, double beta, double L, uint64_t seed,
                                               float *params) {
    clear_error();
    if (!params) return fail(CIA_ERR_INVALID_ARG, "params is NULL");
    if (!std::isfinite(K) || !std::isfinite(sigma) || !std::isfinite(beta) || !(L > 0.0) || !std::isfinite(L))
        return fail(CIA_ERR_INVALID_ARG, "need finite K, sigma, beta and L > 0");
    // coefficients of the periodic extension of g(d) = eta(|d|^2) on
    // [-L, L)^2, rectangle rule on a G x G grid, for |alpha_i| <= A:
    //   c_alpha = G^-2 sum_{j,k} g(x_j, y_k) e^{-i pi (alpha_1 x_j + alpha_2 y_k) / L}
    // evaluated as two one-dimensional sums (first over y, then over x)
    const int G = 256, A = 12, W = 2 * A + 1;
    const double pi = 3.14159265358979323846;
    std::vector<double> x(G), g((size_t)G * G);
    for (int j = 0; j < G; ++j) x[j] = -L + 2.0 * L * j / G;
    const double s2 = sigma * sigma;
    for (int j = 0; j < G; ++j)
        for (int k = 0; k < G; ++k) g[(size_t)j * G + k] = K * std::pow(s2 + x[j] * x[j] + x[k] * x[k], -beta);
    std::vector<std::complex<double>> e((size_t)W * G);   // e^{-i pi a x_k / L}
    for (int a = -A; a <= A; ++a)
        for (int k = 0; k < G; ++k) e[(size_t)(a + A) * G + k] = std::polar(1.0, -pi * a * x[k] / L);
    std::vector<std::complex<double>> h((size_t)G * W);   // h[j][a2] = sum_k g[j][k] e^{-i pi a2 y_k / L}
    for (int j = 0; j < G; ++j)
        for (int a2 = 0; a2 < W; ++a2) {
            std::complex<double> acc = 0.0;
            for (int k = 0; k < G; ++k) acc += g[(size_t)j * G + k] * e[(size_t)a2 * G + k];
            h[(size_t)j * W + a2] = acc;
        }
    struct Mode { int a1, a2; double c; };
    std::vector<Mode> modes;
    for (int a1 = 0; a1 <= A; ++a1)
        for (int a2 = -A; a2 <= A; ++a2) {
            if (a1 == 0 && a2 < 0) continue;   // one representative per +-alpha
            std::complex<double> acc = 0.0;
            for (int j = 0; j < G; ++j) acc += h[(size_t)j * W + (a2 + A)] * e[(size_t)(a1 + A) * G + j];
            const double c = acc.real() / ((double)G * G);
            if (c > 0.0) modes.push_back({a1, a2, c});
        }
    std::stable_sort(modes.begin(), modes.end(), [](const Mode &p, const Mode &q) { return p.c > q.c; });
    std::fill(params, params + kParams, 0.0f);
    SplitMix rng{seed};
    int hid = 0, feat = 0;
    for (const Mode &m : modes) {
        const bool zero = m.a1 == 0 && m.a2 == 0;
        if (feat + (zero ? 1 : 2) > kRank) continue;
        if (zero) {
            params[mlp::kOffB2 + feat++] = (float)std::sqrt(m.c);
            continue;
        }
        const double w1 = pi * m.a1 / L, w2 = pi * m.a2 / L, amp = std::sqrt(2.0 * m.c);
        for (int ph = 0; ph < 2; ++ph) {   // cos = sin(. + pi/2), then sin
            params[mlp::kOffW1 + 2 * hid] = (float)w1;
            params[mlp::kOffW1 + 2 * hid + 1] = (float)w2;
            params[mlp::kOffB1 + hid] = (float)(ph == 0 ? pi / 2 : 0.0);
            params[mlp::kOffW2 + feat * kHidden + hid] = (float)amp;
            ++hid;
            ++feat;
        }
    }
    for (; hid < kHidden; ++hid) {
        // spare plane waves: small random frequencies, no output weight yet
        params[mlp::kOffW1 + 2 * hid] = (float)(0.5 * (2.0 * rng.uniform() - 1.0));
        params[mlp::kOffW1 + 2 * hid + 1] = (float)(0.5 * (2.0 * rng.uniform() - 1.0));
        params[mlp::kOffB1 + hid] = (float)(pi * (2.0 * rng.uniform() - 1.0));
    }
    return CIA_OK;
}

extern "C" cia_status cia_basis_create(const float *params, cia_basis_t **out) {
    clear_error();
    if (!params || !out) return fail(CIA_ERR_INVALID_ARG, "params or out is NULL");
    *out = nullptr;
    for (int i = 0; i < kParams; ++i)
        if (!std::isfinite(params[i])) return fail(CIA_ERR_NUMERIC, "parameter " + std::to_string(i) + " is not finite");
    cia_basis *b = new cia_basis();
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->n_sms, cudaDevAttrMultiProcessorCount, b->device);
    auto alloc = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) e = cudaMemset(*p, 0, bytes);
    };
    alloc((void **)&b->params, kParams * sizeof(float));
    alloc((void **)&b->adam_m, kParams * sizeof(float));
    alloc((void **)&b->adam_v, kParams * sizeof(float));
    alloc((void **)&b->grad, kParams * sizeof(float));
    alloc((void **)&b->partial, (size_t)std::max(b->n_sms, 1) * kParams * sizeof(float));
    alloc((void **)&b->loss_part, (size_t)std::max(b->n_sms, 1) * sizeof(double));
    alloc((void **)&b->fit_loss, 2 * sizeof(double));
    alloc((void **)&b->err_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(b->params, params, kParams * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(basis_pair_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kBwdSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(basis_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kFwdSmem);
    if (e != cudaSuccess) {
        free_basis(b);
        return cuda_fail(e, e == cudaErrorMemoryAllocation ? "cudaMalloc (basis)" : "basis setup");
    }
    *out = b;
    return CIA_OK;
}

extern "C" cia_status cia_basis_destroy(cia_basis_t *basis) {
    clear_error();
    free_basis(basis);
    return CIA_OK;
}

extern "C" cia_status cia_basis_get_params(const cia_basis_t *basis, float *params) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    if (!params) return fail(CIA_ERR_INVALID_ARG, "params is NULL");
    CIA_CUDA_TRY(cudaMemcpy(params, basis->params, kParams * sizeof(float), cudaMemcpyDeviceToHost));
    return CIA_OK;
}

extern "C" cia_status cia_basis_features(cia_basis_t *basis, const float *x, int64_t count, float *phi,
                                         void *stream) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    if (count < 0) return fail(CIA_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return CIA_OK;
    if (!x || !phi) return fail(CIA_ERR_INVALID_ARG, "x or phi is NULL");
    const int64_t tiles = (count + kTileRows - 1) / kTileRows;
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)basis->n_sms * 4);
    basis_features_kernel<<<grid, kThreads, kFwdSmem, (cudaStream_t)stream>>>(basis->params, x, count, phi,
                                                                           basis->err_flag);
    CIA_CUDA_TRY(cudaGetLastError());
    return CIA_OK;
}

extern "C" cia_status cia_basis_pair_grad(cia_basis_t *basis, const float *pairs, int64_t count, float *grad,
                                          double *loss, void *stream) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    if (count <= 0) return fail(CIA_ERR_INVALID_ARG, "count must be positive");
    if (!pairs || !grad) return fail(CIA_ERR_INVALID_ARG, "pairs or grad is NULL");
    return launch_pair_grad(basis, pairs, count, grad, loss, nullptr, false, (cudaStream_t)stream);
}

extern "C" cia_status cia_basis_adam_step(cia_basis_t *basis, const float *grad, const cia_adam_options *opt,
                                          void *stream) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    if (!grad) return fail(CIA_ERR_INVALID_ARG, "grad is NULL");
    st = check_adam(opt);
    if (st != CIA_OK) return st;
    return adam(basis, grad, opt, (cudaStream_t)stream);
}

extern "C" cia_status cia_basis_fit(cia_basis_t *basis, const float *pairs, int64_t count,
                                    const cia_fit_options *opt, cia_fit_report *report, void *stream) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    if (!pairs || !opt) return fail(CIA_ERR_INVALID_ARG, "pairs or options are NULL");
    if (count <= 0) return fail(CIA_ERR_INVALID_ARG, "count must be positive");
    if (opt->batch <= 0 || opt->batch % 64 != 0) return fail(CIA_ERR_INVALID_ARG, "batch must be a positive multiple of 64");
    if (opt->epochs < 0) return fail(CIA_ERR_INVALID_ARG, "epochs < 0");
    st = check_adam(&opt->adam);
    if (st != CIA_OK) return st;
    if (opt->lr_final < 0.0 || !std::isfinite(opt->lr_final)) return fail(CIA_ERR_INVALID_ARG, "lr_final < 0");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t steps = 0;
    double epoch_loss = 0.0, first = 0.0;
    const int64_t per_epoch = (count + opt->batch - 1) / opt->batch;
    const int64_t total_steps = per_epoch * opt->epochs;
    cia_adam_options ad = opt->adam;
    for (int64_t ep = 0; ep < opt->epochs; ++ep) {
        CIA_CUDA_TRY(cudaMemsetAsync(basis->fit_loss + 1, 0, sizeof(double), s));
        int64_t batches = 0;
        for (int64_t b0 = 0; b0 < count; b0 += opt->batch) {
            const int64_t nb = std::min<int64_t>(opt->batch, count - b0);
            st = launch_pair_grad(basis, pairs + b0 * 5, nb, basis->grad, nullptr, basis->fit_loss, steps == 0, s);
            if (st != CIA_OK) return st;
            if (opt->lr_final > 0.0 && total_steps > 1)
                ad.lr = opt->adam.lr * std::pow(opt->lr_final / opt->adam.lr, (double)steps / (double)(total_steps - 1));
            st = adam(basis, basis->grad, &ad, s);
            if (st != CIA_OK) return st;
            ++steps;
            ++batches;
        }
        if (ep + 1 == opt->epochs) {
            double h[2];
            CIA_CUDA_TRY(cudaMemcpyAsync(h, basis->fit_loss, sizeof(h), cudaMemcpyDeviceToHost, s));
            CIA_CUDA_TRY(cudaStreamSynchronize(s));
            first = h[0];
            epoch_loss = h[1] / (double)std::max<int64_t>(batches, 1);
        }
    }
    CIA_CUDA_TRY(cudaStreamSynchronize(s));
    int flag = 0;
    CIA_CUDA_TRY(cudaMemcpy(&flag, basis->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CIA_CUDA_TRY(cudaMemset(basis->err_flag, 0, sizeof(int)));
        return fail(CIA_ERR_TIMEOUT, "a tensor-core wait of the basis kernels gave up");
    }
    if (report) {
        report->steps = steps;
        report->first_loss = first;
        report->last_epoch_loss = epoch_loss;
    }
    return CIA_OK;
}

extern "C" cia_status cia_basis_sync(cia_basis_t *basis, void *stream) {
    clear_error();
    cia_status st = check_basis(basis);
    if (st != CIA_OK) return st;
    CIA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int flag = 0;
    CIA_CUDA_TRY(cudaMemcpy(&flag, basis->err_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CIA_CUDA_TRY(cudaMemset(basis->err_flag, 0, sizeof(int)));
        return fail(CIA_ERR_TIMEOUT, "a tensor-core wait of the basis kernels gave up");
    }
    return CIA_OK;
}

// ---- the basis inside a Cucker--Smale plan -----------------------------------

namespace {

cia_status check_cs_plan(const cia_plan *pl) {
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    if (pl->model != CIA_MODEL_CUCKER_SMALE) return fail(CIA_ERR_INVALID_ARG, "not a Cucker-Smale plan");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(CIA_ERR_INVALID_ARG, "plan belongs to another device");
    return CIA_OK;
}

void reset_check(cia_plan *pl) {
    pl->checks = 0;
    pl->check_last = pl->check_max = 0.0;
    pl->fell_back = false;
    pl->fallback_step = -1;
}

}  // namespace

extern "C" cia_status cia_plan_set_basis(cia_plan_t *plan, const cia_basis_t *basis) {
    clear_error();
    cia_status st = check_cs_plan(plan);
    if (st != CIA_OK) return st;
    if ((st = check_basis(basis)) != CIA_OK) return st;
    CIA_CUDA_TRY(cudaMemcpy(plan->d.cs_params, basis->params, kParams * sizeof(float), cudaMemcpyDeviceToDevice));
    CIA_CUDA_TRY(cs_pack_weights(plan, nullptr));
    CIA_CUDA_TRY(cudaDeviceSynchronize());
    plan->cs_has_basis = true;
    plan->cs_feat_valid = false;
    reset_check(plan);
    return CIA_OK;
}

extern "C" cia_status cia_plan_sample_pairs(cia_plan_t *plan, int64_t count, uint64_t seed, float *pairs,
                                            void *stream) {
    clear_error();
    cia_status st = check_cs_plan(plan);
    if (st != CIA_OK) return st;
    if (count < 0) return fail(CIA_ERR_INVALID_ARG, "count < 0");
    if (count == 0) return CIA_OK;
    if (!pairs) return fail(CIA_ERR_INVALID_ARG, "pairs is NULL");
    if (plan->M < 1 || plan->off[plan->M] < 1) return fail(CIA_ERR_INVALID_ARG, "the plan has no community nodes");
    CIA_CUDA_TRY(cs_launch_sample(plan, plan->state_slot, count, seed, pairs, (cudaStream_t)stream));
    return CIA_OK;
}

extern "C" cia_status cia_plan_set_check(cia_plan_t *plan, int64_t every, double bound) {
    clear_error();
    cia_status st = check_cs_plan(plan);
    if (st != CIA_OK) return st;
    if (every < 0) return fail(CIA_ERR_INVALID_ARG, "every < 0");
    if (every > 0 && !(bound > 0.0 && std::isfinite(bound))) return fail(CIA_ERR_INVALID_ARG, "bound must be positive");
    if (every > 0 && !plan->has_direct)
        return fail(CIA_ERR_INVALID_ARG, "the check needs the direct method (build_direct)");
    if (every > 0 && plan->cs_check_count < 1) return fail(CIA_ERR_INVALID_ARG, "the plan has no community nodes");
    plan->check_every = every;
    plan->check_bound = bound;
    reset_check(plan);
    return CIA_OK;
}

extern "C" cia_status cia_plan_get_check(const cia_plan_t *plan, cia_check_report *report) {
    clear_error();
    if (!plan || !report) return fail(CIA_ERR_INVALID_ARG, "plan or report is NULL");
    report->checks = plan->checks;
    report->last_error = plan->check_last;
    report->max_error = plan->check_max;
    report->fell_back = plan->fell_back ? 1 : 0;
    report->fallback_step = plan->fallback_step;
    return CIA_OK;
}

extern "C" cia_status cia_learn_fit(cia_plan_t *plan, cia_basis_t *basis, const double *x0,
                                    const cia_learn_options *opt, cia_learn_report *report, void *stream) {
    clear_error();
    cia_status st = check_cs_plan(plan);
    if (st != CIA_OK) return st;
    if ((st = check_basis(basis)) != CIA_OK) return st;
    if (!x0 || !opt) return fail(CIA_ERR_INVALID_ARG, "x0 or options are NULL");
    if (!plan->has_direct) return fail(CIA_ERR_INVALID_ARG, "learning from trajectories needs build_direct");
    if (opt->steps < 0 || opt->snapshots < 1 || opt->pairs < opt->snapshots || !std::isfinite(opt->dt))
        return fail(CIA_ERR_INVALID_ARG, "need steps >= 0, snapshots >= 1, pairs >= snapshots and a finite dt");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t per = opt->pairs / opt->snapshots;
    const int64_t total = per * opt->snapshots;
    float *pairs = nullptr;
    CIA_CUDA_TRY(cudaMalloc(&pairs, (size_t)total * 5 * sizeof(float)));
    struct Free {
        float *p;
        ~Free() { cudaFree(p); }
    } guard{pairs};
    if ((st = cia_state_load(plan, x0, stream)) != CIA_OK) return st;
    int64_t done = 0;
    for (int64_t k = 0; k < opt->snapshots; ++k) {
        st = cia_plan_sample_pairs(plan, per, opt->seed + (uint64_t)k * (1ull << 40), pairs + (size_t)k * per * 5,
                                   stream);
        if (st != CIA_OK) return st;
        const int64_t next = (k + 1) * opt->steps / opt->snapshots;
        if (next > done) {
            if ((st = cia_advance(plan, CIA_METHOD_DIRECT, opt->dt, next - done, nullptr, stream)) != CIA_OK) return st;
            done = next;
        }
    }
    cia_fit_report fr{};
    if ((st = cia_basis_fit(basis, pairs, total, &opt->fit, &fr, stream)) != CIA_OK) return st;
    if ((st = cia_plan_set_basis(plan, basis)) != CIA_OK) return st;
    if (report) {
        report->pairs = total;
        report->fit = fr;
    }
    CIA_CUDA_TRY(cudaStreamSynchronize(s));
    return CIA_OK;
}
