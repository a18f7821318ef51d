// Device building blocks of the learned feature map phi (a 2 -> 128 -> 64
// perceptron, see include/cia_basis.h) for one tile of 128 inputs and a CTA
// of 256 threads.
//
// Thread t owns input row r = t & 127 and half h = t >> 7 of the hidden units
// (j in [64h, 64h + 64)) and of the features (columns [32h, 32h + 32)): warp
// w reaches tensor-memory lanes 32 (w & 3) .. 32 (w & 3) + 31, which are
// exactly its rows.
//
// Layer 1 (K = 2) runs on the FP32 cores; its activations, rounded to BF16,
// form the K-major A operand of layer 2, a 128 x 64 x 128 BF16 tcgen05 MMA
// with the FP32 accumulator in tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cia_basis.h"
#include "sync.cuh"
#include "umma.cuh"

namespace cia {
namespace mlp {

constexpr int kIn = CIA_BASIS_IN;
constexpr int kHidden = CIA_BASIS_HIDDEN;
constexpr int kRank = CIA_BASIS_RANK;
constexpr int kParams = CIA_BASIS_PARAMS;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kHidden * kIn;
constexpr int kOffW2 = kOffB1 + kHidden;
constexpr int kOffB2 = kOffW2 + kRank * kHidden;
static_assert(kOffB2 + kRank == kParams, "parameter packing");
static_assert(kIn == 2 && kHidden == 128 && kRank == 64, "the tile code is written for 2 -> 128 -> 64");

constexpr int kTileRows = 128;        // MMA M
constexpr int kThreads = 256;
constexpr uint32_t kIdescL2 = umma::idesc_bf16_f32(kTileRows, kRank);

// Shared-memory image of the parameters: W2, the tensor-core operand, in
// BF16; the first layer (K = 2, FP32 cores) and the biases in FP32.
struct Weights {
    __nv_bfloat16 W2[kRank * kHidden];        // K-major B operand of layer 2: rows r, k = j
    float2 W1[kHidden];                       // (W1[j][0], W1[j][1])
    float b1[kHidden];
    float b2[kRank];
};

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Fill w from the FP32 master parameters, rounding W2 to BF16.
// All kThreads threads call it; the caller synchronises afterwards.
__device__ __forceinline__ void load_weights(const float *__restrict__ params, Weights &w) {
    const int t = threadIdx.x;
    for (int i = t; i < kRank * kHidden / 8; i += kThreads) {
        // 8 consecutive hidden units j of feature row r: one 16-byte store;
        // consecutive threads take consecutive rows of one core-matrix column,
        // so that eight of them fill 128 contiguous bytes (all 32 banks)
        const int r = i % kRank, j0 = (i / kRank) * 8;
        const float *src = params + kOffW2 + r * kHidden + j0;
        uint32_t q[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            __nv_bfloat162 v = __floats2bfloat162_rn(src[2 * e], src[2 * e + 1]);
            q[e] = *reinterpret_cast<uint32_t *>(&v);
        }
        *reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(w.W2) + umma::kmajor_offset(r, j0, kHidden)) =
            make_uint4(q[0], q[1], q[2], q[3]);
    }
    for (int j = t; j < kHidden; j += kThreads) {
        w.W1[j] = make_float2(params[kOffW1 + 2 * j], params[kOffW1 + 2 * j + 1]);
        w.b1[j] = params[kOffB1 + j];
    }
    for (int r = t; r < kRank; r += kThreads) w.b2[r] = params[kOffB2 + r];
}

// Hidden activation sin z.  |z| stays within a few tens (input positions
// relative to a community centroid, frequencies of a few radians per unit),
// where the hardware approximation's absolute error (a few 1e-6) is far below
// the BF16 rounding that follows.
__device__ __forceinline__ float act(float z) { return __sinf(z); }
__device__ __forceinline__ float act_grad(float z) { return __cosf(z); }

// Layer 1 for row r, hidden units [64h, 64h + 64): BF16 activations into the
// K-major A operand (kTileRows x kHidden).  A row that is not `valid` gets
// zeros.  Returns nothing; the caller fences and synchronises.
__device__ __forceinline__ void hidden_to_smem(const Weights &w, float x0, float x1, int r, int h, bool valid,
                                               __nv_bfloat16 *A) {
    unsigned char *base = reinterpret_cast<unsigned char *>(A);
#pragma unroll 2
    for (int q = 0; q < 8; ++q) {
        const int j0 = 64 * h + 8 * q;
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = j0 + 2 * e;
            float a0 = 0.f, a1 = 0.f;
            if (valid) {
                a0 = act(fmaf(w.W1[j].x, x0, fmaf(w.W1[j].y, x1, w.b1[j])));
                a1 = act(fmaf(w.W1[j + 1].x, x0, fmaf(w.W1[j + 1].y, x1, w.b1[j + 1])));
            }
            __nv_bfloat162 v = __floats2bfloat162_rn(a0, a1);
            pk[e] = *reinterpret_cast<uint32_t *>(&v);
        }
        *reinterpret_cast<uint4 *>(base + umma::kmajor_offset(r, j0, kHidden)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// Issue layer 2, D[128 x 64] = A W2^T, from one thread and arrive on bar when
// it completes.
__device__ __forceinline__ void issue_layer2(const __nv_bfloat16 *A, const Weights &w, uint32_t tmem_d,
                                             uint64_t *bar) {
    umma::fence_after_sync();
#pragma unroll
    for (int kk = 0; kk < kHidden / 16; ++kk) {
        const uint64_t ad = umma::smem_desc(reinterpret_cast<const unsigned char *>(A) + 256 * kk, 128, 128 * (kHidden / 8));
        const uint64_t bd = umma::smem_desc(reinterpret_cast<const unsigned char *>(w.W2) + 256 * kk, 128, 128 * (kHidden / 8));
        umma::mma_bf16(tmem_d, ad, bd, kIdescL2, kk > 0);
    }
    umma::mma_commit(bar);
}

// Columns [32h, 32h + 32) of this thread's row of D, plus b2.
__device__ __forceinline__ void load_features(uint32_t tmem_d, const Weights &w, int h, float (&phi)[32]) {
    const uint32_t lane_base = (uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16;
    float v[16];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        umma::tmem_ld16(tmem_d + lane_base + (uint32_t)(32 * h + 16 * c), v);
#pragma unroll
        for (int e = 0; e < 16; ++e) phi[16 * c + e] = v[e] + w.b2[32 * h + 16 * c + e];
    }
}

}  // namespace mlp
}  // namespace cia
