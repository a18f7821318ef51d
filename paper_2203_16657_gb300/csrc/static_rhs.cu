// CIA right-hand side that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// owns the whole device-memory budget through its own pool allocator, or a
// latency-critical loop in which an allocation (which may synchronise the
// device and grow or fragment the pool) is not acceptable.  For them this file
// provides cia_rhs_kuramoto_static: the FP64 Kuramoto CIA right-hand side on
// caller-provided device arrays, whose only scratch memory -- the phasors
// e^{i k x_m} of the state and the community observables Z_{c,k} -- lives in
// one file-scope __device__ array of fixed size.  A device holds that array
// (5 MiB) from the moment this module is loaded there -- at the latest at the
// first call on that device, earlier if modules are loaded eagerly -- until
// the process exits.
//
// The array is shared by all calls: it keeps the last call's contents, every
// element a call reads is written earlier in the same call, and calls whose
// work overlaps on the GPU (different streams, no ordering) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "cia_internal.h"

namespace cia {
namespace {

// Capacity of the scratch array in complex FP64 entries: p * (n + M) of them
// are used by one call (phasors of n nodes and observables of M communities
// for each of the p harmonics).  5 MiB.
constexpr int64_t kScratchEntries = 327680;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double2 g_static_scratch[kScratchEntries];

// Device address of g_static_scratch on each device, resolved once per device
// (with that device current) by cudaGetSymbolAddress: in host code the symbol
// itself is only a host-side stand-in, not a device address.  The address is
// valid for one context: after a device reset the runtime creates a new
// primary context, reloads the module and the array may move, so the address
// is kept together with the unique id of the context it was resolved in and
// resolved again when the current context's id differs.
double2 *g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};
std::mutex g_scratch_mutex;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (0 if none is current),
// through the driver entry points the runtime hands out (no libcuda link).
cudaError_t current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return cudaErrorSymbolNotFound;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
        get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    *id = 0;
    if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

constexpr int kBlock = 256;

struct StaticCoupling {
    int p;
    double d_sin[CIA_MAX_HARMONICS], d_cos[CIA_MAX_HARMONICS];
    double k_over_n;
};

// Phasors u_{m,k} = e^{i k x_m}, k = 1..p, layout [p][n].
__global__ void static_phasor_kernel(int64_t n, int p, const double *x, double2 *u) {
    for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincos(x[m], &s, &c);
        double2 v = make_double2(c, s);
        for (int k = 0; k < p; ++k) {
            u[k * n + m] = v;
            v = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
        }
    }
}

// Z_{c,k} = sum over the community's nodes of u_{l,k} (E1.1), one block per
// community, strided FP64 sums followed by a fixed tree: deterministic.
__global__ void static_observable_kernel(int64_t n, int64_t M, int p, const int64_t *off, const double2 *u,
                                         double2 *z) {
    __shared__ double sre[kBlock], sim[kBlock];
    const int64_t c = blockIdx.x;
    const int64_t lo = off[c], hi = off[c + 1];
    for (int k = 0; k < p; ++k) {
        double re = 0.0, im = 0.0;
        for (int64_t l = lo + threadIdx.x; l < hi; l += kBlock) {
            const double2 v = u[k * n + l];
            re += v.x;
            im += v.y;
        }
        sre[threadIdx.x] = re;
        sim[threadIdx.x] = im;
        __syncthreads();
        for (int s = kBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                sre[threadIdx.x] += sre[threadIdx.x + s];
                sim[threadIdx.x] += sim[threadIdx.x + s];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) z[k * M + c] = make_double2(sre[0], sim[0]);
        __syncthreads();
    }
}

// One warp per node: W = sum_{inter} u_l - sum_{missing} u_l, then the dense
// term (Z_c minus the node's own phasor) and the coupling, as in cia_rhs.
__global__ void static_rhs_kernel(int64_t n, int64_t M, const int64_t *off, const int64_t *miss_rowptr,
                                  const int32_t *miss_col, const int64_t *inter_rowptr, const int32_t *inter_col,
                                  const double *omega, const double2 *u, const double2 *z, StaticCoupling cp,
                                  double *dxdt) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t m = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; m < n; m += warps) {
        // community of m: the c with off[c] <= m < off[c+1], or none
        int64_t c = -1;
        if (M > 0 && m < off[M]) {
            int64_t a = 0, b = M;
            while (b - a > 1) {
                const int64_t mid = (a + b) / 2;
                if (off[mid] <= m) a = mid;
                else b = mid;
            }
            c = a;
        }
        double coup = 0.0;
        for (int k = 0; k < cp.p; ++k) {
            double wr = 0.0, wi = 0.0;
            for (int64_t e = inter_rowptr[m] + lane; e < inter_rowptr[m + 1]; e += 32) {
                const double2 v = u[k * n + inter_col[e]];
                wr += v.x;
                wi += v.y;
            }
            for (int64_t e = miss_rowptr[m] + lane; e < miss_rowptr[m + 1]; e += 32) {
                const double2 v = u[k * n + miss_col[e]];
                wr -= v.x;
                wi -= v.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                wr += __shfl_xor_sync(0xffffffffu, wr, o);
                wi += __shfl_xor_sync(0xffffffffu, wi, o);
            }
            const double2 own = u[k * n + m];
            if (c >= 0) {
                wr += z[k * M + c].x - own.x;
                wi += z[k * M + c].y - own.y;
            }
            const double re = wr * own.x + wi * own.y;
            const double im = wi * own.x - wr * own.y;
            coup += cp.d_sin[k] * im + cp.d_cos[k] * re;
        }
        if (lane == 0) dxdt[m] = (omega ? omega[m] : 0.0) + cp.k_over_n * coup;
    }
}

cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

}  // namespace
}  // namespace cia

using namespace cia;

extern "C" cia_status cia_rhs_kuramoto_static(int64_t n, int64_t M, const int64_t *offsets,
                                              const int64_t *miss_rowptr, const int32_t *miss_col,
                                              const int64_t *inter_rowptr, const int32_t *inter_col,
                                              const double *x, const double *omega,
                                              const cia_coupling *coupling, double *dxdt, void *stream) {
    clear_error();
    if (!coupling || !offsets || !miss_rowptr || !inter_rowptr || !x || !dxdt)
        return fail(CIA_ERR_INVALID_ARG, "a required pointer is NULL");
    if (n < 1 || M < 0) return fail(CIA_ERR_INVALID_ARG, "need n >= 1 and M >= 0");
    if (coupling->model != CIA_MODEL_KURAMOTO) return fail(CIA_ERR_UNSUPPORTED, "only the Kuramoto model");
    const int p = coupling->p;
    if (p < 1 || p > CIA_MAX_HARMONICS) return fail(CIA_ERR_INVALID_ARG, "p must be in [1, CIA_MAX_HARMONICS]");
    if (!std::isfinite(coupling->K)) return fail(CIA_ERR_NUMERIC, "K is not finite");
    // n and M are bounded first so that p * (n + M) cannot overflow
    if (n > kScratchEntries || M > kScratchEntries || (int64_t)p * (n + M) > kScratchEntries)
        return fail(CIA_ERR_INVALID_ARG,
                    "p * (n + M) with n = " + std::to_string(n) + ", M = " + std::to_string(M) +
                        ", p = " + std::to_string(p) + " exceeds the static scratch capacity of " +
                        std::to_string(kScratchEntries) + " complex entries; use cia_plan_create + cia_rhs");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(CIA_ERR_UNSUPPORTED, "device index out of range");
    double2 *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        unsigned long long ctx = 0;
        CIA_CUDA_TRY(current_context_id(&ctx));
        if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
            // cudaGetSymbolAddress makes the device's primary context current if
            // none is, and loads this module in it (no allocation by this code)
            void *addr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&addr, g_static_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
            CIA_CUDA_TRY(current_context_id(&ctx));
            g_scratch_addr[dev] = static_cast<double2 *>(addr);
            g_scratch_ctx[dev] = ctx;
        }
        scratch = g_scratch_addr[dev];
    }
    StaticCoupling cp;
    cp.p = p;
    for (int k = 0; k < CIA_MAX_HARMONICS; ++k) {
        cp.d_sin[k] = k < p ? coupling->d_sin[k] : 0.0;
        cp.d_cos[k] = k < p ? coupling->d_cos[k] : 0.0;
    }
    cp.k_over_n = coupling->K / (double)n;
    double2 *u = scratch;                    // [p][n]
    double2 *z = scratch + (int64_t)p * n;   // [p][M]
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + kBlock - 1) / kBlock, 152 * 16);
    static_phasor_kernel<<<blocks, kBlock, 0, s>>>(n, p, x, u);
    CIA_CUDA_TRY(cudaGetLastError());
    if (M > 0) {
        static_observable_kernel<<<(unsigned)M, kBlock, 0, s>>>(n, M, p, offsets, u, z);
        CIA_CUDA_TRY(cudaGetLastError());
    }
    const unsigned rblocks = (unsigned)std::min<int64_t>((n * 32 + kBlock - 1) / kBlock, 152 * 16);
    static_rhs_kernel<<<rblocks, kBlock, 0, s>>>(n, M, offsets, miss_rowptr, miss_col, inter_rowptr, inter_col,
                                                 omega, u, z, cp, dxdt);
    CIA_CUDA_TRY(cudaGetLastError());
    return CIA_OK;
}
