// C-ABI evaluation and integration entry points of libcia (see include/cia.h).
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "cia_internal.h"

using namespace cia;

namespace {

cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

// Checks shared by every evaluation call: a usable plan on the current
// device, no pending asynchronous error, and a supported kernel shape.
cia_status check_plan(cia_plan *pl, int method) {
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    if (method != CIA_METHOD_CIA && method != CIA_METHOD_DIRECT)
        return fail(CIA_ERR_INVALID_ARG, "unknown method");
    if (method == CIA_METHOD_DIRECT && !pl->has_direct)
        return fail(CIA_ERR_INVALID_ARG, "plan was built without build_direct");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(CIA_ERR_INVALID_ARG, "plan belongs to another device");
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(pending, "pending asynchronous error");
    }
    if (method == CIA_METHOD_CIA && pl->miss_idx_bytes != 2)
        return fail(CIA_ERR_UNSUPPORTED, "communities above 65536 nodes are not supported");
    int optin = 0;
    CIA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
    const size_t need = (method == CIA_METHOD_CIA && pl->staging == 0)
                            ? pipeline_smem_bytes(pl, pl->ring_stages)
                            : stage_smem_bytes(pl, method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA);
    if (method == CIA_METHOD_DIRECT && pl->triadic &&
        (size_t)(pl->precision == CIA_FP64 ? 16 : 8) * (size_t)pl->max_comm > (size_t)optin - 1024)
        return fail(CIA_ERR_UNSUPPORTED, "the direct triadic term stages a whole community in shared memory; "
                                         "community too large");
    if (need > (size_t)optin - 1024)
        return fail(CIA_ERR_UNSUPPORTED, "largest community (" + std::to_string(pl->max_comm) +
                                             " nodes) does not fit the shared-memory community tile");
    return CIA_OK;
}

cia_status rhs_common(cia_plan *pl, int method, const double *x, double *dxdt, void *stream) {
    clear_error();
    cia_status st = check_plan(pl, method);
    if (st != CIA_OK) return st;
    if (!x || !dxdt) return fail(CIA_ERR_INVALID_ARG, "x or dxdt is NULL");
    if (x == dxdt) return fail(CIA_ERR_INVALID_ARG, "x and dxdt alias");
    cudaStream_t s = (cudaStream_t)stream;
    // the slot not holding the resident state is free between calls
    const int slot = pl->state_slot ^ 1;
    CIA_CUDA_TRY(launch_phasors_from_x(pl, x, false, slot, s));
    CIA_CUDA_TRY(launch_rhs(pl, method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA, slot, dxdt, s));
    return CIA_OK;
}

}  // namespace

extern "C" cia_status cia_rhs(cia_plan_t *plan, const double *x, double *dxdt, void *stream) {
    return rhs_common(plan, CIA_METHOD_CIA, x, dxdt, stream);
}

extern "C" cia_status cia_rhs_direct(cia_plan_t *plan, const double *x, double *dxdt, void *stream) {
    return rhs_common(plan, CIA_METHOD_DIRECT, x, dxdt, stream);
}

namespace {

cia_status ensure_omega_constants(cia_plan *pl, double dt, cudaStream_t s) {
    if (!pl->wdt_valid || pl->dt_cached != dt) {
        CIA_CUDA_TRY(launch_omega_constants(pl, dt, s));
        pl->dt_cached = dt;
        pl->wdt_valid = true;
        pl->prof_other++;
    }
    return CIA_OK;
}

// One RK4 stage launch, bracketed by profiling events while recording.
cia_status stage_launch(cia_plan *pl, int m, int stage, int slot, double dt, cudaStream_t s) {
    const bool rec = pl->prof_on && pl->prof_used < pl->prof_cap;
    if (rec) CIA_CUDA_TRY(cudaEventRecord(pl->prof_ev[2 * pl->prof_used], s));
    CIA_CUDA_TRY(launch_rk4_stage(pl, m, stage, slot, dt, s));
    if (rec) {
        CIA_CUDA_TRY(cudaEventRecord(pl->prof_ev[2 * pl->prof_used + 1], s));
        pl->prof_used++;
    }
    return CIA_OK;
}

void destroy_events(cia_plan *pl) {
    for (cudaEvent_t e : pl->prof_ev) cudaEventDestroy(e);
    pl->prof_ev.clear();
    pl->prof_cap = pl->prof_used = 0;
    pl->prof_on = false;
}

}  // namespace

extern "C" cia_status cia_state_load(cia_plan_t *pl, const double *x, void *stream) {
    clear_error();
    cia_status st = check_plan(pl, CIA_METHOD_CIA);
    if (st != CIA_OK && st != CIA_ERR_UNSUPPORTED) return st;
    if (!x) return fail(CIA_ERR_INVALID_ARG, "x is NULL");
    CIA_CUDA_TRY(launch_phasors_from_x(pl, x, true, 0, (cudaStream_t)stream));
    pl->state_slot = 0;
    pl->prof_other++;
    return CIA_OK;
}

extern "C" cia_status cia_state_store(cia_plan_t *pl, double *x, void *stream) {
    clear_error();
    if (!pl || !x) return fail(CIA_ERR_INVALID_ARG, "plan or x is NULL");
    CIA_CUDA_TRY(launch_scatter_master(pl, x, (cudaStream_t)stream));
    pl->prof_other++;
    return CIA_OK;
}

extern "C" cia_status cia_advance(cia_plan_t *pl, int method, double dt, int64_t nsteps, double *r_out,
                                  void *stream) {
    clear_error();
    cia_status st = check_plan(pl, method);
    if (st != CIA_OK) return st;
    if (!std::isfinite(dt)) return fail(CIA_ERR_NUMERIC, "dt is not finite");
    if (nsteps < 0) return fail(CIA_ERR_INVALID_ARG, "nsteps < 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int m = method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA;
    st = ensure_omega_constants(pl, dt, s);
    if (st != CIA_OK) return st;
    int slot = pl->state_slot;
    for (int64_t j = 0; j < nsteps; ++j) {
        for (int stage = 1; stage <= 4; ++stage) {
            st = stage_launch(pl, m, stage, slot, dt, s);
            if (st != CIA_OK) return st;
            slot ^= 1;
        }
        if (r_out) {
            CIA_CUDA_TRY(launch_order_parameter(pl, slot, r_out + j, s));
            pl->prof_other++;
        }
    }
    pl->state_slot = slot;
    return CIA_OK;
}

extern "C" cia_status cia_integrate(cia_plan_t *pl, int method, double *x, double dt, int64_t nsteps,
                                    double *r_out, void *stream) {
    clear_error();
    cia_status st = check_plan(pl, method);
    if (st != CIA_OK) return st;
    if (!x) return fail(CIA_ERR_INVALID_ARG, "x is NULL");
    if ((st = cia_state_load(pl, x, stream)) != CIA_OK) return st;
    if ((st = cia_advance(pl, method, dt, nsteps, r_out, stream)) != CIA_OK) return st;
    return cia_state_store(pl, x, stream);
}

extern "C" cia_status cia_profile_begin(cia_plan_t *pl, int64_t capacity) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    destroy_events(pl);
    pl->prof_other = 0;
    if (capacity <= 0) return CIA_OK;
    pl->prof_ev.resize(2 * capacity);
    for (auto &e : pl->prof_ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            e = nullptr;
            destroy_events(pl);
            return cuda_fail(err, "cudaEventCreate");
        }
    }
    pl->prof_cap = capacity;
    pl->prof_used = 0;
    pl->prof_on = true;
    return CIA_OK;
}

extern "C" cia_status cia_profile_end(cia_plan_t *pl, cia_profile *out) {
    clear_error();
    if (!pl || !out) return fail(CIA_ERR_INVALID_ARG, "plan or out is NULL");
    out->stage_launches = pl->prof_used;
    out->other_launches = pl->prof_other;
    out->stage_ms = 0.0;
    for (int64_t i = 0; i < pl->prof_used; ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(pl->prof_ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pl->prof_ev[2 * i], pl->prof_ev[2 * i + 1]);
        if (e != cudaSuccess) {
            destroy_events(pl);
            return cuda_fail(e, "profiling events");
        }
        out->stage_ms += ms;
    }
    destroy_events(pl);
    return CIA_OK;
}

extern "C" cia_status cia_integrate_host(cia_plan_t *pl, int method, double *x_host, double dt,
                                         int64_t nsteps, double *r_out_host, void *stream) {
    clear_error();
    if (!pl || !x_host) return fail(CIA_ERR_INVALID_ARG, "plan or x_host is NULL");
    if (nsteps < 0) return fail(CIA_ERR_INVALID_ARG, "nsteps < 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (r_out_host && nsteps > pl->d.r_cap) {
        if (pl->d.r_tmp) cudaFree(pl->d.r_tmp);
        pl->d.r_tmp = nullptr;
        pl->d.r_cap = 0;
        CIA_CUDA_TRY(cudaMalloc(&pl->d.r_tmp, nsteps * sizeof(double)));
        pl->d.r_cap = nsteps;
    }
    const size_t xb = (size_t)pl->n * sizeof(double);
    CIA_CUDA_TRY(cudaMemcpyAsync(pl->d.x_tmp, x_host, xb, cudaMemcpyHostToDevice, s));
    cia_status st = cia_integrate(pl, method, pl->d.x_tmp, dt, nsteps, r_out_host ? pl->d.r_tmp : nullptr, stream);
    if (st != CIA_OK) return st;
    CIA_CUDA_TRY(cudaMemcpyAsync(x_host, pl->d.x_tmp, xb, cudaMemcpyDeviceToHost, s));
    if (r_out_host && nsteps)
        CIA_CUDA_TRY(cudaMemcpyAsync(r_out_host, pl->d.r_tmp, nsteps * sizeof(double), cudaMemcpyDeviceToHost, s));
    return cia_sync(pl, stream);
}

extern "C" cia_status cia_sync(cia_plan_t *pl, void *stream) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    CIA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    CIA_CUDA_TRY(cudaGetLastError());
    int flag = 0;
    CIA_CUDA_TRY(cudaMemcpy(&flag, pl->d.err_flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        CIA_CUDA_TRY(cudaMemset(pl->d.err_flag, 0, sizeof(int)));
        return fail(CIA_ERR_TIMEOUT, "a device-side wait gave up; results since the last cia_sync are invalid");
    }
    return CIA_OK;
}
