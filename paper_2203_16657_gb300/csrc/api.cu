// C-ABI evaluation and integration entry points of libcia (see include/cia.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "cia_internal.h"

using namespace cia;

namespace {

cia_status fail(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

// Checks shared by every evaluation call: a usable plan on the current
// device, no pending asynchronous error, and a supported kernel shape.
// A usable plan on the current device with no pending asynchronous error.
cia_status check_device(cia_plan *pl) {
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    int dev = -1;
    CIA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != pl->device) return fail(CIA_ERR_INVALID_ARG, "plan belongs to another device");
    cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(pending, "pending asynchronous error");
    }
    return CIA_OK;
}

cia_status check_plan(cia_plan *pl, int method) {
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    if (method != CIA_METHOD_CIA && method != CIA_METHOD_DIRECT)
        return fail(CIA_ERR_INVALID_ARG, "unknown method");
    if (method == CIA_METHOD_DIRECT && !pl->has_direct)
        return fail(CIA_ERR_INVALID_ARG, "plan was built without build_direct");
    cia_status st = check_device(pl);
    if (st != CIA_OK) return st;
    if (method == CIA_METHOD_CIA && pl->miss_idx_bytes != 2)
        return fail(CIA_ERR_UNSUPPORTED, "communities above 65536 nodes are not supported");
    int optin = 0;
    CIA_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, pl->device));
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        if (method == CIA_METHOD_CIA && !pl->cs_has_basis)
            return fail(CIA_ERR_INVALID_ARG, "the Cucker-Smale CIA needs a basis (cia_plan_set_basis)");
        if (method == CIA_METHOD_CIA && cs_stage_smem_bytes(pl) > (size_t)optin - 4096)
            return fail(CIA_ERR_UNSUPPORTED, "largest community (" + std::to_string(pl->max_comm) +
                                                 " nodes) does not fit the shared-memory community tile");
        return CIA_OK;
    }
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
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        CIA_CUDA_TRY(cs_launch_load(pl, x, false, slot, s));
        if (method == CIA_METHOD_CIA) {
            // the feature buffer is shared with the resident state
            CIA_CUDA_TRY(cs_launch_features(pl, slot, s));
            pl->cs_feat_valid = false;
        }
        CIA_CUDA_TRY(cs_launch_rhs(pl, method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA, slot, dxdt, s));
        return CIA_OK;
    }
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
    if (pl->model == CIA_MODEL_CUCKER_SMALE) CIA_CUDA_TRY(cs_launch_stage(pl, m, stage, slot, dt, s));
    else CIA_CUDA_TRY(launch_rk4_stage(pl, m, stage, slot, dt, s));
    if (rec) {
        CIA_CUDA_TRY(cudaEventRecord(pl->prof_ev[2 * pl->prof_used + 1], s));
        pl->prof_used++;
    }
    return CIA_OK;
}

// Learned-basis check at the resident state: returns err / ref (see cia_plan_set_check).
cia_status cs_check(cia_plan *pl, cudaStream_t s, double *ratio) {
    CIA_CUDA_TRY(cs_launch_check(pl, pl->state_slot, s));
    pl->prof_other++;
    std::vector<double> h(2 * pl->cs_check_count);
    CIA_CUDA_TRY(cudaMemcpyAsync(h.data(), pl->d.cs_check_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    CIA_CUDA_TRY(cudaStreamSynchronize(s));
    double err = 0.0, ref = 0.0;
    for (int64_t k = 0; k < pl->cs_check_count; ++k) {
        err = std::max(err, h[2 * k]);
        ref = std::max(ref, h[2 * k + 1]);
    }
    *ratio = ref > 0.0 ? err / ref : (err > 0.0 ? INFINITY : 0.0);
    return CIA_OK;
}

// cia_advance for the Cucker--Smale model: CIA stages with the learned basis
// (features computed first if the resident state has none), the sampled
// check every check_every steps, direct stages after a failed check.
cia_status cs_advance(cia_plan *pl, int method, double dt, int64_t nsteps, double *r_out, cudaStream_t s) {
    if (r_out) return fail(CIA_ERR_INVALID_ARG, "r_out must be NULL for the Cucker-Smale model");
    bool use_cia = method == CIA_METHOD_CIA && !pl->fell_back;
    int slot = pl->state_slot;
    cia_status st;
    for (int64_t j = 0; j < nsteps; ++j) {
        if (use_cia && !pl->cs_feat_valid) {
            CIA_CUDA_TRY(cs_launch_features(pl, slot, s));
            pl->prof_other++;
            pl->cs_feat_valid = true;
        }
        if (use_cia && pl->check_every > 0 && j % pl->check_every == 0) {
            pl->state_slot = slot;
            double ratio = 0.0;
            if ((st = cs_check(pl, s, &ratio)) != CIA_OK) return st;
            pl->checks++;
            pl->check_last = ratio;
            pl->check_max = std::max(pl->check_max, ratio);
            if (!(ratio <= pl->check_bound)) {
                pl->fell_back = true;
                pl->fallback_step = j;
                use_cia = false;
            }
        }
        const int m = use_cia ? Method::CIA : Method::DIRECT;
        if (!use_cia) pl->cs_feat_valid = false;
        for (int stage = 1; stage <= 4; ++stage) {
            if ((st = stage_launch(pl, m, stage, slot, dt, s)) != CIA_OK) return st;
            slot ^= 1;
        }
    }
    pl->state_slot = slot;
    if (method == CIA_METHOD_CIA && pl->fell_back)
        return fail(CIA_ERR_FALLBACK, "the learned basis failed its check (err/ref " + std::to_string(pl->check_last) +
                                          " > " + std::to_string(pl->check_bound) +
                                          "); the direct method was used from step " +
                                          std::to_string(pl->fallback_step) + " of the failing call");
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
    cia_status st = check_device(pl);
    if (st != CIA_OK) return st;
    if (!x) return fail(CIA_ERR_INVALID_ARG, "x is NULL");
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        CIA_CUDA_TRY(cs_launch_load(pl, x, true, 0, (cudaStream_t)stream));
        pl->cs_feat_valid = false;   // features are computed by the first CIA step
    } else {
        CIA_CUDA_TRY(launch_phasors_from_x(pl, x, true, 0, (cudaStream_t)stream));
    }
    pl->state_slot = 0;
    pl->prof_other++;
    return CIA_OK;
}

extern "C" cia_status cia_state_store(cia_plan_t *pl, double *x, void *stream) {
    clear_error();
    if (!pl || !x) return fail(CIA_ERR_INVALID_ARG, "plan or x is NULL");
    if (pl->model == CIA_MODEL_CUCKER_SMALE) CIA_CUDA_TRY(cs_launch_store(pl, x, (cudaStream_t)stream));
    else CIA_CUDA_TRY(launch_scatter_master(pl, x, (cudaStream_t)stream));
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
    if (pl->model == CIA_MODEL_CUCKER_SMALE) return cs_advance(pl, method, dt, nsteps, r_out, s);
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
    st = cia_advance(pl, method, dt, nsteps, r_out, stream);
    if (st != CIA_OK && st != CIA_ERR_FALLBACK) return st;
    const std::string msg = cia_last_error();
    cia_status st2 = cia_state_store(pl, x, stream);
    if (st2 != CIA_OK) return st2;
    if (st == CIA_ERR_FALLBACK) set_error(msg);
    return st;
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
    const size_t xb = (size_t)pl->n * pl->state_dim * sizeof(double);
    CIA_CUDA_TRY(cudaMemcpyAsync(pl->d.x_tmp, x_host, xb, cudaMemcpyHostToDevice, s));
    cia_status st = cia_integrate(pl, method, pl->d.x_tmp, dt, nsteps, r_out_host ? pl->d.r_tmp : nullptr, stream);
    if (st != CIA_OK && st != CIA_ERR_FALLBACK) return st;
    const std::string msg = cia_last_error();
    CIA_CUDA_TRY(cudaMemcpyAsync(x_host, pl->d.x_tmp, xb, cudaMemcpyDeviceToHost, s));
    if (r_out_host && nsteps)
        CIA_CUDA_TRY(cudaMemcpyAsync(r_out_host, pl->d.r_tmp, nsteps * sizeof(double), cudaMemcpyDeviceToHost, s));
    cia_status st2 = cia_sync(pl, stream);
    if (st2 != CIA_OK) return st2;
    if (st == CIA_ERR_FALLBACK) set_error(msg);
    return st;
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
