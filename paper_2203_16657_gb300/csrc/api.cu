// C-ABI evaluation and integration entry points of libcia (see include/cia.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cia_internal.h"
#include "sync.cuh"

using namespace cia;

namespace cia {

void invalidate_graphs(cia_plan *pl) {
    if (pl->graph_exec) cudaGraphExecDestroy(pl->graph_exec);
    pl->graph_exec = nullptr;
    pl->graph_method = pl->graph_slot = -1;
    pl->graph_r_out = nullptr;
}

}  // namespace cia

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
    // the general-coupling stage kernel reads oversized communities from global memory
    if (pl->model == CIA_MODEL_POLYNOMIAL) return CIA_OK;
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        if (method == CIA_METHOD_CIA && !pl->cs_has_basis)
            return fail(CIA_ERR_INVALID_ARG, "the Cucker-Smale CIA needs a basis (cia_plan_set_basis)");
        if (method == CIA_METHOD_CIA && cs_stage_smem_bytes(pl) > (size_t)optin - 4096)
            return fail(CIA_ERR_UNSUPPORTED, "largest community (" + std::to_string(pl->max_comm) +
                                                 " nodes) does not fit the shared-memory community tile");
        return CIA_OK;
    }
    const size_t need = (method == CIA_METHOD_CIA && pl->staging == 3)   ? pipeline_smem_bytes(pl, pl->ring_stages)
                        : (method == CIA_METHOD_CIA && pl->staging == 2) ? window_smem_bytes(pl)
                        : (method == CIA_METHOD_CIA && pl->staging == 4) ? stream_smem_bytes(pl)
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
    if (pl->model == CIA_MODEL_POLYNOMIAL) {
        CIA_CUDA_TRY(gc_launch_load(pl, x, false, slot, s));
        CIA_CUDA_TRY(gc_launch_rhs(pl, method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA, slot, dxdt, s));
        return CIA_OK;
    }
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
    else if (pl->model == CIA_MODEL_POLYNOMIAL) CIA_CUDA_TRY(gc_launch_stage(pl, m, stage, slot, dt, s));
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

// Capture (or reuse) the CUDA graph of one RK4 step: four stage launches
// starting from `slot`, then the order parameters when r_out is given.
cia_status ensure_step_graph(cia_plan *pl, int m, int slot, double dt, double *r_out) {
    if (pl->graph_exec && pl->graph_method == m && pl->graph_slot == slot && pl->graph_dt == dt &&
        pl->graph_r == (r_out != nullptr) && pl->graph_r_out == r_out)
        return CIA_OK;
    invalidate_graphs(pl);
    if (!pl->capture_stream) CIA_CUDA_TRY(cudaStreamCreateWithFlags(&pl->capture_stream, cudaStreamNonBlocking));
    cudaStream_t cs = pl->capture_stream;
    CIA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    int sl = slot;
    for (int stage = 1; stage <= 4 && err == cudaSuccess; ++stage) {
        err = pl->model == CIA_MODEL_POLYNOMIAL ? gc_launch_stage(pl, m, stage, sl, dt, cs)
                                                : launch_rk4_stage(pl, m, stage, sl, dt, cs);
        sl ^= 1;
    }
    if (err == cudaSuccess && r_out) err = launch_order_parameters(pl, sl, r_out, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(cs, &graph);
    if (err != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(err, "kernel launch during graph capture");
    }
    if (end != cudaSuccess) return cuda_fail(end, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t inst = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) return cuda_fail(inst, "cudaGraphInstantiate");
    pl->graph_exec = exec;
    pl->graph_method = m;
    pl->graph_slot = slot;
    pl->graph_dt = dt;
    pl->graph_r = r_out != nullptr;
    pl->graph_r_out = r_out;
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
    } else if (pl->model == CIA_MODEL_POLYNOMIAL) {
        CIA_CUDA_TRY(gc_launch_load(pl, x, true, 0, (cudaStream_t)stream));
    } else {
        CIA_CUDA_TRY(launch_phasors_from_x(pl, x, true, 0, (cudaStream_t)stream));
    }
    pl->state_slot = 0;
    pl->needs_load = false;
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
    if (pl->needs_load) return fail(CIA_ERR_INVALID_ARG, "the tiling changed: load a state first (cia_state_load)");
    cudaStream_t s = (cudaStream_t)stream;
    if (pl->model == CIA_MODEL_CUCKER_SMALE) return cs_advance(pl, method, dt, nsteps, r_out, s);
    const int m = method == CIA_METHOD_DIRECT ? Method::DIRECT : Method::CIA;
    if (pl->model == CIA_MODEL_POLYNOMIAL) {
        if (r_out) return fail(CIA_ERR_INVALID_ARG, "r_out must be NULL for the polynomial and Fourier couplings");
    } else {
        st = ensure_omega_constants(pl, dt, s);
        if (st != CIA_OK) return st;
    }
    if (r_out) CIA_CUDA_TRY(cudaMemsetAsync(pl->d.r_counter, 0, sizeof(int64_t), s));
    const bool profiling = pl->prof_on && pl->prof_used < pl->prof_cap;
    int slot = pl->state_slot;
    // a step graph captured by an earlier call for the same method, slot, dt
    // and order-parameter buffer is replayed from the first step on
    const bool graph_ready = pl->graph_exec && pl->graph_method == m && pl->graph_slot == slot &&
                             pl->graph_dt == dt && pl->graph_r == (r_out != nullptr) && pl->graph_r_out == r_out;
    const bool graphs = pl->use_graphs == 0 && !profiling && (nsteps >= 2 || graph_ready);
    for (int64_t j = 0; j < nsteps; ++j) {
        if (graphs && (j >= 1 || graph_ready)) {
            // steps 1.. replay one captured step (step 0 of the capturing
            // call ran plain launches, which also configured every kernel);
            // 4 stages return the slot
            if ((st = ensure_step_graph(pl, m, slot, dt, r_out)) != CIA_OK) return st;
            CIA_CUDA_TRY(cudaGraphLaunch(pl->graph_exec, s));
            pl->prof_other += 4 + (r_out ? 1 : 0);
            continue;
        }
        for (int stage = 1; stage <= 4; ++stage) {
            st = stage_launch(pl, m, stage, slot, dt, s);
            if (st != CIA_OK) return st;
            slot ^= 1;
        }
        if (r_out) {
            CIA_CUDA_TRY(launch_order_parameters(pl, slot, r_out, s));
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
    // one order parameter per step and instance, staged in mapped pinned host
    // memory that the order-parameter kernel writes through its device alias
    const int64_t r_count = nsteps * (int64_t)std::max<int64_t>(pl->B, 1);
    if (r_out_host && r_count > pl->d.r_cap) {
        if (pl->d.r_tmp_host) cudaFreeHost(pl->d.r_tmp_host);
        pl->d.r_tmp = pl->d.r_tmp_host = nullptr;
        pl->d.r_cap = 0;
        CIA_CUDA_TRY(cudaHostAlloc((void **)&pl->d.r_tmp_host, (size_t)r_count * sizeof(double), cudaHostAllocMapped));
        CIA_CUDA_TRY(cudaHostGetDevicePointer((void **)&pl->d.r_tmp, pl->d.r_tmp_host, 0));
        pl->d.r_cap = r_count;
    }
    const size_t xb = (size_t)pl->n * pl->state_dim * sizeof(double);
    CIA_CUDA_TRY(cudaMemcpyAsync(pl->d.x_tmp, x_host, xb, cudaMemcpyHostToDevice, s));
    cia_status st = cia_integrate(pl, method, pl->d.x_tmp, dt, nsteps, r_out_host ? pl->d.r_tmp : nullptr, stream);
    if (st != CIA_OK && st != CIA_ERR_FALLBACK) return st;
    const std::string msg = cia_last_error();
    CIA_CUDA_TRY(cudaMemcpyAsync(x_host, pl->d.x_tmp, xb, cudaMemcpyDeviceToHost, s));
    cia_status st2 = cia_sync(pl, stream);
    if (st2 != CIA_OK) return st2;
    if (r_out_host && r_count) std::memcpy(r_out_host, pl->d.r_tmp_host, (size_t)r_count * sizeof(double));
    if (st == CIA_ERR_FALLBACK) set_error(msg);
    return st;
}

extern "C" cia_status cia_plan_set_weights(cia_plan_t *pl, const double *alpha, const double *beta) {
    clear_error();
    cia_status st = check_device(pl);
    if (st != CIA_OK) return st;
    if (pl->model != CIA_MODEL_POLYNOMIAL || pl->gc_basis != 0)
        return fail(CIA_ERR_UNSUPPORTED, "rank-one link weights are for the polynomial models");
    const int64_t n = pl->n;
    if (alpha || beta) {
        std::vector<double> w(2 * n);
        for (int64_t m = 0; m < n; ++m) {
            const int32_t i = pl->perm[m];
            w[m] = alpha ? alpha[i] : 1.0;
            w[n + m] = beta ? beta[i] : 1.0;
            if (!std::isfinite(w[m]) || !std::isfinite(w[n + m])) return fail(CIA_ERR_NUMERIC, "a weight is not finite");
        }
        if (!pl->d.gc_alpha) {
            void *p = nullptr;
            CIA_CUDA_TRY(cudaMalloc(&p, (size_t)2 * n * sizeof(double)));
            pl->allocations.push_back(p);
            pl->device_bytes += (int64_t)(2 * n * sizeof(double));
            pl->d.gc_alpha = static_cast<double *>(p);
            pl->d.gc_beta = pl->d.gc_alpha + n;
        }
        CIA_CUDA_TRY(cudaMemcpy(pl->d.gc_alpha, w.data(), (size_t)2 * n * sizeof(double), cudaMemcpyHostToDevice));
    }
    pl->gc_weighted = alpha || beta;
    // the window holds one more row when weighted; the moments change
    pl->staging = pl->staging_req == 1 ? 1 : 2;
    pl->needs_load = true;
    invalidate_graphs(pl);
    return CIA_OK;
}

extern "C" cia_status cia_sync(cia_plan_t *pl, void *stream) {
    clear_error();
    if (!pl) return fail(CIA_ERR_INVALID_ARG, "plan is NULL");
    // the flag lives in mapped pinned host memory: once the stream's work has
    // finished, whatever a kernel wrote there is visible to the host
    CIA_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    CIA_CUDA_TRY(cudaGetLastError());
    volatile int *flag_host = pl->d.err_flag_host;
    const int flag = flag_host ? *flag_host : 0;
    if (flag) {
        *flag_host = 0;
        return fail(CIA_ERR_TIMEOUT, "a device-side wait gave up; results since the last cia_sync are invalid");
    }
    return CIA_OK;
}

extern "C" cia_status cia_plan_autotune(cia_plan_t *pl, const double *x, double dt, int64_t steps,
                                        cia_tune_report *report, void *stream) {
    clear_error();
    cia_status st = check_plan(pl, CIA_METHOD_CIA);
    if (st != CIA_OK && st != CIA_ERR_UNSUPPORTED) return st;
    if (!x) return fail(CIA_ERR_INVALID_ARG, "x is NULL");
    if (steps < 1 || !std::isfinite(dt)) return fail(CIA_ERR_INVALID_ARG, "need steps >= 1 and a finite dt");
    if (pl->model == CIA_MODEL_POLYNOMIAL)
        return fail(CIA_ERR_UNSUPPORTED, "no tuning candidates for the polynomial and Fourier couplings");
    struct Cand { int tn, tib, staging; };
    std::vector<Cand> cands;
    if (pl->model == CIA_MODEL_CUCKER_SMALE) {
        for (int tn : {64, 128})
            for (int tib : {16384, 32768}) cands.push_back({tn, tib, 1});
    } else {
        for (int tib : {32768, 65536, 98304}) cands.push_back({256, tib, 2});
        cands.push_back({128, 32768, 2});
        cands.push_back({64, 16384, 2});
        cands.push_back({256, 32768, 3});
        cands.push_back({256, 32768, 1});
        for (int tib : {49152, 65536}) cands.push_back({256, tib, 4});
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CIA_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
        }
    } guard{e0, e1};
    double best = INFINITY, worst = 0.0;
    int bi = -1, tried = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        const Cand &c = cands[i];
        if ((st = cia_plan_retile(pl, c.tn, c.tib, c.staging)) != CIA_OK) return st;
        if (c.staging != pl->staging) continue;   // the kernel does not fit: another candidate covers its fallback
        if ((st = cia_state_load(pl, x, stream)) != CIA_OK) return st;
        if ((st = check_plan(pl, CIA_METHOD_CIA)) != CIA_OK) continue;   // does not fit this GPU
        if ((st = cia_advance(pl, CIA_METHOD_CIA, dt, 2, nullptr, stream)) != CIA_OK && st != CIA_ERR_FALLBACK)
            return st;
        CIA_CUDA_TRY(cudaEventRecord(e0, s));
        if ((st = cia_advance(pl, CIA_METHOD_CIA, dt, steps, nullptr, stream)) != CIA_OK && st != CIA_ERR_FALLBACK)
            return st;
        CIA_CUDA_TRY(cudaEventRecord(e1, s));
        CIA_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        CIA_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if ((st = cia_sync(pl, stream)) != CIA_OK) return st;
        const double per = (double)ms / (double)steps;
        ++tried;
        worst = std::max(worst, per);
        if (per < best) {
            best = per;
            bi = (int)i;
        }
    }
    if (bi < 0) return fail(CIA_ERR_UNSUPPORTED, "no candidate tiling fits this GPU");
    const Cand &c = cands[bi];
    if ((st = cia_plan_retile(pl, c.tn, c.tib, c.staging)) != CIA_OK) return st;
    if ((st = cia_state_load(pl, x, stream)) != CIA_OK) return st;
    CIA_CUDA_TRY(cudaStreamSynchronize(s));
    if (report) {
        report->candidates = tried;
        report->tile_nodes = c.tn;
        report->tile_index_bytes = c.tib;
        report->staging = pl->staging;
        report->best_ms_per_step = best;
        report->worst_ms_per_step = worst;
    }
    return CIA_OK;
}

namespace {

// An mbarrier that nothing arrives on: the bounded wait gives up after
// limit_ns and reports it through the plan's error flag, exactly as a stage
// kernel whose producer never delivers.
__global__ void selftest_wait_kernel(int *err_flag, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) cia::mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0 && !cia::mbar_wait_bounded(&bar, 0, limit_ns)) atomicExch(err_flag, 1);
}

}  // namespace

extern "C" cia_status cia_selftest_bounded_wait(cia_plan_t *pl, int64_t limit_ns, void *stream) {
    clear_error();
    cia_status st = check_device(pl);
    if (st != CIA_OK) return st;
    if (limit_ns < 1000 || limit_ns > 1000000000)
        return fail(CIA_ERR_INVALID_ARG, "limit_ns must be in [1e3, 1e9]");
    selftest_wait_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(pl->d.err_flag, (uint64_t)limit_ns);
    CIA_CUDA_TRY(cudaGetLastError());
    return CIA_OK;
}
