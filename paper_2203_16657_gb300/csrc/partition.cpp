// Step P1's trade-off between communities and the CIA's cost per stage
// (Sec. "Community Detection (P1)": fewer, larger communities can pay off,
// more so for a high expansion order): a partition chosen by measuring the
// plan's own kernels.
//
// The modelled time of one stage is
//   T = c_tile * tiles + c_byte * (b_node N + b_miss nnz(S-) + b_inter nnz(S+)),
// a fixed cost per work tile (latency of its set-up, observable and node
// phase) plus a cost per byte the stage touches (index bytes, gathered
// phasors, node state).  With one tile per small community, T equals, up to a
// constant and the factor c_miss + c_inter (c_x = c_byte b_x), the Potts
// Hamiltonian of cia_detect_communities with
//   gamma p = c_miss / (c_miss + c_inter),  mu = c_tile / (c_miss + c_inter),
// because nnz(S-) = sum_c lambda_c (lambda_c - 1) - 2 e_in and
// nnz(S+) = 2 |E| - 2 e_in.  Equal link costs give back gamma p = 1/2, the
// setting that counts nnz(S) exactly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cia_internal.h"

using namespace cia;

namespace {

cia_status fail_p(cia_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

// Bytes one stage touches per node, per missing link and per inter link for
// a Kuramoto plan with p harmonics: index bytes, the gathered phasor, and the
// node's own state (as in the measurement's byte model).
void byte_weights(int precision, int p, double *b_node, double *b_miss, double *b_inter) {
    const double rb = precision == CIA_FP64 ? 8.0 : 4.0, c = 2.0 * rb * p;
    *b_node = c + 8.0 + rb + 0.75 * rb + rb + c + 0.25 * (8.0 + 8.0 - rb);
    *b_miss = 2.0 + c;
    *b_inter = 4.0 + c;
}

// Device time of one RK4 step (ms) of the CIA on a plan, from the state x
// (device, original order): two warm-up steps, then `steps` timed together.
cia_status time_plan(cia_plan_t *plan, const double *x_dev, double dt, int64_t steps, double *ms_per_step) {
    cia_status st = cia_state_load(plan, x_dev, nullptr);
    if (st != CIA_OK) return st;
    if ((st = cia_advance(plan, CIA_METHOD_CIA, dt, 2, nullptr, nullptr)) != CIA_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CIA_CUDA_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "cudaEventCreate");
    }
    float ms = 0.f;
    cudaError_t e = cudaEventRecord(e0, nullptr);
    if (e == cudaSuccess) {
        st = cia_advance(plan, CIA_METHOD_CIA, dt, steps, nullptr, nullptr);
        if (st == CIA_OK) e = cudaEventRecord(e1, nullptr);
        if (st == CIA_OK && e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (st == CIA_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != CIA_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "timing a candidate partition");
    *ms_per_step = (double)ms / (double)steps;
    return cia_sync(plan, nullptr);
}

struct Candidate {
    std::vector<int32_t> labels;
    cia_detect_report det{};
    cia_plan_info info{};
    double ms = INFINITY;
};

cia_status evaluate(const cia_graph *g, const cia_detect_options *dopt, const double *omega, const cia_coupling *cp,
                    const cia_options *opt, const double *x_dev, double dt, int64_t steps, Candidate &out) {
    out.labels.assign(g->n, -1);
    cia_status st = cia_detect_communities(g, dopt, out.labels.data(), &out.det);
    if (st != CIA_OK) return st;
    cia_plan_t *plan = nullptr;
    if ((st = cia_plan_create(g, out.labels.data(), omega, cp, opt, &plan)) != CIA_OK) return st;
    st = cia_plan_get_info(plan, &out.info);
    if (st == CIA_OK) st = time_plan(plan, x_dev, dt, steps, &out.ms);
    cia_plan_destroy(plan);
    return st;
}

}  // namespace

extern "C" cia_status cia_choose_partition(const cia_graph *g, const double *omega, const cia_coupling *coupling,
                                           const cia_options *opt, const double *x, double dt, int64_t steps,
                                           int32_t *labels, cia_partition_report *report) {
    clear_error();
    if (!g || !coupling || !x || !labels) return fail_p(CIA_ERR_INVALID_ARG, "a required pointer is NULL");
    if (coupling->model != CIA_MODEL_KURAMOTO && coupling->model != CIA_MODEL_KURAMOTO_HO)
        return fail_p(CIA_ERR_UNSUPPORTED, "the partition choice models the Kuramoto kernels");
    if (steps < 1 || !std::isfinite(dt)) return fail_p(CIA_ERR_INVALID_ARG, "need steps >= 1 and a finite dt");
    if (g->n < 2) return fail_p(CIA_ERR_INVALID_ARG, "need at least two nodes");
    double *x_dev = nullptr;
    CIA_CUDA_TRY(cudaMalloc(&x_dev, (size_t)g->n * sizeof(double)));
    struct Free {
        double *p;
        ~Free() { cudaFree(p); }
    } guard{x_dev};
    CIA_CUDA_TRY(cudaMemcpy(x_dev, x, (size_t)g->n * sizeof(double), cudaMemcpyHostToDevice));
    Candidate cand[3];
    cia_detect_options d0;
    cia_detect_options_default(&d0);
    // 0: the partition with the fewest entries of S (gamma p = 1/2, mu = 0)
    const double density = (double)g->rowptr[g->n] / ((double)g->n * (double)(g->n - 1));
    if (density > 0.0) d0.gamma = 0.5 / density;
    cia_status st = evaluate(g, &d0, omega, coupling, opt, x_dev, dt, steps, cand[0]);
    if (st != CIA_OK) return st;
    // 1: a coarser probe: a charge of one average block (directed pairs) per community
    cia_detect_options d1 = d0;
    {
        double pairs = 0.0;
        std::vector<int64_t> size(std::max<int64_t>(cand[0].det.communities, 1), 0);
        for (int64_t i = 0; i < g->n; ++i)
            if (cand[0].labels[i] >= 0) ++size[cand[0].labels[i]];
        for (int64_t s : size) pairs += (double)s * (double)(s - 1);
        d1.community_cost = std::max(1.0, pairs / (double)std::max<int64_t>(cand[0].det.communities, 1));
    }
    if ((st = evaluate(g, &d1, omega, coupling, opt, x_dev, dt, steps, cand[1])) != CIA_OK) return st;
    // fit c_tile and c_byte to the two measurements (per stage)
    const int precision = opt ? opt->precision : CIA_FP64;
    const int p = coupling->model == CIA_MODEL_KURAMOTO_HO ? std::max(coupling->p, 2) : coupling->p;
    double bn, bm, bi;
    byte_weights(precision, p, &bn, &bm, &bi);
    auto bytes = [&](const cia_plan_info &f) {
        return bn * (double)f.n + bm * (double)f.nnz_missing + bi * (double)f.nnz_inter;
    };
    const double t0 = cand[0].ms / 4.0, t1 = cand[1].ms / 4.0;
    const double a0 = (double)cand[0].info.n_tiles, a1 = (double)cand[1].info.n_tiles;
    const double b0 = bytes(cand[0].info), b1 = bytes(cand[1].info);
    double c_tile = 0.0, c_byte = 0.0;
    const double det = a0 * b1 - a1 * b0;
    if (std::fabs(det) > 1e-9 * std::fabs(a0 * b1) && std::fabs(det) > 0.0) {
        c_tile = (t0 * b1 - t1 * b0) / det;
        c_byte = (a0 * t1 - a1 * t0) / det;
    }
    if (!(c_byte > 0.0) || !(c_tile >= 0.0) || !std::isfinite(c_tile) || !std::isfinite(c_byte)) {
        // one cost explains the measurements: attribute the larger plan's time to bytes
        c_tile = std::max(0.0, std::isfinite(c_tile) ? c_tile : 0.0);
        c_byte = std::max(1e-30, (t0 - c_tile * a0) / std::max(b0, 1.0));
    }
    const double c_miss = c_byte * bm, c_inter = c_byte * bi;
    cia_detect_options d2 = d0;
    if (density > 0.0) d2.gamma = c_miss / (c_miss + c_inter) / density;
    d2.community_cost = c_tile / (c_miss + c_inter);
    if (!(d2.gamma > 0.0) || !std::isfinite(d2.gamma)) d2.gamma = d0.gamma;
    if (!std::isfinite(d2.community_cost)) d2.community_cost = 0.0;
    if ((st = evaluate(g, &d2, omega, coupling, opt, x_dev, dt, steps, cand[2])) != CIA_OK) return st;
    int best = 0;
    for (int k = 1; k < 3; ++k)
        if (cand[k].ms < cand[best].ms) best = k;
    std::memcpy(labels, cand[best].labels.data(), (size_t)g->n * sizeof(int32_t));
    if (report) {
        for (int k = 0; k < 3; ++k) {
            report->communities[k] = cand[k].det.communities;
            report->tiles[k] = cand[k].info.n_tiles;
            report->ms_per_step[k] = cand[k].ms;
            report->nnz_s[k] = cand[k].info.nnz_missing + cand[k].info.nnz_inter;
        }
        report->per_tile_us = c_tile * 1e3;
        report->per_byte_ps = c_byte * 1e9;
        report->gamma = d2.gamma;
        report->community_cost = d2.community_cost;
        report->probe_community_cost = d1.community_cost;
        report->chosen = best;
    }
    return CIA_OK;
}
