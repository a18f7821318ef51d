/*
 * cia_basis.h -- learned separable coupling basis for the Cucker--Smale model.
 *
 * Step P2 of the CIA (Sec. 3.2, App. A.6) expands the coupling weight in a
 * basis that separates the two agents: the paper uses the Fourier modes
 * e^{i pi <alpha, s>/L} of the Cucker--Smale weight
 *     eta(||s_l - s_m||^2) = K (sigma^2 + ||s_l - s_m||^2)^-beta
 * (eq. Cucker_Smale_etaExpansion).  This library replaces the Fourier modes
 * by a learned rank-R feature map,
 *     eta(||s_l - s_m||^2) ~ phi(s_l) . phi(s_m),
 *     phi(x) = W2 sin(W1 x + b1) + b2,     x in R^2, phi(x) in R^R,
 * a two-layer perceptron 2 -> 128 -> 64 whose second layer runs on the
 * tensor cores with BF16 weights and activations (FP32 accumulation); the
 * first layer (K = 2) runs on the FP32 cores.  With the sine activation the
 * hidden units are plane waves sin(<w_j, x> + b_j): the paper's Fourier
 * modes are one setting of the parameters (cia_basis_params_fourier), which
 * training then improves.  The same features
 * feed the community moments U_c, H_c (eq. Cucker_Smale_orderParams) and the
 * dense evaluation (eq. Cucker_Smale_fast_RHS), so the approximate pair
 * weight is symmetric and the CIA conserves momentum like the exact model.
 * Positions enter phi relative to a point common to the community (its
 * centroid), which leaves every pair difference unchanged.
 *
 * A basis object holds the FP32 master parameters and the Adam moments on
 * the device.  Every evaluation rounds W2 to BF16 first.
 * Training minimises the mean squared pair loss
 *     L = (1/B) sum_b (phi(a_b) . phi(c_b) - t_b)^2
 * over pairs (a_b, c_b) of positions with target t_b = eta(||a_b - c_b||^2).
 *
 * Conventions of include/cia.h apply (status codes, stream, ownership).
 */
#ifndef CIA_BASIS_H
#define CIA_BASIS_H

#include "cia.h"

#ifdef __cplusplus
extern "C" {
#endif

#define CIA_BASIS_IN 2
#define CIA_BASIS_HIDDEN 128
#define CIA_BASIS_RANK 64
/* Packed parameter vector, FP32, in this order:
 *   W1 [HIDDEN][IN] row-major, b1 [HIDDEN], W2 [RANK][HIDDEN] row-major, b2 [RANK]. */
#define CIA_BASIS_PARAMS (CIA_BASIS_HIDDEN * CIA_BASIS_IN + CIA_BASIS_HIDDEN + \
                          CIA_BASIS_RANK * CIA_BASIS_HIDDEN + CIA_BASIS_RANK)

typedef struct cia_basis cia_basis_t;

/* Adam (Kingma & Ba) on the FP32 master parameters. */
typedef struct {
    double lr;                  /* step size, e.g. 1e-3 */
    double beta1, beta2;        /* moment decay rates, e.g. 0.9 and 0.999 */
    double eps;                 /* e.g. 1e-8 */
} cia_adam_options;

typedef struct {
    int64_t batch;              /* pairs per optimiser step, a multiple of 64 (e.g. 16384) */
    int64_t epochs;             /* passes over the pair array */
    cia_adam_options adam;      /* adam.lr is the step size of the first step */
    double lr_final;            /* step size of the last step, geometric decay in between
                                   (0 = constant adam.lr) */
} cia_fit_options;

typedef struct {
    int64_t steps;              /* optimiser steps taken */
    double first_loss;          /* loss of the first batch (before its update) */
    double last_epoch_loss;     /* mean batch loss over the last epoch */
} cia_fit_report;

/* Parameters (host, CIA_BASIS_PARAMS floats) that make phi the rank-64
 * Fourier basis of the weight eta(y) = K (sigma^2 + y)^-beta on the box
 * [-L, L]^2 of differences (App. A.6): the coefficients c_alpha of the
 * periodic extension (rectangle rule on a 256 x 256 grid) of the 32 strongest
 * mode pairs +-alpha, each as two hidden units sin(pi <alpha, x> / L + pi/2)
 * and sin(pi <alpha, x> / L) weighted sqrt(2 c_alpha) (alpha = 0: the bias
 * sqrt(c_0)), so that phi(x) . phi(y) is the truncated series of
 * eta(||x - y||^2).  The remaining hidden units get seeded small random
 * frequencies and zero output weights.  Host-only, no device work. */
cia_status cia_basis_params_fourier(double K, double sigma, double beta, double L, uint64_t seed,
                                    float *params);

/* Create a basis on the current device from host parameters (packed as
 * above, CIA_BASIS_PARAMS floats); Adam moments start at zero. */
cia_status cia_basis_create(const float *params, cia_basis_t **out);

/* Release the basis (NULL is a no-op). */
cia_status cia_basis_destroy(cia_basis_t *basis);

/* Copy the FP32 master parameters to params (host, CIA_BASIS_PARAMS floats). */
cia_status cia_basis_get_params(const cia_basis_t *basis, float *params);

/* phi(x) for `count` inputs.  x: device, count x 2 floats; phi: device,
 * count x RANK floats (row b = phi(x_b), before any rounding of the output).
 * Hidden activations are rounded to BF16 before the second layer. */
cia_status cia_basis_features(cia_basis_t *basis, const float *x, int64_t count, float *phi,
                              void *stream);

/* Gradient of the pair loss L over `count` pairs (count > 0, any size).
 * pairs: device, count x 5 floats (a_x, a_y, c_x, c_y, t) per pair.
 * grad: device, CIA_BASIS_PARAMS floats (same packing as the parameters).
 * loss: device, one double (L of the evaluated model), or NULL.
 * The backward products run on the tensor cores with BF16 operands. */
cia_status cia_basis_pair_grad(cia_basis_t *basis, const float *pairs, int64_t count, float *grad,
                               double *loss, void *stream);

/* One Adam step on the master parameters with gradient grad (device,
 * CIA_BASIS_PARAMS floats). */
cia_status cia_basis_adam_step(cia_basis_t *basis, const float *grad, const cia_adam_options *opt,
                               void *stream);

/* Fit the basis to `count` pairs (device, layout of cia_basis_pair_grad):
 * opt->epochs passes, each cutting the array into consecutive batches of
 * opt->batch pairs (a last partial batch is used as it is), one Adam step per
 * batch.  Synchronises the stream and fills *report (may be NULL). */
cia_status cia_basis_fit(cia_basis_t *basis, const float *pairs, int64_t count,
                         const cia_fit_options *opt, cia_fit_report *report, void *stream);

/* ---- the basis inside a Cucker--Smale plan -------------------------------- */

/* Use the basis' current parameters (copied, rounded to BF16 on use) for the
 * plan's CIA.  Resets the plan's check state.  The copy is ordered after all
 * work issued to the basis on the legacy default stream; synchronise other
 * streams first. */
cia_status cia_plan_set_basis(cia_plan_t *plan, const cia_basis_t *basis);

/* Draw `count` training pairs (layout of cia_basis_pair_grad) from the plan's
 * resident state: node i uniform over the nodes that belong to a community,
 * partner l uniform over the other nodes of i's community, positions relative
 * to that community's centroid, target t = eta(||s_i - s_l||^2) with the
 * plan's K, sigma, beta.  The generator is SplitMix64 (Steele, Lea and Flood
 * 2014) on the counter seed + 2q (+1).  pairs: device, count x 5 floats. */
cia_status cia_plan_sample_pairs(cia_plan_t *plan, int64_t count, uint64_t seed, float *pairs,
                                 void *stream);

/* Sampled check of the learned basis during cia_advance / cia_integrate with
 * the CIA (needs opt.build_direct): before step 0 and every `every` steps,
 * for up to 512 fixed community nodes m (evenly spaced in the permuted order)
 *   err = max_m |dense_m - (1/N) sum_{l in c(m), l != m} eta (v_l - v_m)|,
 *   ref = max_m |(1/N) sum_{l in N(m)} eta (v_l - v_m)|      (max over both components),
 * the first being exactly the CIA's deviation from the direct right-hand side
 * (its sparse corrections are exact).  If err > bound * ref the remaining
 * steps, and later calls, use the direct method (cia_plan_set_check or
 * cia_plan_set_basis re-arms the CIA).  every = 0 turns the check off. */
cia_status cia_plan_set_check(cia_plan_t *plan, int64_t every, double bound);

typedef struct {
    int64_t checks;             /* checks run since the last set_check / set_basis */
    double last_error;          /* err / ref of the last check */
    double max_error;           /* largest err / ref */
    int fell_back;              /* nonzero once a check failed */
    int64_t fallback_step;      /* step (within the call that failed) at which it failed, -1 if none */
} cia_check_report;

cia_status cia_plan_get_check(const cia_plan_t *plan, cia_check_report *report);

typedef struct {
    double dt;                  /* step of the direct RK4 trajectory */
    int64_t steps;              /* its length in steps */
    int64_t snapshots;          /* states where pairs are drawn: steps 0, steps/snapshots, ... */
    int64_t pairs;              /* pairs in total, split evenly over the snapshots */
    uint64_t seed;
    cia_fit_options fit;
} cia_learn_options;

typedef struct {
    int64_t pairs;              /* pairs drawn */
    cia_fit_report fit;
} cia_learn_report;

/* Learn the basis from the dynamics themselves: load x0 (device, n x 4
 * doubles, original order), integrate it with the DIRECT method (needs
 * opt.build_direct) for opt->steps RK4 steps of opt->dt, drawing
 * opt->pairs / opt->snapshots pairs (cia_plan_sample_pairs) at each snapshot,
 * fit the basis to all of them (cia_basis_fit) and set it as the plan's basis.
 * The plan's resident state is left at the end of the trajectory.
 * Synchronises the stream; *report may be NULL. */
cia_status cia_learn_fit(cia_plan_t *plan, cia_basis_t *basis, const double *x0,
                         const cia_learn_options *opt, cia_learn_report *report, void *stream);

/* Wait for the basis' work on `stream`; CIA_ERR_TIMEOUT (flag cleared) if a
 * bounded tensor-core wait of its kernels gave up since the last check. */
cia_status cia_basis_sync(cia_basis_t *basis, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CIA_BASIS_H */
