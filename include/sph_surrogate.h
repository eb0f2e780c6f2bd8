/*
 * sph_surrogate.h -- C ABI of the learned k-step surrogate and of its dense
 * BF16 contraction on the tensor cores.
 *
 * The paper has no learned component; this library adds one: a
 * message-passing network over the SPH neighbour graph that advances the
 * particle state by k plain steps at once, trained on trajectories of the
 * plain method, with the plain method as its fallback and judge.  Return
 * values and error messages follow sph.h (SPH_OK or a negative SPH_E* code,
 * message from sph_last_error()).
 */
#ifndef SPH_SURROGATE_H
#define SPH_SURROGATE_H

#include "sph.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Dense contraction C = A B^T on the tensor cores (tcgen05, BF16 operands,
 * FP32 accumulation).  A: M x K BF16, row-major with leading dimension lda;
 * B: N x K BF16, row-major, ldb; C: M x N FP32, row-major, ldc.  All three are
 * device pointers owned by the caller; A and B 16-byte aligned, lda and ldb
 * multiples of 8.  N in {16, 32, 64, 128, 256}; K a multiple of 16.  With
 * accumulate = 0, C is overwritten; with accumulate = 1, the products are
 * added to C with atomics, and K may be split across CTAs in ranges of
 * k_split (a multiple of 64; 0 = no split).  The call only queues the work on
 * `stream`; a tensor-core wait that exceeded one second sets bit 0 of the
 * device word *err_dev, which the caller reads. */
int sph_mm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                int k_split, int accumulate, void *stream, unsigned *err_dev);

/* State snapshots in original particle order, in device memory owned by the
 * caller: x and u of n * dim doubles (particle-major, each instance in its
 * own frame), rho of n doubles.  sph_snapshot queues the copy; 
 * sph_load_snapshot replaces the handle's state (the next step rebuilds the
 * lists) without changing the step counter. */
int sph_snapshot(sph_handle h, double *x_dev, double *u_dev, double *rho_dev);
int sph_load_snapshot(sph_handle h, const double *x_dev, const double *u_dev, const double *rho_dev);

/* Attaches the learned surrogate to a single-instance handle (or replaces
 * its parameters).  weights: nweights host doubles in the flat format of
 * paper_1702_07760_gb300/surrogate_layout.py (held on the device as FP32
 * master weights, with BF16 copies for the tensor cores); norm: the
 * normalisation block of that format (6 dim + 14 doubles: mu_in, sd_in,
 * mu_out, sd_out, k_ref, the jump time T = k dt, sd_edge_u, sd_edge_rho).
 * Resets the Adam state.  The network, for every particle, maps the state
 * and the plain method's rates at that state (acceleration a, density rate)
 * to its increments over the jump: encoder, two rounds of edge messages over
 * the neighbour pairs closer than 2h (edge inputs: relative position,
 * distance, phase change, velocity and density differences; summed, scaled
 * by 1/k_ref) with a residual node update, decoder giving corrections to the
 * explicit jump: du = T a + c_u, drho = T Drho/Dt + c_rho, and
 * dx = T (u + du / 2) + c_x. */
int sph_surrogate_init(sph_handle h, const double *weights, int64_t nweights, const double *norm, int64_t nnorm);

/* Copies the current FP32 master weights to host doubles. */
int sph_surrogate_get_weights(sph_handle h, double *weights, int64_t nweights);

/* Network increments at the current state, in original particle order:
 * out[p * (2 dim + 1) + c] holds dx (dim), du (dim) and drho (1); walls get
 * zero dx and du.  Evaluates the rates at the current state first (which
 * rebuilds the lists and overwrites the eval fields).  Waits for the
 * stream. */
int sph_surrogate_predict(sph_handle h, double *out_host, int64_t bytes);

/* Advances the state by one rates evaluation and one network evaluation
 * standing for k_steps plain steps: x += dx and u += du on fluid particles,
 * rho += drho on all; adds k_steps to the step counters.  Queues the work. */
int sph_surrogate_advance(sph_handle h, int k_steps);

/* One training step on the pair (current state, state after k plain
 * steps): x1, u1, rho1 are device arrays in the snapshot layout.  Computes
 * the masked mean squared error of the normalised targets (position
 * increment minus T (u + u1) / 2, velocity increment minus T a, density
 * deviation increment minus T (Drho/Dt) / rho0; all channels of fluid
 * particles, the density channel of walls) and its gradient with
 * the hand-written backward pass; with update != 0 applies one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8) of learning rate lr.  Writes the loss
 * to *loss_out and, if grad_out is not NULL, the FP32 gradient (ngrad =
 * number of parameters) as host doubles.  Waits for the stream. */
int sph_surrogate_train_step(sph_handle h, const double *x1_dev, const double *u1_dev, const double *rho1_dev,
                             double lr, int update, double *loss_out, double *grad_out, int64_t ngrad);

/* The judge's second criterion: a judged jump whose oil occupancy differs
 * from the plain steps' by more than tol (|O_jump xor O_plain| / |O_plain|,
 * as sph_oil_occupancy_diff) is rejected too.  0 (the default) reports the
 * interface error without using it to reject. */
int sph_surrogate_set_interface_tol(sph_handle h, double tol);

/* Largest centroid error (over d_ref) and interface error of the judged
 * macro-steps of the last sph_surrogate_run or sph_surrogate_advance_judged. */
int sph_surrogate_judge_stats(sph_handle h, double *max_centroid_err, double *max_interface_err);

/* One judged macro-step: the surrogate jump and k_steps plain steps (of size
 * dt, graph-replayed) from the same state; the plain result is kept.  *err
 * (if not NULL) receives |c_jump - c_plain| / d_ref for the oil centroids
 * (1e30 when the jump left a non-finite value, a particle outside the box or
 * an over-full neighbour list).  Returns SPH_OK when err <= tol and
 * SPH_EFALLBACK when the judge rejects the jump (the state is still the
 * plain result); an interface error above the tolerance of
 * sph_surrogate_set_interface_tol rejects it as well.  k_steps * dt must equal
 * the network's jump span (t_jump of its normalisation block, to 1e-9
 * relative), else SPH_EINVAL.  Waits for the stream. */
int sph_surrogate_advance_judged(sph_handle h, double dt, int k_steps, double tol, double d_ref, double *err);

/* n_macro macro-steps of k_steps plain steps each.  A macro-step is one
 * surrogate evaluation, except every judge_every-th (0: never), where both
 * the surrogate and k_steps plain steps (of size dt, graph-replayed) start
 * from the same state: the plain result is kept, and the distance between
 * the two oil centroids over d_ref is the judged error (the interface error
 * is judged too, see sph_surrogate_set_interface_tol).  An error above tol
 * rejects the surrogate: plain steps replace it until the next judged
 * macro-step.  After every unjudged jump the device error flags are read; a
 * jump that left a non-finite value, a particle outside the box or an
 * over-full neighbour list is rejected too: the state returns to the last
 * verified one (the start, or the result of the last judged or plain
 * stretch), the macro-steps since then are redone with plain steps, and
 * plain steps continue until the next judged macro-step.  The same happens
 * when the plain steps of a judged macro-step fail from the state the
 * unjudged jumps before it left (a non-finite value, a particle outside the
 * box, an over-full list, a step beyond the skin): that judged error counts
 * as 1e30 and the jump as rejected.  Reports the
 * judged count, the rejected count (both kinds) and the largest judged
 * error (1e30 for a judged jump that broke the state).  k_steps * dt must
 * equal the network's jump span (t_jump of its normalisation block, to 1e-9
 * relative), else SPH_EINVAL.  Waits for the stream. */
int sph_surrogate_run(sph_handle h, double dt, int k_steps, int64_t n_macro, int judge_every, double tol,
                      double d_ref, int64_t *n_judged, int64_t *n_rejected, double *max_err);

#ifdef __cplusplus
}
#endif

#endif /* SPH_SURROGATE_H */
