/*
 * mcmcdet_learned.h -- C ABI of the learned proposal of the GB300 (sm_103a) DMALA detector.
 *
 * The paper has no counterpart: its conclusion (Sec. V) names hybrids of model- and data-driven
 * detection as future work. This part adds a small per-antenna network beside the sampler of
 * mcmcdet.h, used in two ways that both leave the target posterior (Eq. (33)) unchanged:
 *  - warm start: the initial level of every chain is drawn from the network's distribution at
 *    the point x = 0 instead of uniformly;
 *  - mixture move: a Metropolis-Hastings transition whose proposal is, per complex antenna i
 *    (real dimensions i and Nt + i, symbol s = kI * L + kQ),
 *        q_mix,i(s | x) = (1 - lambda) q_i(kI | x) q_{Nt+i}(kQ | x) + lambda p_i(s | x),
 *    the product of Algorithm 1's two proposal factors mixed with the network's distribution at
 *    x; the move is accepted with Eq. (18)'s ratio written with q_mix (network evaluated at x
 *    and at x'), so it is an exact MH kernel and may be interleaved with Algorithm 1's
 *    transitions in any fixed pattern. The plain sampler stays available unchanged.
 *
 * Network: 6 features -> 256 (ReLU) -> 256 (ReLU) -> Qc logits. Parameters are one flat FP32
 * vector, in this order and row-major: W1 [256 x 6], b1 [256], W2 [256 x 256], b2 [256],
 * W3 [Qc x 256], b3 [Qc]; mcmc_mlp_param_count gives its length. Features of antenna i at
 * state x, in the detector's level units (xt = 2k - (L - 1), Gt = dmin^2 H^T H and
 * zt = dmin H^T y over the stacked real model):
 *   r = xt + (zt - Gt xt) / diag(Gt)                  (the current gradient as the point a
 *                                                       coordinate step reaches; zt/diag(Gt) at 0)
 *   wt = (Gt + (sigma^2 / 2) I)^{-1} zt               (Remark 1's preconditioned matched filter)
 *   F_i = [r_i, r_{Nt+i}, wt_i, wt_{Nt+i}, log Gt_ii, log sigma^2]   (6 FP32 values per row)
 * Training: softmax cross-entropy of the logits against symbol labels, Adam (Kingma & Ba) with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected, FP32-accurate throughout (the matrix
 * products on tcgen05 from three-term BF16 splits, or on CUDA cores: mcmc_mlp_set_train_engine).
 * Inference: FP32-accurate through the training products, or the BF16 network on tcgen05 tensor
 * cores: the hidden activations and the weights of layers 2 and 3 rounded to BF16 (round to
 * nearest even), layer 1 and every bias FP32-accurate, FP32 accumulation.
 *
 * Random numbers (Philox4x32-10 as in mcmcdet.h): a mixture move numbered t uses transition t's
 * proposal uniforms (dimension n: counter (t, n, channel, chain / 4)) and acceptance uniform;
 * antenna i's component choice comes from counter (t, 0x80000000 + i, channel, chain / 4), word
 * chain % 4: the network's component iff u < lambda. A network draw takes the smallest s with
 * u * S_{Qc-1} < S_s (cumulative weights over s ascending) with u the in-phase dimension's
 * proposal uniform. The warm start draws the same way from dimension i's t = 0 word.
 *
 * Errors as in mcmcdet.h. Every pointer argument is a DEVICE pointer unless marked host; the
 * caller owns them. Calls enqueue on the handle's stream and are asynchronous unless stated.
 */
#ifndef MCMCDET_LEARNED_H
#define MCMCDET_LEARNED_H

#include <stdint.h>

#include "mcmcdet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcmc_mlp mcmc_mlp;

#define MCMC_MLP_FEATURES 6
#define MCMC_MLP_HIDDEN 256

/* Length of the flat parameter vector for a Qc-point constellation (4, 16, 64); 0 otherwise. */
int64_t mcmc_mlp_param_count(int32_t qam);

/* Creates a network for Qc = qam outputs with parameters set to zero. max_rows bounds the rows
 * of one training call (workspace); inference of any number of rows runs in chunks of it.
 * stream: cudaStream_t or NULL for a stream owned by the handle (a blocking stream: it orders
 * with the legacy default stream). */
mcmc_status mcmc_mlp_create(int32_t qam, int32_t max_rows, void *stream, mcmc_mlp **out);
mcmc_status mcmc_mlp_destroy(mcmc_mlp *m);
const char *mcmc_mlp_last_error(const mcmc_mlp *m);

/* Engine of the matrix products of training (loss_grad, train_step) and of the forward that
 * mcmc_mlp_forward runs with tensor_cores = 0: the three layers' products, the input gradients
 * and the weight gradients summed over the rows. tensor_cores = 1 (the default on sm_103):
 * tcgen05 tiles of 128 x 64 or 128 x 128, each FP32 operand split into three BF16 terms (to 2^-26
 * of itself) and the six leading term products accumulated in FP32, as accurate as an FP32
 * product; 0: the FP32 CUDA-core kernel. The bias gradients (column sums) run on CUDA cores
 * either way. Both engines are deterministic. MCMC_EUNSUPPORTED for 1 without sm_103. */
mcmc_status mcmc_mlp_set_train_engine(mcmc_mlp *m, int32_t tensor_cores);

/* Copies the flat parameter vector in or out (host_io = 1: host pointer, synchronous). Setting
 * the parameters resets the Adam state. */
mcmc_status mcmc_mlp_set_params(mcmc_mlp *m, const float *params, int32_t host_io);
mcmc_status mcmc_mlp_get_params(mcmc_mlp *m, float *params, int32_t host_io);

/* logits [rows x Qc] of features X [rows x 6] (row-major FP32). tensor_cores = 1 runs the
 * BF16 network kernel on tcgen05 (as above), 0 the FP32-accurate products of training (on the
 * engine mcmc_mlp_set_train_engine selects). */
mcmc_status mcmc_mlp_forward(mcmc_mlp *m, int64_t rows, const float *X, float *logits,
                             int32_t tensor_cores);

/* Mean cross-entropy over the rows idx[0..rows) of (X, labels) (idx NULL: rows 0..rows-1) and its
 * gradient with respect to the flat parameters: loss -> *loss (device FP32 scalar, may be NULL),
 * gradient -> grad (device, param_count floats). rows <= max_rows. Deterministic. */
mcmc_status mcmc_mlp_loss_grad(mcmc_mlp *m, int32_t rows, const float *X, const int32_t *labels,
                               const int32_t *idx, float *loss, float *grad);

/* loss_grad followed by one Adam step with learning rate lr (step counter kept by the handle). */
mcmc_status mcmc_mlp_train_step(mcmc_mlp *m, int32_t rows, const float *X, const int32_t *labels,
                                const int32_t *idx, float lr, float *loss);

/* Features of the detector's current chain states: X [R x 6] with R = sum_b Np * Nt_b, row
 * Np * (sum_{b' < b} Nt_b') + c * Nt_b + i for antenna i of chain c of channel b. at_zero = 1
 * gives the features of the point x = 0 instead: R = sum_b Nt_b, row (sum_{b' < b} Nt_b') + i.
 * Needs a preconditioned FP32 or MIXED handle (MCMC_EUNSUPPORTED otherwise). */
mcmc_status mcmc_detect_features(mcmc_detector *d, int32_t at_zero, float *X);

/* Attaches a network (not owned: it must outlive its use; NULL detaches) with mixture weight
 * lambda in [0, 1]. Only channels whose constellation has the network's Qc points take learned
 * moves and warm starts; the others are left to the plain sampler. tensor_cores selects the
 * inference kernel as in mcmc_mlp_forward. The detector evaluates the network on its own stream
 * with the network's workspace: no call on the network may run concurrently with the
 * detector's learned calls. */
mcmc_status mcmc_detect_set_model(mcmc_detector *d, mcmc_mlp *m, float lambda,
                                  int32_t tensor_cores);

/* Warm start: redraws the states of every chain of the network's channels from the network at
 * x = 0; their energies are evaluated in FP64 when next needed (the next run, estimate or mixture
 * move), and the running best restarts there. */
mcmc_status mcmc_detect_init_learned(mcmc_detector *d);

/* One mixture move, numbered t (1 .. 2^32 - 1), of every chain of the network's channels. */
mcmc_status mcmc_detect_mix_step(mcmc_detector *d, int64_t t);

#ifdef __cplusplus
}
#endif

#endif /* MCMCDET_LEARNED_H */
