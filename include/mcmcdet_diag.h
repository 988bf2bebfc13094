/* mcmcdet_diag.h -- convergence diagnostics of the DMALA chain for small systems.
 *
 * Sec. III-B analyses the chain through its exact transition kernel: for states x' != x,
 * P(x'|x) = q(x'|x) A(x'|x), and P(x|x) = q(x|x) + sum_{z != x} q(z|x) (1 - A(z|x)) (Eq. (22)),
 * with q the factorised proposal (Eqs. (15)-(17), or (21) with Remark 1's preconditioner) and A
 * the MH acceptance (Eq. (18)). The chain leaves the tempered posterior pi(x) ~ exp(f(x) / tau)
 * invariant (Lemma 1), its convergence rate r is the second largest eigenvalue of P, and the
 * distance of the chain's law from pi after t transitions is measured in total variation
 * (Theorem 1; Figs. 2-3 use a 2x2 QPSK system, 16 states).
 *
 * This entry point forms P for a batch of channels of one shape, in FP64 on the GPU, together
 * with pi, the spectrum of P and the total-variation curve from the uniform start (the law of
 * the detector's random initial states).
 *
 * Conventions shared with the detector (include/mcmcdet.h): the stacked real model
 * x = [Re x_c; Im x_c] (N = 2 Nt real dimensions), PAM levels k in {0..L-1} with value
 * (2k - L + 1) d_min, L = sqrt(qam), d_min = sqrt(3 / (2 (qam - 1))); alpha = alpha_scale sigma^2;
 * preconditioned: beta = d_min^2 / sigma^2 and P~ = (H_r^T H_r + gamma I)^{-1} with
 * gamma = sigma^2 / (2 d_min^2); plain: beta = 1, P~ = I. State index of levels (k_0..k_{N-1}):
 * sum_n k_n L^(N-1-n), i.e. dimension 0 is the most significant digit.
 */
#ifndef MCMCDET_DIAG_H
#define MCMCDET_DIAG_H

#include <stdint.h>

#include "mcmcdet.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Largest state space L^(2 Nt) for which the transition kernel is formed, the largest for which
 * its spectrum is computed, and the largest number of receive antennas. */
#define MCMC_DIAG_MAX_STATES 256
#define MCMC_DIAG_MAX_EIG_STATES 64
#define MCMC_DIAG_MAX_NR 32

/* Exact transition kernels of n_channels channels of one shape (nt, nr, qam).
 *   H          device, complex FP32 (interleaved re, im), channel b at H + b * nr * nt complex
 *              entries, column-major nr x nt;
 *   y          device, complex FP32, channel b at y + b * nr;
 *   noise_var  device, sigma^2 > 0 per channel (complex noise variance); a non-positive value
 *              gives NaN outputs for that channel;
 *   preconditioned, alpha_scale (> 0), tau (>= 1): as in mcmc_detect_preprocess;
 *   P          device [n_channels][S][S] FP64, row i = the law of the next state from state i
 *              (S = L^(2 nt) <= MCMC_DIAG_MAX_STATES), required;
 *   pi         device [n_channels][S] FP64, the tempered posterior, or NULL;
 *   eig        device [n_channels][S] FP64, the eigenvalues of P in descending order (real: P is
 *              reversible), or NULL; requires S <= MCMC_DIAG_MAX_EIG_STATES;
 *   tv_steps   >= 0; tv device [n_channels][tv_steps + 1] FP64 with tv[t] the total-variation
 *              distance between pi and the law after t transitions from the uniform law over the
 *              S states, or NULL (then tv_steps is ignored);
 *   stream     cudaStream_t or NULL (the legacy default stream).
 * The caller owns every buffer. The call validates its arguments on the host (MCMC_EINVAL) and
 * enqueues one kernel on the stream (MCMC_ECUDA if the launch fails); it does not synchronise
 * and allocates nothing (its scratch is the kernel's shared memory). */
mcmc_status mcmc_diag_transition(int32_t n_channels, int32_t nt, int32_t nr, int32_t qam,
                                 const void *H, const void *y, const float *noise_var,
                                 int32_t preconditioned, float alpha_scale, float tau, double *P,
                                 double *pi, double *eig, int32_t tv_steps, double *tv,
                                 void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCMCDET_DIAG_H */
