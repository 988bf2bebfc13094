/*
 * mcmcdet.h -- C ABI of the GB300 (sm_103a) DMALA MIMO detector.
 *
 * Method: "Near-Optimal MIMO Detection Using Gradient-Based MCMC in Discrete Spaces"
 * (arXiv 2407.06042). For every received vector y = Hx + n (Sec. II-A, Eq. (1)) the library runs
 * Np independent DMALA Markov chains (Algorithm 1) on the tempered posterior (Eq. (33)) and reads
 * out a hard decision (the visited sample with the smallest residual, Sec. III-A) and IS-based
 * LLRs (Eq. (34), in the form of Eqs. (35)-(36); Algorithm 2).
 *
 * Conventions shared by every call (identical to the CPU oracle's, which is written separately):
 *  - complex channel H of channel b: Nr x Nt, column-major, interleaved (re, im) float pairs;
 *    element (r, c) at float2 index H_off[b] + c*Nr + r. y: Nr interleaved pairs at y_off[b].
 *  - real-valued model (stacked): x = [Re x_c ; Im x_c] (N = 2Nt), y = [Re y ; Im y] (M = 2Nr).
 *  - alphabet per real dimension: L = sqrt(Qc) PAM levels (2 d_min j - (L-1) d_min), j = 0..L-1,
 *    d_min = sqrt(3 / (2 (Qc - 1))); chain states are these level indices j (int8).
 *  - bits: antenna i carries log2(Qc) bits, first the Gray label (j ^ (j >> 1)) of its in-phase
 *    level (real dimension i), then that of its quadrature level (dimension Nt + i), most
 *    significant bit first; bit 0 <-> b = +1. LLR > 0 favours bit 0. best_idx holds the complex
 *    Gray label (label_I << log2 L) | label_Q.
 *  - parameters (Sec. IV-A): alpha = alpha_scale * sigma^2; preconditioned proposal (Remark 1,
 *    Eqs. (19), (21)) with beta = d_min^2 / sigma^2 and gamma = sigma^2 / (2 d_min^2); plain
 *    proposal (Eqs. (16)-(17)) otherwise; temperature tau (Eq. (33)) replaces f by f / tau in
 *    Algorithm 1, gradient included. sigma^2 is the complex noise variance (sigma^2/2 per real
 *    element).
 *  - random numbers: Philox4x32-10 keyed by the 64-bit seed (lo, hi words); counter
 *    (t, n, channel, chain / 4), word chain % 4, for the proposal uniform of dimension n at
 *    transition t; counter (t, 0xFFFFFFFF, channel, chain / 4) for the acceptance uniform;
 *    t = 0 draws the initial state (level = word >> (32 - log2 L)). Uniform u = (2 (w >> 9) + 1)
 *    * 2^-24. Categorical draws take the smallest level j with u * S_{L-1} < S_j (cumulative
 *    proposal weights, levels ascending). A proposal is accepted iff log u < log A (Eq. (18)).
 *    "channel" is the channel's index in the batch given to mcmc_detect_preprocess.
 *  - a run of T iterations performs T Metropolis-Hastings transitions, numbered
 *    t_offset+1 .. t_offset+T; the hard decision covers every visited state including the
 *    initial one (ties keep the earliest).
 *
 * Errors: every call returns an mcmc_status; no exception crosses the ABI. Arguments are checked
 * on the host before anything is enqueued (MCMC_EINVAL). Calls out of order return MCMC_ESTATE.
 * A numeric fault detected on the device (non-finite energy or logit) is reported as
 * MCMC_ENUMERIC by the next synchronising call. A CUDA runtime failure returns MCMC_ECUDA and the
 * message is kept in mcmc_detect_last_error(). Device waits are bounded; one that runs out sets
 * MCMC_ETIMEOUT instead of hanging.
 *
 * Threading: a handle is not thread-safe; distinct handles are independent.
 */
#ifndef MCMCDET_H
#define MCMCDET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mcmc_detector mcmc_detector;

typedef enum {
    MCMC_OK = 0,
    MCMC_EINVAL = 1,        /* bad argument (checked on the host, nothing enqueued) */
    MCMC_ENOMEM = 2,        /* device or host allocation failed */
    MCMC_ECUDA = 3,         /* CUDA runtime error, see mcmc_detect_last_error */
    MCMC_ETIMEOUT = 4,      /* a bounded device wait ran out */
    MCMC_ENUMERIC = 5,      /* non-finite value met on the device */
    MCMC_ESTATE = 6,        /* call out of order (e.g. run before preprocess) */
    MCMC_EUNSUPPORTED = 7   /* valid request the build does not support (e.g. no sm_103a GPU) */
} mcmc_status;

/* Arithmetic of the chain loop. */
typedef enum {
    MCMC_PREC_FP64 = 0,     /* everything FP64 on CUDA cores (parity mode) */
    MCMC_PREC_FP32 = 1,     /* plain FP32 sampler on CUDA cores */
    MCMC_PREC_MIXED = 2     /* Gram products on tcgen05 tensor cores from split-BF16 G (FP32
                               accumulate), states exact in BF16, FP32 proposal and MH ratio */
} mcmc_prec;

typedef struct {
    int32_t max_channels;   /* capacity: channels per preprocess call */
    int32_t max_nt;         /* capacity: transmit antennas (N = 2 max_nt <= 256) */
    int32_t max_nr;         /* capacity: receive antennas */
    int32_t chains;         /* Np, a multiple of 4, 4..1024 */
    int32_t precision;      /* mcmc_prec */
    int32_t preconditioned; /* 1: Remark 1 proposal (the paper's evaluation setting), 0: plain */
    int32_t refresh_period; /* FP32 / MIXED energies (FP64 mode is exact throughout): the chains
                               add FP32 energy differences to the last exact value. R >= 0: every
                               run_chains ends with an exact evaluation of the energies (so the
                               read-outs see exact values); R > 0 also refreshes them every R
                               transitions inside the run (after each transition t with
                               t % R == 0: the run is cut into chain-kernel launches there, with
                               the exact evaluation between them, unless
                               MCMC_ENGINE_KERNEL_REFRESH); R = -1: never (the tracked values
                               drift; for measuring that drift) */
    int32_t split_terms;    /* MIXED: BF16 terms G is split into (2 = hi+lo, 3 = hi+lo+lo2) */
    int32_t engine;         /* MCMC_ENGINE_AUTO (autotuned per shape class), _SIMT or _TC, optionally
                               OR-ed with the flags MCMC_ENGINE_GRAPH, _NO_CLUSTER, _TRACE,
                               _NO_PACK, _NO_GRAPH and _KERNEL_REFRESH */
    int32_t tile;           /* with an explicit engine: chains per work item (TC: 16 or 32, and 64
                               for channels with N = 2 Nt > 128, which run on thread-block
                               clusters; SIMT: a multiple of 8, at most 64); 0: the engine's
                               default. Must be 0 with MCMC_ENGINE_AUTO (the autotuner picks it) */
    uint64_t seed;          /* Philox key */
    void *stream;           /* cudaStream_t to enqueue on; NULL: the handle creates its own */
} mcmc_config;

/* Chain-kernel engine. AUTO: every shape class (N, L) of a batch gets the launch shape an
 * autotuner found fastest when the class was first seen in the process (probe launches timed on
 * that batch at preprocess): for MIXED precision the tcgen05 kernel at 16 or 32 chains per CTA
 * (also 64 for N > 128) or the CUDA-core kernel (FP32 products, at least as accurate as the split-BF16 ones); for FP32 the
 * CUDA-core kernel's chain tile. SIMT / TC force an engine (TC requires MIXED). Tensor-core
 * channels of N <= 64 of several shape classes with the same tile form one launch group (the
 * packed kernel); every other shape class is a group of its own. A run with several groups
 * enqueues them on parallel streams and, unless NO_GRAPH, replays them from one CUDA graph;
 * GRAPH asks for the graph replay for any batch. */
#define MCMC_ENGINE_AUTO 0
#define MCMC_ENGINE_SIMT 1      /* CUDA-core chain kernel (FP64 / FP32 / MIXED) */
#define MCMC_ENGINE_TC 2        /* tcgen05 chain kernel (MIXED, N <= 256) */
#define MCMC_ENGINE_GRAPH 4     /* flag: replay run_chains from a captured CUDA graph */
#define MCMC_ENGINE_NO_CLUSTER 8 /* flag: channels with N > 128 run the single-CTA tcgen05 kernel,
                                    which streams the Gram operand from L2 every transition,
                                    instead of a thread-block cluster with one resident operand
                                    tile per CTA */
#define MCMC_ENGINE_NO_PACK 32  /* flag: tensor-core channels of N <= 64 from several shape classes
                                   run as one launch per class instead of one packed launch (a
                                   persistent kernel pulling every class's work items, largest
                                   first, from a device queue) */
#define MCMC_ENGINE_NO_GRAPH 64 /* flag: a batch of several launch groups is enqueued directly
                                   instead of being replayed from a CUDA graph */
#define MCMC_ENGINE_KERNEL_REFRESH 128 /* flag: the in-run refreshes of refresh_period > 0 run
                                          inside the chain kernels (one launch per run) instead
                                          of between launches; the states, decisions and draws are
                                          the same either way. Without it a run makes one launch
                                          per R transitions, so for very short periods (a few
                                          transitions) this form can be the faster one */
#define MCMC_ENGINE_TRACE 16    /* flag: every chain records the log acceptance ratio and the log
                                   uniform of its latest transition (Eq. (18)), read back with
                                   mcmc_detect_get_trace (parity diagnostics; one extra store per
                                   chain and transition) */

/* Per-batch statistics (host struct, filled by mcmc_detect_estimate when non-NULL). */
typedef struct {
    int64_t transitions;    /* chain transitions performed since preprocess */
    int64_t accepts;        /* accepted proposals since preprocess */
    int32_t numeric_faults; /* 1 if a chain met a non-finite value since preprocess, else 0 */
    int32_t near_tie_windows; /* entries of near_ties (3) */
    double refresh_drift;   /* max |f_tracked - f_exact| seen at refreshes (FP32/MIXED): the
                               largest correction an exact evaluation made */
    int64_t near_ties[3];   /* Metropolis-Hastings decisions (Eq. (18)) since preprocess whose
                               |log A - log u|, as the chain kernel evaluated it in its own
                               precision, was below 1e-6, 1e-4 and 1e-2 (natural log): the
                               decisions a rounding difference of that size could flip */
    double refresh_drift_rel; /* max |f_tracked - f_exact| / |f_exact| seen at the refreshes
                                 between and after launches (the in-kernel refreshes of
                                 MCMC_ENGINE_KERNEL_REFRESH record refresh_drift only) */
} mcmc_stats;

/* Fills *cfg with defaults: 1 channel, Nt = Nr = 4, 32 chains, FP32, preconditioned, R = 0,
 * split_terms = 2, autotuned engine, seed 0, own stream. */
void mcmc_config_default(mcmc_config *cfg);

/* Creates a detector with the given capacity. Allocates its device workspace lazily at the
 * first preprocess. The config is copied. Returns MCMC_EUNSUPPORTED without an sm_103a device
 * for MIXED (tensor-core) precision. */
mcmc_status mcmc_detect_create(const mcmc_config *cfg, mcmc_detector **out);

/* Sec. II-A / Remark 1 preparation of a batch of n_channels received vectors (Gram matrix G = H^H H,
 * matched filter H^H y, ||y||^2, the preconditioner (G + gamma I)^{-1} when enabled, in FP64),
 * followed by the random initial states (t = 0) and their FP64 energies.
 *  nt, nr, qam, H_off, y_off: HOST arrays [n_channels]; qam in {4, 16, 64}; 1 <= nt <= max_nt,
 *    nt <= nr <= max_nr is not required (nr >= 1).
 *  H, y, noise_var: device pointers when host_io == 0, host pointers when host_io == 1 (copied
 *    inside, on the handle's stream; the call then returns after the copy was enqueued from a
 *    pinned staging buffer, so the host arrays may be reused at once).
 *    noise_var[b] = sigma^2 of channel b (float, > 0, finite).
 *  alpha_scale > 0 (paper: 1), tau >= 1 (paper: 2).
 * Inputs may be released once the stream has passed this call. */
mcmc_status mcmc_detect_preprocess(mcmc_detector *d, int32_t n_channels,
                                   const int32_t *nt, const int32_t *nr, const int32_t *qam,
                                   const void *H, const int64_t *H_off,
                                   const void *y, const int64_t *y_off,
                                   const float *noise_var,
                                   float alpha_scale, float tau, int32_t host_io);

/* Algorithm 1's loop: `iterations` transitions of every chain of every channel, numbered
 * t_offset+1 .. t_offset+iterations (t_offset >= 0). Resuming with t_offset = the number of
 * transitions already done continues the same random stream exactly. The first run after
 * preprocess (or a warm start) first evaluates the states' energies in FP64, where the chains'
 * tracked energies and running best start. */
mcmc_status mcmc_detect_run_chains(mcmc_detector *d, int32_t iterations, int64_t t_offset);

/* Read-out (Sec. III-A hard decision, Algorithm 2 / Eq. (34) soft output) from the chains' final
 * states (S = Np samples per channel, repeats kept). Outputs (any may be NULL):
 *  best_idx [sum Nt_b]          complex Gray label of the best visited sample per antenna
 *  llr      [sum Nt_b log2 Qc_b] IS-based LLRs in the bit order above
 *  best_f   [n_channels]        f(x_best) = -||y - H x_best||^2 / sigma^2 (untempered, FP64)
 *  stats    host mcmc_stats*
 * best_idx/llr/best_f are device pointers when host_io == 0, host pointers when host_io == 1.
 * best_f is an FP64 evaluation of the best state. The energies entering the LLRs are the tracked
 * ones (FP64 in FP64 mode; FP32 steps since the last FP64 refresh otherwise, see refresh_period).
 * Synchronises the handle's stream and reports device-side faults. */
mcmc_status mcmc_detect_estimate(mcmc_detector *d, int8_t *best_idx, float *llr, double *best_f,
                                 mcmc_stats *stats, int32_t host_io);

/* List-based soft output, Eq. (31): the conventional alternative to the IS-LLR of
 * mcmc_detect_estimate. The Np current states of each channel form the sample list, and
 *   llr_k = log sum_{x, bit k of x = 0} exp(f(x)) - log sum_{x, bit k of x = 1} exp(f(x))
 * over its distinct vectors, with f the FP64 energy of each state (Eq. (3)). The paper does not
 * say what an empty side gives: here -clip (no state with bit k = 0) or +clip, and every value
 * is clipped to [-clip, clip]. clip > 0 and finite. llr [sum over channels Nt_b log2 Qc_b]:
 * device or host per host_io, in the bit order of mcmc_detect_estimate. Synchronises. */
mcmc_status mcmc_detect_llr_list(mcmc_detector *d, float *llr, float clip, int32_t host_io);

/* Chain state export: states [sum over channels Np*N_b] int8 level indices, channel-major, then
 * chain-major (chain c of channel b at offset Np*sum_{b'<b} N_b' + c*N_b); f [n_channels*Np]
 * untempered energies f = -||y - Hx||^2 / sigma^2 (Eq. (3)) of those states, FP64 evaluations.
 * Either may be NULL. The call changes nothing in the handle: FP32 and MIXED runs track their
 * energies in FP32 steps (see mcmc_detect_get_tracked), and the FP64 evaluations handed out here
 * are computed beside them. Host or device pointers per host_io. Synchronises. */
mcmc_status mcmc_detect_get_chains(mcmc_detector *d, int8_t *states, double *f, int32_t host_io);

/* The energies the chains track, as they hold them: f [n_channels*Np] of the current states and
 * best_f [n_channels*Np] of each chain's best visited state (the running maximum, Sec. III-A),
 * untempered, layout as in get_chains; either may be NULL. FP64 handles track them exactly; FP32
 * and MIXED runs add FP32 energy differences (Algorithm 1's MH ratio) to the value of the last
 * FP64 evaluation (the first run's initial energies, or the latest refresh, see refresh_period).
 * These are the values the IS-LLR of mcmc_detect_estimate and the hard decision read. Before the
 * first run the initial states' FP64 evaluations are returned. Changes nothing in the handle.
 * Host or device pointers per host_io. Synchronises. */
mcmc_status mcmc_detect_get_tracked(mcmc_detector *d, double *f, double *best_f, int32_t host_io);

/* Handles created with MCMC_ENGINE_TRACE: trace [2*n_channels*Np] doubles, per chain (layout as
 * get_chains' f) the log acceptance ratio log(pi(x')q(x|x') / (pi(x)q(x'|x))) and log u of its
 * latest Metropolis-Hastings test (Eq. (18), tempered target, natural log) as the chain kernel
 * computed them (0, 0 before the first run). MCMC_ESTATE without the flag. Synchronises. */
mcmc_status mcmc_detect_get_trace(mcmc_detector *d, double *trace, int32_t host_io);

/* Chain state import (checkpoint restore, or any start point): same layout as get_chains; every
 * level must lie in [0, L_b). Energies are recomputed in FP64. */
mcmc_status mcmc_detect_set_chains(mcmc_detector *d, const int8_t *states, int32_t host_io);

/* The launch groups of the current batch (after preprocess): returns their number and, for the
 * first `cap` of them, six int32 per group in info: engine (MCMC_ENGINE_SIMT / _TC), chain tile
 * (chains per group of threads or per work item), 1 if it is the packed launch of several shape
 * classes, the largest N of its channels, its work items, and CTAs resident per SM (tcgen05:
 * CTAs per cluster for thread-block clusters). The choices of the autotuner, per shape class,
 * are what they show. 0 for NULL or before preprocess; info may be NULL. */
int32_t mcmc_detect_launch_groups(const mcmc_detector *d, int32_t *info, int32_t cap);

/* Device time (ms) of the chain kernels of the latest n runs, oldest first: from the start of
 * the first launch group to the end of the last (CUDA events on the handle's stream), without
 * the exact energy evaluations before and after them (the in-run refreshes of refresh_period > 0
 * are inside that span, between the launches or inside the kernels). 1 <= n <= min(runs so far,
 * 64), else
 * MCMC_EINVAL. Waits for those runs' events. */
mcmc_status mcmc_detect_run_kernel_ms(mcmc_detector *d, int32_t n, float *ms);

/* Waits for every call enqueued on the handle's stream; reports device faults. */
mcmc_status mcmc_detect_synchronize(mcmc_detector *d);

/* Releases the handle and its workspace (synchronises first). NULL is a no-op returning MCMC_OK. */
mcmc_status mcmc_detect_destroy(mcmc_detector *d);

/* Static description of a status code. */
const char *mcmc_status_string(mcmc_status s);

/* Last error message of the handle ("" when none); the pointer stays valid until the next call. */
const char *mcmc_detect_last_error(const mcmc_detector *d);

/* Chain kernel launches enqueued on this handle since creation (all kernels of the run loop). */
int64_t mcmc_detect_kernel_launches(const mcmc_detector *d);

/* Size of the fixed device scratch array used by mcmc_detect_noalloc (16 MiB). */
#define MCMC_NOALLOC_SCRATCH_BYTES (16u << 20)

/* Whole FP32 detection of a small batch without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc -- real-time loops
 * that must not block on the allocator, hosts whose device memory belongs to a pool they do not
 * control, components whose device memory budget is fixed when they start.
 *
 * It performs what mcmc_detect_create + preprocess + run_chains(iterations, 0) + estimate do
 * for precision MCMC_PREC_FP32 (same kernels, same results), but takes every intermediate buffer
 * from one file-scope device array of MCMC_NOALLOC_SCRATCH_BYTES that every GPU loading this
 * library holds until the process exits. Arguments are those of the handle-based calls:
 *  nt, nr, qam, H_off, y_off: HOST arrays [n_channels]; H, y, noise_var: DEVICE pointers
 *  (layouts as in mcmc_detect_preprocess); chains (Np, multiple of 4), iterations, seed,
 *  preconditioned, alpha_scale, tau as in mcmc_config / preprocess; outputs best_idx, llr, best_f:
 *  DEVICE pointers (layouts as in mcmc_detect_estimate; any may be NULL); stream: cudaStream_t
 *  or NULL for the default stream. The call synchronises that stream before returning.
 * Errors: MCMC_EINVAL for bad arguments and for a batch whose intermediate buffers need more than
 * MCMC_NOALLOC_SCRATCH_BYTES (checked before any work is enqueued); device faults as in estimate.
 * The first call in a CUDA context (per device, and again after cudaDeviceReset) looks up the
 * array's device address (cudaGetSymbolAddress) with that context current: make that first call
 * before any stream capture begins.
 * Every call shares the array and leaves its contents behind; each call re-initialises what it
 * reads, and calls that overlap on the GPU (other threads, other streams) race with each other. */
mcmc_status mcmc_detect_noalloc(int32_t n_channels, const int32_t *nt, const int32_t *nr,
                                const int32_t *qam, const void *H, const int64_t *H_off,
                                const void *y, const int64_t *y_off, const float *noise_var,
                                int32_t chains, int32_t iterations, uint64_t seed,
                                int32_t preconditioned, float alpha_scale, float tau,
                                int8_t *best_idx, float *llr, double *best_f, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCMCDET_H */
