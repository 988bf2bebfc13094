/*
 * dmala_oracle.c -- plain FP64 CPU oracle for the DMALA MIMO detector.
 *
 * TEST INFRASTRUCTURE. This file is the slow, obviously-correct reference that the CUDA
 * library is checked against. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it; the CUDA library neither links nor calls it, and it shares no code
 * with the CUDA library (it includes only the C standard library).
 *
 * Paper: "Near-Optimal MIMO Detection Using Gradient-Based MCMC in Discrete Spaces"
 * (arXiv 2407.06042). Every routine states the passage it follows. All arithmetic is FP64 and
 * follows the paper's definitions directly: the metric f and its gradient are evaluated from the
 * real-valued channel H (never from the Gram matrix), each proposal factor is a softmax over the
 * alphabet, and the acceptance test is the paper's A > u written in the log domain.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *  - real-valued model: x = [Re x_c ; Im x_c], y = [Re y_c ; Im y_c],
 *    H = [[Re H, -Im H], [Im H, Re H]]  (Sec. II-A says only "equivalent real-valued model");
 *  - alphabet A = {(2j - L + 1) d_min : j = 0..L-1} ascending, d_min = sqrt(3 / (2 (Qc - 1)))
 *    (half the minimum distance of unit-average-energy square QAM, Sec. IV-A);
 *  - sigma^2 is the complex noise variance, sigma^2/2 per real element (Sec. II-A);
 *  - tempering (Algorithm 2): f is replaced by f/tau everywhere in Algorithm 1, the gradient
 *    included; alpha, beta, gamma stay functions of sigma^2;
 *  - "T iterations" = T Metropolis-Hastings transitions; the final sample is x^(T+1);
 *  - categorical draws by inverse CDF over the levels in ascending order: the smallest j with
 *    u * S_{L-1} < S_j, S_j the cumulative sum of exp(logit - max logit);
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the 64-bit seed, counter
 *    (t, n, channel, chain / 4) for the proposal uniform of dimension n at transition t, word
 *    chain % 4; counter (t, 0xFFFFFFFF, channel, chain / 4) for the acceptance uniform; t = 0
 *    for the random initial state (level = word >> (32 - log2 L));
 *    uniform u = (2 * (word >> 9) + 1) * 2^-24, exactly representable in FP32 and FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_N 512
#define ORACLE_MAX_L 8

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy  */
/* as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies with a Weyl-sequence key bump.  */
/* ------------------------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1) from one 32-bit word: (2m + 1) / 2^24 with m the top 23 bits */
double oracle_uniform(uint32_t w)
{
    return (double)(2u * (w >> 9) + 1u) * (1.0 / 16777216.0);
}

static uint32_t philox_word(uint64_t seed, uint32_t t, uint32_t n, uint32_t channel,
                            uint32_t chain)
{
    uint32_t ctr[4] = {t, n, channel, chain >> 2};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return out[chain & 3u];
}

/* ------------------------------------------------------------------------------------------ */
/* System model (Sec. II-A, Eq. (1)).                                                           */
/* ------------------------------------------------------------------------------------------ */

/* Stacked real-valued model from a complex Nr x Nt channel (column-major, interleaved re/im)
 * and an Nr-vector y. Output H is (2Nr) x (2Nt) row-major, y is 2Nr. */
void oracle_real_model(int nr, int nt, const double *Hc, const double *yc, double *H, double *y)
{
    int M = 2 * nr, N = 2 * nt;
    for (int r = 0; r < nr; ++r) {
        for (int c = 0; c < nt; ++c) {
            double re = Hc[2 * (c * nr + r)], im = Hc[2 * (c * nr + r) + 1];
            H[r * N + c] = re;
            H[r * N + nt + c] = -im;
            H[(nr + r) * N + c] = im;
            H[(nr + r) * N + nt + c] = re;
        }
        y[r] = yc[2 * r];
        y[nr + r] = yc[2 * r + 1];
    }
    (void)M;
}

/* half of the minimum distance between points of unit-average-energy square Qc-QAM */
double oracle_dmin(int qc)
{
    return sqrt(3.0 / (2.0 * (double)(qc - 1)));
}

/* Eq. (3): f(x) = -||y - Hx||^2 / sigma^2, from the residual. */
double oracle_f(const double *H, const double *y, int M, int N, double sigma2, const double *x)
{
    double s = 0.0;
    for (int m = 0; m < M; ++m) {
        double r = y[m];
        for (int n = 0; n < N; ++n) r -= H[m * N + n] * x[n];
        s += r * r;
    }
    return -s / sigma2;
}

/* Eq. (10): grad f(x) = (2 / sigma^2) H^T (y - Hx). */
void oracle_grad_f(const double *H, const double *y, int M, int N, double sigma2,
                   const double *x, double *g)
{
    double r[2 * ORACLE_MAX_N];
    for (int m = 0; m < M; ++m) {
        double v = y[m];
        for (int n = 0; n < N; ++n) v -= H[m * N + n] * x[n];
        r[m] = v;
    }
    for (int n = 0; n < N; ++n) {
        double s = 0.0;
        for (int m = 0; m < M; ++m) s += H[m * N + n] * r[m];
        g[n] = 2.0 / sigma2 * s;
    }
}

/* Remark 1: M = (H^T H + gamma I)^{-1}, by Gauss-Jordan elimination with partial pivoting.
 * Returns 0 on success, -1 if a pivot vanishes. P is N x N row-major. */
int oracle_preconditioner(const double *H, int M, int N, double gamma, double *P)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(2 * N));
    if (!a) return -1;
    int W = 2 * N;
    for (int i = 0; i < N; ++i) {
        for (int j = 0; j < N; ++j) {
            double s = 0.0;
            for (int m = 0; m < M; ++m) s += H[m * N + i] * H[m * N + j];
            a[i * W + j] = s + (i == j ? gamma : 0.0);
            a[i * W + N + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < N; ++c) {
        int piv = c;
        for (int r = c + 1; r < N; ++r)
            if (fabs(a[r * W + c]) > fabs(a[piv * W + c])) piv = r;
        if (a[piv * W + c] == 0.0) { free(a); return -1; }
        if (piv != c)
            for (int j = 0; j < W; ++j) { double t = a[c * W + j]; a[c * W + j] = a[piv * W + j]; a[piv * W + j] = t; }
        double inv = 1.0 / a[c * W + c];
        for (int j = 0; j < W; ++j) a[c * W + j] *= inv;
        for (int r = 0; r < N; ++r) {
            if (r == c) continue;
            double fct = a[r * W + c];
            if (fct != 0.0)
                for (int j = 0; j < W; ++j) a[r * W + j] -= fct * a[c * W + j];
        }
    }
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) P[i * N + j] = a[i * W + N + j];
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* A DMALA problem instance.                                                                    */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int M, N, L;            /* real rows, real unknowns, PAM levels per real dimension */
    const double *H;        /* M x N row-major real-valued channel */
    const double *y;        /* M real-valued observation */
    const double *P;        /* N x N preconditioner (Remark 1), or NULL for the plain gradient */
    double sigma2;          /* complex noise variance */
    double alpha;           /* step size (Eq. (9)) */
    double beta;            /* perturbation scale of Remark 1 (1 for the plain proposal) */
    double tau;             /* temperature of Eq. (33) (1 = untempered) */
    double dmin;            /* alphabet half-spacing */
} oracle_problem;

static double level_value(const oracle_problem *p, int j)
{
    return (double)(2 * j - p->L + 1) * p->dmin;
}

static void levels_to_x(const oracle_problem *p, const int *k, double *x)
{
    for (int n = 0; n < p->N; ++n) x[n] = level_value(p, k[n]);
}

/* tempered metric f(x)/tau (Algorithm 2, first step) */
static double f_tempered(const oracle_problem *p, const int *k)
{
    double x[ORACLE_MAX_N];
    levels_to_x(p, k, x);
    return oracle_f(p->H, p->y, p->M, p->N, p->sigma2, x) / p->tau;
}

/* Drift entering the proposal: P grad(f/tau)(x) (Remark 1), or grad(f/tau)(x) when P is NULL. */
static void drift(const oracle_problem *p, const int *k, double *d)
{
    double x[ORACLE_MAX_N], g[ORACLE_MAX_N];
    levels_to_x(p, k, x);
    oracle_grad_f(p->H, p->y, p->M, p->N, p->sigma2, x, g);
    for (int n = 0; n < p->N; ++n) g[n] /= p->tau;
    if (!p->P) {
        for (int n = 0; n < p->N; ++n) d[n] = g[n];
        return;
    }
    for (int i = 0; i < p->N; ++i) {
        double s = 0.0;
        for (int j = 0; j < p->N; ++j) s += p->P[i * p->N + j] * g[j];
        d[i] = s;
    }
}

/* Logits of the proposal factor q_n(. | x_n) over the alphabet, given the drift component d_n.
 * Plain proposal, Eq. (16): mu(a) = (1/2) d_n (a - x_n) - (a - x_n)^2 / (2 alpha).
 * Preconditioned, Eq. (21) (Remark 1): nu(a) = (1/(2 beta)) d_n (a - x_n) - (a - x_n)^2 / (2 alpha beta).
 * The first is the second with beta = 1; the caller passes beta = 1 for the plain proposal. */
static void factor_logits(const oracle_problem *p, int kn, double dn, double *logit)
{
    double xn = level_value(p, kn);
    for (int j = 0; j < p->L; ++j) {
        double dl = level_value(p, j) - xn;
        logit[j] = dn * dl / (2.0 * p->beta) - dl * dl / (2.0 * p->alpha * p->beta);
    }
}

/* Eq. (17): log softmax of the logits, evaluated at level j. */
static double log_softmax_at(const double *logit, int L, int j)
{
    double mx = logit[0];
    for (int i = 1; i < L; ++i) if (logit[i] > mx) mx = logit[i];
    double s = 0.0;
    for (int i = 0; i < L; ++i) s += exp(logit[i] - mx);
    return logit[j] - mx - log(s);
}

/* Eqs. (14)-(15): log q(x_to | x_from) = sum_n log q_n(x_to_n | x_from_n). */
double oracle_log_q(const oracle_problem *p, const int *k_from, const int *k_to)
{
    double d[ORACLE_MAX_N], logit[ORACLE_MAX_L];
    drift(p, k_from, d);
    double s = 0.0;
    for (int n = 0; n < p->N; ++n) {
        factor_logits(p, k_from[n], d[n], logit);
        s += log_softmax_at(logit, p->L, k_to[n]);
    }
    return s;
}

/* Eq. (18) in the log domain: log A(x'|x) = min{0, f(x')/tau - f(x)/tau + log q(x|x') - log q(x'|x)}. */
double oracle_log_accept(const oracle_problem *p, const int *k, const int *kp)
{
    double v = f_tempered(p, kp) - f_tempered(p, k) + oracle_log_q(p, kp, k) - oracle_log_q(p, k, kp);
    return v < 0.0 ? v : 0.0;
}

/* Random initial state (Sec. IV-A: "each initialized randomly"): uniform levels from t = 0. */
void oracle_init_state(const oracle_problem *p, uint64_t seed, uint32_t channel, uint32_t chain,
                       int *k)
{
    int bits = (p->L == 2) ? 1 : (p->L == 4) ? 2 : 3;
    for (int n = 0; n < p->N; ++n)
        k[n] = (int)(philox_word(seed, 0u, (uint32_t)n, channel, chain) >> (32 - bits));
}

typedef struct {
    double log_a;        /* log acceptance probability of the proposal */
    double log_u;        /* log of the acceptance uniform */
    double cat_margin;   /* min over n of the distance of u*S_total to the nearest CDF boundary, / S_total */
    double f_new;        /* f(x^(t+1)) / tau */
    int accepted;
} oracle_step_info;

/* One transition of Algorithm 1 (steps of its loop body, in order), number t >= 1.
 * k holds x^(t) on entry and x^(t+1) on return. */
int oracle_step(const oracle_problem *p, uint64_t seed, uint32_t channel, uint32_t chain,
                uint32_t t, int *k, oracle_step_info *info)
{
    int N = p->N, L = p->L;
    double d[ORACLE_MAX_N], logit[ORACLE_MAX_L];
    int kp[ORACLE_MAX_N];
    double margin = 1.0;

    /* Sample x'_n ~ q_n(. | x_n) for every n (inverse CDF). */
    drift(p, k, d);
    for (int n = 0; n < N; ++n) {
        factor_logits(p, k[n], d[n], logit);
        double mx = logit[0];
        for (int j = 1; j < L; ++j) if (logit[j] > mx) mx = logit[j];
        double S[ORACLE_MAX_L], acc = 0.0;
        for (int j = 0; j < L; ++j) { acc += exp(logit[j] - mx); S[j] = acc; }
        double u = oracle_uniform(philox_word(seed, t, (uint32_t)n, channel, chain));
        double target = u * S[L - 1];
        int sel = L - 1;
        for (int j = 0; j < L; ++j) if (target < S[j]) { sel = j; break; }
        kp[n] = sel;
        double lo = sel > 0 ? S[sel - 1] : 0.0;
        double m1 = (target - lo) / S[L - 1], m2 = (S[sel] - target) / S[L - 1];
        if (sel > 0 && m1 < margin) margin = m1;
        if (sel < L - 1 && m2 < margin) margin = m2;
    }
    /* q(x'|x), grad f(x'), q(x|x'), f(x'), then A(x'|x) and u. */
    double log_a = oracle_log_accept(p, k, kp);
    double u = oracle_uniform(philox_word(seed, t, 0xFFFFFFFFu, channel, chain));
    double log_u = log(u);
    int acc = (log_a > log_u);
    if (acc) memcpy(k, kp, sizeof(int) * (size_t)N);
    if (info) {
        info->log_a = log_a;
        info->log_u = log_u;
        info->cat_margin = margin;
        info->f_new = f_tempered(p, k);
        info->accepted = acc;
    }
    return acc;
}

/* Runs transitions t_offset+1 .. t_offset+iters of one chain from the state in k.
 * Tracks the visited state with the largest f (smallest residual, Sec. III-A hard decision):
 * the initial state counts when t_offset == 0; ties keep the earliest. Returns accepts. */
int oracle_run_chain(const oracle_problem *p, uint64_t seed, uint32_t channel, uint32_t chain,
                     uint32_t t_offset, int iters, int *k, double *best_f, int *best_k,
                     double *min_gap)
{
    int accepts = 0;
    double bf = -INFINITY, gap = INFINITY;
    if (best_f && best_k) {
        bf = *best_f;
        if (t_offset == 0) {
            double f0 = f_tempered(p, k) * p->tau;
            if (f0 > bf) { bf = f0; memcpy(best_k, k, sizeof(int) * (size_t)p->N); }
        }
    }
    for (int i = 0; i < iters; ++i) {
        oracle_step_info info;
        accepts += oracle_step(p, seed, channel, chain, t_offset + 1u + (uint32_t)i, k, &info);
        double g = fabs(info.log_a - info.log_u);
        if (g < gap) gap = g;
        if (best_f && best_k) {
            double fu = info.f_new * p->tau;
            if (fu > bf) { bf = fu; memcpy(best_k, k, sizeof(int) * (size_t)p->N); }
        }
    }
    if (best_f) *best_f = bf;
    if (min_gap) *min_gap = gap;
    return accepts;
}

/* ------------------------------------------------------------------------------------------ */
/* Learned proposal (an extension with no counterpart in the paper). Per complex antenna i     */
/* (real dimensions i and Nt + i, symbol s = kI * L + kQ) the proposal is the mixture          */
/*     q_mix,i(s | x) = (1 - lambda) q_i(kI | x) q_{Nt+i}(kQ | x) + lambda p_i(s | x)          */
/* of the product of Algorithm 1's two factors and a network's per-antenna distribution p_i    */
/* evaluated at x (passed in as natural-log probabilities, Nt x Qc). The move is accepted with */
/* the Metropolis-Hastings ratio of Eq. (18) written with q_mix, so every such move keeps the  */
/* target exactly. lambda = 0 is Algorithm 1's transition, uniform for uniform.                */
/* Random numbers: dimension n's proposal uniform and the acceptance uniform as in Algorithm   */
/* 1's transition t; the component choice of antenna i from counter                            */
/* (t, 0x80000000 + i, channel, chain / 4): the network's component iff u < lambda. A network  */
/* draw takes the smallest s with u_i * S_{Qc-1} < S_s (u_i the in-phase dimension's uniform). */
/* ------------------------------------------------------------------------------------------ */

static uint32_t mix_word(uint64_t seed, uint32_t t, int i, uint32_t channel, uint32_t chain)
{
    return philox_word(seed, t, 0x80000000u + (uint32_t)i, channel, chain);
}

static double log_add(double a, double b)
{
    double m = a > b ? a : b;
    if (m == -INFINITY) return -INFINITY;
    return m + log(exp(a - m) + exp(b - m));
}

/* log q_mix(x_to | x_from) with the network's log-probabilities nnlogp evaluated at x_from. */
double oracle_mix_log_q(const oracle_problem *p, double lambda, const int *k_from,
                        const double *nnlogp, const int *k_to)
{
    int N = p->N, L = p->L, nt = N / 2, Q = L * L;
    double d[ORACLE_MAX_N], li[ORACLE_MAX_L], lq[ORACLE_MAX_L];
    drift(p, k_from, d);
    double s = 0.0;
    for (int i = 0; i < nt; ++i) {
        factor_logits(p, k_from[i], d[i], li);
        factor_logits(p, k_from[nt + i], d[nt + i], lq);
        double ld = log_softmax_at(li, L, k_to[i]) + log_softmax_at(lq, L, k_to[nt + i]);
        double ln = nnlogp[i * Q + k_to[i] * L + k_to[nt + i]];
        double a = lambda < 1.0 ? log1p(-lambda) + ld : -INFINITY;
        double b = lambda > 0.0 ? log(lambda) + ln : -INFINITY;
        s += log_add(a, b);
    }
    return s;
}

/* First half of a learned move numbered t: draws x' from q_mix(. | x) into kp. Returns the
 * smallest distance of a deciding uniform to its decision boundary (CDF margins relative to
 * the total, and |u - lambda| of the component choices). */
double oracle_mix_propose(const oracle_problem *p, uint64_t seed, uint32_t channel,
                          uint32_t chain, uint32_t t, double lambda, const int *k,
                          const double *nnlogp, int *kp)
{
    int N = p->N, L = p->L, nt = N / 2, Q = L * L;
    double d[ORACLE_MAX_N], logit[ORACLE_MAX_L];
    double margin = 1.0;
    drift(p, k, d);
    for (int i = 0; i < nt; ++i) {
        double uc = oracle_uniform(mix_word(seed, t, i, channel, chain));
        if (fabs(uc - lambda) < margin) margin = fabs(uc - lambda);
        if (uc < lambda) {
            double S[ORACLE_MAX_L * ORACLE_MAX_L], acc = 0.0;
            for (int s = 0; s < Q; ++s) { acc += exp(nnlogp[i * Q + s]); S[s] = acc; }
            double target = oracle_uniform(philox_word(seed, t, (uint32_t)i, channel, chain)) * S[Q - 1];
            int sel = Q - 1;
            for (int s = 0; s < Q; ++s) if (target < S[s]) { sel = s; break; }
            double lo = sel > 0 ? S[sel - 1] : 0.0;
            double m1 = (target - lo) / S[Q - 1], m2 = (S[sel] - target) / S[Q - 1];
            if (sel > 0 && m1 < margin) margin = m1;
            if (sel < Q - 1 && m2 < margin) margin = m2;
            kp[i] = sel / L;
            kp[nt + i] = sel % L;
            continue;
        }
        for (int h = 0; h < 2; ++h) {
            int n = h ? nt + i : i;
            factor_logits(p, k[n], d[n], logit);
            double mx = logit[0];
            for (int j = 1; j < L; ++j) if (logit[j] > mx) mx = logit[j];
            double S[ORACLE_MAX_L], acc = 0.0;
            for (int j = 0; j < L; ++j) { acc += exp(logit[j] - mx); S[j] = acc; }
            double target = oracle_uniform(philox_word(seed, t, (uint32_t)n, channel, chain)) * S[L - 1];
            int sel = L - 1;
            for (int j = 0; j < L; ++j) if (target < S[j]) { sel = j; break; }
            double lo = sel > 0 ? S[sel - 1] : 0.0;
            double m1 = (target - lo) / S[L - 1], m2 = (S[sel] - target) / S[L - 1];
            if (sel > 0 && m1 < margin) margin = m1;
            if (sel < L - 1 && m2 < margin) margin = m2;
            kp[n] = sel;
        }
    }
    return margin;
}

/* Second half: Metropolis-Hastings test of x' against x with the network evaluated at x
 * (nnlogp_x) and at x' (nnlogp_xp); k becomes the next state. info as for Algorithm 1. */
int oracle_mix_accept(const oracle_problem *p, uint64_t seed, uint32_t channel, uint32_t chain,
                      uint32_t t, double lambda, int *k, const int *kp, const double *nnlogp_x,
                      const double *nnlogp_xp, double margin, oracle_step_info *info)
{
    double v = f_tempered(p, kp) - f_tempered(p, k) +
               oracle_mix_log_q(p, lambda, kp, nnlogp_xp, k) -
               oracle_mix_log_q(p, lambda, k, nnlogp_x, kp);
    double log_a = v < 0.0 ? v : 0.0;
    double log_u = log(oracle_uniform(philox_word(seed, t, 0xFFFFFFFFu, channel, chain)));
    int acc = (log_a > log_u);
    if (acc) memcpy(k, kp, sizeof(int) * (size_t)p->N);
    if (info) {
        info->log_a = log_a;
        info->log_u = log_u;
        info->cat_margin = margin;
        info->f_new = f_tempered(p, k);
        info->accepted = acc;
    }
    return acc;
}

/* Warm start: per antenna i a symbol drawn from the network's distribution at x = 0 (nnlogp,
 * Nt x Qc) by inverse CDF with dimension i's t = 0 word read as a uniform. */
void oracle_init_state_learned(const oracle_problem *p, uint64_t seed, uint32_t channel,
                               uint32_t chain, const double *nnlogp, int *k)
{
    int L = p->L, nt = p->N / 2, Q = L * L;
    for (int i = 0; i < nt; ++i) {
        double S[ORACLE_MAX_L * ORACLE_MAX_L], acc = 0.0;
        for (int s = 0; s < Q; ++s) { acc += exp(nnlogp[i * Q + s]); S[s] = acc; }
        double target = oracle_uniform(philox_word(seed, 0u, (uint32_t)i, channel, chain)) * S[Q - 1];
        int sel = Q - 1;
        for (int s = 0; s < Q; ++s) if (target < S[s]) { sel = s; break; }
        k[i] = sel / L;
        k[nt + i] = sel % L;
    }
}

/* One transition numbered t of each of `chains` chains (chain ids chain0 .. chain0+chains-1)
 * from the states in k (chains x N, row-major), in place; infos may be NULL. */
void oracle_step_chains(const oracle_problem *p, uint64_t seed, uint32_t channel, uint32_t chain0,
                        int chains, uint32_t t, int *k, oracle_step_info *infos)
{
    for (int c = 0; c < chains; ++c)
        oracle_step(p, seed, channel, chain0 + (uint32_t)c, t, k + (size_t)c * (size_t)p->N,
                    infos ? infos + c : NULL);
}

/* ------------------------------------------------------------------------------------------ */
/* Soft output (Sec. III-C).                                                                   */
/* ------------------------------------------------------------------------------------------ */
static int gray_of(int k) { return k ^ (k >> 1); }
static int level_of_gray(int g) { int k = g; k ^= k >> 1; k ^= k >> 2; return k; }
static int log2_levels(int L) { return L == 2 ? 1 : L == 4 ? 2 : 3; }

/* F(a) = log(1 + e^a), evaluated exactly (Eq. (35) allows a table; the oracle does not). */
static double softplus(double a)
{
    return a > 0.0 ? a + log1p(exp(-a)) : log1p(exp(a));
}

/* Position of bit index kb in the per-channel bit vector: antenna i carries bits
 * [i*2B, i*2B+B) for its in-phase level (real dimension i) and [i*2B+B, i*2B+2B) for its
 * quadrature level (real dimension Nt+i), most significant Gray bit first. */
static void bit_position(int N, int B, int kb, int *dim, int *pos)
{
    int nt = N / 2;
    int ant = kb / (2 * B), r = kb % (2 * B);
    *dim = (r < B) ? ant : nt + ant;
    *pos = (r < B) ? r : r - B;
}

/* IS-based LLR, Eq. (34) in its log-sum-exp form Eqs. (35)-(36) with exact F:
 * L_k = log sum_s exp(((tau-1)/tau) f(x+) - F(-gamma)) - log sum_s exp(((tau-1)/tau) f(x-) - F(gamma)),
 * gamma = (f(x+) - f(x-)) / tau, x+- the sample with bit k set to +1 (label bit 0) / -1 (bit 1).
 * f is evaluated from the residual for every x+- (untempered f of Eq. (3)).
 * samples: S x N levels (row-major). llr: N*log2(L) values in the bit order of bit_position. */
void oracle_llr_is(const oracle_problem *p, int S, const int *samples, double *llr)
{
    int N = p->N, B = log2_levels(p->L);
    double x[ORACLE_MAX_N];
    double w = (p->tau - 1.0) / p->tau;
    for (int kb = 0; kb < N * B; ++kb) {
        int n, pos;
        bit_position(N, B, kb, &n, &pos);
        int mask = 1 << (B - 1 - pos);
        double vp = -INFINITY, vm = -INFINITY;    /* running log-sum-exp, Eq. (36) */
        for (int s = 0; s < S; ++s) {
            const int *ks = samples + (size_t)s * (size_t)N;
            levels_to_x(p, ks, x);
            int g = gray_of(ks[n]);
            x[n] = level_value(p, level_of_gray(g & ~mask));
            double fp = oracle_f(p->H, p->y, p->M, N, p->sigma2, x);
            x[n] = level_value(p, level_of_gray(g | mask));
            double fm = oracle_f(p->H, p->y, p->M, N, p->sigma2, x);
            double gam = (fp - fm) / p->tau;
            double ap = w * fp - softplus(-gam);
            double am = w * fm - softplus(gam);
            vp = (vp > ap ? vp : ap) + softplus(-fabs(vp - ap));
            vm = (vm > am ? vm : am) + softplus(-fabs(vm - am));
        }
        llr[kb] = vp - vm;
    }
}

/* List-based LLR, Eq. (31): the sample list stands in for the whole state space,
 * L_k = log sum_{x in list, bit k of x = 0} exp(f(x)) - log sum_{x in list, bit k = 1} exp(f(x)),
 * over the distinct vectors of the list (the two sums run over sets). The paper leaves a side
 * with no vector unspecified: it gives +clip (no vector with bit 1) or -clip (none with bit 0),
 * and every value is clipped to [-clip, clip]. f is untempered (Eq. (3)). */
void oracle_llr_list(const oracle_problem *p, int S, const int *samples, double clip, double *llr)
{
    int N = p->N, B = log2_levels(p->L);
    double *f = (double *)malloc(sizeof(double) * (size_t)S);
    int *keep = (int *)malloc(sizeof(int) * (size_t)S);
    if (!f || !keep) { free(f); free(keep); return; }
    double x[ORACLE_MAX_N];
    for (int s = 0; s < S; ++s) {
        const int *ks = samples + (size_t)s * (size_t)N;
        keep[s] = 1;
        for (int r = 0; r < s && keep[s]; ++r) {
            const int *kr = samples + (size_t)r * (size_t)N;
            int same = 1;
            for (int n = 0; n < N; ++n) same &= ks[n] == kr[n];
            if (same) keep[s] = 0;
        }
        if (keep[s]) {
            levels_to_x(p, ks, x);
            f[s] = oracle_f(p->H, p->y, p->M, N, p->sigma2, x);
        }
    }
    for (int kb = 0; kb < N * B; ++kb) {
        int n, pos;
        bit_position(N, B, kb, &n, &pos);
        int mask = 1 << (B - 1 - pos);
        double vp = -INFINITY, vm = -INFINITY;
        for (int s = 0; s < S; ++s) {
            if (!keep[s]) continue;
            double a = f[s];
            if (gray_of(samples[(size_t)s * (size_t)N + n]) & mask)
                vm = (vm > a ? vm : a) + softplus(-fabs(vm - a));
            else
                vp = (vp > a ? vp : a) + softplus(-fabs(vp - a));
        }
        double v = vp == -INFINITY ? -clip : vm == -INFINITY ? clip : vp - vm;
        llr[kb] = v > clip ? clip : v < -clip ? -clip : v;
    }
    free(f);
    free(keep);
}

/* ------------------------------------------------------------------------------------------ */
/* Exact companions for enumerable systems (L^N states).                                       */
/* ------------------------------------------------------------------------------------------ */
static void state_of_index(int N, int L, long idx, int *k)
{
    for (int n = N - 1; n >= 0; --n) { k[n] = (int)(idx % L); idx /= L; }
}

/* f(x) (untempered, Eq. (3)) for every state; state index = sum_n k_n L^(N-1-n). */
void oracle_all_f(const oracle_problem *p, double *fout)
{
    long S = 1;
    for (int n = 0; n < p->N; ++n) S *= p->L;
    int k[ORACLE_MAX_N];
    double x[ORACLE_MAX_N];
    for (long i = 0; i < S; ++i) {
        state_of_index(p->N, p->L, i, k);
        levels_to_x(p, k, x);
        fout[i] = oracle_f(p->H, p->y, p->M, p->N, p->sigma2, x);
    }
}

/* Eq. (4): exact MAP LLR by enumeration of every state. */
void oracle_exact_llr(const oracle_problem *p, double *llr)
{
    int N = p->N, L = p->L, B = log2_levels(L);
    long S = 1;
    for (int n = 0; n < N; ++n) S *= L;
    double *f = (double *)malloc(sizeof(double) * (size_t)S);
    if (!f) return;
    oracle_all_f(p, f);
    int k[ORACLE_MAX_N];
    for (int kb = 0; kb < N * B; ++kb) {
        int n, pos;
        bit_position(N, B, kb, &n, &pos);
        int mask = 1 << (B - 1 - pos);
        double vp = -INFINITY, vm = -INFINITY;
        for (long i = 0; i < S; ++i) {
            state_of_index(N, L, i, k);
            double a = f[i];
            if (gray_of(k[n]) & mask) vm = (vm > a ? vm : a) + softplus(-fabs(vm - a));
            else vp = (vp > a ? vp : a) + softplus(-fabs(vp - a));
        }
        llr[kb] = vp - vm;
    }
    free(f);
}

/* Eq. (22): the transition matrix of the DMALA chain targeting exp(f/tau), row = from state.
 * Off-diagonal q(x'|x) A(x'|x); diagonal q(x|x) + sum_{z != x} q(z|x) (1 - A(z|x)).
 * Pmat is S x S row-major with S = L^N (the caller keeps S small). */
void oracle_transition_matrix(const oracle_problem *p, double *Pmat)
{
    int N = p->N;
    long S = 1;
    for (int n = 0; n < N; ++n) S *= p->L;
    int *ks = (int *)malloc(sizeof(int) * (size_t)S * (size_t)N);
    double *logq = (double *)malloc(sizeof(double) * (size_t)S * (size_t)S);
    double *ft = (double *)malloc(sizeof(double) * (size_t)S);
    if (!ks || !logq || !ft) { free(ks); free(logq); free(ft); return; }
    for (long i = 0; i < S; ++i) {
        state_of_index(N, p->L, i, ks + i * N);
        ft[i] = f_tempered(p, ks + i * N);
    }
    for (long i = 0; i < S; ++i)
        for (long j = 0; j < S; ++j) logq[i * S + j] = oracle_log_q(p, ks + i * N, ks + j * N);
    for (long i = 0; i < S; ++i) {
        double stay = exp(logq[i * S + i]);
        for (long j = 0; j < S; ++j) {
            if (j == i) continue;
            double la = ft[j] - ft[i] + logq[j * S + i] - logq[i * S + j];
            double A = la < 0.0 ? exp(la) : 1.0;
            double qij = exp(logq[i * S + j]);
            Pmat[i * S + j] = qij * A;
            stay += qij * (1.0 - A);
        }
        Pmat[i * S + i] = stay;
    }
    free(ks); free(logq); free(ft);
}

/* ------------------------------------------------------------------------------------------ */
/* One whole detection (Algorithm 2 around Algorithm 1) for one channel, FP64 end to end.      */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int preconditioned;   /* 1: Remark 1 with beta = dmin^2/sigma^2, gamma = sigma^2/(2 dmin^2) */
    double alpha_scale;   /* alpha = alpha_scale * sigma^2 (Sec. IV-A: 1) */
    double tau;           /* temperature (Sec. IV-A: 2) */
    int chains;           /* Np */
    int iterations;       /* T transitions */
    uint64_t seed;
    uint32_t channel;     /* channel id in the Philox counter */
} oracle_detect_cfg;

/* Hc: column-major Nr x Nt complex (interleaved), yc: Nr complex. Outputs (each may be NULL):
 * final_states [chains x 2Nt] levels, final_f [chains] (untempered f of the final states),
 * best_state [2Nt], best_f (max untempered f over every visited state of every chain; ties keep
 * the lowest chain), llr [Nt log2 Qc], accepts (total). Returns 0, or -1 on bad input. */
int oracle_detect(int nr, int nt, int qc, const double *Hc, const double *yc, double sigma2,
                  const oracle_detect_cfg *cfg, int *final_states, double *final_f,
                  int *best_state, double *best_f, double *llr, long *accepts)
{
    int M = 2 * nr, N = 2 * nt, L = (qc == 4) ? 2 : (qc == 16) ? 4 : (qc == 64) ? 8 : 0;
    if (L == 0 || N > ORACLE_MAX_N || M > 2 * ORACLE_MAX_N || cfg->chains <= 0 || sigma2 <= 0.0)
        return -1;
    double *H = (double *)malloc(sizeof(double) * (size_t)M * (size_t)N);
    double *y = (double *)malloc(sizeof(double) * (size_t)M);
    double *P = NULL;
    int *states = (int *)malloc(sizeof(int) * (size_t)cfg->chains * (size_t)N);
    if (!H || !y || !states) { free(H); free(y); free(states); return -1; }
    oracle_real_model(nr, nt, Hc, yc, H, y);
    double dmin = oracle_dmin(qc);
    oracle_problem p;
    p.M = M; p.N = N; p.L = L; p.H = H; p.y = y; p.sigma2 = sigma2;
    p.alpha = cfg->alpha_scale * sigma2;
    p.tau = cfg->tau;
    p.dmin = dmin;
    p.beta = 1.0;
    p.P = NULL;
    if (cfg->preconditioned) {
        P = (double *)malloc(sizeof(double) * (size_t)N * (size_t)N);
        if (!P || oracle_preconditioner(H, M, N, sigma2 / (2.0 * dmin * dmin), P) != 0) {
            free(H); free(y); free(P); free(states); return -1;
        }
        p.P = P;
        p.beta = dmin * dmin / sigma2;
    }
    double bf_all = -INFINITY;
    long acc = 0;
    int bk[ORACLE_MAX_N];
    for (int c = 0; c < cfg->chains; ++c) {
        int *k = states + (size_t)c * (size_t)N;
        oracle_init_state(&p, cfg->seed, cfg->channel, (uint32_t)c, k);
        double bf = -INFINITY;
        acc += oracle_run_chain(&p, cfg->seed, cfg->channel, (uint32_t)c, 0u, cfg->iterations,
                                k, &bf, bk, NULL);
        if (bf > bf_all) {
            bf_all = bf;
            if (best_state) memcpy(best_state, bk, sizeof(int) * (size_t)N);
        }
        if (final_f) final_f[c] = f_tempered(&p, k) * p.tau;
    }
    if (final_states) memcpy(final_states, states, sizeof(int) * (size_t)cfg->chains * (size_t)N);
    if (best_f) *best_f = bf_all;
    if (llr) oracle_llr_is(&p, cfg->chains, states, llr);
    if (accepts) *accepts = acc;
    free(H); free(y); free(P); free(states);
    return 0;
}

/* Size of the problem struct, so the Python wrapper can check its mirror. */
int oracle_problem_size(void) { return (int)sizeof(oracle_problem); }
