// diag.cu -- convergence diagnostics of the DMALA chain for small systems (Sec. III-B): the
// exact transition kernel P of Eq. (22), the tempered posterior pi it leaves invariant, the
// spectrum of P (its second eigenvalue is the convergence rate r) and the total-variation
// distance of the chain's law from pi over the transitions (Theorem 1). One CTA per channel,
// FP64 throughout, all scratch in shared memory.
//
//  1. the stacked real model H_r (M x N), y_r, and for the preconditioned proposal
//     P~ = (H_r^T H_r + gamma I)^{-1} (Remark 1, Eq. (19)) by Gauss-Jordan (N <= 8);
//  2. per state s (levels k, values x = (2k - L + 1) d): f_tau(x) = -||y_r - H_r x||^2 /
//     (tau sigma^2) (Eq. (3) tempered), the drift P~ grad f_tau(x) and, per dimension n, the log
//     proposal factor log q_n(j | x) over the L levels (Eqs. (15)-(17) / (21));
//  3. P row by row (a warp per row, lanes over the columns): log q(x_j | x_i) is the sum of the
//     factors, the MH acceptance is Eq. (18) in the log domain, and the diagonal is
//     q(x_i | x_i) + sum_{j != i} q(x_j | x_i) (1 - A(x_j | x_i)) (Eq. (22), second line);
//  4. the spectrum: by detailed balance B = D^{1/2} P D^{-1/2} (D = diag pi) is symmetric, with
//     B_ij = exp(min(log q_ij + h_ij, log q_ji - h_ij)), h_ij = (f_tau,i - f_tau,j) / 2, formed so
//     that it is symmetric bit for bit; cyclic Jacobi with round-robin pairs (S / 2 disjoint
//     rotations per step, S - 1 steps per sweep) drives its off-diagonal part to zero;
//  5. TV(t) = (1/2) sum_s |p_t(s) - pi(s)| with p_0 uniform and p_{t+1} = p_t P.
#include "../../include/mcmcdet_diag.h"

#include <cmath>

#include "common.cuh"

namespace mcmcdet {

namespace {

constexpr int kDiagMaxN = 8;        // real dimensions: S = L^N <= 256 with L >= 2
constexpr int kDiagThreads = 256;
constexpr int kDiagMaxSweeps = 40;

struct DiagArgs {
    int n_channels, nt, nr, L, log2L, N, M, S, pre;
    double alpha_scale, tau, dmin;
    const float2 *H, *y;
    const float *s2;
    double *P, *pi, *eig, *tv;
    int tv_steps;
};

// Shared-memory layout (doubles).
struct DiagLayout {
    int hr, yr, pm, ft, lq, pi, b, rot, pv, red, total;
};

__host__ __device__ inline DiagLayout diag_layout(int M, int N, int S, int L, bool eig)
{
    DiagLayout l{};
    int o = 0;
    l.hr = o; o += M * N;
    l.yr = o; o += M;
    l.pm = o; o += N * N;
    l.ft = o; o += S;
    l.lq = o; o += S * N * L;
    l.pi = o; o += S;
    l.b = o; o += eig ? S * S : 0;
    l.rot = o; o += eig ? 2 * S : 0;   // (c, s) of the S / 2 rotations of a step
    l.pv = o; o += 2 * S;              // p_t and p_{t+1}
    l.red = o; o += 32;
    l.total = o;
    return l;
}

__device__ __forceinline__ int level_of(int s, int n, int N, int log2L, int L)
{
    return (s >> (log2L * (N - 1 - n))) & (L - 1);
}

// Block-wide sum (kDiagThreads threads); red holds 32 doubles. Every thread gets the total.
__device__ double block_sum(double v, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// Round-robin pairing of S players (S even) for round r of S - 1: player 0 stays, the others
// rotate; pair k of the round is (pos[k], pos[S - 1 - k]).
__device__ __forceinline__ int rr_player(int pos, int r, int S)
{
    return pos == 0 ? 0 : 1 + (pos - 1 + r) % (S - 1);
}

__global__ void __launch_bounds__(kDiagThreads) diag_kernel(const DiagArgs a)
{
    const int b = blockIdx.x;
    const int N = a.N, M = a.M, S = a.S, L = a.L, nt = a.nt, nr = a.nr;
    const bool want_eig = a.eig != nullptr;
    const DiagLayout lay = diag_layout(M, N, S, L, want_eig);
    extern __shared__ double sm[];
    double *Hr = sm + lay.hr, *yr = sm + lay.yr, *Pm = sm + lay.pm, *ft = sm + lay.ft;
    double *lq = sm + lay.lq, *spi = sm + lay.pi, *B = sm + lay.b, *rot = sm + lay.rot;
    double *pv = sm + lay.pv, *red = sm + lay.red;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

    // 1. real model: H_r = [[Re H, -Im H], [Im H, Re H]], y_r = [Re y; Im y]
    const float2 *Hc = a.H + (size_t)b * nr * nt;
    const float2 *yc = a.y + (size_t)b * nr;
    for (int e = tid; e < M * N; e += blockDim.x) {
        const int m = e / N, n = e % N;
        const bool mi = m >= nr, ni = n >= nt;
        const float2 h = Hc[(ni ? n - nt : n) * nr + (mi ? m - nr : m)];
        Hr[e] = mi == ni ? (double)h.x : (mi ? (double)h.y : -(double)h.y);
    }
    for (int m = tid; m < M; m += blockDim.x) yr[m] = m < nr ? (double)yc[m].x : (double)yc[m - nr].y;
    const double s2 = (double)a.s2[b];
    const double d = a.dmin, tau = a.tau;
    const double alpha = a.alpha_scale * s2;
    const double beta = a.pre ? d * d / s2 : 1.0;
    const double gamma = s2 / (2.0 * d * d);
    __syncthreads();
    if (a.pre && tid == 0) {
        // P~ = (H_r^T H_r + gamma I)^{-1}: Gauss-Jordan on [A | I] (A symmetric positive definite)
        double Aw[kDiagMaxN][2 * kDiagMaxN];
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) {
                double g = i == j ? gamma : 0.0;
                for (int m = 0; m < M; ++m) g += Hr[m * N + i] * Hr[m * N + j];
                Aw[i][j] = g;
                Aw[i][N + j] = i == j ? 1.0 : 0.0;
            }
        for (int k = 0; k < N; ++k) {
            const double inv = 1.0 / Aw[k][k];
            for (int j = 0; j < 2 * N; ++j) Aw[k][j] *= inv;
            for (int i = 0; i < N; ++i) {
                if (i == k) continue;
                const double f = Aw[i][k];
                for (int j = 0; j < 2 * N; ++j) Aw[i][j] -= f * Aw[k][j];
            }
        }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) Pm[i * N + j] = Aw[i][N + j];
    }
    __syncthreads();

    // 2. per state: f_tau, drift and the log proposal factors
    for (int s = tid; s < S; s += blockDim.x) {
        double x[kDiagMaxN], g[kDiagMaxN];
        for (int n = 0; n < N; ++n) {
            x[n] = (2.0 * level_of(s, n, N, a.log2L, L) - (L - 1)) * d;
            g[n] = 0.0;
        }
        double rr = 0.0;
        for (int m = 0; m < M; ++m) {
            double r = yr[m];
            for (int n = 0; n < N; ++n) r -= Hr[m * N + n] * x[n];
            rr += r * r;
            for (int n = 0; n < N; ++n) g[n] += Hr[m * N + n] * r;
        }
        ft[s] = -rr / (tau * s2);
        const double gs = 2.0 / (tau * s2);   // grad f_tau = (2 / (tau sigma^2)) H_r^T (y_r - H_r x)
        for (int n = 0; n < N; ++n) {
            double dn = 0.0;
            if (a.pre)
                for (int j = 0; j < N; ++j) dn += Pm[n * N + j] * g[j];
            else
                dn = g[n];
            dn *= gs;
            // logits of level j: (1 / (2 beta)) dn (a_j - x_n) - (a_j - x_n)^2 / (2 alpha beta)
            double nu[8], mx = -INFINITY;
            for (int j = 0; j < L; ++j) {
                const double dx = (2.0 * j - (L - 1)) * d - x[n];
                nu[j] = dn * dx / (2.0 * beta) - dx * dx / (2.0 * alpha * beta);
                mx = fmax(mx, nu[j]);
            }
            double z = 0.0;
            for (int j = 0; j < L; ++j) z += exp(nu[j] - mx);
            const double lz = mx + log(z);
            for (int j = 0; j < L; ++j) lq[(s * N + n) * L + j] = nu[j] - lz;
        }
    }
    __syncthreads();
    // the tempered posterior
    {
        double mx = -INFINITY;
        for (int s = tid; s < S; s += blockDim.x) mx = fmax(mx, ft[s]);
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[warp] = mx;
        __syncthreads();
        mx = red[0];
        for (int w = 1; w < nw; ++w) mx = fmax(mx, red[w]);
        __syncthreads();
        double part = 0.0;
        for (int s = tid; s < S; s += blockDim.x) {
            spi[s] = exp(ft[s] - mx);
            part += spi[s];
        }
        const double tot = block_sum(part, red);
        for (int s = tid; s < S; s += blockDim.x) {
            spi[s] /= tot;
            if (a.pi) a.pi[(size_t)b * S + s] = spi[s];
        }
    }
    __syncthreads();

    // 3. P, a warp per row i (and the symmetric form for the spectrum)
    double *Pb = a.P + (size_t)b * S * S;
    auto log_q = [&](int from, int to) {
        double v = 0.0;
        for (int n = 0; n < N; ++n) v += lq[(from * N + n) * L + level_of(to, n, N, a.log2L, L)];
        return v;
    };
    for (int i = warp; i < S; i += nw) {
        double stay = 0.0;
        for (int j = lane; j < S; j += 32) {
            if (j == i) continue;
            const double lij = log_q(i, j), lji = log_q(j, i);
            const double la = ft[j] - ft[i] + lji - lij;
            const double A = la < 0.0 ? exp(la) : 1.0;
            const double q = exp(lij);
            Pb[(size_t)i * S + j] = q * A;
            stay += q * (1.0 - A);
            if (want_eig) {
                const double h = 0.5 * (ft[i] - ft[j]);
                B[i * S + j] = exp(fmin(lij + h, lji - h));
            }
        }
        for (int o = 16; o; o >>= 1) stay += __shfl_xor_sync(0xffffffffu, stay, o);
        if (lane == 0) {
            const double pii = exp(log_q(i, i)) + stay;
            Pb[(size_t)i * S + i] = pii;
            if (want_eig) B[i * S + i] = pii;
        }
    }
    __syncthreads();

    // 4. spectrum by parallel cyclic Jacobi on B
    if (want_eig) {
        double nrm = 0.0;
        for (int e = tid; e < S * S; e += blockDim.x) nrm += B[e] * B[e];
        nrm = block_sum(nrm, red);
        for (int sweep = 0; sweep < kDiagMaxSweeps; ++sweep) {
            double off = 0.0;
            for (int e = tid; e < S * S; e += blockDim.x)
                if (e / S != e % S) off += B[e] * B[e];
            off = block_sum(off, red);
            if (!(off > 1e-30 * nrm)) break;
            for (int r = 0; r < S - 1; ++r) {
                // rotation (c, s) zeroing B_pq of each pair: t = sign(th) / (|th| + sqrt(th^2 + 1)),
                // th = (B_qq - B_pp) / (2 B_pq), c = 1 / sqrt(t^2 + 1), s = t c
                for (int k = tid; k < S / 2; k += blockDim.x) {
                    const int p = rr_player(k, r, S), q = rr_player(S - 1 - k, r, S);
                    const double bpq = B[p * S + q];
                    double c = 1.0, sn = 0.0;
                    if (bpq != 0.0) {
                        const double th = (B[q * S + q] - B[p * S + p]) / (2.0 * bpq);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                    }
                    rot[2 * k] = c;
                    rot[2 * k + 1] = sn;
                }
                __syncthreads();
                // B <- B J (columns p, q of every row), then B <- J^T B (rows p, q)
                for (int e = tid; e < S * (S / 2); e += blockDim.x) {
                    const int row = e / (S / 2), k = e % (S / 2);
                    const int p = rr_player(k, r, S), q = rr_player(S - 1 - k, r, S);
                    const double c = rot[2 * k], sn = rot[2 * k + 1];
                    const double bp = B[row * S + p], bq = B[row * S + q];
                    B[row * S + p] = c * bp - sn * bq;
                    B[row * S + q] = sn * bp + c * bq;
                }
                __syncthreads();
                for (int e = tid; e < S * (S / 2); e += blockDim.x) {
                    const int col = e / (S / 2), k = e % (S / 2);
                    const int p = rr_player(k, r, S), q = rr_player(S - 1 - k, r, S);
                    const double c = rot[2 * k], sn = rot[2 * k + 1];
                    const double bp = B[p * S + col], bq = B[q * S + col];
                    B[p * S + col] = c * bp - sn * bq;
                    B[q * S + col] = sn * bp + c * bq;
                }
                __syncthreads();
            }
        }
        if (tid == 0) {
            // eigenvalues: the diagonal, in descending order
            double *ev = a.eig + (size_t)b * S;
            for (int i = 0; i < S; ++i) {
                const double v = B[i * S + i];
                int j = i;
                while (j > 0 && ev[j - 1] < v) {
                    ev[j] = ev[j - 1];
                    --j;
                }
                ev[j] = v;
            }
        }
        __syncthreads();
    }

    // 5. total variation from the uniform start
    if (a.tv) {
        double *p0 = pv, *p1 = pv + S;
        for (int s = tid; s < S; s += blockDim.x) p0[s] = 1.0 / S;
        __syncthreads();
        for (int t = 0; t <= a.tv_steps; ++t) {
            double part = 0.0;
            for (int s = tid; s < S; s += blockDim.x) part += fabs(p0[s] - spi[s]);
            const double tv = 0.5 * block_sum(part, red);
            if (tid == 0) a.tv[(size_t)b * (a.tv_steps + 1) + t] = tv;
            if (t == a.tv_steps) break;
            for (int s = tid; s < S; s += blockDim.x) {
                double v = 0.0;
                for (int i = 0; i < S; ++i) v += p0[i] * Pb[(size_t)i * S + s];
                p1[s] = v;
            }
            __syncthreads();
            double *tmp = p0;
            p0 = p1;
            p1 = tmp;
        }
    }
}

}  // namespace

}  // namespace mcmcdet

extern "C" mcmc_status mcmc_diag_transition(int32_t n_channels, int32_t nt, int32_t nr, int32_t qam,
                                            const void *H, const void *y, const float *noise_var,
                                            int32_t preconditioned, float alpha_scale, float tau,
                                            double *P, double *pi, double *eig, int32_t tv_steps,
                                            double *tv, void *stream)
{
    using namespace mcmcdet;
    const int L = qam == 4 ? 2 : qam == 16 ? 4 : qam == 64 ? 8 : 0;
    if (n_channels < 1 || nt < 1 || nr < 1 || nr > MCMC_DIAG_MAX_NR || !L || !H || !y ||
        !noise_var || !P || (preconditioned != 0 && preconditioned != 1) ||
        !(alpha_scale > 0.f) || !std::isfinite(alpha_scale) || !(tau >= 1.f) || !std::isfinite(tau) ||
        (tv && tv_steps < 0))
        return MCMC_EINVAL;
    const int N = 2 * nt;
    long long S = 1;
    for (int n = 0; n < N && S <= MCMC_DIAG_MAX_STATES; ++n) S *= L;
    if (N > kDiagMaxN || S > MCMC_DIAG_MAX_STATES) return MCMC_EINVAL;
    if (eig && S > MCMC_DIAG_MAX_EIG_STATES) return MCMC_EINVAL;
    DiagArgs a{};
    a.n_channels = n_channels;
    a.nt = nt;
    a.nr = nr;
    a.L = L;
    a.log2L = L == 2 ? 1 : L == 4 ? 2 : 3;
    a.N = N;
    a.M = 2 * nr;
    a.S = (int)S;
    a.pre = preconditioned;
    a.alpha_scale = alpha_scale;
    a.tau = tau;
    a.dmin = std::sqrt(3.0 / (2.0 * (qam - 1)));
    a.H = static_cast<const float2 *>(H);
    a.y = static_cast<const float2 *>(y);
    a.s2 = noise_var;
    a.P = P;
    a.pi = pi;
    a.eig = eig;
    a.tv = tv;
    a.tv_steps = tv ? tv_steps : 0;
    const DiagLayout lay = diag_layout(a.M, N, a.S, L, eig != nullptr);
    const size_t smem = sizeof(double) * (size_t)lay.total;
    if (allow_max_dyn_smem(diag_kernel) != cudaSuccess) {
        cudaGetLastError();
        return MCMC_ECUDA;
    }
    diag_kernel<<<n_channels, kDiagThreads, smem, static_cast<cudaStream_t>(stream)>>>(a);
    return cudaGetLastError() == cudaSuccess ? MCMC_OK : MCMC_ECUDA;
}
