// mix.cu -- kernels of the learned proposal on the detector's chains: Gram products and network
// features at a set of states, the mixture draw, the Metropolis-Hastings test of the mixture
// move, and the warm start (declarations and conventions in include/mcmcdet_learned.h).
//
// A mixture move numbered t runs as: gram_features(x) -> network(x) -> propose -> gram_features(x')
// -> network(x') -> accept. All arithmetic is FP32 on the emitted FP32 operands
// [Gt | P~ Gt], zt and wt; proposal densities are kept in log2 units (ex2 / lg2), as in the
// chain kernels.
#include "kernels.h"
#include "proposal.cuh"

namespace mcmcdet {

namespace {

constexpr int kGramChains = 32;   // chains per CTA of the Gram/feature kernel

// Gt x and P~ Gt x of chains [c0, c0 + 32) of one channel (one CTA), then the network features
// of every (chain, antenna) of the tile.
__global__ void __launch_bounds__(256) gram_features_kernel(MixGramArgs a)
{
    __shared__ __align__(16) float xs[kMaxN * kGramChains];   // xs[n * 32 + c]
    const int b = blockIdx.y;
    const ChannelDesc d = a.desc[b];
    if (a.L && d.L != a.L) return;
    const int N = d.N, Nt = d.Nt, NOp = d.NOp, NO = d.NO;
    const int c0 = blockIdx.x * kGramChains;
    const int nc = min(kGramChains, a.chains - c0);
    if (nc <= 0) return;
    const int8_t *x = a.x + d.state_off + (long long)c0 * N;
    for (int e = threadIdx.x; e < N * kGramChains; e += blockDim.x) {
        const int n = e / kGramChains, c = e % kGramChains;
        xs[e] = c < nc ? (float)odd_of(x[c * N + n], d.L) : 0.f;
    }
    __syncthreads();
    const float *bt = a.bt32 + d.bt_off;
    const long long sbase = d.state_off + (long long)c0 * N;
    for (int u = threadIdx.x; u < NO * (kGramChains / 8); u += blockDim.x) {
        const int o = u % NO, g = u / NO;
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int m = 0; m < N; ++m) {
            const float bv = __ldg(bt + (long long)m * NOp + o);
            const float4 x0 = *reinterpret_cast<const float4 *>(&xs[m * kGramChains + 8 * g]);
            const float4 x1 = *reinterpret_cast<const float4 *>(&xs[m * kGramChains + 8 * g + 4]);
            acc[0] = fmaf(bv, x0.x, acc[0]);
            acc[1] = fmaf(bv, x0.y, acc[1]);
            acc[2] = fmaf(bv, x0.z, acc[2]);
            acc[3] = fmaf(bv, x0.w, acc[3]);
            acc[4] = fmaf(bv, x1.x, acc[4]);
            acc[5] = fmaf(bv, x1.y, acc[5]);
            acc[6] = fmaf(bv, x1.z, acc[6]);
            acc[7] = fmaf(bv, x1.w, acc[7]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = 8 * g + j;
            if (c >= nc) continue;
            if (o < N) a.gx[sbase + (long long)c * N + o] = acc[j];
            else a.px[sbase + (long long)c * N + (o - N)] = acc[j];
        }
    }
    if (!a.X) return;
    __syncthreads();
    const float *z = a.z32 + d.vec_off, *w = a.w32 + d.vec_off;
    const float ls2 = logf((float)d.sigma2);
    for (int e = threadIdx.x; e < nc * Nt; e += blockDim.x) {
        const int c = e / Nt, i = e % Nt;
        const long long base = sbase + (long long)c * N;
        const float gI = bt[(long long)i * NOp + i], gQ = bt[(long long)(Nt + i) * NOp + Nt + i];
        const float rI = xs[i * kGramChains + c] + (z[i] - a.gx[base + i]) / gI;
        const float rQ = xs[(Nt + i) * kGramChains + c] + (z[Nt + i] - a.gx[base + Nt + i]) / gQ;
        float *row = a.X + (d.state_off / 2 + (long long)(c0 + c) * Nt + i) * 6;
        row[0] = rI;
        row[1] = rQ;
        row[2] = w[i];
        row[3] = w[Nt + i];
        row[4] = logf(gI);
        row[5] = ls2;
    }
}

// Features of the point x = 0 (one thread per antenna).
__global__ void features_zero_kernel(MixGramArgs a)
{
    const int b = blockIdx.y;
    const ChannelDesc d = a.desc[b];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d.Nt) return;
    const int Nt = d.Nt, NOp = d.NOp;
    const float *bt = a.bt32 + d.bt_off;
    const float *z = a.z32 + d.vec_off, *w = a.w32 + d.vec_off;
    const float gI = bt[(long long)i * NOp + i], gQ = bt[(long long)(Nt + i) * NOp + Nt + i];
    float *row = a.X + (d.ant_off + i) * 6;
    row[0] = z[i] / gI;
    row[1] = z[Nt + i] / gQ;
    row[2] = w[i];
    row[3] = w[Nt + i];
    row[4] = logf(gI);
    row[5] = logf((float)d.sigma2);
}

__device__ __forceinline__ float log2_add(float a, float b)
{
    const float m = fmaxf(a, b);
    if (m == -INFINITY) return -INFINITY;
    return m + lg2_approx(ex2_approx(a - m) + ex2_approx(b - m));
}

// Network distribution of one row in log2 units: max logit2, the sum of the weights
// 2^(l2(s) - mx) (summed in s order) and the log2 normaliser.
template <int Q>
__device__ __forceinline__ void nn_norm(const float *logits, float &mx, float &lse2, float &tot)
{
    mx = -INFINITY;
#pragma unroll 8
    for (int s = 0; s < Q; ++s) mx = fmaxf(mx, logits[s] * kLog2e);
    float S = 0.f;
#pragma unroll 8
    for (int s = 0; s < Q; ++s) S += ex2_approx(fmaf(logits[s], kLog2e, -mx));
    tot = S;
    lse2 = mx + lg2_approx(S);
}

template <int Q>
__device__ __forceinline__ void nn_norm(const float *logits, float &mx, float &lse2)
{
    float tot;
    nn_norm<Q>(logits, mx, lse2, tot);
}

// Smallest s with u * S_{Q-1} < S_s over the network's weights 2^(l2(s) - mx) (tot = S_{Q-1}).
template <int Q>
__device__ __forceinline__ int nn_draw(const float *logits, float mx, float tot, float u)
{
    const float target = u * tot;
    float acc = 0.f;
    int sel = Q - 1;
#pragma unroll 8
    for (int s = 0; s < Q; ++s) {
        acc += ex2_approx(fmaf(logits[s], kLog2e, -mx));
        if (target < acc) { sel = s; break; }
    }
    return sel;
}

__device__ __forceinline__ uint32_t philox_word(const MixStepArgs &a, uint32_t t, uint32_t stream,
                                                int b, int c)
{
    const U4 v = philox4x32_10(t, stream, (uint32_t)b, (uint32_t)(c >> 2), a.key0, a.key1);
    return word_of(v, c & 3);
}

// Proposal slope of dimension n (log2 units) at a state with products g (Gt x) and p (P~ Gt x).
__device__ __forceinline__ float slope2(const ChannelDesc &d, bool pre, float z, float w, float g,
                                        float p)
{
    return (float)d.clin * kLog2e * (pre ? (w - p) : (z - g));
}

// Draw of x' for one (chain, antenna) and log2 q_mix of it.
template <int L>
__global__ void __launch_bounds__(128) propose_kernel(MixStepArgs a)
{
    constexpr int Q = L * L;
    const int b = blockIdx.y;
    const ChannelDesc d = a.desc[b];
    if (d.L != L) return;
    const int Nt = d.Nt, N = d.N;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.chains * Nt) return;
    const int c = e / Nt, i = e % Nt;
    const long long base = d.state_off + (long long)c * N;
    const long long row = d.state_off / 2 + e;
    const bool pre = d.NO > N;
    const float *z = a.z32 + d.vec_off, *w = a.w32 + d.vec_off;
    const int kI = a.states[base + i], kQ = a.states[base + Nt + i];
    const float c2 = (float)d.cquad * kLog2e, inv2c = 0.5f / c2;
    const float aI = slope2(d, pre, z[i], w[i], a.gx[base + i], a.px[base + i]);
    const float aQ = slope2(d, pre, z[Nt + i], w[Nt + i], a.gx[base + Nt + i], a.px[base + Nt + i]);
    const float *lg = a.logits + row * Q;
    float mx, lse2, tot;
    nn_norm<Q>(lg, mx, lse2, tot);
    const uint32_t t = a.t;
    const float uc = uniform_f(philox_word(a, t, 0x80000000u + (uint32_t)i, b, c));
    const float uI = uniform_f(philox_word(a, t, (uint32_t)i, b, c));
    const float uQ = uniform_f(philox_word(a, t, (uint32_t)(Nt + i), b, c));
    int jI, jQ;
    float lDI, lDQ;
    if (uc < a.lambda) {
        const int s = nn_draw<Q>(lg, mx, tot, uI);
        jI = s / L;
        jQ = s % L;
        lDI = factor_log2q<L>(aI, c2, inv2c, kI, jI);
        lDQ = factor_log2q<L>(aQ, c2, inv2c, kQ, jQ);
    } else {
        jI = factor_draw<L>(aI, c2, inv2c, kI, uI, lDI);
        jQ = factor_draw<L>(aQ, c2, inv2c, kQ, uQ, lDQ);
    }
    const float lN = fmaf(lg[jI * L + jQ], kLog2e, -lse2);
    a.prop[base + i] = (int8_t)jI;
    a.prop[base + Nt + i] = (int8_t)jQ;
    a.lqf[row] = log2_add(a.l2w_plain + lDI + lDQ, a.l2w_nn + lN);
}

// Metropolis-Hastings test of the mixture move (one warp per chain).
template <int L>
__global__ void __launch_bounds__(128) accept_kernel(MixStepArgs a)
{
    constexpr int Q = L * L;
    const int b = blockIdx.y;
    const ChannelDesc d = a.desc[b];
    if (d.L != L) return;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (c >= a.chains) return;
    const int Nt = d.Nt, N = d.N;
    const long long base = d.state_off + (long long)c * N;
    const bool pre = d.NO > N;
    const float *z = a.z32 + d.vec_off, *w = a.w32 + d.vec_off;
    const float c2 = (float)d.cquad * kLog2e, inv2c = 0.5f / c2;
    float lq = 0.f;   // sum over antennas of log2 q_mix(x | x') - log2 q_mix(x' | x)
    for (int i = lane; i < Nt; i += 32) {
        const long long row = d.state_off / 2 + (long long)c * Nt + i;
        const int kI = a.states[base + i], kQ = a.states[base + Nt + i];
        const int jI = a.prop[base + i], jQ = a.prop[base + Nt + i];
        const float aI = slope2(d, pre, z[i], w[i], a.gxp[base + i], a.pxp[base + i]);
        const float aQ = slope2(d, pre, z[Nt + i], w[Nt + i], a.gxp[base + Nt + i], a.pxp[base + Nt + i]);
        const float lD = factor_log2q<L>(aI, c2, inv2c, jI, kI) + factor_log2q<L>(aQ, c2, inv2c, jQ, kQ);
        const float *lg = a.logits + row * Q;
        float mx, lse2;
        nn_norm<Q>(lg, mx, lse2);
        const float lN = fmaf(lg[kI * L + kQ], kLog2e, -lse2);
        lq += log2_add(a.l2w_plain + lD, a.l2w_nn + lN) - a.lqf[row];
    }
    float sd = 0.f;   // sum_n (x'_n - x_n)(2 zt_n - (Gt x)_n - (Gt x')_n)
    for (int n = lane; n < N; n += 32) {
        const int dk = a.prop[base + n] - a.states[base + n];
        if (dk) sd = fmaf(2.f * (float)dk, 2.f * z[n] - a.gx[base + n] - a.gxp[base + n], sd);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lq += __shfl_xor_sync(0xffffffffu, lq, o);
        sd += __shfl_xor_sync(0xffffffffu, sd, o);
    }
    int ok = 0, impr = 0;
    if (lane == 0) {
        const float logr = fmaf((float)d.cf * kLog2e, sd, lq);
        const float loga = logr < 0.f ? logr : 0.f;
        const float u = uniform_f(philox_word(a, a.t, kMhStream, b, c));
        ok = lg2_approx(u) < loga;
        if (!isfinite(logr)) {
            ok = 0;
            set_status(a.status, kStatusNumeric);
        }
        if (ok) {
            const long long ci = (long long)b * a.chains + c;
            const double fn = a.f[ci] + d.inv_s2 * (double)sd;
            a.f[ci] = fn;
            a.accepts[ci] += 1;
            if (fn > a.best_f[ci]) {
                a.best_f[ci] = fn;
                impr = 1;
            }
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    impr = __shfl_sync(0xffffffffu, impr, 0);
    if (ok) {
        for (int n = lane; n < N; n += 32) {
            const int8_t v = a.prop[base + n];
            a.states_out[base + n] = v;
            if (impr) a.best_states[base + n] = v;
        }
    }
}

// Warm start: per channel and group of antennas, the network's cumulative weights at x = 0 are
// formed once in shared memory (one thread per antenna); then one thread per (antenna, chain)
// draws with its t = 0 uniform.
constexpr int kWarmAnt = 4;   // antennas per CTA (block = kWarmAnt x 64 threads)

template <int L>
__global__ void __launch_bounds__(256) init_learned_kernel(MixStepArgs a)
{
    constexpr int Q = L * L;
    __shared__ float S[kWarmAnt][Q];
    const int b = blockIdx.y;
    const ChannelDesc d = a.desc[b];
    if (d.L != L) return;
    const int Nt = d.Nt, N = d.N;
    const int i0 = blockIdx.x * kWarmAnt;
    if (i0 >= Nt) return;
    if (threadIdx.x < kWarmAnt && i0 + (int)threadIdx.x < Nt) {
        const float *lg = a.logits + (d.ant_off + i0 + threadIdx.x) * Q;
        float mx, lse2;
        nn_norm<Q>(lg, mx, lse2);
        float acc = 0.f;
        for (int s = 0; s < Q; ++s) {
            acc += ex2_approx(fmaf(lg[s], kLog2e, -mx));
            S[threadIdx.x][s] = acc;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kWarmAnt * a.chains; e += blockDim.x) {
        const int ia = e % kWarmAnt, c = e / kWarmAnt;
        const int i = i0 + ia;
        if (i >= Nt) continue;
        const float target = uniform_f(philox_word(a, 0u, (uint32_t)i, b, c)) * S[ia][Q - 1];
        int sel = Q - 1;
        for (int s = 0; s < Q; ++s)
            if (target < S[ia][s]) { sel = s; break; }
        const long long base = d.state_off + (long long)c * N;
        a.states_out[base + i] = (int8_t)(sel / L);
        a.states_out[base + Nt + i] = (int8_t)(sel % L);
    }
}

}  // namespace

cudaError_t launch_gram_features(const MixGramArgs &a, int n_channels, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    dim3 grid((a.chains + kGramChains - 1) / kGramChains, n_channels);
    gram_features_kernel<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_features_zero(const MixGramArgs &a, int n_channels, int max_nt, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    features_zero_kernel<<<dim3((max_nt + 127) / 128, n_channels), 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mix(int which, const MixStepArgs &a, int n_channels, int max_nt, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    const dim3 gthreads((a.chains * max_nt + 127) / 128, n_channels);
    const dim3 gwarps((a.chains + 3) / 4, n_channels);
    const dim3 gwarm((max_nt + kWarmAnt - 1) / kWarmAnt, n_channels);
    switch (which * 10 + a.L) {
    case 2: propose_kernel<2><<<gthreads, 128, 0, s>>>(a); break;
    case 4: propose_kernel<4><<<gthreads, 128, 0, s>>>(a); break;
    case 8: propose_kernel<8><<<gthreads, 128, 0, s>>>(a); break;
    case 12: accept_kernel<2><<<gwarps, 128, 0, s>>>(a); break;
    case 14: accept_kernel<4><<<gwarps, 128, 0, s>>>(a); break;
    case 18: accept_kernel<8><<<gwarps, 128, 0, s>>>(a); break;
    case 22: init_learned_kernel<2><<<gwarm, 256, 0, s>>>(a); break;
    case 24: init_learned_kernel<4><<<gwarm, 256, 0, s>>>(a); break;
    case 28: init_learned_kernel<8><<<gwarm, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace mcmcdet
