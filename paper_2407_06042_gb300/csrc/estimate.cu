// estimate.cu -- read-out of the chains (Sec. III-A hard decision; Sec. III-C, Algorithm 2).
//
// One CTA per channel:
//  * hard decision: the visited state with the largest f (smallest residual), ties to the lowest
//    chain; its f is recomputed in FP64 and its levels are mapped to complex Gray labels;
//  * soft output: IS-based LLR of Eq. (34) in the log-sum-exp form of Eqs. (35)-(36) over the
//    S = Np final states, with F(a) = log(1 + e^a) for the weights (F(gamma) taken as
//    gamma + F(-gamma); exact in FP64, within 6e-8 in FP32) and a running maximum-and-scaled-sum
//    for each log-sum-exp. For bit k on
//    dimension n, x+ and x- differ from the sample in dimension n only (Sec. III-D), so
//        f(x with level k') - f(x) = (1/sigma^2) (2 D (zt_n - (Gt xt)_n) - D^2 Gt_nn),
//    D = 2 (k' - k), needs (Gt xt)_n of the sample only.
#include "common.cuh"
#include "kernels.h"

namespace mcmcdet {

namespace {

template <typename T> struct E;
template <> struct E<float> {
    // F(a) = max(a, 0) + log(1 + e^-|a|); the log of 1 + e^-|a| drops terms below 2^-24
    // (an absolute error under 6e-8, far inside the FP32 read-out's tolerance)
    static __device__ __forceinline__ float softplus(float a)
    {
        return fmaxf(a, 0.f) + __logf(1.f + __expf(-fabsf(a)));
    }
    static __device__ __forceinline__ float ex(float a) { return __expf(a); }
    static __device__ __forceinline__ float lg(float a) { return __logf(a); }
};
template <> struct E<double> {
    static __device__ __forceinline__ double softplus(double a)
    {
        return a > 0.0 ? a + log1p(exp(-a)) : log1p(exp(a));
    }
    static __device__ __forceinline__ double ex(double a) { return exp(a); }
    static __device__ __forceinline__ double lg(double a) { return log(a); }
};

// Running log-sum-exp of Eq. (36) as (m, s), value m + log s, without branches: the running
// maximum moves to max(m, a) and both the sum and the new term are scaled to it (one of the two
// exponentials is exp(0) = 1; exp(-inf) = 0 for the first term).
template <typename T>
struct Lse {
    T m = -INFINITY, s = T(0);
    __device__ __forceinline__ void add(T a)
    {
        if (a == -INFINITY) return;
        const T mn = m > a ? m : a;
        s = s * E<T>::ex(m - mn) + E<T>::ex(a - mn);
        m = mn;
    }
    __device__ __forceinline__ T value() const { return s > T(0) ? m + E<T>::lg(s) : T(-INFINITY); }
};

// running log-sum-exp, Eq. (36)
template <typename T>
__device__ __forceinline__ T lse_push(T v, T a)
{
    if (v == -INFINITY) return a;
    if (a == -INFINITY) return v;
    const T m = v > a ? v : a;
    const T dlt = v > a ? a - v : v - a;
    return m + E<T>::softplus(dlt);
}

// launched with 256 threads (8 warps)
template <typename T>
__global__ void __launch_bounds__(256) estimate_kernel(const EstimateArgs A)
{
    const int b = blockIdx.x;
    const ChannelDesc d = A.desc[b];
    const int N = d.N, L = d.L, B = d.log2L, Np = A.chains, nt = d.Nt;
    const int8_t *S = A.states + d.state_off;
    const double *f = A.f + (long long)b * Np;
    const T *G = reinterpret_cast<const T *>(A.G) + (A.g_is_bt ? d.bt_off : d.mat_off);
    const int gstride = A.g_is_bt ? d.NOp : N;
    const T *z = reinterpret_cast<const T *>(A.z) + d.vec_off;
    const T inv_s2 = (T)d.inv_s2;
    const T tau = (T)d.tau;
    const T w = (tau - T(1)) / tau;
    const T inv_tau = T(1) / tau;
    __shared__ int s_best;
    __shared__ double s_fref;
    __shared__ T s_part[2 * 3 * kMaxN];      // partial LSEs (split 0 stored, others merged)
    __shared__ T s_fs[1024];                 // f(x_s) - f_ref of every sample (FP64 difference)

    // hard decision and the reference energy of the soft output
    if (threadIdx.x < 32) {
        double bv = -INFINITY, fm = -INFINITY;
        int bi = 0x7fffffff;
        for (int c = threadIdx.x; c < Np; c += 32) {
            const double v = A.best_f[(long long)b * Np + c];
            if (v > bv || (v == bv && c < bi)) { bv = v; bi = c; }
            fm = f[c] > fm ? f[c] : fm;
        }
        for (int o = 16; o; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            const double of = __shfl_xor_sync(0xffffffffu, fm, o);
            fm = of > fm ? of : fm;
        }
        if (threadIdx.x == 0) { s_best = bi; s_fref = fm; }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < Np; c += blockDim.x) s_fs[c] = (T)(f[c] - s_fref);
    const int8_t *kb = A.best_states + d.state_off + (long long)s_best * N;
    // FP64 energy of the best sample, x^T Gt x row by row: a warp takes every 8th row and its
    // lanes the columns (coalesced rows), all rows in flight at once
    __shared__ double s_x[kMaxN];
    __shared__ double s_ql[2 * 8];
    for (int n = threadIdx.x; n < N; n += blockDim.x) s_x[n] = (double)odd_of(kb[n], L);
    __syncthreads();
    {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const double *G64 = A.G64 + d.mat_off;
        const double *z64 = A.z64 + d.vec_off;
        double quad = 0.0, lin = 0.0;
        for (int n = warp; n < N; n += 8) {
            const double *g = G64 + (long long)n * N;
            double sr = 0.0;
            for (int m = lane; m < N; m += 32) sr = fma(g[m], s_x[m], sr);
            quad = fma(s_x[n], sr, quad);
        }
        for (int n = threadIdx.x; n < N; n += blockDim.x) lin = fma(s_x[n], z64[n], lin);
        for (int o = 16; o; o >>= 1) {
            quad += __shfl_xor_sync(0xffffffffu, quad, o);
            lin += __shfl_xor_sync(0xffffffffu, lin, o);
        }
        if (lane == 0) {
            s_ql[2 * warp] = quad;
            s_ql[2 * warp + 1] = lin;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && A.best_f_out) {
        double quad = 0.0, lin = 0.0;
        for (int w8 = 0; w8 < 8; ++w8) {
            quad += s_ql[2 * w8];
            lin += s_ql[2 * w8 + 1];
        }
        A.best_f_out[b] = -(A.yy[b] - 2.0 * lin + quad) * d.inv_s2;
    }
    if (A.best_idx) {
        for (int i = threadIdx.x; i < nt; i += blockDim.x)
            A.best_idx[d.ant_off + i] = (int8_t)((gray_of(kb[i]) << B) | gray_of(kb[nt + i]));
    }
    if (!A.llr) return;

    // soft output: thread (n, sp) handles samples s = sp, sp + split, ...
    const int split = max(1, (int)blockDim.x / N);
    const int n = threadIdx.x % N, sp = threadIdx.x / N;
    const bool active = sp < split && (int)threadIdx.x < split * N;
    Lse<T> vp[3], vm[3];
    if (active) {
        const T gnn = G[(long long)n * gstride + n];
        for (int s = sp; s < Np; s += split) {
            const int8_t *ks = S + (long long)s * N;
            T Dn = T(0);
            if (A.dexp) Dn = (T)A.dexp[d.state_off + (long long)s * N + n];
            else
                for (int m = 0; m < N; ++m) Dn = fma(G[(long long)n * gstride + m], (T)odd_of(ks[m], L), Dn);
            const int k = ks[n];
            const T r = z[n] - Dn;
            const T fs = s_fs[s];
            const int g = gray_of(k);
            for (int p = 0; p < B; ++p) {
                const int mask = 1 << (B - 1 - p);
                const int kpl = level_of_gray(g & ~mask), kmi = level_of_gray(g | mask);
                const T dp = T(2 * (kpl - k)), dm = T(2 * (kmi - k));
                const T dfp = inv_s2 * (T(2) * dp * r - dp * dp * gnn);
                const T dfm = inv_s2 * (T(2) * dm * r - dm * dm * gnn);
                const T gam = (dfp - dfm) * inv_tau;
                const T fmg = E<T>::softplus(-gam);   // F(gam) = gam + F(-gam)
                vp[p].add(w * (fs + dfp) - fmg);
                vm[p].add(w * (fs + dfm) - (gam + fmg));
            }
        }
    }
    // merge the partial sums of the split threads of each dimension
    for (int r = 0; r < split; ++r) {
        __syncthreads();
        if (active && sp == r) {
            for (int p = 0; p < B; ++p) {
                T *slot = s_part + 2 * (p * kMaxN + n);
                const T a = vp[p].value(), c = vm[p].value();
                if (r == 0) { slot[0] = a; slot[1] = c; }
                else { slot[0] = lse_push(slot[0], a); slot[1] = lse_push(slot[1], c); }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < N * B; e += blockDim.x) {
        const int nn = e / B, p = e % B;
        const T *slot = s_part + 2 * (p * kMaxN + nn);
        const T llr = slot[0] - slot[1];
        if (!isfinite((double)llr)) set_status(A.status, kStatusNumeric);
        const int ant = nn % nt, part = nn / nt;
        A.llr[d.bit_off + (long long)ant * 2 * B + part * B + p] = (float)llr;
    }
}

// List-based soft output, Eq. (31): the sample list (the Np final states) stands in for the whole
// state space, over its distinct vectors. One CTA per channel: a 64-bit FNV-1a hash of every
// chain's levels, a chain kept unless an earlier one holds the same levels (hash match, then a
// full comparison), the FP64 energies relative to the largest kept one, then per bit a running
// log-sum-exp over the kept states on each side. A side with no state gives -clip or +clip, and
// every value is clipped to [-clip, clip] (the paper leaves empty sides open).
template <typename T>
__global__ void __launch_bounds__(256) list_llr_kernel(const ListLlrArgs A)
{
    const int b = blockIdx.x;
    const ChannelDesc d = A.desc[b];
    const int N = d.N, B = d.log2L, Np = A.chains, nt = d.Nt;
    const int8_t *S = A.states + d.state_off;
    const double *f = A.f + (long long)b * Np;
    __shared__ unsigned long long s_h[1024];
    __shared__ unsigned char s_keep[1024];
    __shared__ T s_fs[1024];
    __shared__ double s_red[8];
    const int tid = threadIdx.x;
    for (int c = tid; c < Np; c += blockDim.x) {
        unsigned long long h = 14695981039346656037ull;
        for (int n = 0; n < N; ++n) {
            h ^= (unsigned char)S[(long long)c * N + n];
            h *= 1099511628211ull;
        }
        s_h[c] = h;
    }
    __syncthreads();
    double fm = -INFINITY;
    for (int c = tid; c < Np; c += blockDim.x) {
        bool keep = true;
        for (int r = 0; r < c && keep; ++r) {
            if (s_h[r] != s_h[c]) continue;
            bool same = true;
            for (int n = 0; n < N && same; ++n) same = S[(long long)r * N + n] == S[(long long)c * N + n];
            keep = !same;
        }
        s_keep[c] = keep;
        if (keep) fm = fmax(fm, f[c]);
    }
    for (int o = 16; o; o >>= 1) fm = fmax(fm, __shfl_xor_sync(0xffffffffu, fm, o));
    if ((tid & 31) == 0) s_red[tid >> 5] = fm;
    __syncthreads();
    fm = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) fm = fmax(fm, s_red[w]);
    for (int c = tid; c < Np; c += blockDim.x) s_fs[c] = (T)(f[c] - fm);
    __syncthreads();
    const T clip = (T)A.clip;
    for (int kb = tid; kb < N * B; kb += blockDim.x) {
        const int ant = kb / (2 * B), r = kb % (2 * B);
        const int n = r < B ? ant : nt + ant, pos = r < B ? r : r - B;
        const int mask = 1 << (B - 1 - pos);
        Lse<T> vp, vm;
        for (int c = 0; c < Np; ++c) {
            if (!s_keep[c]) continue;
            if (gray_of(S[(long long)c * N + n]) & mask) vm.add(s_fs[c]);
            else vp.add(s_fs[c]);
        }
        T v = !(vp.s > T(0)) ? -clip : !(vm.s > T(0)) ? clip : vp.value() - vm.value();
        if (!isfinite((double)v)) set_status(A.status, kStatusNumeric);
        v = v > clip ? clip : (v < -clip ? -clip : v);
        A.llr[d.bit_off + kb] = (float)v;
    }
}

}  // namespace

cudaError_t launch_list_llr(const ListLlrArgs &a, bool fp64, cudaStream_t s)
{
    if (a.n_channels <= 0) return cudaSuccess;
    if (fp64) list_llr_kernel<double><<<a.n_channels, 256, 0, s>>>(a);
    else list_llr_kernel<float><<<a.n_channels, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_estimate(const EstimateArgs &a, bool fp64, cudaStream_t s)
{
    if (a.n_channels <= 0) return cudaSuccess;
    if (fp64) estimate_kernel<double><<<a.n_channels, 256, 0, s>>>(a);
    else estimate_kernel<float><<<a.n_channels, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mcmcdet
