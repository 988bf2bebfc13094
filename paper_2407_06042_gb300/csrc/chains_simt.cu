// chains_simt.cu -- DMALA chain kernel on CUDA cores (FP64 parity mode and the plain FP32
// sampler): Algorithm 1's loop for a group of chains of one channel per CTA.
//
// Per transition t (Algorithm 1, loop body, in order):
//   1. x'_n ~ q_n(. | x_n) for every (chain, n) from the cached drift slope of the current
//      state (Eqs. (15)-(17) / (21)); log q(x'|x) accumulated;
//   2. one small GEMM  D' = X' [Gt | P~ Gt]  gives Gt x' (energy) and the drift at x' (Eq. (10));
//   3. the reverse factors q_n(x_n | x'_n) and the energy difference (Eqs. (3), (18));
//   4. per chain: log A = min(0, df/tau + log q(x|x') - log q(x'|x)); accept iff log u < log A;
//   5. accepted chains take x', Gt x' and the drift slope of x' (the proposal cache of
//      Algorithm 1's accept branch).
// The drift slope and Gt x of a state are pure functions of that state, so a run split into
// several launches (resume) makes exactly the same decisions as one launch.
#include "common.cuh"
#include "kernels.h"
#include "proposal.cuh"

namespace mcmcdet {

namespace {

template <typename T> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg(float x) { return __logf(x); }
    static __device__ __forceinline__ float uni(uint32_t w) { return uniform_f(w); }
};
template <> struct M<double> {
    static __device__ __forceinline__ double ex(double x) { return exp(x); }
    static __device__ __forceinline__ double lg(double x) { return log(x); }
    static __device__ __forceinline__ double uni(uint32_t w) { return uniform_d(w); }
};

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout (byte offsets), identical for every work item of a launch.
struct Layout {
    size_t bt, zt, wt, a, D, Dp, xsT, term, dterm, fcur, fbest, acc, impr, cnt, tie, k, kp, kb, total;
};

__host__ __device__ inline Layout make_layout(int es, int cg, int N, int NOp, bool bt_smem)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 16); return r; };
    L.bt = take(bt_smem ? (size_t)N * NOp * es : 0);
    L.zt = take((size_t)N * es);
    L.wt = take((size_t)N * es);
    L.a = take((size_t)cg * N * es);
    L.D = take((size_t)cg * N * es);
    L.Dp = take((size_t)cg * NOp * es);
    L.xsT = take((size_t)N * (cg + 4) * es);   // row stride cg + 4: conflict-light column writes
    L.term = take((size_t)cg * N * es);
    L.dterm = take((size_t)cg * N * es);
    L.fcur = take((size_t)cg * 8);
    L.fbest = take((size_t)cg * 8);
    L.acc = take((size_t)cg * 4);
    L.impr = take((size_t)cg * 4);
    L.cnt = take((size_t)cg * 4);
    L.tie = take(3 * 4);                        // near-tie counts of the work item, three windows
    L.k = take((size_t)cg * N);
    L.kp = take((size_t)cg * N);
    L.kb = take((size_t)cg * N);
    L.total = o;
    return L;
}

template <typename T, int NV> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<double, 2> { using type = double2; };

template <typename T, int CNT>
__device__ __forceinline__ void load_row(const T *p, T (&v)[CNT])
{
    constexpr int NV = sizeof(T) == 4 ? 4 : 2;
    using V = typename Vec<T, NV>::type;
#pragma unroll
    for (int i = 0; i < CNT / NV; ++i) {
        const V q = reinterpret_cast<const V *>(p)[i];
        if constexpr (NV == 4) { v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w; }
        else { v[2 * i] = q.x; v[2 * i + 1] = q.y; }
    }
}

template <typename T, int CNT>
__device__ __forceinline__ void store_row(T *p, const T (&v)[CNT])
{
    constexpr int NV = sizeof(T) == 4 ? 4 : 2;
    using V = typename Vec<T, NV>::type;
#pragma unroll
    for (int i = 0; i < CNT / NV; ++i) {
        V q;
        if constexpr (NV == 4) { q.x = v[4 * i]; q.y = v[4 * i + 1]; q.z = v[4 * i + 2]; q.w = v[4 * i + 3]; }
        else { q.x = v[2 * i]; q.y = v[2 * i + 1]; }
        reinterpret_cast<V *>(p)[i] = q;
    }
}

// D'[c][o] = sum_m bt[m][o] xsT[m][c] for the active chains; register tile TCH x TO.
template <typename T, int TCH, int TO>
__device__ __forceinline__ void gemm(const T *__restrict__ bt, int NOp, const T *xsT, int xld, int N,
                                     T *Dp, int nC)
{
    const int nOT = NOp / TO, nCT = (nC + TCH - 1) / TCH;
    for (int tile = threadIdx.x; tile < nOT * nCT; tile += blockDim.x) {
        const int o0 = (tile % nOT) * TO, c0 = (tile / nOT) * TCH;
        T acc[TCH][TO];
#pragma unroll
        for (int i = 0; i < TCH; ++i)
#pragma unroll
            for (int j = 0; j < TO; ++j) acc[i][j] = T(0);
#pragma unroll 2
        for (int m = 0; m < N; ++m) {
            T xv[TCH], bv[TO];
            load_row<T, TCH>(xsT + (size_t)m * xld + c0, xv);
            load_row<T, TO>(bt + (size_t)m * NOp + o0, bv);
#pragma unroll
            for (int i = 0; i < TCH; ++i)
#pragma unroll
                for (int j = 0; j < TO; ++j) acc[i][j] = fma(xv[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < TCH; ++i) store_row<T, TO>(Dp + (size_t)(c0 + i) * NOp + o0, acc[i]);
    }
}

// Proposal factor of one dimension: logits a (j - k) - cq (j - k)^2 for j < L, their maximum,
// the cumulative weights S_j = sum_{i<=j} exp(logit_i - max) and their total S_{L-1}.
template <typename T>
struct Factor {
    T mx;
    T total;
    T S[kMaxL];
};

template <typename T>
__device__ __forceinline__ T logit_of(T a, T cq, int j, int k)
{
    const T dj = T(j - k);
    return a * dj - cq * dj * dj;
}

template <typename T, int L>
__device__ __forceinline__ void factor(T a, T cq, int k, Factor<T> &F)
{
    T lg[L];
    T mx = -T(1e30);
#pragma unroll
    for (int j = 0; j < L; ++j) {
        lg[j] = logit_of(a, cq, j, k);
        mx = lg[j] > mx ? lg[j] : mx;
    }
    F.mx = mx;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < L; ++j) {
        acc += M<T>::ex(lg[j] - mx);
        F.S[j] = acc;
    }
    F.total = acc;
}

// Draw of one factor and log q of the drawn level. FP64: natural logs, every weight exp'd
// directly (as the definition reads). FP32: the shared log2-unit arithmetic of proposal.cuh.
template <typename T, int L>
__device__ __forceinline__ int draw_level(T a, T cq, T inv2c, int k, uint32_t word, T &logq)
{
    if constexpr (sizeof(T) == 8) {
        Factor<T> F;
        factor<T, L>(a, cq, k, F);
        const T target = M<T>::uni(word) * F.total;
        int sel = L - 1;
#pragma unroll
        for (int l = L - 1; l >= 0; --l)
            if (target < F.S[l]) sel = l;
        logq = logit_of(a, cq, sel, k) - F.mx - M<T>::lg(F.total);
        return sel;
    } else {
        float lq;
        const int sel = factor_draw<L>(a, cq, inv2c, k, uniform_f(word), lq);
        logq = lq;
        return sel;
    }
}

template <typename T, int L>
__device__ __forceinline__ T log_q_of(T a, T cq, T inv2c, int k, int j_eval)
{
    if constexpr (sizeof(T) == 8) {
        Factor<T> F;
        factor<T, L>(a, cq, k, F);
        return logit_of(a, cq, j_eval, k) - F.mx - M<T>::lg(F.total);
    } else {
        return factor_log2q<L>(a, cq, inv2c, k, j_eval);
    }
}

// Units: FP64 works in natural logs; FP32 in log2 units (slopes, curvature and the energy
// scale pre-multiplied by log2 e), as in proposal.cuh.
template <typename T, int TCH, int TO, int L>
__device__ void simt_item(const ChainArgs &A, const WorkItem &it, const ChannelDesc &d)
{
    const int N = d.N, NOp = d.NOp, cg = A.cg, nC = it.nc;
    const int xld = cg + 4;                        // row stride of xsT
    const bool pre = d.NO > N;
    const T unit = sizeof(T) == 8 ? T(1) : (T)kLog2e;
    const T clin = (T)d.clin * unit, cq = (T)d.cquad * unit, cf = (T)d.cf * unit;
    const T inv2c = T(0.5) / cq;
    const Layout lay = make_layout(sizeof(T), cg, A.max_n, A.max_nop, A.bt_in_smem);
    extern __shared__ __align__(16) unsigned char smem[];
    T *zt = reinterpret_cast<T *>(smem + lay.zt);
    T *wt = reinterpret_cast<T *>(smem + lay.wt);
    T *sa = reinterpret_cast<T *>(smem + lay.a);
    T *sD = reinterpret_cast<T *>(smem + lay.D);
    T *Dp = reinterpret_cast<T *>(smem + lay.Dp);
    T *xsT = reinterpret_cast<T *>(smem + lay.xsT);
    T *term = reinterpret_cast<T *>(smem + lay.term);
    T *dterm = reinterpret_cast<T *>(smem + lay.dterm);
    double *fcur = reinterpret_cast<double *>(smem + lay.fcur);
    double *fbest = reinterpret_cast<double *>(smem + lay.fbest);
    int *acc = reinterpret_cast<int *>(smem + lay.acc);
    int *impr = reinterpret_cast<int *>(smem + lay.impr);
    unsigned *cnt = reinterpret_cast<unsigned *>(smem + lay.cnt);
    unsigned *ties = reinterpret_cast<unsigned *>(smem + lay.tie);
    int8_t *sk = reinterpret_cast<int8_t *>(smem + lay.k);
    int8_t *skp = reinterpret_cast<int8_t *>(smem + lay.kp);
    int8_t *skb = reinterpret_cast<int8_t *>(smem + lay.kb);

    const T *gbt = reinterpret_cast<const T *>(A.bt) + d.bt_off;
    const T *bt = gbt;
    if (A.bt_in_smem) {
        T *sbt = reinterpret_cast<T *>(smem + lay.bt);
        for (int e = threadIdx.x; e < N * NOp; e += blockDim.x) sbt[e] = gbt[e];
        bt = sbt;
    }
    const T *gz = reinterpret_cast<const T *>(A.z) + d.vec_off;
    const T *gw = reinterpret_cast<const T *>(A.w) + d.vec_off;
    for (int n = threadIdx.x; n < N; n += blockDim.x) { zt[n] = gz[n]; wt[n] = gw[n]; }
    const long long sbase = d.state_off + (long long)it.c0 * N;
    for (int e = threadIdx.x; e < nC * N; e += blockDim.x) {
        const int c = e / N, n = e % N;
        const int8_t kv = A.states[sbase + e];
        sk[c * N + n] = kv;
        skb[c * N + n] = A.best_states[sbase + e];
        xsT[n * xld + c] = (T)odd_of(kv, L);
    }
    for (int c = threadIdx.x; c < cg; c += blockDim.x) {
        const long long ci = (long long)it.b * A.chains + it.c0 + c;
        fcur[c] = c < nC ? A.f[ci] : 0.0;
        fbest[c] = c < nC ? A.best_f[ci] : 0.0;
        cnt[c] = 0;
    }
    if (threadIdx.x < 3) ties[threadIdx.x] = 0u;
    __syncthreads();
    // Gt x and the drift slope of the current states
    gemm<T, TCH, TO>(bt, NOp, xsT, xld, N, Dp, nC);
    __syncthreads();
    for (int e = threadIdx.x; e < nC * N; e += blockDim.x) {
        const int c = e / N, n = e % N;
        const T dg = Dp[c * NOp + n];
        sD[e] = dg;
        sa[e] = clin * (pre ? (wt[n] - Dp[c * NOp + N + n]) : (zt[n] - dg));
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    if (A.init_f) {
        // tracked energies of the current states from Gt x (FP32 products, FP64 sums); the
        // running best restarts from them
        for (int c = warp; c < nC; c += nwarps) {
            double quad = 0.0, lin = 0.0;
            for (int n = lane; n < N; n += 32) {
                const double xn = odd_of(sk[c * N + n], L);
                quad += xn * (double)sD[c * N + n];
                lin += xn * (double)zt[n];
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                quad += __shfl_xor_sync(0xffffffffu, quad, o);
                lin += __shfl_xor_sync(0xffffffffu, lin, o);
            }
            if (lane == 0) {
                const double f0 = -(A.yy[it.b] - 2.0 * lin + quad) * d.inv_s2;
                fcur[c] = f0;
                fbest[c] = f0;
            }
        }
        for (int e = threadIdx.x; e < nC * N; e += blockDim.x) skb[e] = sk[e];
        __syncthreads();
    }
    for (int i = 0; i < A.iterations; ++i) {
        const uint32_t t = (uint32_t)(A.t_offset + 1 + i);
        // 1. proposal draw, four chains per Philox block
        for (int q = threadIdx.x; q < (nC / 4) * N; q += blockDim.x) {
            const int cq4 = q / N, n = q % N;
            const U4 w = philox4x32_10_rk(t, (uint32_t)n, (uint32_t)it.b,
                                          (uint32_t)((it.c0 >> 2) + cq4), A.philox_rk);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * cq4 + j;
                const int e = c * N + n;
                const int kn = sk[e];
                T lq;
                const int sel = draw_level<T, L>(sa[e], cq, inv2c, kn, word_of(w, j), lq);
                skp[e] = (int8_t)sel;
                term[e] = -lq;
                xsT[n * xld + c] = (T)odd_of(sel, L);
            }
        }
        __syncthreads();
        // 2. D' = X' [Gt | P~ Gt]
        gemm<T, TCH, TO>(bt, NOp, xsT, xld, N, Dp, nC);
        __syncthreads();
        // 3. reverse factor and energy difference per (chain, n)
        for (int e = threadIdx.x; e < nC * N; e += blockDim.x) {
            const int c = e / N, n = e % N;
            const int kn = sk[e], kpn = skp[e];
            const T dgp = Dp[c * NOp + n];
            const T ap = clin * (pre ? (wt[n] - Dp[c * NOp + N + n]) : (zt[n] - dgp));
            term[e] += log_q_of<T, L>(ap, cq, inv2c, kpn, kn);
            dterm[e] = T(2 * (kpn - kn)) * (T(2) * zt[n] - sD[e] - dgp);
        }
        __syncthreads();
        // 4. Metropolis-Hastings decision, one warp per chain
        for (int c = warp; c < nC; c += nwarps) {
            T s = T(0), sd = T(0);
            for (int n = lane; n < N; n += 32) { s += term[c * N + n]; sd += dterm[c * N + n]; }
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                s += __shfl_xor_sync(0xffffffffu, s, o);
                sd += __shfl_xor_sync(0xffffffffu, sd, o);
            }
            if (lane == 0) {
                const int cc = it.c0 + c;
                const U4 w = philox4x32_10_rk(t, kMhStream, (uint32_t)it.b, (uint32_t)(cc >> 2),
                                              A.philox_rk);
                const T logr = s + cf * sd;
                const T loga = logr < T(0) ? logr : T(0);
                const T u = M<T>::uni(word_of(w, cc & 3));
                const T logu = sizeof(T) == 8 ? M<T>::lg(u) : (T)lg2_approx((float)u);
                int ok = logu < loga;
                if (!isfinite((double)logr)) { ok = 0; set_status(A.status, kStatusNumeric); }
                // near-tie bands |log A - log u| < 1e-6, 1e-4, 1e-2 (natural log; the kernel's
                // units are log2 in FP32, natural in FP64)
                const T gap = loga > logu ? loga - logu : logu - loga;
                if (gap < T(1e-2) * unit) {
                    atomicAdd(&ties[2], 1u);
                    if (gap < T(1e-4) * unit) atomicAdd(&ties[1], 1u);
                    if (gap < T(1e-6) * unit) atomicAdd(&ties[0], 1u);
                }
                if (A.trace)
                    reinterpret_cast<double2 *>(A.trace)[(long long)it.b * A.chains + cc] =
                        make_double2((double)logr / (double)unit, (double)logu / (double)unit);
                acc[c] = ok;
                int im = 0;
                if (ok) {
                    const double fn = fcur[c] + d.inv_s2 * (double)sd;
                    fcur[c] = fn;
                    cnt[c] += 1;
                    if (fn > fbest[c]) { fbest[c] = fn; im = 1; }
                }
                impr[c] = im;
            }
        }
        __syncthreads();
        // 5. accepted chains take x' and its caches
        for (int e = threadIdx.x; e < nC * N; e += blockDim.x) {
            const int c = e / N, n = e % N;
            if (acc[c]) {
                const int8_t kv = skp[e];
                sk[e] = kv;
                const T dgp = Dp[c * NOp + n];
                sD[e] = dgp;
                sa[e] = clin * (pre ? (wt[n] - Dp[c * NOp + N + n]) : (zt[n] - dgp));
                if (impr[c]) skb[e] = kv;
            }
        }
        __syncthreads();
        // periodic FP64 refresh of the tracked energies (decisions never read them)
        if (sizeof(T) == 4 && A.refresh_period > 0 && (t % (uint32_t)A.refresh_period) == 0u) {
            const double *G = A.G64 + d.mat_off;
            const double *z = A.z64 + d.vec_off;
            for (int c = warp; c < nC; c += nwarps) {
                double quad, lin;
                quad_lin_fp64(G, z, N, lane, [&](int n) { return (double)odd_of(sk[c * N + n], L); },
                              quad, lin);
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    quad += __shfl_xor_sync(0xffffffffu, quad, o);
                    lin += __shfl_xor_sync(0xffffffffu, lin, o);
                }
                if (lane == 0) {
                    const double f64 = -(A.yy[it.b] - 2.0 * lin + quad) * d.inv_s2;
                    const double dr = fabs(f64 - fcur[c]);
                    atomicMax(A.drift_bits, (unsigned long long)__double_as_longlong(dr));
                    fcur[c] = f64;
                }
            }
            __syncthreads();
        }
    }
    // write back
    for (int e = threadIdx.x; e < nC * N; e += blockDim.x) {
        A.states[sbase + e] = sk[e];
        A.best_states[sbase + e] = skb[e];
        if (A.dexp) A.dexp[sbase + e] = (float)sD[e];
    }
    for (int c = threadIdx.x; c < nC; c += blockDim.x) {
        const long long ci = (long long)it.b * A.chains + it.c0 + c;
        A.f[ci] = fcur[c];
        A.best_f[ci] = fbest[c];
        A.accepts[ci] += cnt[c];
    }
    if (threadIdx.x < 3 && A.near_ties && ties[threadIdx.x])
        atomicAdd(&A.near_ties[threadIdx.x], (unsigned long long)ties[threadIdx.x]);
}

template <typename T, int TCH, int TO>
__global__ void __launch_bounds__(256) chains_simt_kernel(const ChainArgs A)
{
    const WorkItem it = A.items[blockIdx.x];
    const ChannelDesc d = A.desc[it.b];
    switch (d.L) {
    case 2: simt_item<T, TCH, TO, 2>(A, it, d); break;
    case 4: simt_item<T, TCH, TO, 4>(A, it, d); break;
    default: simt_item<T, TCH, TO, 8>(A, it, d); break;
    }
}

}  // namespace

size_t chain_smem_bytes_simt(int elem_size, int cg, int max_n, int max_nop, bool bt_in_smem)
{
    return make_layout(elem_size, cg, max_n, max_nop, bt_in_smem).total;
}

cudaError_t launch_chains_simt(const ChainArgs &a_in, bool fp64, size_t smem, cudaStream_t s)
{
    if (a_in.n_items <= 0) return cudaSuccess;
    ChainArgs a = a_in;
    philox_round_keys(a.key0, a.key1, a.philox_rk);
    cudaError_t e;
    if (fp64) {
        auto k = chains_simt_kernel<double, 4, 4>;
        if ((e = allow_max_dyn_smem(k)) != cudaSuccess) return e;
        k<<<a.n_items, 256, smem, s>>>(a);
    } else {
        auto k = chains_simt_kernel<float, 8, 4>;
        if ((e = allow_max_dyn_smem(k)) != cudaSuccess) return e;
        k<<<a.n_items, 256, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace mcmcdet
