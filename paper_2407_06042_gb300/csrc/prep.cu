// prep.cu -- per-channel preparation (Sec. II-A, Eq. (10); Remark 1, Eq. (19); Sec. III-D):
// the complex Gram matrix G = H^H H, the matched filter z = H^H y and ||y||^2 in FP64, the
// damped inverse (G + gamma I)^{-1} for the preconditioned proposal, the scaled real-valued
// operands every chain kernel reads, the random initial states (t = 0) and their FP64 energies.
//
// One CTA per channel; the work is O(Nr Nt^2 + Nt^3) per channel, done once per batch.
#include "common.cuh"
#include "kernels.h"

#include <cuda_bf16.h>

namespace mcmcdet {

namespace {

struct cd { double x, y; };   // complex double
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cd cmulc(cd a, cd b) { return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x}; } // conj(a) b
__device__ __forceinline__ cd csub(cd a, cd b) { return {a.x - b.x, a.y - b.y}; }

// ------------------------------------------------------------------------------------------
// K1: complex Gram matrix, matched filter, ||y||^2 (FP64 accumulation of FP32 inputs: every
// product of two FP32 values is exact in FP64).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gram_kernel(PrepArgs a)
{
    const int b = blockIdx.x;
    const ChannelDesc d = a.desc[b];
    const int nt = d.Nt, nr = d.Nr;
    const float2 *H = a.H + d.h_off;
    const float2 *y = a.y + d.y_off;
    extern __shared__ float2 sh[];
    const bool staged = a.stage_h;
    float2 *Hs = staged ? sh : nullptr;
    float2 *ys = staged ? sh + (size_t)nt * nr : nullptr;
    if (staged) {
        for (int i = threadIdx.x; i < nt * nr; i += blockDim.x) Hs[i] = H[i];
        for (int i = threadIdx.x; i < nr; i += blockDim.x) ys[i] = y[i];
        __syncthreads();
    }
    const float2 *Hp = staged ? Hs : H;
    const float2 *yp = staged ? ys : y;
    cd *G = reinterpret_cast<cd *>(a.Gc) + d.mat_off / 4;   // Nt^2 complex per channel (mat_off counts N^2 = 4 Nt^2)
    // upper triangle incl. diagonal, mirrored
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        const int i = e / nt, j = e % nt;
        if (j < i) continue;
        double re = 0.0, im = 0.0;
        const float2 *ci = Hp + (size_t)i * nr, *cj = Hp + (size_t)j * nr;
        for (int r = 0; r < nr; ++r) {
            const double ar = ci[r].x, ai = ci[r].y, br = cj[r].x, bi = cj[r].y;
            re = fma(ar, br, re); re = fma(ai, bi, re);
            im = fma(ar, bi, im); im = fma(-ai, br, im);
        }
        G[i * nt + j] = {re, im};
        if (i != j) G[j * nt + i] = {re, -im};
    }
    cd *z = reinterpret_cast<cd *>(a.zc) + d.vec_off / 2;
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        double re = 0.0, im = 0.0;
        const float2 *ci = Hp + (size_t)i * nr;
        for (int r = 0; r < nr; ++r) {
            const double ar = ci[r].x, ai = ci[r].y, br = yp[r].x, bi = yp[r].y;
            re = fma(ar, br, re); re = fma(ai, bi, re);
            im = fma(ar, bi, im); im = fma(-ai, br, im);
        }
        z[i] = {re, im};
    }
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int r = threadIdx.x; r < nr; r += 32) s += (double)yp[r].x * yp[r].x + (double)yp[r].y * yp[r].y;
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) a.yy[b] = s;
    }
}

// ------------------------------------------------------------------------------------------
// K2: (G + gamma I)^{-1} by Gauss-Jordan elimination on [G + gamma I | I] (Hermitian positive
// definite: every pivot is real and positive, no pivoting). The working block lives in shared
// memory when it fits, else in the global scratch block of this channel.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) precond_kernel(PrepArgs a)
{
    const int b = blockIdx.x;
    const ChannelDesc d = a.desc[b];
    const int nt = d.Nt, W = 2 * nt;
    const double gamma = d.gamma_t / (d.dmin * d.dmin);   // gamma in the unscaled model
    extern __shared__ double shd[];
    cd *fac = reinterpret_cast<cd *>(shd);                  // nt factors
    cd *blk = a.stage_gj ? reinterpret_cast<cd *>(shd) + nt
                         : reinterpret_cast<cd *>(a.gj) + d.mat_off / 2;   // nt x 2nt
    const cd *G = reinterpret_cast<const cd *>(a.Gc) + d.mat_off / 4;
    for (int e = threadIdx.x; e < nt * W; e += blockDim.x) {
        const int i = e / W, j = e % W;
        cd v;
        if (j < nt) { v = G[i * nt + j]; if (i == j) v.x += gamma; }
        else v = {(j - nt) == i ? 1.0 : 0.0, 0.0};
        blk[e] = v;
    }
    __syncthreads();
    for (int k = 0; k < nt; ++k) {
        const double piv = blk[k * W + k].x;
        if (threadIdx.x == 0 && !(piv > 0.0)) set_status(a.status, kStatusNumeric);
        const double inv = 1.0 / piv;
        __syncthreads();
        for (int j = threadIdx.x; j < W; j += blockDim.x) {
            cd v = blk[k * W + j];
            blk[k * W + j] = {v.x * inv, v.y * inv};
        }
        for (int i = threadIdx.x; i < nt; i += blockDim.x) fac[i] = blk[i * W + k];
        __syncthreads();
        for (int e = threadIdx.x; e < nt * W; e += blockDim.x) {
            const int i = e / W, j = e % W;
            if (i == k) continue;
            blk[e] = csub(blk[e], cmul(fac[i], blk[k * W + j]));
        }
        __syncthreads();
    }
    cd *M = reinterpret_cast<cd *>(a.Mc) + d.mat_off / 4;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        const int i = e / nt, j = e % nt;
        M[e] = blk[i * W + nt + j];
    }
}

// ------------------------------------------------------------------------------------------
// Emission of the scaled real-valued operands:
//   Gt = d^2 [[Re G, -Im G], [Im G, Re G]]   (FP64, N x N)
//   GMt = P~ Gt = real([(G + gamma I)^{-1} G]) = real(I - gamma M)   (preconditioned only)
//   zt = d [Re z; Im z],  wt = P~ zt = [Re(M z); Im(M z)] / d
//   Bt (N x NOp, the CUDA-core GEMM operand): row m = [Gt row m | GMt row m | 0 pad]
// ------------------------------------------------------------------------------------------
template <typename T>
__device__ void emit_bt(const PrepArgs &a, const ChannelDesc &d, T *bt)
{
    const int N = d.N;
    for (int e = threadIdx.x; e < N * d.NOp; e += blockDim.x) {
        const int m = e / d.NOp, o = e % d.NOp;
        double v = 0.0;
        if (o < N) v = a.G64[d.mat_off + (long long)m * N + o];
        else if (o < d.NO) v = a.GM64[d.mat_off + (long long)m * N + (o - N)];
        bt[e] = (T)v;
    }
}

__global__ void __launch_bounds__(256) emit_kernel(PrepArgs a)
{
    const int b = blockIdx.x;
    const ChannelDesc d = a.desc[b];
    const int nt = d.Nt, N = d.N;
    const double d2 = d.dmin * d.dmin;
    const cd *G = reinterpret_cast<const cd *>(a.Gc) + d.mat_off / 4;
    const cd *z = reinterpret_cast<const cd *>(a.zc) + d.vec_off / 2;
    double *G64 = a.G64 + d.mat_off;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int r = e / N, c = e % N;
        const cd g = G[(r % nt) * nt + (c % nt)];
        const int q = (r >= nt) * 2 + (c >= nt);
        const double v = (q == 0 || q == 3) ? g.x : (q == 1 ? -g.y : g.y);
        G64[e] = d2 * v;
    }
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        a.z64[d.vec_off + i] = d.dmin * z[i].x;
        a.z64[d.vec_off + nt + i] = d.dmin * z[i].y;
    }
    const bool pre = d.NO > N;
    if (pre) {
        const cd *M = reinterpret_cast<const cd *>(a.Mc) + d.mat_off / 4;
        const double gamma = d.gamma_t / d2;
        double *GM = a.GM64 + d.mat_off;
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const int r = e / N, c = e % N;
            const cd m = M[(r % nt) * nt + (c % nt)];
            const int q = (r >= nt) * 2 + (c >= nt);
            double v = (q == 0 || q == 3) ? m.x : (q == 1 ? -m.y : m.y);
            v = -gamma * v + (r == c ? 1.0 : 0.0);
            GM[e] = v;
        }
        for (int i = threadIdx.x; i < nt; i += blockDim.x) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < nt; ++j) {
                const cd p = cmul(M[i * nt + j], z[j]);
                re += p.x; im += p.y;
            }
            a.w64[d.vec_off + i] = re / d.dmin;
            a.w64[d.vec_off + nt + i] = im / d.dmin;
        }
    } else {
        for (int i = threadIdx.x; i < N; i += blockDim.x) a.w64[d.vec_off + i] = 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        a.z32[d.vec_off + i] = (float)a.z64[d.vec_off + i];
        a.w32[d.vec_off + i] = (float)a.w64[d.vec_off + i];
    }
    if (a.bt64) emit_bt<double>(a, d, a.bt64 + d.bt_off);
    if (a.bt32) emit_bt<float>(a, d, a.bt32 + d.bt_off);
}

// ------------------------------------------------------------------------------------------
// Random initial states (t = 0): level = Philox word >> (32 - log2 L); one thread per
// (channel, chain quad, dimension).
// ------------------------------------------------------------------------------------------
__global__ void init_states_kernel(InitArgs a)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = (int)(gid / a.items_per_channel);
    if (b >= a.n_channels) return;
    const int r = (int)(gid % a.items_per_channel);
    const ChannelDesc d = a.desc[b];
    const int quads = a.chains / 4;
    if (r >= quads * d.N) return;
    const int q = r / d.N, n = r % d.N;
    const U4 w = philox4x32_10(0u, (uint32_t)n, (uint32_t)b, (uint32_t)q, a.key0, a.key1);
    for (int j = 0; j < 4; ++j) {
        const int c = 4 * q + j;
        const int lev = (int)(word_of(w, j) >> (32 - d.log2L));
        a.states[d.state_off + (long long)c * d.N + n] = (int8_t)lev;
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// FP64 energies of the current states: f = -(||y||^2 - 2 xt^T zt + xt^T Gt xt) / sigma^2.
// One warp per chain. Optionally also resets the running best to the current state.
// ------------------------------------------------------------------------------------------
__global__ void refresh_kernel(RefreshArgs a)
{
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= (long long)a.n_channels * a.chains) return;
    const int b = (int)(warp / a.chains), c = (int)(warp % a.chains);
    const ChannelDesc d = a.desc[b];
    const int N = d.N, L = d.L;
    const int8_t *k = a.states + d.state_off + (long long)c * N;
    const double *G = a.G64 + d.mat_off;
    const double *z = a.z64 + d.vec_off;
    double quad = 0.0, lin = 0.0;
    bool bad = false;
    for (int n = lane; n < N; n += 32) {
        const int kn = k[n];
        bad |= (kn < 0 || kn >= L);
        const double xn = odd_of(kn, L);
        double s = 0.0;
        for (int m = 0; m < N; ++m) s = fma(G[(long long)n * N + m], (double)odd_of(k[m], L), s);
        quad = fma(xn, s, quad);
        lin = fma(xn, z[n], lin);
    }
    for (int o = 16; o; o >>= 1) {
        quad += __shfl_xor_sync(0xffffffffu, quad, o);
        lin += __shfl_xor_sync(0xffffffffu, lin, o);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) {
        const double f = -(a.yy[b] - 2.0 * lin + quad) * d.inv_s2;
        if (bad) set_status(a.status, kStatusBadState);
        if (!isfinite(f)) set_status(a.status, kStatusNumeric);
        const long long ci = (long long)b * a.chains + c;
        a.f[ci] = f;
        if (a.reset_best) a.best_f[ci] = f;
    }
    if (a.reset_best) {
        int8_t *bk = a.best_states + d.state_off + (long long)c * N;
        for (int n = lane; n < N; n += 32) bk[n] = k[n];
    }
}

// ------------------------------------------------------------------------------------------
// Host launchers
// ------------------------------------------------------------------------------------------
cudaError_t launch_prep(const PrepArgs &a, int n_channels, size_t h_stage_bytes,
                        size_t gj_stage_bytes, bool preconditioned, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    cudaError_t e;
    if (h_stage_bytes > 48 * 1024) {
        e = cudaFuncSetAttribute(gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)h_stage_bytes);
        if (e != cudaSuccess) return e;
    }
    gram_kernel<<<n_channels, 256, a.stage_h ? h_stage_bytes : 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (preconditioned) {
        if (gj_stage_bytes > 48 * 1024) {
            e = cudaFuncSetAttribute(precond_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)gj_stage_bytes);
            if (e != cudaSuccess) return e;
        }
        precond_kernel<<<n_channels, 256, gj_stage_bytes, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    emit_kernel<<<n_channels, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_init_states(const InitArgs &a, cudaStream_t s)
{
    const long long total = (long long)a.n_channels * a.items_per_channel;
    if (total <= 0) return cudaSuccess;
    const int bs = 256;
    init_states_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const RefreshArgs &a, cudaStream_t s)
{
    const long long warps = (long long)a.n_channels * a.chains;
    if (warps <= 0) return cudaSuccess;
    const int bs = 256;
    refresh_kernel<<<(unsigned)((warps * 32 + bs - 1) / bs), bs, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mcmcdet
