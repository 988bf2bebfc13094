// prep.cu -- per-channel preparation (Sec. II-A, Eq. (10); Remark 1, Eq. (19); Sec. III-D):
// the complex Gram matrix G = H^H H, the matched filter z = H^H y and ||y||^2 in FP64, the
// damped inverse (G + gamma I)^{-1} for the preconditioned proposal, the scaled real-valued
// operands every chain kernel reads and the random initial states (t = 0).
//
// One CTA per channel; the work is O(Nr Nt^2 + Nt^3) per channel, done once per batch.
#include "common.cuh"
#include "kernels.h"

#include <cuda_bf16.h>

namespace mcmcdet {

namespace {

struct cd { double x, y; };   // complex double
__device__ __forceinline__ cd cmul(cd a, cd b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

// Float-float accumulator: s is the FP32 running sum, e gathers the exact rounding errors of the
// additions (TwoSum) and of the products (FMA split), so s + e carries ~48 significant bits.
struct FF {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = a * b;
        const float pe = fmaf(a, b, -p);          // exact: a b = p + pe
        const float t = s + p;                    // TwoSum(s, p)
        const float z = t - s;
        const float te = (s - (t - z)) + (p - z);
        s = t;
        e += te + pe;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

// ------------------------------------------------------------------------------------------
// K1: complex Gram matrix, matched filter, ||y||^2 (FP64 accumulation of FP32 inputs: every
// product of two FP32 values is exact in FP64).
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) gram_kernel(PrepArgs a)
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
    // 2 x 2 complex blocks (i0, i0+1) x (j0, j0+1) with i0 <= j0 (upper block triangle); each
    // column pair is read once per r for four complex products
    const int nb = (nt + 1) / 2;
    const int nblk = nb * (nb + 1) / 2;
    for (int e = threadIdx.x; e < nblk; e += blockDim.x) {
        int bi = 0, rem = e;
        while (rem >= nb - bi) { rem -= nb - bi; ++bi; }   // row-major over the block triangle
        const int bj = bi + rem;
        const int i0 = 2 * bi, j0 = 2 * bj;
        const bool i1v = i0 + 1 < nt, j1v = j0 + 1 < nt;
        // float-float accumulation (Ogita-Rump-Oishi Sum2 over exact products): hi / lo per real
        // and imaginary part; every product of two FP32 inputs is split exactly with an FMA
        FF acc[2][2][2];
        const float2 *ci0 = Hp + (size_t)i0 * nr, *ci1 = Hp + (size_t)(i1v ? i0 + 1 : i0) * nr;
        const float2 *cj0 = Hp + (size_t)j0 * nr, *cj1 = Hp + (size_t)(j1v ? j0 + 1 : j0) * nr;
        for (int r = 0; r < nr; ++r) {
            const float2 u0 = ci0[r], u1 = ci1[r], v0 = cj0[r], v1 = cj1[r];
            const float ur[2] = {u0.x, u1.x}, ui[2] = {u0.y, u1.y};
            const float vr[2] = {v0.x, v1.x}, vi[2] = {v0.y, v1.y};
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    // conj(u_p) v_q = (ur vr + ui vi) + i (ur vi - ui vr)
                    acc[p][q][0].add_prod(ur[p], vr[q]);
                    acc[p][q][0].add_prod(ui[p], vi[q]);
                    acc[p][q][1].add_prod(ur[p], vi[q]);
                    acc[p][q][1].add_prod(-ui[p], vr[q]);
                }
        }
#pragma unroll
        for (int p = 0; p < 2; ++p)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int i = i0 + p, j = j0 + q;
                if (i >= nt || j >= nt || j < i) continue;
                const double gr = acc[p][q][0].value(), gi = acc[p][q][1].value();
                G[i * nt + j] = {gr, gi};
                if (i != j) G[j * nt + i] = {gr, -gi};
            }
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

template <typename R> struct CT;
template <> struct CT<float> { struct type { float x, y; }; };
template <> struct CT<double> { using type = cd; };

// ------------------------------------------------------------------------------------------
// K2: M = (G + gamma I)^{-1} (Remark 1, Eq. (19)) by in-place Gauss-Jordan elimination without
// pivoting (G + gamma I is Hermitian positive definite for gamma > 0, so every pivot is real and
// positive in exact arithmetic), in FP64 (FP64 mode) or FP32 (FP32 / MIXED: any deterministic
// preconditioner keeps the chain exact, the proposal staying a function of the state). Step k
// copies row k (times the pivot's inverse) and column k, then every element updates in place:
//     A_kk <- 1/p,  A_kj <- A_kj / p,  A_ik <- -A_ik / p,  A_ij <- A_ij - A_ik A_kj / p.
// The matrix lives in shared memory when it fits, else in the channel's global scratch block.
// ------------------------------------------------------------------------------------------
// Register-tiled form for nt <= 16 T (FP32, 256 threads): thread (ti, tj) of a 16 x 16 grid
// holds rows [T ti, T ti + T) x columns [T tj, T tj + T) of A in registers. At step k the owners
// of row k and column k publish their old values (double-buffered, so one barrier per step
// suffices: a buffer is rewritten two steps later, after every reader has passed the barrier
// between), then every thread updates its tile with the same four rules.
template <int T>
__global__ void __launch_bounds__(256, T == 4 ? 3 : 6) precond_regs_kernel(PrepArgs a)
{
    const ChannelDesc d = a.desc[blockIdx.x];
    const int nt = d.Nt;
    const double gamma = d.gamma_t / (d.dmin * d.dmin);   // gamma in the unscaled model
    using C2 = CT<float>::type;
    __shared__ C2 srow[2][64], scol[2][64];
    const int ti = threadIdx.x >> 4, tj = threadIdx.x & 15;
    const int i0 = T * ti, j0 = T * tj;
    const cd *G = reinterpret_cast<const cd *>(a.Gc) + d.mat_off / 4;
    C2 A[T][T];
#pragma unroll
    for (int r = 0; r < T; ++r)
#pragma unroll
        for (int c = 0; c < T; ++c) {
            const int i = i0 + r, j = j0 + c;
            A[r][c] = {0.f, 0.f};
            if (i < nt && j < nt) {
                const cd g = G[i * nt + j];
                A[r][c] = {(float)(g.x + (i == j ? gamma : 0.0)), (float)g.y};
            }
        }
    for (int k = 0; k < nt; ++k) {
        const int buf = k & 1;
#pragma unroll
        for (int r = 0; r < T; ++r)
            if (i0 + r == k)
#pragma unroll
                for (int c = 0; c < T; ++c) srow[buf][j0 + c] = A[r][c];
#pragma unroll
        for (int c = 0; c < T; ++c)
            if (j0 + c == k)
#pragma unroll
                for (int r = 0; r < T; ++r) scol[buf][i0 + r] = A[r][c];
        __syncthreads();
        const C2 piv = srow[buf][k];
        if (threadIdx.x == 0 && !(piv.x > 0.f)) set_status(a.status, kStatusNumeric);
        const float den = piv.x * piv.x + piv.y * piv.y;
        const C2 pinv = {piv.x / den, -piv.y / den};
        C2 rk[T], ck[T];
#pragma unroll
        for (int c = 0; c < T; ++c) {
            const C2 r = srow[buf][j0 + c];
            rk[c] = {r.x * pinv.x - r.y * pinv.y, r.x * pinv.y + r.y * pinv.x};
        }
#pragma unroll
        for (int r = 0; r < T; ++r) ck[r] = scol[buf][i0 + r];
#pragma unroll
        for (int r = 0; r < T; ++r)
#pragma unroll
            for (int c = 0; c < T; ++c) {
                const bool ik = i0 + r == k, jk = j0 + c == k;
                const C2 cc = ck[r], rr = rk[c], o = A[r][c];
                C2 v = {o.x - (cc.x * rr.x - cc.y * rr.y), o.y - (cc.x * rr.y + cc.y * rr.x)};
                if (jk) v = {-(cc.x * pinv.x - cc.y * pinv.y), -(cc.x * pinv.y + cc.y * pinv.x)};
                if (ik) v = jk ? pinv : rr;
                A[r][c] = v;
            }
    }
    cd *M = reinterpret_cast<cd *>(a.Mc) + d.mat_off / 4;
#pragma unroll
    for (int r = 0; r < T; ++r)
#pragma unroll
        for (int c = 0; c < T; ++c) {
            const int i = i0 + r, j = j0 + c;
            if (i < nt && j < nt) M[i * nt + j] = {(double)A[r][c].x, (double)A[r][c].y};
        }
}

template <typename R>
__global__ void __launch_bounds__(256) precond_kernel(PrepArgs a)
{
    const int b = blockIdx.x;
    const ChannelDesc d = a.desc[b];
    const int nt = d.Nt;
    const double gamma = d.gamma_t / (d.dmin * d.dmin);   // gamma in the unscaled model
    using C2 = typename CT<R>::type;
    extern __shared__ double shd[];
    C2 *rowk = reinterpret_cast<C2 *>(shd);               // A_kj / p
    C2 *colk = rowk + nt;                                 // A_ik
    C2 *Am = a.stage_gj ? colk + nt : reinterpret_cast<C2 *>(a.gj) + d.mat_off / 2;
    const cd *G = reinterpret_cast<const cd *>(a.Gc) + d.mat_off / 4;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        const cd g = G[e];
        Am[e] = {(R)(g.x + (e / nt == e % nt ? gamma : 0.0)), (R)g.y};
    }
    __syncthreads();
    for (int k = 0; k < nt; ++k) {
        const C2 piv = Am[k * nt + k];
        if (threadIdx.x == 0 && !(piv.x > R(0))) set_status(a.status, kStatusNumeric);
        const R den = piv.x * piv.x + piv.y * piv.y;
        const C2 pinv = {piv.x / den, -piv.y / den};
        for (int j = threadIdx.x; j < nt; j += blockDim.x) {
            const C2 r = Am[k * nt + j];
            rowk[j] = {r.x * pinv.x - r.y * pinv.y, r.x * pinv.y + r.y * pinv.x};
            colk[j] = Am[j * nt + k];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
            const int i = e / nt, j = e % nt;
            C2 v;
            if (i == k) {
                v = j == k ? pinv : rowk[j];
            } else if (j == k) {
                const C2 c = colk[i];
                v = {-(c.x * pinv.x - c.y * pinv.y), -(c.x * pinv.y + c.y * pinv.x)};
            } else {
                const C2 c = colk[i], r = rowk[j], o = Am[e];
                v = {o.x - (c.x * r.x - c.y * r.y), o.y - (c.x * r.y + c.y * r.x)};
            }
            Am[e] = v;
        }
        __syncthreads();
    }
    cd *M = reinterpret_cast<cd *>(a.Mc) + d.mat_off / 4;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
        const C2 v = Am[e];
        M[e] = {(double)v.x, (double)v.y};
    }
}

// ------------------------------------------------------------------------------------------
// Emission of the scaled real-valued operands:
//   Gt = d^2 [[Re G, -Im G], [Im G, Re G]]   (FP64, N x N)
//   GMt = P~ Gt = real([(G + gamma I)^{-1} G]) = real(I - gamma M)   (preconditioned only)
//   zt = d [Re z; Im z],  wt = P~ zt = [Re(M z); Im(M z)] / d
//   Bt (N x NOp, the CUDA-core GEMM operand): row m = [Gt row m | GMt row m | 0 pad]
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) emit_kernel(PrepArgs a)
{
    const int b = blockIdx.x;
    const ChannelDesc d = a.desc[b];
    const int nt = d.Nt, N = d.N, NO = d.NO, NOp = d.NOp;
    const double d2 = d.dmin * d.dmin;
    const bool pre = NO > N;
    const double gamma = d.gamma_t / d2;
    const cd *__restrict__ G = reinterpret_cast<const cd *>(a.Gc) + d.mat_off / 4;
    const cd *__restrict__ M = reinterpret_cast<const cd *>(a.Mc) + d.mat_off / 4;
    const cd *__restrict__ z = reinterpret_cast<const cd *>(a.zc) + d.vec_off / 2;
    double *__restrict__ G64 = a.G64 + d.mat_off;
    double *__restrict__ GM = (pre && a.GM64) ? a.GM64 + d.mat_off : nullptr;
    double *__restrict__ bt64 = a.bt64 ? a.bt64 + d.bt_off : nullptr;
    float *__restrict__ bt32 = a.bt32 ? a.bt32 + d.bt_off : nullptr;
    // Every element (r, c) of the N x NOp operand [Gt | GMt | 0], one pass: consecutive threads
    // take consecutive elements, and (r, c) advance by (blockDim / NOp, blockDim % NOp) without
    // divisions. In the stacked embedding, entry (r, c) of Gt (or of GMt) takes the complex entry
    // (r mod nt, c mod nt) of G (or M): Re on the diagonal blocks, -Im above, +Im below.
    const int dr = blockDim.x / NOp, dc = blockDim.x % NOp;
    int r = threadIdx.x / NOp, c = threadIdx.x % NOp;
    for (int e = threadIdx.x; e < N * NOp; e += blockDim.x) {
        double v = 0.0;
        if (c < NO) {
            const bool gpart = c < N;
            const int cc = gpart ? c : c - N;
            const int ri = r < nt ? r : r - nt, ci = cc < nt ? cc : cc - nt;
            const bool rlo = r >= nt, clo = cc >= nt;
            const cd g = (gpart ? G : M)[ri * nt + ci];
            const double q = rlo == clo ? g.x : (clo ? -g.y : g.y);
            if (gpart) {
                v = d2 * q;
                G64[r * N + c] = v;
            } else {
                v = -gamma * q + (r == cc ? 1.0 : 0.0);   // real(I - gamma M)
                if (GM) GM[r * N + cc] = v;
            }
        }
        if (bt64) bt64[e] = v;
        else if (bt32) bt32[e] = (float)v;
        c += dc;
        r += dr;
        if (c >= NOp) {
            c -= NOp;
            ++r;
        }
    }
    // zt = d [Re z; Im z] and wt = [Re(M z); Im(M z)] / d (zero without the preconditioner); wt
    // in FP32 when M came from the FP32 factorisation (FP64 would add no accuracy there)
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
        const double zr = d.dmin * z[i].x, zi = d.dmin * z[i].y;
        double re = 0.0, im = 0.0;
        if (pre && a.precond_fp32) {
            float fr = 0.f, fi = 0.f;
            for (int j = 0; j < nt; ++j) {
                const cd m = M[i * nt + j], v = z[j];
                const float mr = (float)m.x, mi = (float)m.y, vr = (float)v.x, vi = (float)v.y;
                fr = fmaf(mr, vr, fmaf(-mi, vi, fr));
                fi = fmaf(mr, vi, fmaf(mi, vr, fi));
            }
            re = fr;
            im = fi;
        } else if (pre) {
            for (int j = 0; j < nt; ++j) {
                const cd p = cmul(M[i * nt + j], z[j]);
                re += p.x;
                im += p.y;
            }
        }
        const double wr = re / d.dmin, wi = im / d.dmin;
        a.z64[d.vec_off + i] = zr;
        a.z64[d.vec_off + nt + i] = zi;
        a.z32[d.vec_off + i] = (float)zr;
        a.z32[d.vec_off + nt + i] = (float)zi;
        a.w64[d.vec_off + i] = wr;
        a.w64[d.vec_off + nt + i] = wi;
        a.w32[d.vec_off + i] = (float)wr;
        a.w32[d.vec_off + nt + i] = (float)wi;
    }
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
// Host launchers
// ------------------------------------------------------------------------------------------
// Threads of the Gram kernel: its work items are the nb (nb + 1) / 2 upper-triangle 2 x 2 blocks
// (nb = ceil(Nt / 2)) of equal cost; pick the warp multiple in [128, 512] that wastes the fewest
// thread-slots over the rounds (ties to more threads). 256 when the batch's Nt is unknown.
int gram_threads(int max_nt)
{
    if (max_nt <= 0) return 256;
    const int nb = (max_nt + 1) / 2, nblk = nb * (nb + 1) / 2;
    int best = 256;
    double best_eff = -1.0;
    for (int t = 128; t <= 512; t += 32) {
        const int rounds = (nblk + t - 1) / t;
        const double eff = (double)nblk / ((double)rounds * t);
        if (eff >= best_eff) { best_eff = eff; best = t; }
    }
    return best;
}

cudaError_t launch_prep(const PrepArgs &a, int n_channels, size_t h_stage_bytes,
                        size_t gj_stage_bytes, bool preconditioned, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    cudaError_t e;
    if (h_stage_bytes > 48 * 1024) {
        if ((e = allow_max_dyn_smem(gram_kernel)) != cudaSuccess) return e;
    }
    gram_kernel<<<n_channels, gram_threads(a.max_nt), a.stage_h ? h_stage_bytes : 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (preconditioned) {
        auto k = a.precond_fp32 ? precond_kernel<float> : precond_kernel<double>;
        // FP32 batches of Nt <= 64: the matrix in registers (no dynamic shared memory)
        if (a.precond_fp32 && a.max_nt > 0 && a.max_nt <= 64) {
            k = a.max_nt <= 32 ? precond_regs_kernel<2> : precond_regs_kernel<4>;
            gj_stage_bytes = 0;
        }
        if (gj_stage_bytes > 48 * 1024) {
            if ((e = allow_max_dyn_smem(k)) != cudaSuccess) return e;
        }
        k<<<n_channels, 256, gj_stage_bytes, s>>>(a);
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

}  // namespace mcmcdet
