// refresh.cu -- energies of the current chain states, f(x) = -||y - Hx||^2 / sigma^2 (Eq. (3)),
// evaluated exactly enough to stand for the FP64 value:
//     f = -(||y||^2 - 2 xt^T zt + xt^T Gt xt) / sigma^2
// in the scaled units of common.cuh (xt odd integers, Gt = d^2 H^T H, zt = d H^T y).
//
// The quadratic form is the expensive part (N^2 per state) and this GPU's FP64 pipe runs at a
// small fraction of its integer rate, so it is summed in integers. Gt is rounded to the fixed
// point 2^-sh with sh = 53 - exponent(max_n Gt_nn): Gt is positive semidefinite, so every
// |Gt_nm| <= max_n Gt_nn and |Gt_nm 2^sh| < 2^53. The integer Gt_nm 2^sh is split into seven
// balanced int8 digits, Gt_nm 2^sh = sum_k 256^k d_k,nm (k = 0..6), and
//     Q_k = sum_n xt_n sum_m d_k,nm xt_m
// is an exact int32 sum of DP4A products (|Q_k| < 7 * N * 128 * 7 * N < 2^31 for N <= 256).
// One FP64 Horner pass gives xt^T Gt xt = 2^-sh sum_k 256^k Q_k. Each entry of Gt is off by at
// most half a unit of 2^-sh <= 2^-52 max Gt_nn, so the quadratic form is off by at most
// 2^-53 max Gt_nn (sum_n |xt_n|)^2, comparable to the rounding of an FP64 sum. The linear term
// xt^T zt is formed the same way: zt at the fixed point 2^-sz, sz = 53 - exponent(max_m |zt_m|),
// in seven int8 digits, exact DP4A sums, one Horner pass (off by at most
// 2^-53 max_m |zt_m| sum_m |xt_m|).
//
// One CTA per (channel, block of chains): the channel's digits are generated 32 rows at a time
// into shared memory; each warp takes four chains at a time and each lane one row of the block,
// so every digit word loaded serves four chains' DP4A products. Gt is symmetric, so a block of
// rows needs only its own 32 x 32 diagonal block (each ordered pair once) and the columns to its
// right (counted twice, for the mirrored pairs below the diagonal): about (N + 32) / 2N of the
// digits and products of the full form, with the same integer sums.
#include "common.cuh"
#include "kernels.h"

namespace mcmcdet {

namespace {

constexpr int kRefreshThreads = 256;
constexpr int kRowBlock = 32;     // rows of Gt whose digits are held at once (one per lane)
constexpr int kDigits = 7;

// Chains per CTA: the states of a block of chains are held as int8 words in shared memory.
__host__ __device__ inline int refresh_chains_per_cta(int chains, int N)
{
    const int cap = (32768 / ((N + 3) / 4 * 4)) / 4 * 4;
    return chains < cap ? chains : (cap < 4 ? 4 : cap);
}

// Row stride (words) of a digit plane: odd, so that the 32 lanes reading one column word of 32
// different rows hit 32 different banks.
__host__ __device__ inline int refresh_row_stride(int N) { return ((N + 3) / 4) | 1; }

__host__ __device__ inline size_t refresh_smem_bytes(int chains, int N)
{
    const int cpb = refresh_chains_per_cta(chains, N);
    const int nw = (N + 3) / 4;
    return (size_t)cpb * nw * 4                                   // states (odd integers, int8)
           + (size_t)kDigits * kRowBlock * refresh_row_stride(N) * 4   // digit planes of one block
           + (size_t)cpb * kDigits * 4                            // Q_k per chain
           + (size_t)kDigits * nw * 4                             // digit planes of zt
           + 16;                                                  // shifts, flags
}

__global__ void __launch_bounds__(kRefreshThreads) refresh_kernel(RefreshArgs a, int cpb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int blocks_per_channel = (a.chains + cpb - 1) / cpb;
    const int b = blockIdx.x / blocks_per_channel;
    const int c0 = (blockIdx.x % blocks_per_channel) * cpb;
    const int nc = min(cpb, a.chains - c0);
    const ChannelDesc d = a.desc[b];
    const int N = d.N, L = d.L, nw = (N + 3) / 4, rs = refresh_row_stride(N);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    uint32_t *sX = reinterpret_cast<uint32_t *>(smem);                       // [cpb][nw]
    uint32_t *sD = sX + (size_t)cpb * nw;                                    // [7][32][rs]
    int *sQ = reinterpret_cast<int *>(sD + (size_t)kDigits * kRowBlock * rs);  // [cpb][7]
    uint32_t *sZ = reinterpret_cast<uint32_t *>(sQ + (size_t)cpb * kDigits); // [7][nw]
    int *sflag = reinterpret_cast<int *>(sZ + (size_t)kDigits * nw);        // [0] shift, [1] bad,
                                                                             // [2] shift of zt
    const double *G = a.G64 + d.mat_off;
    const double *z = a.z64 + d.vec_off;
    const int8_t *states = a.states + d.state_off + (long long)c0 * N;

    // states as odd integers, packed four per word (padding dimensions hold 0)
    bool bad = false;
    for (int e = tid; e < cpb * nw; e += blockDim.x) {
        const int c = e / nw, w = e - c * nw;
        uint32_t word = 0;
        if (c < nc) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = 4 * w + j;
                if (m < N) {
                    const int k = states[(long long)c * N + m];
                    bad |= (k < 0 || k >= L);
                    word |= (uint32_t)(odd_of(k, L) & 255) << (8 * j);
                }
            }
        }
        sX[e] = word;
    }
    for (int e = tid; e < cpb * kDigits; e += blockDim.x) sQ[e] = 0;
    if (warp == 0) {
        double mx = 0.0;
        for (int n = lane; n < N; n += 32) mx = fmax(mx, G[(long long)n * N + n]);
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int ex = 0;
            frexp(mx, &ex);
            sflag[0] = 53 - ex;               // |Gt_nm| 2^sh < 2^53
            sflag[1] = 0;
        }
    } else if (warp == 1) {
        double mx = 0.0;
        for (int n = lane; n < N; n += 32) mx = fmax(mx, fabs(z[n]));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            int ex = 0;
            frexp(mx, &ex);
            sflag[2] = 53 - ex;               // |zt_m| 2^sz < 2^53
        }
    }
    __syncthreads();
    if (bad) atomicOr(&sflag[1], 1);
    const int sh = sflag[0], sz = sflag[2];
    // zt at the fixed point 2^-sz in seven balanced int8 digits, four values per word (the
    // linear term x^T zt then is an exact int32 sum per digit, like the quadratic form)
    for (int w = tid; w < nw; w += blockDim.x) {
        uint32_t dw[kDigits] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = 4 * w + j;
            long long v = m < N ? fixed_of(z[m], sz) : 0;
#pragma unroll
            for (int k = 0; k < kDigits; ++k) {
                const int lo = (int)(v & 255), dk = lo >= 128 ? lo - 256 : lo;
                v = (v - dk) >> 8;
                dw[k] |= (uint32_t)(dk & 255) << (8 * j);
            }
        }
#pragma unroll
        for (int k = 0; k < kDigits; ++k) sZ[k * nw + w] = dw[k];
    }

    for (int r0 = 0; r0 < N; r0 += kRowBlock) {
        // digit planes of rows r0 .. r0 + 31, columns r0 .. N - 1 (word w0 onwards)
        const int w0 = r0 / 4, nwb = nw - w0, wd = min(nwb, kRowBlock / 4);
        for (int u = tid; u < kRowBlock * nwb; u += blockDim.x) {
            const int i = u / nwb, wr = u - i * nwb, w = w0 + wr, n = r0 + i;
            uint32_t dw[kDigits] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
            if (n < N) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = 4 * w + j;
                    long long v = m < N ? fixed_of(G[(long long)n * N + m], sh) : 0;
#pragma unroll
                    for (int k = 0; k < kDigits; ++k) {
                        const int lo = (int)(v & 255), dk = lo >= 128 ? lo - 256 : lo;
                        v = (v - dk) >> 8;
                        dw[k] |= (uint32_t)(dk & 255) << (8 * j);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kDigits; ++k) sD[(k * kRowBlock + i) * rs + wr] = dw[k];
        }
        __syncthreads();
        // lane = row r0 + lane; a warp takes four chains at a time
        const int n = r0 + lane;
        for (int cq = warp; 4 * cq < nc; cq += nwarps) {
            int t[4][kDigits];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int k = 0; k < kDigits; ++k) t[j][k] = 0;
            const uint32_t *x0 = sX + (size_t)(4 * cq) * nw;
            // the diagonal block's words once, the words to its right with x doubled (each byte
            // 2 x, |2 x| <= 14: the shift's carries into the next byte are masked off)
            for (int wr = 0; wr < nwb; ++wr) {
                uint32_t dv[kDigits];
#pragma unroll
                for (int k = 0; k < kDigits; ++k) dv[k] = sD[(k * kRowBlock + lane) * rs + wr];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t xw = x0[(size_t)j * nw + w0 + wr];   // rows past nc hold zeros
                    const int xs = (int)(wr < wd ? xw : (xw << 1) & 0xFEFEFEFEu);
#pragma unroll
                    for (int k = 0; k < kDigits; ++k) t[j][k] = __dp4a((int)dv[k], xs, t[j][k]);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * cq + j;
                int xn = 0;
                if (n < N && c < nc) {
                    const uint32_t word = x0[(size_t)j * nw + (n >> 2)];
                    xn = (int)(int8_t)((word >> (8 * (n & 3))) & 255u);
                }
#pragma unroll
                for (int k = 0; k < kDigits; ++k) {
                    const int v = __reduce_add_sync(0xffffffffu, xn * t[j][k]);
                    if (lane == 0 && c < nc) sQ[c * kDigits + k] += v;   // exact in any order
                }
            }
        }
        __syncthreads();
    }

    // f per chain: the integer sums recombined once in FP64, the linear term in FP64; the
    // largest corrections (non-negative doubles, ordered as their bit patterns) per warp
    unsigned long long mdr = 0ull, mdr_rel = 0ull;
    for (int c = tid; c < nc; c += blockDim.x) {
        double q = 0.0;
#pragma unroll
        for (int k = kDigits - 1; k >= 0; --k) q = fma(q, 256.0, (double)sQ[c * kDigits + k]);
        q = ldexp(q, -sh);
        int lk[kDigits] = {0, 0, 0, 0, 0, 0, 0};
        const uint32_t *xc = sX + (size_t)c * nw;
        for (int w = 0; w < nw; ++w) {
            const int xw = (int)xc[w];
#pragma unroll
            for (int k = 0; k < kDigits; ++k) lk[k] = __dp4a((int)sZ[k * nw + w], xw, lk[k]);
        }
        double l = 0.0;
#pragma unroll
        for (int k = kDigits - 1; k >= 0; --k) l = fma(l, 256.0, (double)lk[k]);
        l = ldexp(l, -sz);
        const double f = -(a.yy[b] - 2.0 * l + q) * d.inv_s2;
        if (!isfinite(f)) set_status(a.status, kStatusNumeric);
        const long long ci = (long long)b * a.chains + c0 + c;
        if (a.drift_bits) {
            const double dr = fabs(a.f[ci] - f);
            mdr = max(mdr, (unsigned long long)__double_as_longlong(dr));
            mdr_rel = max(mdr_rel, (unsigned long long)__double_as_longlong(dr / fmax(fabs(f), 1e-300)));
        }
        a.f[ci] = f;
        if (a.reset_best) a.best_f[ci] = f;
    }
    if (a.drift_bits) {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            mdr = max(mdr, __shfl_xor_sync(0xffffffffu, mdr, o));
            mdr_rel = max(mdr_rel, __shfl_xor_sync(0xffffffffu, mdr_rel, o));
        }
        if (lane == 0 && mdr) atomicMax(a.drift_bits, mdr);
        if (lane == 0 && mdr_rel && a.drift_rel_bits) atomicMax(a.drift_rel_bits, mdr_rel);
    }
    if (sflag[1]) {
        if (tid == 0) set_status(a.status, kStatusBadState);
    }
    if (a.reset_best) {
        int8_t *bk = a.best_states + d.state_off + (long long)c0 * N;
        for (long long e = tid; e < (long long)nc * N; e += blockDim.x) bk[e] = states[e];
    }
}

}  // namespace

cudaError_t launch_refresh(const RefreshArgs &a, cudaStream_t s)
{
    if (a.n_channels <= 0 || a.chains <= 0) return cudaSuccess;
    // the largest channel of the batch sets the launch shape
    const int maxn = a.max_n > 0 && a.max_n <= kMaxN ? a.max_n : kMaxN;
    const int cpb = refresh_chains_per_cta(a.chains, maxn);
    const size_t smem = refresh_smem_bytes(a.chains, maxn);
    cudaError_t e = allow_max_dyn_smem(refresh_kernel);
    if (e != cudaSuccess) return e;
    const long long grid = (long long)a.n_channels * ((a.chains + cpb - 1) / cpb);
    refresh_kernel<<<(unsigned)grid, kRefreshThreads, smem, s>>>(a, cpb);
    return cudaGetLastError();
}

}  // namespace mcmcdet
