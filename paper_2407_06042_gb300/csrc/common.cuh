// common.cuh -- shared device definitions of the DMALA detector kernels (sm_103a).
//
// Scaled units used by every kernel: with d = d_min, the state x = d * xt where xt = 2k - (L-1)
// is an odd integer (k the PAM level index), Gt = d^2 H^T H (real-valued, stacked, N x N),
// zt = d H^T y. Then (Sec. II-A, Eq. (3))
//     f(x) = -(||y||^2 - 2 xt^T zt + xt^T Gt xt) / sigma^2,
// and the tempered energy difference of a move x -> x' (Algorithm 2 with Eq. (18)) is
//     df_tau = (1 / (tau sigma^2)) sum_n (xt'_n - xt_n)(2 zt_n - (Gt xt)_n - (Gt xt')_n),
// which needs only the cached Gt xt of both states (no ||y||^2 cancellation).
// The proposal factor of dimension n (Eq. (16), or Eq. (21) with Remark 1's preconditioner) is,
// in level units j (target level) and k (current level),
//     logit(j) = a_n (j - k) - c_quad (j - k)^2,   a_n = c_lin g_n,
// with g = P~ (zt - Gt xt): P~ = I for the plain proposal (c_lin = 2 / (tau sigma^2),
// c_quad = 2 d^2 / alpha), P~ = (Gt + gamma d^2 I)^{-1} for the preconditioned one
// (c_lin = 2 d^2 / (beta tau sigma^2), c_quad = 2 d^2 / (alpha beta)). For the preconditioned
// drift the kernels use g = wt - (P~ Gt) xt with wt = P~ zt, so one GEMM against [Gt | P~ Gt]
// yields both the energy terms and the drift.
#pragma once

#include <cstdint>
#include <mutex>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

namespace mcmcdet {

constexpr int kMaxN = 256;     // real unknowns per channel (Nt <= 128)
constexpr int kMaxL = 8;       // PAM levels per real dimension (64-QAM)

// Lets kernel `func` take up to the device's opt-in maximum of dynamic shared memory, less its
// static shared memory (each launch then asks for what it needs). Every launch site sets this
// same value, so handles used from different host threads cannot lower the limit between another
// thread's setting and its launch. The attribute is set once per kernel and device (a table of
// the (kernel, device) pairs done, shared by every kernel); later calls only look it up.
inline bool dyn_smem_done(const void *func, int dev, bool mark)
{
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto &e : done)
        if (e.first == func && e.second == dev) return true;
    if (mark) done.emplace_back(func, dev);
    return false;
}

template <typename F>
inline cudaError_t allow_max_dyn_smem(F *func)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const void *key = reinterpret_cast<const void *>(func);
    if (dyn_smem_done(key, dev, false)) return cudaSuccess;
    int mx = 0;
    cudaFuncAttributes fa{};
    e = cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, func);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 mx - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess) dyn_smem_done(key, dev, true);
    return e;
}

// Per-channel description, built on the host at preprocess time.
struct ChannelDesc {
    int N;             // real unknowns 2 Nt
    int L;             // PAM levels
    int log2L;
    int Nt;
    int Nr;
    int NO;            // GEMM outputs per chain: N (plain) or 2N (preconditioned)
    int NOp;           // NO rounded up to a multiple of 8
    int pad0;
    long long state_off;   // int8 offset of chain 0's state: Np * sum_{b'<b} N_b'
    long long mat_off;     // offset of this channel's N x N matrices (elements)
    long long bt_off;      // offset of this channel's N x NOp GEMM operand (elements)
    long long tc_off;      // offset of this channel's tcgen05 operand block (bytes)
    long long vec_off;     // offset of this channel's N-vectors
    long long bit_off;     // offset of this channel's LLRs
    long long ant_off;     // offset of this channel's antennas (best_idx)
    long long h_off;       // input offset of H (complex elements)
    long long y_off;       // input offset of y (complex elements)
    double sigma2;
    double dmin;
    double cf;         // 1 / (tau sigma^2)
    double clin;       // logit slope per drift unit (level units)
    double cquad;      // logit curvature (level units)
    double inv_s2;     // 1 / sigma^2
    double gamma_t;    // gamma d^2 (preconditioner damping in scaled units)
    double tau;
};

// Device status word bits (OR-ed by kernels, read by the host at synchronising calls).
constexpr unsigned kStatusNumeric = 1u;
constexpr unsigned kStatusTimeout = 2u;
constexpr unsigned kStatusBadState = 4u;

// ------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32->64-bit products
// with a Weyl-sequence key schedule.
// ------------------------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit product per multiplier (low and high words together)
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;
        const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

// The same generator with the ten round keys (k0 + r W0, k1 + r W1) precomputed on the host and
// read from the kernel's parameters, so that each round's key is an immediate operand of its XOR.
constexpr int kPhiloxRounds = 10;

__host__ __device__ inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t (&rk)[2 * kPhiloxRounds])
{
    for (int r = 0; r < kPhiloxRounds; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

__device__ __forceinline__ U4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const uint32_t (&rk)[2 * kPhiloxRounds])
{
#pragma unroll
    for (int r = 0; r < kPhiloxRounds; ++r) {
        const uint64_t p0 = (uint64_t)c0 * 0xD2511F53u;
        const uint64_t p1 = (uint64_t)c2 * 0xCD9E8D57u;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ rk[2 * r];
        const uint32_t n2 = hi0 ^ c3 ^ rk[2 * r + 1];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ uint32_t word_of(const U4 &v, int i)
{
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Uniform in (0,1): (2 (w >> 9) + 1) * 2^-24, exactly representable in FP32 and FP64. In FP32
// it is formed without a conversion: 1 + m 2^-23 (m = w >> 9 in the mantissa of 1.0f) minus
// (1 - 2^-24) is exact (Sterbenz) and equals (2m + 1) 2^-24.
__device__ __forceinline__ float uniform_f(uint32_t w)
{
    return __fsub_rn(__uint_as_float(0x3F800000u | (w >> 9)), 0.99999994039535522f);
}
__device__ __forceinline__ double uniform_d(uint32_t w)
{
    return (double)(2u * (w >> 9) + 1u) * 5.9604644775390625e-8;
}

constexpr uint32_t kMhStream = 0xFFFFFFFFu;   // counter word 1 of the acceptance uniforms

// Level index -> odd integer 2k - (L-1).
__device__ __forceinline__ int odd_of(int k, int L) { return 2 * k - (L - 1); }

__device__ __forceinline__ int gray_of(int k) { return k ^ (k >> 1); }
__device__ __forceinline__ int level_of_gray(int g) { int k = g; k ^= k >> 1; k ^= k >> 2; return k; }

__device__ __forceinline__ void set_status(unsigned *status, unsigned bit)
{
    atomicOr(status, bit);
}

// round(g 2^sh) for |g 2^sh| < 2^62, from the bits of g (integer operations only: this GPU's FP64
// pipe runs at a small fraction of its integer and FP32 rates). Ties round away from zero.
__device__ __forceinline__ long long fixed_of(double g, int sh)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(g);
    const int ex = (int)((b >> 52) & 0x7FFull);
    if (ex == 0) return 0;                                  // zero or subnormal
    const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
    const int p = ex - 1075 + sh;                           // g 2^sh = mant 2^p
    long long v;
    if (p >= 0) v = p < 10 ? mant << p : 0;                 // p > 0 is outside the contract
    else if (p > -64) v = (mant + (1ll << (-p - 1))) >> (-p);
    else v = 0;
    return (b >> 63) ? -v : v;
}

// FP64 x^T G x and x^T z for one state (G symmetric N x N), one share of the work: the row pairs
// (r, N - 1 - r) for r = first, first + stride, ..., each row contributing
// x_n (G_nn x_n + 2 sum_{m>n} G_nm x_m), so every pair costs N - 1 products (half of the full N^2
// over all pairs). level(n) returns the odd-integer value of dimension n. The caller sums quad
// and lin over the shares.
template <typename Level>
__device__ __forceinline__ void quad_lin_fp64_part(const double *G, const double *z, int N, int first,
                                                   int stride, Level level, double &quad, double &lin)
{
    quad = 0.0;
    lin = 0.0;
    for (int r = first; r < (N + 1) / 2; r += stride) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int n = h ? N - 1 - r : r;
            if (h && n == r) break;
            const double xn = level(n);
            const double *g = G + (long long)n * N;
            double s = 0.0;
            for (int m = n + 1; m < N; ++m) s = fma(g[m], level(m), s);
            quad = fma(xn, fma(2.0, s, g[n] * xn), quad);
            lin = fma(xn, z[n], lin);
        }
    }
}
// A lane's share of a warp's work (row pairs r = lane, lane + 32, ...).
template <typename Level>
__device__ __forceinline__ void quad_lin_fp64(const double *G, const double *z, int N, int lane,
                                              Level level, double &quad, double &lin)
{
    quad_lin_fp64_part(G, z, N, lane, 32, level, quad, lin);
}

}  // namespace mcmcdet
