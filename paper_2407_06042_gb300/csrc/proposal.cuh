// proposal.cuh -- FP32 arithmetic of one proposal factor q_n(. | x_n) (Eqs. (15)-(17), or (21)
// with Remark 1's preconditioner), shared by the CUDA-core FP32 kernel and the tensor-core
// (MIXED) kernel so that the two differ only in how the Gram products are formed.
//
// In level units the logits are  l(j) = a (j - k) - c (j - k)^2,  j = 0..L-1,  k the current
// level. The kernels work in log2 units (a2 = a log2 e, c2 = c log2 e) so that every weight is
// one ex2. The largest logit sits at the level nearest the vertex of the parabola,
//     j* = clamp(rint(k + a / (2c)), 0, L - 1),
// and every weight is taken relative to it:
//     w_j = 2^(l2(j) - l2(j*)),  l2(j) - l2(j*) = (j - j*) (a2 - c2 (j + j* - 2k)),
// which is <= 0 (no overflow) with w_{j*} = 1 (the total never underflows). The cumulative
// weights S_j are summed in ascending level order, and a draw with uniform u takes the smallest
// j with u S_{L-1} < S_j (binary search over the S_j).
#pragma once

#include "common.cuh"

namespace mcmcdet {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float lg2_approx(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Vertex level j* of the factor (a2, c2 in log2 units, k the current level, inv2c = 1/(2c2)).
template <int L>
__device__ __forceinline__ float vertex_level(float a2, float inv2c, float kf)
{
    float m = rintf(fmaf(a2, inv2c, kf));
    m = fminf(fmaxf(m, 0.f), (float)(L - 1));
    return m;
}

// The relative logit as a polynomial in j: l2(j) - l2(j*) = (j - j*) (P - c2 j)
// = (-c2 j + B) j + C0 with P = a2 - c2 (j* - 2k), B = P + c2 j*, C0 = -j* P, evaluated by Horner
// (two FMAs per level for compile-time j).
struct Poly {
    float B, C0;
};

__device__ __forceinline__ Poly rel_poly(float a2, float c2, float js, float kf)
{
    const float P = fmaf(-c2, js - 2.f * kf, a2);
    return Poly{fmaf(c2, js, P), -js * P};
}

__device__ __forceinline__ float rel_logit2(const Poly &p, float c2, float jf)
{
    return fmaf(fmaf(-c2, jf, p.B), jf, p.C0);
}

// Cumulative weights S_j (levels ascending) of the factor and the vertex polynomial.
template <int L>
__device__ __forceinline__ Poly factor_cumulative(float a2, float c2, float inv2c, float kf,
                                                  float (&S)[L])
{
    const float js = vertex_level<L>(a2, inv2c, kf);
    const Poly p = rel_poly(a2, c2, js, kf);
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        acc += ex2_approx(rel_logit2(p, c2, (float)j));
        S[j] = acc;
    }
    return p;
}

// Smallest j with target < S_j (S nondecreasing, target < S_{L-1} in exact arithmetic): a binary
// search over the cumulative weights, log2 L compares.
template <int L>
__device__ __forceinline__ int cdf_search(const float (&S)[L], float target)
{
    if constexpr (L == 2) {
        return S[0] <= target ? 1 : 0;
    } else if constexpr (L == 4) {
        const bool b1 = S[1] <= target;
        const float m = b1 ? S[2] : S[0];
        const bool b0 = m <= target;
        return (b1 ? 2 : 0) + (b0 ? 1 : 0);
    } else {
        const bool b2 = S[3] <= target;
        const bool b1 = (b2 ? S[5] : S[1]) <= target;
        const float m = b2 ? (b1 ? S[6] : S[4]) : (b1 ? S[2] : S[0]);
        const bool b0 = m <= target;
        return (b2 ? 4 : 0) + (b1 ? 2 : 0) + (b0 ? 1 : 0);
    }
}

// Draw from the factor with uniform u; returns the level and log2 q of it.
template <int L>
__device__ __forceinline__ int factor_draw(float a2, float c2, float inv2c, int k, float u,
                                           float &log2q)
{
    float S[L];
    const float kf = (float)k;
    const Poly p = factor_cumulative<L>(a2, c2, inv2c, kf, S);
    const int sel = cdf_search<L>(S, u * S[L - 1]);
    log2q = rel_logit2(p, c2, (float)sel) - lg2_approx(S[L - 1]);
    return sel;
}

// log2 q(j_eval | level k) of the factor (a2 at level k).
template <int L>
__device__ __forceinline__ float factor_log2q(float a2, float c2, float inv2c, int k, int j_eval)
{
    float S[L];
    const float kf = (float)k;
    const Poly p = factor_cumulative<L>(a2, c2, inv2c, kf, S);
    return rel_logit2(p, c2, (float)j_eval) - lg2_approx(S[L - 1]);
}

// Float-level forms (levels held as exact small floats, no integer conversions): draw returns the
// level as a float.
template <int L>
__device__ __forceinline__ float factor_draw_f(float a2, float c2, float inv2c, float kf, float u,
                                               float &log2q)
{
    float S[L];
    const Poly p = factor_cumulative<L>(a2, c2, inv2c, kf, S);
    const float target = u * S[L - 1];
    float sel;
    if constexpr (L == 2) {
        sel = S[0] <= target ? 1.f : 0.f;
    } else if constexpr (L == 4) {
        const bool b1 = S[1] <= target;
        const bool b0 = (b1 ? S[2] : S[0]) <= target;
        sel = (b1 ? 2.f : 0.f) + (b0 ? 1.f : 0.f);
    } else {
        const bool b2 = S[3] <= target;
        const bool b1 = (b2 ? S[5] : S[1]) <= target;
        const float m = b2 ? (b1 ? S[6] : S[4]) : (b1 ? S[2] : S[0]);
        const bool b0 = m <= target;
        sel = (b2 ? 4.f : 0.f) + (b1 ? 2.f : 0.f) + (b0 ? 1.f : 0.f);
    }
    log2q = rel_logit2(p, c2, sel) - lg2_approx(S[L - 1]);
    return sel;
}

template <int L>
__device__ __forceinline__ float factor_log2q_f(float a2, float c2, float inv2c, float kf,
                                                float jf)
{
    float S[L];
    const Poly p = factor_cumulative<L>(a2, c2, inv2c, kf, S);
    return rel_logit2(p, c2, jf) - lg2_approx(S[L - 1]);
}

}  // namespace mcmcdet
