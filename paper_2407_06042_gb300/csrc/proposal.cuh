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
// j with u S_{L-1} < S_j (the count of j < L-1 with S_j <= u S_{L-1}).
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

// Weights of every level and their total; returns j* (as float).
template <int L>
__device__ __forceinline__ float factor_weights(float a2, float c2, float inv2c, float kf,
                                                float (&w)[L], float &total)
{
    const float js = vertex_level<L>(a2, inv2c, kf);
    const float P = fmaf(-c2, js - 2.f * kf, a2);   // a2 - c2 (j* - 2k)
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        const float dj = (float)j - js;
        const float e = dj * fmaf(-c2, (float)j, P);
        w[j] = ex2_approx(e);
        acc += w[j];
    }
    total = acc;
    return js;
}

// log2 of the unnormalised weight of level j relative to the vertex (same formula as above).
__device__ __forceinline__ float rel_logit2(float a2, float c2, float js, float kf, float jf)
{
    const float P = fmaf(-c2, js - 2.f * kf, a2);
    return (jf - js) * fmaf(-c2, jf, P);
}

// Draw from the factor with uniform u; returns the level and log2 q of it.
template <int L>
__device__ __forceinline__ int factor_draw(float a2, float c2, float inv2c, int k, float u,
                                           float &log2q)
{
    float w[L], total;
    const float kf = (float)k;
    const float js = factor_weights<L>(a2, c2, inv2c, kf, w, total);
    const float target = u * total;
    float S = 0.f;
    int sel = 0;
#pragma unroll
    for (int j = 0; j < L - 1; ++j) {
        S += w[j];
        sel += (S <= target) ? 1 : 0;
    }
    log2q = rel_logit2(a2, c2, js, kf, (float)sel) - lg2_approx(total);
    return sel;
}

// log2 q(j_eval | level k) of the factor (a2 at level k).
template <int L>
__device__ __forceinline__ float factor_log2q(float a2, float c2, float inv2c, int k, int j_eval)
{
    float w[L], total;
    const float kf = (float)k;
    const float js = factor_weights<L>(a2, c2, inv2c, kf, w, total);
    return rel_logit2(a2, c2, js, kf, (float)j_eval) - lg2_approx(total);
}

}  // namespace mcmcdet
