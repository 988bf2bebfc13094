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

// Round to nearest even by adding and removing 1.5 * 2^23 (exact for |x| < 2^22; beyond that the
// callers' clamp to [0, L-1] gives what rintf would).
__device__ __forceinline__ float round_even(float x)
{
    return __fadd_rn(__fadd_rn(x, 12582912.f), -12582912.f);
}

// Vertex level j* of the factor (a2, c2 in log2 units, k the current level, inv2c = 1/(2c2)).
template <int L>
__device__ __forceinline__ float vertex_level(float a2, float inv2c, float kf)
{
    float m = round_even(fmaf(a2, inv2c, kf));
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

// ------------------------------------------------------------------------------------------
// Two chains per instruction: the same arithmetic on packed FP32 pairs (sm_100+ f32x2 add / mul
// / fma, each lane rounded like its scalar counterpart), so a pair's results are bit-identical
// to two scalar evaluations. A pair lives in one 64-bit register (low word = first chain).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t f2_pack(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_splat(float a) { return f2_pack(a, a); }
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// Vertex levels and relative-logit polynomials of two factors (as vertex_level / rel_poly).
template <int L>
struct Poly2 {
    uint64_t B, C0;
};

template <int L>
__device__ __forceinline__ Poly2<L> rel_poly2(uint64_t a2, float c2, float inv2c, uint64_t kf)
{
    float v0, v1;
    f2_unpack(f2_fma(a2, f2_splat(inv2c), kf), v0, v1);
    float r0, r1;
    f2_unpack(f2_add(f2_add(f2_pack(v0, v1), f2_splat(12582912.f)), f2_splat(-12582912.f)), r0, r1);
    const float js0 = fminf(fmaxf(r0, 0.f), (float)(L - 1));
    const float js1 = fminf(fmaxf(r1, 0.f), (float)(L - 1));
    const uint64_t js = f2_pack(js0, js1);
    const uint64_t P = f2_fma(f2_splat(-c2), f2_fma(f2_splat(-2.f), kf, js), a2);
    return Poly2<L>{f2_fma(f2_splat(c2), js, P), f2_mul(f2_pack(-js0, -js1), P)};
}

template <int L>
__device__ __forceinline__ uint64_t rel_logit2_2(const Poly2<L> &p, uint64_t mc2, uint64_t jf)
{
    return f2_fma(f2_fma(mc2, jf, p.B), jf, p.C0);
}

// The proposal factor of two chains at their current levels, as Algorithm 1 carries it from one
// transition to the next: the cumulative weights S_j of each chain, the relative-logit
// polynomial and log2 of each total weight.
template <int L>
struct Table2 {
    float S0[L], S1[L];
    uint64_t B, C0, lgS;
};

template <int L>
__device__ __forceinline__ void factor_table_f2(uint64_t a2, float c2, float inv2c, uint64_t kf,
                                                Table2<L> &tb)
{
    const Poly2<L> p = rel_poly2<L>(a2, c2, inv2c, kf);
    const uint64_t mc2 = f2_splat(-c2);
    uint64_t acc = 0ull;   // (+0.f, +0.f)
#pragma unroll
    for (int j = 0; j < L; ++j) {
        float l0, l1;
        f2_unpack(rel_logit2_2(p, mc2, f2_splat((float)j)), l0, l1);
        acc = f2_add(acc, f2_pack(ex2_approx(l0), ex2_approx(l1)));
        f2_unpack(acc, tb.S0[j], tb.S1[j]);
    }
    tb.B = p.B;
    tb.C0 = p.C0;
    tb.lgS = f2_pack(lg2_approx(tb.S0[L - 1]), lg2_approx(tb.S1[L - 1]));
}

// Draw from a table with uniforms (u0, u1): the levels (as floats) and log2 q of them.
template <int L>
__device__ __forceinline__ void table_draw_f2(const Table2<L> &tb, float c2, float u0, float u1,
                                              uint64_t &sel, uint64_t &log2q)
{
    const float *S0 = tb.S0, *S1 = tb.S1;
    float t0, t1;
    f2_unpack(f2_mul(f2_pack(u0, u1), f2_pack(S0[L - 1], S1[L - 1])), t0, t1);
    float s0, s1;
    if constexpr (L == 2) {
        s0 = S0[0] <= t0 ? 1.f : 0.f;
        s1 = S1[0] <= t1 ? 1.f : 0.f;
    } else if constexpr (L == 4) {
        const bool a1 = S0[1] <= t0, b1 = S1[1] <= t1;
        const bool a0 = (a1 ? S0[2] : S0[0]) <= t0, b0 = (b1 ? S1[2] : S1[0]) <= t1;
        s0 = (a1 ? 2.f : 0.f) + (a0 ? 1.f : 0.f);
        s1 = (b1 ? 2.f : 0.f) + (b0 ? 1.f : 0.f);
    } else {
        const bool a2b = S0[3] <= t0, b2b = S1[3] <= t1;
        const bool a1 = (a2b ? S0[5] : S0[1]) <= t0, b1 = (b2b ? S1[5] : S1[1]) <= t1;
        const float ma = a2b ? (a1 ? S0[6] : S0[4]) : (a1 ? S0[2] : S0[0]);
        const float mb = b2b ? (b1 ? S1[6] : S1[4]) : (b1 ? S1[2] : S1[0]);
        const bool a0 = ma <= t0, b0 = mb <= t1;
        s0 = (a2b ? 4.f : 0.f) + (a1 ? 2.f : 0.f) + (a0 ? 1.f : 0.f);
        s1 = (b2b ? 4.f : 0.f) + (b1 ? 2.f : 0.f) + (b0 ? 1.f : 0.f);
    }
    sel = f2_pack(s0, s1);
    // log2 q = l2(sel) - log2 S_{L-1}, each lane rounded once as r - lg
    log2q = f2_fma(f2_splat(-1.f), tb.lgS, rel_logit2_2(Poly2<L>{tb.B, tb.C0}, f2_splat(-c2), sel));
}

// factor_draw for two chains: levels (as exact small floats) and log2 q of the drawn levels.
template <int L>
__device__ __forceinline__ void factor_draw_f2(uint64_t a2, float c2, float inv2c, uint64_t kf,
                                               float u0, float u1, uint64_t &sel, uint64_t &log2q)
{
    Table2<L> tb;
    factor_table_f2<L>(a2, c2, inv2c, kf, tb);
    table_draw_f2<L>(tb, c2, u0, u1, sel, log2q);
}

// factor_log2q for two chains: log2 q(j_eval | level k) of each (levels as floats).
template <int L>
__device__ __forceinline__ uint64_t factor_log2q_f2(uint64_t a2, float c2, float inv2c, uint64_t kf,
                                                    uint64_t jf)
{
    const Poly2<L> p = rel_poly2<L>(a2, c2, inv2c, kf);
    const uint64_t mc2 = f2_splat(-c2);
    uint64_t acc = 0ull;
#pragma unroll
    for (int j = 0; j < L; ++j) {
        float l0, l1;
        f2_unpack(rel_logit2_2(p, mc2, f2_splat((float)j)), l0, l1);
        acc = f2_add(acc, f2_pack(ex2_approx(l0), ex2_approx(l1)));
    }
    float S0, S1, r0, r1;
    f2_unpack(acc, S0, S1);
    f2_unpack(rel_logit2_2(p, mc2, jf), r0, r1);
    return f2_pack(r0 - lg2_approx(S0), r1 - lg2_approx(S1));
}

}  // namespace mcmcdet
