// mlp.cu -- the learned proposal's network: FP32 CUDA-core training and inference kernels, a
// tcgen05 inference kernel, and the mcmc_mlp_* entry points of include/mcmcdet_learned.h.
//
// Network (no counterpart in the paper): 6 -> 256 (ReLU) -> 256 (ReLU) -> Qc logits, softmax
// cross-entropy, Adam. Every reduction has a fixed order (split-K partials summed by a second
// kernel, column sums by fixed row groups), so training is deterministic.
//
// Tensor-core inference (one CTA of 256 threads per SM, persistent over 128-row tiles; two
// threads per row, each taking half of the hidden units and logits):
//   1. each thread computes its half of its row's first layer on the CUDA cores (K = 6) and
//      stores the BF16 activations into the A operand (K-major core matrices, 128 x 256);
//   2. one thread issues 16 MMAs (M = 128, N = 256, K = 16) against W2 (BF16, staged once per
//      CTA by a bulk copy) into tensor memory columns 0..255;
//   3. each warp reads its 32 lanes back (tcgen05.ld; warps w and w + 4 share lane quadrant
//      w % 4 and split the columns), adds b2, applies ReLU, rounds to BF16 and overwrites the A
//      operand with the second hidden layer;
//   4. 16 MMAs against W3 (N = Qc padded to 16) into columns 256.., then bias and store.
// Every mbarrier wait is bounded; one that runs out sets the timeout status bit and the CTA
// frees its tensor memory and returns.
#include "../../include/mcmcdet_learned.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_bf16.h>

#include "common.cuh"
#include "mlp.h"
#include "tc_ptx.cuh"
#include "tcgemm.h"

namespace mcmcdet {

namespace {

// ------------------------------------------------------------------------------------------
// FP32 GEMM with generic strides: C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak],
// B(k, n) = B[k sbk + n sbn]; epilogue + bias(n), ReLU, or times [mask(m, n) > 0]. With
// `partial` set, each blockIdx.z sums its K range into partial[z][m][n] (no epilogue).
// ------------------------------------------------------------------------------------------
struct GemmArgs {
    int M, N, K;
    const float *A;
    long long sam, sak;
    const float *B;
    long long sbk, sbn;
    float *C;
    long long ldc;
    const float *bias;
    const float *mask;
    long long ldm;
    int relu;
    int kchunk;
    float *partial;
};

constexpr int kBM = 64, kBN = 64, kBK = 16;

__global__ void __launch_bounds__(256) sgemm_kernel(GemmArgs g)
{
    __shared__ float As[kBK][kBM + 4];
    __shared__ __align__(16) float Bs[kBK][kBN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * g.kchunk;
    const int ke = min(g.K, kb + g.kchunk);
    const bool a_kfast = g.sak == 1, b_nfast = g.sbn == 1;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = kb; k0 < ke; k0 += kBK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + 256 * i;
            int mm, ka, nn, kq;
            if (a_kfast) { ka = e & 15; mm = e >> 4; } else { mm = e & 63; ka = e >> 6; }
            if (b_nfast) { nn = e & 63; kq = e >> 6; } else { kq = e & 15; nn = e >> 4; }
            const int gm = m0 + mm, gka = k0 + ka, gn = n0 + nn, gkb = k0 + kq;
            As[ka][mm] = (gm < g.M && gka < ke) ? g.A[(long long)gm * g.sam + (long long)gka * g.sak] : 0.f;
            Bs[kq][nn] = (gn < g.N && gkb < ke) ? g.B[(long long)gkb * g.sbk + (long long)gn * g.sbn] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                acc[i][0] = fmaf(a[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(a[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(a[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(a[i], b.w, acc[i][3]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if (g.partial) {
                g.partial[((long long)blockIdx.z * g.M + m) * g.N + n] = v;
                continue;
            }
            if (g.bias) v += g.bias[n];
            if (g.relu) v = fmaxf(v, 0.f);
            if (g.mask && !(g.mask[(long long)m * g.ldm + n] > 0.f)) v = 0.f;
            g.C[(long long)m * g.ldc + n] = v;
        }
    }
}

// Sum of the split-K partials in split order.
__global__ void splitk_reduce_kernel(const float *partial, int splits, int M, int N, float *C,
                                     long long ldc)
{
    const long long MN = (long long)M * N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
         e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += partial[z * MN + e];
        C[(e / N) * ldc + (e % N)] = s;
    }
}

// Column sums out[n] = sum_r A[r lda + n] in two deterministic stages: CTA (x, y) sums rows
// [y rpc, (y + 1) rpc) of columns 32x .. 32x + 31 into part[y N + n] (eight row groups of 32
// lanes, added in group order), then colsum_final_kernel adds the chunks in a fixed order.
__global__ void colsum_kernel(const float *A, int R, int N, long long lda, int rpc, float *part)
{
    __shared__ float red[8][33];
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int r0 = blockIdx.y * rpc, r1 = min(R, r0 + rpc);
    float s0 = 0.f, s1 = 0.f;
    if (col < N) {
        int r = r0 + grp;
        for (; r + 8 < r1; r += 16) {
            s0 += A[(long long)r * lda + col];
            s1 += A[(long long)(r + 8) * lda + col];
        }
        if (r < r1) s0 += A[(long long)r * lda + col];
    }
    red[grp][lane] = s0 + s1;
    __syncthreads();
    if (grp == 0 && col < N) {
        float t = 0.f;
        for (int q = 0; q < 8; ++q) t += red[q][lane];
        part[(long long)blockIdx.y * N + col] = t;
    }
}

// Chunk partials added in a fixed order: warp w of CTA x sums chunks w, w + 8, ... of columns
// 32x .. 32x + 31, then warp 0 adds the eight sums in warp order.
__global__ void __launch_bounds__(256) colsum_final_kernel(const float *part, int chunks, int N, float *out)
{
    __shared__ float red[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    float t = 0.f;
    if (n < N)
        for (int c = w; c < chunks; c += 8) t += part[(long long)c * N + n];
    red[w][lane] = t;
    __syncthreads();
    if (w == 0 && n < N) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += red[q][lane];
        out[n] = s;
    }
}

// Softmax cross-entropy per row (one warp per row, Q <= 64): dlog = (softmax - onehot) * inv_r,
// rowloss = -log softmax(label).
__global__ void ce_loss_kernel(const float *logits, const int *labels, int R, int Q, float inv_r,
                               float *dlog, float *rowloss, unsigned *status)
{
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= R) return;
    const float *z = logits + w * Q;
    const float z0 = lane < Q ? z[lane] : -INFINITY;
    const float z1 = lane + 32 < Q ? z[lane + 32] : -INFINITY;
    float m = fmaxf(z0, z1);
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    const float e0 = lane < Q ? expf(z0 - m) : 0.f;
    const float e1 = lane + 32 < Q ? expf(z1 - m) : 0.f;
    float S = e0 + e1;
#pragma unroll
    for (int o = 16; o; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
    int lab = labels[w];
    if (lab < 0 || lab >= Q) {
        if (lane == 0) set_status(status, kStatusBadState);
        lab = 0;
    }
    const float inv = 1.f / S;
    if (lane < Q) dlog[w * Q + lane] = (e0 * inv - (lane == lab ? 1.f : 0.f)) * inv_r;
    if (lane + 32 < Q) dlog[w * Q + lane + 32] = (e1 * inv - (lane + 32 == lab ? 1.f : 0.f)) * inv_r;
    if (lane == 0) {
        const float l = -(z[lab] - m - logf(S));
        if (!isfinite(l)) set_status(status, kStatusNumeric);
        rowloss[w] = l;
    }
}

// out = scale * sum_r v[r] (one block, fixed order).
__global__ void sum_kernel(const float *v, int R, float scale, float *out)
{
    __shared__ float red[256];
    float s = 0.f;
    for (int r = threadIdx.x; r < R; r += 256) s += v[r];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 128; h; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] * scale;
}

__global__ void gather_kernel(const float *X, const int *labels, const int *idx, int R,
                              long long n_src, float *xg, int *lg, unsigned *status)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    long long s = idx[r];
    if (s < 0 || s >= n_src) {
        set_status(status, kStatusBadState);
        s = 0;
    }
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) xg[(long long)r * kMlpIn + j] = X[s * kMlpIn + j];
    lg[r] = labels[s];
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr (m c1) / (sqrt(v c2) + eps) with c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, long long n, float lr,
                            float c1, float c2)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// ------------------------------------------------------------------------------------------
// Tensor-core inference
// ------------------------------------------------------------------------------------------
// All three layers run on the tensor cores.
// Layer 1 (K = 6 features) is evaluated to FP32 accuracy from BF16 terms: every feature x and
// weight w is split into three terms, x = x0 + x1 + x2 (each the round-to-nearest BF16 of what
// the previous leave; the remainder is below 2^-26 |x|), and the six products x_i w_j with
// i + j <= 2 are laid side by side along K (the dropped ones are below 2^-26 |x w|), followed by
// the bias's three terms against constant 1.0 columns: K = 6 x 6 + 3, padded to 48.
// Layers 2 and 3 contract over the 256 BF16 hidden values plus their bias, again three BF16
// terms against 1.0 columns: K = 256 + 3, padded to 272. Every MMA adds its bias itself.
constexpr int kMlpK = kMlpHidden + 16;                         // 272
constexpr int kMlpK1 = 48;
constexpr uint32_t kCoreSbo = (kMlpK / 8) * 128;              // 8-row group stride, K = 272
constexpr uint32_t kCoreSbo1 = (kMlpK1 / 8) * 128;            // 8-row group stride, K = 48
constexpr uint32_t kW2Bytes = kMlpHidden * kMlpK * 2;         // 139264
constexpr uint32_t kW1Bytes = kMlpHidden * kMlpK1 * 2;        // 24576
constexpr uint32_t kA0Bytes = 128 * kMlpK1 * 2;               // 12288, one tile's layer-1 A operand
constexpr int kMlpTmemCols = 512;

__host__ __device__ inline uint32_t mlp_w3_bytes(int Qp) { return (uint32_t)Qp * kMlpK * 2u; }

__host__ __device__ inline uint32_t mlp_smem_bytes(int Qp)
{
    return kW2Bytes + mlp_w3_bytes(Qp) + kW1Bytes + 2 * kA0Bytes + 256u;   // + mbarriers, TMEM slot
}

// Byte offset of element (row, k) in a K-major, no-swizzle core-matrix image of stride sbo.
__device__ __forceinline__ uint32_t core_off(int row, int k, uint32_t sbo = kCoreSbo)
{
    return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Three-term BF16 split of an FP32 value (as floats).
__device__ __forceinline__ void split3(float v, float (&t)[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        t[i] = __bfloat162float(__float2bfloat16_rn(v));
        v -= t[i];
    }
}

// Term of a layer-1 weight (B side) and of a feature (A side) at position t = 0..5 of a
// feature's six K slots: the products x0 w0, x0 w1, x1 w0, x0 w2, x1 w1, x2 w0.
__host__ __device__ constexpr int l1_wterm(int t) { return t == 1 || t == 4 ? 1 : (t == 3 ? 2 : 0); }
__host__ __device__ constexpr int l1_xterm(int t) { return t == 2 || t == 4 ? 1 : (t == 5 ? 2 : 0); }

// Operand images in global memory, one thread per 8 K values of a row:
//   W2 | b2 (256 x 272), W3 | b3 (rows padded to Qp with zeros), W1 terms | b1 (256 x 48).
__global__ void mlp_pack_kernel(const float *params, int Q, int Qp, uint8_t *ops)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n23 = (kMlpHidden + Qp) * (kMlpK / 8);
    if (e >= n23 + kMlpHidden * (kMlpK1 / 8)) return;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = 0.f;
    uint8_t *dst;
    if (e < n23) {
        const int n = e / (kMlpK / 8), c = e % (kMlpK / 8);
        const float *w = nullptr;   // the row's weights
        float bias = 0.f;
        if (n < kMlpHidden) {
            w = params + mlp_off_W2() + (long long)n * kMlpHidden;
            bias = params[mlp_off_b2() + n];
            dst = ops + core_off(n, 8 * c);
        } else {
            const int nn = n - kMlpHidden;
            if (nn < Q) {
                w = params + mlp_off_W3() + (long long)nn * kMlpHidden;
                bias = params[mlp_off_b3(Q) + nn];
            }
            dst = ops + kW2Bytes + core_off(nn, 8 * c);
        }
        if (w && 8 * c < kMlpHidden) {
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] = w[8 * c + j];
        } else if (w && 8 * c == kMlpHidden) {
            float t[3];   // k = 256, 257, 258: the bias's three terms (k = 259 .. 271 stay zero)
            split3(bias, t);
            v[0] = t[0]; v[1] = t[1]; v[2] = t[2];
        }
    } else {
        const int f = e - n23, u = f / (kMlpK1 / 8), c = f % (kMlpK1 / 8);
        dst = ops + kW2Bytes + mlp_w3_bytes(Qp) + core_off(u, 8 * c, kCoreSbo1);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * c + j;
            float t[3];
            if (k < 6 * kMlpIn) {
                split3(params[(long long)u * kMlpIn + k / 6], t);
                v[j] = t[l1_wterm(k % 6)];
            } else if (k < 6 * kMlpIn + 3) {
                split3(params[mlp_off_b1() + u], t);
                v[j] = t[k - 6 * kMlpIn];
            }
        }
    }
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) pk[j] = pack_bf16(v[2 * j], v[2 * j + 1]);
    *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&p)[16])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(p[0]), "r"(p[1]), "r"(p[2]), "r"(p[3]), "r"(p[4]), "r"(p[5]), "r"(p[6]),
        "r"(p[7]), "r"(p[8]), "r"(p[9]), "r"(p[10]), "r"(p[11]), "r"(p[12]), "r"(p[13]), "r"(p[14]),
        "r"(p[15])
        : "memory");
}

// The bias columns of an A operand in tensor memory (k = 256 .. 271: 1, 1, 1, then zeros).
__device__ __forceinline__ void tmem_st_bias_cols(uint32_t taddr)
{
    const uint32_t one2 = 0x3F803F80u, one = 0x00003F80u;   // BF16 1.0 = 0x3F80
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%3,%3,%3,%3,%3};" ::"r"(taddr), "r"(one2),
        "r"(one), "r"(0u)
        : "memory");
}

template <int Q>
struct MlpTcArgs {
    long long rows;
    const float *X;
    const uint8_t *ops;     // W2 | b2, W3 | b3 and W1 | b1 images
    float *logits;
    unsigned *status;
    int vec_out;            // logits 16-byte aligned
};

// Roles of the inference kernel's warps: four feature warps (layer 1's A operand), four layer-1
// epilogue warps, four layer-2/3 epilogue warps (an epilogue warp w serves TMEM lane quadrant
// w % 4, one row per thread) and one MMA warp.
constexpr int kXWarps = 4, kE0Warps = 4, kE1Warps = 4;
constexpr int kMmaWarpId = kXWarps + kE0Warps + kE1Warps;
constexpr int kMlpThreads = 32 * (kMmaWarpId + 1);
// Tensor-memory columns. Region 0: layer-1 accumulators, over whose first 136 columns the
// epilogue writes h1 with its bias columns (layer 2's A operand) once it has read them. Region
// 1: layer-2 accumulators, then h2 with its bias columns in the same way (layer 3's A operand),
// and the logits' accumulators in its last 64 columns (written once h2 is there).
constexpr uint32_t kColR0 = 0, kColR1 = 256, kColD2 = 448;
// mbarriers: weights loaded, and the full / empty hand-overs of the pipeline
enum : int { kBarW, kBarA0Full0, kBarA0Full1, kBarA0Empty0, kBarA0Empty1, kBarD0Full, kBarA1Full,
             kBarA1Empty, kBarD1Full, kBarA2Full, kBarD2Full, kBarR1Free, kBarDone, kMlpBars };

// max(lo, 0) and max(hi, 0) rounded to BF16, lo in the low half.
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// BF16 MMA whose A operand (M = 128 rows in the 128 lanes, K along the columns, two values per
// column) is in tensor memory.
__device__ __forceinline__ void mma_bf16_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t db, uint32_t idesc,
                                            uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
        "r"(tmem_a), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mlp_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mlp_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Layer 1's A operand for one row: the six feature terms of each input, then 1.0 three times
// (the bias terms), zeros to K = 48.
__device__ __forceinline__ void mlp_features(const float (&x)[kMlpIn], unsigned char *img, int row)
{
    float v[kMlpK1];
#pragma unroll
    for (int k = 0; k < kMlpK1; ++k) v[k] = 0.f;
#pragma unroll
    for (int q = 0; q < kMlpIn; ++q) {
        float t[3];
        split3(x[q], t);
#pragma unroll
        for (int i = 0; i < 6; ++i) v[6 * q + i] = t[l1_xterm(i)];
    }
    v[6 * kMlpIn] = v[6 * kMlpIn + 1] = v[6 * kMlpIn + 2] = 1.f;
#pragma unroll
    for (int g = 0; g < kMlpK1 / 8; ++g)
        *reinterpret_cast<uint4 *>(img + core_off(row, 8 * g, kCoreSbo1)) =
            make_uint4(pack_bf16(v[8 * g], v[8 * g + 1]), pack_bf16(v[8 * g + 2], v[8 * g + 3]),
                       pack_bf16(v[8 * g + 4], v[8 * g + 5]), pack_bf16(v[8 * g + 6], v[8 * g + 7]));
}

// ReLU and BF16 of one row's 256 accumulators (the bias is in them) at column col, written in
// place as the next layer's A operand over the columns already read, then its bias columns.
__device__ __forceinline__ void mlp_relu_inplace(uint32_t col)
{
#pragma unroll 1
    for (int c = 0; c < kMlpHidden / 32; ++c) {
        float v[32];
        tmem_ld32(col + (uint32_t)(32 * c), v);
        uint32_t pk[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) pk[j] = pack_relu_bf16(v[2 * j], v[2 * j + 1]);
        tmem_st16(col + (uint32_t)(16 * c), pk);
    }
    tmem_st_bias_cols(col + kMlpHidden / 2);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Layer-3 epilogue of one row: the logits (bias included) -> global memory, 16-byte stores when
// the output is aligned.
template <int Q>
__device__ __forceinline__ void mlp_logits(const MlpTcArgs<Q> &a, uint32_t lane_base, long long r)
{
    constexpr int Qp = (Q + 15) / 16 * 16;
    float v[Qp];
#pragma unroll
    for (int c = 0; c < Qp / 8; ++c) {
        float t[8];
        tmem_ld8(lane_base + kColD2 + (uint32_t)(8 * c), t);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[8 * c + j] = t[j];
    }
    if (r >= a.rows) return;
    float *out = a.logits + r * Q;
    if (a.vec_out) {
#pragma unroll
        for (int n = 0; n < Q; n += 4)
            *reinterpret_cast<float4 *>(out + n) = make_float4(v[n], v[n + 1], v[n + 2], v[n + 3]);
    } else {
#pragma unroll
        for (int n = 0; n < Q; ++n) out[n] = v[n];
    }
}

// Persistent, one CTA per SM, 128-row tiles through a pipeline:
//   feature warps:  X -> layer 1's A operand (three BF16 terms per feature) in shared memory,
//                   two buffers;
//   MMA warp:       D0 = A0 [W1 | b1]^T (3 MMAs, N = 256), D1 = [h1 | 1] [W2 | b2]^T (17 MMAs,
//                   N = 256, A in tensor memory), D2 = [h2 | 1] [W3 | b3]^T (17 MMAs, N = Qp,
//                   A in tensor memory), issued in the order D1(t), D0(t + 1), D2(t);
//   layer-1 epilogue warps: D0 -> h1 = BF16(ReLU(D0)) in place;
//   layer-2/3 epilogue warps: D1 -> h2 = BF16(ReLU(D1)) in place, D2 -> logits.
// So layer 1 of the next tile and its epilogue run beside this tile's layer-2 epilogue and
// layer 3. Every hand-over is an mbarrier (MMA completion through tcgen05.commit). Every wait is
// bounded and the warp-collective roles take each wait's verdict for the whole warp: a role that
// gives up sets the timeout status and leaves its loop, the others run out of their own waits,
// and the CTA waits (bounded) for its last MMAs before it frees the tensor memory.
template <int Q>
__global__ void __launch_bounds__(kMlpThreads, 1) mlp_tc_kernel(const __grid_constant__ MlpTcArgs<Q> a)
{
    constexpr int Qp = (Q + 15) / 16 * 16;
    constexpr int kSteps = kMlpK / 16;   // 17
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char *sW2 = smem;
    unsigned char *sW3 = sW2 + kW2Bytes;
    unsigned char *sW1 = sW3 + mlp_w3_bytes(Qp);
    unsigned char *sA0 = sW1 + kW1Bytes;                   // two buffers
    uint64_t *bars = reinterpret_cast<uint64_t *>(sA0 + 2 * kA0Bytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + kMlpBars);
    auto bar = [&](int i) { return smem_u32(&bars[i]); };
    if (tid == 0) {
        mbar_init(bar(kBarW), 1);
        mbar_init(bar(kBarA0Full0), 32 * kXWarps);
        mbar_init(bar(kBarA0Full1), 32 * kXWarps);
        mbar_init(bar(kBarA0Empty0), 1);
        mbar_init(bar(kBarA0Empty1), 1);
        mbar_init(bar(kBarD0Full), 1);
        mbar_init(bar(kBarA1Full), 32 * kE0Warps);
        mbar_init(bar(kBarA1Empty), 1);
        mbar_init(bar(kBarD1Full), 1);
        mbar_init(bar(kBarA2Full), 32 * kE1Warps);
        mbar_init(bar(kBarD2Full), 1);
        mbar_init(bar(kBarR1Free), 32 * kE1Warps);
        mbar_init(bar(kBarDone), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarpId) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kMlpTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // the three weight images: one bulk copy per CTA
    const uint32_t wbytes = kW2Bytes + mlp_w3_bytes(Qp) + kW1Bytes;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(kBarW)),
                     "r"(wbytes)
                     : "memory");
        const uint32_t chunk = 1u << 15;
        for (uint32_t off = 0; off < wbytes; off += chunk) {
            const uint32_t n = wbytes - off < chunk ? wbytes - off : chunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                "%2, [%3];" ::"r"(smem_u32(sW2) + off),
                "l"(a.ops + off), "r"(n), "r"(bar(kBarW))
                : "memory");
        }
    }
    bool ok = !__syncthreads_or(!mbar_wait(bar(kBarW), 0));
    const long long ntiles = (a.rows + 127) / 128;
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    // a wait whose verdict the whole warp takes (the tensor-memory loads and stores that follow
    // are warp-collective)
    auto wwait = [&](int b, uint32_t parity) {
        return __all_sync(0xffffffffu, mbar_wait(bar(b), parity)) != 0;
    };
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    auto row_of = [&](int j) {
        return ((long long)blockIdx.x + (long long)j * gridDim.x) * 128 + 32 * (warp & 3) + lane;
    };

    if (ok && warp < kXWarps) {
        // features: thread = row 32 w + lane
        const int row_l = 32 * warp + lane;
        float x[kMlpIn];
        auto load_x = [&](int j) {
            const long long r = row_of(j);
#pragma unroll
            for (int q = 0; q < kMlpIn; ++q) x[q] = r < a.rows ? a.X[r * kMlpIn + q] : 0.f;
        };
        load_x(0);
        for (int j = 0; j < my_tiles; ++j) {
            const int b = j & 1;
            // layer 1 of tile j - 2 read this buffer: wait for its commit
            if (j >= 2 && !wwait(b ? kBarA0Empty1 : kBarA0Empty0, (uint32_t)((j >> 1) - 1) & 1u)) {
                ok = false;
                break;
            }
            mlp_features(x, sA0 + b * kA0Bytes, row_l);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mlp_arrive(bar(b ? kBarA0Full1 : kBarA0Full0));
            if (j + 1 < my_tiles) load_x(j + 1);
        }
    } else if (ok && warp < kXWarps + kE0Warps) {
        // layer-1 epilogue: thread = row = its TMEM lane
        for (int j = 0; j < my_tiles; ++j) {
            if (!wwait(kBarD0Full, (uint32_t)j & 1u)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mlp_relu_inplace(lane_base + kColR0);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mlp_arrive(bar(kBarA1Full));
        }
    } else if (ok && warp < kMmaWarpId) {
        // layer-2 and layer-3 epilogues: thread = row = its TMEM lane
        for (int j = 0; j < my_tiles; ++j) {
            const uint32_t ph = (uint32_t)j & 1u;
            if (!wwait(kBarD1Full, ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mlp_relu_inplace(lane_base + kColR1);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mlp_arrive(bar(kBarA2Full));
            if (!wwait(kBarD2Full, ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            mlp_logits<Q>(a, lane_base, row_of(j));
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mlp_arrive(bar(kBarR1Free));
        }
    } else if (ok && lane == 0) {
        // MMA warp, one lane
        const uint32_t idesc_h = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMlpHidden >> 3) << 17) |
                                 ((uint32_t)(128 >> 4) << 24);
        const uint32_t idesc_q = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Qp >> 3) << 17) |
                                 ((uint32_t)(128 >> 4) << 24);
        const uint32_t sb1 = smem_u32(sW1), sb2 = smem_u32(sW2), sb3 = smem_u32(sW3), sa0 = smem_u32(sA0);
        // layer 1 of tile j: its features, and region 0 free (layer 2 of tile j - 1 complete)
        auto layer1 = [&](int j) {
            const int b = j & 1;
            if (!mbar_wait(bar(b ? kBarA0Full1 : kBarA0Full0), (uint32_t)(j >> 1) & 1u)) return false;
            if (j > 0 && !mbar_wait(bar(kBarA1Empty), (uint32_t)(j - 1) & 1u)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < kMlpK1 / 16; ++ks)
                mma_bf16(tmem + kColR0, smem_desc(sa0 + b * kA0Bytes + ks * 256u, 128u, kCoreSbo1),
                         smem_desc(sb1 + ks * 256u, 128u, kCoreSbo1), idesc_h, ks ? 1u : 0u);
            mlp_commit(bar(b ? kBarA0Empty1 : kBarA0Empty0));
            mlp_commit(bar(kBarD0Full));
            return true;
        };
        if (my_tiles > 0) ok = layer1(0);
        for (int j = 0; j < my_tiles && ok; ++j) {
            const uint32_t ph = (uint32_t)j & 1u, pp = (uint32_t)(j - 1) & 1u;
            // layer 2: h1 of this tile, and region 1 free (the previous tile's logits read out)
            if (!mbar_wait(bar(kBarA1Full), ph) || (j > 0 && !mbar_wait(bar(kBarR1Free), pp))) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < kSteps; ++ks)
                mma_bf16_ta(tmem + kColR1, tmem + kColR0 + (uint32_t)(8 * ks),
                            smem_desc(sb2 + ks * 256u, 128u, kCoreSbo), idesc_h, ks ? 1u : 0u);
            mlp_commit(bar(kBarA1Empty));
            mlp_commit(bar(kBarD1Full));
            // layer 1 of the next tile while this tile's layer-2 epilogue runs
            if (j + 1 < my_tiles && !layer1(j + 1)) { ok = false; break; }
            // layer 3: h2 of this tile
            if (!mbar_wait(bar(kBarA2Full), ph)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < kSteps; ++ks)
                mma_bf16_ta(tmem + kColD2, tmem + kColR1 + (uint32_t)(8 * ks),
                            smem_desc(sb3 + ks * 256u, 128u, kCoreSbo), idesc_q, ks ? 1u : 0u);
            mlp_commit(bar(kBarD2Full));
        }
        // completes once every MMA issued above has (at once when there were none)
        mlp_commit(bar(kBarDone));
    }
    if (!ok) set_status(a.status, kStatusTimeout);
    __syncwarp();
    // no thread frees the tensor memory while an MMA may still write it
    if (warp == kMmaWarpId) {
        const bool done = __shfl_sync(0xffffffffu, lane == 0 ? mbar_wait(bar(kBarDone), 0) : false, 0);
        if (!done && lane == 0) set_status(a.status, kStatusTimeout);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kMmaWarpId)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kMlpTmemCols));
}

int g_sm_count = 0;

cudaError_t gemm_simt(const GemmArgs &in, float *partial, size_t partial_floats, cudaStream_t s, int *launches)
{
    GemmArgs g = in;
    const int tm = (g.M + kBM - 1) / kBM, tn = (g.N + kBN - 1) / kBN;
    int splits = 1;
    if (partial && g.K > 4 * kBK && !g.bias && !g.relu && !g.mask) {
        const int want = (2 * std::max(g_sm_count, 1) + tm * tn - 1) / (tm * tn);
        const int kmax = (g.K + kBK - 1) / kBK;
        splits = std::max(1, std::min(want, kmax));
        while (splits > 1 && (size_t)splits * g.M * g.N > partial_floats) --splits;
    }
    g.kchunk = ((g.K + splits - 1) / splits + kBK - 1) / kBK * kBK;
    splits = (g.K + g.kchunk - 1) / g.kchunk;
    if (splits < 1) splits = 1;
    g.partial = splits > 1 ? partial : nullptr;
    sgemm_kernel<<<dim3(tn, tm, splits), 256, 0, s>>>(g);
    cudaError_t e = cudaGetLastError();
    *launches = 1;
    if (e != cudaSuccess || splits == 1) return e;
    const long long MN = (long long)g.M * g.N;
    const int blocks = (int)std::min<long long>((MN + 255) / 256, 4096);
    splitk_reduce_kernel<<<blocks, 256, 0, s>>>(partial, splits, g.M, g.N, g.C, g.ldc);
    *launches = 2;
    return cudaGetLastError();
}

// A product of the network: on tcgen05 (split-BF16 operands, FP32 accumulation) when the handle
// trains on tensor cores, else the CUDA-core kernel.
cudaError_t gemm(mcmc_mlp *m, const GemmArgs &in, float *partial, size_t partial_floats,
                 cudaStream_t s)
{
    int launches = 0;
    cudaError_t e;
    if (m->tc_train) {
        TcGemmArgs t{};
        t.M = in.M; t.N = in.N; t.K = in.K;
        t.A = in.A; t.sam = in.sam; t.sak = in.sak;
        t.B = in.B; t.sbk = in.sbk; t.sbn = in.sbn;
        t.C = in.C; t.ldc = in.ldc;
        t.bias = in.bias; t.mask = in.mask; t.ldm = in.ldm; t.relu = in.relu;
        t.status = m->status;
        e = tc_gemm(t, partial, partial_floats, m->sm_count, s, &launches);
    } else {
        e = gemm_simt(in, partial, partial_floats, s, &launches);
    }
    m->launches += launches;
    return e;
}

GemmArgs gargs(int M, int N, int K, const float *A, long long sam, long long sak, const float *B,
               long long sbk, long long sbn, float *C, long long ldc)
{
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.sam = sam; g.sak = sak;
    g.B = B; g.sbk = sbk; g.sbn = sbn;
    g.C = C; g.ldc = ldc;
    return g;
}

// Column sums of an R x N row-major block (colsum_kernel), staged in the split-K buffer (free
// between products on the handle's stream); two launches.
cudaError_t colsum(mcmc_mlp *m, const float *A, int R, int N, float *out, cudaStream_t s)
{
    const int cgroups = (N + 31) / 32;
    int chunks = std::max(1, std::min((R + 255) / 256, 2 * std::max(m->sm_count, 1) / cgroups));
    while (chunks > 1 && (size_t)chunks * N > m->partial_floats) --chunks;
    const int rpc = std::max(1, (R + chunks - 1) / chunks);
    chunks = std::max(1, (R + rpc - 1) / rpc);
    colsum_kernel<<<dim3(cgroups, chunks), 256, 0, s>>>(A, R, N, N, rpc, m->partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    colsum_final_kernel<<<(N + 31) / 32, 256, 0, s>>>(m->partial, chunks, N, out);
    m->launches += 2;
    return cudaGetLastError();
}

// Forward of R rows (R <= max_rows) keeping h1, h2 and the logits in the workspace.
cudaError_t forward_rows(mcmc_mlp *m, int R, const float *X, float *logits, cudaStream_t s)
{
    const float *P = m->params;
    const int H = kMlpHidden;
    GemmArgs g = gargs(R, H, kMlpIn, X, kMlpIn, 1, P, 1, kMlpIn, m->h1, H);
    g.bias = P + mlp_off_b1();
    g.relu = 1;
    cudaError_t e = gemm(m, g, nullptr, 0, s);
    if (e != cudaSuccess) return e;
    g = gargs(R, H, H, m->h1, H, 1, P + mlp_off_W2(), 1, H, m->h2, H);
    g.bias = P + mlp_off_b2();
    g.relu = 1;
    if ((e = gemm(m, g, nullptr, 0, s)) != cudaSuccess) return e;
    g = gargs(R, m->Q, H, m->h2, H, 1, P + mlp_off_W3(), 1, H, logits, m->Q);
    g.bias = P + mlp_off_b3(m->Q);
    return gemm(m, g, nullptr, 0, s);
}

template <int Q>
cudaError_t launch_tc(mcmc_mlp *m, long long rows, const float *X, float *logits, int grid,
                      cudaStream_t s)
{
    constexpr int Qp = (Q + 15) / 16 * 16;
    const uint32_t smem = mlp_smem_bytes(Qp);
    cudaError_t e = cudaFuncSetAttribute(mlp_tc_kernel<Q>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    MlpTcArgs<Q> a;
    a.rows = rows;
    a.X = X;
    a.ops = m->tc_ops;
    a.logits = logits;
    a.status = m->status;
    a.vec_out = ((uintptr_t)logits & 15u) == 0;
    mlp_tc_kernel<Q><<<grid, kMlpThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlp_forward_simt(mcmc_mlp *m, long long rows, const float *X, float *logits,
                             cudaStream_t s)
{
    for (long long r0 = 0; r0 < rows; r0 += m->max_rows) {
        const int R = (int)std::min<long long>(m->max_rows, rows - r0);
        cudaError_t e = forward_rows(m, R, X + r0 * kMlpIn, logits + r0 * m->Q, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t mlp_forward_tc(mcmc_mlp *m, long long rows, const float *X, float *logits,
                           cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    if (!m->tc_valid) {
        const int n = (kMlpHidden + m->Qp) * (kMlpK / 8) + kMlpHidden * (kMlpK1 / 8);
        mlp_pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(m->params, m->Q, m->Qp, m->tc_ops);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        m->launches++;
        m->tc_valid = true;
    }
    const long long tiles = (rows + 127) / 128;
    const int grid = (int)std::min<long long>(tiles, std::max(g_sm_count, 1));
    cudaError_t e = cudaSuccess;
    switch (m->Q) {
    case 4: e = launch_tc<4>(m, rows, X, logits, grid, s); break;
    case 16: e = launch_tc<16>(m, rows, X, logits, grid, s); break;
    default: e = launch_tc<64>(m, rows, X, logits, grid, s); break;
    }
    if (e == cudaSuccess) m->launches++;
    return e;
}

}  // namespace mcmcdet

using namespace mcmcdet;

namespace {

mcmc_status mfail(mcmc_mlp *m, mcmc_status s, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

mcmc_status mfail(mcmc_mlp *m, mcmc_status s, const char *fmt, ...)
{
    if (m) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        m->err = buf;
    }
    return s;
}

mcmc_status mcuda(mcmc_mlp *m, cudaError_t e, const char *what)
{
    return mfail(m, e == cudaErrorMemoryAllocation ? MCMC_ENOMEM : MCMC_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

#define MCK(call, what)                                     \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return mcuda(m, e_, what);   \
    } while (0)

bool valid_q(int q) { return q == 4 || q == 16 || q == 64; }

mcmc_status read_mlp_status(mcmc_mlp *m)
{
    unsigned st = 0;
    MCK(cudaMemcpyAsync(&st, m->status, 4, cudaMemcpyDeviceToHost, m->stream), "copy status");
    MCK(cudaStreamSynchronize(m->stream), "stream synchronize");
    if (st == 0) return MCMC_OK;
    MCK(cudaMemsetAsync(m->status, 0, 4, m->stream), "clear status");
    if (st & kStatusTimeout) return mfail(m, MCMC_ETIMEOUT, "a bounded device wait ran out");
    if (st & kStatusBadState) return mfail(m, MCMC_EINVAL, "label or row index out of range");
    return mfail(m, MCMC_ENUMERIC, "non-finite loss");
}

// Loss and gradient of R gathered rows (xs, ls) into grad.
mcmc_status loss_grad_rows(mcmc_mlp *m, int R, const float *xs, const int *ls, float *loss,
                           float *grad)
{
    const int H = kMlpHidden, Q = m->Q;
    cudaStream_t s = m->stream;
    const float *P = m->params;
    MCK(forward_rows(m, R, xs, m->logit, s), "mlp forward");
    ce_loss_kernel<<<(unsigned)(((long long)R * 32 + 255) / 256), 256, 0, s>>>(
        m->logit, ls, R, Q, 1.f / (float)R, m->dlog, m->rowloss, m->status);
    MCK(cudaGetLastError(), "loss kernel");
    if (loss) {
        sum_kernel<<<1, 256, 0, s>>>(m->rowloss, R, 1.f / (float)R, loss);
        MCK(cudaGetLastError(), "loss sum");
        m->launches++;
    }
    // layer 3: gW3 = dlog^T h2, gb3 = colsum(dlog), da2 = (dlog W3) * [h2 > 0]
    MCK(gemm(m, gargs(Q, H, R, m->dlog, 1, Q, m->h2, H, 1, grad + mlp_off_W3(), H), m->partial,
             m->partial_floats, s), "gW3");
    MCK(colsum(m, m->dlog, R, Q, grad + mlp_off_b3(Q), s), "gb3");
    GemmArgs g = gargs(R, H, Q, m->dlog, Q, 1, P + mlp_off_W3(), H, 1, m->dh, H);
    g.mask = m->h2;
    g.ldm = H;
    MCK(gemm(m, g, nullptr, 0, s), "da2");
    // layer 2: gW2 = da2^T h1, gb2, da1 = (da2 W2) * [h1 > 0] (into the h2 buffer)
    MCK(gemm(m, gargs(H, H, R, m->dh, 1, H, m->h1, H, 1, grad + mlp_off_W2(), H), m->partial,
             m->partial_floats, s), "gW2");
    MCK(colsum(m, m->dh, R, H, grad + mlp_off_b2(), s), "gb2");
    g = gargs(R, H, H, m->dh, H, 1, P + mlp_off_W2(), H, 1, m->h2, H);
    g.mask = m->h1;
    g.ldm = H;
    MCK(gemm(m, g, nullptr, 0, s), "da1");
    // layer 1: gW1 = da1^T X, gb1
    MCK(gemm(m, gargs(H, kMlpIn, R, m->h2, 1, H, xs, kMlpIn, 1, grad, kMlpIn), m->partial,
             m->partial_floats, s), "gW1");
    MCK(colsum(m, m->h2, R, H, grad + mlp_off_b1(), s), "gb1");
    m->launches++;   // the loss kernel; products and column sums count their own
    return MCMC_OK;
}

mcmc_status prepare_rows(mcmc_mlp *m, int rows, const float *X, const int *labels, const int *idx,
                         const float **xs, const int **ls)
{
    if (rows < 1 || rows > m->max_rows) return mfail(m, MCMC_EINVAL, "rows must be in 1..%d", m->max_rows);
    if (!X || !labels) return mfail(m, MCMC_EINVAL, "null features or labels");
    *xs = X;
    *ls = labels;
    if (idx) {
        gather_kernel<<<(rows + 255) / 256, 256, 0, m->stream>>>(X, labels, idx, rows, 1ll << 40,
                                                                 m->xg, m->lg, m->status);
        MCK(cudaGetLastError(), "gather");
        m->launches++;
        *xs = m->xg;
        *ls = m->lg;
    }
    return MCMC_OK;
}

}  // namespace

extern "C" {

int64_t mcmc_mlp_param_count(int32_t qam)
{
    return valid_q(qam) ? (int64_t)mlp_param_count(qam) : 0;
}

const char *mcmc_mlp_last_error(const mcmc_mlp *m)
{
    return m ? m->err.c_str() : "null handle";
}

mcmc_status mcmc_mlp_create(int32_t qam, int32_t max_rows, void *stream, mcmc_mlp **out)
{
    if (!out) return MCMC_EINVAL;
    *out = nullptr;
    if (!valid_q(qam) || max_rows < 1 || max_rows > (1 << 24)) return MCMC_EINVAL;
    mcmc_mlp *m = new (std::nothrow) mcmc_mlp();
    if (!m) return MCMC_ENOMEM;
    m->Q = qam;
    m->Qp = (qam + 15) / 16 * 16;
    m->max_rows = max_rows;
    auto bail = [&](cudaError_t e) {
        mcmc_status st = e == cudaErrorMemoryAllocation ? MCMC_ENOMEM : MCMC_ECUDA;
        mcmc_mlp_destroy(m);
        return st;
    };
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) return bail(e);
    if (!g_sm_count) cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, m->device);
    {
        int mj = 0, mn = 0;
        cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, m->device);
        cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, m->device);
        m->tc_train = mj == 10 && mn == 3;
        cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    }
    if (stream) {
        m->stream = (cudaStream_t)stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&m->stream, cudaStreamDefault)) != cudaSuccess) return bail(e);
        m->own_stream = true;
    }
    const size_t P = (size_t)mlp_param_count(qam);
    const size_t R = (size_t)max_rows, H = kMlpHidden;
    m->partial_floats = (size_t)64 * H * H;
    struct { void **p; size_t bytes; } allocs[] = {
        {(void **)&m->params, 4 * P}, {(void **)&m->grad, 4 * P}, {(void **)&m->adam_m, 4 * P},
        {(void **)&m->adam_v, 4 * P}, {(void **)&m->xg, 4 * R * kMlpIn}, {(void **)&m->lg, 4 * R},
        {(void **)&m->h1, 4 * R * H}, {(void **)&m->h2, 4 * R * H}, {(void **)&m->dh, 4 * R * H},
        {(void **)&m->dlog, 4 * R * qam}, {(void **)&m->logit, 4 * R * qam},
        {(void **)&m->rowloss, 4 * R}, {(void **)&m->partial, 4 * m->partial_floats},
        {(void **)&m->status, 256}, {(void **)&m->tc_ops, mlp_tc_bytes(m->Qp)},
    };
    for (auto &a : allocs)
        if ((e = cudaMalloc(a.p, a.bytes)) != cudaSuccess) return bail(e);
    for (void *p : {(void *)m->params, (void *)m->adam_m, (void *)m->adam_v})
        if ((e = cudaMemsetAsync(p, 0, 4 * P, m->stream)) != cudaSuccess) return bail(e);
    if ((e = cudaMemsetAsync(m->status, 0, 256, m->stream)) != cudaSuccess) return bail(e);
    if ((e = cudaStreamSynchronize(m->stream)) != cudaSuccess) return bail(e);
    *out = m;
    return MCMC_OK;
}

mcmc_status mcmc_mlp_destroy(mcmc_mlp *m)
{
    if (!m) return MCMC_EINVAL;
    if (m->stream) cudaStreamSynchronize(m->stream);
    for (void *p : {(void *)m->params, (void *)m->grad, (void *)m->adam_m, (void *)m->adam_v,
                    (void *)m->xg, (void *)m->lg, (void *)m->h1, (void *)m->h2, (void *)m->dh,
                    (void *)m->dlog, (void *)m->logit, (void *)m->rowloss, (void *)m->partial,
                    (void *)m->status, (void *)m->tc_ops})
        if (p) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
    return MCMC_OK;
}

mcmc_status mcmc_mlp_set_train_engine(mcmc_mlp *m, int32_t tensor_cores)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (tensor_cores != 0 && tensor_cores != 1) return mfail(m, MCMC_EINVAL, "tensor_cores must be 0 or 1");
    if (tensor_cores) {
        int mj = 0, mn = 0;
        cudaDeviceGetAttribute(&mj, cudaDevAttrComputeCapabilityMajor, m->device);
        cudaDeviceGetAttribute(&mn, cudaDevAttrComputeCapabilityMinor, m->device);
        if (!(mj == 10 && mn == 3)) return mfail(m, MCMC_EUNSUPPORTED, "tensor-core training needs sm_103");
    }
    m->tc_train = tensor_cores != 0;
    return MCMC_OK;
}

mcmc_status mcmc_mlp_set_params(mcmc_mlp *m, const float *params, int32_t host_io)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (!params || (host_io != 0 && host_io != 1)) return mfail(m, MCMC_EINVAL, "bad arguments");
    const size_t bytes = 4 * (size_t)mlp_param_count(m->Q);
    MCK(cudaMemcpyAsync(m->params, params, bytes, host_io ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                        m->stream), "copy params");
    MCK(cudaMemsetAsync(m->adam_m, 0, bytes, m->stream), "reset adam");
    MCK(cudaMemsetAsync(m->adam_v, 0, bytes, m->stream), "reset adam");
    if (host_io) MCK(cudaStreamSynchronize(m->stream), "stream synchronize");
    m->adam_step = 0;
    m->tc_valid = false;
    return MCMC_OK;
}

mcmc_status mcmc_mlp_get_params(mcmc_mlp *m, float *params, int32_t host_io)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (!params || (host_io != 0 && host_io != 1)) return mfail(m, MCMC_EINVAL, "bad arguments");
    const size_t bytes = 4 * (size_t)mlp_param_count(m->Q);
    MCK(cudaMemcpyAsync(params, m->params, bytes, host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                        m->stream), "copy params");
    if (host_io) MCK(cudaStreamSynchronize(m->stream), "stream synchronize");
    return MCMC_OK;
}

mcmc_status mcmc_mlp_forward(mcmc_mlp *m, int64_t rows, const float *X, float *logits,
                             int32_t tensor_cores)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (rows < 0 || !X || !logits || (tensor_cores != 0 && tensor_cores != 1))
        return mfail(m, MCMC_EINVAL, "bad arguments");
    if (tensor_cores) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, m->device);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, m->device);
        if (major * 10 + minor != 103) return mfail(m, MCMC_EUNSUPPORTED, "tcgen05 kernel needs sm_103");
        MCK(mlp_forward_tc(m, rows, X, logits, m->stream), "tensor-core mlp forward");
    } else {
        MCK(mlp_forward_simt(m, rows, X, logits, m->stream), "mlp forward");
    }
    return MCMC_OK;
}

mcmc_status mcmc_mlp_loss_grad(mcmc_mlp *m, int32_t rows, const float *X, const int32_t *labels,
                               const int32_t *idx, float *loss, float *grad)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (!grad) return mfail(m, MCMC_EINVAL, "null gradient");
    const float *xs;
    const int *ls;
    mcmc_status st = prepare_rows(m, rows, X, labels, idx, &xs, &ls);
    if (st != MCMC_OK) return st;
    st = loss_grad_rows(m, rows, xs, ls, loss, grad);
    if (st != MCMC_OK) return st;
    return read_mlp_status(m);
}

mcmc_status mcmc_mlp_train_step(mcmc_mlp *m, int32_t rows, const float *X, const int32_t *labels,
                                const int32_t *idx, float lr, float *loss)
{
    if (!m) return MCMC_EINVAL;
    m->err.clear();
    if (!(lr > 0.f) || !std::isfinite(lr)) return mfail(m, MCMC_EINVAL, "learning rate must be > 0");
    const float *xs;
    const int *ls;
    mcmc_status st = prepare_rows(m, rows, X, labels, idx, &xs, &ls);
    if (st != MCMC_OK) return st;
    st = loss_grad_rows(m, rows, xs, ls, loss, m->grad);
    if (st != MCMC_OK) return st;
    m->adam_step++;
    const double c1 = 1.0 / (1.0 - std::pow(0.9, (double)m->adam_step));
    const double c2 = 1.0 / (1.0 - std::pow(0.999, (double)m->adam_step));
    const long long P = mlp_param_count(m->Q);
    adam_kernel<<<(unsigned)std::min<long long>((P + 255) / 256, 1024), 256, 0, m->stream>>>(
        m->params, m->adam_m, m->adam_v, m->grad, P, lr, (float)c1, (float)c2);
    MCK(cudaGetLastError(), "adam");
    m->launches++;
    m->tc_valid = false;
    return MCMC_OK;
}

}  // extern "C"
