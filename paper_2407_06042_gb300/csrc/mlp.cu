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
constexpr uint32_t kW2Bytes = kMlpHidden * kMlpHidden * 2;   // 131072
constexpr uint32_t kHBytes = 128 * kMlpHidden * 2;           // 65536
constexpr uint32_t kCoreSbo = (kMlpHidden / 8) * 128;        // 8-row group stride, K = 256
constexpr int kMlpTmemCols = 512;

__host__ __device__ inline uint32_t mlp_smem_bytes(int Qp)
{
    return kW2Bytes + (uint32_t)Qp * 512u + kHBytes + 64u;
}

// Byte offset of element (row, k) in a K-major, no-swizzle core-matrix image with K = 256.
__device__ __forceinline__ uint32_t core_off(int row, int k)
{
    return (uint32_t)(row >> 3) * kCoreSbo + (uint32_t)(k >> 3) * 128u + (uint32_t)(row & 7) * 16u +
           (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// W2 and W3 (rows padded to Qp with zeros) as BF16 core-matrix images; one thread per 8 K values.
__global__ void mlp_pack_kernel(const float *params, int Q, int Qp, uint8_t *ops)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (kMlpHidden + Qp) * 32) return;
    const int n = e >> 5, c = e & 31;
    const float *src = nullptr;
    uint8_t *dst;
    if (n < kMlpHidden) {
        src = params + mlp_off_W2() + (long long)n * kMlpHidden + 8 * c;
        dst = ops + core_off(n, 8 * c);
    } else {
        const int nn = n - kMlpHidden;
        if (nn < Q) src = params + mlp_off_W3() + (long long)nn * kMlpHidden + 8 * c;
        dst = ops + kW2Bytes + core_off(nn, 8 * c);
    }
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) w[j] = src ? pack_bf16(src[2 * j], src[2 * j + 1]) : 0u;
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
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

// Small weights travel in the kernel's parameter block (constant bank): the CUDA-core layers read
// them as direct FMA operands. W2 and W3 are the BF16 operand images in global memory.
template <int Q>
struct MlpTcArgs {
    long long rows;
    const float *X;
    const uint8_t *ops;
    float *logits;
    unsigned *status;
    float W1[kMlpHidden * kMlpIn];
    float b1[kMlpHidden];
    float b2[kMlpHidden];
    float b3[Q];
};

// Issue K = 256 worth of MMAs (16 x K16) from the A image at sa and the B image at sb into
// tensor memory column tcol, then commit to the barrier (one thread).
__device__ __forceinline__ void mlp_issue(uint32_t tmem_d, uint32_t sa, uint32_t sb, uint32_t idesc,
                                          uint32_t bar)
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
    for (int ks = 0; ks < kMlpHidden / 16; ++ks)
        mma_bf16(tmem_d, smem_desc(sa + ks * 256u, 128u, kCoreSbo),
                 smem_desc(sb + ks * 256u, 128u, kCoreSbo), idesc, ks ? 1u : 0u);
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// The CUDA-core parts of one 128-row tile for one half of the hidden units / logits (HALF_ID a
// compile-time constant, so every weight is a direct constant-bank operand).
template <int Q, int HALF_ID>
__device__ __forceinline__ void mlp_layer1(const MlpTcArgs<Q> &a, const float (&x)[kMlpIn],
                                           unsigned char *hrow)
{
    constexpr int HALF = kMlpHidden / 2;
#pragma unroll
    for (int c = 0; c < HALF / 8; ++c) {
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int u = HALF * HALF_ID + 8 * c + 2 * j + h;
                float s = a.b1[u];
#pragma unroll
                for (int q = 0; q < kMlpIn; ++q) s = fmaf(a.W1[u * kMlpIn + q], x[q], s);
                v[h] = fmaxf(s, 0.f);
            }
            pk[j] = pack_bf16(v[0], v[1]);
        }
        *reinterpret_cast<uint4 *>(hrow + c * 128) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

template <int Q, int HALF_ID>
__device__ __forceinline__ void mlp_epilogue2(const MlpTcArgs<Q> &a, uint32_t lane_base,
                                              unsigned char *hrow)
{
    constexpr int HALF = kMlpHidden / 2;
#pragma unroll
    for (int c4 = 0; c4 < HALF / 32; ++c4) {
        float v[32];
        tmem_ld32(lane_base + (uint32_t)(HALF * HALF_ID + 32 * c4), v);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t pk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int u = HALF * HALF_ID + 32 * c4 + 8 * c + 2 * j;
                pk[j] = pack_bf16(fmaxf(v[8 * c + 2 * j] + a.b2[u], 0.f),
                                  fmaxf(v[8 * c + 2 * j + 1] + a.b2[u + 1], 0.f));
            }
            *reinterpret_cast<uint4 *>(hrow + (4 * c4 + c) * 128) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

template <int Q, int HALF_ID>
__device__ __forceinline__ void mlp_epilogue3(const MlpTcArgs<Q> &a, uint32_t lane_base,
                                              long long r)
{
    constexpr int Qp = (Q + 15) / 16 * 16;
    constexpr int base = (Qp / 2) * HALF_ID;
#pragma unroll
    for (int c = 0; c < Qp / 16; ++c) {
        float v[8];
        tmem_ld8(lane_base + (uint32_t)(kMlpHidden + base + 8 * c), v);
        if (r < a.rows) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = base + 8 * c + j;
                if (n < Q) a.logits[r * Q + n] = v[j] + a.b3[n < Q ? n : 0];
            }
        }
    }
}

// 256 threads: warps w and w + 4 own the rows of TMEM lane quadrant w % 4 and split each row's
// hidden units (and logits) in halves.
template <int Q>
__global__ void __launch_bounds__(256, 1) mlp_tc_kernel(const __grid_constant__ MlpTcArgs<Q> a)
{
    constexpr int Qp = (Q + 15) / 16 * 16;
    constexpr int HALF = kMlpHidden / 2;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quad = warp & 3, half = warp >> 2;
    const int row_l = 32 * quad + lane;            // row of the tile (TMEM lane)
    unsigned char *sW2 = smem;
    unsigned char *sW3 = smem + kW2Bytes;
    unsigned char *sH = sW3 + (uint32_t)Qp * 512u;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sH + kHBytes);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    const uint32_t bar_ld = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tslot)),
                     "r"(kMlpTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    // W2 and W3 images: one bulk copy per CTA
    const uint32_t wbytes = kW2Bytes + (uint32_t)Qp * 512u;
    if (tid == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_ld),
                     "r"(wbytes)
                     : "memory");
        const uint32_t chunk = 1u << 15;
        for (uint32_t off = 0; off < wbytes; off += chunk) {
            const uint32_t n = wbytes - off < chunk ? wbytes - off : chunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                "%2, [%3];" ::"r"(smem_u32(sW2) + off),
                "l"(a.ops + off), "r"(n), "r"(bar_ld)
                : "memory");
        }
    }
    bool alive = !__syncthreads_or(!mbar_wait(bar_ld, 0));
    if (!alive && tid == 0) set_status(a.status, kStatusTimeout);

    const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMlpHidden >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);
    const uint32_t idesc3 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Qp >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);
    const uint32_t sa = smem_u32(sH), sb2 = smem_u32(sW2), sb3 = smem_u32(sW3);
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);
    unsigned char *hrow = sH + core_off(row_l, HALF * half);
    uint32_t phase = 0;
    const long long ntiles = (a.rows + 127) / 128;

    float x[kMlpIn];
    {
        const long long r0 = (long long)blockIdx.x * 128 + row_l;
#pragma unroll
        for (int j = 0; j < kMlpIn; ++j) x[j] = r0 < a.rows ? a.X[r0 * kMlpIn + j] : 0.f;
    }
    for (long long tile = blockIdx.x; tile < ntiles && alive; tile += gridDim.x) {
        const long long r = tile * 128 + row_l;
        // layer 1 on the CUDA cores (this thread's half of the hidden units) -> BF16 A operand
        if (half == 0) mlp_layer1<Q, 0>(a, x, hrow);
        else mlp_layer1<Q, 1>(a, x, hrow);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) mlp_issue(tmem, sa, sb2, idesc2, bar_mma);
        {   // the next tile's features, loaded while the MMAs run
            const long long rn = (tile + gridDim.x) * 128 + row_l;
#pragma unroll
            for (int j = 0; j < kMlpIn; ++j) x[j] = rn < a.rows ? a.X[rn * kMlpIn + j] : 0.f;
        }
        bool ok = mbar_wait(bar_mma, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            alive = false;
            if (tid == 0) set_status(a.status, kStatusTimeout);
            break;
        }
        // layer 2 epilogue (this thread's half of the columns): + b2, ReLU, BF16 -> A operand
        if (half == 0) mlp_epilogue2<Q, 0>(a, lane_base, hrow);
        else mlp_epilogue2<Q, 1>(a, lane_base, hrow);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) mlp_issue(tmem + kMlpHidden, sa, sb3, idesc3, bar_mma);
        ok = mbar_wait(bar_mma, phase);
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (__syncthreads_or(!ok)) {
            alive = false;
            if (tid == 0) set_status(a.status, kStatusTimeout);
            break;
        }
        // layer 3 epilogue: + b3 -> logits (this thread's half of the Qp columns)
        if (half == 0) mlp_epilogue3<Q, 0>(a, lane_base, r);
        else mlp_epilogue3<Q, 1>(a, lane_base, r);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
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
    const float *h = m->small_host;   // W1, b1 | b2 | b3
    std::memcpy(a.W1, h, sizeof a.W1);
    std::memcpy(a.b1, h + kMlpHidden * kMlpIn, sizeof a.b1);
    std::memcpy(a.b2, h + mlp_off_W2(), sizeof a.b2);
    std::memcpy(a.b3, h + mlp_off_W2() + kMlpHidden, sizeof a.b3);
    mlp_tc_kernel<Q><<<grid, 256, smem, s>>>(a);
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
        const int n = (kMlpHidden + m->Qp) * 32;
        mlp_pack_kernel<<<(n + 255) / 256, 256, 0, s>>>(m->params, m->Q, m->Qp, m->tc_ops);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        m->launches++;
        // the small weights travel in the launch parameters: read them back once
        float *h = m->small_host;
        const long long P = mlp_param_count(m->Q);
        if ((e = cudaMemcpyAsync(h, m->params, 4 * (size_t)mlp_off_W2(), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h + mlp_off_W2(), m->params + mlp_off_b2(), 4 * kMlpHidden,
                                 cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h + mlp_off_W2() + kMlpHidden, m->params + mlp_off_b3(m->Q),
                                 4 * (size_t)(P - mlp_off_b3(m->Q)), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return e;
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
    if ((e = cudaMallocHost(&m->small_host, 4 * (size_t)(kMlpHidden * kMlpIn + 3 * kMlpHidden))) != cudaSuccess)
        return bail(e);
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
    if (m->small_host) cudaFreeHost(m->small_host);
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
