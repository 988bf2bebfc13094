// tcgemm.cu -- FP32 matrix products on tcgen05 tensor cores, for the learned proposal's network
// training (forward hidden layer, backward input and weight gradients):
//     C(m, n) = sum_k A(m, k) B(k, n),  A(m, k) = A[m sam + k sak],  B(k, n) = B[k sbk + n sbn],
// with an epilogue (+ bias(n), ReLU, or times [mask(m, n) > 0]) or, for a split K range, raw
// partial sums that a second kernel adds in split order.
//
// Each FP32 operand is split into three BF16 terms, x = x0 + x1 + x2 with x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (the two differences are exact in FP32, and the
// remainder is below 2^-26 |x|), and the product is accumulated in FP32 in tensor memory as the
// six term products a_i b_j with i + j <= 2 (the dropped ones are below 2^-26 |a b|), so that
// the result is as accurate as an FP32 product: the ReLU masks of the backward pass then agree
// with an FP32 evaluation except where FP32 itself is too coarse to decide them.
//
// One CTA of 256 threads per 128 x TN output tile (TMEM lanes x TN FP32 columns, TN = 64 or
// 128, the wider when that still gives every SM work), two CTAs per SM. K runs in stages of 32
// through two shared-memory buffers. The threads hold the next stage's FP32 values in registers:
// they split the ones they hold into BF16 terms and store them as K-major core-matrix images,
// then issue the global loads of the stage after, whose latency the MMAs of this stage and the
// wait for the buffer cover. Thread 0 issues a stage's twelve MMAs (M = 128, N = TN, K = 16)
// and commits them to the buffer's mbarrier, which the threads wait for before they refill that
// buffer two stages later. Every wait is bounded; one that runs out sets the timeout status
// bit, and the CTA waits (bounded) for its last MMAs, frees its tensor memory and returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tcgemm.h"

namespace mcmcdet {

namespace {

constexpr int kTM = 128, kTK = 32, kThreads = 256;
constexpr int kMinStagesPerSplit = 4;
constexpr uint32_t kSbo = (kTK / 8) * 128;              // 8-row group stride of a stage image
constexpr uint32_t kATerm = kTM * kTK * 2;              // 8 KB per BF16 term
constexpr int kTerms = 3;

template <int TN>
struct Tile {
    static constexpr uint32_t kBTerm = TN * kTK * 2;
    static constexpr uint32_t kStage = kTerms * (kATerm + kBTerm);
    static constexpr uint32_t kSmem = 2 * kStage + 64;  // two stages, barriers, TMEM slot
    static constexpr int kBUnits = TN * kTK / 8 / kThreads;
};

__device__ __forceinline__ uint32_t img_off(int r, int kg) { return (uint32_t)(r >> 3) * kSbo + (uint32_t)kg * 128u + (uint32_t)(r & 7) * 16u; }

// 8 FP32 values -> three 16-byte BF16 rows (terms 0, 1, 2) of a core matrix.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&t)[kTerms])
{
    uint32_t w[kTerms][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float r0 = v[2 * j], r1 = v[2 * j + 1];
#pragma unroll
        for (int q = 0; q < kTerms; ++q) {
            const __nv_bfloat16 b0 = __float2bfloat16_rn(r0), b1 = __float2bfloat16_rn(r1);
            r0 -= __bfloat162float(b0);
            r1 -= __bfloat162float(b1);
            w[q][j] = (uint32_t)__bfloat16_as_ushort(b0) | ((uint32_t)__bfloat16_as_ushort(b1) << 16);
        }
    }
#pragma unroll
    for (int q = 0; q < kTerms; ++q) t[q] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// One operand's share of a stage: R image rows x kTK, in units of 8 consecutive k (U per
// thread). P(row, k) = P[row sr + k sk]; units run along k first when sk == 1 (kfast), else
// along the rows, so that a warp's loads are coalesced either way. vec: 16-byte loads are
// aligned (kfast, P and sr multiples of 16 bytes).
template <int R, int U>
__device__ __forceinline__ void load_units(const float *P, long long sr, long long sk, bool kfast, bool vec,
                                           int rows, int r0, int k0, int ke, int tid, float (&v)[U][8])
{
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int u = tid + kThreads * i;
        const int r = kfast ? u >> 2 : u & (R - 1), kg = kfast ? u & 3 : u / R;
        const int row = r0 + r, k = k0 + 8 * kg;
        if (row < rows && vec && k + 8 <= ke) {
            const float4 *p = reinterpret_cast<const float4 *>(P + (long long)row * sr + k);
            const float4 x = __ldg(p), y = __ldg(p + 1);
            v[i][0] = x.x; v[i][1] = x.y; v[i][2] = x.z; v[i][3] = x.w;
            v[i][4] = y.x; v[i][5] = y.y; v[i][6] = y.z; v[i][7] = y.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                v[i][j] = (row < rows && k + j < ke) ? __ldg(P + (long long)row * sr + (long long)(k + j) * sk) : 0.f;
        }
    }
}

template <int R, int U>
__device__ __forceinline__ void store_units(unsigned char *img, uint32_t term, bool kfast, int tid,
                                            const float (&v)[U][8])
{
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int u = tid + kThreads * i;
        const int r = kfast ? u >> 2 : u & (R - 1), kg = kfast ? u & 3 : u / R;
        uint4 t[kTerms];
        split8(v[i], t);
#pragma unroll
        for (int q = 0; q < kTerms; ++q) *reinterpret_cast<uint4 *>(img + q * term + img_off(r, kg)) = t[q];
    }
}

template <int TN>
__global__ void __launch_bounds__(kThreads, 2) tc_gemm_kernel(const TcGemmArgs g)
{
    using T = Tile<TN>;
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + 2 * T::kStage);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + 2 * T::kStage + 32);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
    const int nst = (ke - kb + kTK - 1) / kTK;
    const uint32_t bar[2] = {smem_u32(&bars[0]), smem_u32(&bars[1])};
    if (tid == 0) {
        mbar_init(bar[0], 1);
        mbar_init(bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                           ((uint32_t)(kTM >> 4) << 24);
    const bool a_kfast = g.sak == 1, b_kfast = g.sbk == 1;
    bool ok = true;
    uint32_t uses0 = 0u, uses1 = 0u;   // completed commits awaited per buffer
    int issued = -1;               // last stage whose MMAs were issued and committed

    float va[2][8], vb[T::kBUnits][8];
    if (nst > 0) {
        load_units<kTM, 2>(g.A, g.sam, g.sak, a_kfast, g.a_vec, g.M, m0, kb, ke, tid, va);
        load_units<TN, T::kBUnits>(g.B, g.sbn, g.sbk, b_kfast, g.b_vec, g.N, n0, kb, ke, tid, vb);
    }
    for (int s = 0; s < nst; ++s) {
        const int buf = s & 1;
        unsigned char *base = smem + (uint32_t)buf * T::kStage;
        // the MMAs of stage s - 2 read this buffer: wait for their commit
        const uint32_t bb = buf ? bar[1] : bar[0];
        bool free_ok = true;
        if (s >= 2) {
            uint32_t &u = buf ? uses1 : uses0;
            free_ok = mbar_wait(bb, u & 1u);
            ++u;
        }
        store_units<kTM, 2>(base, kATerm, a_kfast, tid, va);
        store_units<TN, T::kBUnits>(base + kTerms * kATerm, T::kBTerm, b_kfast, tid, vb);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!free_ok)) { ok = false; break; }
        if (s + 1 < nst) {
            const int k1 = kb + (s + 1) * kTK;
            load_units<kTM, 2>(g.A, g.sam, g.sak, a_kfast, g.a_vec, g.M, m0, k1, ke, tid, va);
            load_units<TN, T::kBUnits>(g.B, g.sbn, g.sbk, b_kfast, g.b_vec, g.N, n0, k1, ke, tid, vb);
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(base), b0 = a0 + kTerms * kATerm;
            // (A term, B term) with term indices summing to at most 2, smallest first
            constexpr int ai[6] = {1, 0, 2, 1, 0, 0}, bi[6] = {1, 2, 0, 0, 1, 0};
#pragma unroll
            for (int ks = 0; ks < kTK / 16; ++ks)
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t da = smem_desc(a0 + ai[p] * kATerm + (uint32_t)ks * 256u, 128u, kSbo);
                    const uint64_t db = smem_desc(b0 + bi[p] * T::kBTerm + (uint32_t)ks * 256u, 128u, kSbo);
                    mma_bf16(tmem, da, db, idesc, (s | ks | p) ? 1u : 0u);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bb)
                         : "memory");
        }
        issued = s;
    }
    // the last commit covers every MMA issued before it: wait for it (also after a timeout, so
    // that no MMA still writes the tensor memory freed below)
    if (issued >= 0) {
        const bool lb = issued & 1;
        if (!mbar_wait(lb ? bar[1] : bar[0], (lb ? uses1 : uses0) & 1u)) ok = false;
    }
    if (!ok && tid == 0) set_status(g.status, kStatusTimeout);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(!ok) == 0) {
        // epilogue: warp w reads lane quadrant w % 4 (rows) and column half w / 4, 32 x 32 at a
        // time (thread = row), and turns each block around in shared memory (the stage buffers
        // are idle now) so that its global loads and stores run along rows (thread = column)
        const int q = warp & 3, hc = warp >> 2;
        float *tile = reinterpret_cast<float *>(smem) + warp * (32 * 33);
        const bool masked = g.mask && !g.partial;
#pragma unroll 1
        for (int c = 0; c < TN / 64; ++c) {
            const int cb = (TN / 2) * hc + 32 * c;
            const int n = n0 + cb + lane;
            // the mask rows first: 32 loads in flight per lane while the accumulators are read
            float mk[32];
            if (masked) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int m = m0 + 32 * q + i;
                    mk[i] = m < g.M && n < g.N ? __ldg(&g.mask[(long long)m * g.ldm + n]) : 0.f;
                }
            }
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)cb;
            uint32_t r[32];
            if (nst > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                    "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                      "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                      "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) r[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            if (n < g.N) {
                const float bias = g.bias && !g.partial ? g.bias[n] : 0.f;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int m = m0 + 32 * q + i;
                    if (m < g.M) {
                        float x = tile[i * 33 + lane];
                        if (g.partial) {
                            g.partial[((long long)blockIdx.z * g.M + m) * g.N + n] = x;
                        } else {
                            x += bias;
                            if (g.relu) x = fmaxf(x, 0.f);
                            if (masked && !(mk[i] > 0.f)) x = 0.f;
                            g.C[(long long)m * g.ldc + n] = x;
                        }
                    }
                }
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// Sum of the split-K partials in split order, with the epilogue.
__global__ void tc_gemm_reduce_kernel(const TcGemmArgs g, int splits)
{
    const long long MN = (long long)g.M * g.N;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < MN;
         e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += g.partial[z * MN + e];
        const long long m = e / g.N, n = e % g.N;
        if (g.bias) s += g.bias[n];
        if (g.relu) s = fmaxf(s, 0.f);
        if (g.mask && !(g.mask[m * g.ldm + n] > 0.f)) s = 0.f;
        g.C[m * g.ldc + n] = s;
    }
}

template <int TN>
cudaError_t launch_tile(const TcGemmArgs &g, int tm, int splits, cudaStream_t s)
{
    cudaError_t e = allow_max_dyn_smem(tc_gemm_kernel<TN>);
    if (e != cudaSuccess) return e;
    tc_gemm_kernel<TN><<<dim3((g.N + TN - 1) / TN, tm, splits), kThreads, Tile<TN>::kSmem, s>>>(g);
    return cudaGetLastError();
}

bool aligned16(const float *p, long long stride)
{
    return ((uintptr_t)p & 15u) == 0 && (stride & 3) == 0;
}

}  // namespace

cudaError_t tc_gemm(const TcGemmArgs &in, float *partial, size_t partial_floats, int sms, cudaStream_t s,
                    int *launches)
{
    *launches = 0;
    TcGemmArgs g = in;
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    sms = std::max(sms, 1);
    const int tm = (g.M + kTM - 1) / kTM;
    // split count for a tile width: enough CTAs to cover the GPU, each split at least
    // kMinStagesPerSplit stages deep, within the partial buffer
    auto split_count = [&](int tn) {
        const int tiles = tm * ((g.N + tn - 1) / tn);
        if (!partial || g.K <= kMinStagesPerSplit * kTK) return 1;
        const int want = (sms + tiles - 1) / tiles;
        const int kmax = (g.K + kMinStagesPerSplit * kTK - 1) / (kMinStagesPerSplit * kTK);
        int sp = std::max(1, std::min(want, kmax));
        while (sp > 1 && (size_t)sp * g.M * g.N > partial_floats) --sp;
        return sp;
    };
    // the wider tile when it is at least half used and still gives every SM a CTA
    const int tn = 128 < 2 * g.N && (long long)tm * ((g.N + 127) / 128) * split_count(128) >= sms ? 128 : 64;
    int splits = split_count(tn);
    g.kchunk = std::max(kTK, ((g.K + splits - 1) / splits + kTK - 1) / kTK * kTK);
    splits = std::max(1, (g.K + g.kchunk - 1) / g.kchunk);
    g.partial = splits > 1 ? partial : nullptr;
    g.a_vec = g.sak == 1 && aligned16(g.A, g.sam);
    g.b_vec = g.sbk == 1 && aligned16(g.B, g.sbn);
    cudaError_t e = tn == 128 ? launch_tile<128>(g, tm, splits, s) : launch_tile<64>(g, tm, splits, s);
    *launches = 1;
    if (e != cudaSuccess || splits == 1) return e;
    const long long MN = (long long)g.M * g.N;
    *launches = 2;
    tc_gemm_reduce_kernel<<<(int)std::min<long long>((MN + 255) / 256, 4096), 256, 0, s>>>(g, splits);
    return cudaGetLastError();
}

}  // namespace mcmcdet
