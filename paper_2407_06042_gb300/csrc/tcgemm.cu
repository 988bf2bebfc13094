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
// One CTA per 128 x TN output tile (TMEM lanes x TN FP32 columns, TN = 64 or 128, the wider when
// that still gives every SM two CTAs), two CTAs per SM, warp-specialised: eight loader warps and
// one MMA warp. K runs in stages of 32 through a ring of shared-memory buffers (three for
// TN = 64, two for TN = 128). The loaders hold the next stage's FP32 values in registers: they
// split the ones they hold into BF16 terms, store them as K-major core-matrix images, arrive on
// the buffer's "full" mbarrier and issue the global loads of the stage after. The MMA warp waits
// for "full", one lane issues the stage's twelve MMAs (M = 128, N = TN, K = 16) and commits them
// to the buffer's "empty" mbarrier, which the loaders wait for before they refill it; its last
// commit goes to a "done" mbarrier that the epilogue waits for. So the tensor core works on one
// stage while the loaders prepare the next. Every wait is bounded; one that runs out sets the
// timeout status bit, and the CTA waits (bounded) for its last MMAs, frees its tensor memory and
// returns.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tcgemm.h"

namespace mcmcdet {

namespace {

constexpr int kTM = 128, kTK = 32;
constexpr int kLoaders = 256;                 // warps 0-7 load, split and store; warp 8 issues MMAs
constexpr int kThreads = kLoaders + 32;
constexpr int kMmaWarp = kLoaders / 32;
constexpr int kMinStagesPerSplit = 4;
constexpr uint32_t kSbo = (kTK / 8) * 128;              // 8-row group stride of a stage image
constexpr uint32_t kATerm = kTM * kTK * 2;              // 8 KB per BF16 term
constexpr int kTerms = 3;

template <int TN>
struct Tile {
    static constexpr uint32_t kBTerm = TN * kTK * 2;
    static constexpr uint32_t kStage = kTerms * (kATerm + kBTerm);
    static constexpr int kStages = TN == 64 ? 3 : 2;
    static constexpr uint32_t kBars = kStages * kStage;                   // full[], empty[], done
    static constexpr uint32_t kSmem = kBars + 8 * (2 * kStages + 1) + 8;  // + the TMEM slot
    static constexpr int kBUnits = TN * kTK / 8 / kLoaders;
    static_assert(8 * 32 * 33 * 4 <= kBars, "epilogue tiles reuse the stage buffers");
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t img_off(int r, int kg) { return (uint32_t)(r >> 3) * kSbo + (uint32_t)kg * 128u + (uint32_t)(r & 7) * 16u; }

// 8 FP32 values -> three 16-byte BF16 rows (terms 0, 1, 2) of a core matrix. Pairs are rounded
// with the packed conversion (one instruction per two values) and unpacked by shifts.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 (&t)[kTerms])
{
    uint32_t w[kTerms][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float r0 = v[2 * j], r1 = v[2 * j + 1];
#pragma unroll
        for (int q = 0; q < kTerms; ++q) {
            const __nv_bfloat162 b = __floats2bfloat162_rn(r0, r1);   // .x = r0 (low half)
            const uint32_t u = *reinterpret_cast<const uint32_t *>(&b);
            w[q][j] = u;
            if (q + 1 < kTerms) {
                r0 -= __uint_as_float(u << 16);
                r1 -= __uint_as_float(u & 0xffff0000u);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kTerms; ++q) t[q] = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

// Image row r and k group kg (8 consecutive k) of unit u of a stage. When the operand is
// contiguous along k (kfast), a warp takes 8 rows x the 4 k groups, the 8 threads of each
// quarter-warp one k group of the 8 rows: every row's 128 bytes of the stage are read whole,
// and a quarter-warp's 16-byte stores fill one 128-byte run of the core-matrix image (all 32
// banks once). Otherwise consecutive units take consecutive rows of one k group, which is both
// the coalesced read (the operand is contiguous along the rows) and a conflict-free store.
template <int R>
__device__ __forceinline__ void unit_of(int u, bool kfast, int &r, int &kg)
{
    if (kfast) {
        r = ((u >> 5) << 3) | (u & 7);
        kg = (u >> 3) & 3;
    } else {
        r = u & (R - 1);
        kg = u / R;
    }
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
        int r, kg;
        unit_of<R>(tid + kLoaders * i, kfast, r, kg);
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
        int r, kg;
        unit_of<R>(tid + kLoaders * i, kfast, r, kg);
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
    constexpr int NB = T::kStages;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bars = smem_u32(smem + T::kBars);
    uint32_t *slot = reinterpret_cast<uint32_t *>(smem + T::kBars + 8 * (2 * NB + 1));
    const uint32_t done = bars + 16u * NB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * g.kchunk, ke = min(g.K, kb + g.kchunk);
    const int nst = (ke - kb + kTK - 1) / kTK;
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) {
            mbar_init(bars + 8u * b, kLoaders);        // full[b]: every loader thread arrives
            mbar_init(bars + 8u * (NB + b), 1);        // empty[b]: the MMA commit
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot;
    bool ok = true;

    if (warp < kMmaWarp) {
        // loaders
        const bool a_kfast = g.sak == 1, b_kfast = g.sbk == 1;
        float va[2][8], vb[T::kBUnits][8];
        if (nst > 0) {
            load_units<kTM, 2>(g.A, g.sam, g.sak, a_kfast, g.a_vec, g.M, m0, kb, ke, tid, va);
            load_units<TN, T::kBUnits>(g.B, g.sbn, g.sbk, b_kfast, g.b_vec, g.N, n0, kb, ke, tid, vb);
        }
        for (int s = 0; s < nst; ++s) {
            const int b = s % NB;
            // the MMAs of stage s - NB read this buffer: wait for their commit
            if (s >= NB && !mbar_wait(bars + 8u * (NB + b), (uint32_t)(s / NB - 1) & 1u)) {
                ok = false;
                break;
            }
            unsigned char *base = smem + (uint32_t)b * T::kStage;
            store_units<kTM, 2>(base, kATerm, a_kfast, tid, va);
            store_units<TN, T::kBUnits>(base + kTerms * kATerm, T::kBTerm, b_kfast, tid, vb);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(bars + 8u * b);
            if (s + 1 < nst) {
                const int k1 = kb + (s + 1) * kTK;
                load_units<kTM, 2>(g.A, g.sam, g.sak, a_kfast, g.a_vec, g.M, m0, k1, ke, tid, va);
                load_units<TN, T::kBUnits>(g.B, g.sbn, g.sbk, b_kfast, g.b_vec, g.N, n0, k1, ke, tid, vb);
            }
        }
    } else {
        // MMA warp: lane 0 waits and issues, the verdict is shared with the warp
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                               ((uint32_t)(kTM >> 4) << 24);
        for (int s = 0; s < nst; ++s) {
            const int b = s % NB;
            const bool got = __shfl_sync(0xffffffffu, lane == 0 ? mbar_wait(bars + 8u * b, (uint32_t)(s / NB) & 1u) : false, 0);
            if (!got) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (lane == 0) {
                const uint32_t a0 = smem_u32(smem + (uint32_t)b * T::kStage), b0 = a0 + kTerms * kATerm;
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
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 bars + 8u * (NB + b))
                             : "memory");
            }
            __syncwarp();
        }
        // completes once every MMA issued above has (at once when there were none)
        if (lane == 0)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(done)
                         : "memory");
        __syncwarp();
    }
    // no thread leaves (nor frees the tensor memory) while an MMA still runs
    if (!mbar_wait(done, 0u)) ok = false;
    if (!ok && tid == 0) set_status(g.status, kStatusTimeout);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_or(!ok) == 0 && warp < kMmaWarp) {
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
                // 16 rows at a time: their mask values are loaded together (16 loads in flight)
#pragma unroll 1
                for (int h = 0; h < 32; h += 16) {
                    float mk[16];
                    if (masked) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int m = m0 + 32 * q + h + i;
                            mk[i] = m < g.M ? __ldg(&g.mask[(long long)m * g.ldm + n]) : 0.f;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int m = m0 + 32 * q + h + i;
                        if (m < g.M) {
                            float x = tile[(h + i) * 33 + lane];
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
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
}

// Sum of the split-K partials with the epilogue: CTA x takes 32 consecutive outputs, its eight
// warps the splits z = w, w + 8, ... each, and warp 0 adds the eight sums in warp order (the same
// order on every run).
__global__ void __launch_bounds__(256) tc_gemm_reduce_kernel(const TcGemmArgs g, int splits)
{
    __shared__ float red[8][33];
    const long long MN = (long long)g.M * g.N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long e = (long long)blockIdx.x * 32 + lane;
    float s0 = 0.f, s1 = 0.f;
    if (e < MN) {
        int z = w;
        for (; z + 8 < splits; z += 16) {
            s0 += g.partial[z * MN + e];
            s1 += g.partial[(z + 8) * MN + e];
        }
        if (z < splits) s0 += g.partial[z * MN + e];
    }
    red[w][lane] = s0 + s1;
    __syncthreads();
    if (w == 0 && e < MN) {
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) s += red[q][lane];
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
    // split count for a tile width: enough CTAs to fill the GPU (two per SM), each split at least
    // kMinStagesPerSplit stages deep, within the partial buffer
    auto split_count = [&](int tn) {
        const int tiles = tm * ((g.N + tn - 1) / tn);
        if (!partial || g.K <= kMinStagesPerSplit * kTK) return 1;
        const int want = (2 * sms + tiles - 1) / tiles;
        const int kmax = (g.K + kMinStagesPerSplit * kTK - 1) / (kMinStagesPerSplit * kTK);
        int sp = std::max(1, std::min(want, kmax));
        while (sp > 1 && (size_t)sp * g.M * g.N > partial_floats) --sp;
        return sp;
    };
    // the wider tile when it is at least half used and still gives every SM two CTAs
    const int tn = 128 < 2 * g.N && (long long)tm * ((g.N + 127) / 128) * split_count(128) >= 2 * sms ? 128 : 64;
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
    tc_gemm_reduce_kernel<<<(unsigned)((MN + 31) / 32), 256, 0, s>>>(g, splits);
    return cudaGetLastError();
}

}  // namespace mcmcdet
