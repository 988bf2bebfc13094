// chains_tc.cu -- DMALA chain kernel with the Gram products on tcgen05 tensor cores (MIXED).
//
// Each CTA owns a group of C chains of one channel (persistent over work items). Per transition
// (Algorithm 1's loop body):
//   1. every thread draws x'_n for its (dimension, 4 chains) from the proposal factors of the
//      current state (Eqs. (15)-(17) / (21)), two chains per packed f32x2 instruction, and writes
//      x' as BF16 (exact odd integers) into the shared-memory B operand [C chains x K]. The
//      factors are carried from transition to transition in tensor memory (Algorithm 1 keeps
//      q(.|x) while x stays); a warp rebuilds its tables from the drift slopes only after one of
//      its chains moved;
//   2. one thread issues D = A * X'^T on the tensor core: A = [Gt | P~ Gt] rows (split into
//      `split_terms` BF16 terms, FP32 accumulation in TMEM); completion is signalled through an
//      mbarrier, and the chains' acceptance uniforms are drawn meanwhile. For N <= 128 the A
//      operand is staged once per work item by a bulk copy. Beyond, a thread-block cluster
//      keeps one 128-row tile resident per CTA (see the cluster section below), or, as a
//      fallback, one CTA streams the operand from L2 in 128-row chunks through two buffers
//      (full / empty mbarriers) every transition;
//   3. every thread reads its TMEM lane (one row of A = one dimension of Gt or P~Gt) for its
//      8 columns (chains), swaps halves with its partner lane, and evaluates the reverse factor
//      and the energy difference (Eqs. (3), (18));
//   4. per chain the log acceptance ratio is reduced over dimensions (warp shuffles, then the
//      four TMEM lane quadrants through shared memory) and the MH test is taken;
//   5. accepted chains keep x', Gt x' and the drift slope of x'.
// A-operand row layout (128 rows per tile t): row 32q + l holds dimension 64t + 16q + (l & 15) of
// Gt (l < 16) or of P~ Gt (l >= 16), so each warp's TMEM quadrant carries both quantities of
// 16 dimensions; each thread owns one dimension of 4 chains per tile. Channels of N <= 32 hold
// their rows twice (quadrants 0-1 and 2-3: dimension 16 (q mod 2) + (l & 15)), and each copy
// serves its own group of chains, so a CTA runs twice the chains with the same threads. Both
// operands are K-major, no swizzle, in 8 x 16-byte core matrices. A: K-adjacent core matrices
// 128 B apart (LBO), 8-row groups (K/8)*128 B apart (SBO). B: 144 B and a stride 32 B past a
// multiple of 128 B (b_lbo, b_sbo), which keeps the threads' 16-bit stores free of bank conflicts.
// Every wait is bounded: a wait that runs out sets the timeout status bit, the CTA stops issuing
// work, waits (bounded) for its copies in flight, frees its TMEM and returns (in a cluster, after
// the exit barrier that keeps every CTA's shared memory alive for the others' stores).
//
// The in-run FP64 refreshes (refresh_period > 0) normally run between launches (the refresh
// kernel); the kernels here carry none of that code. chains_tc_kr.cu compiles this file a second
// time with MCMC_TC_IN_KERNEL_REFRESH = 1: the same kernels with the refresh inside, launched by
// tc_launch_chains_kr (MCMC_ENGINE_KERNEL_REFRESH), and none of the host-side planning.
#include "tc_plan.h"

#include <cuda_bf16.h>

#include "proposal.cuh"
#include "tc_ptx.cuh"

#ifndef MCMC_TC_IN_KERNEL_REFRESH
#define MCMC_TC_IN_KERNEL_REFRESH 0
#endif

namespace mcmcdet {

namespace {

constexpr bool kInKernelRefresh = MCMC_TC_IN_KERNEL_REFRESH != 0;

// Launch bounds of the one-tile kernel: at most TC_MAX_THREADS threads per CTA (16 per chain),
// registers sized for TC_MIN_BLOCKS such CTAs per SM.
#ifndef TC_MAX_THREADS
#define TC_MAX_THREADS 512
#endif
#ifndef TC_MIN_BLOCKS
#define TC_MIN_BLOCKS 2
#endif

// 4 values per lane, summed over the 16 lanes of a half warp and scattered: afterwards lanes
// 4j .. 4j+3 of the half hold the sum of value j.
__device__ __forceinline__ float reduce_scatter16(const float (&v)[4], int dl)
{
    float a[2];
    const bool hi8 = dl & 8, hi4 = dl & 4;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = hi8 ? v[i] : v[2 + i];
        const float recv = __shfl_xor_sync(0xffffffffu, send, 8);
        a[i] = (hi8 ? v[2 + i] : v[i]) + recv;
    }
    const float send = hi4 ? a[0] : a[1];
    const float recv = __shfl_xor_sync(0xffffffffu, send, 4);
    float c = (hi4 ? a[1] : a[0]) + recv;
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

// Shared-memory layout of the kernel (bytes).
struct TcLayout {
    uint32_t a, b, red, dred, acc, ref, fst, cnt, tie, fref, kb, dg, xs, dsc, bar, tmem, total;
};

// The A operand of a single CTA stays resident for MT <= 2 (N <= 128). Beyond that it no longer
// fits one SM's shared memory: the cluster kernels (instantiated with MT = 1 per CTA) keep one
// tile per CTA, and the single-CTA fallback streams it from L2 in 128-row x Kp chunks through
// two buffers.
__host__ __device__ constexpr bool tc_streamed(int MT) { return MT >= 3; }

// Row stride (bytes) of the per-chain state copies in shared memory (best visited state, the
// states of an FP64 refresh): the CTA's dimensions, 64 per tile (a cluster CTA: its own 64).
__host__ __device__ constexpr int tc_state_stride(int MT, int CL) { return CL > 1 ? 64 : 64 * MT; }

// Chain groups per CTA: channels of N <= 32 use half of the 64 dimension rows of a tile, so the
// tile holds their rows twice and each copy serves its own group of chains.
__host__ __device__ inline int tc_groups(int N) { return (N + 15) / 16 * 16 <= 32 ? 2 : 1; }

// CL > 1: one CTA of a CL-CTA cluster (MT = 1 local tile, Kp the whole channel's K extent).
__host__ __device__ inline TcLayout tc_layout(int S, int MT, int Kp, int C, int CL = 1)
{
    TcLayout L{};
    uint32_t o = 0;
    auto take = [&](uint32_t bytes, uint32_t al) {
        o = (o + al - 1) / al * al;
        const uint32_t r = o;
        o += bytes;
        return r;
    };
    L.a = take((uint32_t)(tc_streamed(MT) ? 2 : S * MT) * 128 * Kp * 2, 1024);
    L.b = take((uint32_t)(C / 8) * (((uint32_t)(Kp / 8) * 144u + 127u) / 128u * 128u + 32u), 1024);
    L.red = take(4u * C * 4, 16);
    L.dred = take(4u * C * 4, 16);
    L.acc = take((uint32_t)C * 4, 16);
    L.ref = take((uint32_t)C * 16, 16);      // FP64 refresh results per chain
    L.fst = take((uint32_t)C * 16, 16);      // tracked and best energies per chain
    L.cnt = take((uint32_t)C * 4, 16);       // accepted moves per chain
    L.tie = take((uint32_t)C * 12, 16);      // near-tie counts per chain slot, three windows
    // states for the FP64 refresh (a cluster CTA reads them from its B operand instead) and the
    // best visited state of every chain (a cluster CTA: its own 64 dimensions)
    L.fref = take(CL > 1 ? 0u : (uint32_t)C * tc_state_stride(MT, CL), 16);
    L.kb = take((uint32_t)C * tc_state_stride(MT, CL), 16);
    // streamed kernels: Gt x of every thread's (tile, chain pair), [2 MT][threads] packed pairs
    L.dg = take(tc_streamed(MT) ? (uint32_t)(2 * MT) * (16u * C) * 8u : 0u, 16);
    // cluster exchange slots: [2 alternating buffers][CL ranks][C chains] x 16 bytes
    L.xs = take(CL > 1 ? 2u * (uint32_t)CL * (uint32_t)C * 16u : 0u, 16);
    // MMA descriptor pairs of a transition (resident operand: split terms x tiles x K steps)
    L.dsc = take(tc_streamed(MT) ? 0u : (uint32_t)(S * MT * (Kp / 16)) * 16u, 16);
    // TMA, MMA, streamed chunks full[2] / empty[2], cluster B slices and exchange
    L.bar = take(8 * 8, 8);
    L.tmem = take(8, 4);                     // TMEM base address, work-queue item (packed kernel)
    L.total = (o + 127) / 128 * 128;
    return L;
}

// B operand (x', [C chains x Kp]) core-matrix strides: K-adjacent core matrices 144 B apart and
// 8-chain groups at a stride that is 32 B past a multiple of 128 B, so that the 16-bit stores of
// a warp (16 dimensions x 2 chain groups) fall into distinct shared-memory banks.
__host__ __device__ inline uint32_t b_lbo() { return 144u; }
__host__ __device__ inline uint32_t b_sbo(int Kp)
{
    return ((uint32_t)(Kp / 8) * 144u + 127u) / 128u * 128u + 32u;
}

struct TcCtx {
    unsigned char *sA, *sB;
    float *red, *dred;
    int *sacc;
    double *sref;
    double *sfc, *sfb;            // tracked and best energies of the CTA's chains
    unsigned *scnt;
    unsigned *stie;               // [3][C] near-tie counts of the CTA's chain slots (all items)
    int8_t *sfs;
    int8_t *skb;
    uint64_t *sdg;                // Gt x pairs in shared memory (streamed kernels)
    uint4 *sdsc;                  // (A, B) descriptor pairs of a transition's MMAs, in issue order
                                  // (resident operand; written by thread 0 for each work item)
    int nthr;
    uint32_t bar_mma;
    uint32_t tmem;
    uint32_t idesc;
    uint32_t sbo_a, sbo_b;
    int tid, warp, lane, q, cgi, h, dl, C, S, Kp;
    // chain groups: with N <= 32 the four TMEM lane quadrants hold two copies of the operand rows
    // (quadrants 0-1 and 2-3), and each copy serves its own C / 2 chains
    int gofs;                     // first chain of this thread's group
    uint32_t mma_phase;
    // streamed A operand (thread 0's pipeline state)
    const uint8_t *asrc;          // this work item's operand block in global memory
    uint32_t bar_full[2], bar_empty[2];
    uint32_t full_phase[2], empty_phase[2];
    bool pend[2];                 // a chunk copy into buffer b is requested and not yet waited for
    bool fail;                    // a streamed wait (or a cluster B-slice wait) ran out
    // cluster kernels: this CTA's rank (its 128-row tile and 64 dimensions), the barrier that
    // counts the other CTAs' slices of the B operand, the one that counts exchange arrivals,
    // their phases, and the exchange slots (two alternating buffers)
    int rank;
    uint32_t bar_b, bar_x, b_phase, x_phase, x_buf;
    unsigned char *sx;
    uint32_t bar_tma, tma_phase;  // the per-work-item operand copy (and its reload after a refresh)
};

// ------------------------------------------------------------------------------------------
// Thread-block clusters (N > 128): CTA r of a cluster of CL keeps tile r of the A operand
// resident and owns dimensions 64r .. 64r + 63 of every chain of the work item. Per transition
//   - each CTA writes its part of x' into its own B operand and sends that slice (its K groups,
//     for every 8-chain group) to the other CTAs by bulk shared::cta -> shared::cluster copies
//     that complete on their B-slice barrier; the MMA waits for the other slices;
//   - per-chain partial sums (log q and energy terms) are exchanged through distributed shared
//     memory: every CTA stores its partials into a slot of every CTA and arrives on that CTA's
//     exchange barrier, so each CTA sums the same values in the same (rank) order and takes the
//     same MH decisions.
// The exchanges alternate with the B-slice transfers (every CTA joins an exchange only after its
// MMA consumed the previous slices), which orders every write into another CTA's shared memory
// after that CTA's last read of the same bytes.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cl_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_count()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(uint32_t addr, int rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Bounded wait with cluster-scope acquire (the exchange barrier's arrivals come from other CTAs).
__device__ __forceinline__ bool mbar_wait_cl(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < kWaitLimit; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// K groups (8 dimensions) of the B operand that CTA r of the cluster writes.
__device__ __forceinline__ int cl_kg0(int r) { return 8 * r; }
__device__ __forceinline__ int cl_kg1(int r, int Kp) { return min(8 * r + 8, Kp / 8); }

// Thread 0: arm this CTA's B-slice barrier for the other CTAs' slices and send this CTA's slice
// (for every 8-chain group: its K groups, contiguous at a 144-byte K stride) to every other CTA.
template <int CL>
__device__ __forceinline__ void cl_send_b(const TcCtx &x)
{
    const uint32_t groups = (uint32_t)x.C / 8u;
    uint32_t expect = 0;
#pragma unroll
    for (int r = 0; r < CL; ++r)
        if (r != x.rank) expect += (uint32_t)(cl_kg1(r, x.Kp) - cl_kg0(r)) * b_lbo() * groups;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(x.bar_b), "r"(expect)
                 : "memory");
    const uint32_t bytes = (uint32_t)(cl_kg1(x.rank, x.Kp) - cl_kg0(x.rank)) * b_lbo();
    const uint32_t base = smem_u32(x.sB) + (uint32_t)cl_kg0(x.rank) * b_lbo();
#pragma unroll
    for (int r = 0; r < CL; ++r) {
        if (r == x.rank) continue;
        const uint32_t bar = cl_map(x.bar_b, r);
        for (uint32_t g = 0; g < groups; ++g) {
            const uint32_t src = base + g * x.sbo_b;
            asm volatile(
                "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], "
                "%2, [%3];" ::"r"(cl_map(src, r)),
                "r"(src), "r"(bytes), "r"(bar)
                : "memory");
        }
    }
}

// Threads 0 .. C-1 (chain c): publish 16 bytes into slot [buffer][this rank][c] of every CTA of
// the cluster and wait (bounded) until every CTA has published. The C threads store into every
// CTA's slots, meet (a warp or named barrier), and then thread r alone releases them to CTA r
// with one cluster-scope fence and one remote arrival: CL arrivals per CTA and exchange instead
// of CL x C release-arrivals. The caller reads the CL slots of chain c with cl_slot() and then
// calls cl_next() (all threads).
template <int CL>
__device__ __forceinline__ bool cl_exchange(const TcCtx &x, int c, uint4 v)
{
    const uint32_t slot =
        smem_u32(x.sx) + (uint32_t)(((x.x_buf * CL + x.rank) * x.C + c) * 16);
#pragma unroll
    for (int r = 0; r < CL; ++r)
        asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(cl_map(slot, r)),
                     "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                     : "memory");
    // every exchanging thread's stores happen before the releases below
    if (x.C <= 32) __syncwarp(x.C == 32 ? 0xffffffffu : (1u << x.C) - 1u);
    else asm volatile("bar.sync 1, %0;" ::"r"(x.C) : "memory");
    if (c < CL) {
        asm volatile("fence.acq_rel.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cl_map(x.bar_x, c))
                     : "memory");
    }
    return mbar_wait_cl(x.bar_x, x.x_phase);
}
__device__ __forceinline__ uint4 cl_slot(const TcCtx &x, int CL, int r, int c)
{
    return reinterpret_cast<const uint4 *>(x.sx)[(x.x_buf * CL + r) * x.C + c];
}
__device__ __forceinline__ void cl_next(TcCtx &x)
{
    x.x_phase ^= 1u;
    x.x_buf ^= 1u;
}

// Issue the MMAs of one transition (thread 0, after a CTA barrier that publishes the B operand)
// and, separately, wait for them (everyone). The wait returns false on a bounded-wait expiry of
// this thread's wait; callers combine the verdicts in a CTA-wide vote.
// Streamed A operand: bulk copy of chunk c (tile c / S, term c % S) into buffer b.
__device__ __forceinline__ void tc_load_chunk(TcCtx &x, int MT, int c, int b)
{
    const uint32_t cb = 128u * (uint32_t)x.Kp * 2u;
    const int t = c / x.S, s = c % x.S;
    const uint8_t *src = x.asrc + (size_t)(s * MT + t) * cb;
    const uint32_t dst = smem_u32(x.sA) + (uint32_t)b * cb;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(x.bar_full[b]), "r"(cb)
                 : "memory");
    x.pend[b] = true;
    const uint32_t chunk = 1u << 15;
    for (uint32_t off = 0; off < cb; off += chunk) {
        const uint32_t n = cb - off < chunk ? cb - off : chunk;
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                dst + off),
            "l"(src + off), "r"(n), "r"(x.bar_full[b])
            : "memory");
    }
}

// Thread 0: MMAs of one transition over the streamed chunks, two buffers deep. Chunk c's buffer
// is refilled with chunk c + 2 once c's MMAs have completed (their commit to empty[b]); the last
// two chunks are covered by the final commit only, so every full / empty phase is waited once.
template <int MT>
__device__ __forceinline__ void tc_stream_mmas(TcCtx &x)
{
    const int nch = x.S * MT;
    const uint32_t cb = 128u * (uint32_t)x.Kp * 2u;
    const uint32_t b0 = smem_u32(x.sB);
    for (int c = 0; c < 2 && c < nch; ++c)
        if (!x.pend[c]) tc_load_chunk(x, MT, c, c);   // else requested at the end of the last one
    for (int c = 0; c < nch && !x.fail; ++c) {
        const int b = c & 1;
        if (!mbar_wait(x.bar_full[b], x.full_phase[b])) { x.fail = true; break; }
        x.full_phase[b] ^= 1u;
        x.pend[b] = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int t = c / x.S, s = c % x.S;
        const uint32_t ab = smem_u32(x.sA) + (uint32_t)b * cb;
        for (int ks = 0; ks < x.Kp / 16; ++ks) {
            const uint64_t da = smem_desc(ab + ks * 256u, 128u, x.sbo_a);
            const uint64_t db = smem_desc(b0 + ks * 2u * b_lbo(), b_lbo(), x.sbo_b);
            mma_bf16(x.tmem + (uint32_t)(t * x.C), da, db, x.idesc, (s | ks) ? 1u : 0u);
        }
        if (c + 2 < nch) {
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    x.bar_empty[b])
                : "memory");
            if (!mbar_wait(x.bar_empty[b], x.empty_phase[b])) { x.fail = true; break; }
            x.empty_phase[b] ^= 1u;
            tc_load_chunk(x, MT, c + 2, b);
        }
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(x.bar_mma)
        : "memory");
}

// Thread 0, after the transition's MMAs completed: request chunks 0 and 1 for the next one (the
// operand is the same every transition of a work item).
template <int MT>
__device__ __forceinline__ void tc_stream_prefetch(TcCtx &x)
{
    if (x.fail) return;
    for (int c = 0; c < 2 && c < x.S * MT; ++c) tc_load_chunk(x, MT, c, c);
}

// Thread 0, at the end of a work item (or after a failed wait): wait (bounded) for every chunk copy
// requested and not yet waited for, so that none is in flight when the buffers are reused or the
// CTA exits. Returns false if a wait ran out.
__device__ __forceinline__ bool tc_stream_drain(TcCtx &x)
{
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        if (!x.pend[b]) continue;
        if (!mbar_wait(x.bar_full[b], x.full_phase[b])) ok = false;
        x.full_phase[b] ^= 1u;
        x.pend[b] = false;
    }
    return ok;
}

// Thread 0, for each work item of a resident-operand kernel: the (A, B) shared-memory descriptors
// of a transition's MMAs (tile t: split terms s, K steps ks, in accumulation order), so that the
// transitions only load and issue them.
template <int MT>
__device__ __forceinline__ void tc_mma_descs(TcCtx &x)
{
    if constexpr (!tc_streamed(MT)) {
        const uint32_t a0 = smem_u32(x.sA), b0 = smem_u32(x.sB);
        const int nk = x.Kp / 16;
        int e = 0;
        for (int t = 0; t < MT; ++t)
            for (int s = 0; s < x.S; ++s) {
                const uint32_t ab = a0 + (uint32_t)((s * MT + t) * 128 * x.Kp * 2);
                for (int ks = 0; ks < nk; ++ks, ++e) {
                    const uint64_t da = smem_desc(ab + ks * 256u, 128u, x.sbo_a);
                    const uint64_t db = smem_desc(b0 + ks * 2u * b_lbo(), b_lbo(), x.sbo_b);
                    x.sdsc[e] = make_uint4((uint32_t)da, (uint32_t)(da >> 32), (uint32_t)db, (uint32_t)(db >> 32));
                }
            }
    }
}

template <int MT, int CL = 1>
__device__ __forceinline__ void tc_gemm_issue(TcCtx &x)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if constexpr (tc_streamed(MT)) {
        if (x.tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_stream_mmas<MT>(x);
        }
        return;
    }
    if (x.tid == 0 || (CL > 1 && x.tid == 32)) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        bool go = true;
        if constexpr (CL > 1) {
            // the other CTAs' slices of x' complete on the B-slice barrier
            if (x.tid == 0) cl_send_b<CL>(x);
            if (!mbar_wait(x.bar_b, x.b_phase)) { x.fail = true; go = false; }
        }
        // the descriptors were laid out for this work item by tc_mma_descs: only the issue is left
        const int nk = x.Kp / 16, per_tile = x.S * nk;
        const uint32_t idesc = x.idesc;
        if constexpr (CL > 1) {
            // a cluster CTA's K = N > 128 is long: two issuers take the first and the second half
            // of the K steps into two accumulator blocks (the second 7 C columns further, past
            // the carried tables), which the reads add, so the two dependent MMA chains run side
            // by side in the tensor pipe
            const int h = (nk + 1) / 2, k0 = x.tid == 0 ? 0 : h, k1 = x.tid == 0 ? h : nk;
            const uint32_t d = x.tmem + (x.tid == 0 ? 0u : 7u * (uint32_t)x.C);
            bool first = true;
            for (int sterm = 0; sterm < x.S && go; ++sterm)
                for (int ks = k0; ks < k1; ++ks) {
                    const uint4 v = x.sdsc[sterm * nk + ks];
                    mma_bf16(d, ((uint64_t)v.y << 32) | v.x, ((uint64_t)v.w << 32) | v.z, idesc, first ? 0u : 1u);
                    first = false;
                }
        } else {
            for (int t = 0; t < MT && go; ++t) {
                const uint32_t d = x.tmem + (uint32_t)(t * x.C);
                const uint4 *dl = x.sdsc + t * per_tile;
#pragma unroll 4
                for (int e = 0; e < per_tile; ++e) {
                    const uint4 v = dl[e];
                    mma_bf16(d, ((uint64_t)v.y << 32) | v.x, ((uint64_t)v.w << 32) | v.z, idesc, e ? 1u : 0u);
                }
            }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                x.bar_mma)
            : "memory");
    }
    if constexpr (CL > 1) x.b_phase ^= 1u;   // every thread tracks the B-slice phase
}

// prefetch_next: another transition of the same work item follows (streamed operand only).
// In a cluster, thread 0's verdict includes its wait for the other CTAs' B slices.
template <int MT, int CL = 1>
__device__ __forceinline__ bool tc_gemm_wait(TcCtx &x, bool prefetch_next)
{
    const bool ok = mbar_wait(x.bar_mma, x.mma_phase);
    x.mma_phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if constexpr (CL > 1) return ok && !((x.tid == 0 || x.tid == 32) && x.fail);
    if constexpr (tc_streamed(MT)) {
        if (x.tid == 0) {
            if (ok && prefetch_next) tc_stream_prefetch<MT>(x);
            return ok && !x.fail;
        }
    }
    return ok;
}

// TMEM -> registers: Gt x (g) and P~ Gt x (m) of this thread's dimension for its 8 chains
// (a cluster CTA adds its second accumulator block, 7 C columns further).
template <int MT, int CL = 1>
__device__ __forceinline__ void tc_read(const TcCtx &x, float (&g)[MT][4], float (&m)[MT][4])
{
#pragma unroll
    for (int t = 0; t < MT; ++t) {
        float v[8];
        const uint32_t ta = x.tmem + ((uint32_t)(32 * x.q) << 16) + (uint32_t)(t * x.C + x.gofs + 8 * x.cgi);
        tmem_ld8(ta, v);
        if constexpr (CL > 1) {
            float v1[8];
            tmem_ld8(ta + 7u * (uint32_t)x.C, v1);
#pragma unroll
            for (int j = 0; j < 8; ++j) v[j] += v1[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float send = x.h ? v[j] : v[4 + j];
            const float recv = __shfl_xor_sync(0xffffffffu, send, 16);
            g[t][j] = x.h ? recv : v[j];
            m[t][j] = x.h ? v[4 + j] : recv;
        }
    }
}


// TMEM -> registers for one 128-row tile t: Gt x (g) and P~ Gt x (m) of this thread's dimension
// for its 4 chains (the streamed kernels read tile by tile to bound register pressure).
template <int CL = 1>
__device__ __forceinline__ void tc_read_tile(const TcCtx &x, int t, float (&g)[4], float (&m)[4])
{
    float v[8];
    const uint32_t ta = x.tmem + ((uint32_t)(32 * x.q) << 16) + (uint32_t)(t * x.C + x.gofs + 8 * x.cgi);
    tmem_ld8(ta, v);
    if constexpr (CL > 1) {
        float v1[8];
        tmem_ld8(ta + 7u * (uint32_t)x.C, v1);
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] += v1[j];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float send = x.h ? v[j] : v[4 + j];
        const float recv = __shfl_xor_sync(0xffffffffu, send, 16);
        g[j] = x.h ? recv : v[j];
        m[j] = x.h ? v[4 + j] : recv;
    }
}

// Carried proposal factors in tensor memory (tiles of resident-operand kernels): per thread and
// tile 48 columns past the accumulators, the cumulative weights of its two chain pairs at +0 and
// +16 and their polynomial and log-normalisers at +32 and +40.
__host__ __device__ constexpr int tc_table_cols(int MT, int C) { return tc_streamed(MT) ? 0 : 6 * MT * C; }

template <int L>
__device__ __forceinline__ void table_store(uint32_t ta, uint32_t te, const Table2<L> &tb)
{
    uint32_t s[2 * L], e[8];
#pragma unroll
    for (int j = 0; j < L; ++j) {
        s[j] = __float_as_uint(tb.S0[j]);
        s[L + j] = __float_as_uint(tb.S1[j]);
    }
    float v[6];
    f2_unpack(tb.B, v[0], v[1]);
    f2_unpack(tb.C0, v[2], v[3]);
    f2_unpack(tb.lgS, v[4], v[5]);
#pragma unroll
    for (int j = 0; j < 6; ++j) e[j] = __float_as_uint(v[j]);
    e[6] = e[7] = 0u;
    tmem_st_pair<2 * L>(ta, te, s, e);
}

template <int L>
__device__ __forceinline__ void table_load(uint32_t ta, uint32_t te, Table2<L> &tb)
{
    uint32_t s[2 * L], e[8];
    tmem_ld_pair<2 * L>(ta, te, s, e);
#pragma unroll
    for (int j = 0; j < L; ++j) {
        tb.S0[j] = __uint_as_float(s[j]);
        tb.S1[j] = __uint_as_float(s[L + j]);
    }
    tb.B = f2_pack(__uint_as_float(e[0]), __uint_as_float(e[1]));
    tb.C0 = f2_pack(__uint_as_float(e[2]), __uint_as_float(e[3]));
    tb.lgS = f2_pack(__uint_as_float(e[4]), __uint_as_float(e[5]));
}

// Thread 0: bulk copy of this channel's resident A operand into shared memory, completing on the
// TMA barrier (a cluster CTA copies the S terms of its own tile of the channel's CL tiles).
template <int MT, int CL>
__device__ __forceinline__ void tc_stage_a(const TcCtx &x, const unsigned char *ops)
{
    const uint32_t tbytes = 128u * (uint32_t)x.Kp * 2u;
    const uint32_t abytes = (uint32_t)x.S * MT * tbytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(x.bar_tma), "r"(abytes)
                 : "memory");
    const uint32_t chunk = 1u << 16;
    for (int sc = 0; sc < (CL > 1 ? x.S : 1); ++sc) {
        const unsigned char *src = ops + (CL > 1 ? (size_t)(sc * CL + x.rank) * tbytes : 0);
        const uint32_t dst = smem_u32(x.sA) + (CL > 1 ? (uint32_t)sc * tbytes : 0u);
        const uint32_t nb = CL > 1 ? tbytes : abytes;
        for (uint32_t off = 0; off < nb; off += chunk) {
            const uint32_t n = nb - off < chunk ? nb - off : chunk;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    dst + off),
                "l"(src + off), "r"(n), "r"(x.bar_tma)
                : "memory");
        }
    }
}

// One work item (chains [c0, c0 + nC) of one channel). FULL: every dimension of every tile and
// every chain column is live, so no per-(dimension, chain) validity test is needed. Levels are
// held as exact small floats.
template <int MT, int L, bool FULL, int G, int CL>
__device__ void tc_item(const ChainArgs &A, TcCtx &x, const WorkItem &it, const ChannelDesc &d,
                        bool &alive)
{
    const int N = d.N, nC = it.nc, C = x.C;
    const bool pre = d.NO > N;
    const float a2s = (float)d.clin * kLog2e;     // slope -> log2 units
    const float c2 = (float)d.cquad * kLog2e;
    const float inv2c = 0.5f / c2;
    const float cf2 = (float)d.cf * kLog2e;       // df_tau -> log2 units
    const float lm1 = (float)(L - 1);
    static_assert(G == 1 || (G == 2 && MT == 1), "two chain groups only for one tile");
    static_assert(CL == 1 || (MT == 1 && G == 1), "a cluster CTA holds one tile of one group");
    const int Cq = C / G;                                  // chains per group
    const int gofs = G == 1 ? 0 : (x.q >> 1) * Cq;         // this thread's group's first chain
    const int cbase = gofs + 8 * x.cgi + 4 * x.h;          // first of its 4 chains (CTA-local)
    // sum of the per-quadrant partials of chain c over the quadrants holding its dimensions
    auto quad_sum = [&](const float *v, int c) {
        if constexpr (G == 1) {
            return v[c] + v[Cq + c] + v[2 * Cq + c] + v[3 * Cq + c];
        } else {
            const bool hi = c >= Cq;
            const int cl = hi ? c - Cq : c, g0 = hi ? 2 : 0;
            return v[g0 * Cq + cl] + v[(g0 + 1) * Cq + cl];
        }
    };
    float zt[MT], wt[MT];
    int nd[MT];
    bool live[MT][4];
    // per (tile, chain pair): levels, Gt x and the drift slope (log2 units), as packed pairs
    uint64_t k2[MT][2], sl2[MT][2];
    // Gt x of the current states: registers, or shared memory for more than two tiles
    constexpr bool kDgSmem = tc_streamed(MT);
    uint64_t Dg2r[kDgSmem ? 1 : MT][2] = {};
    auto dg_get = [&](int t, int p) -> uint64_t {
        if constexpr (kDgSmem) return x.sdg[(2 * t + p) * x.nthr + x.tid];
        else return Dg2r[t][p];
    };
    auto dg_set = [&](int t, int p, uint64_t v) {
        if constexpr (kDgSmem) x.sdg[(2 * t + p) * x.nthr + x.tid] = v;
        else Dg2r[t][p] = v;
    };
    int8_t *skb = x.skb;   // best visited states [C][64 MT] (cluster CTAs: [C][64], own dimensions)
    constexpr int kKs = tc_state_stride(MT, CL);
    auto kbi = [&](int c, int n) { return CL > 1 ? c * 64 + (n & 63) : c * kKs + n; };
    const float *gz = reinterpret_cast<const float *>(A.z) + d.vec_off;
    const float *gw = reinterpret_cast<const float *>(A.w) + d.vec_off;
    uint32_t boff[MT];                             // byte offset of this thread's B element, chain cbase
#pragma unroll
    for (int t = 0; t < MT; ++t) {
        const int n = 64 * (CL > 1 ? x.rank : t) + 16 * (G == 1 ? x.q : (x.q & 1)) + x.dl;
        nd[t] = n;
        const bool v = FULL || n < N;
        zt[t] = v ? gz[n] : 0.f;
        wt[t] = v ? gw[n] : 0.f;
        boff[t] = (uint32_t)(cbase >> 3) * x.sbo_b + (uint32_t)(n >> 3) * b_lbo() +
                  (uint32_t)(cbase & 7) * 16u + (uint32_t)(n & 7) * 2u;
        float kv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = cbase + j;
            live[t][j] = FULL || (v && c < nC);
            kv[j] = 0.f;
            if (live[t][j]) {
                const long long e = d.state_off + (long long)(it.c0 + c) * N + n;
                kv[j] = (float)A.states[e];
                skb[kbi(c, n)] = A.best_states[e];
            }
        }
        k2[t][0] = f2_pack(kv[0], kv[1]);
        k2[t][1] = f2_pack(kv[2], kv[3]);
    }
    // Algorithm 1 carries q(.|x) of the current state from one transition to the next: the
    // resident-operand kernels keep every thread's factor tables in tensor memory and rebuild
    // them (for the whole warp) only after one of its chains moved. Rebuilt tables equal the
    // carried ones bit for bit, so the draws do not depend on where a table came from.
    constexpr bool kCache = !tc_streamed(MT);
    const uint32_t tcache =
        x.tmem + ((32u * (uint32_t)x.q) << 16) + (uint32_t)(MT * C + 48 * MT * x.cgi);
    // per chain pair: the carried tables are not those of the current states (a chain of the
    // pair moved, or the work item just started); a warp rebuilds a pair's tables when any of
    // its lanes needs it, the other pair's it reloads
    bool stale[2] = {true, true};
    // chain x.tid's tracked and best energies and accept count live in shared memory (read and
    // written by that thread only)
    if (x.tid < nC) {
        const long long ci = (long long)it.b * A.chains + it.c0 + x.tid;
        x.sfc[x.tid] = A.f[ci];
        x.sfb[x.tid] = A.best_f[ci];
        x.scnt[x.tid] = 0u;
    }
    const uint64_t two2 = f2_splat(2.f), mlm1 = f2_splat(-lm1), mone = f2_splat(-1.f);
    // x as BF16 into the B operand: bits of the exact float 2k - (L-1); dead slots write 0
    auto write_b = [&](const uint64_t (&kk)[MT][2]) {
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            if (!FULL && nd[t] >= x.Kp) continue;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                float xv[2];
                f2_unpack(f2_fma(two2, kk[t][p], mlm1), xv[0], xv[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int j = 2 * p + h;
                    if (!FULL && cbase + j >= C) continue;
                    const float v = live[t][j] ? xv[h] : 0.f;
                    *reinterpret_cast<unsigned short *>(x.sB + boff[t] + 16u * j) =
                        (unsigned short)(__float_as_uint(v) >> 16);
                }
            }
        }
    };
    // slope of a state from its products (log2 units): c_lin (w~ - P~Gt x) or c_lin (z~ - Gt x)
    auto slope2 = [&](int t, uint64_t g, uint64_t m) {
        return f2_mul(f2_splat(a2s), f2_fma(mone, pre ? m : g, f2_splat(pre ? wt[t] : zt[t])));
    };
    // x (BF16 bits of an odd level) of chain c, dimension n, from the B operand
    auto b_level = [&](int c, int n) -> float {
        const unsigned short bits = *reinterpret_cast<const unsigned short *>(
            x.sB + (uint32_t)(c >> 3) * x.sbo_b + (uint32_t)(n >> 3) * b_lbo() + (uint32_t)(c & 7) * 16u +
            (uint32_t)(n & 7) * 2u);
        return __uint_as_float((uint32_t)bits << 16);
    };
    write_b(k2);
    if (x.tid == 0) tc_mma_descs<MT>(x);
    bool lf0 = false;   // cluster: a failed first MMA wait, reported through the first exchange
    if (alive) {
        tc_gemm_issue<MT, CL>(x);
        const bool ok = tc_gemm_wait<MT, CL>(x, A.iterations > 0);
        if constexpr (CL > 1) lf0 = __syncthreads_or(!ok);
        else if (__syncthreads_or(!ok)) { alive = false; set_status(A.status, kStatusTimeout); }
    }
    {
        float g[MT][4], m[MT][4];
        if (alive) tc_read<MT, CL>(x, g, m);
#pragma unroll
        for (int t = 0; t < MT; ++t)
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const uint64_t gg = alive ? f2_pack(g[t][2 * p], g[t][2 * p + 1]) : 0ull;
                const uint64_t mm = alive ? f2_pack(m[t][2 * p], m[t][2 * p + 1]) : 0ull;
                dg_set(t, p, gg);
                sl2[t][p] = alive ? slope2(t, gg, mm) : 0ull;
            }
    }
    // tracked energies of the current states from the tensor-core Gt x; the running best
    // restarts from them. Per-quadrant partial sums of chain c go to red / dred.
    auto init_partials = [&]() {
        float lin[4], quad[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) { lin[j] = 0.f; quad[j] = 0.f; }
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            float kv[4], dg[4];
            f2_unpack(k2[t][0], kv[0], kv[1]);
            f2_unpack(k2[t][1], kv[2], kv[3]);
            f2_unpack(dg_get(t, 0), dg[0], dg[1]);
            f2_unpack(dg_get(t, 1), dg[2], dg[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (!live[t][j]) continue;
                const float xn = fmaf(2.f, kv[j], -lm1);
                lin[j] = fmaf(xn, zt[t], lin[j]);
                quad[j] = fmaf(xn, dg[j], quad[j]);
                skb[kbi(cbase + j, nd[t])] = (int8_t)kv[j];
            }
        }
        const float rl = reduce_scatter16(lin, x.dl);
        const float rq = reduce_scatter16(quad, x.dl);
        if ((x.dl & 3) == 0) {
            const int c = cbase + (x.dl >> 2);
            x.red[x.q * Cq + c - gofs] = rl;
            x.dred[x.q * Cq + c - gofs] = rq;
        }
    };
    if constexpr (CL > 1) {
        // the first exchange always runs: it carries the energies' partial sums (or zeros) and the
        // first MMA's verdict, and it separates this work item's first B-slice transfer from the next
        if (A.init_f) init_partials();
        __syncthreads();
        bool xf = false;
        if (x.tid < C) {
            const int c = x.tid;
            const float l = A.init_f ? quad_sum(x.red, c) : 0.f;
            const float qd = A.init_f ? quad_sum(x.dred, c) : 0.f;
            xf = !cl_exchange<CL>(x, c, make_uint4(__float_as_uint(l), __float_as_uint(qd), lf0 ? 1u : 0u, 0u));
            if (!xf) {
                float sl = 0.f, sq = 0.f;
#pragma unroll
                for (int r = 0; r < CL; ++r) {
                    const uint4 v = cl_slot(x, CL, r, c);
                    sl += __uint_as_float(v.x);
                    sq += __uint_as_float(v.y);
                    xf |= v.z != 0u;
                }
                if (A.init_f && c < nC) {
                    const double f0 = -(A.yy[it.b] - 2.0 * (double)sl + (double)sq) * d.inv_s2;
                    x.sfc[c] = f0;
                    x.sfb[c] = f0;
                }
            }
        }
        cl_next(x);
        if (__syncthreads_or(xf)) { alive = false; set_status(A.status, kStatusTimeout); }
    } else if (A.init_f && alive) {
        init_partials();
        __syncthreads();
        if (x.tid < nC) {
            const int c = x.tid;
            const double l = (double)quad_sum(x.red, c);
            const double qd = (double)quad_sum(x.dred, c);
            const double f0 = -(A.yy[it.b] - 2.0 * l + qd) * d.inv_s2;
            x.sfc[c] = f0;
            x.sfb[c] = f0;
        }
        __syncthreads();
    }

    for (int i = 0; i < A.iterations && alive; ++i) {
        const uint32_t t_it = (uint32_t)(A.t_offset + 1 + i);
        uint64_t part2[2] = {0ull, 0ull}, dpart2[2] = {0ull, 0ull};
        uint64_t kp2[MT][2];
        // 1. proposal draw (log2 q(x'|x) accumulated with a minus sign) from the carried factors
        bool fresh[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            fresh[p] = !kCache || __any_sync(0xffffffffu, stale[p]);
            stale[p] = false;
        }
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const int n = nd[t];
            U4 w = {0, 0, 0, 0};
            if (FULL || live[t][0])
                w = philox4x32_10_rk(t_it, (uint32_t)n, (uint32_t)it.b,
                                     (uint32_t)((it.c0 + cbase) >> 2), A.philox_rk);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                Table2<L> tb;
                const uint32_t ta = tcache + 48u * t + 16u * p, te = tcache + 48u * t + 32u + 8u * p;
                if (fresh[p]) {
                    factor_table_f2<L>(sl2[t][p], c2, inv2c, k2[t][p], tb);
                    if constexpr (kCache) table_store<L>(ta, te, tb);
                } else {
                    table_load<L>(ta, te, tb);
                }
                uint64_t sel, lq;
                table_draw_f2<L>(tb, c2, uniform_f(word_of(w, 2 * p)), uniform_f(word_of(w, 2 * p + 1)),
                                 sel, lq);
                if (!FULL) {
                    float s[2], kk[2], q[2];
                    f2_unpack(sel, s[0], s[1]);
                    f2_unpack(k2[t][p], kk[0], kk[1]);
                    f2_unpack(lq, q[0], q[1]);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (!live[t][2 * p + h]) { s[h] = kk[h]; q[h] = 0.f; }
                    sel = f2_pack(s[0], s[1]);
                    lq = f2_pack(q[0], q[1]);
                }
                kp2[t][p] = sel;
                part2[p] = f2_fma(mone, lq, part2[p]);
            }
        }
        write_b(kp2);
        // 2. D' = A X'^T on the tensor core; while it runs, the chains' acceptance uniforms
        //    (the timeout verdict joins the next CTA barrier)
        tc_gemm_issue<MT, CL>(x);
        float logu = 0.f;
        if (x.tid < nC) {
            const int cc = it.c0 + x.tid;
            const U4 w = philox4x32_10_rk(t_it, kMhStream, (uint32_t)it.b, (uint32_t)(cc >> 2),
                                          A.philox_rk);
            logu = lg2_approx(uniform_f(word_of(w, cc & 3)));
        }
        const bool mma_ok = tc_gemm_wait<MT, CL>(x, i + 1 < A.iterations);
        // 3. reverse factor and energy difference (with more than two tiles, the products and
        //    levels of x' are not kept in registers: the update reads them again)
        constexpr bool kReread = tc_streamed(MT);
        constexpr int MTK = kReread ? 1 : MT;   // tiles whose x' caches stay live
        uint64_t gp2[MTK][2], sp2[MTK][2];
#pragma unroll
        for (int t = 0; t < MT; ++t) {
            const uint64_t z2 = f2_splat(2.f * zt[t]);
            float gpt[4], mpt[4];
            tc_read_tile<CL>(x, t, gpt, mpt);
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const uint64_t gg = f2_pack(gpt[2 * p], gpt[2 * p + 1]);
                const uint64_t ap = slope2(t, gg, f2_pack(mpt[2 * p], mpt[2 * p + 1]));
                if constexpr (!kReread) {
                    gp2[t < MTK ? t : 0][p] = gg;
                    sp2[t < MTK ? t : 0][p] = ap;   // slope of x', kept for the update
                }
                uint64_t lr = factor_log2q_f2<L>(ap, c2, inv2c, kp2[t][p], k2[t][p]);
                // (x'_n - x_n)(2 zt_n - (Gt x)_n - (Gt x')_n), the levels' difference doubled
                const uint64_t dk = f2_mul(two2, f2_fma(mone, k2[t][p], kp2[t][p]));
                const uint64_t e = f2_fma(mone, gg, f2_fma(mone, dg_get(t, p), z2));
                uint64_t dd = f2_mul(dk, e);
                if (!FULL) {
                    float a[2], b[2];
                    f2_unpack(lr, a[0], a[1]);
                    f2_unpack(dd, b[0], b[1]);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (!live[t][2 * p + h]) { a[h] = 0.f; b[h] = 0.f; }
                    lr = f2_pack(a[0], a[1]);
                    dd = f2_pack(b[0], b[1]);
                }
                part2[p] = f2_add(part2[p], lr);
                dpart2[p] = f2_add(dpart2[p], dd);
            }
        }
        // 4. per-chain reduction and the MH decision (log2 units)
        float part[4], dpart[4];
        f2_unpack(part2[0], part[0], part[1]);
        f2_unpack(part2[1], part[2], part[3]);
        f2_unpack(dpart2[0], dpart[0], dpart[1]);
        f2_unpack(dpart2[1], dpart[2], dpart[3]);
        const float rs = reduce_scatter16(part, x.dl);
        const float rd = reduce_scatter16(dpart, x.dl);
        if ((x.dl & 3) == 0) {
            const int c = cbase + (x.dl >> 2);
            x.red[x.q * Cq + c - gofs] = rs;
            x.dred[x.q * Cq + c - gofs] = rd;
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        // MH decision of chain c (thread c) from its summed log q terms s and energy terms sd
        auto decide = [&](int c, float s, float sd) {
            const float logr = fmaf(cf2, sd, s);
            const float loga = logr < 0.f ? logr : 0.f;
            int ok = logu < loga;
            if (!isfinite(logr)) { ok = 0; set_status(A.status, kStatusNumeric); }
            if (CL == 1 || x.rank == 0) {
                // near-tie bands |log A - log u| < 1e-6, 1e-4, 1e-2 (natural log; log2 units here)
                const float gap = fabsf(loga - logu);
                x.stie[c] += gap < 1e-6f * kLog2e ? 1u : 0u;
                x.stie[C + c] += gap < 1e-4f * kLog2e ? 1u : 0u;
                x.stie[2 * C + c] += gap < 1e-2f * kLog2e ? 1u : 0u;
                if (A.trace)
                    reinterpret_cast<double2 *>(A.trace)[(long long)it.b * A.chains + it.c0 + c] =
                        make_double2((double)logr * (double)kLn2, (double)logu * (double)kLn2);
            }
            int im = 0;
            if (ok) {
                const double fc = x.sfc[c] + d.inv_s2 * (double)sd;
                x.sfc[c] = fc;
                x.scnt[c] += 1u;
                if (fc > x.sfb[c]) { x.sfb[c] = fc; im = 1; }
            }
            x.sacc[c] = ok | (im << 1);
        };
        if constexpr (CL == 1) {
            if (__syncthreads_or(!mma_ok)) { alive = false; set_status(A.status, kStatusTimeout); break; }
            if (x.tid < nC) decide(x.tid, quad_sum(x.red, x.tid), quad_sum(x.dred, x.tid));
            __syncthreads();
        } else {
            // the CTA's partial sums (its 64 dimensions) to every CTA of the cluster; every CTA
            // adds the CL partials in rank order and takes the same decisions
            const bool lf = __syncthreads_or(!mma_ok);
            bool xf = false;
            if (x.tid < C) {
                const int c = x.tid;
                xf = !cl_exchange<CL>(x, c,
                                      make_uint4(__float_as_uint(quad_sum(x.red, c)),
                                                 __float_as_uint(quad_sum(x.dred, c)), lf ? 1u : 0u, 0u));
                if (!xf) {
                    float ss = 0.f, sd = 0.f;
#pragma unroll
                    for (int r = 0; r < CL; ++r) {
                        const uint4 v = cl_slot(x, CL, r, c);
                        ss += __uint_as_float(v.x);
                        sd += __uint_as_float(v.y);
                        xf |= v.z != 0u;
                    }
                    if (!xf && c < nC) decide(c, ss, sd);
                }
            }
            cl_next(x);
            if (__syncthreads_or(xf)) { alive = false; set_status(A.status, kStatusTimeout); break; }
        }
        // 5. accepted chains take x' and its caches
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            int fl[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = cbase + 2 * p + h;
                fl[h] = (FULL || c < nC) ? x.sacc[c] : 0;
                if (fl[h] & 1) stale[p] = true;   // x' taken: its factors are not the carried ones
            }
            if constexpr (kReread) continue;
#pragma unroll
            for (int t = 0; t < MTK; ++t) {
                float ka[2], kb[2], da[2], db[2], sa[2], sb[2];
                f2_unpack(k2[t][p], ka[0], ka[1]);
                f2_unpack(kp2[t][p], kb[0], kb[1]);
                f2_unpack(dg_get(t, p), da[0], da[1]);
                f2_unpack(gp2[t][p], db[0], db[1]);
                f2_unpack(sl2[t][p], sa[0], sa[1]);
                f2_unpack(sp2[t][p], sb[0], sb[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const bool ok = fl[h] & 1, im = fl[h] & 2;
                    ka[h] = ok ? kb[h] : ka[h];
                    da[h] = ok ? db[h] : da[h];
                    sa[h] = ok ? sb[h] : sa[h];
                    if (im && live[t][2 * p + h]) skb[kbi(cbase + 2 * p + h, nd[t])] = (int8_t)kb[h];
                }
                k2[t][p] = f2_pack(ka[0], ka[1]);
                dg_set(t, p, f2_pack(da[0], da[1]));
                sl2[t][p] = f2_pack(sa[0], sa[1]);
            }
        }
        if constexpr (kReread) {
            // accepted chains: x' levels from the B operand, Gt x' and the slope from TMEM (the
            // loads are warp-collective: a warp reads when any of its lanes has an acceptance)
            int fl[4];
            bool any = false;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = cbase + j;
                fl[j] = (FULL || c < nC) ? x.sacc[c] : 0;
                any |= (fl[j] & 1);
            }
            if (__any_sync(0xffffffffu, any)) {
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    float g[4], m[4];
                    tc_read_tile<CL>(x, t, g, m);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        float ka[2], da[2], sa[2], sb[2];
                        f2_unpack(k2[t][p], ka[0], ka[1]);
                        f2_unpack(dg_get(t, p), da[0], da[1]);
                        f2_unpack(sl2[t][p], sa[0], sa[1]);
                        f2_unpack(slope2(t, f2_pack(g[2 * p], g[2 * p + 1]), f2_pack(m[2 * p], m[2 * p + 1])),
                                  sb[0], sb[1]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int j = 2 * p + h;
                            if (!(fl[j] & 1)) continue;
                            const unsigned short bits =
                                *reinterpret_cast<const unsigned short *>(x.sB + boff[t] + 16u * j);
                            const float kb = 0.5f * (__uint_as_float((uint32_t)bits << 16) + lm1);
                            ka[h] = kb;
                            da[h] = g[j];
                            sa[h] = sb[h];
                            if ((fl[j] & 2) && live[t][j]) skb[kbi(cbase + j, nd[t])] = (int8_t)kb;
                        }
                        k2[t][p] = f2_pack(ka[0], ka[1]);
                        dg_set(t, p, f2_pack(da[0], da[1]));
                        sl2[t][p] = f2_pack(sa[0], sa[1]);
                    }
                }
            }
        }
        // periodic FP64 refresh of the tracked energies (decisions never read them); compiled
        // into the kernels of the second translation unit only
        if constexpr (!kInKernelRefresh) {
        } else if constexpr (CL > 1) {
            if (A.refresh_period > 0 && (t_it % (uint32_t)A.refresh_period) == 0u) {
                // every CTA needs the whole state: x goes through the B operand's slice transfer.
                // Then x^T G x over this CTA's rows n (all columns m) is evaluated exactly for
                // G rounded to 53 bits below its largest entry (|G_nm| <= max_n G_nn, G being
                // positive semidefinite): G_nm 2^sh = sum_k d_k,nm 256^k with balanced int8 digits
                // d_k (k = 0..6), and Q_k = sum_n x_n sum_m d_k,nm x_m is an exact int32 sum of
                // DP4A products. The partial sums sum_k Q_k 256^k 2^-sh (FP64) and z^T x over the
                // rows are exchanged and added in rank order, identically in every CTA. The A
                // operand's shared memory holds the scratch and is reloaded afterwards.
                write_b(k2);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (x.tid == 0) cl_send_b<CL>(x);
                bool okb = mbar_wait(x.bar_b, x.b_phase);
                x.b_phase ^= 1u;
                const double *Gm = A.G64 + d.mat_off;
                const double *z = A.z64 + d.vec_off;
                const int Kp = x.Kp, XS = Kp + 16, nw = Kp / 4, n0 = 64 * x.rank;
                int8_t *sX = reinterpret_cast<int8_t *>(x.sA);                    // [C][XS] states
                uint32_t *sD = reinterpret_cast<uint32_t *>(x.sA + C * XS);       // [7][16][nw] digits
                int *sQ = reinterpret_cast<int *>(x.sA + C * XS + 112 * Kp);     // [C][7] Q_k
                if (x.warp == 0) {
                    double mx = 0.0;
                    for (int n = x.lane; n < N; n += 32) mx = fmax(mx, Gm[(long long)n * N + n]);
#pragma unroll
                    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    if (x.lane == 0) x.sref[0] = mx;
                }
                for (int e = x.tid; e < C * Kp; e += x.nthr) {
                    const int c = e / Kp, m = e - c * Kp;
                    sX[c * XS + m] = (int8_t)b_level(c, m);
                }
                for (int e = x.tid; e < 7 * C; e += x.nthr) sQ[e] = 0;
                __syncthreads();
                int ex2;
                frexp(x.sref[0], &ex2);
                const int sh = 53 - ex2;                         // |G_nm| 2^sh < 2^53
                const int cc = x.tid % C, rg = x.tid / C;        // chain; row rg of each 16-row block
                int pk[7] = {0, 0, 0, 0, 0, 0, 0};
                for (int rb = 0; rb < 4; ++rb) {
                    if (rb) __syncthreads();                     // the last block's digits are read
                    for (int u = x.tid; u < 16 * nw; u += x.nthr) {
                        const int i = u / nw, w = u - i * nw, n = n0 + 16 * rb + i;
                        uint32_t dw[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
                        if (n < N) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int m = 4 * w + j;
                                long long v = m < N ? fixed_of(Gm[(long long)n * N + m], sh) : 0;
#pragma unroll
                                for (int k = 0; k < 7; ++k) {
                                    const int lo = (int)(v & 255), dk = lo >= 128 ? lo - 256 : lo;
                                    v = (v - dk) >> 8;
                                    dw[k] |= (uint32_t)(dk & 255) << (8 * j);
                                }
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 7; ++k) sD[(k * 16 + i) * nw + w] = dw[k];
                    }
                    __syncthreads();
                    int tk[7] = {0, 0, 0, 0, 0, 0, 0};
                    const uint32_t *xw = reinterpret_cast<const uint32_t *>(sX + cc * XS);
                    for (int w = 0; w < nw; w += 4) {
                        const uint4 xv = *reinterpret_cast<const uint4 *>(xw + w);
#pragma unroll
                        for (int k = 0; k < 7; ++k) {
                            const uint4 dv = *reinterpret_cast<const uint4 *>(sD + (k * 16 + rg) * nw + w);
                            int a = tk[k];
                            a = __dp4a((int)dv.x, (int)xv.x, a);
                            a = __dp4a((int)dv.y, (int)xv.y, a);
                            a = __dp4a((int)dv.z, (int)xv.z, a);
                            a = __dp4a((int)dv.w, (int)xv.w, a);
                            tk[k] = a;
                        }
                    }
                    const int n = n0 + 16 * rb + rg;
                    const int xn = n < N ? (int)sX[cc * XS + n] : 0;
#pragma unroll
                    for (int k = 0; k < 7; ++k) pk[k] += xn * tk[k];
                }
                // integer sums: exact in any order
#pragma unroll
                for (int k = 0; k < 7; ++k) atomicAdd(&sQ[cc * 7 + k], pk[k]);
                __syncthreads();
                if (x.tid < nC) {
                    const int c = x.tid;
                    double q = 0.0;
                    for (int k = 6; k >= 0; --k) q = fma(q, 256.0, (double)sQ[c * 7 + k]);
                    double l = 0.0;
                    for (int n = n0; n < n0 + 64 && n < N; ++n) l = fma(z[n], (double)sX[c * XS + n], l);
                    x.sref[2 * c] = ldexp(q, -sh);
                    x.sref[2 * c + 1] = l;
                }
                // the scratch is read: reload the resident operand (complete before the next MMA)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
                if (x.tid == 0) tc_stage_a<MT, CL>(x, A.tc_ops + d.tc_off);
                okb = mbar_wait(x.bar_tma, x.tma_phase) && okb;
                x.tma_phase ^= 1u;
                bool xf = __syncthreads_or(!okb);
                if (x.tid < C) {
                    const int c = x.tid;
                    const double q = c < nC ? x.sref[2 * c] : 0.0, l = c < nC ? x.sref[2 * c + 1] : 0.0;
                    const unsigned long long qb = (unsigned long long)__double_as_longlong(q);
                    const unsigned long long lb = (unsigned long long)__double_as_longlong(l);
                    const bool okx = cl_exchange<CL>(
                        x, c, make_uint4((uint32_t)qb, (uint32_t)(qb >> 32), (uint32_t)lb, (uint32_t)(lb >> 32)));
                    xf |= !okx;
                    if (okx && c < nC) {
                        double sq = 0.0, sl = 0.0;
#pragma unroll
                        for (int r = 0; r < CL; ++r) {
                            const uint4 v = cl_slot(x, CL, r, c);
                            sq += __longlong_as_double((long long)(((unsigned long long)v.y << 32) | v.x));
                            sl += __longlong_as_double((long long)(((unsigned long long)v.w << 32) | v.z));
                        }
                        const double fr = -(A.yy[it.b] - 2.0 * sl + sq) * d.inv_s2;
                        if (x.rank == 0)
                            atomicMax(A.drift_bits, (unsigned long long)__double_as_longlong(fabs(fr - x.sfc[c])));
                        x.sfc[c] = fr;
                    }
                }
                cl_next(x);
                if (__syncthreads_or(xf)) { alive = false; set_status(A.status, kStatusTimeout); break; }
            }
        } else if (A.refresh_period > 0 && (t_it % (uint32_t)A.refresh_period) == 0u) {
#pragma unroll
            for (int t = 0; t < MT; ++t) {
                float kv[4];
                f2_unpack(k2[t][0], kv[0], kv[1]);
                f2_unpack(k2[t][1], kv[2], kv[3]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (live[t][j]) x.sfs[(cbase + j) * kKs + nd[t]] = (int8_t)kv[j];
            }
            __syncthreads();
            const double *Gm = A.G64 + d.mat_off;
            const double *z = A.z64 + d.vec_off;
            for (int c = x.warp; c < nC; c += blockDim.x >> 5) {
                double quad, lin;
                quad_lin_fp64(Gm, z, N, x.lane,
                              [&](int n) { return (double)odd_of(x.sfs[c * kKs + n], L); }, quad, lin);
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    quad += __shfl_xor_sync(0xffffffffu, quad, o);
                    lin += __shfl_xor_sync(0xffffffffu, lin, o);
                }
                if (x.lane == 0) x.sref[c] = -(A.yy[it.b] - 2.0 * lin + quad) * d.inv_s2;
            }
            __syncthreads();
            if (x.tid < nC) {
                const double dr = fabs(x.sref[x.tid] - x.sfc[x.tid]);
                atomicMax(A.drift_bits, (unsigned long long)__double_as_longlong(dr));
                x.sfc[x.tid] = x.sref[x.tid];
            }
        }
    }
    // write back this work item
#pragma unroll
    for (int t = 0; t < MT; ++t) {
        float kv[4], dg[4];
        f2_unpack(k2[t][0], kv[0], kv[1]);
        f2_unpack(k2[t][1], kv[2], kv[3]);
        f2_unpack(dg_get(t, 0), dg[0], dg[1]);
        f2_unpack(dg_get(t, 1), dg[2], dg[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!live[t][j]) continue;
            const long long e = d.state_off + (long long)(it.c0 + cbase + j) * N + nd[t];
            A.states[e] = (int8_t)kv[j];
            A.best_states[e] = skb[kbi(cbase + j, nd[t])];
            if (A.dexp) A.dexp[e] = dg[j];
        }
    }
    if (x.tid < nC && (CL == 1 || x.rank == 0)) {
        const long long ci = (long long)it.b * A.chains + it.c0 + x.tid;
        A.f[ci] = x.sfc[x.tid];
        A.best_f[ci] = x.sfb[x.tid];
        A.accepts[ci] += x.scnt[x.tid];
    }
}

template <int MT, int L, int G, int CL>
__device__ __forceinline__ void tc_item_dispatch(const ChainArgs &A, TcCtx &x, const WorkItem &it,
                                                 const ChannelDesc &d, bool &alive)
{
    if (d.N == 64 * MT * CL / G && it.nc == x.C) tc_item<MT, L, true, G, CL>(A, x, it, d, alive);
    else tc_item<MT, L, false, G, CL>(A, x, it, d, alive);
}

// G: chain groups per CTA (2 for N <= 32, one tile); C: chains per CTA over all groups.
// CL > 1: one CTA of a cluster of CL (MT = 1 local tile of a channel with CL tiles).
// G = 0: the packed kernel for a batch of uneven one-tile channels (N <= 64): every CTA pulls
// work items from a device queue (largest first) and takes each item's chain groups (1 or 2,
// by N), K extent and operand layouts from its channel; C is then the largest chains per CTA
// (two groups of C / 2) and Kp = 64, the extents the shared memory and TMEM are sized for.
template <int MT, int G, int CL>
__global__ void __launch_bounds__(CL > 1 ? 1024 : TC_MAX_THREADS, MT == 1 && CL == 1 ? TC_MIN_BLOCKS : 1)
    chains_tc_kernel(const ChainArgs A, const int C, const int S, const int Kp)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcLayout lay = tc_layout(S, MT, Kp, C, CL);
    TcCtx x;
    x.sA = smem + lay.a;
    x.sB = smem + lay.b;
    x.red = reinterpret_cast<float *>(smem + lay.red);
    x.dred = reinterpret_cast<float *>(smem + lay.dred);
    x.sacc = reinterpret_cast<int *>(smem + lay.acc);
    x.sref = reinterpret_cast<double *>(smem + lay.ref);
    x.sfc = reinterpret_cast<double *>(smem + lay.fst);
    x.sfb = x.sfc + C;
    x.scnt = reinterpret_cast<unsigned *>(smem + lay.cnt);
    x.stie = reinterpret_cast<unsigned *>(smem + lay.tie);
    x.sfs = reinterpret_cast<int8_t *>(smem + lay.fref);
    x.skb = reinterpret_cast<int8_t *>(smem + lay.kb);
    x.sdg = reinterpret_cast<uint64_t *>(smem + lay.dg);
    x.sdsc = reinterpret_cast<uint4 *>(smem + lay.dsc);
    x.nthr = blockDim.x;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + lay.bar);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + lay.tmem);
    x.bar_tma = smem_u32(&bars[0]);
    x.tma_phase = 0;
    x.bar_mma = smem_u32(&bars[1]);
    x.tid = threadIdx.x;
    x.warp = x.tid >> 5;
    x.lane = x.tid & 31;
    x.q = x.warp & 3;
    x.cgi = x.warp >> 2;
    x.h = x.lane >> 4;
    x.dl = x.lane & 15;
    constexpr bool kPacked = G == 0;
    static_assert(!kPacked || (MT == 1 && CL == 1), "the packed kernel runs one-tile items");
    x.C = C;
    x.gofs = G == 2 ? (x.q >> 1) * (C / 2) : 0;   // first chain of this thread's group
    x.S = S;
    x.Kp = Kp;
    x.sbo_a = (uint32_t)(Kp / 8) * 128u;
    x.sbo_b = b_sbo(Kp);
    x.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(C >> 3) << 17) |
              ((uint32_t)(128 >> 4) << 24);
    x.mma_phase = 0;
    x.asrc = nullptr;
    for (int b = 0; b < 2; ++b) {
        x.bar_full[b] = smem_u32(&bars[2 + b]);
        x.bar_empty[b] = smem_u32(&bars[4 + b]);
        x.full_phase[b] = 0;
        x.empty_phase[b] = 0;
        x.pend[b] = false;
    }
    x.fail = false;
    x.rank = CL > 1 ? (int)cl_rank() : 0;
    x.bar_b = smem_u32(&bars[6]);
    x.bar_x = smem_u32(&bars[7]);
    x.b_phase = 0;
    x.x_phase = 0;
    x.x_buf = 0;
    x.sx = smem + lay.xs;
    const int ncols_alloc = A.tc_tmem_cols;   // TMEM columns to allocate (power of 2, >= 32)

    if (x.tid == 0) {
        mbar_init(x.bar_tma, 1);
        mbar_init(x.bar_mma, CL > 1 ? 2 : 1);   // clusters: two issuers commit
        for (int b = 0; b < 2; ++b) {
            mbar_init(x.bar_full[b], 1);
            mbar_init(x.bar_empty[b], 1);
        }
        mbar_init(x.bar_b, 1);
        mbar_init(x.bar_x, (uint32_t)CL);         // one release-arrival from every CTA
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (x.warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(ncols_alloc));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    x.tmem = *tmem_slot;
    // zero the B operand once: padding columns / chains stay zero, the rest is rewritten
    for (int e = x.tid; e < (int)(lay.red - lay.b) / 16; e += blockDim.x)
        reinterpret_cast<uint4 *>(x.sB)[e] = make_uint4(0, 0, 0, 0);
    for (int e = x.tid; e < 3 * C; e += blockDim.x) x.stie[e] = 0u;
    bool alive = true;
    // a cluster's CTAs start exchanging only once every CTA's barriers and B operand are set up
    if constexpr (CL > 1) cl_sync();
    const int item0 = CL > 1 ? (int)cl_id() : (int)blockIdx.x;
    const int istep = CL > 1 ? (int)cl_count() : (int)gridDim.x;
    volatile int *qslot = reinterpret_cast<volatile int *>(tmem_slot + 1);

    for (int item = item0; alive; item += istep) {
        if constexpr (kPacked) {
            // the next item of the batch's queue (every CTA of the launch draws from it)
            if (x.tid == 0) *qslot = atomicAdd(A.queue, 1);
            __syncthreads();
            item = *qslot;
            __syncthreads();
        }
        if (item >= A.n_items) break;
        const WorkItem it = A.items[item];
        const ChannelDesc d = A.desc[it.b];
        x.asrc = A.tc_ops + d.tc_off;
        if constexpr (kPacked) {
            // this item's chain groups and K extent, and the operand layouts that follow from them
            const int g = tc_groups(d.N), tile = C / 2, kp = (d.N + 15) / 16 * 16;
            x.C = g * tile;
            x.gofs = g == 1 ? 0 : (x.q >> 1) * tile;
            x.Kp = kp;
            x.sbo_a = (uint32_t)(kp / 8) * 128u;
            x.sbo_b = b_sbo(kp);
            x.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(x.C >> 3) << 17) |
                      ((uint32_t)(128 >> 4) << 24);
            // the B operand's layout follows K: clear it, so that padding stays zero (the
            // previous item's MMAs have completed; the staging barrier below orders the rest)
            for (int e = x.tid; e < (int)(lay.red - lay.b) / 16; e += blockDim.x)
                reinterpret_cast<uint4 *>(x.sB)[e] = make_uint4(0, 0, 0, 0);
        }
        if constexpr (tc_streamed(MT)) {
            // chunks are streamed by the transitions themselves
            switch (d.L) {
            case 2: tc_item_dispatch<MT, 2, G, CL>(A, x, it, d, alive); break;
            case 4: tc_item_dispatch<MT, 4, G, CL>(A, x, it, d, alive); break;
            default: tc_item_dispatch<MT, 8, G, CL>(A, x, it, d, alive); break;
            }
            const bool drained = x.tid != 0 || tc_stream_drain(x);
            if (__syncthreads_or(!drained || (x.tid == 0 && x.fail)) && alive) {
                alive = false;
                set_status(A.status, kStatusTimeout);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            continue;
        }
        // stage this channel's A operand (TMA bulk copy, mbarrier completion)
        if (x.tid == 0) tc_stage_a<MT, CL>(x, A.tc_ops + d.tc_off);
        if (__syncthreads_or(!mbar_wait(x.bar_tma, x.tma_phase))) {
            alive = false;
            set_status(A.status, kStatusTimeout);
        }
        x.tma_phase ^= 1u;
        if (!alive) break;
        if constexpr (kPacked) {
            if (tc_groups(d.N) == 2) {
                switch (d.L) {
                case 2: tc_item_dispatch<1, 2, 2, 1>(A, x, it, d, alive); break;
                case 4: tc_item_dispatch<1, 4, 2, 1>(A, x, it, d, alive); break;
                default: tc_item_dispatch<1, 8, 2, 1>(A, x, it, d, alive); break;
                }
            } else {
                switch (d.L) {
                case 2: tc_item_dispatch<1, 2, 1, 1>(A, x, it, d, alive); break;
                case 4: tc_item_dispatch<1, 4, 1, 1>(A, x, it, d, alive); break;
                default: tc_item_dispatch<1, 8, 1, 1>(A, x, it, d, alive); break;
                }
            }
        } else {
            switch (d.L) {
            case 2: tc_item_dispatch<MT, 2, G, CL>(A, x, it, d, alive); break;
            case 4: tc_item_dispatch<MT, 4, G, CL>(A, x, it, d, alive); break;
            default: tc_item_dispatch<MT, 8, G, CL>(A, x, it, d, alive); break;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    // near-tie counts of the CTA (every item it ran): one sum per window
    __syncthreads();
    if (x.warp == 0 && A.near_ties && (CL == 1 || x.rank == 0)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            unsigned v = 0;
            for (int c = x.lane; c < C; c += 32) v += x.stie[k * C + c];
            v = __reduce_add_sync(0xffffffffu, v);
            if (x.lane == 0 && v) atomicAdd(&A.near_ties[k], (unsigned long long)v);
        }
    }
    // no CTA leaves while another may still store into its shared memory: after a wait that ran
    // out, the B-slice phase this CTA armed last may still receive the other CTAs' bulk copies,
    // so thread 0 waits (bounded) for it before the exit barrier (on the normal path it has
    // completed and the wait returns at once)
    if constexpr (CL > 1) {
        if (x.tid == 0 && !alive) mbar_wait(x.bar_b, x.b_phase ^ 1u);
        cl_sync();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (x.warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(x.tmem),
                     "r"(ncols_alloc));
}

#if !MCMC_TC_IN_KERNEL_REFRESH
// ------------------------------------------------------------------------------------------
// Operand packing: [Gt | P~Gt] (FP32) -> `S` BF16 split terms in the core-matrix image. One
// thread builds one 16-byte core-matrix row (8 consecutive K values of one A row) per term.
// ------------------------------------------------------------------------------------------
__global__ void pack_kernel(const ChannelDesc *desc, const float *bt32, uint8_t *ops, int S)
{
    const ChannelDesc d = desc[blockIdx.x];
    const int N = d.N;
    if (N > kMaxN) return;
    const int MT = (N + 63) / 64, Kp = (N + 15) / 16 * 16;
    const bool pre = d.NO > N;
    const float *bt = bt32 + d.bt_off;
    uint8_t *base = ops + d.tc_off;
    const int kgs = Kp / 8;
    const int units = MT * 128 * kgs;
    for (int u = threadIdx.x; u < units; u += blockDim.x) {
        const int t = u / (128 * kgs), rem = u % (128 * kgs);
        const int r = rem / kgs, kg = rem % kgs;
        const int q = r >> 5, l = r & 31;
        const int qpg = tc_groups(N) == 2 ? 2 : 4;     // two copies of the rows for N <= 32
        const int n = 64 * t + 16 * (q % qpg) + (l & 15), part = l >> 4;
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int kk = 8 * kg + i;
            float x = 0.f;
            if (n < N && kk < N && (part == 0 || pre)) x = bt[(size_t)kk * d.NOp + part * N + n];
            v[i] = x;   // Bt row kk holds [Gt row kk | P~Gt row kk]; both blocks are symmetric
        }
        const size_t off = (size_t)((r >> 3) * kgs + kg) * 128 + (r & 7) * 16;
        for (int s = 0; s < S; ++s) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const __nv_bfloat16 lo = __float2bfloat16_rn(v[2 * i]);
                const __nv_bfloat16 hi = __float2bfloat16_rn(v[2 * i + 1]);
                v[2 * i] -= __bfloat162float(lo);
                v[2 * i + 1] -= __bfloat162float(hi);
                w[i] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
            }
            *reinterpret_cast<uint4 *>(base + (size_t)(s * MT + t) * 128 * Kp * 2 + off) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

int pow2_at_least(int v)
{
    int p = 32;
    while (p < v) p <<= 1;
    return p;
}
#endif  // !MCMC_TC_IN_KERNEL_REFRESH

}  // namespace

namespace {

using TcKernel = void (*)(const ChainArgs, const int, const int, const int);

TcKernel cluster_kernel(int CL) { return CL == 3 ? chains_tc_kernel<1, 1, 3> : chains_tc_kernel<1, 1, 4>; }

#if !MCMC_TC_IN_KERNEL_REFRESH
// Clusters of CL CTAs (smem bytes, threads each) that can be resident at once; 0 if none.
int cluster_capacity(int CL, size_t smem, int threads)
{
    const TcKernel k = cluster_kernel(CL);
    if (allow_max_dyn_smem(k) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)CL, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}
#endif  // !MCMC_TC_IN_KERNEL_REFRESH

}  // namespace

#if !MCMC_TC_IN_KERNEL_REFRESH
bool tc_make_plan(int max_n, int chains_per_cta, int split_terms, size_t smem_optin, bool allow_cluster,
                  TcPlan *plan)
{
    *plan = TcPlan{};
    if (max_n < 1 || max_n > kMaxN) return false;
    if (max_n > 128 && allow_cluster) {
        // three or four tiles: a cluster with one resident tile per CTA, where it fits
        const int CL = (max_n + 63) / 64, Kp = (max_n + 15) / 16 * 16, C = chains_per_cta;
        if (C == 16 || C == 32 || C == 64) {
            const TcLayout L = tc_layout(split_terms, 1, Kp, C, CL);
            // the FP64 refresh's scratch (states, one 16-row block of digits, sums) lives in the
            // A operand's shared memory
            const long long scratch = (long long)C * (Kp + 16) + 112LL * Kp + 28LL * C;
            const int ncl = L.total <= smem_optin && scratch <= (long long)split_terms * 256 * Kp
                                ? cluster_capacity(CL, L.total, 16 * C) : 0;
            if (ncl > 0) {
                plan->valid = 1;
                plan->chains_per_cta = C;
                plan->groups = 1;
                plan->m_tiles = CL;
                plan->kdim = Kp;
                plan->max_n = max_n;
                plan->split_terms = split_terms;
                plan->threads = 16 * C;
                plan->tmem_cols = pow2_at_least(C + tc_table_cols(1, C));
                plan->ctas_per_sm = 1;
                plan->smem = L.total;
                plan->cluster = CL;
                plan->max_clusters = ncl;
                return true;
            }
        }
    }
    if (chains_per_cta < 16 || chains_per_cta > 32 || chains_per_cta % 16) return false;
    if (16 * chains_per_cta > TC_MAX_THREADS) return false;
    const int MT = (max_n + 63) / 64;
    const int Kp = (max_n + 15) / 16 * 16;
    const int C = chains_per_cta;                  // chains per group (one group of threads each)
    const int Ct = tc_groups(max_n) * C;           // chains per CTA and work item
    const int S = split_terms;
    const TcLayout L = tc_layout(S, MT, Kp, Ct);
    if (L.total > smem_optin) return false;
    plan->valid = 1;
    plan->chains_per_cta = Ct;
    plan->groups = Ct / C;
    plan->m_tiles = MT;
    plan->kdim = Kp;
    plan->max_n = max_n;
    plan->split_terms = S;
    plan->threads = 16 * C;                   // 4 TMEM quadrants x C/8 column groups x 32
    plan->tmem_cols = pow2_at_least(MT * Ct + tc_table_cols(MT, C));   // accumulators + carried factors
    // resident CTAs per SM: shared memory, threads, registers (as the launch bounds allow: 64
    // per thread for one tile, 128 beyond, at the default bounds), and TMEM
    const int regs = std::min(255, (MT == 1 ? 65536 / (TC_MIN_BLOCKS * TC_MAX_THREADS)
                                            : 65536 / TC_MAX_THREADS) / 8 * 8);
    const int by_smem = (int)(228 * 1024 / (L.total + 1024));
    const int by_thr = std::min(2048 / plan->threads, 65536 / (plan->threads * regs));
    const int by_occ = std::min(by_smem, by_thr);
    const int by_tmem = 512 / plan->tmem_cols;
    plan->ctas_per_sm = std::max(1, std::min(by_occ, by_tmem));
    plan->smem = L.total;
    plan->cluster = 1;
    return true;
}

bool tc_make_plan_packed(int tile, int split_terms, size_t smem_optin, TcPlan *plan)
{
    *plan = TcPlan{};
    if (tile < 16 || tile > 32 || tile % 16 || 16 * tile > TC_MAX_THREADS) return false;
    const int Kp = 64, Ct = 2 * tile, S = split_terms;
    const TcLayout L = tc_layout(S, 1, Kp, Ct);
    if (L.total > smem_optin) return false;
    plan->valid = 1;
    plan->packed = 1;
    plan->chains_per_cta = Ct;
    plan->groups = 0;
    plan->m_tiles = 1;
    plan->kdim = Kp;
    plan->max_n = 64;
    plan->split_terms = S;
    plan->threads = 16 * tile;
    // accumulators of two groups and the carried factors of the threads' chains
    plan->tmem_cols = pow2_at_least(Ct + tc_table_cols(1, tile));
    const int regs = std::min(255, 65536 / (TC_MIN_BLOCKS * TC_MAX_THREADS) / 8 * 8);
    const int by_smem = (int)(228 * 1024 / (L.total + 1024));
    const int by_thr = std::min(2048 / plan->threads, 65536 / (plan->threads * regs));
    plan->ctas_per_sm = std::max(1, std::min(std::min(by_smem, by_thr), 512 / plan->tmem_cols));
    plan->smem = L.total;
    plan->cluster = 1;
    return true;
}

long long tc_operand_bytes(int N, int split_terms)
{
    if (N > kMaxN) return 0;
    const int MT = (N + 63) / 64, Kp = (N + 15) / 16 * 16;
    return (long long)split_terms * MT * 128 * Kp * 2;
}

cudaError_t tc_launch_pack(int split_terms, const ChannelDesc *desc, int n_channels,
                           const float *bt32, uint8_t *tc_ops, cudaStream_t s)
{
    if (n_channels <= 0) return cudaSuccess;
    pack_kernel<<<n_channels, 256, 0, s>>>(desc, bt32, tc_ops, split_terms);
    return cudaGetLastError();
}

#endif  // !MCMC_TC_IN_KERNEL_REFRESH

// The launch of a group's work items: tc_launch_chains runs the kernels without the in-run
// refresh (refresh_period must be 0 in a_in), tc_launch_chains_kr those with it.
#if MCMC_TC_IN_KERNEL_REFRESH
cudaError_t tc_launch_chains_kr(const ChainArgs &a_in, const TcPlan &plan, cudaStream_t s)
#else
cudaError_t tc_launch_chains(const ChainArgs &a_in, const TcPlan &plan, cudaStream_t s)
#endif
{
    if (a_in.n_items <= 0) return cudaSuccess;
    ChainArgs a = a_in;
    a.tc_tmem_cols = plan.tmem_cols;
    philox_round_keys(a.key0, a.key1, a.philox_rk);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e;
    if (plan.cluster > 1) {
        const int CL = plan.cluster, ncl = plan.max_clusters;
        if (ncl <= 0) return cudaErrorInvalidConfiguration;
        if ((e = allow_max_dyn_smem(cluster_kernel(CL))) != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(CL * std::min(a.n_items, ncl)), 1, 1);
        cfg.blockDim = dim3((unsigned)plan.threads, 1, 1);
        cfg.dynamicSmemBytes = plan.smem;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)CL;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, cluster_kernel(CL), a, plan.chains_per_cta, plan.split_terms, plan.kdim);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    const int grid = std::min(a.n_items, std::max(1, sms * plan.ctas_per_sm));
    auto go = [&](auto k) {
        if ((e = allow_max_dyn_smem(k)) != cudaSuccess) return e;
        k<<<grid, plan.threads, plan.smem, s>>>(a, plan.chains_per_cta, plan.split_terms, plan.kdim);
        return cudaSuccess;
    };
    switch (plan.m_tiles) {
    case 1:
        e = plan.packed ? go(chains_tc_kernel<1, 0, 1>)
                        : plan.groups == 2 ? go(chains_tc_kernel<1, 2, 1>) : go(chains_tc_kernel<1, 1, 1>);
        break;
    case 2: e = go(chains_tc_kernel<2, 1, 1>); break;
    case 3: e = go(chains_tc_kernel<3, 1, 1>); break;
    default: e = go(chains_tc_kernel<4, 1, 1>); break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace mcmcdet
