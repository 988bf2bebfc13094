// tc_plan.h -- launch plan of the tcgen05 (MIXED precision) chain kernel.
#pragma once

#include <cstdint>
#include <vector>

#include "kernels.h"

namespace mcmcdet {

struct TcPlan {
    int valid;
    int chains_per_cta;     // MMA N extent: chains of one channel per CTA (multiple of 16)
    int groups;             // chain groups per CTA: 2 when N <= 32 (the operand rows held twice)
    int m_tiles;            // 128-row tiles of the A operand (interleaved Gt / P~Gt rows)
    int kdim;               // K extent: N rounded up to 16
    int max_n;
    int split_terms;        // BF16 terms of Gt (P~Gt uses the first term only)
    int threads;
    int tmem_cols;
    int ctas_per_sm;
    size_t smem;            // dynamic shared memory per CTA (bytes)
    int cluster;            // CTAs per thread-block cluster: m_tiles for N > 128 (one resident
                            // tile per CTA, chains_per_cta 16, 32 or 64), else 1
    int max_clusters;       // clusters that can be resident at once (queried when planning, so
                            // that launches, also inside a stream capture, need no query)
    int packed;             // 1: the packed kernel (one-tile items of every N <= 64 from a work
                            // queue); chains_per_cta is then two groups of the tile
};

// Kernel shape for a group of channels with the same K extent (N rounded up to 16) and tile
// count, `chains_per_cta` chains (multiple of 16) per group of threads (twice that per CTA and
// work item when N <= 32); false if it does not fit. N > 128 takes a thread-block cluster of
// one CTA per tile where allowed, its shared memory fits and such clusters can be resident (then
// 64 chains per CTA are allowed too), else the single-CTA kernel that streams the operand from L2.
bool tc_make_plan(int max_n, int chains_per_cta, int split_terms, size_t smem_optin, bool allow_cluster,
                  TcPlan *plan);

// Kernel shape of the packed launch: one persistent kernel for every channel of N <= 64 in a
// batch (one or two chain groups of `tile` chains per item, by N; K extent up to 64), whose CTAs
// pull work items from a device queue. False if it does not fit.
bool tc_make_plan_packed(int tile, int split_terms, size_t smem_optin, TcPlan *plan);

// Bytes of one channel's packed BF16 operand block (depends on its N only).
long long tc_operand_bytes(int N, int split_terms);

// Packs [Gt | P~Gt] (the FP32 CUDA-core operand, N x NOp per channel) into the BF16 split
// operand block of every channel with N <= 256, in the canonical tcgen05 layout (each block
// sized for the channel's own K extent and tile count).
cudaError_t tc_launch_pack(int split_terms, const ChannelDesc *desc, int n_channels,
                           const float *bt32, uint8_t *tc_ops, cudaStream_t s);

// Launches the chain kernels of a plan for a.n_items work items. tc_launch_chains: kernels
// without the in-run FP64 refresh (a.refresh_period must be 0: the caller refreshes between
// launches); tc_launch_chains_kr: the same kernels with the refresh every a.refresh_period
// transitions inside them.
cudaError_t tc_launch_chains(const ChainArgs &a, const TcPlan &plan, cudaStream_t s);
cudaError_t tc_launch_chains_kr(const ChainArgs &a, const TcPlan &plan, cudaStream_t s);

}  // namespace mcmcdet
