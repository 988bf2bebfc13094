// tc_plan.h -- launch plan of the tcgen05 (MIXED precision) chain kernel.
#pragma once

#include <cstdint>
#include <vector>

#include "kernels.h"

namespace mcmcdet {

struct TcPlan {
    int valid;
    int chains_per_cta;     // MMA N extent: chains of one channel per CTA (multiple of 16)
    int m_tiles;            // 128-row tiles of the A operand (interleaved Gt / P~Gt rows)
    int kdim;               // K extent: N rounded up to 16
    int max_n;
    int split_terms;        // BF16 terms of Gt (P~Gt uses the first term only)
    int threads;
    int tmem_cols;
    int ctas_per_sm;
    size_t smem;            // dynamic shared memory per CTA (bytes)
};

// Chooses the kernel shape for a batch; false if the batch cannot run on this engine.
bool tc_make_plan(const std::vector<ChannelDesc> &desc, int chains, int split_terms,
                  size_t smem_optin, int sm_count, TcPlan *plan);

// Bytes of one channel's packed BF16 operand block.
long long tc_operand_bytes(const ChannelDesc &c, const TcPlan &plan);

// Packs [Gt | P~Gt] (the FP32 CUDA-core operand, N x NOp per channel) into the BF16 split
// operand blocks in the canonical tcgen05 layout.
cudaError_t tc_launch_pack(const TcPlan &plan, const ChannelDesc *desc, int n_channels,
                           const float *bt32, uint8_t *tc_ops, cudaStream_t s);

cudaError_t tc_launch_chains(const ChainArgs &a, const TcPlan &plan, cudaStream_t s);

}  // namespace mcmcdet
