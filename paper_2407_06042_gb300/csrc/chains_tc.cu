// chains_tc.cu -- tcgen05 chain kernel (MIXED precision). Placeholder plan: not yet available.
#include "tc_plan.h"

namespace mcmcdet {

bool tc_make_plan(const std::vector<ChannelDesc> &, int, int, size_t, int, TcPlan *plan)
{
    *plan = TcPlan{};
    return false;
}

long long tc_operand_bytes(const ChannelDesc &, const TcPlan &) { return 0; }

cudaError_t tc_launch_pack(const TcPlan &, const ChannelDesc *, int, const double *, const double *,
                           uint8_t *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t tc_launch_chains(const ChainArgs &, const TcPlan &, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace mcmcdet
