// chains_tc_kr.cu -- the tcgen05 chain kernels of chains_tc.cu with the in-run FP64 energy
// refresh (every refresh_period transitions, MCMC_ENGINE_KERNEL_REFRESH) compiled into them.
// A second translation unit of the same source, so that the default kernels, which leave the
// refresh to a kernel between launches, carry none of its code or register pressure; it defines
// only tc_launch_chains_kr.
#define MCMC_TC_IN_KERNEL_REFRESH 1
#include "chains_tc.cu"
