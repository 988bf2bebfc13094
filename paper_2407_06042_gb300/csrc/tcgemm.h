// tcgemm.h -- FP32 matrix products on tcgen05 tensor cores with split-BF16 operands (tcgemm.cu).
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace mcmcdet {

// C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn];
// epilogue + bias(n), ReLU, or times [mask(m, n) > 0]. kchunk, partial and the vector flags are
// set by tc_gemm.
struct TcGemmArgs {
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
    int a_vec, b_vec;       // 16-byte operand loads are aligned (set by tc_gemm)
    float *partial;
    unsigned *status;       // timeout bit of a bounded wait that ran out
};

// Launches the product (split over K into `partial`, summed in split order by a second kernel,
// when K is long enough and partial has room); sms = the device's SM count; *launches = the
// kernels launched (1 or 2).
cudaError_t tc_gemm(const TcGemmArgs &g, float *partial, size_t partial_floats, int sms, cudaStream_t s,
                    int *launches);

}  // namespace mcmcdet
