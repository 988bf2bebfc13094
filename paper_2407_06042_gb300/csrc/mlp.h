// mlp.h -- the learned proposal's network handle and its launchers (private to the library).
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

struct mcmc_mlp {
    int Q = 0;               // outputs (constellation points)
    int Qp = 0;              // Q rounded up to a multiple of 16 (tensor-core N)
    int max_rows = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    std::string err;
    long long launches = 0;
    long long adam_step = 0;
    float *params = nullptr, *grad = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    // training / CUDA-core inference workspace (max_rows rows)
    float *xg = nullptr;        // gathered features [max_rows x 6]
    int *lg = nullptr;          // gathered labels
    float *h1 = nullptr, *h2 = nullptr, *dlog = nullptr, *dh = nullptr, *logit = nullptr;
    float *rowloss = nullptr, *partial = nullptr;
    size_t partial_floats = 0;
    unsigned *status = nullptr;
    // tensor-core operand images of W2 and W3 (BF16), rebuilt when the parameters change
    uint8_t *tc_ops = nullptr;
    bool tc_valid = false;
    // the large products of a forward or training pass (hidden layer, input and weight
    // gradients) on tcgen05 with split-BF16 operands (default on sm_103), else on CUDA cores
    bool tc_train = false;
    int sm_count = 0;
};

namespace mcmcdet {

constexpr int kMlpIn = 6;
constexpr int kMlpHidden = 256;

__host__ __device__ inline long long mlp_param_count(int Q)
{
    return (long long)kMlpHidden * kMlpIn + kMlpHidden + (long long)kMlpHidden * kMlpHidden +
           kMlpHidden + (long long)Q * kMlpHidden + Q;
}
__host__ __device__ inline long long mlp_off_b1() { return (long long)kMlpHidden * kMlpIn; }
__host__ __device__ inline long long mlp_off_W2() { return mlp_off_b1() + kMlpHidden; }
__host__ __device__ inline long long mlp_off_b2() { return mlp_off_W2() + (long long)kMlpHidden * kMlpHidden; }
__host__ __device__ inline long long mlp_off_W3() { return mlp_off_b2() + kMlpHidden; }
__host__ __device__ inline long long mlp_off_b3(int Q) { return mlp_off_W3() + (long long)Q * kMlpHidden; }

// Bytes of the tensor-core operand images, BF16: W2 | b2 (256 x 272) and W3 | b3 (Qp x 272), the
// bias split into three terms in the extra K columns, and the layer-1 terms of W1 | b1 (256 x 48).
inline size_t mlp_tc_bytes(int Qp) { return (size_t)(kMlpHidden + Qp) * (kMlpHidden + 16) * 2 + (size_t)kMlpHidden * 48 * 2; }

// logits [rows x Q] of X [rows x 6]: FP32 CUDA-core kernels in chunks of max_rows rows.
cudaError_t mlp_forward_simt(mcmc_mlp *m, long long rows, const float *X, float *logits,
                             cudaStream_t s);
// The same on tcgen05 (BF16 operands, FP32 accumulation); packs the operand images if needed.
cudaError_t mlp_forward_tc(mcmc_mlp *m, long long rows, const float *X, float *logits,
                           cudaStream_t s);

}  // namespace mcmcdet
