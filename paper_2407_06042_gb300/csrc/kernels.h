// kernels.h -- argument blocks and host launchers shared by the CUDA translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mcmcdet {

struct PrepArgs {
    const ChannelDesc *desc;
    const float2 *H;        // packed complex channels (FP32)
    const float2 *y;        // packed received vectors (FP32)
    double *Gc;             // complex Gram matrices, Nt^2 complex per channel (scratch)
    double *zc;             // complex matched filters, Nt complex per channel (scratch)
    double *Mc;             // complex (G + gamma I)^{-1}, Nt^2 complex per channel (scratch)
    double *gj;             // Gauss-Jordan block in global memory when not staged (scratch)
    double *yy;             // ||y||^2 per channel
    double *G64;            // Gt, N x N per channel
    double *GM64;           // P~ Gt, N x N per channel (preconditioned)
    double *z64, *w64;      // zt, wt (FP64)
    float *z32, *w32;       // zt, wt (FP32)
    float *bt32;            // CUDA-core GEMM operand (FP32), N x NOp per channel, or null
    double *bt64;           // CUDA-core GEMM operand (FP64), or null
    unsigned *status;
    int stage_h;            // stage H and y in shared memory
    int stage_gj;           // factorise the preconditioner in shared memory
    int precond_fp32;       // FP32 Gauss-Jordan (FP32 / MIXED modes) instead of FP64
    int max_nt;             // largest Nt of the batch (0: unknown)
};

struct InitArgs {
    const ChannelDesc *desc;
    int8_t *states;
    int n_channels;
    int chains;
    long long items_per_channel;   // (chains / 4) * max N
    uint32_t key0, key1;
};

struct RefreshArgs {
    const ChannelDesc *desc;
    const int8_t *states;
    const double *G64;
    const double *z64;
    const double *yy;
    double *f;
    double *best_f;
    int8_t *best_states;
    unsigned *status;
    int n_channels;
    int chains;
    int reset_best;
    int max_n;              // largest N of the batch (sizes the launch; 0: kMaxN)
    // or null: max |f_old - f| and max |f_old - f| / |f| over the chains (ordered bits), the
    // correction this refresh makes to the energies the chains tracked
    unsigned long long *drift_bits;
    unsigned long long *drift_rel_bits;
};

// One chain-kernel work item: chains [c0, c0 + nc) of channel b.
struct WorkItem {
    int b;
    int c0;
    int nc;
    int pad;
};

struct ChainArgs {
    const ChannelDesc *desc;
    const WorkItem *items;
    int n_items;
    int chains;             // Np
    int cg;                 // chains per work item (capacity of the shared-memory arrays)
    int max_n;              // largest N in the batch
    int max_nop;            // largest NOp in the batch
    int bt_in_smem;         // copy the GEMM operand to shared memory
    int iterations;
    long long t_offset;
    int refresh_period;
    uint32_t key0, key1;
    const void *bt;         // float* or double* operand (N x NOp per channel)
    const void *z;          // float* or double* zt
    const void *w;          // float* or double* wt
    const double *G64;      // FP64 Gt for the periodic refresh
    const double *z64;
    const double *yy;
    int8_t *states;
    int8_t *best_states;
    double *f;
    double *best_f;
    unsigned long long *accepts;
    unsigned long long *drift_bits;   // max |f_tracked - f_fp64| as ordered bits
    unsigned *status;
    int init_f;             // derive the tracked energies of the current states from the first
                            // GEMM (FP32 / MIXED) and restart the running best from them
    float *dexp;            // Gt x of the final states (FP32), same layout as the states
    unsigned long long *near_ties;   // [3] MH decisions with |log A - log u| below 1e-6, 1e-4 and
                                     // 1e-2 (natural log), as the kernel evaluated them
    double *trace;          // or null: per chain (channel-major) the log acceptance ratio and log u
                            // (natural log) of its latest transition, as pairs
    // tcgen05 engine only
    const uint8_t *tc_ops;  // per-channel packed BF16 operand blocks
    int split_terms;
    int tc_tmem_cols;       // TMEM columns each CTA allocates
    int *queue;             // packed kernel: the next work item to hand out (zero at launch)
    uint32_t philox_rk[2 * kPhiloxRounds];   // round keys of (key0, key1), set at launch
};

struct ListLlrArgs {
    const ChannelDesc *desc;
    const int8_t *states;
    const double *f;        // FP64 energies of the states
    int n_channels;
    int chains;
    float clip;
    float *llr;
    unsigned *status;
};

struct EstimateArgs {
    const ChannelDesc *desc;
    const int8_t *states;
    const int8_t *best_states;
    const double *f;
    const double *best_f;
    const void *G;          // float* or double* Gt (N x N per channel), or the Bt operand
    const float *dexp;      // Gt x of every chain's state from the chain kernel (FP32), or null
    int g_is_bt;            // G points at the N x NOp operand (row stride NOp)
    const void *z;          // float* or double* zt
    const double *G64;
    const double *z64;
    const double *yy;
    int n_channels;
    int chains;
    int8_t *best_idx;       // out
    float *llr;             // out
    double *best_f_out;     // out
    unsigned *status;
};

// Learned proposal: Gram products and features at a set of states (one kernel), and the
// mixture move / warm start kernels.
struct MixGramArgs {
    const ChannelDesc *desc;
    int chains;
    int L;                  // channels with this many levels (0: every channel)
    const float *bt32;      // [Gt | P~ Gt] FP32 operand, N x NOp per channel
    const float *z32, *w32;
    const int8_t *x;        // states the products are taken at
    float *gx, *px;         // out: Gt x, P~ Gt x (state layout)
    float *X;               // out: features [rows x 6], or null
};

struct MixStepArgs {
    const ChannelDesc *desc;
    int chains;
    int L;                  // the network's channels: L levels, Q = L^2 outputs
    const float *z32, *w32;
    const int8_t *states;   // x
    int8_t *states_out;     // next state (may alias states)
    int8_t *prop;           // x'
    const float *gx, *px;   // products at x
    const float *gxp, *pxp; // products at x'
    const float *logits;    // network logits at x (propose), at x' (accept), at 0 (warm start)
    float *lqf;             // log2 q_mix(x' | x) per (chain, antenna)
    float lambda;
    float l2w_plain, l2w_nn;   // log2(1 - lambda), log2(lambda)
    uint32_t t;
    uint32_t key0, key1;
    double *f, *best_f;
    int8_t *best_states;
    unsigned long long *accepts;
    unsigned *status;
};

cudaError_t launch_gram_features(const MixGramArgs &a, int n_channels, cudaStream_t s);
cudaError_t launch_features_zero(const MixGramArgs &a, int n_channels, int max_nt, cudaStream_t s);
// which: 0 propose, 1 accept, 2 warm start
cudaError_t launch_mix(int which, const MixStepArgs &a, int n_channels, int max_nt, cudaStream_t s);

size_t chain_smem_bytes_simt(int elem_size, int cg, int max_n, int max_nop, bool bt_in_smem);

cudaError_t launch_prep(const PrepArgs &a, int n_channels, size_t h_stage_bytes,
                        size_t gj_stage_bytes, bool preconditioned, cudaStream_t s);
cudaError_t launch_init_states(const InitArgs &a, cudaStream_t s);
cudaError_t launch_refresh(const RefreshArgs &a, cudaStream_t s);
cudaError_t launch_chains_simt(const ChainArgs &a, bool fp64, size_t smem, cudaStream_t s);
cudaError_t launch_estimate(const EstimateArgs &a, bool fp64, cudaStream_t s);
cudaError_t launch_list_llr(const ListLlrArgs &a, bool fp64, cudaStream_t s);

}  // namespace mcmcdet
