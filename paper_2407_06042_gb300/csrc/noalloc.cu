// noalloc.cu -- one-call detection of a small batch that allocates no device memory.
//
// Some callers cannot call cudaMalloc: real-time loops that must never block on the allocator,
// hosts whose device memory is carved up in advance by a pool they do not control, and
// components whose device memory budget is fixed when they start. For them this entry point runs
// the whole FP32 detection (preparation, chains, read-out) with every intermediate buffer taken
// from one fixed array in device global memory, declared below at file scope. The array exists
// on every GPU that loads this library, from load until the process exits.
//
// The caller still owns the inputs (H, y, noise variances) and the outputs (labels, LLRs,
// energies). The array is shared by every call on a device and keeps the contents of the last
// call: each call re-initialises everything it reads (the status word, the acceptance counters,
// the chain states), and calls that overlap on the GPU race with each other.
#include "../../include/mcmcdet.h"

#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace mcmcdet;

namespace {

// The fixed scratch of the no-allocation entry point (size: MCMC_NOALLOC_SCRATCH_BYTES).
__device__ __align__(256) unsigned char g_noalloc_scratch[MCMC_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per CUDA context. In host code the symbol's name is only a
// host-side stand-in, never a device address: the real address is looked up (with the context
// current) the first time a call runs in a context, and kept for that context. A context that is
// destroyed (cudaDeviceReset) and a new one created at the same handle value has a new unique
// id, so entries are matched on both and the new context gets its own lookup.
struct ScratchEntry {
    CUcontext ctx;
    unsigned long long ctx_id;
    void *addr;
};
std::vector<ScratchEntry> g_scratch_addr;
std::mutex g_scratch_mu;

// The two driver calls used to identify the current context, looked up through the runtime (the
// library does not link against the driver, so it also loads on machines without one).
using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

cudaError_t current_context(CUcontext *ctx, unsigned long long *id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *p0 = nullptr, *p1 = nullptr;
        cudaDriverEntryPointQueryResult q0{}, q1{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p0, 4000, cudaEnableDefault, &q0);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &p1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess || !p0 || !p1) return e != cudaSuccess ? e : cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(p0);
        get_id = reinterpret_cast<CtxGetIdFn>(p1);
    }
    *ctx = nullptr;
    if (get_current(ctx) != CUDA_SUCCESS || !*ctx) return cudaErrorInvalidDevice;
    return get_id(*ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidDevice;
}

cudaError_t scratch_address(unsigned char **out)
{
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (current_context(&ctx, &id) != cudaSuccess) {
        // no context current yet: the runtime call makes the current device's primary context
        // current (and loads this library's module on it)
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        const cudaError_t c = current_context(&ctx, &id);
        if (c != cudaSuccess) return c;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    for (const ScratchEntry &e : g_scratch_addr)
        if (e.ctx == ctx && e.ctx_id == id) {
            *out = static_cast<unsigned char *>(e.addr);
            return cudaSuccess;
        }
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr.push_back(ScratchEntry{ctx, id, p});
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

// sigma^2-dependent constants of every channel (same formulas as the handle-based path).
__global__ void noalloc_desc_kernel(ChannelDesc *desc, const float *noise_var, int n,
                                    double alpha_scale, double tau, int preconditioned,
                                    unsigned *status)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    ChannelDesc &c = desc[b];
    const double s2 = noise_var[b];
    if (!(s2 > 0.0) || !isfinite(s2)) {
        atomicOr(status, kStatusNumeric);
        c.sigma2 = 1.0;
    } else {
        c.sigma2 = s2;
    }
    const double d2 = c.dmin * c.dmin;
    const double alpha = alpha_scale * c.sigma2;
    c.tau = tau;
    c.inv_s2 = 1.0 / c.sigma2;
    c.cf = 1.0 / (tau * c.sigma2);
    if (preconditioned) {
        const double beta = d2 / c.sigma2;
        c.clin = 2.0 * d2 / (beta * tau * c.sigma2);
        c.cquad = 2.0 * d2 / (alpha * beta);
        c.gamma_t = d2 * (c.sigma2 / (2.0 * d2));
    } else {
        c.clin = 2.0 / (tau * c.sigma2);
        c.cquad = 2.0 * d2 / alpha;
        c.gamma_t = 0.0;
    }
}

struct Carver {
    unsigned char *base;
    size_t off = 0;
    template <typename T> T *take(size_t count)
    {
        off = (off + 255) / 256 * 256;
        T *p = reinterpret_cast<T *>(base + off);
        off += std::max<size_t>(count * sizeof(T), 1);
        return p;
    }
};

}  // namespace

extern "C" mcmc_status mcmc_detect_noalloc(int32_t n_channels, const int32_t *nt,
                                           const int32_t *nr, const int32_t *qam, const void *H,
                                           const int64_t *H_off, const void *y,
                                           const int64_t *y_off, const float *noise_var,
                                           int32_t chains, int32_t iterations, uint64_t seed,
                                           int32_t preconditioned, float alpha_scale, float tau,
                                           int8_t *best_idx, float *llr, double *best_f,
                                           void *stream)
{
    if (n_channels < 1 || !nt || !nr || !qam || !H || !H_off || !y || !y_off || !noise_var)
        return MCMC_EINVAL;
    if (chains < 4 || chains > 1024 || (chains % 4) != 0 || iterations < 0 ||
        (preconditioned != 0 && preconditioned != 1) || !(alpha_scale > 0.f) ||
        !std::isfinite(alpha_scale) || !(tau >= 1.f) || !std::isfinite(tau))
        return MCMC_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int Np = chains;
    const bool pre = preconditioned != 0;

    // per-channel descriptors (host)
    std::vector<ChannelDesc> desc(n_channels);
    long long st = 0, mat = 0, bt = 0, vec = 0, bits = 0, ant = 0;
    int maxn = 0, maxnop = 0, maxnt = 0, maxnr = 0;
    for (int b = 0; b < n_channels; ++b) {
        const int L = qam[b] == 4 ? 2 : qam[b] == 16 ? 4 : qam[b] == 64 ? 8 : 0;
        if (!L || nt[b] < 1 || 2 * nt[b] > kMaxN || nr[b] < 1 || nr[b] > 4096 || H_off[b] < 0 ||
            y_off[b] < 0)
            return MCMC_EINVAL;
        ChannelDesc &c = desc[b];
        std::memset(&c, 0, sizeof c);
        c.N = 2 * nt[b];
        c.L = L;
        c.log2L = L == 2 ? 1 : L == 4 ? 2 : 3;
        c.Nt = nt[b];
        c.Nr = nr[b];
        c.NO = pre ? 2 * c.N : c.N;
        c.NOp = (c.NO + 7) / 8 * 8;
        c.state_off = st;
        c.mat_off = mat;
        c.bt_off = bt;
        c.vec_off = vec;
        c.bit_off = bits;
        c.ant_off = ant;
        c.h_off = H_off[b];
        c.y_off = y_off[b];
        c.dmin = std::sqrt(3.0 / (2.0 * (qam[b] - 1)));
        st += (long long)Np * c.N;
        mat += (long long)c.N * c.N;
        bt += (long long)c.N * c.NOp;
        vec += c.N;
        bits += (long long)c.N * c.log2L;
        ant += c.Nt;
        maxn = std::max(maxn, c.N);
        maxnop = std::max(maxnop, c.NOp);
        maxnt = std::max(maxnt, c.Nt);
        maxnr = std::max(maxnr, c.Nr);
    }
    // CUDA-core FP32 chain kernel plan (shared-memory budget as in the handle-based path)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return MCMC_EUNSUPPORTED;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return MCMC_ECUDA;
    const size_t budget = std::min<size_t>((size_t)optin, 110 * 1024);
    bool bt_smem = true;
    int cg = std::min(64, (Np + 7) / 8 * 8);
    for (;;) {
        const size_t need = chain_smem_bytes_simt(4, cg, maxn, maxnop, bt_smem);
        if (need <= budget) break;
        if (bt_smem && (size_t)maxn * maxnop * 4 > budget / 2) { bt_smem = false; continue; }
        if (cg > 8) { cg -= 8; continue; }
        if (bt_smem) { bt_smem = false; continue; }
        return MCMC_EUNSUPPORTED;
    }
    std::vector<WorkItem> items;
    for (int b = 0; b < n_channels; ++b)
        for (int c0 = 0; c0 < Np; c0 += cg) items.push_back(WorkItem{b, c0, std::min(cg, Np - c0), 0});

    // carve the fixed scratch; requests that do not fit are rejected before any work
    unsigned char *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return MCMC_ECUDA;
    }
    // FP32 Gauss-Jordan block and the copies of its pivot row and column (always in shared
    // memory, also when the block itself lives in global memory)
    const size_t gj_stage = (size_t)(maxnt * maxnt + 2 * maxnt) * 8;
    const bool stage_gj = pre && gj_stage <= std::min<size_t>((size_t)optin, 160 * 1024);
    Carver cv{scratch};
    const long long ntc = mat / 4;
    ChannelDesc *d_desc = cv.take<ChannelDesc>(n_channels);
    WorkItem *d_items = cv.take<WorkItem>(items.size());
    unsigned *d_misc = cv.take<unsigned>(64);
    double *d_Gc = cv.take<double>(2 * ntc);
    double *d_zc = cv.take<double>(vec);
    double *d_Mc = pre ? cv.take<double>(2 * ntc) : nullptr;
    double *d_gj = (pre && !stage_gj) ? cv.take<double>(4 * ntc) : nullptr;
    double *d_yy = cv.take<double>(n_channels);
    double *d_G64 = cv.take<double>(mat);
    double *d_z64 = cv.take<double>(vec);
    double *d_w64 = cv.take<double>(vec);
    float *d_z32 = cv.take<float>(vec);
    float *d_w32 = cv.take<float>(vec);
    float *d_bt32 = cv.take<float>(bt);
    int8_t *d_states = cv.take<int8_t>(st);
    int8_t *d_best_states = cv.take<int8_t>(st);
    double *d_f = cv.take<double>((size_t)n_channels * Np);
    double *d_best_f = cv.take<double>((size_t)n_channels * Np);
    unsigned long long *d_acc = cv.take<unsigned long long>((size_t)n_channels * Np);
    float *d_dexp = cv.take<float>(st);
    if (cv.off > (size_t)MCMC_NOALLOC_SCRATCH_BYTES) return MCMC_EINVAL;
    unsigned *status = d_misc;
    unsigned long long *drift = reinterpret_cast<unsigned long long *>(d_misc + 2);

#define NA_CK(call)                                       \
    do {                                                  \
        if ((call) != cudaSuccess) {                      \
            cudaGetLastError();                           \
            return MCMC_ECUDA;                            \
        }                                                 \
    } while (0)

    NA_CK(cudaMemcpyAsync(d_desc, desc.data(), sizeof(ChannelDesc) * n_channels,
                          cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemcpyAsync(d_items, items.data(), sizeof(WorkItem) * items.size(),
                          cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemsetAsync(d_misc, 0, 64 * sizeof(unsigned), s));
    NA_CK(cudaMemsetAsync(d_acc, 0, 8 * (size_t)n_channels * Np, s));
    noalloc_desc_kernel<<<(n_channels + 127) / 128, 128, 0, s>>>(d_desc, noise_var, n_channels,
                                                                 alpha_scale, tau, pre, status);
    NA_CK(cudaGetLastError());

    PrepArgs pa{};
    pa.desc = d_desc;
    pa.H = static_cast<const float2 *>(H);
    pa.y = static_cast<const float2 *>(y);
    pa.Gc = d_Gc;
    pa.zc = d_zc;
    pa.Mc = d_Mc;
    pa.gj = d_gj;
    pa.yy = d_yy;
    pa.G64 = d_G64;
    pa.GM64 = nullptr;   // FP32 mode: the preconditioned operand is emitted straight to FP32
    pa.z64 = d_z64;
    pa.w64 = d_w64;
    pa.z32 = d_z32;
    pa.w32 = d_w32;
    pa.bt32 = d_bt32;
    pa.bt64 = nullptr;
    pa.status = status;
    const size_t h_stage = 8 * (size_t)(maxnt * maxnr + maxnr);
    pa.stage_h = h_stage <= std::min<size_t>((size_t)optin, 128 * 1024);
    pa.stage_gj = stage_gj;
    pa.precond_fp32 = 1;
    pa.max_nt = maxnt;   // the register-tiled Gauss-Jordan for Nt <= 64, as the handle path picks
    NA_CK(launch_prep(pa, n_channels, h_stage, stage_gj ? gj_stage : (size_t)(2 * maxnt) * 8, pre, s));

    InitArgs ia{};
    ia.desc = d_desc;
    ia.states = d_states;
    ia.n_channels = n_channels;
    ia.chains = Np;
    ia.items_per_channel = (long long)(Np / 4) * maxn;
    ia.key0 = (uint32_t)(seed & 0xFFFFFFFFu);
    ia.key1 = (uint32_t)(seed >> 32);
    NA_CK(launch_init_states(ia, s));

    // exact energies of the initial states; the running best starts there
    RefreshArgs ra{};
    ra.desc = d_desc;
    ra.states = d_states;
    ra.G64 = d_G64;
    ra.z64 = d_z64;
    ra.yy = d_yy;
    ra.f = d_f;
    ra.best_f = d_best_f;
    ra.best_states = d_best_states;
    ra.status = status;
    ra.n_channels = n_channels;
    ra.chains = Np;
    ra.reset_best = 1;
    ra.max_n = maxn;
    NA_CK(launch_refresh(ra, s));

    if (iterations > 0) {
        ChainArgs ca{};
        ca.desc = d_desc;
        ca.items = d_items;
        ca.n_items = (int)items.size();
        ca.chains = Np;
        ca.cg = cg;
        ca.max_n = maxn;
        ca.max_nop = maxnop;
        ca.bt_in_smem = bt_smem;
        ca.iterations = iterations;
        ca.t_offset = 0;
        ca.refresh_period = 0;
        ca.key0 = ia.key0;
        ca.key1 = ia.key1;
        ca.bt = d_bt32;
        ca.z = d_z32;
        ca.w = d_w32;
        ca.G64 = d_G64;
        ca.z64 = d_z64;
        ca.yy = d_yy;
        ca.states = d_states;
        ca.best_states = d_best_states;
        ca.f = d_f;
        ca.best_f = d_best_f;
        ca.accepts = d_acc;
        ca.drift_bits = drift;
        ca.status = status;
        ca.init_f = 0;
        ca.dexp = d_dexp;
        NA_CK(launch_chains_simt(ca, false, chain_smem_bytes_simt(4, cg, maxn, maxnop, bt_smem), s));
        // exact energies of the final states (the chains tracked them in FP32 steps)
        ra.reset_best = 0;
        ra.best_f = nullptr;
        ra.best_states = nullptr;
        NA_CK(launch_refresh(ra, s));
    }

    EstimateArgs ea{};
    ea.desc = d_desc;
    ea.states = d_states;
    ea.best_states = d_best_states;
    ea.f = d_f;
    ea.best_f = d_best_f;
    ea.G = d_bt32;
    ea.g_is_bt = 1;
    ea.dexp = iterations > 0 ? d_dexp : nullptr;
    ea.z = d_z32;
    ea.G64 = d_G64;
    ea.z64 = d_z64;
    ea.yy = d_yy;
    ea.n_channels = n_channels;
    ea.chains = Np;
    ea.best_idx = best_idx;
    ea.llr = llr;
    ea.best_f_out = best_f;
    ea.status = status;
    NA_CK(launch_estimate(ea, false, s));

    unsigned hs = 0;
    NA_CK(cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
    if (hs & kStatusBadState) return MCMC_EINVAL;
    if (hs & kStatusTimeout) return MCMC_ETIMEOUT;
    if (hs & kStatusNumeric) return MCMC_ENUMERIC;
    return MCMC_OK;
}
