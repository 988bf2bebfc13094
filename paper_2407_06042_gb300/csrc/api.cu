// api.cu -- host side of the C ABI declared in include/mcmcdet.h: handle, argument checks,
// workspace management, batch planning and kernel launches. No torch types, no exceptions
// across the ABI.
#include "../../include/mcmcdet.h"
#include "../../include/mcmcdet_learned.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "mlp.h"
#include "tc_plan.h"

using namespace mcmcdet;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
};

// One chain-kernel launch: channels of one shape class on one engine.
struct Group {
    int engine = 0;            // MCMC_ENGINE_SIMT or MCMC_ENGINE_TC
    int tile = 0;              // TC: chains per CTA; SIMT: chains per work item
    TcPlan plan{};             // TC
    bool bt_smem = false;      // SIMT: GEMM operand staged in shared memory
    size_t smem = 0;           // SIMT: dynamic shared memory
    int max_n = 0, max_nop = 0;
    bool packed = false;       // TC: the packed kernel over several one-tile shape classes
    std::vector<WorkItem> items;
    DevBuf d_items;
};

// Engine choice of one shape class.
struct Choice {
    int engine = 0;
    int tile = 0;
};

}  // namespace

struct mcmc_detector {
    mcmc_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // a run with several launch groups forks them onto these streams (parallel graph branches)
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    // start / end of the chain kernels of the latest runs (the refreshes around them excluded)
    static constexpr int kRunSlots = 64;
    cudaEvent_t ev_run[kRunSlots][2] = {};
    long long runs = 0;
    int device = 0;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    size_t smem_optin = 0;
    std::string err;
    long long launches = 0;

    // batch state
    bool prepared = false;
    int n_channels = 0;
    std::vector<ChannelDesc> desc;
    std::vector<Choice> choice;     // per channel
    std::vector<Group> groups;
    std::vector<DevBuf> spare_items;   // work-item buffers of earlier batches, reused
    cudaGraphExec_t graph = nullptr;
    int tuned_classes = 0;
    int max_n = 0, max_nop = 0, max_nt = 0, max_nr = 0;
    long long tot_states = 0, tot_mat = 0, tot_bt = 0, tot_vec = 0, tot_bits = 0, tot_ant = 0;
    long long tot_tc = 0;
    long long transitions = 0;
    bool f_valid = false;   // tracked energies hold the current states' values
    bool f_exact = true;    // ... to FP64 accuracy (FP32 / MIXED runs track them in FP32 steps)
    bool d_valid = false;   // d_dexp holds Gt x of the current states

    // device workspace
    DevBuf d_desc, d_Gc, d_zc, d_Mc, d_gj, d_yy, d_G64, d_GM64, d_z64, d_w64, d_z32,
        d_w32, d_bt32, d_bt64, d_tc, d_states, d_best_states, d_f, d_best_f, d_accepts,
        d_misc, d_in_H, d_in_y, d_in_s2, d_out_idx, d_out_llr, d_out_bf, d_dexp, d_fx, d_trace,
        d_queue;
    HostBuf h_stage;
    // pinned staging ring for the per-batch tables (descriptors, work items): a slot is rewritten
    // only after the copy that last read it has completed
    static constexpr int kUpSlots = 4;
    HostBuf h_up[kUpSlots];
    cudaEvent_t up_done[kUpSlots] = {};
    int up_next = 0;

    // learned proposal (not owned network; scratch of the mixture move)
    mcmc_mlp *mlp = nullptr;
    float mix_lambda = 0.f;
    int mix_tc = 0;
    DevBuf d_mx_gx, d_mx_px, d_mx_gxp, d_mx_pxp, d_mx_prop, d_mx_X, d_mx_logits, d_mx_lqf;
};

namespace {

mcmc_status fail(mcmc_detector *d, mcmc_status s, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

mcmc_status fail(mcmc_detector *d, mcmc_status s, const char *fmt, ...)
{
    if (d) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        d->err = buf;
    }
    return s;
}

mcmc_status cuda_fail(mcmc_detector *d, cudaError_t e, const char *what)
{
    return fail(d, e == cudaErrorMemoryAllocation ? MCMC_ENOMEM : MCMC_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return cuda_fail(d, e_, what);   \
    } while (0)

cudaError_t ensure(DevBuf &b, size_t bytes)
{
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

cudaError_t ensure_host(HostBuf &b, size_t bytes)
{
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMallocHost(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

template <typename T> T *P(DevBuf &b) { return reinterpret_cast<T *>(b.p); }

int log2_levels(int L) { return L == 2 ? 1 : L == 4 ? 2 : L == 8 ? 3 : -1; }

bool is_pinned_or_device(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeHost || at.type == cudaMemoryTypeDevice ||
           at.type == cudaMemoryTypeManaged;
}

// Host-to-device copy of a host table built by the library (descriptors, work items) through the
// pinned staging ring. A copy from pageable memory would first wait for all work queued on the
// stream; this one waits, at most, for the copy issued kUpSlots uploads earlier.
cudaError_t upload(mcmc_detector *d, void *dst, const void *src, size_t bytes)
{
    if (bytes == 0) return cudaSuccess;
    const int k = d->up_next;
    d->up_next = (k + 1) % mcmc_detector::kUpSlots;
    cudaError_t e;
    if (!d->up_done[k]) {
        if ((e = cudaEventCreateWithFlags(&d->up_done[k], cudaEventDisableTiming)) != cudaSuccess) return e;
    } else if ((e = cudaEventSynchronize(d->up_done[k])) != cudaSuccess) {
        return e;
    }
    if ((e = ensure_host(d->h_up[k], bytes)) != cudaSuccess) return e;
    std::memcpy(d->h_up[k].p, src, bytes);
    if ((e = cudaMemcpyAsync(dst, d->h_up[k].p, bytes, cudaMemcpyHostToDevice, d->stream)) != cudaSuccess)
        return e;
    return cudaEventRecord(d->up_done[k], d->stream);
}

// Host-to-device copy: direct from pinned memory, else through the handle's pinned staging
// buffer (the call blocks only for the memcpy into the staging buffer).
cudaError_t h2d(mcmc_detector *d, void *dst, const void *src, size_t bytes, size_t stage_off)
{
    if (bytes == 0) return cudaSuccess;
    if (is_pinned_or_device(src)) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, d->stream);
    std::memcpy(static_cast<char *>(d->h_stage.p) + stage_off, src, bytes);
    return cudaMemcpyAsync(dst, static_cast<char *>(d->h_stage.p) + stage_off, bytes,
                           cudaMemcpyHostToDevice, d->stream);
}

mcmc_status ensure_energies(mcmc_detector *d);
mcmc_status fp64_energies(mcmc_detector *d, const double **out);
mcmc_status refresh_energies(mcmc_detector *d, double *f, bool reset_best, bool measure);

mcmc_status read_status(mcmc_detector *d)
{
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, P<unsigned>(d->d_misc), sizeof st, cudaMemcpyDeviceToHost, d->stream),
       "status read");
    CK(cudaStreamSynchronize(d->stream), "stream synchronize");
    if (st & kStatusBadState) return fail(d, MCMC_EINVAL, "chain state level out of range");
    if (st & kStatusTimeout) return fail(d, MCMC_ETIMEOUT, "bounded device wait expired");
    if (st & kStatusNumeric) return fail(d, MCMC_ENUMERIC, "non-finite value on the device");
    return MCMC_OK;
}

// misc block layout: [0] status (unsigned), [8] drift bits (u64), [16] relative drift bits (u64),
// [32] near-tie counts (3 x u64)
unsigned *status_ptr(mcmc_detector *d) { return P<unsigned>(d->d_misc); }
unsigned long long *drift_ptr(mcmc_detector *d) { return reinterpret_cast<unsigned long long *>(P<char>(d->d_misc) + 8); }
unsigned long long *drift_rel_ptr(mcmc_detector *d) { return reinterpret_cast<unsigned long long *>(P<char>(d->d_misc) + 16); }
unsigned long long *ties_ptr(mcmc_detector *d) { return reinterpret_cast<unsigned long long *>(P<char>(d->d_misc) + 32); }

__global__ void finalize_desc_kernel(ChannelDesc *desc, const float *noise_var, int n,
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
        c.gamma_t = d2 * (c.sigma2 / (2.0 * d2));   // gamma d^2 with gamma = sigma^2 / (2 dmin^2)
    } else {
        c.clin = 2.0 / (tau * c.sigma2);
        c.cquad = 2.0 * d2 / alpha;
        c.gamma_t = 0.0;
    }
}

}  // namespace

namespace {

// Energies of the current states, evaluated exactly (refresh.cu) into `f`: the tracked energies
// (d_f) or a scratch buffer. reset_best restarts every chain's running best at its current state;
// measure records the correction made to the tracked values in the drift statistics.
mcmc_status refresh_energies(mcmc_detector *d, double *f, bool reset_best, bool measure)
{
    RefreshArgs ra{};
    ra.desc = P<ChannelDesc>(d->d_desc);
    ra.states = P<int8_t>(d->d_states);
    ra.G64 = P<double>(d->d_G64);
    ra.z64 = P<double>(d->d_z64);
    ra.yy = P<double>(d->d_yy);
    ra.f = f;
    ra.best_f = reset_best ? P<double>(d->d_best_f) : nullptr;
    ra.best_states = reset_best ? P<int8_t>(d->d_best_states) : nullptr;
    ra.status = status_ptr(d);
    ra.n_channels = d->n_channels;
    ra.chains = d->cfg.chains;
    ra.reset_best = reset_best ? 1 : 0;
    ra.max_n = d->max_n;
    ra.drift_bits = measure ? drift_ptr(d) : nullptr;
    ra.drift_rel_bits = measure ? drift_rel_ptr(d) : nullptr;
    CK(launch_refresh(ra, d->stream), "energies");
    d->launches++;
    return MCMC_OK;
}

// Exact energies of the current states (and a restart of the running best) when the tracked
// energies are not valid: after a warm start without a run in between.
mcmc_status ensure_energies(mcmc_detector *d)
{
    if (d->f_valid) return MCMC_OK;
    mcmc_status st = refresh_energies(d, P<double>(d->d_f), true, false);
    if (st != MCMC_OK) return st;
    d->f_valid = true;
    d->f_exact = true;
    return MCMC_OK;
}

// Exact evaluations of the current states' energies for read-outs that need them. When the tracked
// energies are exact they are handed out directly; otherwise the values are computed into a
// scratch buffer and the tracked energies (which the IS-LLR and the running best read) stay as the
// chains left them.
mcmc_status fp64_energies(mcmc_detector *d, const double **out)
{
    if (d->f_valid && d->f_exact) {
        *out = P<double>(d->d_f);
        return MCMC_OK;
    }
    CK(ensure(d->d_fx, 8 * (size_t)d->n_channels * d->cfg.chains), "alloc FP64 energies");
    mcmc_status st = refresh_energies(d, P<double>(d->d_fx), false, false);
    if (st != MCMC_OK) return st;
    *out = P<double>(d->d_fx);
    return MCMC_OK;
}

// ---- shape classes, engine choice, autotuner --------------------------------------------
using ClassKey = std::tuple<int, int, int, int, int, int, int>;   // N, L, Np, prec, pre, S, engine cfg
std::map<ClassKey, Choice> g_tuned;                               // process-wide tuning results
std::mutex g_tuned_mu;

ClassKey class_key(const mcmc_detector *d, const ChannelDesc &c)
{
    return ClassKey{c.N, c.L, d->cfg.chains, d->cfg.precision, d->cfg.preconditioned,
                    d->cfg.split_terms, d->cfg.engine & (3 | MCMC_ENGINE_NO_CLUSTER)};
}

// SIMT launch shape for chains-per-item cg: whether the operand fits shared memory and the size.
bool simt_fit(const mcmc_detector *d, int cg, int max_n, int max_nop, bool *bt_smem, size_t *smem)
{
    const int es = d->cfg.precision == MCMC_PREC_FP64 ? 8 : 4;
    const size_t budget = std::min<size_t>(d->smem_optin, 110 * 1024);
    for (int s = 0; s < 2; ++s) {
        const bool bs = s == 0;
        if (bs && (size_t)max_n * max_nop * es > budget / 2) continue;
        const size_t need = chain_smem_bytes_simt(es, cg, max_n, max_nop, bs);
        if (need <= budget) { *bt_smem = bs; *smem = need; return true; }
    }
    return false;
}

int simt_default_tile(const mcmc_detector *d, int max_n, int max_nop)
{
    for (int cg = std::min(64, (d->cfg.chains + 7) / 8 * 8); cg >= 8; cg -= 8) {
        bool bs;
        size_t sm;
        if (simt_fit(d, cg, max_n, max_nop, &bs, &sm)) return cg;
    }
    return 0;
}

Choice default_choice(const mcmc_detector *d, const ChannelDesc &c)
{
    const int eng = d->cfg.engine & 3;
    if (d->cfg.precision == MCMC_PREC_MIXED && c.N <= kMaxN && eng != MCMC_ENGINE_SIMT)
        return Choice{MCMC_ENGINE_TC, d->cfg.tile ? d->cfg.tile : 32};
    if (eng == MCMC_ENGINE_SIMT && d->cfg.tile) return Choice{MCMC_ENGINE_SIMT, d->cfg.tile};
    return Choice{MCMC_ENGINE_SIMT, simt_default_tile(d, c.N, c.NOp)};
}

// Groups of channels with one engine and one launch shape; items cover every chain. Tensor-core
// channels of N <= 64 (one 128-row operand tile) of several shape classes with the same tile are
// packed into one group run by the packed kernel, which pulls their work items, largest first,
// from a device queue (unless MCMC_ENGINE_NO_PACK).
mcmc_status build_groups(mcmc_detector *d)
{
    const int Np = d->cfg.chains;
    using GroupKey = std::tuple<int, int, int>;   // (engine, tile, N-class)
    std::map<GroupKey, std::vector<int>> by;
    GroupKey last{-1, -1, -1};
    std::vector<int> *last_v = nullptr;           // batches usually repeat one class for long runs
    for (int b = 0; b < d->n_channels; ++b) {
        const Choice ch = d->choice[b];
        const ChannelDesc &c = d->desc[b];
        const int cls = ch.engine == MCMC_ENGINE_TC ? (c.N + 15) / 16 * 16 : c.N;
        const GroupKey key{ch.engine, ch.tile, cls};
        if (!last_v || key != last) {
            last = key;
            last_v = &by[key];
        }
        last_v->push_back(b);
    }
    // one-tile tensor-core classes per tile: packed when there are two or more
    std::map<int, std::vector<GroupKey>> one_tile;
    if (!(d->cfg.engine & MCMC_ENGINE_NO_PACK))
        for (auto &kv : by)
            if (std::get<0>(kv.first) == MCMC_ENGINE_TC && std::get<2>(kv.first) <= 64)
                one_tile[std::get<1>(kv.first)].push_back(kv.first);
    // keep the work-item buffers: freeing device memory would synchronise the device
    for (auto &g : d->groups)
        if (g.d_items.p) d->spare_items.push_back(g.d_items);
    d->groups.clear();
    auto finish = [&](Group &g) -> mcmc_status {
        if (!d->spare_items.empty()) {
            g.d_items = d->spare_items.back();
            d->spare_items.pop_back();
        }
        CK(ensure(g.d_items, sizeof(WorkItem) * g.items.size()), "alloc items");
        CK(upload(d, g.d_items.p, g.items.data(), sizeof(WorkItem) * g.items.size()), "copy items");
        d->groups.push_back(std::move(g));
        return MCMC_OK;
    };
    for (auto &tk : one_tile) {
        if (tk.second.size() < 2) continue;
        Group g;
        g.engine = MCMC_ENGINE_TC;
        g.tile = tk.first;
        g.packed = true;
        if (!tc_make_plan_packed(g.tile, d->cfg.split_terms, d->smem_optin, &g.plan)) continue;
        for (const GroupKey &k : tk.second) {
            for (int b : by[k]) {
                const ChannelDesc &c = d->desc[b];
                g.max_n = std::max(g.max_n, c.N);
                g.max_nop = std::max(g.max_nop, c.NOp);
                const int per = (c.N <= 32 ? 2 : 1) * g.tile;
                for (int c0 = 0; c0 < Np; c0 += per)
                    g.items.push_back(WorkItem{b, c0, std::min(per, Np - c0), 0});
            }
            by.erase(k);
        }
        // largest work first (chains x dimensions x levels), so that the queue ends on small items
        std::stable_sort(g.items.begin(), g.items.end(), [&](const WorkItem &a, const WorkItem &b) {
            const ChannelDesc &ca = d->desc[a.b], &cb = d->desc[b.b];
            return (long long)a.nc * ca.N * ca.L > (long long)b.nc * cb.N * cb.L;
        });
        mcmc_status st = finish(g);
        if (st != MCMC_OK) return st;
    }
    for (auto &kv : by) {
        Group g;
        g.engine = std::get<0>(kv.first);
        g.tile = std::get<1>(kv.first);
        for (int b : kv.second) {
            g.max_n = std::max(g.max_n, d->desc[b].N);
            g.max_nop = std::max(g.max_nop, d->desc[b].NOp);
        }
        if (g.engine == MCMC_ENGINE_TC) {
            if (!tc_make_plan(g.max_n, g.tile, d->cfg.split_terms, d->smem_optin,
                              !(d->cfg.engine & MCMC_ENGINE_NO_CLUSTER), &g.plan))
                return fail(d, MCMC_EUNSUPPORTED, "no tensor-core plan for N = %d", g.max_n);
        } else {
            if (g.tile <= 0 || !simt_fit(d, g.tile, g.max_n, g.max_nop, &g.bt_smem, &g.smem))
                return fail(d, MCMC_EUNSUPPORTED, "channels of N = %d do not fit the CUDA-core kernel", g.max_n);
        }
        // chains per work item: the SIMT tile, or the tcgen05 plan's chains per CTA (the tile
        // times its chain groups)
        const int per = g.engine == MCMC_ENGINE_TC ? g.plan.chains_per_cta : g.tile;
        g.items.reserve(kv.second.size() * (size_t)((Np + per - 1) / per));
        for (int b : kv.second)
            for (int c0 = 0; c0 < Np; c0 += per)
                g.items.push_back(WorkItem{b, c0, std::min(per, Np - c0), 0});
        mcmc_status st = finish(g);
        if (st != MCMC_OK) return st;
    }
    // one queue counter per group (the packed kernel's), and the streams / events that let a
    // run's groups proceed in parallel
    CK(ensure(d->d_queue, 4 * d->groups.size()), "alloc queues");
    const size_t need = d->groups.size() > 1 ? d->groups.size() - 1 : 0;
    if (need && !d->ev_fork) CK(cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming), "event");
    while (d->aux.size() < need) {
        cudaStream_t s = nullptr;
        CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "aux stream");
        d->aux.push_back(s);
        cudaEvent_t e = nullptr;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
        d->ev_join.push_back(e);
    }
    return MCMC_OK;
}

ChainArgs chain_args(mcmc_detector *d, int32_t iterations, int64_t t_offset)
{
    const bool fp64 = d->cfg.precision == MCMC_PREC_FP64;
    ChainArgs ca{};
    ca.desc = P<ChannelDesc>(d->d_desc);
    ca.chains = d->cfg.chains;
    ca.iterations = iterations;
    ca.t_offset = t_offset;
    ca.refresh_period = d->cfg.refresh_period;
    ca.key0 = (uint32_t)(d->cfg.seed & 0xFFFFFFFFu);
    ca.key1 = (uint32_t)(d->cfg.seed >> 32);
    ca.bt = fp64 ? (const void *)P<double>(d->d_bt64) : (const void *)P<float>(d->d_bt32);
    ca.z = fp64 ? (const void *)P<double>(d->d_z64) : (const void *)P<float>(d->d_z32);
    ca.w = fp64 ? (const void *)P<double>(d->d_w64) : (const void *)P<float>(d->d_w32);
    ca.G64 = P<double>(d->d_G64);
    ca.z64 = P<double>(d->d_z64);
    ca.yy = P<double>(d->d_yy);
    ca.states = P<int8_t>(d->d_states);
    ca.best_states = P<int8_t>(d->d_best_states);
    ca.f = P<double>(d->d_f);
    ca.best_f = P<double>(d->d_best_f);
    ca.accepts = P<unsigned long long>(d->d_accepts);
    ca.drift_bits = drift_ptr(d);
    ca.status = status_ptr(d);
    ca.tc_ops = P<uint8_t>(d->d_tc);
    ca.split_terms = d->cfg.split_terms;
    ca.init_f = d->f_valid ? 0 : 1;
    ca.dexp = fp64 ? nullptr : P<float>(d->d_dexp);
    ca.near_ties = ties_ptr(d);
    ca.trace = (d->cfg.engine & MCMC_ENGINE_TRACE) ? P<double>(d->d_trace) : nullptr;
    return ca;
}

cudaError_t launch_group(mcmc_detector *d, const Group &g, ChainArgs ca, cudaStream_t s, int *queue)
{
    const bool fp64 = d->cfg.precision == MCMC_PREC_FP64;
    ca.items = static_cast<const WorkItem *>(g.d_items.p);
    ca.n_items = (int)g.items.size();
    ca.cg = g.tile;
    ca.max_n = g.max_n;
    ca.max_nop = g.max_nop;
    ca.bt_in_smem = g.bt_smem;
    if (g.engine == MCMC_ENGINE_TC) {
        if (g.packed) {
            cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
            if (e != cudaSuccess) return e;
            ca.queue = queue;
        }
        return ca.refresh_period > 0 ? tc_launch_chains_kr(ca, g.plan, s) : tc_launch_chains(ca, g.plan, s);
    }
    return launch_chains_simt(ca, fp64, g.smem, s);
}

// Autotuner: for every shape class not seen before (in this process, for this configuration),
// time each candidate launch shape on a sample of the class's channels and keep the fastest.
// Probe runs overwrite chain state; the caller redraws the initial states afterwards.
mcmc_status autotune(mcmc_detector *d, bool *probed)
{
    *probed = false;
    const int prec = d->cfg.precision;
    if (prec == MCMC_PREC_FP64 || (d->cfg.engine & 3) != MCMC_ENGINE_AUTO) return MCMC_OK;
    std::map<ClassKey, std::vector<int>> classes;
    for (int b = 0; b < d->n_channels; ++b) classes[class_key(d, d->desc[b])].push_back(b);
    std::vector<Choice> saved = d->choice;
    for (auto &kv : classes) {
        {
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            auto it = g_tuned.find(kv.first);
            if (it != g_tuned.end()) {
                for (int b : kv.second) saved[b] = it->second;
                continue;
            }
        }
        const ChannelDesc &c0 = d->desc[kv.second[0]];
        std::vector<Choice> cands;
        if (prec == MCMC_PREC_MIXED && c0.N <= kMaxN) {
            if (c0.N > 128) cands.push_back(Choice{MCMC_ENGINE_TC, 64});   // cluster kernel only
            cands.push_back(Choice{MCMC_ENGINE_TC, 32});
            cands.push_back(Choice{MCMC_ENGINE_TC, 16});
        }
        for (int cg : {64, 32, 16}) {
            bool bs;
            size_t sm;
            if (cg <= (d->cfg.chains + 7) / 8 * 8 && simt_fit(d, cg, c0.N, c0.NOp, &bs, &sm))
                cands.push_back(Choice{MCMC_ENGINE_SIMT, cg});
        }
        // probe sample: enough channels to fill the GPU twice, at most the class
        const int want = std::max(1, 4 * d->sm_count * 32 / std::max(1, d->cfg.chains));
        std::vector<int> sample(kv.second.begin(),
                                kv.second.begin() + std::min<size_t>(kv.second.size(), (size_t)want));
        Choice best = cands.empty() ? default_choice(d, c0) : cands[0];
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0), "event");
        CK(cudaEventCreate(&e1), "event");
        for (const Choice &cand : cands) {
            Group g;   // the sample channels only
            g.engine = cand.engine;
            g.tile = cand.tile;
            g.max_n = c0.N;
            g.max_nop = c0.NOp;
            bool ok = cand.engine == MCMC_ENGINE_TC
                          ? tc_make_plan(g.max_n, g.tile, d->cfg.split_terms, d->smem_optin,
                                         !(d->cfg.engine & MCMC_ENGINE_NO_CLUSTER), &g.plan)
                          : simt_fit(d, g.tile, g.max_n, g.max_nop, &g.bt_smem, &g.smem);
            if (!ok) continue;
            const int per = cand.engine == MCMC_ENGINE_TC ? g.plan.chains_per_cta : g.tile;
            for (int b : sample)
                for (int cc = 0; cc < d->cfg.chains; cc += per)
                    g.items.push_back(WorkItem{b, cc, std::min(per, d->cfg.chains - cc), 0});
            CK(ensure(g.d_items, sizeof(WorkItem) * g.items.size()), "alloc probe items");
            CK(cudaMemcpyAsync(g.d_items.p, g.items.data(), sizeof(WorkItem) * g.items.size(),
                               cudaMemcpyHostToDevice, d->stream), "copy probe items");
            ChainArgs ca = chain_args(d, 2, 0);
            ca.init_f = 1;
            // the kernels the run will launch: without the in-run refresh unless it stays inside
            if (!(d->cfg.engine & MCMC_ENGINE_KERNEL_REFRESH)) ca.refresh_period = 0;
            ca.near_ties = nullptr;   // probe transitions are not the batch's
            ca.trace = nullptr;
            cudaError_t e = launch_group(d, g, ca, d->stream, nullptr);   // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, d->stream);
            ca.iterations = 24;   // long enough to amortise per-item set-up (streamed operands)
            if (e == cudaSuccess) e = launch_group(d, g, ca, d->stream, nullptr);
            if (e == cudaSuccess) e = cudaEventRecord(e1, d->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            cudaFree(g.d_items.p);
            d->launches += 2;
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(d, e, "autotuner probe");
            }
            if (ms < best_ms) { best_ms = ms; best = cand; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (sample.size() == (size_t)want) {
            // only a probe over a full sample speaks for other batches of this class: with a few
            // channels the engines' parallelism differs from a full batch's
            std::lock_guard<std::mutex> lk(g_tuned_mu);
            g_tuned[kv.first] = best;
        }
        for (int b : kv.second) saved[b] = best;
        *probed = true;
        d->tuned_classes++;
    }
    d->choice = saved;
    return MCMC_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

void mcmc_config_default(mcmc_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->max_channels = 1;
    cfg->max_nt = 4;
    cfg->max_nr = 4;
    cfg->chains = 32;
    cfg->precision = MCMC_PREC_FP32;
    cfg->preconditioned = 1;
    cfg->refresh_period = 0;
    cfg->split_terms = 2;
    cfg->engine = MCMC_ENGINE_AUTO;
    cfg->seed = 0;
    cfg->stream = nullptr;
}

const char *mcmc_status_string(mcmc_status s)
{
    switch (s) {
    case MCMC_OK: return "ok";
    case MCMC_EINVAL: return "invalid argument";
    case MCMC_ENOMEM: return "out of memory";
    case MCMC_ECUDA: return "CUDA error";
    case MCMC_ETIMEOUT: return "bounded device wait expired";
    case MCMC_ENUMERIC: return "non-finite value on the device";
    case MCMC_ESTATE: return "call out of order";
    case MCMC_EUNSUPPORTED: return "unsupported on this device or build";
    }
    return "unknown status";
}

const char *mcmc_detect_last_error(const mcmc_detector *d)
{
    return d ? d->err.c_str() : "null handle";
}

int64_t mcmc_detect_kernel_launches(const mcmc_detector *d)
{
    return d ? d->launches : 0;
}

mcmc_status mcmc_detect_create(const mcmc_config *cfg, mcmc_detector **out)
{
    if (!cfg || !out) return MCMC_EINVAL;
    *out = nullptr;
    if (cfg->max_channels < 1 || cfg->max_nt < 1 || 2 * cfg->max_nt > kMaxN || cfg->max_nr < 1 ||
        cfg->max_nr > 4096 || cfg->chains < 4 || cfg->chains > 1024 || (cfg->chains % 4) != 0 ||
        cfg->precision < MCMC_PREC_FP64 || cfg->precision > MCMC_PREC_MIXED ||
        (cfg->preconditioned != 0 && cfg->preconditioned != 1) || cfg->refresh_period < -1 ||
        cfg->split_terms < 1 || cfg->split_terms > 3 || cfg->engine < 0 ||
        (cfg->engine & ~(3 | MCMC_ENGINE_GRAPH | MCMC_ENGINE_NO_CLUSTER | MCMC_ENGINE_TRACE |
                         MCMC_ENGINE_NO_PACK | MCMC_ENGINE_NO_GRAPH | MCMC_ENGINE_KERNEL_REFRESH)) != 0 ||
        (cfg->engine & 3) == 3 ||
        cfg->tile < 0 || (cfg->tile != 0 && (cfg->engine & 3) == MCMC_ENGINE_AUTO) ||
        ((cfg->engine & 3) == MCMC_ENGINE_TC && cfg->tile != 0 && cfg->tile != 16 && cfg->tile != 32 &&
         cfg->tile != 64) ||
        ((cfg->engine & 3) == MCMC_ENGINE_SIMT && (cfg->tile % 8 != 0 || cfg->tile > 64)))
        return MCMC_EINVAL;
    if (cfg->precision != MCMC_PREC_MIXED && (cfg->engine & 3) == MCMC_ENGINE_TC) return MCMC_EINVAL;
    mcmc_detector *d = new (std::nothrow) mcmc_detector();
    if (!d) return MCMC_ENOMEM;
    d->cfg = *cfg;
    cudaError_t e = cudaGetDevice(&d->device);
    if (e != cudaSuccess) { cudaGetLastError(); delete d; return MCMC_EUNSUPPORTED; }
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, d->device) != cudaSuccess) { cudaGetLastError(); delete d; return MCMC_ECUDA; }
    d->sm_count = prop.multiProcessorCount;
    d->cc_major = prop.major;
    d->cc_minor = prop.minor;
    d->smem_optin = prop.sharedMemPerBlockOptin;
    if (cfg->precision == MCMC_PREC_MIXED && !(prop.major == 10 && prop.minor == 3)) {
        delete d;
        return MCMC_EUNSUPPORTED;
    }
    if (cfg->stream) {
        d->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        if (cudaStreamCreateWithFlags(&d->stream, cudaStreamDefault) != cudaSuccess) {
            cudaGetLastError();
            delete d;
            return MCMC_ECUDA;
        }
        d->own_stream = true;
    }
    if (ensure(d->d_misc, 256) != cudaSuccess ||
        cudaMemsetAsync(d->d_misc.p, 0, 256, d->stream) != cudaSuccess) {
        cudaGetLastError();
        mcmc_detect_destroy(d);
        return MCMC_ENOMEM;
    }
    *out = d;
    return MCMC_OK;
}

mcmc_status mcmc_detect_destroy(mcmc_detector *d)
{
    if (!d) return MCMC_OK;
    if (d->stream) cudaStreamSynchronize(d->stream);
    DevBuf *bufs[] = {&d->d_desc, &d->d_Gc, &d->d_zc, &d->d_Mc, &d->d_gj, &d->d_yy,
                      &d->d_G64, &d->d_GM64, &d->d_z64, &d->d_w64, &d->d_z32, &d->d_w32,
                      &d->d_bt32, &d->d_bt64, &d->d_tc, &d->d_states, &d->d_best_states, &d->d_f,
                      &d->d_best_f, &d->d_accepts, &d->d_misc, &d->d_in_H, &d->d_in_y,
                      &d->d_in_s2, &d->d_out_idx, &d->d_out_llr, &d->d_out_bf, &d->d_dexp,
                      &d->d_fx, &d->d_trace, &d->d_queue,
                      &d->d_mx_gx, &d->d_mx_px, &d->d_mx_gxp, &d->d_mx_pxp, &d->d_mx_prop,
                      &d->d_mx_X, &d->d_mx_logits, &d->d_mx_lqf};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto &g : d->groups)
        if (g.d_items.p) cudaFree(g.d_items.p);
    for (auto &b : d->spare_items)
        if (b.p) cudaFree(b.p);
    if (d->graph) cudaGraphExecDestroy(d->graph);
    if (d->h_stage.p) cudaFreeHost(d->h_stage.p);
    for (int k = 0; k < mcmc_detector::kUpSlots; ++k) {
        if (d->up_done[k]) cudaEventDestroy(d->up_done[k]);
        if (d->h_up[k].p) cudaFreeHost(d->h_up[k].p);
    }
    for (cudaStream_t a : d->aux) cudaStreamDestroy(a);
    for (cudaEvent_t e : d->ev_join) cudaEventDestroy(e);
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    for (auto &pr : d->ev_run)
        for (cudaEvent_t e : pr)
            if (e) cudaEventDestroy(e);
    if (d->own_stream && d->stream) cudaStreamDestroy(d->stream);
    cudaGetLastError();
    delete d;
    return MCMC_OK;
}

mcmc_status mcmc_detect_preprocess(mcmc_detector *d, int32_t n_channels, const int32_t *nt,
                                   const int32_t *nr, const int32_t *qam, const void *H,
                                   const int64_t *H_off, const void *y, const int64_t *y_off,
                                   const float *noise_var, float alpha_scale, float tau,
                                   int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (n_channels < 1 || n_channels > d->cfg.max_channels)
        return fail(d, MCMC_EINVAL, "n_channels %d outside [1, %d]", n_channels, d->cfg.max_channels);
    if (!nt || !nr || !qam || !H || !H_off || !y || !y_off || !noise_var)
        return fail(d, MCMC_EINVAL, "null argument");
    if (!(alpha_scale > 0.f) || !std::isfinite(alpha_scale) || !(tau >= 1.f) || !std::isfinite(tau))
        return fail(d, MCMC_EINVAL, "alpha_scale must be > 0 and tau >= 1");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const int Np = d->cfg.chains;
    const bool pre = d->cfg.preconditioned != 0;
    d->prepared = false;
    d->desc.assign(n_channels, ChannelDesc{});
    long long st = 0, mat = 0, bt = 0, vec = 0, bits = 0, ant = 0, hmax = 0, ymax = 0;
    int maxn = 0, maxnop = 0, maxnt = 0, maxnr = 0;
    for (int b = 0; b < n_channels; ++b) {
        const int L = qam[b] == 4 ? 2 : qam[b] == 16 ? 4 : qam[b] == 64 ? 8 : 0;
        if (!L) return fail(d, MCMC_EINVAL, "channel %d: qam %d not in {4,16,64}", b, qam[b]);
        if (nt[b] < 1 || nt[b] > d->cfg.max_nt || nr[b] < 1 || nr[b] > d->cfg.max_nr)
            return fail(d, MCMC_EINVAL, "channel %d: nt=%d nr=%d outside capacity", b, nt[b], nr[b]);
        if (H_off[b] < 0 || y_off[b] < 0) return fail(d, MCMC_EINVAL, "channel %d: negative offset", b);
        ChannelDesc &c = d->desc[b];
        c.N = 2 * nt[b];
        c.L = L;
        c.log2L = log2_levels(L);
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
        hmax = std::max(hmax, (long long)H_off[b] + (long long)nt[b] * nr[b]);
        ymax = std::max(ymax, (long long)y_off[b] + nr[b]);
        maxn = std::max(maxn, c.N);
        maxnop = std::max(maxnop, c.NOp);
        maxnt = std::max(maxnt, c.Nt);
        maxnr = std::max(maxnr, c.Nr);
    }
    d->n_channels = n_channels;
    d->max_n = maxn;
    d->max_nop = maxnop;
    d->max_nt = maxnt;
    d->max_nr = maxnr;
    d->tot_states = st;
    d->tot_mat = mat;
    d->tot_bt = bt;
    d->tot_vec = vec;
    d->tot_bits = bits;
    d->tot_ant = ant;

    // chain-kernel plan: one engine / launch shape per channel (tuned or default)
    const bool fp64 = d->cfg.precision == MCMC_PREC_FP64;
    const bool mixed = d->cfg.precision == MCMC_PREC_MIXED;
    d->choice.assign(n_channels, Choice{});
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        int lastN = -1, lastL = -1;
        Choice lastc{};
        for (int b = 0; b < n_channels; ++b) {
            const ChannelDesc &c = d->desc[b];
            if (c.N != lastN || c.L != lastL) {   // the key varies with (N, L) only within a call
                auto it = g_tuned.find(class_key(d, c));
                lastc = (it != g_tuned.end() && (d->cfg.engine & 3) == MCMC_ENGINE_AUTO) ? it->second
                                                                                        : default_choice(d, c);
                lastN = c.N;
                lastL = c.L;
            }
            d->choice[b] = lastc;
        }
    }
    long long tot_tc = 0;
    if (mixed) {
        for (auto &c : d->desc) {
            c.tc_off = tot_tc;
            tot_tc += tc_operand_bytes(c.N, d->cfg.split_terms);
        }
    }
    if (d->graph) {
        cudaGraphExecDestroy(d->graph);
        d->graph = nullptr;
    }

    // workspace
    const long long ntc = mat / 4;   // complex Nt^2 elements over the batch
    CK(ensure(d->d_desc, sizeof(ChannelDesc) * n_channels), "alloc desc");
    CK(ensure(d->d_Gc, 16 * ntc), "alloc Gc");
    CK(ensure(d->d_zc, 8 * vec), "alloc zc");
    CK(ensure(d->d_yy, 8 * n_channels), "alloc yy");
    CK(ensure(d->d_G64, 8 * mat), "alloc G64");
    CK(ensure(d->d_z64, 8 * vec), "alloc z64");
    CK(ensure(d->d_w64, 8 * vec), "alloc w64");
    CK(ensure(d->d_z32, 4 * vec), "alloc z32");
    CK(ensure(d->d_w32, 4 * vec), "alloc w32");
    if (pre) {
        CK(ensure(d->d_Mc, 16 * ntc), "alloc Mc");
        if (fp64) CK(ensure(d->d_GM64, 8 * mat), "alloc GM64");
    }
    // Gauss-Jordan block (FP64 complex in FP64 mode, FP32 complex otherwise) and the copies of
    // its pivot row and column
    const size_t gj_elem = fp64 ? 16 : 8;
    const size_t gj_stage = (size_t)(maxnt * maxnt + 2 * maxnt) * gj_elem;
    const bool stage_gj = pre && gj_stage <= std::min<size_t>(d->smem_optin, 160 * 1024);
    if (pre && !stage_gj) CK(ensure(d->d_gj, 16 * 2 * ntc), "alloc gj");
    if (fp64) CK(ensure(d->d_bt64, 8 * bt), "alloc bt64");
    else CK(ensure(d->d_bt32, 4 * bt), "alloc bt32");   // FP32 chains; FP32 read-out of every non-FP64 mode
    if (mixed) CK(ensure(d->d_tc, (size_t)tot_tc), "alloc tc operands");
    CK(ensure(d->d_states, st), "alloc states");
    CK(ensure(d->d_best_states, st), "alloc best states");
    CK(ensure(d->d_f, 8 * (size_t)n_channels * Np), "alloc f");
    CK(ensure(d->d_best_f, 8 * (size_t)n_channels * Np), "alloc best f");
    CK(ensure(d->d_accepts, 8 * (size_t)n_channels * Np), "alloc accepts");
    if (!fp64) CK(ensure(d->d_dexp, 4 * (size_t)st), "alloc Gt x export");
    if (d->cfg.engine & MCMC_ENGINE_TRACE) {
        CK(ensure(d->d_trace, 16 * (size_t)n_channels * Np), "alloc trace");
        CK(cudaMemsetAsync(d->d_trace.p, 0, 16 * (size_t)n_channels * Np, d->stream), "reset trace");
    }

    // inputs
    const float2 *Hd = static_cast<const float2 *>(H);
    const float2 *yd = static_cast<const float2 *>(y);
    const float *sd = noise_var;
    if (host_io) {
        const size_t hb = 8 * (size_t)hmax, yb = 8 * (size_t)ymax, sb = 4 * (size_t)n_channels;
        CK(ensure(d->d_in_H, hb), "alloc H");
        CK(ensure(d->d_in_y, yb), "alloc y");
        CK(ensure(d->d_in_s2, sb), "alloc noise_var");
        const bool all_pinned = is_pinned_or_device(H) && is_pinned_or_device(y) && is_pinned_or_device(noise_var);
        if (!all_pinned) {
            CK(cudaStreamSynchronize(d->stream), "stream synchronize");
            CK(ensure_host(d->h_stage, hb + yb + sb), "alloc pinned staging");
        }
        CK(h2d(d, d->d_in_H.p, H, hb, 0), "copy H");
        CK(h2d(d, d->d_in_y.p, y, yb, hb), "copy y");
        CK(h2d(d, d->d_in_s2.p, noise_var, sb, hb + yb), "copy noise_var");
        Hd = P<float2>(d->d_in_H);
        yd = P<float2>(d->d_in_y);
        sd = P<float>(d->d_in_s2);
    }
    CK(upload(d, d->d_desc.p, d->desc.data(), sizeof(ChannelDesc) * n_channels), "copy desc");
    CK(cudaMemsetAsync(d->d_misc.p, 0, 256, d->stream), "reset status");
    CK(cudaMemsetAsync(d->d_accepts.p, 0, 8 * (size_t)n_channels * Np, d->stream), "reset accepts");
    finalize_desc_kernel<<<(n_channels + 127) / 128, 128, 0, d->stream>>>(
        P<ChannelDesc>(d->d_desc), sd, n_channels, alpha_scale, tau, pre, status_ptr(d));
    CK(cudaGetLastError(), "finalize desc");
    d->launches++;

    PrepArgs pa{};
    pa.desc = P<ChannelDesc>(d->d_desc);
    pa.H = Hd;
    pa.y = yd;
    pa.Gc = P<double>(d->d_Gc);
    pa.zc = P<double>(d->d_zc);
    pa.Mc = P<double>(d->d_Mc);
    pa.gj = P<double>(d->d_gj);
    pa.yy = P<double>(d->d_yy);
    pa.G64 = P<double>(d->d_G64);
    pa.GM64 = (pre && fp64) ? P<double>(d->d_GM64) : nullptr;
    pa.z64 = P<double>(d->d_z64);
    pa.w64 = P<double>(d->d_w64);
    pa.z32 = P<float>(d->d_z32);
    pa.w32 = P<float>(d->d_w32);
    pa.bt32 = fp64 ? nullptr : P<float>(d->d_bt32);
    pa.bt64 = fp64 ? P<double>(d->d_bt64) : nullptr;
    pa.status = status_ptr(d);
    const size_t h_stage = 8 * (size_t)(maxnt * maxnr + maxnr);
    pa.stage_h = h_stage <= std::min<size_t>(d->smem_optin, 128 * 1024);
    pa.stage_gj = stage_gj;
    pa.precond_fp32 = fp64 ? 0 : 1;
    pa.max_nt = maxnt;
    CK(launch_prep(pa, n_channels, h_stage, stage_gj ? gj_stage : 2 * maxnt * gj_elem, pre, d->stream),
       "prep kernels");
    d->launches += pre ? 3 : 2;
    if (mixed) {
        CK(tc_launch_pack(d->cfg.split_terms, P<ChannelDesc>(d->d_desc), n_channels,
                          P<float>(d->d_bt32), P<uint8_t>(d->d_tc), d->stream), "pack operands");
        d->launches++;
    }

    InitArgs ia{};
    ia.desc = P<ChannelDesc>(d->d_desc);
    ia.states = P<int8_t>(d->d_states);
    ia.n_channels = n_channels;
    ia.chains = Np;
    ia.items_per_channel = (long long)(Np / 4) * maxn;
    ia.key0 = (uint32_t)(d->cfg.seed & 0xFFFFFFFFu);
    ia.key1 = (uint32_t)(d->cfg.seed >> 32);
    CK(launch_init_states(ia, d->stream), "init states");
    d->launches++;

    // autotune unseen shape classes on this batch, then redraw the states the probes touched
    d->f_valid = fp64;
    {
        bool probed = false;
        mcmc_status ts = autotune(d, &probed);
        if (ts != MCMC_OK) return ts;
        if (probed) {
            CK(launch_init_states(ia, d->stream), "init states");
            CK(cudaMemsetAsync(d->d_accepts.p, 0, 8 * (size_t)n_channels * Np, d->stream), "reset accepts");
            d->launches++;
        }
    }
    {
        mcmc_status gs = build_groups(d);
        if (gs != MCMC_OK) return gs;
    }

    // the exact energies of the initial states (every precision), where the running best
    // starts, are evaluated when first needed: by the next run, estimate or mixture move (the
    // read-outs hand out FP64 evaluations meanwhile); a warm start that replaces the states
    // first does not pay for them twice
    d->f_valid = false;
    d->f_exact = false;
    d->d_valid = false;
    d->transitions = 0;
    d->prepared = true;
    return MCMC_OK;
}

mcmc_status mcmc_detect_run_chains(mcmc_detector *d, int32_t iterations, int64_t t_offset)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "run_chains before preprocess");
    if (iterations < 0 || t_offset < 0 || t_offset + (int64_t)iterations > 0xFFFFFFFFll)
        return fail(d, MCMC_EINVAL, "iterations/t_offset out of range");
    if (iterations == 0) return MCMC_OK;
    const bool fp64 = d->cfg.precision == MCMC_PREC_FP64;
    // the chains start from exact energies of their states (after preprocess or a warm start)
    {
        mcmc_status es = ensure_energies(d);
        if (es != MCMC_OK) return es;
    }
    ChainArgs ca = chain_args(d, iterations, t_offset);
    // FP32 / MIXED: the energies the chains tracked in FP32 steps are replaced by exact
    // evaluations when the run ends (refresh_period >= 0), and the correction is recorded
    const bool final_refresh = !fp64 && d->cfg.refresh_period >= 0;
    // In-run refreshes (refresh_period R > 0) after every transition t with t % R == 0: by
    // default the run is cut into launches at those transitions and the exact refresh kernel runs
    // between them. The draws follow the transition number, so the states and decisions are those
    // of one launch; MCMC_ENGINE_KERNEL_REFRESH keeps the refreshes inside the chain kernels.
    const int R = d->cfg.refresh_period;
    const bool cut = !fp64 && R > 0 && !(d->cfg.engine & MCMC_ENGINE_KERNEL_REFRESH);
    std::vector<std::pair<int64_t, int32_t>> segs;   // (t_offset, iterations) of each launch
    if (cut) {
        ca.refresh_period = 0;
        const int64_t end = t_offset + iterations;
        for (int64_t s0 = t_offset; s0 < end;) {
            const int64_t e = std::min<int64_t>((s0 / R + 1) * R, end);
            segs.emplace_back(s0, (int32_t)(e - s0));
            s0 = e;
        }
    } else {
        segs.emplace_back(t_offset, iterations);
    }
    RefreshArgs fr{};
    if (final_refresh) {
        fr.desc = P<ChannelDesc>(d->d_desc);
        fr.states = P<int8_t>(d->d_states);
        fr.G64 = P<double>(d->d_G64);
        fr.z64 = P<double>(d->d_z64);
        fr.yy = P<double>(d->d_yy);
        fr.f = P<double>(d->d_f);
        fr.status = status_ptr(d);
        fr.n_channels = d->n_channels;
        fr.chains = d->cfg.chains;
        fr.max_n = d->max_n;
        fr.drift_bits = drift_ptr(d);
        fr.drift_rel_bits = drift_rel_ptr(d);
    }
    // every group's launch, forked onto its own stream when there are several (parallel
    // branches: the groups' kernels share the GPU instead of running one after the other), then
    // the final refresh once all have joined
    auto enqueue = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        const size_t ng = d->groups.size();
        int *queues = P<int>(d->d_queue);
        for (size_t si = 0; si < segs.size() && e == cudaSuccess; ++si) {
            ChainArgs cs = ca;
            cs.t_offset = segs[si].first;
            cs.iterations = segs[si].second;
            if (ng > 1) e = cudaEventRecord(d->ev_fork, d->stream);
            for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) {
                cudaStream_t s = gi == 0 ? d->stream : d->aux[gi - 1];
                if (gi > 0) e = cudaStreamWaitEvent(s, d->ev_fork, 0);
                if (e == cudaSuccess) e = launch_group(d, d->groups[gi], cs, s, queues + gi);
                if (e == cudaSuccess && gi > 0) e = cudaEventRecord(d->ev_join[gi - 1], s);
            }
            for (size_t gi = 1; gi < ng && e == cudaSuccess; ++gi)
                e = cudaStreamWaitEvent(d->stream, d->ev_join[gi - 1], 0);
            // an in-run refresh (the last cut is the run's end: the final refresh follows it)
            if (e == cudaSuccess && si + 1 < segs.size()) e = launch_refresh(fr, d->stream);
        }
        return e;
    };
    const int slot = (int)(d->runs % mcmc_detector::kRunSlots);
    for (int k = 0; k < 2; ++k)
        if (!d->ev_run[slot][k]) CK(cudaEventCreate(&d->ev_run[slot][k]), "event");
    CK(cudaEventRecord(d->ev_run[slot][0], d->stream), "record run start");
    // one CUDA graph per run (replayed; updated in place when only the arguments changed) when
    // asked for, and by default for a batch of several launch groups
    const bool graph = (d->cfg.engine & MCMC_ENGINE_GRAPH) ||
                       (d->groups.size() > 1 && !(d->cfg.engine & MCMC_ENGINE_NO_GRAPH));
    if (graph) {
        CK(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        const cudaError_t le = enqueue();
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(d->stream, &g);
        if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(d, le, "chain kernel"); }
        CK(ce, "end capture");
        bool updated = false;
        if (d->graph) {
            cudaGraphExecUpdateResultInfo info{};
            updated = cudaGraphExecUpdate(d->graph, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(d->graph);
                d->graph = nullptr;
            }
        }
        if (!updated) {
            const cudaError_t ie = cudaGraphInstantiate(&d->graph, g, 0);
            if (ie != cudaSuccess) { cudaGraphDestroy(g); return cuda_fail(d, ie, "instantiate graph"); }
        }
        cudaGraphDestroy(g);
        CK(cudaGraphLaunch(d->graph, d->stream), "graph launch");
    } else {
        CK(enqueue(), "chain kernel");
    }
    CK(cudaEventRecord(d->ev_run[slot][1], d->stream), "record run end");
    d->runs++;
    if (final_refresh) CK(launch_refresh(fr, d->stream), "energies");
    d->launches += (long long)(d->groups.size() + 1) * segs.size() - 1 + (final_refresh ? 1 : 0);
    d->f_valid = true;
    d->f_exact = fp64 || final_refresh;
    d->d_valid = !fp64;
    d->transitions += (long long)iterations * d->n_channels * d->cfg.chains;
    return MCMC_OK;
}

mcmc_status mcmc_detect_estimate(mcmc_detector *d, int8_t *best_idx, float *llr, double *best_f,
                                 mcmc_stats *stats, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "estimate before preprocess");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const bool fp64 = d->cfg.precision == MCMC_PREC_FP64;
    {
        mcmc_status es = ensure_energies(d);
        if (es != MCMC_OK) return es;
    }
    int8_t *o_idx = best_idx;
    float *o_llr = llr;
    double *o_bf = best_f;
    if (host_io) {
        if (best_idx) { CK(ensure(d->d_out_idx, d->tot_ant), "alloc out"); o_idx = P<int8_t>(d->d_out_idx); }
        if (llr) { CK(ensure(d->d_out_llr, 4 * d->tot_bits), "alloc out"); o_llr = P<float>(d->d_out_llr); }
        if (best_f) { CK(ensure(d->d_out_bf, 8 * (size_t)d->n_channels), "alloc out"); o_bf = P<double>(d->d_out_bf); }
    }
    EstimateArgs ea{};
    ea.desc = P<ChannelDesc>(d->d_desc);
    ea.states = P<int8_t>(d->d_states);
    ea.best_states = P<int8_t>(d->d_best_states);
    ea.f = P<double>(d->d_f);
    ea.best_f = P<double>(d->d_best_f);
    ea.G = fp64 ? (const void *)P<double>(d->d_G64) : (const void *)P<float>(d->d_bt32);
    ea.g_is_bt = fp64 ? 0 : 1;
    ea.dexp = (!fp64 && d->d_valid) ? P<float>(d->d_dexp) : nullptr;
    ea.z = fp64 ? (const void *)P<double>(d->d_z64) : (const void *)P<float>(d->d_z32);
    ea.G64 = P<double>(d->d_G64);
    ea.z64 = P<double>(d->d_z64);
    ea.yy = P<double>(d->d_yy);
    ea.n_channels = d->n_channels;
    ea.chains = d->cfg.chains;
    ea.best_idx = o_idx;
    ea.llr = o_llr;
    ea.best_f_out = o_bf;
    ea.status = status_ptr(d);
    CK(launch_estimate(ea, fp64, d->stream), "estimate kernel");
    d->launches++;
    if (host_io) {
        if (best_idx) CK(cudaMemcpyAsync(best_idx, o_idx, d->tot_ant, cudaMemcpyDeviceToHost, d->stream), "copy out");
        if (llr) CK(cudaMemcpyAsync(llr, o_llr, 4 * d->tot_bits, cudaMemcpyDeviceToHost, d->stream), "copy out");
        if (best_f) CK(cudaMemcpyAsync(best_f, o_bf, 8 * (size_t)d->n_channels, cudaMemcpyDeviceToHost, d->stream), "copy out");
    }
    mcmc_status s = read_status(d);
    if (stats) {
        std::memset(stats, 0, sizeof *stats);
        stats->transitions = d->transitions;
        std::vector<unsigned long long> acc((size_t)d->n_channels * d->cfg.chains);
        CK(cudaMemcpy(acc.data(), d->d_accepts.p, 8 * acc.size(), cudaMemcpyDeviceToHost), "copy accepts");
        unsigned long long tot = 0;
        for (auto v : acc) tot += v;
        stats->accepts = (int64_t)tot;
        unsigned long long db = 0;
        CK(cudaMemcpy(&db, drift_ptr(d), 8, cudaMemcpyDeviceToHost), "copy drift");
        double dr;
        std::memcpy(&dr, &db, 8);
        stats->refresh_drift = dr;
        CK(cudaMemcpy(&db, drift_rel_ptr(d), 8, cudaMemcpyDeviceToHost), "copy drift");
        std::memcpy(&dr, &db, 8);
        stats->refresh_drift_rel = dr;
        unsigned long long ties[3] = {0, 0, 0};
        CK(cudaMemcpy(ties, ties_ptr(d), sizeof ties, cudaMemcpyDeviceToHost), "copy near ties");
        for (int k = 0; k < 3; ++k) stats->near_ties[k] = (int64_t)ties[k];
        unsigned stw = 0;
        CK(cudaMemcpy(&stw, status_ptr(d), sizeof stw, cudaMemcpyDeviceToHost), "copy status");
        stats->numeric_faults = (stw & kStatusNumeric) ? 1 : 0;
        stats->near_tie_windows = 3;
    }
    return s;
}

mcmc_status mcmc_detect_llr_list(mcmc_detector *d, float *llr, float clip, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "llr_list before preprocess");
    if (!llr) return fail(d, MCMC_EINVAL, "null llr");
    if (!(clip > 0.f) || !std::isfinite(clip)) return fail(d, MCMC_EINVAL, "clip must be > 0 and finite");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const double *fx = nullptr;   // FP64 energies of the current states
    {
        mcmc_status es = fp64_energies(d, &fx);
        if (es != MCMC_OK) return es;
    }
    float *o_llr = llr;
    if (host_io) {
        CK(ensure(d->d_out_llr, 4 * d->tot_bits), "alloc out");
        o_llr = P<float>(d->d_out_llr);
    }
    ListLlrArgs la{};
    la.desc = P<ChannelDesc>(d->d_desc);
    la.states = P<int8_t>(d->d_states);
    la.f = fx;
    la.n_channels = d->n_channels;
    la.chains = d->cfg.chains;
    la.clip = clip;
    la.llr = o_llr;
    la.status = status_ptr(d);
    CK(launch_list_llr(la, d->cfg.precision == MCMC_PREC_FP64, d->stream), "list LLR kernel");
    d->launches++;
    if (host_io) CK(cudaMemcpyAsync(llr, o_llr, 4 * d->tot_bits, cudaMemcpyDeviceToHost, d->stream), "copy out");
    return read_status(d);
}

mcmc_status mcmc_detect_get_chains(mcmc_detector *d, int8_t *states, double *f, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "get_chains before preprocess");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const double *fx = nullptr;
    if (f) {
        mcmc_status es = fp64_energies(d, &fx);
        if (es != MCMC_OK) return es;
    }
    const cudaMemcpyKind k = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (states) CK(cudaMemcpyAsync(states, d->d_states.p, d->tot_states, k, d->stream), "copy states");
    if (f) CK(cudaMemcpyAsync(f, fx, 8 * (size_t)d->n_channels * d->cfg.chains, k, d->stream), "copy f");
    return read_status(d);
}

mcmc_status mcmc_detect_get_tracked(mcmc_detector *d, double *f, double *best_f, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "get_tracked before preprocess");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const size_t bytes = 8 * (size_t)d->n_channels * d->cfg.chains;
    const cudaMemcpyKind k = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (!d->f_valid) {
        // no run yet: the chains have no tracked energies; hand out FP64 evaluations of the
        // initial states (the running best is the initial state) and leave the handle as it is
        const double *fx = nullptr;
        mcmc_status es = fp64_energies(d, &fx);
        if (es != MCMC_OK) return es;
        if (f) CK(cudaMemcpyAsync(f, fx, bytes, k, d->stream), "copy f");
        if (best_f) CK(cudaMemcpyAsync(best_f, fx, bytes, k, d->stream), "copy best f");
        return read_status(d);
    }
    if (f) CK(cudaMemcpyAsync(f, d->d_f.p, bytes, k, d->stream), "copy f");
    if (best_f) CK(cudaMemcpyAsync(best_f, d->d_best_f.p, bytes, k, d->stream), "copy best f");
    return read_status(d);
}

mcmc_status mcmc_detect_get_trace(mcmc_detector *d, double *trace, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "get_trace before preprocess");
    if (!(d->cfg.engine & MCMC_ENGINE_TRACE)) return fail(d, MCMC_ESTATE, "handle created without MCMC_ENGINE_TRACE");
    if (!trace) return fail(d, MCMC_EINVAL, "null trace");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    const cudaMemcpyKind k = host_io ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(trace, d->d_trace.p, 16 * (size_t)d->n_channels * d->cfg.chains, k, d->stream),
       "copy trace");
    return read_status(d);
}

mcmc_status mcmc_detect_set_chains(mcmc_detector *d, const int8_t *states, int32_t host_io)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!d->prepared) return fail(d, MCMC_ESTATE, "set_chains before preprocess");
    if (!states) return fail(d, MCMC_EINVAL, "null states");
    if (host_io != 0 && host_io != 1) return fail(d, MCMC_EINVAL, "host_io must be 0 or 1");
    if (host_io) {
        const int Np = d->cfg.chains;
        for (int b = 0; b < d->n_channels; ++b) {
            const ChannelDesc &c = d->desc[b];
            for (long long i = 0; i < (long long)Np * c.N; ++i) {
                const int v = states[c.state_off + i];
                if (v < 0 || v >= c.L) return fail(d, MCMC_EINVAL, "channel %d: level %d out of range", b, v);
            }
        }
        CK(cudaMemcpyAsync(d->d_states.p, states, d->tot_states, cudaMemcpyHostToDevice, d->stream), "copy states");
        CK(cudaStreamSynchronize(d->stream), "stream synchronize");
    } else {
        CK(cudaMemcpyAsync(d->d_states.p, states, d->tot_states, cudaMemcpyDeviceToDevice, d->stream), "copy states");
    }
    {
        mcmc_status es = refresh_energies(d, P<double>(d->d_f), true, false);
        if (es != MCMC_OK) return es;
    }
    d->f_valid = true;
    d->f_exact = true;
    d->d_valid = false;
    return read_status(d);
}

int32_t mcmc_detect_launch_groups(const mcmc_detector *d, int32_t *info, int32_t cap)
{
    if (!d || !d->prepared) return 0;
    const int32_t n = (int32_t)d->groups.size();
    for (int32_t i = 0; i < n && info && i < cap; ++i) {
        const Group &g = d->groups[(size_t)i];
        int32_t *r = info + 6 * i;
        r[0] = g.engine;
        r[1] = g.tile;
        r[2] = g.packed ? 1 : 0;
        r[3] = g.max_n;
        r[4] = (int32_t)g.items.size();
        r[5] = g.engine == MCMC_ENGINE_TC ? (g.plan.cluster > 1 ? g.plan.cluster : g.plan.ctas_per_sm) : 0;
    }
    return n;
}

mcmc_status mcmc_detect_run_kernel_ms(mcmc_detector *d, int32_t n, float *ms)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!ms || n < 1 || n > mcmc_detector::kRunSlots || n > d->runs)
        return fail(d, MCMC_EINVAL, "n must lie in 1 .. min(runs so far, %d)", mcmc_detector::kRunSlots);
    for (int32_t i = 0; i < n; ++i) {
        const int slot = (int)((d->runs - n + i) % mcmc_detector::kRunSlots);
        CK(cudaEventSynchronize(d->ev_run[slot][1]), "event synchronize");
        CK(cudaEventElapsedTime(&ms[i], d->ev_run[slot][0], d->ev_run[slot][1]), "event time");
    }
    return MCMC_OK;
}

mcmc_status mcmc_detect_synchronize(mcmc_detector *d)
{
    if (!d) return MCMC_EINVAL;
    return read_status(d);
}

}  // extern "C"

// ---- learned proposal (include/mcmcdet_learned.h) -----------------------------------------

namespace {

mcmc_status learned_ok(mcmc_detector *d)
{
    if (!d->prepared) return fail(d, MCMC_ESTATE, "learned proposal before preprocess");
    if (d->cfg.precision == MCMC_PREC_FP64)
        return fail(d, MCMC_EUNSUPPORTED, "the learned proposal runs on FP32 or MIXED handles");
    if (!d->cfg.preconditioned)
        return fail(d, MCMC_EUNSUPPORTED, "the learned proposal needs the preconditioned proposal");
    return MCMC_OK;
}

MixGramArgs gram_args(mcmc_detector *d, const int8_t *x, float *gx, float *px, float *X, int L)
{
    MixGramArgs g{};
    g.desc = P<ChannelDesc>(d->d_desc);
    g.chains = d->cfg.chains;
    g.L = L;
    g.bt32 = P<float>(d->d_bt32);
    g.z32 = P<float>(d->d_z32);
    g.w32 = P<float>(d->d_w32);
    g.x = x;
    g.gx = gx;
    g.px = px;
    g.X = X;
    return g;
}

MixStepArgs step_args(mcmc_detector *d)
{
    MixStepArgs a{};
    a.desc = P<ChannelDesc>(d->d_desc);
    a.chains = d->cfg.chains;
    a.L = 0;
    if (d->mlp) a.L = d->mlp->Q == 4 ? 2 : d->mlp->Q == 16 ? 4 : 8;
    a.z32 = P<float>(d->d_z32);
    a.w32 = P<float>(d->d_w32);
    a.states = P<int8_t>(d->d_states);
    a.states_out = P<int8_t>(d->d_states);
    a.prop = P<int8_t>(d->d_mx_prop);
    a.gx = P<float>(d->d_mx_gx);
    a.px = P<float>(d->d_mx_px);
    a.gxp = P<float>(d->d_mx_gxp);
    a.pxp = P<float>(d->d_mx_pxp);
    a.logits = P<float>(d->d_mx_logits);
    a.lqf = P<float>(d->d_mx_lqf);
    a.lambda = d->mix_lambda;
    a.l2w_plain = d->mix_lambda < 1.f ? (float)std::log2(1.0 - (double)d->mix_lambda) : -INFINITY;
    a.l2w_nn = d->mix_lambda > 0.f ? (float)std::log2((double)d->mix_lambda) : -INFINITY;
    a.key0 = (uint32_t)(d->cfg.seed & 0xFFFFFFFFu);
    a.key1 = (uint32_t)(d->cfg.seed >> 32);
    a.f = P<double>(d->d_f);
    a.best_f = P<double>(d->d_best_f);
    a.best_states = P<int8_t>(d->d_best_states);
    a.accepts = P<unsigned long long>(d->d_accepts);
    a.status = status_ptr(d);
    return a;
}

cudaError_t net_forward(mcmc_detector *d, long long rows, const float *X, float *logits)
{
    d->launches++;
    return d->mix_tc ? mlp_forward_tc(d->mlp, rows, X, logits, d->stream)
                     : mlp_forward_simt(d->mlp, rows, X, logits, d->stream);
}

}  // namespace

extern "C" {

mcmc_status mcmc_detect_features(mcmc_detector *d, int32_t at_zero, float *X)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!X || (at_zero != 0 && at_zero != 1)) return fail(d, MCMC_EINVAL, "bad arguments");
    mcmc_status st = learned_ok(d);
    if (st != MCMC_OK) return st;
    if (at_zero) {
        CK(launch_features_zero(gram_args(d, nullptr, nullptr, nullptr, X, 0), d->n_channels,
                                d->max_nt, d->stream), "features kernel");
    } else {
        CK(ensure(d->d_mx_gx, 4 * d->tot_states), "alloc scratch");
        CK(ensure(d->d_mx_px, 4 * d->tot_states), "alloc scratch");
        CK(launch_gram_features(gram_args(d, P<int8_t>(d->d_states), P<float>(d->d_mx_gx),
                                          P<float>(d->d_mx_px), X, 0),
                                d->n_channels, d->stream), "features kernel");
    }
    d->launches++;
    return MCMC_OK;
}

mcmc_status mcmc_detect_set_model(mcmc_detector *d, mcmc_mlp *m, float lambda, int32_t tensor_cores)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    if (!m) {
        d->mlp = nullptr;
        return MCMC_OK;
    }
    if (!(lambda >= 0.f && lambda <= 1.f)) return fail(d, MCMC_EINVAL, "lambda must be in [0, 1]");
    if (tensor_cores != 0 && tensor_cores != 1) return fail(d, MCMC_EINVAL, "tensor_cores must be 0 or 1");
    if (d->cfg.precision == MCMC_PREC_FP64)
        return fail(d, MCMC_EUNSUPPORTED, "the learned proposal runs on FP32 or MIXED handles");
    if (!d->cfg.preconditioned)
        return fail(d, MCMC_EUNSUPPORTED, "the learned proposal needs the preconditioned proposal");
    if (tensor_cores && d->cc_major * 10 + d->cc_minor != 103)
        return fail(d, MCMC_EUNSUPPORTED, "tensor-core inference needs sm_103");
    d->mlp = m;
    d->mix_lambda = lambda;
    d->mix_tc = tensor_cores;
    return MCMC_OK;
}

mcmc_status mcmc_detect_init_learned(mcmc_detector *d)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    mcmc_status st = learned_ok(d);
    if (st != MCMC_OK) return st;
    if (!d->mlp) return fail(d, MCMC_ESTATE, "no network attached");
    const long long rows = d->tot_ant;
    CK(ensure(d->d_mx_X, 4 * 6 * (size_t)rows), "alloc scratch");
    CK(ensure(d->d_mx_logits, 4 * (size_t)d->mlp->Q * rows), "alloc scratch");
    CK(launch_features_zero(gram_args(d, nullptr, nullptr, nullptr, P<float>(d->d_mx_X), 0),
                            d->n_channels, d->max_nt, d->stream), "features kernel");
    d->launches++;
    CK(net_forward(d, rows, P<float>(d->d_mx_X), P<float>(d->d_mx_logits)), "network forward");
    CK(launch_mix(2, step_args(d), d->n_channels, d->max_nt, d->stream), "warm start kernel");
    d->launches++;
    // exact energies of the warm-start states, where the running best restarts: evaluated when
    // first needed, as after preprocess
    d->f_valid = false;
    d->f_exact = false;
    d->d_valid = false;
    return MCMC_OK;
}

mcmc_status mcmc_detect_mix_step(mcmc_detector *d, int64_t t)
{
    if (!d) return MCMC_EINVAL;
    d->err.clear();
    mcmc_status st = learned_ok(d);
    if (st != MCMC_OK) return st;
    if (!d->mlp) return fail(d, MCMC_ESTATE, "no network attached");
    if (t < 1 || t > 0xFFFFFFFFll) return fail(d, MCMC_EINVAL, "t out of range");
    st = ensure_energies(d);
    if (st != MCMC_OK) return st;
    const long long rows = d->tot_states / 2;
    for (DevBuf *b : {&d->d_mx_gx, &d->d_mx_px, &d->d_mx_gxp, &d->d_mx_pxp, &d->d_mx_lqf})
        CK(ensure(*b, 4 * (size_t)d->tot_states), "alloc scratch");
    CK(ensure(d->d_mx_prop, d->tot_states), "alloc scratch");
    CK(ensure(d->d_mx_X, 4 * 6 * (size_t)rows), "alloc scratch");
    CK(ensure(d->d_mx_logits, 4 * (size_t)d->mlp->Q * rows), "alloc scratch");
    MixStepArgs a = step_args(d);
    a.t = (uint32_t)t;
    const int L = a.L;
    float *X = P<float>(d->d_mx_X), *lg = P<float>(d->d_mx_logits);
    CK(launch_gram_features(gram_args(d, P<int8_t>(d->d_states), P<float>(d->d_mx_gx),
                                      P<float>(d->d_mx_px), X, L), d->n_channels, d->stream),
       "features kernel");
    CK(net_forward(d, rows, X, lg), "network forward");
    CK(launch_mix(0, a, d->n_channels, d->max_nt, d->stream), "mixture draw kernel");
    CK(launch_gram_features(gram_args(d, P<int8_t>(d->d_mx_prop), P<float>(d->d_mx_gxp),
                                      P<float>(d->d_mx_pxp), X, L), d->n_channels, d->stream),
       "features kernel");
    CK(net_forward(d, rows, X, lg), "network forward");
    CK(launch_mix(1, a, d->n_channels, d->max_nt, d->stream), "mixture accept kernel");
    d->launches += 4;
    d->d_valid = false;
    d->f_exact = false;
    if (d->cfg.refresh_period >= 0) {
        // exact energies after the move, as at the end of a run
        st = refresh_energies(d, P<double>(d->d_f), false, true);
        if (st != MCMC_OK) return st;
        d->f_exact = true;
    }
    long long moved = 0;
    for (const ChannelDesc &c : d->desc)
        if (c.L == L) moved += d->cfg.chains;
    d->transitions += moved;
    return MCMC_OK;
}

}  // extern "C"
