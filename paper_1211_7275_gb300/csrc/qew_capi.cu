// qew_capi.cu -- runtime behind the C ABI declared in include/qew.h: handle, chain and tile
// layout, device buffers, the launch schedule of Euler segments and fused observations, the
// autotuner, and argument checking.
//
// The schedule follows the protocol of arXiv:1211.7275 (Sec. II-III): chains start flat, are
// integrated with explicit Euler steps of size dt, and are observed at chosen step counts; a
// segment of the fused FP32-split kernel never crosses an observation step, so every
// observation sees exactly the state after that many steps.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "qew.h"
#include "qew_internal.h"

using namespace qew;

namespace {

thread_local std::string g_last_error;

static_assert(QEW_RF_GAUSS_LINEAR == kRF && QEW_RB_UNIFORM_CATMULLROM == kRB && QEW_NONE == kNone &&
                  QEW_RB_GAUSS_LINEAR == kRBGLinear && QEW_RB_GAUSS_CATMULLROM == kRBGCubic,
              "the C ABI's disorder kinds index the kernels' kind table");
constexpr int32_t kBlockTile = 1024;   // sites per block tile (FP64 path, init, conversions)
constexpr int64_t kMaxSites = int64_t(1) << 40;

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard()
    {
        if (changed)
            cudaSetDevice(prev);
    }
};

struct TuneKey {
    int64_t n_sites;
    int32_t n_chains;
    int32_t kinds_mask;
    int64_t min_L, max_L;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(n_sites, n_chains, kinds_mask, min_L, max_L) <
               std::tie(o.n_sites, o.n_chains, o.kinds_mask, o.min_L, o.max_L);
    }
};

std::mutex g_tune_mu;
std::map<TuneKey, std::tuple<int, int, int>> g_tune_cache;

}  // namespace

struct qew_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t n_chains = 0;
    std::vector<int64_t> L;
    std::vector<double> f;
    std::vector<int32_t> kind;
    std::vector<uint32_t> sample;   // sample index s of each chain (counter word 2)
    std::vector<int64_t> offset;
    double dt = 0.1;
    uint64_t seed = 0;
    int precision = QEW_FP32_SPLIT;
    int64_t n_sites = 0;
    int64_t step = 0;
    int kinds_mask = 0;
    int n_cache = 2;
    int32_t period = 0;   // disorder period M in u (0: aperiodic)

    // launch shape of the fused kernel (defaults: the best measured shapes on a GB300)
    int S = 23, K = 16, tpc = 2;
    bool autotune_pending = false;

    std::vector<ChainDesc> h_chains;
    ChainDesc* d_chains = nullptr;
    TileDesc* d_tiles[kNumKinds] = {};
    int32_t n_tiles[kNumKinds] = {};
    int32_t tile_base[kNumKinds] = {};
    int32_t w_own[kNumKinds] = {};   // sites a warp tile owns, per disorder kind
    TileDesc* d_btiles = nullptr;
    int32_t n_btiles = 0;

    SplitState sp[2] = {};
    int cur = 0;
    F64State f64 = {};
    double* u64[2] = {nullptr, nullptr};

    double* d_shift = nullptr;
    double* d_partial = nullptr;
    size_t partial_slots = 0;
    double* d_obs = nullptr;
    size_t obs_cap = 0;
    double* h_obs = nullptr;
    size_t h_obs_cap = 0;

    // statistics (qew_enable_stats / qew_get_stats)
    int64_t sites_of_kind[kNumKinds] = {};
    bool stats_on = false;
    int64_t n_launches = 0;
    int64_t n_fused = 0;
    int64_t n_site_updates = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    unsigned long long* d_crossings = nullptr;
    int32_t* d_error = nullptr;   // set by a kernel whose bounded wait gave up

    // structure factor: cuFFT plan of the handle's chain length and batch (made on first use)
    cufftHandle sq_plan = 0;
    bool sq_plan_made = false;

    // stream owned by the handle (used unless the caller sets one) and the captured observation graph
    cudaStream_t own_stream = nullptr;
    bool use_graphs = true;
    cudaGraphExec_t gexec = nullptr;
    std::vector<int64_t> g_steps;
    int64_t g_step0 = -1, g_step1 = 0;
    int g_cur0 = -1, g_cur1 = 0;
    int g_shape[4] = {0, 0, 0, 0};
    int64_t g_launches = 0, g_fused = 0, g_su = 0;

    std::string err;
};

namespace {

int fail(qew_ctx* h, int code, const std::string& msg)
{
    if (h)
        h->err = msg;
    g_last_error = msg;
    return code;
}

int cuda_fail(qew_ctx* h, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error where possible
    return fail(h, e == cudaErrorMemoryAllocation ? QEW_ENOMEM : QEW_ECUDA, m);
}

#define QEW_CUDA(h, call, where)                     \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess)                       \
            return cuda_fail((h), e_, (where));      \
    } while (0)

template <class T>
cudaError_t dev_alloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0)
        return cudaSuccess;
    return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

template <class T>
void dev_free(T*& p)
{
    if (p)
        cudaFree(p);
    p = nullptr;
}

void free_split(qew_ctx* h)
{
    for (int b = 0; b < 2; ++b) {
        dev_free(h->sp[b].cell);
        dev_free(h->sp[b].off);
        dev_free(h->sp[b].rf);
        dev_free(h->sp[b].qn);
        dev_free(h->sp[b].q3);
        dev_free(h->sp[b].qab);
        dev_free(h->sp[b].qc);
    }
}

void free_f64(qew_ctx* h)
{
    dev_free(h->u64[0]);
    dev_free(h->u64[1]);
    dev_free(h->f64.ncache);
    for (int c = 0; c < 4; ++c)
        dev_free(h->f64.c[c]);
    h->f64.u = nullptr;
}

void free_events(qew_ctx* h)
{
    for (cudaEvent_t e : h->ev_pool)
        cudaEventDestroy(e);
    h->ev_pool.clear();
    h->ev_used = 0;
}

void drop_graph(qew_ctx* h)
{
    if (h->gexec)
        cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->g_steps.clear();
    h->g_step0 = -1;
}

void free_all(qew_ctx* h)
{
    drop_graph(h);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    h->own_stream = nullptr;
    free_events(h);
    dev_free(h->d_crossings);
    dev_free(h->d_error);
    free_split(h);
    free_f64(h);
    dev_free(h->d_chains);
    for (int k = 0; k < kNumKinds; ++k)
        dev_free(h->d_tiles[k]);
    dev_free(h->d_btiles);
    dev_free(h->d_shift);
    dev_free(h->d_partial);
    dev_free(h->d_obs);
    if (h->h_obs)
        cudaFreeHost(h->h_obs);
    h->h_obs = nullptr;
    if (h->sq_plan_made)
        cufftDestroy(h->sq_plan);
    h->sq_plan_made = false;
}

int alloc_state(qew_ctx* h)
{
    const size_t N = static_cast<size_t>(h->n_sites);
    if (h->precision == QEW_FP32_SPLIT) {
        free_f64(h);
        if (h->sp[0].cell)
            return QEW_OK;
        for (int b = 0; b < 2; ++b) {
            QEW_CUDA(h, dev_alloc(&h->sp[b].cell, N), "allocating the cell array");
            QEW_CUDA(h, dev_alloc(&h->sp[b].off, N), "allocating the offset array");
            if (h->kinds_mask & kPairMask)
                QEW_CUDA(h, dev_alloc(&h->sp[b].rf, N), "allocating the two-node disorder cache");
            if (h->kinds_mask & kQuadMask) {
                QEW_CUDA(h, dev_alloc(&h->sp[b].qn, N), "allocating the cubic disorder cache");
                QEW_CUDA(h, dev_alloc(&h->sp[b].q3, N), "allocating the cubic disorder cache");
                QEW_CUDA(h, dev_alloc(&h->sp[b].qab, N), "allocating the cubic disorder cache");
                QEW_CUDA(h, dev_alloc(&h->sp[b].qc, N), "allocating the cubic disorder cache");
            }
        }
    } else {
        free_split(h);
        if (h->u64[0])
            return QEW_OK;
        QEW_CUDA(h, dev_alloc(&h->u64[0], N), "allocating the FP64 state");
        QEW_CUDA(h, dev_alloc(&h->u64[1], N), "allocating the FP64 state");
        QEW_CUDA(h, dev_alloc(&h->f64.ncache, N), "allocating the FP64 cache cells");
        for (int c = 0; c < h->n_cache; ++c)
            QEW_CUDA(h, dev_alloc(&h->f64.c[c], N), "allocating the FP64 disorder cache");
    }
    return QEW_OK;
}

// Sites per lane that chains of `kind` use under the requested S: the largest width the kind
// supports up to S (every kind supports 7), so that in a mixed batch each kind gets its own
// widest tile.
int kind_S(int kind, int S)
{
    const int all[] = {39, 31, 23, 15, 7};
    for (int s : all)
        if (s <= S && split_supported(kind, s))
            return s;
    return 7;
}

// The narrowest tile among the kinds present: K is bounded by it.
int min_kind_S(const qew_ctx* h, int S)
{
    int m = S;
    for (int k = 0; k < kNumKinds; ++k)
        if (h->kinds_mask >> k & 1)
            m = std::min(m, kind_S(k, S));
    return m;
}

// Largest shared-memory footprint among the kinds present, for S sites per lane requested.
size_t max_kind_smem(const qew_ctx* h, int S, int tiles_per_cta)
{
    size_t m = 0;
    for (int k = 0; k < kNumKinds; ++k)
        if (h->kinds_mask >> k & 1)
            m = std::max(m, split_smem_bytes(k, kind_S(k, S), tiles_per_cta));
    return m;
}

// Tile lists for the current precision and launch shape; uploads chain descriptors and sizes
// the partial-sum buffer.
int build_layout(qew_ctx* h)
{
    drop_graph(h);   // captured launches point at the descriptors rebuilt here
    for (int k = 0; k < kNumKinds; ++k)
        h->w_own[k] = 32 * kind_S(k, h->S) - 2 * h->K;
    std::vector<TileDesc> lists[kNumKinds];
    std::vector<TileDesc> blocks;
    h->h_chains.assign(h->n_chains, ChainDesc{});
    std::vector<int32_t> first(h->n_chains), count(h->n_chains);
    for (int32_t c = 0; c < h->n_chains; ++c) {
        ChainDesc& d = h->h_chains[c];
        d.offset = h->offset[c];
        d.L = static_cast<int32_t>(h->L[c]);
        d.s = h->sample[c];
        d.kind = h->kind[c];
        d.f32 = static_cast<float>(h->f[c]);
        d.period = h->period;
        d.f64 = h->f[c];
        for (int64_t st = 0; st < d.L; st += kBlockTile)   // 64-bit: L may reach 2^31 - 1
            blocks.push_back(TileDesc{c, static_cast<int32_t>(st)});
        if (h->precision == QEW_FP32_SPLIT) {
            auto& lst = lists[d.kind];
            first[c] = static_cast<int32_t>(lst.size());
            for (int64_t st = 0; st < d.L; st += h->w_own[d.kind])
                lst.push_back(TileDesc{c, static_cast<int32_t>(st)});
            count[c] = static_cast<int32_t>(lst.size()) - first[c];
        }
    }
    size_t slots = 0;
    if (h->precision == QEW_FP32_SPLIT) {
        int32_t base = 0;
        for (int k = 0; k < kNumKinds; ++k) {
            h->tile_base[k] = base;
            h->n_tiles[k] = static_cast<int32_t>(lists[k].size());
            base += h->n_tiles[k];
        }
        for (int32_t c = 0; c < h->n_chains; ++c) {
            h->h_chains[c].tile0 = h->tile_base[h->kind[c]] + first[c];
            h->h_chains[c].ntiles = count[c];
        }
        slots = static_cast<size_t>(base);
    } else {
        int32_t b = 0;
        for (int32_t c = 0; c < h->n_chains; ++c) {
            const int32_t nb = static_cast<int32_t>((h->L[c] + kBlockTile - 1) / kBlockTile);
            h->h_chains[c].tile0 = b;
            h->h_chains[c].ntiles = nb;
            b += nb;
        }
        slots = static_cast<size_t>(b);
        for (int k = 0; k < kNumKinds; ++k)
            h->n_tiles[k] = 0;
    }
    dev_free(h->d_chains);
    for (int k = 0; k < kNumKinds; ++k)
        dev_free(h->d_tiles[k]);
    dev_free(h->d_btiles);
    QEW_CUDA(h, dev_alloc(&h->d_chains, h->h_chains.size()), "allocating chain descriptors");
    QEW_CUDA(h, cudaMemcpy(h->d_chains, h->h_chains.data(), h->h_chains.size() * sizeof(ChainDesc),
                           cudaMemcpyHostToDevice), "uploading chain descriptors");
    for (int k = 0; k < kNumKinds; ++k) {
        if (lists[k].empty())
            continue;
        QEW_CUDA(h, dev_alloc(&h->d_tiles[k], lists[k].size()), "allocating tile lists");
        QEW_CUDA(h, cudaMemcpy(h->d_tiles[k], lists[k].data(), lists[k].size() * sizeof(TileDesc),
                               cudaMemcpyHostToDevice), "uploading tile lists");
    }
    h->n_btiles = static_cast<int32_t>(blocks.size());
    QEW_CUDA(h, dev_alloc(&h->d_btiles, blocks.size()), "allocating block tiles");
    QEW_CUDA(h, cudaMemcpy(h->d_btiles, blocks.data(), blocks.size() * sizeof(TileDesc), cudaMemcpyHostToDevice),
             "uploading block tiles");
    if (slots > h->partial_slots) {
        dev_free(h->d_partial);
        QEW_CUDA(h, dev_alloc(&h->d_partial, slots * 3), "allocating partial sums");
        h->partial_slots = slots;
    }
    return QEW_OK;
}

// Flat start (u_in == nullptr) or the given device FP64 state; step counter to 0 and the
// reference shifts to `shift0`.
int init_state(qew_ctx* h, const double* d_u_in, const std::vector<double>& shift0)
{
    h->cur = 0;
    h->step = 0;
    if (h->precision == QEW_FP32_SPLIT) {
        QEW_CUDA(h, split_init(h->d_chains, h->n_chains, h->d_btiles, h->n_btiles, kBlockTile, h->sp[0], h->seed,
                               h->kinds_mask & kQuadMask, d_u_in, h->stream), "launching the state initialisation");
    } else {
        h->f64.u = h->u64[0];
        QEW_CUDA(h, f64_init(h->d_chains, h->d_btiles, h->n_btiles, kBlockTile, h->f64, h->seed, h->kinds_mask & kQuadMask,
                             d_u_in, h->stream), "launching the FP64 state initialisation");
    }
    h->n_launches += 1;
    QEW_CUDA(h, cudaMemcpyAsync(h->d_shift, shift0.data(), shift0.size() * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream), "setting reference shifts");
    QEW_CUDA(h, cudaStreamSynchronize(h->stream), "initialising the state");
    return QEW_OK;
}

SplitLaunch split_args(qew_ctx* h, int kind, int K, int do_obs, SplitState in, SplitState out)
{
    SplitLaunch a{};
    a.tiles = h->d_tiles[kind];
    a.n_tiles = h->n_tiles[kind];
    a.tile_base = h->tile_base[kind];
    a.chains = h->d_chains;
    a.in = in;
    a.out = out;
    a.K = K;
    a.w_own = h->w_own[kind];
    a.dt = static_cast<float>(h->dt);
    a.seed = h->seed;
    a.do_obs = do_obs;
    a.shift = h->d_shift;
    a.partial = h->d_partial;
    a.crossings = h->stats_on ? h->d_crossings : nullptr;
    a.error = h->d_error;
    a.keys = philox_key_schedule(h->seed);
    return a;
}

int next_event(qew_ctx* h, cudaEvent_t* ev)
{
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        QEW_CUDA(h, cudaEventCreate(&e), "creating a timing event");
        h->ev_pool.push_back(e);
    }
    *ev = h->ev_pool[h->ev_used++];
    return QEW_OK;
}

int launch_split_all(qew_ctx* h, int K, int do_obs, SplitState in, SplitState out)
{
    for (int k = 0; k < kNumKinds; ++k) {
        if (h->n_tiles[k] == 0)
            continue;
        const SplitLaunch a = split_args(h, k, K, do_obs, in, out);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (h->stats_on) {
            int rc = next_event(h, &e0);
            if (rc == QEW_OK)
                rc = next_event(h, &e1);
            if (rc != QEW_OK)
                return rc;
            QEW_CUDA(h, cudaEventRecord(e0, h->stream), "recording a timing event");
        }
        QEW_CUDA(h, split_step(k, kind_S(k, h->S), h->tpc, a, h->stream), "launching the fused step kernel");
        if (h->stats_on)
            QEW_CUDA(h, cudaEventRecord(e1, h->stream), "recording a timing event");
        h->n_launches += 1;
        h->n_fused += 1;
        h->n_site_updates += h->sites_of_kind[k] * K;
    }
    return QEW_OK;
}

F64Launch f64_args(qew_ctx* h)
{
    F64Launch a{};
    a.tiles = h->d_btiles;
    a.n_tiles = h->n_btiles;
    a.w_tile = kBlockTile;
    a.chains = h->d_chains;
    a.st = h->f64;
    a.u_in = h->u64[h->cur];
    a.u_out = h->u64[h->cur ^ 1];
    a.dt = h->dt;
    a.seed = h->seed;
    a.shift = h->d_shift;
    a.partial = h->d_partial;
    return a;
}

int autotune(qew_ctx* h);

// Range check of the FP32-split state (neighbouring cells less than 2^12 apart), at the end of every
// call that advances the chains; a violation is reported by the next check_device_error.
int guard_range(qew_ctx* h)
{
    if (h->precision != QEW_FP32_SPLIT)
        return QEW_OK;
    QEW_CUDA(h, split_range_guard(h->d_chains, h->n_chains, *std::max_element(h->L.begin(), h->L.end()),
                                  h->sp[h->cur].cell, h->d_error, h->stream), "launching the range guard");
    h->n_launches += 1;
    return QEW_OK;
}

// The autotuner times candidate shapes only once the chains are this many steps past the flat
// start.  The best shape changes while the crossing rate decays: measured on 4 x 2^25 random-
// field chains at f_c, 736-site tiles are 4% faster than 992-site ones over steps 0-256, equal
// over 256-768, and 6% slower after step 2048 (the larger tiles fill their regeneration rounds
// better).  Step 1024 is past the crossover.
constexpr int64_t kTuneAfterSteps = 1024;

// Advance to `target` (>= current step); with `obs` record the observables there into obs.
int run_to(qew_ctx* h, int64_t target, double* obs)
{
    if (h->precision == QEW_FP32_SPLIT) {
        bool observed = false;
        while (h->step < target) {
            if (h->autotune_pending && h->step >= kTuneAfterSteps) {
                int rc = autotune(h);
                if (rc != QEW_OK)
                    return rc;
            }
            int64_t seg_end = target;
            if (h->autotune_pending && h->step < kTuneAfterSteps)
                seg_end = std::min<int64_t>(target, kTuneAfterSteps);
            const int Keff = static_cast<int>(std::min<int64_t>(h->K, seg_end - h->step));
            const bool last = (h->step + Keff == target);
            const int do_obs = (obs != nullptr && last) ? 1 : 0;
            int rc = launch_split_all(h, Keff, do_obs, h->sp[h->cur], h->sp[h->cur ^ 1]);
            if (rc != QEW_OK)
                return rc;
            h->cur ^= 1;
            h->step += Keff;
            observed = observed || do_obs;
        }
        if (obs && !observed) {
            int rc = launch_split_all(h, 0, 1, h->sp[h->cur], h->sp[h->cur ^ 1]);
            if (rc != QEW_OK)
                return rc;
        }
        if (obs) {
            QEW_CUDA(h, reduce_chains(h->d_chains, h->n_chains, h->d_partial, h->d_shift, obs, 1, h->stream),
                     "launching the observable reduction");
            h->n_launches += 1;
        }
    } else {
        while (h->step < target) {
            QEW_CUDA(h, f64_step(f64_args(h), h->stream), "launching the FP64 step kernel");
            h->cur ^= 1;
            h->f64.u = h->u64[h->cur];
            ++h->step;
            h->n_launches += 1;
            h->n_site_updates += h->n_sites;
        }
        if (obs) {
            QEW_CUDA(h, f64_observe(f64_args(h), h->stream), "launching the FP64 observation kernel");
            QEW_CUDA(h, reduce_chains(h->d_chains, h->n_chains, h->d_partial, h->d_shift, obs, 1, h->stream),
                     "launching the observable reduction");
            h->n_launches += 2;
        }
    }
    return QEW_OK;
}

// Times candidate launch shapes on the handle's own chains: each trial launch reads the
// current state and writes the other ping-pong buffer, so the state is unchanged.
int autotune(qew_ctx* h)
{
    h->autotune_pending = false;
    TuneKey key{h->n_sites, h->n_chains, h->kinds_mask,
                *std::min_element(h->L.begin(), h->L.end()), *std::max_element(h->L.begin(), h->L.end())};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            std::tie(h->S, h->K, h->tpc) = it->second;
            return build_layout(h);
        }
    }
    const int S_all[] = {7, 15, 23, 31, 39};
    const int K_all[] = {4, 8, 16, 32};
    const int T_all[] = {1, 2, 4};
    float best = 1e30f;
    int bS = h->S, bK = h->K, bT = h->tpc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess)
        ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        if (e0)
            cudaEventDestroy(e0);
        return cuda_fail(h, ce, "creating tuning events");
    }
    int rc = QEW_OK;
    for (int S : S_all) {
        // a requested width that no kind present runs would repeat a narrower candidate
        bool used = false;
        for (int k = 0; k < kNumKinds; ++k)
            if ((h->kinds_mask >> k & 1) && kind_S(k, S) == S)
                used = true;
        if (!used)
            continue;
        for (int K : K_all) {
            if (4 * K > 32 * min_kind_S(h, S))
                continue;
            for (int T : T_all) {
                if (max_kind_smem(h, S, T) > 200 * 1024)
                    continue;
                h->S = S;
                h->K = K;
                h->tpc = T;
                rc = build_layout(h);
                // best of four timed repetitions (after one untimed), each two launches long, so a
                // shape wins by its throughput rather than by the noise of a single launch
                float ms_best = 1e30f;
                for (int rep = 0; rep < 5 && rc == QEW_OK; ++rep) {
                    cudaEventRecord(e0, h->stream);
                    for (int l = 0; l < 2 && rc == QEW_OK; ++l)
                        rc = launch_split_all(h, K, 0, h->sp[h->cur], h->sp[h->cur ^ 1]);
                    if (rc != QEW_OK)
                        break;
                    cudaEventRecord(e1, h->stream);
                    ce = cudaEventSynchronize(e1);
                    if (ce != cudaSuccess) {
                        rc = cuda_fail(h, ce, "timing a tuning candidate");
                        break;
                    }
                    float ms = 0;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0)
                        ms_best = std::min(ms_best, 0.5f * ms);
                }
                if (rc != QEW_OK)
                    break;
                const float per = ms_best / static_cast<float>(K);
                if (per < best) {
                    best = per;
                    bS = S;
                    bK = K;
                    bT = T;
                }
            }
            if (rc != QEW_OK)
                break;
        }
        if (rc != QEW_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != QEW_OK)
        return rc;
    h->S = bS;
    h->K = bK;
    h->tpc = bT;
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        g_tune_cache[key] = std::make_tuple(bS, bK, bT);
    }
    return build_layout(h);
}

int validate_common(double dt, uint64_t)
{
    if (!(dt > 0.0 && dt < 0.5))
        return fail(nullptr, QEW_EINVAL, "dt must lie in (0, 0.5)");
    return QEW_OK;
}

int create_impl(qew_handle* out, int32_t n_chains, const int64_t* L, const double* f, const int32_t* kind, double dt,
                uint64_t seed, int32_t precision)
{
    if (!out)
        return fail(nullptr, QEW_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n_chains < 1)
        return fail(nullptr, QEW_EINVAL, "need at least one chain");
    if (!L || !f || !kind)
        return fail(nullptr, QEW_EINVAL, "L, f and kind must not be NULL");
    int rc = validate_common(dt, seed);
    if (rc != QEW_OK)
        return rc;
    if (precision != QEW_FP32_SPLIT && precision != QEW_FP64)
        return fail(nullptr, QEW_EINVAL, "precision must be QEW_FP32_SPLIT or QEW_FP64");
    int64_t total = 0;
    for (int32_t c = 0; c < n_chains; ++c) {
        if (L[c] < 1 || L[c] >= (int64_t(1) << 31))
            return fail(nullptr, QEW_EINVAL, "chain length " + std::to_string(L[c]) + " outside [1, 2^31)");
        if (!std::isfinite(f[c]) || std::fabs(f[c]) >= 4096.0)
            return fail(nullptr, QEW_EINVAL, "drive f must be finite with |f| < 2^12");
        if (kind[c] < QEW_RF_GAUSS_LINEAR || kind[c] > QEW_RB_GAUSS_CATMULLROM)
            return fail(nullptr, QEW_EINVAL, "unknown disorder kind " + std::to_string(kind[c]));
        total += L[c];
        if (total >= kMaxSites)
            return fail(nullptr, QEW_EINVAL, "total number of sites must be below 2^40");
    }
    qew_ctx* h = new (std::nothrow) qew_ctx();
    if (!h)
        return fail(nullptr, QEW_ENOMEM, "host allocation of the handle failed");
    try {
        cudaGetDevice(&h->device);
        if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return fail(nullptr, QEW_ECUDA, "creating the handle's stream failed");
        }
        h->stream = h->own_stream;
        h->n_chains = n_chains;
        h->L.assign(L, L + n_chains);
        h->f.assign(f, f + n_chains);
        h->kind.assign(kind, kind + n_chains);
        h->sample.resize(n_chains);
        for (int32_t c = 0; c < n_chains; ++c)
            h->sample[c] = static_cast<uint32_t>(c);
        h->offset.resize(n_chains);
        int64_t off = 0;
        for (int32_t c = 0; c < n_chains; ++c) {
            h->offset[c] = off;
            off += L[c];
            h->kinds_mask |= 1 << kind[c];
            h->sites_of_kind[kind[c]] += L[c];
        }
        h->n_sites = off;
        h->n_cache = (h->kinds_mask & kQuadMask) ? 4 : 2;
        h->dt = dt;
        h->seed = seed;
        h->precision = precision;
        if (h->kinds_mask & kQuadMask)
            h->S = 7;   // four-node caches are larger: 7 sites per lane
        rc = build_layout(h);
        if (rc == QEW_OK)
            rc = alloc_state(h);
        if (rc == QEW_OK) {
            cudaError_t e = dev_alloc(&h->d_shift, static_cast<size_t>(n_chains));
            if (e == cudaSuccess)
                e = dev_alloc(&h->d_error, 1);
            if (e == cudaSuccess)
                e = cudaMemset(h->d_error, 0, sizeof(int32_t));
            if (e != cudaSuccess)
                rc = cuda_fail(h, e, "allocating reference shifts");
        }
        if (rc == QEW_OK)
            rc = init_state(h, nullptr, std::vector<double>(n_chains, 0.0));
    } catch (const std::bad_alloc&) {
        rc = fail(h, QEW_ENOMEM, "host allocation failed");
    }
    if (rc != QEW_OK) {
        g_last_error = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return QEW_OK;
}

int check_handle(qew_handle h)
{
    if (!h)
        return fail(nullptr, QEW_EINVAL, "handle must not be NULL");
    return QEW_OK;
}

// A kernel whose bounded wait on a bulk copy gave up leaves 1 in d_error; one whose range guard
// found neighbouring cells 2^12 or more apart leaves 2.  Report it once.
int check_device_error(qew_ctx* h)
{
    int32_t flag = 0;
    QEW_CUDA(h, cudaMemcpy(&flag, h->d_error, sizeof(flag), cudaMemcpyDeviceToHost), "reading the error flag");
    if (flag) {
        cudaMemset(h->d_error, 0, sizeof(int32_t));
        if (flag == 2)
            return fail(h, QEW_ESTATE, "neighbouring displacements reached 2^12 cells, outside the range the "
                                       "FP32-split kernel represents exactly; the state is no longer valid");
        return fail(h, QEW_ETIMEOUT, "a bounded wait for a bulk copy gave up; the state is no longer valid");
    }
    return QEW_OK;
}

int ensure_obs(qew_ctx* h, size_t n)
{
    if (n > h->obs_cap || n > h->h_obs_cap)
        drop_graph(h);   // the captured copy-out targets these buffers
    if (n > h->obs_cap) {
        dev_free(h->d_obs);
        QEW_CUDA(h, dev_alloc(&h->d_obs, n), "allocating observation buffer");
        h->obs_cap = n;
    }
    if (n > h->h_obs_cap) {
        if (h->h_obs)
            cudaFreeHost(h->h_obs);
        h->h_obs = nullptr;
        QEW_CUDA(h, cudaMallocHost(reinterpret_cast<void**>(&h->h_obs), n * sizeof(double)),
                 "allocating pinned observation buffer");
        h->h_obs_cap = n;
    }
    return QEW_OK;
}

int observe_impl(qew_ctx* h, const int64_t* steps, int32_t n_times, double* v_out, double* ubar_out,
                 double* w2_out)
{
    if (n_times < 0)
        return fail(h, QEW_EINVAL, "n_times must be >= 0");
    if (n_times == 0)
        return QEW_OK;
    if (!steps)
        return fail(h, QEW_EINVAL, "steps must not be NULL");
    if (steps[0] < h->step)
        return fail(h, QEW_EINVAL, "steps[0] = " + std::to_string(steps[0]) + " lies before the current step " +
                                       std::to_string(h->step));
    for (int32_t k = 1; k < n_times; ++k)
        if (steps[k] <= steps[k - 1])
            return fail(h, QEW_EINVAL, "steps must be strictly increasing");
    const size_t per = static_cast<size_t>(h->n_chains) * 4;
    int rc = ensure_obs(h, per * n_times);
    if (rc != QEW_OK)
        return rc;
    if (h->autotune_pending && h->precision == QEW_FP32_SPLIT && h->step >= kTuneAfterSteps) {
        rc = autotune(h);   // allocates: never inside a capture
        if (rc != QEW_OK)
            return rc;
    }
    // launches this schedule needs (a graph is worth it, and stays small, only up to a bound)
    int64_t n_launch = 0, at = h->step;
    for (int32_t k = 0; k < n_times; ++k) {
        const int64_t seg = steps[k] - at;
        n_launch += (h->precision == QEW_FP32_SPLIT) ? (seg + h->K - 1) / h->K + 2 : seg + 2;
        at = steps[k];
    }
    const int shape[4] = {h->S, h->K, h->tpc, h->precision};
    const bool graphable = h->use_graphs && !h->stats_on && !h->autotune_pending && n_launch <= 20000 &&
                           h->stream != nullptr;
    const bool replay = graphable && h->gexec && h->g_step0 == h->step && h->g_cur0 == h->cur &&
                        std::memcmp(h->g_shape, shape, sizeof(shape)) == 0 &&
                        h->g_steps.size() == static_cast<size_t>(n_times) &&
                        std::equal(h->g_steps.begin(), h->g_steps.end(), steps);
    if (replay) {
        QEW_CUDA(h, cudaGraphLaunch(h->gexec, h->stream), "replaying the observation graph");
        h->step = h->g_step1;
        h->cur = h->g_cur1;
        h->f64.u = h->u64[h->cur];
        h->n_launches += h->g_launches;
        h->n_fused += h->g_fused;
        h->n_site_updates += h->g_su;
    } else {
        const int64_t step0 = h->step;
        const int cur0 = h->cur;
        const int64_t l0 = h->n_launches, f0 = h->n_fused, s0 = h->n_site_updates;
        bool capturing = false;
        if (graphable) {
            drop_graph(h);
            capturing = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (!capturing)
                cudaGetLastError();
        }
        for (int32_t k = 0; k < n_times && rc == QEW_OK; ++k)
            rc = run_to(h, steps[k], h->d_obs + per * k);
        if (rc == QEW_OK)
            rc = guard_range(h);
        cudaError_t ce = cudaSuccess;
        if (rc == QEW_OK)
            ce = cudaMemcpyAsync(h->h_obs, h->d_obs, per * n_times * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (capturing) {
            cudaGraph_t graph = nullptr;
            cudaError_t ee = cudaStreamEndCapture(h->stream, &graph);
            if (rc != QEW_OK || ce != cudaSuccess || ee != cudaSuccess) {
                if (graph)
                    cudaGraphDestroy(graph);
                h->step = step0;   // nothing ran: undo the host-side bookkeeping
                h->cur = cur0;
                h->f64.u = h->u64[h->cur];
                if (rc != QEW_OK)
                    return rc;
                return cuda_fail(h, ce != cudaSuccess ? ce : ee, "capturing the observation graph");
            }
            ce = cudaGraphInstantiate(&h->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) {
                h->gexec = nullptr;
                h->step = step0;
                h->cur = cur0;
                h->f64.u = h->u64[h->cur];
                return cuda_fail(h, ce, "instantiating the observation graph");
            }
            h->g_steps.assign(steps, steps + n_times);
            h->g_step0 = step0;
            h->g_cur0 = cur0;
            h->g_step1 = h->step;
            h->g_cur1 = h->cur;
            std::memcpy(h->g_shape, shape, sizeof(shape));
            h->g_launches = h->n_launches - l0;
            h->g_fused = h->n_fused - f0;
            h->g_su = h->n_site_updates - s0;
            QEW_CUDA(h, cudaGraphLaunch(h->gexec, h->stream), "launching the observation graph");
        } else {
            if (rc != QEW_OK)
                return rc;
            QEW_CUDA(h, ce, "copying observables to the host");
        }
    }
    QEW_CUDA(h, cudaStreamSynchronize(h->stream), "running the relaxation");
    if (int rc2 = check_device_error(h))
        return rc2;
    bool finite = true;
    for (int32_t k = 0; k < n_times; ++k) {
        for (int32_t c = 0; c < h->n_chains; ++c) {
            const double* o = h->h_obs + per * k + 4 * c;
            const double Ld = static_cast<double>(h->L[c]);
            const double m1 = o[1] / Ld;
            const double v = h->f[c] + o[0] / Ld;
            const double ub = o[3] + m1;
            const double w2 = o[2] / Ld - m1 * m1;
            const size_t idx = static_cast<size_t>(k) * h->n_chains + c;
            if (v_out)
                v_out[idx] = v;
            if (ubar_out)
                ubar_out[idx] = ub;
            if (w2_out)
                w2_out[idx] = w2;
            finite = finite && std::isfinite(v) && std::isfinite(ub) && std::isfinite(w2);
        }
    }
    if (!finite)
        return fail(h, QEW_ENONFINITE, "an observable is not finite");
    return QEW_OK;
}

int get_state_impl(qew_ctx* h, double* u_out, int32_t* cells_out, int64_t* step_out)
{
    const size_t N = static_cast<size_t>(h->n_sites);
    if (step_out)
        *step_out = h->step;
    if (!u_out && !cells_out)
        return QEW_OK;
    double* d_u = nullptr;
    int32_t* d_c = nullptr;
    int rc = QEW_OK;
    cudaError_t e = cudaSuccess;
    if (u_out && h->precision == QEW_FP32_SPLIT)
        e = dev_alloc(&d_u, N);
    if (e == cudaSuccess && cells_out)
        e = dev_alloc(&d_c, N);
    if (e != cudaSuccess) {
        rc = cuda_fail(h, e, "allocating a state copy");
    } else if (h->precision == QEW_FP32_SPLIT) {
        e = split_to_f64(h->d_chains, h->d_btiles, h->n_btiles, kBlockTile, h->sp[h->cur], d_u, d_c, h->stream);
        if (e == cudaSuccess && u_out)
            e = cudaMemcpyAsync(u_out, d_u, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    } else {
        if (cells_out)
            e = f64_cells(h->d_chains, h->d_btiles, h->n_btiles, kBlockTile, h->u64[h->cur], d_c, h->stream);
        if (e == cudaSuccess && u_out)
            e = cudaMemcpyAsync(u_out, h->u64[h->cur], N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    }
    if (rc == QEW_OK && e == cudaSuccess && cells_out)
        e = cudaMemcpyAsync(cells_out, d_c, N * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (rc == QEW_OK && e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    if (rc == QEW_OK && e != cudaSuccess)
        rc = cuda_fail(h, e, "reading the state");
    if (rc == QEW_OK)
        rc = check_device_error(h);
    dev_free(d_u);
    dev_free(d_c);
    return rc;
}

int set_state_impl(qew_ctx* h, const double* u_in)
{
    const size_t N = static_cast<size_t>(h->n_sites);
    std::vector<double> shift0(h->n_chains, 0.0);
    for (int32_t c = 0; c < h->n_chains; ++c) {
        double acc = 0.0;
        const double* uc = u_in + h->offset[c];
        for (int64_t i = 0; i < h->L[c]; ++i) {
            const double u = uc[i];
            if (!std::isfinite(u) || std::fabs(u) >= 1073741824.0)
                return fail(h, QEW_EINVAL, "state values must be finite with |u| < 2^30");
            const double un = uc[i + 1 == h->L[c] ? 0 : i + 1];
            if (std::isfinite(un) && std::fabs(un - u) >= 4096.0)
                return fail(h, QEW_EINVAL, "neighbouring displacements must differ by less than 2^12");
            acc += u;
        }
        shift0[c] = std::floor(acc / static_cast<double>(h->L[c]) + 0.5);
    }
    double* d_u = nullptr;
    cudaError_t e = dev_alloc(&d_u, N);
    if (e != cudaSuccess)
        return cuda_fail(h, e, "allocating a state copy");
    e = cudaMemcpy(d_u, u_in, N * sizeof(double), cudaMemcpyHostToDevice);
    int rc = (e == cudaSuccess) ? init_state(h, d_u, shift0) : cuda_fail(h, e, "uploading the state");
    dev_free(d_u);
    return rc;
}

}  // namespace

void qew::set_last_error(const std::string& msg)
{
    g_last_error = msg;
}

extern "C" {

int qew_create(qew_handle* out, int64_t L, int32_t batch, double f, double dt, int32_t disorder_kind, uint64_t seed)
{
    if (batch < 1)
        return fail(nullptr, QEW_EINVAL, "batch must be >= 1");
    try {
        std::vector<int64_t> Ls(batch, L);
        std::vector<double> fs(batch, f);
        std::vector<int32_t> ks(batch, disorder_kind);
        return create_impl(out, batch, Ls.data(), fs.data(), ks.data(), dt, seed, QEW_FP32_SPLIT);
    } catch (const std::bad_alloc&) {
        return fail(nullptr, QEW_ENOMEM, "host allocation failed");
    }
}

int qew_create_batch(qew_handle* out, int32_t n_chains, const int64_t* L, const double* f, const int32_t* kind,
                     double dt, uint64_t seed, int32_t precision)
{
    return create_impl(out, n_chains, L, f, kind, dt, seed, precision);
}

int qew_set_precision(qew_handle h, int32_t precision)
{
    if (int rc = check_handle(h))
        return rc;
    if (precision != QEW_FP32_SPLIT && precision != QEW_FP64)
        return fail(h, QEW_EINVAL, "precision must be QEW_FP32_SPLIT or QEW_FP64");
    if (h->step != 0)
        return fail(h, QEW_ESTATE, "precision can only change before the first step");
    DeviceGuard g(h->device);
    h->precision = precision;
    int rc = build_layout(h);
    if (rc == QEW_OK)
        rc = alloc_state(h);
    if (rc == QEW_OK)
        rc = init_state(h, nullptr, std::vector<double>(h->n_chains, 0.0));
    return rc;
}

int qew_set_disorder_period(qew_handle h, int64_t period)
{
    if (int rc = check_handle(h))
        return rc;
    if (period < 0 || period >= (int64_t(1) << 31))
        return fail(h, QEW_EINVAL, "period must lie in [0, 2^31)");
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    h->period = static_cast<int32_t>(period);
    int rc = build_layout(h);
    if (rc == QEW_OK)
        rc = init_state(h, nullptr, std::vector<double>(h->n_chains, 0.0));
    return rc;
}

int qew_set_samples(qew_handle h, const uint32_t* s)
{
    if (int rc = check_handle(h))
        return rc;
    if (!s)
        return fail(h, QEW_EINVAL, "s must not be NULL");
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    h->sample.assign(s, s + h->n_chains);
    int rc = build_layout(h);
    if (rc == QEW_OK)
        rc = init_state(h, nullptr, std::vector<double>(h->n_chains, 0.0));
    return rc;
}

int qew_set_stream(qew_handle h, void* stream)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    drop_graph(h);
    h->stream = stream ? static_cast<cudaStream_t>(stream) : h->own_stream;
    return QEW_OK;
}

int qew_set_tuning(qew_handle h, int32_t tile_w, int32_t K, int32_t tiles_per_cta)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    if (tile_w == 0 && K == 0 && tiles_per_cta == 0) {
        h->autotune_pending = true;
        return QEW_OK;
    }
    if (tile_w % 32 != 0)
        return fail(h, QEW_EINVAL, "tile_w must be one of 224, 480, 736, 992, 1248");
    const int S = tile_w / 32;
    if (S != 7 && S != 15 && S != 23 && S != 31 && S != 39)
        return fail(h, QEW_EINVAL, "tile_w must be one of 224, 480, 736, 992, 1248");
    if (K < 1 || 4 * K > 32 * min_kind_S(h, S))
        return fail(h, QEW_EINVAL, "K must lie in [1, tile_w / 4] for the narrowest tile in use");
    if (tiles_per_cta != 1 && tiles_per_cta != 2 && tiles_per_cta != 4 && tiles_per_cta != 8)
        return fail(h, QEW_EINVAL, "tiles_per_cta must be 1, 2, 4 or 8");
    if (max_kind_smem(h, S, tiles_per_cta) > 227 * 1024)
        return fail(h, QEW_EINVAL, "tile_w * tiles_per_cta needs more shared memory than a block has");
    h->S = S;
    h->K = K;
    h->tpc = tiles_per_cta;
    h->autotune_pending = false;
    return build_layout(h);
}

int qew_get_tuning(qew_handle h, int32_t* tile_w, int32_t* K, int32_t* tiles_per_cta)
{
    if (int rc = check_handle(h))
        return rc;
    if (tile_w) {
        int S = 7;
        for (int k = 0; k < kNumKinds; ++k)
            if (h->kinds_mask >> k & 1)
                S = std::max(S, kind_S(k, h->S));
        *tile_w = 32 * S;
    }
    if (K)
        *K = h->K;
    if (tiles_per_cta)
        *tiles_per_cta = h->tpc;
    return QEW_OK;
}

int qew_advance(qew_handle h, int64_t n_steps)
{
    if (int rc = check_handle(h))
        return rc;
    if (n_steps < 0)
        return fail(h, QEW_EINVAL, "n_steps must be >= 0");
    DeviceGuard g(h->device);
    int rc = run_to(h, h->step + n_steps, nullptr);
    if (rc == QEW_OK && n_steps > 0)
        rc = guard_range(h);
    if (rc == QEW_OK) {
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess)
            return cuda_fail(h, e, "advancing");
    }
    return rc;
}

int qew_observe(qew_handle h, const int64_t* steps, int32_t n_times, double* v_out, double* w2_out)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    return observe_impl(h, steps, n_times, v_out, nullptr, w2_out);
}

int qew_observe_ex(qew_handle h, const int64_t* steps, int32_t n_times, double* v_out, double* ubar_out,
                   double* w2_out)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    return observe_impl(h, steps, n_times, v_out, ubar_out, w2_out);
}

int qew_get_state(qew_handle h, double* u_out, int64_t* step_out)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    return get_state_impl(h, u_out, nullptr, step_out);
}

int qew_get_cells(qew_handle h, int32_t* cells_out)
{
    if (int rc = check_handle(h))
        return rc;
    if (!cells_out)
        return fail(h, QEW_EINVAL, "cells_out must not be NULL");
    DeviceGuard g(h->device);
    return get_state_impl(h, nullptr, cells_out, nullptr);
}

int qew_set_state(qew_handle h, const double* u_in)
{
    if (int rc = check_handle(h))
        return rc;
    if (!u_in)
        return fail(h, QEW_EINVAL, "u_in must not be NULL");
    DeviceGuard g(h->device);
    return set_state_impl(h, u_in);
}

int qew_structure_factor(qew_handle h, int32_t n_modes, double* S_out)
{
    if (int rc = check_handle(h))
        return rc;
    if (!S_out)
        return fail(h, QEW_EINVAL, "S_out must not be NULL");
    const int64_t L = h->L[0];
    for (int32_t c = 1; c < h->n_chains; ++c)
        if (h->L[c] != L)
            return fail(h, QEW_EINVAL, "the structure factor needs chains of one length");
    if (n_modes < 1 || n_modes > L / 2)
        return fail(h, QEW_EINVAL, "n_modes must lie in [1, L/2]");
    DeviceGuard g(h->device);
    const int32_t Li = static_cast<int32_t>(L);
    const int32_t B = h->n_chains;
    if (!h->sq_plan_made) {
        int n = Li, inembed = 2 * (Li / 2 + 1), onembed = Li / 2 + 1;
        const cufftResult r = cufftPlanMany(&h->sq_plan, 1, &n, &inembed, 1, inembed, &onembed, 1, onembed, CUFFT_D2Z, B);
        if (r != CUFFT_SUCCESS)
            return fail(h, r == CUFFT_ALLOC_FAILED ? QEW_ENOMEM : QEW_ECUDA,
                        "cuFFT plan of the structure factor failed (status " + std::to_string(static_cast<int>(r)) + ")");
        h->sq_plan_made = true;
    }
    if (cufftSetStream(h->sq_plan, h->stream) != CUFFT_SUCCESS)
        return fail(h, QEW_ECUDA, "cuFFT could not take the handle's stream");
    const size_t rows_n = static_cast<size_t>(B) * 2 * (static_cast<size_t>(Li) / 2 + 1);
    double* d_rows = nullptr;
    double* d_S = nullptr;
    int rc = QEW_OK;
    cudaError_t e = dev_alloc(&d_rows, rows_n);
    if (e == cudaSuccess)
        e = dev_alloc(&d_S, static_cast<size_t>(n_modes));
    if (e != cudaSuccess) {
        rc = cuda_fail(h, e, "allocating the structure-factor work area");
    } else {
        if (h->precision == QEW_FP32_SPLIT)
            e = sq_rows(h->d_chains, B, Li, &h->sp[h->cur], nullptr, d_rows, h->stream);
        else
            e = sq_rows(h->d_chains, B, Li, nullptr, h->u64[h->cur], d_rows, h->stream);
        if (e == cudaSuccess) {
            const cufftResult r = cufftExecD2Z(h->sq_plan, d_rows, reinterpret_cast<cufftDoubleComplex*>(d_rows));
            if (r != CUFFT_SUCCESS)
                rc = fail(h, QEW_ECUDA, "cuFFT transform failed (status " + std::to_string(static_cast<int>(r)) + ")");
        }
        if (rc == QEW_OK && e == cudaSuccess)
            e = sq_power(d_rows, Li, B, n_modes, d_S, h->stream);
        if (rc == QEW_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(S_out, d_S, static_cast<size_t>(n_modes) * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream);
        if (rc == QEW_OK && e == cudaSuccess)
            e = cudaStreamSynchronize(h->stream);
        if (rc == QEW_OK && e != cudaSuccess)
            rc = cuda_fail(h, e, "computing the structure factor");
    }
    dev_free(d_rows);
    dev_free(d_S);
    return rc;
}

int qew_reset(qew_handle h)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    return init_state(h, nullptr, std::vector<double>(h->n_chains, 0.0));
}

int qew_num_sites(qew_handle h, int64_t* n_sites)
{
    if (int rc = check_handle(h))
        return rc;
    if (!n_sites)
        return fail(h, QEW_EINVAL, "n_sites must not be NULL");
    *n_sites = h->n_sites;
    return QEW_OK;
}

int qew_disorder_values(int32_t kind, int32_t precision, uint64_t seed, uint32_t s, const int64_t* i,
                        const int64_t* n, int64_t count, double* out)
{
    if (kind < QEW_RF_GAUSS_LINEAR || kind > QEW_RB_GAUSS_CATMULLROM || kind == QEW_NONE)
        return fail(nullptr, QEW_EINVAL, "kind must name a disorder (not QEW_NONE)");
    if (precision != QEW_FP32_SPLIT && precision != QEW_FP64)
        return fail(nullptr, QEW_EINVAL, "unknown precision");
    if (count < 0 || (count > 0 && (!i || !n || !out)))
        return fail(nullptr, QEW_EINVAL, "bad count or NULL array");
    if (count == 0)
        return QEW_OK;
    int64_t *di = nullptr, *dn = nullptr;
    double* dout = nullptr;
    cudaError_t e = dev_alloc(&di, count);
    if (e == cudaSuccess)
        e = dev_alloc(&dn, count);
    if (e == cudaSuccess)
        e = dev_alloc(&dout, count);
    if (e == cudaSuccess)
        e = cudaMemcpy(di, i, count * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dn, n, count * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = disorder_values(kind, precision == QEW_FP64, seed, s, di, dn, count, dout, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, count * sizeof(double), cudaMemcpyDeviceToHost);
    dev_free(di);
    dev_free(dn);
    dev_free(dout);
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "qew_disorder_values");
    return QEW_OK;
}

int qew_philox_words(const uint32_t* ctr, const uint32_t* key, int64_t n_blocks, uint32_t* out)
{
    if (n_blocks < 0 || (n_blocks > 0 && (!ctr || !key || !out)))
        return fail(nullptr, QEW_EINVAL, "bad count or NULL array");
    if (n_blocks == 0)
        return QEW_OK;
    uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr;
    cudaError_t e = dev_alloc(&dc, 4 * n_blocks);
    if (e == cudaSuccess)
        e = dev_alloc(&dk, 2 * n_blocks);
    if (e == cudaSuccess)
        e = dev_alloc(&dout, 4 * n_blocks);
    if (e == cudaSuccess)
        e = cudaMemcpy(dc, ctr, 16 * n_blocks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(dk, key, 8 * n_blocks, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = philox_words(dc, dk, n_blocks, dout, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, dout, 16 * n_blocks, cudaMemcpyDeviceToHost);
    dev_free(dc);
    dev_free(dk);
    dev_free(dout);
    if (e != cudaSuccess)
        return cuda_fail(nullptr, e, "qew_philox_words");
    return QEW_OK;
}

int qew_enable_stats(qew_handle h, int32_t enable)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    QEW_CUDA(h, cudaStreamSynchronize(h->stream), "synchronising before enabling stats");
    if (enable && !h->d_crossings)
        QEW_CUDA(h, dev_alloc(&h->d_crossings, 1), "allocating the crossing counter");
    if (h->d_crossings)
        QEW_CUDA(h, cudaMemset(h->d_crossings, 0, sizeof(unsigned long long)), "clearing the crossing counter");
    h->stats_on = enable != 0;
    h->n_launches = h->n_fused = h->n_site_updates = 0;
    h->ev_used = 0;
    return QEW_OK;
}

int qew_get_stats(qew_handle h, int64_t* launches, int64_t* fused_launches, double* fused_ms, int64_t* site_updates,
                  int64_t* crossings)
{
    if (int rc = check_handle(h))
        return rc;
    DeviceGuard g(h->device);
    QEW_CUDA(h, cudaStreamSynchronize(h->stream), "synchronising for stats");
    double ms = 0.0;
    for (size_t k = 0; k + 1 < h->ev_used; k += 2) {
        float t = 0.0f;
        QEW_CUDA(h, cudaEventElapsedTime(&t, h->ev_pool[k], h->ev_pool[k + 1]), "reading a timing event");
        ms += t;
    }
    unsigned long long cr = 0;
    if (h->stats_on && h->d_crossings) {
        QEW_CUDA(h, cudaMemcpy(&cr, h->d_crossings, sizeof(cr), cudaMemcpyDeviceToHost), "reading crossings");
        QEW_CUDA(h, cudaMemset(h->d_crossings, 0, sizeof(cr)), "clearing the crossing counter");
    }
    if (launches)
        *launches = h->n_launches;
    if (fused_launches)
        *fused_launches = h->n_fused;
    if (fused_ms)
        *fused_ms = ms;
    if (site_updates)
        *site_updates = h->n_site_updates;
    if (crossings)
        *crossings = static_cast<int64_t>(cr);
    h->n_launches = h->n_fused = h->n_site_updates = 0;
    h->ev_used = 0;
    return QEW_OK;
}

int qew_selftest_bounded_wait(qew_handle h, int32_t spin_limit)
{
    if (int rc = check_handle(h))
        return rc;
    if (spin_limit < 1 || spin_limit > (1 << 22))
        return fail(h, QEW_EINVAL, "spin_limit must lie in [1, 2^22]");
    DeviceGuard g(h->device);
    QEW_CUDA(h, bounded_wait_selftest(h->d_error, spin_limit, h->stream), "launching the bounded-wait probe");
    QEW_CUDA(h, cudaStreamSynchronize(h->stream), "running the bounded-wait probe");
    return check_device_error(h);
}

const char* qew_last_error(qew_handle h)
{
    return h ? h->err.c_str() : g_last_error.c_str();
}

void qew_destroy(qew_handle h)
{
    if (!h)
        return;
    {
        DeviceGuard g(h->device);
        cudaStreamSynchronize(h->stream);
        free_all(h);
    }
    delete h;
}

}  // extern "C"
