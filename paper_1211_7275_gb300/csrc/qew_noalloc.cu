// qew_noalloc.cu -- observables of a caller-owned FP32-split state with no device allocation.
//
// This is a variant of the observation path of the fused kernel (per-tile partial sums followed
// by a fixed-order per-chain reduction).  Its scratch memory -- the per-tile partial sums and
// the per-chain totals -- lives in one file-scope __device__ array of fixed size instead of
// memory the library allocates, so that callers who cannot let a library call cudaMalloc can
// still use it.  Host code never hands the array's name to a kernel: in host code that name is
// only a host-side stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "qew.h"
#include "qew_internal.h"

namespace {

constexpr int kNaTile = 256;             // sites per warp tile
constexpr int kNaWarps = 4;              // warp tiles per block
constexpr int kNaMaxTiles = 1 << 16;     // -> at most 2^24 sites per call
constexpr int kNaMaxChains = 4096;
constexpr size_t kNaDoubles = static_cast<size_t>(kNaMaxTiles) * 3 + static_cast<size_t>(kNaMaxChains) * 4;

// [kNaMaxTiles][3] per-tile sums (F, y, y^2), then [kNaMaxChains][4] per-chain totals
// (sum F, S1, S2, reference cell).  Every call overwrites what it reads, so nothing has to
// start at zero; the contents of the last call remain until the next one.
static __device__ __align__(256) double g_noalloc_scratch[kNaDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_na_mu;
double* g_na_ptr[kMaxDevices] = {};

int na_fail(int code, const std::string& msg)
{
    qew::set_last_error(msg);   // readable through qew_last_error(NULL)
    return code;
}

// Device address of the scratch array on the current device (looked up on first use).
int na_scratch(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return na_fail(QEW_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return na_fail(QEW_EINVAL, "device ordinal outside the supported range");
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
        double* p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_scratch);
        if (e != cudaSuccess)
            return na_fail(QEW_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return QEW_OK;
}

// One warp per tile of 256 sites of chain c = tile / tiles_per_chain.  Per site: the pinning
// force at the state (values regenerated exactly as the fused kernel caches them), y = u minus
// the tile's reference cell; FP32 sums, warp reduction, FP64 shift to the chain's reference cell
// (its site 0) in lane 0.
__global__ void __launch_bounds__(kNaWarps * 32) na_tile_sums(const int32_t* __restrict__ cell,
                                                              const float* __restrict__ off, int32_t L,
                                                              int32_t tiles_per_chain, int32_t n_tiles, float f,
                                                              int kind, uint64_t seed, double* scratch)
{
    const int lane = threadIdx.x & 31;
    const int tile = blockIdx.x * kNaWarps + (threadIdx.x >> 5);
    if (tile >= n_tiles)
        return;
    const int32_t c = tile / tiles_per_chain;
    const int32_t start = (tile % tiles_per_chain) * kNaTile;
    const int64_t base = static_cast<int64_t>(c) * L;
    const int32_t c_ref = __ldg(cell + base);
    const int32_t nref = __ldg(cell + base + start);
    float sF = 0.0f, sy = 0.0f, syy = 0.0f;
    int cnt = 0;
    for (int x = lane; x < kNaTile; x += 32) {
        const int32_t i = start + x;
        if (i >= L)
            break;
        const int32_t n = __ldg(cell + base + i);
        const float d = __ldg(off + base + i);
        float g = f;
        if (kind == qew::kRF) {
            const float q0 = qew::rf_plus_f32(seed, static_cast<uint32_t>(c), i, n, f);
            const float q1 = qew::rf_plus_f32(seed, static_cast<uint32_t>(c), i, n + 1, f);
            g = fmaf(d, q1 - q0, q0);
        } else if (kind == qew::kRBGLinear) {
            g = (qew::rbg_f32(seed, c, i, n) - qew::rbg_f32(seed, c, i, n + 1)) + f;
        } else if (kind == qew::kRB) {
            float A, B, C;
            qew::rb_coefficients(qew::rb_f32(seed, c, i, n - 1), qew::rb_f32(seed, c, i, n),
                                 qew::rb_f32(seed, c, i, n + 1), qew::rb_f32(seed, c, i, n + 2), f, A, B, C);
            g = fmaf(d, fmaf(d, C, B), A);
        } else if (kind == qew::kRBGCubic) {
            float A, B, C;
            qew::rb_coefficients(qew::rbg_f32(seed, c, i, n - 1), qew::rbg_f32(seed, c, i, n),
                                 qew::rbg_f32(seed, c, i, n + 1), qew::rbg_f32(seed, c, i, n + 2), f, A, B, C);
            g = fmaf(d, fmaf(d, C, B), A);
        }
        sF += g - f;
        const float y = static_cast<float>(n - nref) + d;   // the cell difference is exact below 2^24
        sy += y;
        syy = fmaf(y, y, syy);
        ++cnt;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sF += __shfl_down_sync(0xffffffffu, sF, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        syy += __shfl_down_sync(0xffffffffu, syy, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        const double rel = static_cast<double>(nref) - static_cast<double>(c_ref);
        const double dsy = sy;
        double* dst = scratch + static_cast<size_t>(tile) * 3;
        dst[0] = sF;
        dst[1] = dsy + cnt * rel;
        dst[2] = static_cast<double>(syy) + rel * (2.0 * dsy + cnt * rel);
    }
}

// One block per chain: fixed-order sum of its tiles' partials -> totals[c] = (sum F, S1, S2, c_ref).
__global__ void __launch_bounds__(256) na_chain_sums(const int32_t* __restrict__ cell, int32_t L,
                                                     int32_t tiles_per_chain, double* scratch)
{
    __shared__ double red[3][256];
    const int32_t c = blockIdx.x;
    const double* part = scratch + static_cast<size_t>(c) * tiles_per_chain * 3;
    double a = 0.0, b = 0.0, q = 0.0;
    for (int t = threadIdx.x; t < tiles_per_chain; t += blockDim.x) {
        a += part[3 * t];
        b += part[3 * t + 1];
        q += part[3 * t + 2];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    red[2][threadIdx.x] = q;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (static_cast<int>(threadIdx.x) < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
            red[2][threadIdx.x] += red[2][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* tot = scratch + static_cast<size_t>(kNaMaxTiles) * 3 + static_cast<size_t>(c) * 4;
        tot[0] = red[0][0];
        tot[1] = red[1][0];
        tot[2] = red[2][0];
        tot[3] = static_cast<double>(cell[static_cast<int64_t>(c) * L]);
    }
}

}  // namespace

extern "C" int qew_observe_state_noalloc(const int32_t* cell, const float* off, int64_t L, int32_t batch,
                                         double f, int32_t disorder_kind, uint64_t seed, void* stream,
                                         double* v_out, double* ubar_out, double* w2_out)
{
    if (!cell || !off)
        return na_fail(QEW_EINVAL, "cell and off must be device pointers, not NULL");
    if (L < 1 || L >= (int64_t(1) << 31) || batch < 1)
        return na_fail(QEW_EINVAL, "need 1 <= L < 2^31 and batch >= 1");
    if (disorder_kind < QEW_RF_GAUSS_LINEAR || disorder_kind > QEW_RB_GAUSS_CATMULLROM)
        return na_fail(QEW_EINVAL, "unknown disorder kind");
    const int64_t tiles_per_chain = (L + kNaTile - 1) / kNaTile;
    if (batch > kNaMaxChains || tiles_per_chain * batch > kNaMaxTiles)
        return na_fail(QEW_EINVAL, "state too large for the fixed scratch: at most " + std::to_string(kNaMaxChains) +
                                       " chains and " + std::to_string(static_cast<long long>(kNaMaxTiles) * kNaTile) +
                                       " sites (whole 256-site tiles per chain)");
    double* scratch = nullptr;
    if (int rc = na_scratch(&scratch))
        return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int32_t n_tiles = static_cast<int32_t>(tiles_per_chain * batch);
    na_tile_sums<<<(n_tiles + kNaWarps - 1) / kNaWarps, kNaWarps * 32, 0, st>>>(
        cell, off, static_cast<int32_t>(L), static_cast<int32_t>(tiles_per_chain), n_tiles, static_cast<float>(f),
        disorder_kind, seed, scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        na_chain_sums<<<batch, 256, 0, st>>>(cell, static_cast<int32_t>(L), static_cast<int32_t>(tiles_per_chain),
                                             scratch);
        e = cudaGetLastError();
    }
    double tot[4 * 64];
    for (int32_t c0 = 0; e == cudaSuccess && c0 < batch; c0 += 64) {
        const int32_t nb = batch - c0 < 64 ? batch - c0 : 64;
        e = cudaMemcpyAsync(tot, scratch + static_cast<size_t>(kNaMaxTiles) * 3 + static_cast<size_t>(c0) * 4,
                            sizeof(double) * 4 * nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        for (int32_t k = 0; e == cudaSuccess && k < nb; ++k) {
            const double* o = tot + 4 * k;
            const double Ld = static_cast<double>(L);
            const double m1 = o[1] / Ld;
            if (v_out)
                v_out[c0 + k] = f + o[0] / Ld;
            if (ubar_out)
                ubar_out[c0 + k] = o[3] + m1;
            if (w2_out)
                w2_out[c0 + k] = o[2] / Ld - m1 * m1;
        }
    }
    if (e != cudaSuccess)
        return na_fail(QEW_ECUDA, std::string("qew_observe_state_noalloc: ") + cudaGetErrorString(e));
    return QEW_OK;
}
