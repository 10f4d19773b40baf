// qew_reduce.cu -- second pass of the checkpoint reductions, the range guard of the FP32-split
// state at observations, and the generator diagnostics.
//
// Observables (arXiv:1211.7275, Sec. II, Eqs. 3-5) per chain, from the per-tile partial sums
// written by the step kernels: sum F_p, S1 = sum (u - c) and S2 = sum (u - c)^2, c the chain's
// reference shift.  The host forms v = f + sum F_p / L, ubar = c + S1 / L and
// w2 = S2 / L - (S1 / L)^2.  The shift follows the centre of mass from one observation to the
// next, so S1 / L stays of the order of the displacement between observations and the
// one-pass variance keeps its precision.  One block per chain sums its partials in a fixed
// order, so results are bitwise reproducible from run to run.
#include <algorithm>

#include "qew_internal.h"
#include "qew_tma.cuh"

namespace qew {
namespace {

__global__ void __launch_bounds__(256) reduce_chains_kernel(const ChainDesc* chains, const double* partial,
                                                            double* shift, double* obs, int integer_shift)
{
    __shared__ double red[3][256];
    const ChainDesc ch = chains[blockIdx.x];
    double a = 0.0, b = 0.0, c = 0.0;
    for (int t = threadIdx.x; t < ch.ntiles; t += blockDim.x) {
        const double* q = partial + static_cast<size_t>(ch.tile0 + t) * 3;
        a += q[0];
        b += q[1];
        c += q[2];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    red[2][threadIdx.x] = c;
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
        const double c_used = shift[blockIdx.x];
        double* o = obs + static_cast<size_t>(blockIdx.x) * 4;
        o[0] = red[0][0];
        o[1] = red[1][0];
        o[2] = red[2][0];
        o[3] = c_used;
        const double mean_rel = red[1][0] / static_cast<double>(ch.L);
        double next = c_used + (integer_shift ? floor(mean_rel + 0.5) : mean_rel);
        if (!isfinite(next) || fabs(next) > 1.0e9)
            next = c_used;  // keep a usable reference if the state went non-finite
        shift[blockIdx.x] = next;
    }
}

__global__ void philox_words_kernel(const uint4* ctr, const uint2* key, int64_t n, uint4* out)
{
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x)
        out[k] = philox4x32_10(ctr[k], key[k].x, key[k].y);
}

__global__ void disorder_values_kernel(int kind, int fp64, uint64_t seed, uint32_t s, const int64_t* i,
                                       const int64_t* n, int64_t count, double* out)
{
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < count;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t ii = static_cast<int32_t>(i[k]);
        const int32_t nn = static_cast<int32_t>(n[k]);
        double v;
        if (kind == kRF)
            v = fp64 ? rf_f64(seed, s, ii, nn) : static_cast<double>(rf_f32(seed, s, ii, nn));
        else if (kind == kRB)
            v = fp64 ? rb_f64(seed, s, ii, nn) : static_cast<double>(rb_f32(seed, s, ii, nn));
        else
            v = fp64 ? rbg_f64(seed, s, ii, nn) : static_cast<double>(rbg_f32(seed, s, ii, nn));
        out[k] = v;
    }
}

// One warp waits on an mbarrier that nothing will ever complete: the bounded wait must give up
// and record it in `error`, exactly as the fused kernel does when a bulk copy does not land.
__global__ void bounded_wait_probe(int32_t* error, int limit)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const bool done = __all_sync(0xffffffffu, mbar_wait(&bar, 0, limit));
    if (!done && threadIdx.x == 0)
        atomicExch(error, 1);
}

// Range guard of the FP32-split state, run at every observation: the fused kernel carries cells as
// exact small floats relative to a cell of its tile window and (compact layout) decodes a step's
// move from 16 bits of the cell.  Both hold while neighbouring cells differ by less than 2^12: then
// no Euler step moves a site by 2^15 cells (the Euler map grows a neighbour difference by at most
// 2 dt max|F_p| per step) and a 992-site window spans less than 2^22 cells.  A violation sets the
// error flag to 2.  Blocks (x, y) stride over the sites of chains y, y + gridDim.y, ...; the
// chain descriptor is read once per chain, so a thread's loads are independent of one another.
__global__ void __launch_bounds__(256) split_range_guard_kernel(const ChainDesc* chains, int32_t n_chains,
                                                               const int32_t* __restrict__ cell, int32_t* error)
{
    bool bad = false;
    for (int32_t c = blockIdx.y; c < n_chains; c += gridDim.y) {
        const ChainDesc ch = chains[c];
        const int32_t* cc = cell + ch.offset;
        const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
#pragma unroll 4
        for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < ch.L; i += stride) {
            const int64_t j = (i + 1 == ch.L) ? 0 : i + 1;   // 64-bit: chains reach 2^31 - 1 sites
            const int64_t dn = static_cast<int64_t>(__ldg(cc + j)) - __ldg(cc + i);
            bad = bad || dn >= 4096 || dn <= -4096;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicExch(error, 2);
}

}  // namespace

cudaError_t split_range_guard(const ChainDesc* chains, int32_t n_chains, int64_t max_L, const int32_t* cell,
                              int32_t* error, cudaStream_t stream)
{
    if (n_chains == 0)
        return cudaSuccess;
    // about 16 sites per thread along x, at most 1024 blocks per chain
    const int64_t bx = std::min<int64_t>(std::max<int64_t>((max_L + 256 * 16 - 1) / (256 * 16), 1), 1024);
    const dim3 grid(static_cast<unsigned>(bx), static_cast<unsigned>(std::min<int32_t>(n_chains, 65535)));
    split_range_guard_kernel<<<grid, 256, 0, stream>>>(chains, n_chains, cell, error);
    return cudaGetLastError();
}

cudaError_t bounded_wait_selftest(int32_t* d_error, int spin_limit, cudaStream_t stream)
{
    bounded_wait_probe<<<1, 32, 0, stream>>>(d_error, spin_limit);
    return cudaGetLastError();
}

cudaError_t reduce_chains(const ChainDesc* chains, int32_t n_chains, const double* partial, double* shift,
                          double* obs, int integer_shift, cudaStream_t stream)
{
    if (n_chains == 0)
        return cudaSuccess;
    reduce_chains_kernel<<<n_chains, 256, 0, stream>>>(chains, partial, shift, obs, integer_shift);
    return cudaGetLastError();
}

cudaError_t philox_words(const uint32_t* ctr, const uint32_t* key, int64_t n_blocks, uint32_t* out,
                         cudaStream_t stream)
{
    if (n_blocks == 0)
        return cudaSuccess;
    const int grid = static_cast<int>(n_blocks / 256 + 1 < 4096 ? n_blocks / 256 + 1 : 4096);
    philox_words_kernel<<<grid, 256, 0, stream>>>(reinterpret_cast<const uint4*>(ctr),
                                                  reinterpret_cast<const uint2*>(key), n_blocks,
                                                  reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

cudaError_t disorder_values(int kind, int fp64, uint64_t seed, uint32_t s, const int64_t* i, const int64_t* n,
                            int64_t count, double* out, cudaStream_t stream)
{
    if (count == 0)
        return cudaSuccess;
    const int grid = static_cast<int>(count / 256 + 1 < 4096 ? count / 256 + 1 : 4096);
    disorder_values_kernel<<<grid, 256, 0, stream>>>(kind, fp64, seed, s, i, n, count, out);
    return cudaGetLastError();
}

}  // namespace qew
