// qew_peaks.cu -- measured rates of the lane arithmetic that bounds the relaxation kernels.
//
// The fused FP32-split kernel is bound by instruction issue, not by memory, so its roofline is a
// lane-operation rate: SMs x 128 lanes x SM clock, one FP32 FMA per lane and cycle.  These
// microbenchmarks measure that rate and two others on the device:
//   - FP32 FMA: independent fmaf chains, the unit of the lane-operation roofline;
//   - FP64 FMA: the same for double, the arithmetic of the plain FP64 comparison path;
//   - Philox4x32-10 blocks with a precomputed key schedule, the generator that redraws the
//     disorder at every cell crossing (Sec. III.B, memory-free disorder of Sec. IV.D).
// Each runs on a grid that fills every SM at its occupancy limit, once untimed and then three
// times between CUDA events (best of three).  One thread also reads the SM cycle counter against
// the global nanosecond timer across the FP32 run, which gives the SM clock it ran at.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "qew.h"
#include "qew_internal.h"

namespace {

using qew::PhiloxKeys;

constexpr int kThreads = 256;
constexpr int kChains = 8;     // independent dependency chains per thread
constexpr int kUnroll = 16;    // FMAs per chain per loop trip
constexpr int kBlocksPhilox = 4;   // independent Philox counters per thread

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float fma_t(float x, float a, float b) { return fmaf(x, a, b); }
__device__ __forceinline__ double fma_t(double x, double a, double b) { return ::fma(x, a, b); }

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_rate_kernel(T* out, int iters, T a, T b, unsigned long long* clk)
{
    const bool timer = clk && blockIdx.x == 0 && threadIdx.x == 0;
    unsigned long long c0 = 0, t0 = 0;
    if (timer) {
        t0 = global_ns();
        c0 = clock64();
    }
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = static_cast<T>(threadIdx.x + c) * static_cast<T>(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c)
                x[c] = fma_t(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    out[static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x] = s;
    if (timer) {
        const unsigned long long c1 = clock64();
        const unsigned long long t1 = global_ns();
        clk[0] = c1 - c0;
        clk[1] = t1 - t0;
    }
}

__global__ void __launch_bounds__(kThreads) philox_rate_kernel(uint32_t* out, int iters, PhiloxKeys ks)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint4 c[kBlocksPhilox];
#pragma unroll
    for (int j = 0; j < kBlocksPhilox; ++j)
        c[j] = make_uint4(t, static_cast<uint32_t>(j), 0u, 0u);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < kBlocksPhilox; ++j)
            c[j] = qew::philox4x32_10_ks(c[j], ks);
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < kBlocksPhilox; ++j)
        r ^= c[j].x ^ c[j].y ^ c[j].z ^ c[j].w;
    out[t] = r;
}

int peaks_fail(int code, const std::string& msg)
{
    qew::set_last_error(msg);
    return code;
}

// Best of three event-timed launches (after one untimed) of `launch`, in seconds.
template <typename F>
cudaError_t best_of_three(F launch, double* seconds)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
        e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess)
            e = launch();
        if (e == cudaSuccess)
            e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rep > 0)
            best = std::min(best, ms);
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    *seconds = 1e-3 * best;
    return e;
}

template <typename T>
cudaError_t fma_rate(int sms, int iters, double* ops_per_s, double* sm_mhz)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel<T>, kThreads, 0);
    if (e != cudaSuccess)
        return e;
    const int blocks = sms * std::max(per_sm, 1);
    T* out = nullptr;
    unsigned long long* clk = nullptr;
    e = cudaMalloc(&out, sizeof(T) * static_cast<size_t>(blocks) * kThreads);
    if (e == cudaSuccess)
        e = cudaMalloc(&clk, 2 * sizeof(unsigned long long));
    double s = 0.0;
    if (e == cudaSuccess)
        e = best_of_three([&] {
                fma_rate_kernel<T><<<blocks, kThreads>>>(out, iters, static_cast<T>(0.999999), static_cast<T>(1e-7),
                                                         clk);
                return cudaGetLastError();
            }, &s);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess)
        e = cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(clk);
    if (e != cudaSuccess)
        return e;
    *ops_per_s = static_cast<double>(blocks) * kThreads * iters * kUnroll * kChains / s;
    if (sm_mhz)
        *sm_mhz = h[1] ? 1e3 * static_cast<double>(h[0]) / static_cast<double>(h[1]) : 0.0;
    return cudaSuccess;
}

cudaError_t philox_rate(int sms, int iters, double* blocks_per_s)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, philox_rate_kernel, kThreads, 0);
    if (e != cudaSuccess)
        return e;
    const int blocks = sms * std::max(per_sm, 1);
    uint32_t* out = nullptr;
    e = cudaMalloc(&out, sizeof(uint32_t) * static_cast<size_t>(blocks) * kThreads);
    const PhiloxKeys ks = qew::philox_key_schedule(0x2d7f5a3c9b1e4f60ull);
    double s = 0.0;
    if (e == cudaSuccess)
        e = best_of_three([&] {
                philox_rate_kernel<<<blocks, kThreads>>>(out, iters, ks);
                return cudaGetLastError();
            }, &s);
    cudaFree(out);
    if (e != cudaSuccess)
        return e;
    *blocks_per_s = static_cast<double>(blocks) * kThreads * iters * kBlocksPhilox / s;
    return cudaSuccess;
}

}  // namespace

extern "C" int qew_measure_alu_peaks(double* out, int32_t n_out)
{
    if (!out || n_out < 4)
        return peaks_fail(QEW_EINVAL, "qew_measure_alu_peaks: out must hold 4 values");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double f32 = 0.0, f64 = 0.0, philox = 0.0, mhz = 0.0;
    // loop trips sized for launches of a few to a few tens of milliseconds on a full GPU
    if (e == cudaSuccess)
        e = fma_rate<float>(sms, 4096, &f32, &mhz);
    if (e == cudaSuccess)
        e = fma_rate<double>(sms, 128, &f64, nullptr);
    if (e == cudaSuccess)
        e = philox_rate(sms, 1024, &philox);
    if (e != cudaSuccess)
        return peaks_fail(QEW_ECUDA, std::string("qew_measure_alu_peaks: ") + cudaGetErrorString(e));
    out[0] = f32;
    out[1] = f64;
    out[2] = philox;
    out[3] = mhz;
    return QEW_OK;
}
