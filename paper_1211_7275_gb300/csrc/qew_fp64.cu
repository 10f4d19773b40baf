// qew_fp64.cu -- the plain FP64 path of the qEW relaxation: one Euler step per launch, one
// thread per site, FP64 state in HBM (ping-pong), and each site's disorder values cached in
// HBM for the cell they were drawn for (regenerated when the site changes cell).
//
// Method: Eq. 1 of arXiv:1211.7275 with eta = c = 1, periodic in x, explicit Euler with all
// forces from the old state (Sec. III.B); pinning force by linear interpolation of R (RF), as
// minus the derivative of the Catmull-Rom spline through V or G (cubic random bond, Cases 1-2),
// or as G(n) - G(n+1) (linear-spline random bond, Case 3) (Sec. III.B, Sec. IV.C); observables
// of Eqs. 3-5.  Every FP64 operation is an explicit round-to-nearest intrinsic so that no
// multiply-add is contracted: the rounding sequence is the textbook one, operation by operation,
// (1 - d) R(n) + d R(n+1) for the force and u + dt ((lap + f) + F) for the update, with
// lap = (u_{i+1} + u_{i-1}) - 2 u_i.
#include "qew_internal.h"

namespace qew {
namespace {

// One disorder node in FP64: R (RF), V (uniform random bond) or G (Gaussian random bond).
// (n is the cell-relative node index; `period` > 0 makes the disorder periodic in u)
template <int KIND>
__device__ __forceinline__ double node_f64(uint64_t seed, uint32_t s, int32_t i, int32_t n, int32_t period)
{
    n = wrap_node(n, period);
    if constexpr (KIND == kRF)
        return rf_f64(seed, s, i, n);
    else if constexpr (KIND == kRB)
        return rb_f64(seed, s, i, n);
    else
        return rbg_f64(seed, s, i, n);
}

template <int KIND>
__device__ __forceinline__ double pinning_f64(double u, int64_t p, int32_t i, uint32_t s, uint64_t seed,
                                              const F64State& st, int32_t period)
{
    if constexpr (KIND == kNone) {
        return 0.0;
    } else {
        const double fl = floor(u);
        const int32_t n = static_cast<int32_t>(fl);
        const double d = __dsub_rn(u, fl);
        const int32_t nc = st.ncache[p];
        if constexpr (pair_kind(KIND)) {
            double r0, r1;
            if (n == nc) {
                r0 = st.c[0][p];
                r1 = st.c[1][p];
            } else {
                if (n == nc + 1) {
                    r0 = st.c[1][p];
                    r1 = node_f64<KIND>(seed, s, i, n + 1, period);
                } else if (n == nc - 1) {
                    r1 = st.c[0][p];
                    r0 = node_f64<KIND>(seed, s, i, n, period);
                } else {
                    r0 = node_f64<KIND>(seed, s, i, n, period);
                    r1 = node_f64<KIND>(seed, s, i, n + 1, period);
                }
                st.ncache[p] = n;
                st.c[0][p] = r0;
                st.c[1][p] = r1;
            }
            if constexpr (KIND == kRF)
                return __dadd_rn(__dmul_rn(__dsub_rn(1.0, d), r0), __dmul_rn(d, r1));
            else
                return __dsub_rn(r0, r1);   // minus the slope of the linear spline through G
        } else {
            double p0, p1, p2, p3;
            if (n == nc) {
                p0 = st.c[0][p];
                p1 = st.c[1][p];
                p2 = st.c[2][p];
                p3 = st.c[3][p];
            } else {
                if (n == nc + 1) {
                    p0 = st.c[1][p];
                    p1 = st.c[2][p];
                    p2 = st.c[3][p];
                    p3 = node_f64<KIND>(seed, s, i, n + 2, period);
                } else if (n == nc - 1) {
                    p1 = st.c[0][p];
                    p2 = st.c[1][p];
                    p3 = st.c[2][p];
                    p0 = node_f64<KIND>(seed, s, i, n - 1, period);
                } else {
                    p0 = node_f64<KIND>(seed, s, i, n - 1, period);
                    p1 = node_f64<KIND>(seed, s, i, n, period);
                    p2 = node_f64<KIND>(seed, s, i, n + 1, period);
                    p3 = node_f64<KIND>(seed, s, i, n + 2, period);
                }
                st.ncache[p] = n;
                st.c[0][p] = p0;
                st.c[1][p] = p1;
                st.c[2][p] = p2;
                st.c[3][p] = p3;
            }
            // -1/2 [(p2 - p0) + 2 b d + 3 c d^2], b = 2p0 - 5p1 + 4p2 - p3, c = -p0 + 3p1 - 3p2 + p3
            const double ca = __dsub_rn(p2, p0);
            const double cb = __dsub_rn(__dadd_rn(__dsub_rn(__dmul_rn(2.0, p0), __dmul_rn(5.0, p1)), __dmul_rn(4.0, p2)), p3);
            const double cc = __dadd_rn(__dsub_rn(__dsub_rn(__dmul_rn(3.0, p1), p0), __dmul_rn(3.0, p2)), p3);
            const double t1 = __dmul_rn(__dmul_rn(2.0, cb), d);
            const double t2 = __dmul_rn(__dmul_rn(__dmul_rn(3.0, cc), d), d);
            return __dmul_rn(-0.5, __dadd_rn(__dadd_rn(ca, t1), t2));
        }
    }
}

template <int KIND>
__device__ __forceinline__ void f64_step_body(const F64Launch& a)
{
    const TileDesc td = a.tiles[blockIdx.x];
    const ChainDesc ch = a.chains[td.chain];
    const int32_t L = ch.L;
    for (int x = threadIdx.x; x < a.w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= L)
            break;
        const int64_t p = ch.offset + i;
        const double u = a.u_in[p];
        const double ul = a.u_in[ch.offset + (i == 0 ? L - 1 : i - 1)];
        const double ur = a.u_in[ch.offset + (i + 1 == L ? 0 : i + 1)];
        const double F = pinning_f64<KIND>(u, p, i, ch.s, a.seed, a.st, ch.period);
        const double lap = __dsub_rn(__dadd_rn(ur, ul), __dmul_rn(2.0, u));
        a.u_out[p] = __dadd_rn(u, __dmul_rn(a.dt, __dadd_rn(__dadd_rn(lap, ch.f64), F)));
    }
}

// Per block tile: sum F, sum (u - c), sum (u - c)^2 of the current state u_in, c the chain's
// reference shift.
template <int KIND>
__device__ __forceinline__ void f64_observe_body(const F64Launch& a, double (*red)[256 / 32])
{
    const TileDesc td = a.tiles[blockIdx.x];
    const ChainDesc ch = a.chains[td.chain];
    const double c = a.shift[td.chain];
    double tF = 0.0, t1 = 0.0, t2 = 0.0;
    for (int x = threadIdx.x; x < a.w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= ch.L)
            break;
        const int64_t p = ch.offset + i;
        const double u = a.u_in[p];
        tF = __dadd_rn(tF, pinning_f64<KIND>(u, p, i, ch.s, a.seed, a.st, ch.period));
        const double y = __dsub_rn(u, c);
        t1 = __dadd_rn(t1, y);
        t2 = __dadd_rn(t2, __dmul_rn(y, y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tF += __shfl_down_sync(0xffffffffu, tF, o);
        t1 += __shfl_down_sync(0xffffffffu, t1, o);
        t2 += __shfl_down_sync(0xffffffffu, t2, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][warp] = tF;
        red[1][warp] = t1;
        red[2][warp] = t2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sF = 0.0, s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) {
            sF += red[0][w];
            s1 += red[1][w];
            s2 += red[2][w];
        }
        double* dst = a.partial + static_cast<size_t>(blockIdx.x) * 3;
        dst[0] = sF;
        dst[1] = s1;
        dst[2] = s2;
    }
}

__global__ void f64_init_kernel(const ChainDesc* chains, const TileDesc* tiles, int32_t w_tile, F64State st,
                                uint64_t seed, const double* u_in)
{
    const TileDesc td = tiles[blockIdx.x];
    const ChainDesc ch = chains[td.chain];
    for (int x = threadIdx.x; x < w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= ch.L)
            break;
        const int64_t p = ch.offset + i;
        const double u = u_in ? u_in[p] : 0.0;
        st.u[p] = u;
        const int32_t n = static_cast<int32_t>(floor(u));
        st.ncache[p] = n;
        const int32_t M = ch.period;
        if (ch.kind == kRF) {
            st.c[0][p] = rf_f64(seed, ch.s, i, wrap_node(n, M));
            st.c[1][p] = rf_f64(seed, ch.s, i, wrap_node(n + 1, M));
        } else if (ch.kind == kRBGLinear) {
            st.c[0][p] = rbg_f64(seed, ch.s, i, wrap_node(n, M));
            st.c[1][p] = rbg_f64(seed, ch.s, i, wrap_node(n + 1, M));
        } else if (ch.kind == kRB) {
            for (int c = 0; c < 4; ++c)
                st.c[c][p] = rb_f64(seed, ch.s, i, wrap_node(n - 1 + c, M));
        } else if (ch.kind == kRBGCubic) {
            for (int c = 0; c < 4; ++c)
                st.c[c][p] = rbg_f64(seed, ch.s, i, wrap_node(n - 1 + c, M));
        }
    }
}

__global__ void f64_cells_kernel(const ChainDesc* chains, const TileDesc* tiles, int32_t w_tile, const double* u,
                                 int32_t* cells_out)
{
    const TileDesc td = tiles[blockIdx.x];
    const ChainDesc ch = chains[td.chain];
    for (int x = threadIdx.x; x < w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= ch.L)
            break;
        const int64_t p = ch.offset + i;
        cells_out[p] = static_cast<int32_t>(floor(u[p]));
    }
}

// Block tiles of mixed kinds share one launch: the kind is uniform per block (one chain).
__global__ void __launch_bounds__(256) f64_step_any(F64Launch a)
{
    const int kind = a.chains[a.tiles[blockIdx.x].chain].kind;
    if (kind == kRF)
        f64_step_body<kRF>(a);
    else if (kind == kRB)
        f64_step_body<kRB>(a);
    else if (kind == kRBGLinear)
        f64_step_body<kRBGLinear>(a);
    else if (kind == kRBGCubic)
        f64_step_body<kRBGCubic>(a);
    else
        f64_step_body<kNone>(a);
}

__global__ void __launch_bounds__(256) f64_observe_any(F64Launch a)
{
    __shared__ double red[3][256 / 32];
    const int kind = a.chains[a.tiles[blockIdx.x].chain].kind;
    if (kind == kRF)
        f64_observe_body<kRF>(a, red);
    else if (kind == kRB)
        f64_observe_body<kRB>(a, red);
    else if (kind == kRBGLinear)
        f64_observe_body<kRBGLinear>(a, red);
    else if (kind == kRBGCubic)
        f64_observe_body<kRBGCubic>(a, red);
    else
        f64_observe_body<kNone>(a, red);
}

}  // namespace

cudaError_t f64_step(const F64Launch& a, cudaStream_t st)
{
    if (a.n_tiles == 0)
        return cudaSuccess;
    f64_step_any<<<a.n_tiles, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t f64_observe(const F64Launch& a, cudaStream_t st)
{
    if (a.n_tiles == 0)
        return cudaSuccess;
    f64_observe_any<<<a.n_tiles, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t f64_init(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile, F64State st,
                     uint64_t seed, int, const double* u_in, cudaStream_t stream)
{
    if (n_tiles == 0)
        return cudaSuccess;
    f64_init_kernel<<<n_tiles, 256, 0, stream>>>(chains, tiles, w_tile, st, seed, u_in);
    return cudaGetLastError();
}

cudaError_t f64_cells(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                      const double* u, int32_t* cells_out, cudaStream_t stream)
{
    if (n_tiles == 0)
        return cudaSuccess;
    f64_cells_kernel<<<n_tiles, 256, 0, stream>>>(chains, tiles, w_tile, u, cells_out);
    return cudaGetLastError();
}

}  // namespace qew
