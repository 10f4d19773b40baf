// qew_split.cu -- the fused FP32-split kernel of the qEW relaxation: elastic force + pinning
// force + Euler update + cell renormalisation + disorder regeneration, K Euler steps per HBM
// round trip (temporal blocking), with the checkpoint partial sums fused after the last step.
//
// Method: Eq. 1 of arXiv:1211.7275 with eta = c = 1, discretised in x with periodic boundary
// conditions and integrated by explicit Euler (Sec. III.B); pinning force interpolated from
// random values at integer (i, n) (Sec. III.B and the cases of Sec. IV.C); observables of
// Eqs. 3-5 (Sec. II).
//
// State of a site: integer cell n and FP32 offset d in [0, 1) (u = n + d), plus its disorder
// cache: RF keeps R(n) + f and R(n+1) + f, RB keeps V(n-1 .. n+2).  The drive f is folded into
// the RF cache so that F_p + f costs one subtraction and one FMA per site-step.
//
// Work decomposition: one warp owns one tile of 32 * S sites of a chain, S consecutive sites
// per lane held in registers.  A tile advanced K steps needs K extra sites on each side (the
// stencil's light cone), so the window is [start - K, start - K + 32 S) and the owned sites
// [start, start + w_own), w_own <= 32 S - 2K; the outermost sites of the window go stale one
// per step from each edge and are never stored.  Windows wrap around periodic chains (any
// number of times for chains shorter than a tile).  Halo exchange inside a step is two warp
// shuffles per neighbour; there is no shared-memory traffic and no barrier inside the K loop.
#include <cstdio>

#include "qew_internal.h"
#include "qew_tma.cuh"

namespace qew {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Offset outside [0, 1) (or NaN / -0): compare the bit pattern; every float in [0, 1) is
// below the pattern of 1.0f, negative values have the sign bit set.
__device__ __forceinline__ unsigned out_of_cell(float d)
{
    return __float_as_uint(d) >= 0x3F800000u ? 1u : 0u;
}

// Move a site whose offset left [0, 1) to its new cell: returns the cell shift k and leaves
// d in [0, 1).  A tiny negative offset can round to 1.0f after the shift; then the site stays
// in the upper cell with d = 0.
__device__ __forceinline__ int renormalise(float& d)
{
    const float fk = floorf(d);
    int k = static_cast<int>(fk);
    float r = d - fk;
    if (r >= 1.0f) {
        r = 0.0f;
        k += 1;
    }
    d = r;
    return k;
}

// Chain-local index of window position x (window start wstart).
__device__ __forceinline__ int32_t site_index(int64_t wstart, int x, bool contiguous, int32_t L)
{
    const int64_t g = wstart + x;
    return contiguous ? static_cast<int32_t>(g) : wrap_site(g, L);
}

template <int KIND>
struct CacheWidth {
    static constexpr int value = (KIND == kRB) ? 4 : 2;
};

template <int KIND, int S>
__global__ void __launch_bounds__(256) split_step_kernel(SplitLaunch a)
{
    constexpr int NC = CacheWidth<KIND>::value;
    constexpr int TW = 32 * S;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t s_bar[8];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * (blockDim.x >> 5) + warp;
    if (tile >= a.n_tiles)
        return;  // whole warp; the kernel uses no block-wide barrier

    int32_t* s_cell = reinterpret_cast<int32_t*>(smem_raw) + static_cast<size_t>(warp) * TW * (2 + NC);
    float* s_off = reinterpret_cast<float*>(s_cell + TW);
    float* s_c = s_off + TW;

    const TileDesc td = a.tiles[tile];
    const ChainDesc ch = a.chains[td.chain];
    const int32_t L = ch.L;
    const int K = a.K;
    const int owned = min(a.w_own, L - td.start);
    const int64_t wstart = static_cast<int64_t>(td.start) - K;
    const bool contiguous = (wstart >= 0) && (wstart + TW <= L);
    const float f = ch.f32;
    const float dt = a.dt;
    const uint64_t seed = a.seed;
    const uint32_t s = ch.s;

    // ---- stage the window in this warp's shared-memory slice ----
    // Contiguous, 16-byte aligned windows arrive by TMA bulk copies (one per array, completion
    // on the warp's mbarrier); windows that wrap around the chain or start unaligned use
    // coalesced read-only loads.
    const bool tma_in = contiguous && (((ch.offset + wstart) & 3) == 0);
    if (tma_in) {
        uint64_t* bar = &s_bar[warp];
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncwarp();
        if (lane == 0) {
            constexpr uint32_t bytes = TW * 4;
            const int64_t p0 = ch.offset + wstart;
            mbar_arrive_expect_tx(bar, bytes * (2 + NC));
            tma_load_1d(s_cell, a.in.cell + p0, bytes, bar);
            tma_load_1d(s_off, a.in.off + p0, bytes, bar);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                tma_load_1d(s_c + c * TW, a.in.c[c] + p0, bytes, bar);
        }
        const bool landed = __all_sync(kFull, mbar_wait(bar, 0));   // warp-uniform outcome
        if (!landed) {
            // the copy did not land: flag it, give the copies one more bounded wait, drop the tile
            if (lane == 0)
                atomicExch(a.error, 1);
            mbar_wait(bar, 0);
            return;
        }
    } else {
        const int32_t* __restrict__ g_cell = a.in.cell;
        const float* __restrict__ g_off = a.in.off;
        for (int x = lane; x < TW; x += 32) {
            const int32_t g = contiguous ? static_cast<int32_t>(wstart + x) : wrap_site(wstart + x, L);
            const int64_t p = ch.offset + g;
            s_cell[x] = __ldg(g_cell + p);
            s_off[x] = __ldg(g_off + p);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                s_c[c * TW + x] = __ldg(a.in.c[c] + p);
        }
        __syncwarp();
    }

    int n[S];
    float d[S];
    float q[NC][S];   // RF: R(n)+f, R(n+1)+f.  RB: V(n-1..n+2)
    float A[KIND == kRB ? S : 1], B[KIND == kRB ? S : 1], C[KIND == kRB ? S : 1];
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const int x = lane * S + j;
        n[j] = s_cell[x];
        d[j] = s_off[x];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            q[c][j] = s_c[c * TW + x];
        if constexpr (KIND == kRB)
            rb_coefficients(q[0][j], q[1][j], q[2][j], q[3][j], f, A[j], B[j], C[j]);
    }
    __syncwarp();   // the staging area is reused by the regeneration queue below

    // ---- K Euler steps, all in registers ----
    unsigned n_cross = 0;
    // per-warp request queue of the cooperative regeneration, in the staging area (idle here)
    int32_t* q_site = s_cell;
    int32_t* q_cell = s_cell + 32;
    float* q_val = s_off;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        const int nl = __shfl_up_sync(kFull, n[S - 1], 1);
        const float dl = __shfl_up_sync(kFull, d[S - 1], 1);
        const int nr = __shfl_down_sync(kFull, n[0], 1);
        const float drn = __shfl_down_sync(kFull, d[0], 1);
        float Dm = small_int_to_float(n[0] - nl) + (d[0] - dl);   // u_j - u_{j-1}
        unsigned cross = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int nn = (j + 1 < S) ? n[j + 1] : nr;
            const float dd = (j + 1 < S) ? d[j + 1] : drn;
            const float Dp = small_int_to_float(nn - n[j]) + (dd - d[j]);   // u_{j+1} - u_j
            float g;                                                         // F_p + f
            if constexpr (KIND == kRB)
                g = fmaf(d[j], fmaf(d[j], C[j], B[j]), A[j]);
            else
                g = fmaf(d[j], q[1][j] - q[0][j], q[0][j]);
            const float dn = fmaf(dt, (Dp - Dm) + g, d[j]);
            Dm = Dp;
            d[j] = dn;
            cross |= out_of_cell(dn) << j;
        }
        if (__any_sync(kFull, cross)) {
            // Cell changes.  A one-cell move needs one new disorder value (RF: R(n+1) after an
            // upward move, R(n) after a downward one; RB: V(n+2) / V(n-1)); the others shift
            // within the cache.  These requests are evaluated warp-cooperatively below.  A jump
            // of several cells (rare) regenerates the whole cache of that site in place.
            unsigned req = 0, up = 0;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                if (!((cross >> j) & 1u))
                    continue;
                const int kk = renormalise(d[j]);
                if (kk == 0)
                    continue;
                const int nn = n[j] + kk;
                n[j] = nn;
                ++n_cross;
                if constexpr (KIND == kNone)
                    continue;
                if (kk == 1 || kk == -1) {
                    req |= 1u << j;
                    if (kk == 1) {
                        up |= 1u << j;
#pragma unroll
                        for (int c = 0; c + 1 < NC; ++c)
                            q[c][j] = q[c + 1][j];
                    } else {
#pragma unroll
                        for (int c = NC - 1; c > 0; --c)
                            q[c][j] = q[c - 1][j];
                    }
                } else {
                    const int32_t i = site_index(wstart, lane * S + j, contiguous, L);
                    if constexpr (KIND == kRF) {
                        q[0][j] = rf_f32(seed, s, i, nn) + f;
                        q[1][j] = rf_f32(seed, s, i, nn + 1) + f;
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            q[c][j] = rb_f32(seed, s, i, nn - 1 + c);
                        rb_coefficients(q[0][j], q[1][j], q[2][j], q[3][j], f, A[j], B[j], C[j]);
                    }
                }
            }
            if constexpr (KIND != kNone) {
                // warp-wide exclusive scan of the request counts -> queue positions
                const int cnt = __popc(req);
                int incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                const int total = __shfl_sync(kFull, incl, 31);
                const int first = incl - cnt;
                for (int base = 0; base < total; base += 32) {
                    // enqueue (site, cell) of the requests with positions base .. base+31
                    int p = first - base;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        if ((req >> j) & 1u) {
                            if (static_cast<unsigned>(p) < 32u) {
                                q_site[p] = site_index(wstart, lane * S + j, contiguous, L);
                                // RF: R(n+1) after an up move, R(n) after a down move.
                                // RB: V(n+2) after an up move, V(n-1) after a down move.
                                const int off_up = (KIND == kRF) ? 1 : 2;
                                const int off_dn = (KIND == kRF) ? 0 : -1;
                                q_cell[p] = n[j] + (((up >> j) & 1u) ? off_up : off_dn);
                            }
                            ++p;
                        }
                    }
                    __syncwarp();
                    if (base + lane < total) {
                        if constexpr (KIND == kRF)
                            q_val[lane] = rf_f32(seed, s, q_site[lane], q_cell[lane]) + f;
                        else
                            q_val[lane] = rb_f32(seed, s, q_site[lane], q_cell[lane]);
                    }
                    __syncwarp();
                    p = first - base;
#pragma unroll
                    for (int j = 0; j < S; ++j) {
                        if ((req >> j) & 1u) {
                            if (static_cast<unsigned>(p) < 32u) {
                                const float v = q_val[p];
                                if ((up >> j) & 1u)
                                    q[NC - 1][j] = v;
                                else
                                    q[0][j] = v;
                            }
                            ++p;
                        }
                    }
                    __syncwarp();
                }
                if constexpr (KIND == kRB) {
#pragma unroll
                    for (int j = 0; j < S; ++j)
                        if ((req >> j) & 1u)
                            rb_coefficients(q[0][j], q[1][j], q[2][j], q[3][j], f, A[j], B[j], C[j]);
                }
            }
        }
    }

    if (a.crossings) {
        unsigned tot = __reduce_add_sync(kFull, n_cross);
        if (lane == 0 && tot)
            atomicAdd(a.crossings, static_cast<unsigned long long>(tot));
    }

    // ---- checkpoint partial sums of the state after the K steps (owned sites only) ----
    // FP32 sums relative to the warp's reference cell (lane 0's first site; the spread inside a
    // tile is small), FP32 warp reduction, then one FP64 shift to the chain reference in lane 0.
    if (a.do_obs) {
        const int32_t c_ref = static_cast<int32_t>(a.shift[td.chain]);
        const int32_t nref = __shfl_sync(kFull, n[0], 0);
        float sF = 0.0f, sy = 0.0f, syy = 0.0f;
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int o = lane * S + j - K;
            if (o >= 0 && o < owned) {
                float g;
                if constexpr (KIND == kRB)
                    g = fmaf(d[j], fmaf(d[j], C[j], B[j]), A[j]);
                else
                    g = fmaf(d[j], q[1][j] - q[0][j], q[0][j]);
                sF += g - f;
                const float y = small_int_to_float(n[j] - nref) + d[j];
                sy += y;
                syy = fmaf(y, y, syy);
                ++cnt;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            sF += __shfl_down_sync(kFull, sF, o);
            sy += __shfl_down_sync(kFull, sy, o);
            syy += __shfl_down_sync(kFull, syy, o);
            cnt += __shfl_down_sync(kFull, cnt, o);
        }
        if (lane == 0) {
            const double rel = static_cast<double>(nref) - static_cast<double>(c_ref);
            const double dsy = sy;
            double* dst = a.partial + static_cast<size_t>(a.tile_base + tile) * 3;
            dst[0] = sF;
            dst[1] = dsy + cnt * rel;
            dst[2] = static_cast<double>(syy) + rel * (2.0 * dsy + cnt * rel);
        }
    }

    if (K == 0)
        return;

    // ---- write the owned sites back: registers -> shared -> global ----
    __syncwarp();
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const int x = lane * S + j;
        s_cell[x] = n[j];
        s_off[x] = d[j];
#pragma unroll
        for (int c = 0; c < NC; ++c)
            s_c[c * TW + x] = q[c][j];
    }
    const int64_t out0 = ch.offset + td.start;
    const bool tma_out = ((K & 3) == 0) && ((out0 & 3) == 0) && ((owned & 3) == 0);
    if (tma_out) {
        fence_proxy_async_shared();   // generic-proxy writes above -> visible to the bulk copy
        __syncwarp();
        if (lane == 0) {
            const uint32_t bytes = static_cast<uint32_t>(owned) * 4;
            tma_store_1d(a.out.cell + out0, s_cell + K, bytes);
            tma_store_1d(a.out.off + out0, s_off + K, bytes);
#pragma unroll
            for (int c = 0; c < NC; ++c)
                tma_store_1d(a.out.c[c] + out0, s_c + c * TW + K, bytes);
            tma_store_commit();
            tma_store_wait_all();
        }
    } else {
        __syncwarp();
        for (int o = lane; o < owned; o += 32) {
            const int x = o + K;
            const int64_t p = out0 + o;
            a.out.cell[p] = s_cell[x];
            a.out.off[p] = s_off[x];
#pragma unroll
            for (int c = 0; c < NC; ++c)
                a.out.c[c][p] = s_c[c * TW + x];
        }
    }
}

template <int KIND, int S>
cudaError_t launch_split(int tiles_per_cta, const SplitLaunch& a, cudaStream_t st)
{
    constexpr int NC = CacheWidth<KIND>::value;
    const size_t smem = static_cast<size_t>(tiles_per_cta) * 32 * S * 4 * (2 + NC);
    auto kern = split_step_kernel<KIND, S>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess)
        return e;
    const int grid = (a.n_tiles + tiles_per_cta - 1) / tiles_per_cta;
    if (grid == 0)
        return cudaSuccess;
    kern<<<grid, 32 * tiles_per_cta, smem, st>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Initialisation (flat start or a given FP64 state) and conversion back to FP64.
// Block tiles of w_tile sites, one thread per site.
// ---------------------------------------------------------------------------------------
__global__ void split_init_kernel(const ChainDesc* chains, const TileDesc* tiles, int32_t w_tile, SplitState st,
                                  uint64_t seed, const double* u_in)
{
    const TileDesc td = tiles[blockIdx.x];
    const ChainDesc ch = chains[td.chain];
    for (int x = threadIdx.x; x < w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= ch.L)
            break;
        const int64_t p = ch.offset + i;
        int32_t n = 0;
        float d = 0.0f;
        if (u_in) {
            const double u = u_in[p];
            const double fl = floor(u);
            n = static_cast<int32_t>(fl);
            d = static_cast<float>(u - fl);
            if (d >= 1.0f) {
                d = 0.0f;
                n += 1;
            }
        }
        st.cell[p] = n;
        st.off[p] = d;
        if (ch.kind == kRF) {
            st.c[0][p] = rf_f32(seed, ch.s, i, n) + ch.f32;
            st.c[1][p] = rf_f32(seed, ch.s, i, n + 1) + ch.f32;
        } else if (ch.kind == kRB) {
            for (int c = 0; c < 4; ++c)
                st.c[c][p] = rb_f32(seed, ch.s, i, n - 1 + c);
        } else {
            st.c[0][p] = ch.f32;
            st.c[1][p] = ch.f32;
        }
    }
}

__global__ void split_to_f64_kernel(const ChainDesc* chains, const TileDesc* tiles, int32_t w_tile, SplitState st,
                                    double* u_out, int32_t* cells_out)
{
    const TileDesc td = tiles[blockIdx.x];
    const ChainDesc ch = chains[td.chain];
    for (int x = threadIdx.x; x < w_tile; x += blockDim.x) {
        const int32_t i = td.start + x;
        if (i >= ch.L)
            break;
        const int64_t p = ch.offset + i;
        if (u_out)
            u_out[p] = static_cast<double>(st.cell[p]) + static_cast<double>(st.off[p]);
        if (cells_out)
            cells_out[p] = st.cell[p];
    }
}

}  // namespace

bool split_supported(int kind, int S)
{
    if (kind == kRB)
        return S == 8 || S == 16;
    return S == 8 || S == 16 || S == 24 || S == 32;
}

size_t split_smem_bytes(int kind, int S, int tiles_per_cta)
{
    const int nc = (kind == kRB) ? 4 : 2;
    return static_cast<size_t>(tiles_per_cta) * 32 * S * 4 * (2 + nc);
}

cudaError_t split_step(int kind, int S, int tiles_per_cta, const SplitLaunch& a, cudaStream_t st)
{
    if (kind == kRF) {
        switch (S) {
        case 8: return launch_split<kRF, 8>(tiles_per_cta, a, st);
        case 16: return launch_split<kRF, 16>(tiles_per_cta, a, st);
        case 24: return launch_split<kRF, 24>(tiles_per_cta, a, st);
        case 32: return launch_split<kRF, 32>(tiles_per_cta, a, st);
        }
    } else if (kind == kRB) {
        switch (S) {
        case 8: return launch_split<kRB, 8>(tiles_per_cta, a, st);
        case 16: return launch_split<kRB, 16>(tiles_per_cta, a, st);
        }
    } else {
        switch (S) {
        case 8: return launch_split<kNone, 8>(tiles_per_cta, a, st);
        case 16: return launch_split<kNone, 16>(tiles_per_cta, a, st);
        case 24: return launch_split<kNone, 24>(tiles_per_cta, a, st);
        case 32: return launch_split<kNone, 32>(tiles_per_cta, a, st);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t split_init(const ChainDesc* chains, int32_t, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                       SplitState st, uint64_t seed, int, const double* u_in, cudaStream_t stream)
{
    if (n_tiles == 0)
        return cudaSuccess;
    split_init_kernel<<<n_tiles, 256, 0, stream>>>(chains, tiles, w_tile, st, seed, u_in);
    return cudaGetLastError();
}

cudaError_t split_to_f64(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                         SplitState st, double* u_out, int32_t* cells_out, cudaStream_t stream)
{
    if (n_tiles == 0)
        return cudaSuccess;
    split_to_f64_kernel<<<n_tiles, 256, 0, stream>>>(chains, tiles, w_tile, st, u_out, cells_out);
    return cudaGetLastError();
}

}  // namespace qew
