// qew_split.cu -- the fused FP32-split kernel of the qEW relaxation: elastic force + pinning
// force + Euler update + cell renormalisation + disorder regeneration, K Euler steps per HBM
// round trip (temporal blocking), with the checkpoint partial sums fused after the last step.
//
// Method: Eq. 1 of arXiv:1211.7275 with eta = c = 1, discretised in x with periodic boundary
// conditions and integrated by explicit Euler (Sec. III.B); pinning force interpolated from
// random values at integer (i, n) (Sec. III.B and the cases of Sec. IV.C); observables of
// Eqs. 3-5 (Sec. II).
//
// State of a site: integer cell n and FP32 offset d in [0, 1) (u = n + d), held in registers,
// plus its disorder cache, held in shared memory.  Pair kinds keep the two nodes of the cell:
// RF (R(n) + f, R(n+1) + f) -- the drive f is folded in, so F_p + f is one subtraction and one
// FMA -- and the linear-spline random bond (G(n), G(n+1)), F_p + f = (G(n) - G(n+1)) + f.  Quad
// kinds (cubic random bond, uniform V or Gaussian G) keep the coefficients A, B, C of
// F_p + f = A + d (B + d C) over the cell (from the spline nodes V(n-1 .. n+2)) and the three
// nodes V(n), V(n+1), V(n+2) that a move to a neighbouring cell reuses.
//
// Work decomposition: one warp owns one tile of 32 * S sites of a chain, S consecutive sites
// per lane.  A tile advanced K steps needs K extra sites on each side (the stencil's light
// cone), so the window is [start - K, start - K + 32 S) and the owned sites
// [start, start + w_own), w_own <= 32 S - 2K; the outermost sites of the window go stale one
// per step from each edge and are never stored.  Windows wrap around periodic chains (any
// number of times for chains shorter than a tile).  Halo exchange inside a step is two warp
// shuffles per neighbour and there is no block-wide barrier.
//
// Cell crossings: renormalisation is branch-free (n += floor(d), d -= floor(d)) and leaves one
// bit per moved site.  After the update loop each lane stores its cells to shared memory (one
// store per site; a store inside the update loop would keep the compiler from hoisting the cache
// loads there), and a warp prefix sum of the lanes' move counts gives each lane its queue slots,
// which it fills by walking the set bits of its mask (no atomics, deterministic order): all of
// a step's requests in one pass where the queue holds a whole step, else 32 slots per chunk,
// resuming in the next chunk where it stopped.  The queued Philox values are then evaluated 32
// lanes at a time and written straight into the shared-memory cache of the requesting sites; the
// direction of each move is recovered from the cell the cache was drawn for, kept per site in
// shared memory.
#include <cstdio>
#include <mutex>
#include <type_traits>

#include "qew_internal.h"
#include "qew_tma.cuh"

namespace qew {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Chain-local index of window position x (window start wstart, |wstart| <= K).  A window wraps
// at most once around a chain at least as long as the window; shorter chains take the modulo.
// The wrap is taken in 64 bits: past the end of a chain of up to 2^31 - 1 sites, g itself may
// not fit in an int32.
__device__ __forceinline__ int32_t site_index(int64_t wstart, int x, bool contiguous, int32_t L)
{
    const int64_t g = wstart + x;
    if (contiguous)
        return static_cast<int32_t>(g);
    if (g >= -static_cast<int64_t>(L) && g < 2 * static_cast<int64_t>(L))
        return static_cast<int32_t>(g < 0 ? g + L : (g >= L ? g - L : g));
    return wrap_site(g, L);
}

// Bytes of disorder cache per site in HBM.
template <int KIND>
struct CacheBytes {
    static constexpr int hbm = pair_kind(KIND) ? 8 : quad_kind(KIND) ? 24 : 0;
};

// Shared memory per site.  Random-field tiles of 31 or more sites per lane use a compact layout
// of 14 B: one 4-byte staging slot (cells, then offsets, at load and store; each step's new
// cells in between), the 8-byte node pair, and the low 16 bits of the cell the pair was drawn
// for.  At 992-site tiles this fits 16 instead of 14 warps per SM (measured: +3.3%); smaller
// tiles are register-limited, and there the two-pass staging only costs (measured on 736-site
// random-field tiles in a mixed batch and on Case 3).  The other layouts keep 8 bytes of staging
// (cell and offset side by side, the cell half doubling as the cache cell) plus the cache: a
// node pair (8 B), or for the cubic kinds the coefficients and three nodes (24 B, the same in
// HBM, so a tile loads them without recomputing the coefficients).  The cubic kinds are bound by
// the shared-memory data path and by latency; measured on the uniform random bond:
//   - the coefficients as (A, B) pairs and C alone, so the update loop reads 12 bytes per site
//     and step rather than a 16-byte vector with an unused lane: +5% (12 instead of 11 warps per
//     SM at 480-site tiles, one load instruction more per site);
//   - three nodes instead of four (V(n-1) is dropped; a down move draws it again, and at the
//     thresholds down moves are a few in 10^4) and no coefficient recompute at tile load: +10%
//     (14 warps per SM, 108 instead of 124 registers).
__host__ __device__ constexpr bool compact_layout(int kind, int S) { return kind == kRF && S >= 31; }
__host__ __device__ constexpr int site_smem_bytes(int kind, int S)
{
    return compact_layout(kind, S) ? 4 + 8 + 2 : pair_kind(kind) ? 8 + 8 : quad_kind(kind) ? 8 + 24 : 8;
}

// Per warp after its sites, the request queue.  The two-node kinds below 31 sites per lane have
// shared memory to spare: their queue holds every request of a step (a 16-bit window position per
// site of the tile), so each lane walks its move mask once per step instead of once per chunk of
// 32 requests (measured: Case 3, about 90 requests per step and tile, +18.5%; the random field at
// 736-site tiles +2.5%).  The others keep one chunk of 32 requests: the compact random-field
// layout and the cubic kinds are bound by shared memory, and their steps rarely make more than 32
// requests.
__host__ __device__ constexpr bool full_queue(int kind, int S) { return pair_kind(kind) && S < 31; }
__host__ __device__ constexpr int queue_bytes(int kind, int S) { return full_queue(kind, S) ? 32 * S * 2 : 32 * 4; }

// F_p + f at window position x with offset d, from the shared-memory cache.
template <int KIND>
__device__ __forceinline__ float drive_plus_pinning(const float2* s_rf, const float2* s_ab, const float* s_c, int x, float d, float f)
{
    if constexpr (KIND == kRF) {
        const float2 q = s_rf[x];
        return fmaf(d, q.y - q.x, q.x);
    } else if constexpr (KIND == kRBGLinear) {
        const float2 q = s_rf[x];
        return (q.x - q.y) + f;
    } else if constexpr (quad_kind(KIND)) {
        const float2 ab = s_ab[x];
        return fmaf(d, fmaf(d, s_c[x], ab.y), ab.x);
    } else {
        return f;
    }
}

// Per-lane mask of the sites that moved in a step: 32 bits while a lane holds at most 32 sites,
// 64 beyond.  The bit of site j is a compile-time constant in the unrolled update loop, so each
// site still sets one bit of one 32-bit word.
template <int S>
using MoveMask = typename std::conditional<(S <= 32), unsigned, unsigned long long>::type;

__device__ __forceinline__ int mask_popc(unsigned m) { return __popc(m); }
__device__ __forceinline__ int mask_popc(unsigned long long m) { return __popcll(m); }
__device__ __forceinline__ int mask_ffs(unsigned m) { return __ffs(m); }
__device__ __forceinline__ int mask_ffs(unsigned long long m) { return __ffsll(static_cast<long long>(m)); }

// Kinds of cell move.
constexpr int kMoveUp = 1;
constexpr int kMoveDown = 2;
constexpr int kMoveFar = 3;

// Resident 256-thread blocks per SM asked of the register allocator, per kind and lanes' sites.
// Measured: on Case 3 (which regenerates often) a lower-occupancy budget lost 10%, and on the
// random field at S = 31 the 144 registers the allocator takes unasked lost 3% against the
// 128 asked here.
template <int KIND, int S>
struct MinBlocks {
    static constexpr int value = (S <= 8) ? (quad_kind(KIND) ? 3 : 4) : (S <= 16) ? (quad_kind(KIND) ? 2 : 3) : (S <= 31) ? 2 : 1;
};

// Sites per lane are odd: lane l reads its cache at word offsets 2 S l (pair) or 4 S l (quad), and
// an odd S spreads a half-warp (quarter-warp for 16-byte loads) over distinct shared-memory banks.

template <int KIND, int S>
__global__ void __launch_bounds__(256, MinBlocks<KIND, S>::value) split_step_kernel(SplitLaunch a)
{
    constexpr int TW = 32 * S;
    constexpr bool kCompact = compact_layout(KIND, S);
    constexpr bool kFullQueue = full_queue(KIND, S);
    constexpr int WARP_SMEM = TW * site_smem_bytes(KIND, S) + queue_bytes(KIND, S);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ uint64_t s_bar[8];

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int tile = blockIdx.x * (blockDim.x >> 5) + warp;
    if (tile >= a.n_tiles)
        return;  // whole warp; the kernel uses no block-wide barrier

    unsigned char* wsm = smem_raw + static_cast<size_t>(warp) * WARP_SMEM;
    int32_t* s_cell = reinterpret_cast<int32_t*>(wsm);          // staging of n (load/store)
    float* s_off = reinterpret_cast<float*>(wsm + (kCompact ? 0 : 4 * TW));   // staging of d (load/store)
    // During the K loop the staged cells are the cells the caches were drawn for, and the staged
    // offsets' slot of each site takes its cell after the step (relative to N0, as a float).
    int32_t* s_ccell = s_cell;
    float* s_newc = s_off;
    int* s_q = reinterpret_cast<int*>(wsm + TW * site_smem_bytes(KIND, S));   // request chunk
    uint16_t* s_q16 = reinterpret_cast<uint16_t*>(s_q);                       // or all of a step
    // compact layout: staging at 0, the node pair at 4 TW, cache cells (low 16 bits) at 12 TW
    float2* s_rf = reinterpret_cast<float2*>(wsm + (kCompact ? 4 : 8) * TW);
    uint16_t* s_cc16 = reinterpret_cast<uint16_t*>(wsm + 12 * TW);
    float2* s_qn = reinterpret_cast<float2*>(wsm + 8 * TW);     // cubic nodes V(n), V(n+1)
    float* s_q3 = reinterpret_cast<float*>(wsm + 16 * TW);      // and V(n+2)
    float2* s_ab = reinterpret_cast<float2*>(wsm + 20 * TW);    // cubic coefficients (A, B)
    float* s_c = reinterpret_cast<float*>(wsm + 28 * TW);       // and C

    const TileDesc td = a.tiles[tile];
    const ChainDesc ch = a.chains[td.chain];
    const int32_t L = ch.L;
    const int K = a.K;
    const int owned = min(a.w_own, L - td.start);
    const int64_t wstart = static_cast<int64_t>(td.start) - K;
    const bool contiguous = (wstart >= 0) && (wstart + TW <= L);
    const float f = ch.f32;
    const float dt = a.dt;
    const uint32_t s = ch.s;
    const int32_t M = ch.period;

    // ---- stage the window in this warp's shared-memory slice ----
    // Contiguous, 16-byte aligned windows arrive by TMA bulk copies (one per array, completion
    // on the warp's mbarrier); windows that wrap around the chain or start unaligned use
    // coalesced read-only loads.
    // The compact layout stages cells and offsets one after the other through the same slot:
    // cells (with the node pairs) first, then offsets.
    const bool tma_in = contiguous && (((ch.offset + wstart) & 3) == 0);
    const int64_t p0 = ch.offset + wstart;
    uint64_t* bar = &s_bar[warp];
    if (tma_in) {
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncwarp();
        if (lane == 0) {
            if constexpr (kCompact) {
                mbar_arrive_expect_tx(bar, TW * (4 + CacheBytes<KIND>::hbm));
                tma_load_1d(s_cell, a.in.cell + p0, TW * 4, bar);
                tma_load_1d(s_rf, a.in.rf + p0, TW * 8, bar);
            } else {
                mbar_arrive_expect_tx(bar, TW * (8 + CacheBytes<KIND>::hbm));
                tma_load_1d(s_cell, a.in.cell + p0, TW * 4, bar);
                tma_load_1d(s_off, a.in.off + p0, TW * 4, bar);
                if constexpr (pair_kind(KIND))
                    tma_load_1d(s_rf, a.in.rf + p0, TW * 8, bar);
                if constexpr (quad_kind(KIND)) {
                    tma_load_1d(s_qn, a.in.qn + p0, TW * 8, bar);
                    tma_load_1d(s_q3, a.in.q3 + p0, TW * 4, bar);
                    tma_load_1d(s_ab, a.in.qab + p0, TW * 8, bar);
                    tma_load_1d(s_c, a.in.qc + p0, TW * 4, bar);
                }
            }
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
            const int64_t p = ch.offset + site_index(wstart, x, contiguous, L);
            s_cell[x] = __ldg(g_cell + p);
            if constexpr (!kCompact)
                s_off[x] = __ldg(g_off + p);
            if constexpr (pair_kind(KIND))
                s_rf[x] = __ldg(a.in.rf + p);
            if constexpr (quad_kind(KIND)) {
                s_qn[x] = __ldg(a.in.qn + p);
                s_q3[x] = __ldg(a.in.q3 + p);
                s_ab[x] = __ldg(a.in.qab + p);
                s_c[x] = __ldg(a.in.qc + p);
            }
        }
        __syncwarp();
    }

    // Cells are carried as exact small floats relative to the warp's reference cell N0 (window
    // position 0): a neighbour difference is then (c' - c) + (d' - d), three FP32 operations.
    // Neighbouring displacements differ by less than 2^12, so a tile's cells stay far below 2^24.
    const int32_t N0 = s_cell[0];
    float c[S];
    float d[S];
    if constexpr (kCompact) {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int x = lane * S + j;
            const int32_t n = s_cell[x];
            c[j] = static_cast<float>(n - N0);
            s_cc16[x] = static_cast<uint16_t>(n);
        }
        // every lane has read its cells: the offsets may now overwrite the staging slot
        fence_proxy_async_shared();
        __syncwarp();
        if (tma_in) {
            if (lane == 0) {
                mbar_arrive_expect_tx(bar, TW * 4);
                tma_load_1d(s_off, a.in.off + p0, TW * 4, bar);
            }
            const bool landed = __all_sync(kFull, mbar_wait(bar, 1));
            if (!landed) {
                if (lane == 0)
                    atomicExch(a.error, 1);
                mbar_wait(bar, 1);
                return;
            }
        } else {
            for (int x = lane; x < TW; x += 32)
                s_off[x] = __ldg(a.in.off + ch.offset + site_index(wstart, x, contiguous, L));
            __syncwarp();
        }
    }
#pragma unroll
    for (int j = 0; j < S; ++j) {
        const int x = lane * S + j;
        if constexpr (!kCompact)
            c[j] = static_cast<float>(s_cell[x] - N0);
        d[j] = s_off[x];
    }
    __syncwarp();   // the staging area becomes the request queue below

    // ---- K Euler steps: state in registers, cache in shared memory ----
    unsigned n_cross = 0;
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        // Window positions 0 and TW - 1 take themselves as their outer neighbour: they go stale
        // either way, and a zero slope there keeps the stale edge from drifting off and making
        // spurious cell moves (each of which would draw disorder values).
        const float cl0 = __shfl_up_sync(kFull, c[S - 1], 1);
        const float dl0 = __shfl_up_sync(kFull, d[S - 1], 1);
        const float cr0 = __shfl_down_sync(kFull, c[0], 1);
        const float dr0 = __shfl_down_sync(kFull, d[0], 1);
        const float cl = (lane == 0) ? c[0] : cl0;
        const float dl = (lane == 0) ? d[0] : dl0;
        const float cr = (lane == 31) ? c[S - 1] : cr0;
        const float drn = (lane == 31) ? d[S - 1] : dr0;
        float Dm = (c[0] - cl) + (d[0] - dl);   // u_j - u_{j-1}
        MoveMask<S> mv = 0;   // sites that changed cell in this step (bit j: the lane's site j)
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int x = lane * S + j;
            const float cn = (j + 1 < S) ? c[j + 1] : cr;
            const float dd = (j + 1 < S) ? d[j + 1] : drn;
            const float Dp = (cn - c[j]) + (dd - d[j]);   // u_{j+1} - u_j
            const float g = drive_plus_pinning<KIND>(s_rf, s_ab, s_c, x, d[j], f);   // F_p + f
            const float dn = fmaf(dt, (Dp - Dm) + g, d[j]);
            Dm = Dp;
            // Branch-free renormalisation.  d - floor(d) is exact; a tiny negative d can round up
            // to exactly 1, which is a valid representation (the interpolated force is continuous).
            const float fl = floorf(dn);
            c[j] += fl;
            d[j] = dn - fl;
            mv |= (fl != 0.0f) ? (MoveMask<S>(1) << j) : MoveMask<S>(0);
        }
        const unsigned anymv = __reduce_or_sync(kFull, mv);
        if (anymv) {
            // the lane's cells after the step, read by the consumers below for the moved sites
            if constexpr (KIND != kNone) {
#pragma unroll
                for (int j = 0; j < S; ++j)
                    s_newc[lane * S + j] = c[j];
            }
            // queue slots: warp prefix sum of the lanes' move counts; each lane then walks the set
            // bits of its mask.  Chunks of 32 requests, one Philox value per lane and chunk.
            const int cnt = mask_popc(mv);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl += y;
            }
            const int qn = __shfl_sync(kFull, incl, 31);
            n_cross += static_cast<unsigned>(qn);   // the same in every lane
            if constexpr (KIND != kNone) {
                // each lane's walk resumes in the next chunk where it stopped
                int q = incl - cnt;
                MoveMask<S> m = mv;
                if constexpr (kFullQueue) {
                    // every request of the step at once (a site is queued at most once: qn <= TW)
                    while (m != 0) {
                        const int b = mask_ffs(m) - 1;
                        m &= m - 1;
                        s_q16[q] = static_cast<uint16_t>(lane * S + b);
                        ++q;
                    }
                    __syncwarp();
                }
                for (int base = 0; base < qn; base += 32) {
                    if constexpr (!kFullQueue) {
                        while (m != 0 && q < base + 32) {
                            const int b = mask_ffs(m) - 1;
                            m &= m - 1;
                            s_q[q - base] = lane * S + b;   // window position of the site
                            ++q;
                        }
                        __syncwarp();
                    }
                    if (base + lane < qn) {
                        const int x = kFullQueue ? static_cast<int>(s_q16[base + lane]) : s_q[lane];
                        const int nn = N0 + __float2int_rn(s_newc[x]);
                        int move;   // cells moved in this step
                        if constexpr (kCompact) {
                            // from the low 16 bits: exact while a step moves a site by less than
                            // 2^15 cells (|dt (lap + f + F_p)| < 2^15; split_range_guard checks the
                            // neighbour differences that keep it so at every observation)
                            move = static_cast<int16_t>(static_cast<uint16_t>(nn) - s_cc16[x]);
                            s_cc16[x] = static_cast<uint16_t>(nn);
                        } else {
                            move = nn - s_ccell[x];
                            s_ccell[x] = nn;
                        }
                        const int code = (move == 1) ? kMoveUp : (move == -1) ? kMoveDown : kMoveFar;
                        const int32_t i = contiguous ? static_cast<int32_t>(wstart) + x
                                                     : site_index(wstart, x, contiguous, L);
                        if constexpr (pair_kind(KIND) && S < 31) {
                            // one new node, n+1 after an up move and n after a down move; a far move
                            // draws n and n+1.  One call site, with a second trip only for far moves:
                            // a second inlined transform would spill registers at S <= 15.
                            const float2 o = s_rf[x];
                            float2 q = (code == kMoveUp) ? make_float2(o.y, 0.0f) : make_float2(0.0f, o.x);
                            const int n0 = (code == kMoveUp) ? nn + 1 : nn;
                            const int trips = (code == kMoveFar) ? 2 : 1;
#pragma unroll 1
                            for (int r = 0; r < trips; ++r) {
                                const float v = pair_node_f32<KIND>(a.keys, s, i, wrap_node(n0 + r, M), f);
                                if (code == kMoveUp || r == 1)
                                    q.y = v;
                                else
                                    q.x = v;
                            }
                            s_rf[x] = q;
                        } else if constexpr (pair_kind(KIND)) {
                            // the same draws with the far-move node inline: at S = 31 the register
                            // budget binds either way and this form measured 0.5% faster
                            const float v =
                                pair_node_f32<KIND>(a.keys, s, i, wrap_node(code == kMoveUp ? nn + 1 : nn, M), f);
                            const float2 o = s_rf[x];
                            float2 q;
                            if (code == kMoveUp)
                                q = make_float2(o.y, v);
                            else if (code == kMoveDown)
                                q = make_float2(v, o.x);
                            else
                                q = make_float2(v, pair_node_f32<KIND>(a.keys, s, i, wrap_node(nn + 1, M), f));
                            s_rf[x] = q;
                        } else {
                            // The spline over the new cell nn needs V(nn-1 .. nn+2).  The cache
                            // holds V(n), V(n+1), V(n+2) of the old cell n: an up move draws
                            // V(nn+2); a down move draws V(nn-1) and V(nn) (V(n-1) is not kept:
                            // at the thresholds down moves are a few in 10^4); a far move draws
                            // all four.
                            const float v =
                                quad_node_f32<KIND>(a.keys, s, i, wrap_node(code == kMoveUp ? nn + 2 : nn - 1, M));
                            const float2 o = s_qn[x];
                            float p0, p1, p2, p3;
                            if (code == kMoveUp) {
                                p0 = o.x;
                                p1 = o.y;
                                p2 = s_q3[x];
                                p3 = v;
                            } else {
                                p0 = v;
                                p1 = quad_node_f32<KIND>(a.keys, s, i, wrap_node(nn, M));
                                if (code == kMoveDown) {
                                    p2 = o.x;
                                    p3 = o.y;
                                } else {
                                    p2 = quad_node_f32<KIND>(a.keys, s, i, wrap_node(nn + 1, M));
                                    p3 = quad_node_f32<KIND>(a.keys, s, i, wrap_node(nn + 2, M));
                                }
                            }
                            s_qn[x] = make_float2(p1, p2);
                            s_q3[x] = p3;
                            float A, B, C;
                            rb_coefficients(p0, p1, p2, p3, f, A, B, C);
                            s_ab[x] = make_float2(A, B);
                            s_c[x] = C;
                        }
                    }
                    __syncwarp();
                }
            }
        }
    }

    if (a.crossings) {
        const unsigned tot = n_cross;
        if (lane == 0 && tot)
            atomicAdd(a.crossings, static_cast<unsigned long long>(tot));
    }

    // ---- checkpoint partial sums of the state after the K steps (owned sites only) ----
    // FP32 sums relative to the warp's reference cell (lane 0's first site; the spread inside a
    // tile is small), FP32 warp reduction, then one FP64 shift to the chain reference in lane 0.
    if (a.do_obs) {
        const int32_t c_ref = static_cast<int32_t>(a.shift[td.chain]);
        float sF = 0.0f, sy = 0.0f, syy = 0.0f;
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int x = lane * S + j;
            const int o = x - K;
            if (o >= 0 && o < owned) {
                if constexpr (KIND == kRBGLinear) {
                    const float2 q = s_rf[x];
                    sF += q.x - q.y;
                } else {
                    sF += drive_plus_pinning<KIND>(s_rf, s_ab, s_c, x, d[j], f) - f;
                }
                const float y = c[j] + d[j];   // u - N0
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
            const double rel = static_cast<double>(N0) - static_cast<double>(c_ref);
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
    const int64_t out0 = ch.offset + td.start;
    const bool tma_out = ((K & 3) == 0) && ((out0 & 3) == 0) && ((owned & 3) == 0);
    if constexpr (kCompact) {
        // cells and node pairs first, then the offsets through the same staging slot
#pragma unroll
        for (int j = 0; j < S; ++j)
            s_cell[lane * S + j] = N0 + __float2int_rn(c[j]);
        if (tma_out) {
            fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
                const uint32_t cnt = static_cast<uint32_t>(owned);
                tma_store_1d(a.out.cell + out0, s_cell + K, cnt * 4);
                tma_store_1d(a.out.rf + out0, s_rf + K, cnt * 8);
                tma_store_commit();
                tma_store_wait_read_all();   // the staging slot may be overwritten
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < S; ++j)
                s_off[lane * S + j] = d[j];
            fence_proxy_async_shared();
            __syncwarp();
            if (lane == 0) {
                tma_store_1d(a.out.off + out0, s_off + K, static_cast<uint32_t>(owned) * 4);
                tma_store_commit();
                tma_store_wait_all();
            }
        } else {
            __syncwarp();
            for (int o = lane; o < owned; o += 32) {
                a.out.cell[out0 + o] = s_cell[o + K];
                a.out.rf[out0 + o] = s_rf[o + K];
            }
            __syncwarp();
#pragma unroll
            for (int j = 0; j < S; ++j)
                s_off[lane * S + j] = d[j];
            __syncwarp();
            for (int o = lane; o < owned; o += 32)
                a.out.off[out0 + o] = s_off[o + K];
        }
    } else {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const int x = lane * S + j;
            s_cell[x] = N0 + __float2int_rn(c[j]);
            s_off[x] = d[j];
        }
        if (tma_out) {
            fence_proxy_async_shared();   // generic-proxy writes above -> visible to the bulk copy
            __syncwarp();
            if (lane == 0) {
                const uint32_t cnt = static_cast<uint32_t>(owned);
                tma_store_1d(a.out.cell + out0, s_cell + K, cnt * 4);
                tma_store_1d(a.out.off + out0, s_off + K, cnt * 4);
                if constexpr (pair_kind(KIND))
                    tma_store_1d(a.out.rf + out0, s_rf + K, cnt * 8);
                if constexpr (quad_kind(KIND))
                {
                    tma_store_1d(a.out.qn + out0, s_qn + K, cnt * 8);
                    tma_store_1d(a.out.q3 + out0, s_q3 + K, cnt * 4);
                    tma_store_1d(a.out.qab + out0, s_ab + K, cnt * 8);
                    tma_store_1d(a.out.qc + out0, s_c + K, cnt * 4);
                }
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
                if constexpr (pair_kind(KIND))
                    a.out.rf[p] = s_rf[x];
                if constexpr (quad_kind(KIND)) {
                    a.out.qn[p] = s_qn[x];
                    a.out.q3[p] = s_q3[x];
                    a.out.qab[p] = s_ab[x];
                    a.out.qc[p] = s_c[x];
                }
            }
        }
    }
}

template <int KIND, int S>
cudaError_t launch_split(int tiles_per_cta, const SplitLaunch& a, cudaStream_t st)
{
    const size_t smem = static_cast<size_t>(tiles_per_cta) * (32 * S * site_smem_bytes(KIND, S) + queue_bytes(KIND, S));
    auto kern = split_step_kernel<KIND, S>;
    // raise the dynamic shared-memory limit of this kernel on this device to the largest shape in
    // use; under a lock, so that two threads raising it at once cannot leave the smaller value
    static std::mutex s_mu;
    static int s_limit[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    {
        std::lock_guard<std::mutex> g(s_mu);
        const bool tracked = dev >= 0 && dev < 64;
        if (!tracked || static_cast<int>(smem) > s_limit[dev]) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess)
                return e;
            if (tracked)
                s_limit[dev] = static_cast<int>(smem);
        }
    }
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
        const int32_t M = ch.period;
        const int32_t m0 = wrap_node(n - 1, M), m1 = wrap_node(n, M), m2 = wrap_node(n + 1, M), m3 = wrap_node(n + 2, M);
        if (ch.kind == kRF)
            st.rf[p] = make_float2(rf_plus_f32(seed, ch.s, i, m1, ch.f32), rf_plus_f32(seed, ch.s, i, m2, ch.f32));
        else if (ch.kind == kRBGLinear)
            st.rf[p] = make_float2(rbg_f32(seed, ch.s, i, m1), rbg_f32(seed, ch.s, i, m2));
        else if (ch.kind == kRB || ch.kind == kRBGCubic) {
            const bool uni = ch.kind == kRB;
            const float p0 = uni ? rb_f32(seed, ch.s, i, m0) : rbg_f32(seed, ch.s, i, m0);
            const float p1 = uni ? rb_f32(seed, ch.s, i, m1) : rbg_f32(seed, ch.s, i, m1);
            const float p2 = uni ? rb_f32(seed, ch.s, i, m2) : rbg_f32(seed, ch.s, i, m2);
            const float p3 = uni ? rb_f32(seed, ch.s, i, m3) : rbg_f32(seed, ch.s, i, m3);
            float A, B, C;
            rb_coefficients(p0, p1, p2, p3, ch.f32, A, B, C);
            st.qn[p] = make_float2(p1, p2);
            st.q3[p] = p3;
            st.qab[p] = make_float2(A, B);
            st.qc[p] = C;
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
    if (quad_kind(kind))
        return S == 7 || S == 15;
    if (kind == kNone)
        return S == 7 || S == 15 || S == 23 || S == 31;
    return S == 7 || S == 15 || S == 23 || S == 31 || S == 39;
}

size_t split_smem_bytes(int kind, int S, int tiles_per_cta)
{
    return static_cast<size_t>(tiles_per_cta) * (32 * S * site_smem_bytes(kind, S) + queue_bytes(kind, S));
}

cudaError_t split_step(int kind, int S, int tiles_per_cta, const SplitLaunch& a, cudaStream_t st)
{
    if (kind == kRF) {
        switch (S) {
        case 7: return launch_split<kRF, 7>(tiles_per_cta, a, st);
        case 15: return launch_split<kRF, 15>(tiles_per_cta, a, st);
        case 23: return launch_split<kRF, 23>(tiles_per_cta, a, st);
        case 31: return launch_split<kRF, 31>(tiles_per_cta, a, st);
        case 39: return launch_split<kRF, 39>(tiles_per_cta, a, st);
        }
    } else if (kind == kRBGLinear) {
        switch (S) {
        case 7: return launch_split<kRBGLinear, 7>(tiles_per_cta, a, st);
        case 15: return launch_split<kRBGLinear, 15>(tiles_per_cta, a, st);
        case 23: return launch_split<kRBGLinear, 23>(tiles_per_cta, a, st);
        case 31: return launch_split<kRBGLinear, 31>(tiles_per_cta, a, st);
        case 39: return launch_split<kRBGLinear, 39>(tiles_per_cta, a, st);
        }
    } else if (kind == kRB) {
        switch (S) {
        case 7: return launch_split<kRB, 7>(tiles_per_cta, a, st);
        case 15: return launch_split<kRB, 15>(tiles_per_cta, a, st);
        }
    } else if (kind == kRBGCubic) {
        switch (S) {
        case 7: return launch_split<kRBGCubic, 7>(tiles_per_cta, a, st);
        case 15: return launch_split<kRBGCubic, 15>(tiles_per_cta, a, st);
        }
    } else if (kind == kNone) {
        switch (S) {
        case 7: return launch_split<kNone, 7>(tiles_per_cta, a, st);
        case 15: return launch_split<kNone, 15>(tiles_per_cta, a, st);
        case 23: return launch_split<kNone, 23>(tiles_per_cta, a, st);
        case 31: return launch_split<kNone, 31>(tiles_per_cta, a, st);
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
