// qew_internal.h -- declarations shared by the translation units of the qEW library (kernel
// launchers and the buffers they work on).  Not part of the public C ABI (include/qew.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <string>

#include "qew_device.cuh"

namespace qew {

// FP32-split state: cell n (int32), in-cell offset d (float, [0,1)) and the disorder cache
// of each site.  The two-node kinds keep (R(n) + f, R(n+1) + f) or (G(n), G(n+1)) in rf.  The
// cubic kinds keep the nodes V(n), V(n+1) in qn, V(n+2) in q3, and the coefficients of
// F_p + f = A + d (B + d C) over cell n (from V(n-1) .. V(n+2)) in qab (A, B) and qc (C).  A
// chain of kind NONE uses none of them.
struct SplitState {
    int32_t* cell;
    float* off;
    float2* rf;
    float2* qn;
    float* q3;
    float2* qab;
    float* qc;
};

// FP64 state: displacement u, and the disorder cache of the cell `ncache` it was drawn for:
// RF R(n), R(n+1) in c[0], c[1]; RB V(n-1..n+2) in c[0..3].
struct F64State {
    double* u;
    int32_t* ncache;
    double* c[4];
};

struct SplitLaunch {
    const TileDesc* tiles;   // tiles of one disorder kind
    int32_t n_tiles;
    int32_t tile_base;       // partial-sum slot of tiles[0]
    const ChainDesc* chains;
    SplitState in, out;
    int32_t K;               // Euler steps in this launch (0: observe only)
    int32_t w_own;           // owned sites per tile
    float dt;
    uint64_t seed;
    int32_t do_obs;          // write per-tile partial sums of the state after the K steps
    const double* shift;     // per-chain reference cell c of the sums
    double* partial;         // [n_tiles_total][3]: sum F, sum (u - c), sum (u - c)^2
    unsigned long long* crossings;  // if not null: cell crossings are added here
    int32_t* error;          // 1: a bounded wait on a bulk copy gave up; 2: neighbouring cells 2^12 apart
    PhiloxKeys keys;         // round keys of `seed`
};

// Sites per lane of the fused kernel for each supported tile width (tile_w = 32 * S).
bool split_supported(int kind, int sites_per_lane);
size_t split_smem_bytes(int kind, int sites_per_lane, int tiles_per_cta);
cudaError_t split_step(int kind, int sites_per_lane, int tiles_per_cta, const SplitLaunch& a, cudaStream_t st);
cudaError_t split_init(const ChainDesc* chains, int32_t n_chains, const TileDesc* tiles, int32_t n_tiles,
                       int32_t w_tile, SplitState st, uint64_t seed, int any_rb, const double* u_in,
                       cudaStream_t stream);
cudaError_t split_to_f64(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                         SplitState st, double* u_out, int32_t* cells_out, cudaStream_t stream);
// Sets *error to 2 if neighbouring cells of the FP32-split state differ by 2^12 or more (the range
// in which the fused kernel's cell arithmetic is exact); max_L is the longest chain.
cudaError_t split_range_guard(const ChainDesc* chains, int32_t n_chains, int64_t max_L, const int32_t* cell,
                              int32_t* error, cudaStream_t stream);

struct F64Launch {
    const TileDesc* tiles;   // block tiles of w_tile sites
    int32_t n_tiles;
    int32_t w_tile;
    const ChainDesc* chains;
    F64State st;             // cache is updated in place
    const double* u_in;
    double* u_out;
    double dt;
    uint64_t seed;
    const double* shift;
    double* partial;
};

cudaError_t f64_step(const F64Launch& a, cudaStream_t st);
cudaError_t f64_observe(const F64Launch& a, cudaStream_t st);
cudaError_t f64_init(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                     F64State st, uint64_t seed, int any_rb, const double* u_in, cudaStream_t stream);
cudaError_t f64_cells(const ChainDesc* chains, const TileDesc* tiles, int32_t n_tiles, int32_t w_tile,
                      const double* u, int32_t* cells_out, cudaStream_t stream);

// Second pass: per chain, sum the partials of its tiles in a fixed order, record
// (sum F, S1, S2, c) into obs[chain] and move the chain's reference c to the new centre of
// mass (rounded to an integer cell when `integer_shift`).
cudaError_t reduce_chains(const ChainDesc* chains, int32_t n_chains, const double* partial, double* shift,
                          double* obs, int integer_shift, cudaStream_t stream);

// Structure factor (Eq. 6): rows of u(x) - c0 per chain in the padded layout of an in-place
// real-to-complex FFT (row stride 2 (L/2 + 1) doubles), from the split state (split != NULL) or
// the FP64 state; then the mean over chains of |Z(n)|^2 / L^2 for n = 1 .. n_modes.
cudaError_t sq_rows(const ChainDesc* chains, int32_t n_chains, int32_t L, const SplitState* split, const double* u64,
                    double* rows, cudaStream_t stream);
cudaError_t sq_power(const void* Z, int32_t L, int32_t n_chains, int32_t n_modes, double* S, cudaStream_t stream);

// Message returned by qew_last_error(NULL) for calls without a handle (this thread).
void set_last_error(const std::string& msg);

// Launch one warp whose mbarrier wait cannot complete; it sets *d_error after spin_limit polls.
cudaError_t bounded_wait_selftest(int32_t* d_error, int spin_limit, cudaStream_t stream);

cudaError_t philox_words(const uint32_t* ctr, const uint32_t* key, int64_t n_blocks, uint32_t* out,
                         cudaStream_t stream);
cudaError_t disorder_values(int kind, int fp64, uint64_t seed, uint32_t s, const int64_t* i, const int64_t* n,
                            int64_t count, double* out, cudaStream_t stream);

}  // namespace qew
