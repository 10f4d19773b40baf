// qew_sq.cu -- the structure factor of Eq. 6 (Sec. II of arXiv:1211.7275):
//     S_q = mean over chains of |(1/L) sum_x u(x) e^{-iqx}|^2,  q = 2 pi n / L,  n = 1 .. L/2.
// The line is written as FP64 rows of 2 (L/2 + 1) values per chain (the padded layout of an
// in-place real-to-complex FFT), transformed by cuFFT, and the mode powers are averaged over the
// chains by sq_power_kernel, in a fixed order.
#include "qew_internal.h"

namespace qew {
namespace {

// Row c holds u(x) - c0 for chain c, where c0 is the cell (FP32-split) or the floor (FP64) of
// site 0: the shift leaves every mode n >= 1 unchanged and keeps the values small, so the
// transform's rounding error stays at the scale of the line's width, not of its position.
__global__ void sq_rows_split_kernel(const ChainDesc* chains, int32_t n_chains, SplitState st, int32_t L, int64_t P,
                                     double* rows)
{
    for (int c = blockIdx.y; c < n_chains; c += gridDim.y) {
        const ChainDesc ch = chains[c];
        const int32_t c0 = st.cell[ch.offset];
        double* row = rows + static_cast<int64_t>(c) * P;
        for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < L;
             i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
            const int64_t p = ch.offset + i;
            row[i] = static_cast<double>(st.cell[p] - c0) + static_cast<double>(st.off[p]);   // exact
        }
    }
}

__global__ void sq_rows_f64_kernel(const ChainDesc* chains, int32_t n_chains, const double* u, int32_t L, int64_t P,
                                   double* rows)
{
    for (int c = blockIdx.y; c < n_chains; c += gridDim.y) {
        const ChainDesc ch = chains[c];
        const double c0 = floor(u[ch.offset]);
        double* row = rows + static_cast<int64_t>(c) * P;
        for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < L;
             i += static_cast<int64_t>(gridDim.x) * blockDim.x)
            row[i] = u[ch.offset + i] - c0;
    }
}

// S[k] = scale * sum over chains c (in order) of |Z_c(k + 1)|^2, k < n_modes.  One thread per
// mode: a warp reads 32 consecutive complex values of a row, coalesced.
__global__ void sq_power_kernel(const double2* Z, int64_t Pz, int32_t n_chains, int32_t n_modes, double scale,
                                double* S)
{
    for (int64_t k = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; k < n_modes;
         k += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        double acc = 0.0;
        for (int c = 0; c < n_chains; ++c) {
            const double2 z = Z[static_cast<int64_t>(c) * Pz + k + 1];
            acc = fma(z.x, z.x, fma(z.y, z.y, acc));
        }
        S[k] = acc * scale;
    }
}

int sq_grid(int64_t n)
{
    const int64_t blocks = (n + 255) / 256;
    return static_cast<int>(blocks < 4 * 152 ? (blocks < 1 ? 1 : blocks) : 4 * 152);
}

}  // namespace

cudaError_t sq_rows(const ChainDesc* chains, int32_t n_chains, int32_t L, const SplitState* split, const double* u64,
                    double* rows, cudaStream_t stream)
{
    const int64_t P = 2 * (static_cast<int64_t>(L) / 2 + 1);
    const dim3 grid(sq_grid(L) / 4 + 1, n_chains < 4096 ? n_chains : 4096);
    if (split)
        sq_rows_split_kernel<<<grid, 256, 0, stream>>>(chains, n_chains, *split, L, P, rows);
    else
        sq_rows_f64_kernel<<<grid, 256, 0, stream>>>(chains, n_chains, u64, L, P, rows);
    return cudaGetLastError();
}

cudaError_t sq_power(const void* Z, int32_t L, int32_t n_chains, int32_t n_modes, double* S, cudaStream_t stream)
{
    const int64_t Pz = static_cast<int64_t>(L) / 2 + 1;
    const double scale = 1.0 / (static_cast<double>(L) * static_cast<double>(L) * n_chains);
    sq_power_kernel<<<sq_grid(n_modes), 256, 0, stream>>>(static_cast<const double2*>(Z), Pz, n_chains, n_modes,
                                                          scale, S);
    return cudaGetLastError();
}

}  // namespace qew
