// qew_device.cuh -- device-side building blocks of the qEW engine: the Philox4x32-10 block
// function, the transforms of its output words to disorder values, and the descriptors that
// map warp tiles to chains.
//
// Disorder (arXiv:1211.7275, Sec. III.B): uncorrelated random numbers drawn at the integer
// points (i, n) of the (x, u) plane, generated on demand (the memory-free variant of
// Sec. IV.D).  The generator is Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), keyed by
// the seed and counted by (i, (uint32) n, s, tag).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace qew {

// Disorder kinds (the cases of Sec. IV.C).
constexpr int kRF = 0;         // random field: Gaussian R at the integers, linear interpolation (Case 4)
constexpr int kRB = 1;         // random bond: uniform V, Catmull-Rom spline (Case 2)
constexpr int kNone = 2;       // no disorder
constexpr int kRBGLinear = 3;  // random bond: Gaussian G, linear spline, F = G(n) - G(n+1) (Case 3)
constexpr int kRBGCubic = 4;   // random bond: Gaussian G, Catmull-Rom spline (Case 1)
constexpr int kNumKinds = 5;

// Cache families: "pair" kinds keep the two nodes of the current cell per site, "quad" kinds
// the cubic spline's coefficients over the cell (from the four nodes V(n-1 .. n+2)) and the
// nodes V(n), V(n+1), V(n+2).
__host__ __device__ constexpr bool pair_kind(int k) { return k == kRF || k == kRBGLinear; }
__host__ __device__ constexpr bool quad_kind(int k) { return k == kRB || k == kRBGCubic; }
constexpr int kPairMask = (1 << kRF) | (1 << kRBGLinear);
constexpr int kQuadMask = (1 << kRB) | (1 << kRBGCubic);

constexpr uint32_t kTagRF = 0u;   // counter word 3 of random-field force values
constexpr uint32_t kTagRB = 1u;   // counter word 3 of uniform random-bond potential values
constexpr uint32_t kTagRBG = 2u;  // counter word 3 of Gaussian random-bond potential values (Cases 1, 3)

// One chain of the batch.
struct ChainDesc {
    int64_t offset;   // first site of the chain in the concatenated state arrays
    int32_t L;        // number of sites
    uint32_t s;       // sample index (counter word 2)
    int32_t kind;     // kRF / kRB / kNone
    int32_t tile0;    // first partial-sum slot of this chain (tiles of its list)
    int32_t ntiles;   // number of tiles (partial-sum slots) of this chain
    float f32;        // drive f, FP32
    int32_t period;   // disorder period M in u (node index taken mod M); 0: aperiodic
    double f64;       // drive f, FP64
};

// Node index that keys the generator: n itself, or n mod M in [0, M) for a disorder periodic in
// u with period M (the L x M system of Sec. III.B).
__host__ __device__ __forceinline__ int32_t wrap_node(int32_t n, int32_t period)
{
    if (period <= 0)
        return n;
    const int32_t r = n % period;
    return r < 0 ? r + period : r;
}

// One warp tile of the fused kernel (or one block tile of the FP64 kernels): chain and first
// owned site.
struct TileDesc {
    int32_t chain;
    int32_t start;
};

// ---------------------------------------------------------------------------------------
// Philox4x32-10.  Round: multiply words 0 and 2 by the two round multipliers (full 64-bit
// products); the new words are (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1,
// lo(M0 x0)); the key advances by the two Weyl increments between rounds.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c.y ^ k0;
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c.w ^ k1;
        c = make_uint4(n0, static_cast<uint32_t>(p1), n2, static_cast<uint32_t>(p0));
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The ten round keys of a seed, (k0 + r W0, k1 + r W1) for r = 0..9, computed once on the host:
// passed as kernel parameters they are read from the constant bank as XOR operands, so a block
// evaluation needs no key additions.
struct PhiloxKeys {
    uint32_t k[20];
};

__host__ __device__ inline PhiloxKeys philox_key_schedule(uint64_t seed)
{
    PhiloxKeys ks;
    uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        ks.k[2 * r] = k0;
        ks.k[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ks;
}

// Philox4x32-10 with a precomputed key schedule (same function as philox4x32_10).
__device__ __forceinline__ uint4 philox4x32_10_ks(uint4 c, const PhiloxKeys& ks)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = static_cast<uint64_t>(0xD2511F53u) * c.x;
        const uint64_t p1 = static_cast<uint64_t>(0xCD9E8D57u) * c.z;
        const uint32_t n0 = static_cast<uint32_t>(p1 >> 32) ^ c.y ^ ks.k[2 * r];
        const uint32_t n2 = static_cast<uint32_t>(p0 >> 32) ^ c.w ^ ks.k[2 * r + 1];
        c = make_uint4(n0, static_cast<uint32_t>(p1), n2, static_cast<uint32_t>(p0));
    }
    return c;
}

__device__ __forceinline__ uint4 disorder_words(uint64_t seed, uint32_t s, int32_t i, int32_t n, uint32_t tag)
{
    return philox4x32_10(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(n), s, tag),
                         static_cast<uint32_t>(seed), static_cast<uint32_t>(seed >> 32));
}

// ln U1 for U1 = (x + 1/2) 2^-32, in FP32, from the odd series of the inverse hyperbolic tangent,
// 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + ...), with s in [0, 1/3] in both halves:
//   x < 2^31:   U1 = 2^e m with m in [1, 2) read from the float's bits, and
//               ln U1 = e ln 2 + ln m,  ln m = 2 atanh((m - 1) / (m + 1));
//   x >= 2^31:  1 - U1 = t = (~x + 1/2) 2^-32 is exact in the word arithmetic, and
//               ln U1 = ln(1 - t) = -2 atanh(t / (2 - t)),
// so values of U1 near 1 keep their relative accuracy (forming 1 - U1 from a rounded U1 would
// cancel).  Nine terms reach FP32 resolution for s <= 1/3 (the next is below 3e-9 s).  Both
// halves are evaluated and selected, so a warp of mixed words does not diverge; the quotient is
// an approximate reciprocal refined by one Newton step.
__device__ __forceinline__ float ln_u1_f32(uint32_t x)
{
    const bool upper = (x & 0x80000000u) != 0;
    const float u1 = fmaf(static_cast<float>(x), 0x1p-32f, 0x1p-33f);
    const uint32_t bits = __float_as_uint(u1);
    const float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);   // exact
    const float e = static_cast<float>(static_cast<int>(bits >> 23) - 127);
    const float t = fmaf(static_cast<float>(~x), 0x1p-32f, 0x1p-33f);
    const float num = upper ? t : m - 1.0f;
    const float den = upper ? 2.0f - t : m + 1.0f;
    const float rc = __fdividef(1.0f, den);
    const float s0 = num * rc;
    const float s = fmaf(fmaf(-s0, den, num), rc, s0);   // one Newton correction of num / den
    const float z = s * s;
    float p = 1.0f / 17.0f;
    p = fmaf(p, z, 1.0f / 15.0f);
    p = fmaf(p, z, 1.0f / 13.0f);
    p = fmaf(p, z, 1.0f / 11.0f);
    p = fmaf(p, z, 1.0f / 9.0f);
    p = fmaf(p, z, 1.0f / 7.0f);
    p = fmaf(p, z, 1.0f / 5.0f);
    p = fmaf(p, z, 1.0f / 3.0f);
    p = fmaf(p, z, 1.0f);
    const float at2 = 2.0f * s * p;   // 2 atanh(s)
    return upper ? -at2 : fmaf(e, 0.693147180559945f, at2);
}

// cos(2 pi U2) for U2 = (x + 1/2) 2^-32, in FP32.  The octant k = x >> 29 and, within it, the
// distance to the nearest multiple of pi/2 (in units of pi/4, formed exactly from the low 29 bits)
// reduce the angle to theta in (0, pi/4); cos(2 pi U2) is then +-cos(theta) or +-sin(theta), from
// their Taylor polynomials (truncation below 2e-9).  The reduction is exact, so the result keeps
// a relative accuracy of about 1e-7 also near the zeros of the cosine.
__device__ __forceinline__ float cos_2pi_word(uint32_t x)
{
    const uint32_t k = x >> 29;
    const uint32_t r = x & 0x1FFFFFFFu;
    const uint32_t q = (k & 1u) ? (0x1FFFFFFFu - r) : r;
    const float th = fmaf(static_cast<float>(q), 0x1p-29f, 0x1p-30f) * 0.785398163397448f;
    const float z = th * th;
    float sp = 1.0f / 362880.0f;
    sp = fmaf(sp, z, -1.0f / 5040.0f);
    sp = fmaf(sp, z, 1.0f / 120.0f);
    sp = fmaf(sp, z, -1.0f / 6.0f);
    const float sn = fmaf(sp * z, th, th);
    float cp = -1.0f / 3628800.0f;
    cp = fmaf(cp, z, 1.0f / 40320.0f);
    cp = fmaf(cp, z, -1.0f / 720.0f);
    cp = fmaf(cp, z, 1.0f / 24.0f);
    cp = fmaf(cp, z, -0.5f);
    const float cs = fmaf(cp, z, 1.0f);
    const float v = (((k + 1u) >> 1) & 1u) ? sn : cs;   // octants 1, 2, 5, 6 take the sine
    return (((k + 2u) >> 2) & 1u) ? -v : v;             // octants 2 .. 5 are negative
}

// N(0, 1) value sqrt(-2 ln U1) cos(2 pi U2), U_k = (x_k + 1/2) 2^-32 (Box-Muller, cosine
// branch): the random-field force R and the Gaussian random-bond potential G.  The value plus
// `add` is rounded once (the random-field cache holds R + f), by an explicit fused multiply-add,
// so every kernel that draws a value rounds it the same way.  -2 ln U1 > 0 always (U1 < 1), so
// its square root is a rsqrt(a), refined by one Newton step.
__device__ __forceinline__ float gauss_value_plus_f32(uint4 w, float add)
{
    const float a = -2.0f * ln_u1_f32(w.x);
    const float y = rsqrtf(a);
    const float r0 = a * y;
    const float r = fmaf(fmaf(-r0, r0, a), 0.5f * y, r0);   // one Newton correction of sqrt(a)
    return __fmaf_rn(r, cos_2pi_word(w.y), add);
}

__device__ __forceinline__ float gauss_value_f32(uint4 w)
{
    return gauss_value_plus_f32(w, 0.0f);
}

__device__ __forceinline__ double gauss_value_f64(uint4 w)
{
    const double u1 = (static_cast<double>(w.x) + 0.5) * 0x1p-32;
    const double u2 = (static_cast<double>(w.y) + 0.5) * 0x1p-32;
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// V = (x0 + 1/2) 2^-31 - 1, uniform on (-1, 1).
__device__ __forceinline__ float rb_value_f32(uint4 w)
{
    return fmaf(static_cast<float>(w.x), 0x1p-31f, -1.0f);
}

__device__ __forceinline__ double rb_value_f64(uint4 w)
{
    return (static_cast<double>(w.x) + 0.5) * 0x1p-31 - 1.0;
}

__device__ __forceinline__ float rf_f32(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f32(disorder_words(seed, s, i, n, kTagRF));
}

// R(i, n) + f, rounded once: the random-field cache value.
__device__ __forceinline__ float rf_plus_f32(uint64_t seed, uint32_t s, int32_t i, int32_t n, float f)
{
    return gauss_value_plus_f32(disorder_words(seed, s, i, n, kTagRF), f);
}

__device__ __forceinline__ float rbg_f32(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f32(disorder_words(seed, s, i, n, kTagRBG));
}

__device__ __forceinline__ float rb_f32(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return rb_value_f32(disorder_words(seed, s, i, n, kTagRB));
}

__device__ __forceinline__ float rf_f32(const PhiloxKeys& ks, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f32(
        philox4x32_10_ks(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(n), s, kTagRF), ks));
}

__device__ __forceinline__ float rbg_f32(const PhiloxKeys& ks, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f32(
        philox4x32_10_ks(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(n), s, kTagRBG), ks));
}

__device__ __forceinline__ float rb_f32(const PhiloxKeys& ks, uint32_t s, int32_t i, int32_t n)
{
    return rb_value_f32(
        philox4x32_10_ks(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(n), s, kTagRB), ks));
}

__device__ __forceinline__ double rf_f64(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f64(disorder_words(seed, s, i, n, kTagRF));
}

__device__ __forceinline__ double rbg_f64(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return gauss_value_f64(disorder_words(seed, s, i, n, kTagRBG));
}

// The two cell nodes of a pair kind (FP32): R + f for RF (the drive is folded into the cache), G
// for the linear-spline random bond.
template <int KIND>
__device__ __forceinline__ float pair_node_f32(const PhiloxKeys& ks, uint32_t s, int32_t i, int32_t n, float f)
{
    if constexpr (KIND == kRF)
        return gauss_value_plus_f32(
            philox4x32_10_ks(make_uint4(static_cast<uint32_t>(i), static_cast<uint32_t>(n), s, kTagRF), ks), f);
    else
        return rbg_f32(ks, s, i, n);
}

// A spline node of a quad kind (FP32): uniform V or Gaussian G.
template <int KIND>
__device__ __forceinline__ float quad_node_f32(const PhiloxKeys& ks, uint32_t s, int32_t i, int32_t n)
{
    if constexpr (KIND == kRB)
        return rb_f32(ks, s, i, n);
    else
        return rbg_f32(ks, s, i, n);
}

__device__ __forceinline__ double rb_f64(uint64_t seed, uint32_t s, int32_t i, int32_t n)
{
    return rb_value_f64(disorder_words(seed, s, i, n, kTagRB));
}

// Exact int -> float for -2^22 <= k < 2^22 without the conversion pipe: adding the bit pattern
// of 1.5 * 2^23 places k in the mantissa of a float whose unit in the last place is 1; the
// subtraction then removes the bias exactly (the "magic number" conversion).
__device__ __forceinline__ float small_int_to_float(int k)
{
    return __int_as_float(k + 0x4B400000) - 12582912.0f;
}

// RB cubic coefficients of F_p + f = A + d (B + d C) for the Catmull-Rom spline through
// p0..p3 = V(n-1 .. n+2):  -dV/du = -1/2 [(p2 - p0) + 2 b d + 3 c d^2],
// b = 2 p0 - 5 p1 + 4 p2 - p3, c = -p0 + 3 p1 - 3 p2 + p3.
// Every operation is an explicit round-to-nearest intrinsic: left to itself the compiler may
// contract a multiply and an add differently in different kernel instantiations, and the cache
// coefficients (hence the trajectory) would then depend on the launch shape.
__device__ __forceinline__ void rb_coefficients(float p0, float p1, float p2, float p3, float f, float& A,
                                                float& B, float& C)
{
    A = __fmaf_rn(-0.5f, __fsub_rn(p2, p0), f);
    B = -__fsub_rn(__fadd_rn(__fsub_rn(__fmul_rn(2.0f, p0), __fmul_rn(5.0f, p1)), __fmul_rn(4.0f, p2)), p3);
    C = __fmul_rn(-1.5f, __fadd_rn(__fsub_rn(__fsub_rn(__fmul_rn(3.0f, p1), p0), __fmul_rn(3.0f, p2)), p3));
}

// Site index i modulo L for any int64 position (windows may wrap more than once on short chains).
__device__ __forceinline__ int32_t wrap_site(int64_t g, int32_t L)
{
    int64_t r = g % L;
    return static_cast<int32_t>(r < 0 ? r + L : r);
}

}  // namespace qew
