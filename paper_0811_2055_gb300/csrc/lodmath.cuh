// Device arithmetic of the octree build: the counter-based generator that drives the
// density-weighted random subselection (octree paragraph), the specified log and cube-root
// series, exact fixed-point masses and Morton keys.  Every floating-point operation is an
// explicit round-to-nearest intrinsic so that nothing is contracted into an FMA.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace gbd {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): counter (id, code_lo, code_hi, 0),
// key (seed_lo, seed_hi); the 64-bit draw is (r0 << 32) | r1.
__device__ __forceinline__ uint64_t node_draw(uint64_t seed, uint64_t code, uint32_t id)
{
    uint32_t x0 = id, x1 = (uint32_t)code, x2 = (uint32_t)(code >> 32), x3 = 0u;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t a = 0xD2511F53u * x0, ah = __umulhi(0xD2511F53u, x0);
        const uint32_t b = 0xCD9E8D57u * x2, bh = __umulhi(0xCD9E8D57u, x2);
        const uint32_t y0 = bh ^ x1 ^ k0;
        const uint32_t y2 = ah ^ x3 ^ k1;
        x0 = y0;
        x1 = b;
        x2 = y2;
        x3 = a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return ((uint64_t)x0 << 32) | (uint64_t)x1;
}

// -ln U for U = ((u >> 12) + 1/2) 2^-52, by range reduction to m in [sqrt(1/2), sqrt(2)) and
// the series ln m = 2 s sum_{k=0}^{12} s^(2k)/(2k+1), s = (m-1)/(m+1), Horner from k = 12.
__device__ __forceinline__ double neg_log_unit(uint64_t u)
{
    const double U = __dmul_rn(__dadd_rn(__ull2double_rn(u >> 12), 0.5), 0x1p-52);
    // frexp by the bit pattern (U is a normal number in [2^-53, 1))
    const uint64_t bits = (uint64_t)__double_as_longlong(U);
    int e = (int)((bits >> 52) & 0x7FF) - 1022;
    double m = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FE0000000000000ull));
    if (m < 0x1.6a09e667f3bcdp-1) {
        m = __dmul_rn(m, 2.0);
        e -= 1;
    }
    const double s = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
    const double z = __dmul_rn(s, s);
    double p = __ddiv_rn(1.0, 25.0);
#pragma unroll
    for (int k = 11; k >= 0; --k) p = __dadd_rn(__dmul_rn(p, z), __ddiv_rn(1.0, (double)(2 * k + 1)));
    const double lnm = __dmul_rn(__dmul_rn(2.0, s), p);
    const double lnU = __dadd_rn(__dmul_rn((double)e, 0x1.62e42fefa39efp-1), lnm);
    return -lnU;
}

// Cube root of t >= 1: eight Newton steps s <- (2 s + t / s^2) / 3 from s0 = 2^ceil(e/3),
// t = f 2^e with f in [1/2, 1).
__device__ __forceinline__ double cube_root_ge1(double t)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(t);
    const int e = (int)((bits >> 52) & 0x7FF) - 1022;
    const int k = e >= 0 ? (e + 2) / 3 : -((-e) / 3);
    double s = ldexp(1.0, k);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const double q = __ddiv_rn(t, __dmul_rn(s, s));
        s = __ddiv_rn(__dadd_rn(__dmul_rn(2.0, s), q), 3.0);
    }
    return s;
}

// mass * 2^47 as an exact 128-bit integer (mass is a normal float in [2^-24, 2^24]).
__device__ __forceinline__ gb::U128 mass_fixed(float m)
{
    const uint32_t b = __float_as_uint(m);
    const uint64_t mant = (uint64_t)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = (int)((b >> 23) & 0xFFu) - 103; // (E - 150) + 47
    gb::U128 r;
    if (sh <= 0) {
        r.lo = mant >> (-sh);
        r.hi = 0ull;
    } else {
        r.lo = mant << sh;
        r.hi = sh >= 41 ? (mant >> (64 - sh)) : 0ull;
    }
    return r;
}

// spread the low 21 bits of v to every third bit (bit i -> bit 3i)
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// gather every third bit (inverse of spread3)
__device__ __forceinline__ uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x | (x >> 8)) & 0x001F0000FF0000FFull;
    x = (x | (x >> 16)) & 0x001F00000000FFFFull;
    x = (x | (x >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)x;
}

// q = clamp(floor((double(x) - lo) * scale), 0, 2^21 - 1); NaN -> 0
__device__ __forceinline__ uint32_t quantize_axis(float x, double lo, double scale)
{
    const double t = __dmul_rn(__dsub_rn((double)x, lo), scale);
    if (!(t >= 0.0)) return 0u;
    if (!(t < 2097152.0)) return 2097151u;
    return (uint32_t)__double2uint_rz(t);
}

// The same when the root cube starts at 0 and scale is a power of two (within fp32 range): x * scale
// is then exact in fp32 (scaling by a power of two; a result below 1 truncates to 0 either way), so
// the fp32 product gives the identical q without FP64 arithmetic.
__device__ __forceinline__ uint32_t quantize_axis_pow2(float x, float scale)
{
    const float t = __fmul_rn(x, scale);
    if (!(t >= 0.0f)) return 0u;
    if (!(t < 2097152.0f)) return 2097151u;
    return (uint32_t)__float2uint_rz(t);
}

__device__ __forceinline__ uint64_t morton_key_pow2(float x, float y, float z, float scale)
{
    const uint32_t qx = quantize_axis_pow2(x, scale), qy = quantize_axis_pow2(y, scale),
                   qz = quantize_axis_pow2(z, scale);
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

__device__ __forceinline__ uint64_t morton_key(float x, float y, float z, double lx, double ly, double lz,
                                               double scale)
{
    const uint32_t qx = quantize_axis(x, lx, scale), qy = quantize_axis(y, ly, scale), qz = quantize_axis(z, lz, scale);
    return (spread3(qx) << 2) | (spread3(qy) << 1) | spread3(qz);
}

} // namespace gbd
