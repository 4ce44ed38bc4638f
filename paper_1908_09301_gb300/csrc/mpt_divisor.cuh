// mpt_divisor.cuh -- division of 32-bit integers by a small invariant
// divisor with a multiplier and shifts (host and device), used by the closes of
// Eq. (3)'s brackets (division by m + 1) and of the Horner steps of Eq. (2).
#pragma once
#include <cstdint>

namespace mpt {

// ------------------------------------------------------------------ division by an invariant

// Division of a 32-bit n by d (1 <= d < 2^31) with a multiplier and shifts:
// the method of Granlund and Montgomery, "Division by invariant integers
// using multiplication" (PLDI 1994), Sec. 4: with l = ceil(log2 d),
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// q = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct Divisor {
    uint32_t d, m;
    int s1, s2;
};

__host__ __device__ inline Divisor make_divisor(uint32_t d)
{
    Divisor v;
    v.d = d;
    int l = 0;
    while (l < 32 && (1ull << l) < d) l++;
    v.m = (uint32_t)((((1ull << l) - d) << 32) / d + 1);
    v.s1 = l < 1 ? l : 1;
    v.s2 = l - 1 > 0 ? l - 1 : 0;
    return v;
}

// make_divisor for 1 <= d < 2^16 without a 64-bit division: l from a count of
// leading zeros, and floor(2^32 (2^l - d) / d) from two 32-by-16-bit steps
// (2^l - d < d, so each step's quotient fits in 16 bits).  Same result.
__host__ __device__ inline Divisor make_divisor16(uint32_t d)
{
    Divisor v;
    v.d = d;
#ifdef __CUDA_ARCH__
    const int l = d > 1u ? 32 - __clz((int)(d - 1u)) : 0;
#else
    int l = 0;
    while ((1u << l) < d) l++;
#endif
    const uint32_t A = (uint32_t)((1u << l) - d);  // < d
    const uint32_t n1 = A << 16, q1 = n1 / d, r1 = n1 - q1 * d;
    const uint32_t n0 = r1 << 16, q0 = n0 / d;
    v.m = ((q1 << 16) | q0) + 1u;
    v.s1 = l < 1 ? l : 1;
    v.s2 = l - 1 > 0 ? l - 1 : 0;
    return v;
}

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ uint32_t div_inv(uint32_t n, const Divisor &v)
{
    uint32_t t = mulhi32(v.m, n);
    return (t + ((n - t) >> v.s1)) >> v.s2;
}

// (r * 2^32 + x) div d with r < d < 2^16 on entry; r becomes the remainder
__host__ __device__ __forceinline__ uint32_t divstep(uint32_t &r, uint32_t x, const Divisor &v)
{
    uint32_t n1 = (r << 16) | (x >> 16);
    uint32_t q1 = div_inv(n1, v);
    uint32_t r1 = n1 - q1 * v.d;
    uint32_t n0 = (r1 << 16) | (x & 0xffffu);
    uint32_t q0 = div_inv(n0, v);
    r = n0 - q0 * v.d;
    return (q1 << 16) | q0;
}

__host__ __device__ __forceinline__ uint32_t mod_inv(uint32_t n, const Divisor &v)
{
    return n - div_inv(n, v) * v.d;
}

}  // namespace mpt
