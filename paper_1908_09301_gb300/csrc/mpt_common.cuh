// mpt_common.cuh -- device building blocks of the multiple-precision Taylor
// step (Sec. 2 of Dimova et al., arXiv 1908.09301): exact limb products into
// int64 column windows, carry normalisation, division by a small integer with
// truncation to L limbs.  Shared by the kernels of this library.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "mpt_kernel.cuh"

namespace mpt {

constexpr unsigned FULL = 0xffffffffu;

// Shared-memory layout of an operand vector: one padding word every 8 words,
// so that lanes reading words 8 apart hit different banks.
__host__ __device__ __forceinline__ int phys(int x) { return x + (x >> 3); }

// int64 accumulator windows use the same skew (one padding column every 8).
__host__ __device__ __forceinline__ int wphys(int c) { return c + (c >> 3); }
__host__ __device__ __forceinline__ int wsize(int Wcap) { return wphys(Wcap) + 1; }

// one 32x32 limb product added into a 96-bit column (c0, c1, c2)
__device__ __forceinline__ void mac_cc(uint32_t a, uint32_t b, uint32_t &c0, uint32_t &c1,
                                       uint32_t &c2)
{
    asm volatile(
        "mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
        "addc.u32 %2, %2, 0;"
        : "+r"(c0), "+r"(c1), "+r"(c2)
        : "r"(a), "r"(b));
}

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

// ------------------------------------------------------------------ limb-product units

// Columns of the exact product A*B (Lp x Lp limbs, column c = sum_i a_i b_{c-i}).
// A thread owns column pair q: block1 = [qW, qW+W), block2 = [qW+Lp, qW+Lp+W);
// the pair holds W*Lp products and is walked as s = 0 .. (P+1)W-1 (block1
// for s < (q+1)W with i = s, block2 after with i = s - W).  The W b-limbs in
// registers slide down one limb per step through a cyclic copy C of B padded
// with W zeros (C[x] = b_x for x < Lp, 0 below M = Lp + W), so the hand-over
// from block1 to block2 needs no reload.  A unit covers steps [s0, s1)
// (multiples of W).  The block1 sums are saved at the hand-over; the copy is
// predicated per lane and only issued in chunks where some lane among the
// ones running together hands over (a vote over the active lanes: a lane that
// needs the copy always takes it, the others copy nothing), so lanes of one
// warp never diverge and callers may run units in loops of unequal length.
//
// Output: v1[t] (t < W+2) is the block1 contribution to column qW + t,
// v2[t] the block2 contribution to column qW + Lp + t, as signed int64
// digits of the exact 96-bit column sums.
template <bool SPARSE>
__device__ __forceinline__ void mac_unit_vals(const uint32_t *A, const uint32_t *C, int q, int s0,
                                              int s1, int Lp, int M, long long v1[W + 2],
                                              long long v2[W + 2])
{
    uint32_t a0[W], a1[W], a2[W], k0[W], k1[W], k2[W], bw[W];
    {
        int x0 = q * W - s0;
        if (x0 < 0) x0 += M;  // aligned to W, so the W limbs do not wrap
        const uint32_t *Cp = C + phys(x0);
#pragma unroll
        for (int k = 0; k < W; k++) {
            a0[k] = a1[k] = a2[k] = 0u;
            k0[k] = k1[k] = k2[k] = 0u;
            bw[k] = Cp[k];
        }
    }
    const int jt = q + 1;  // chunk at which block2 starts
    for (int j = s0 / W; j < s1 / W; j++) {
        const bool snap = (j == jt);
        if (__any_sync(__activemask(), snap)) {
#pragma unroll
            for (int k = 0; k < W; k++) {
                k0[k] = snap ? a0[k] : k0[k];
                k1[k] = snap ? a1[k] : k1[k];
                k2[k] = snap ? a2[k] : k2[k];
            }
        }
        const int ib = (j < jt) ? j * W : (j - 1) * W;
        const uint32_t *Ap = A + phys(ib);
        int xg = (q - j - 1) * W;
        if (xg < 0) xg += M;
        const uint32_t *Cp = C + phys(xg);
        uint32_t av[W], bn[W];
#pragma unroll
        for (int u = 0; u < W; u++) {
            av[u] = Ap[u];
            bn[u] = Cp[W - 1 - u];
        }
#pragma unroll
        for (int u = 0; u < W; u++) {
            if (!SPARSE || av[u] != 0u) {
#pragma unroll
                for (int k = W - 1; k >= 0; k--) mac_cc(av[u], bw[k], a0[k], a1[k], a2[k]);
            }
#pragma unroll
            for (int k = W - 1; k > 0; k--) bw[k] = bw[k - 1];
            bw[0] = bn[u];
        }
    }
    // block1 = saved sums (or all of it when the hand-over lies beyond s1)
    if (jt * W >= s1) {
#pragma unroll
        for (int k = 0; k < W; k++) {
            k0[k] = a0[k];
            k1[k] = a1[k];
            k2[k] = a2[k];
        }
    }
#pragma unroll
    for (int t = 0; t < W + 2; t++) {
        long long x1 = 0, x2 = 0;
        if (t < W) {
            x1 += k0[t];
            x2 += (long long)a0[t] - k0[t];
        }
        if (t >= 1 && t - 1 < W) {
            x1 += k1[t - 1];
            x2 += (long long)a1[t - 1] - k1[t - 1];
        }
        if (t >= 2 && t - 2 < W) {
            x1 += k2[t - 2];
            x2 += (long long)a2[t - 2] - k2[t - 2];
        }
        v1[t] = x1;
        v2[t] = x2;
    }
}

// the unit's contributions added (negated when `neg`) into an int64 column
// window `win` (skewed layout) at column offset `off`
template <bool SPARSE>
__device__ __forceinline__ void mac_unit(const uint32_t *A, const uint32_t *C, int q, int s0,
                                         int s1, int Lp, int M, long long *win, int off, bool neg)
{
    long long v1[W + 2], v2[W + 2];
    mac_unit_vals<SPARSE>(A, C, q, s0, s1, Lp, M, v1, v2);
    const int c1 = off + q * W, c2 = c1 + Lp;
#pragma unroll
    for (int t = 0; t < W + 2; t++) {
        long long x1 = neg ? -v1[t] : v1[t];
        long long x2 = neg ? -v2[t] : v2[t];
        if (x1) atomicAdd((unsigned long long *)&win[wphys(c1 + t)], (unsigned long long)x1);
        if (x2) atomicAdd((unsigned long long *)&win[wphys(c2 + t)], (unsigned long long)x2);
    }
}

// a lone number +-c (staged in A layout): limbs [qW, qW+W) into the window
__device__ __forceinline__ void add_unit(const uint32_t *A, int q, long long *win, int off, bool neg)
{
#pragma unroll
    for (int k = 0; k < W; k++) {
        long long v = A[phys(q * W + k)];
        if (v) atomicAdd((unsigned long long *)&win[wphys(off + q * W + k)],
                         (unsigned long long)(neg ? -v : v));
    }
}

// v * c for a one-limb multiplier v (c staged in A layout): limbs [qW, qW+W)
__device__ __forceinline__ void scaled_unit(uint32_t v, const uint32_t *A, int q, long long *win,
                                            int off, bool neg)
{
    long long lo[W + 1];
#pragma unroll
    for (int k = 0; k <= W; k++) lo[k] = 0;
#pragma unroll
    for (int k = 0; k < W; k++) {
        uint64_t p = (uint64_t)v * A[phys(q * W + k)];
        lo[k] += (long long)(uint32_t)p;
        lo[k + 1] += (long long)(p >> 32);
    }
#pragma unroll
    for (int k = 0; k <= W; k++) {
        long long x = neg ? -lo[k] : lo[k];
        if (x) atomicAdd((unsigned long long *)&win[wphys(off + q * W + k)], (unsigned long long)x);
    }
}

// ------------------------------------------------------------------ close: normalise, divide

struct Norm {
    int neg;
    int top;  // index of the top non-zero digit, -1 for zero
};

// Exact value of Wn int64 columns (sum col[c] 2^(32c), skewed layout in
// shared memory) as sign and magnitude digits.  One warp; lane l owns columns
// [lK, lK+K).  Local carries first, then carries that cross lanes ride up one
// lane per round until none is left (a carry is absorbed or passed on, so 32
// rounds always suffice).
__device__ Norm warp_normalize(const long long *col, uint32_t *dig, int Wn, int *status)
{
    const int lane = threadIdx.x & 31;
    const int K = (Wn + 31) >> 5;
    const int c0 = lane * K;
    const int c1 = min(c0 + K, Wn);
    long long carry = 0;
    for (int c = c0; c < c1; c += 8) {
        long long v[8];
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = (c + k < c1) ? col[wphys(c + k)] : 0;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (c + k < c1) {
                long long t = v[k] + carry;
                dig[c + k] = (uint32_t)t;
                carry = t >> 32;
            }
        }
    }
    long long top = 0;
    bool settled = false;
    for (int round = 0; round < 40; round++) {
        top += __shfl_sync(FULL, carry, 31);
        long long cin = __shfl_up_sync(FULL, carry, 1);
        if (lane == 0) cin = 0;
        if (!__any_sync(FULL, cin != 0)) {
            settled = true;
            break;
        }
        long long c = cin;
        for (int cc = c0; cc < c1 && c != 0; cc++) {
            long long v = (long long)dig[cc] + c;
            dig[cc] = (uint32_t)v;
            c = v >> 32;
        }
        carry = c;
    }
    if (!settled && lane == 0) atomicCAS(status, 0, DEV_INTERNAL);
    Norm r;
    r.neg = top < 0;
    if (r.neg) {
        // |V| = 2^(32 Wn) - D: digits below the lowest non-zero one stay 0,
        // that one becomes 2^32 - d, the ones above are complemented
        int zl = 0x7fffffff;
        for (int c = c1 - 1; c >= c0; c--)
            if (dig[c]) zl = c;
        int z = zl;
        for (int o = 16; o; o >>= 1) z = min(z, __shfl_xor_sync(FULL, z, o));
        for (int c = c0; c < c1; c++) {
            if (c > z) dig[c] = ~dig[c];
            else if (c == z) dig[c] = 0u - dig[c];
        }
    }
    int tl = -1;
    for (int c = c0; c < c1; c++)
        if (dig[c]) tl = c;
    for (int o = 16; o; o >>= 1) tl = max(tl, __shfl_xor_sync(FULL, tl, o));
    r.top = tl;
    __syncwarp();
    return r;
}

// trunc_L(|E| / d) for |E| = sum_c dig[c] 2^(32(base+c)) with top digit t:
// writes L limbs to out and returns the exponent.  Only limbs of |E| at or
// above the quotient's lowest kept position matter,
// floor(|E| / (d 2^(32 s))) = floor(floor(|E| / 2^(32 s)) / d); below the
// window's lowest limb they are zero.  The long division runs on 32 lanes at
// once: each lane's chunk is the affine map r -> (2^(32 len) r + chunk) mod d
// on the running remainder, the maps are composed with a shuffle scan, then
// every lane divides its chunk starting from its incoming remainder.
__device__ long long warp_divide(const uint32_t *dig, int t, long long base, uint32_t d, int L,
                                 uint32_t *out)
{
    const int lane = threadIdx.x & 31;
    const long long T = base + t + 1;
    const long long eq = (dig[t] >= d) ? T : T - 1;
    const long long s = eq - L;
    const int nX = (int)(T - s);
    const int KX = (nX + 31) >> 5;
    const int jhi = min(nX - lane * KX, nX);
    const int jlo = max(jhi - KX, 0);
    auto X = [&](int j) -> uint32_t {
        long long idx = s + j - base;
        return idx >= 0 ? dig[idx] : 0u;
    };
    if (d == 1u) {
        for (int j = jhi - 1; j >= jlo; j--)
            if (j < L) out[j] = X(j);
        __syncwarp();
        return eq;
    }
    const Divisor dv = make_divisor(d);
    uint32_t t32 = 1;
    (void)divstep(t32, 0u, dv);  // 2^32 mod d
    uint32_t V = 0, Pm = 1;
    for (int j = jhi - 1; j >= jlo; j--) {
        (void)divstep(V, X(j), dv);
        Pm = mod_inv(Pm * t32, dv);
    }
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t Po = __shfl_up_sync(FULL, Pm, o);
        uint32_t Vo = __shfl_up_sync(FULL, V, o);
        if (lane >= o) {
            V = mod_inv(Pm * Vo + V, dv);
            Pm = mod_inv(Pm * Po, dv);
        }
    }
    uint32_t r = __shfl_up_sync(FULL, V, 1);
    if (lane == 0) r = 0;
    for (int j = jhi - 1; j >= jlo; j--) {
        uint32_t qd = divstep(r, X(j), dv);
        if (j < L) out[j] = qd;
    }
    __syncwarp();
    return eq;
}

// ------------------------------------------------------------------ async copies

__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src_gmem)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// ------------------------------------------------------------------ flags

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_int(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

}  // namespace mpt
