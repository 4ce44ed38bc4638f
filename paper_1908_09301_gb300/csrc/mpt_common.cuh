// mpt_common.cuh -- device building blocks of the pipelined multiple-precision
// Taylor step (Sec. 2 of Dimova et al., arXiv 1908.09301): exact sums of limb
// products in int64 column windows, carry normalisation, division by a small
// integer with truncation to L limbs.  The block-level routines assume PT
// threads per CTA.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "mpt_divisor.cuh"
#include "mpt_kernel.cuh"

namespace mpt {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NWARPS = PT / 32;

// ------------------------------------------------------------------ operand layout

// Operand vectors in shared memory: limb x sits at gpos(x); every group of
// W = 8 limbs starts on a 48-byte boundary, so a group is two 128-bit loads and
// eight consecutive groups start on eight different 4-bank windows.
constexpr int GS = 12;  // words per limb group
__host__ __device__ __forceinline__ int gpos(int x) { return (x >> 3) * GS + (x & 7); }
// words of a vector of n limbs (n a multiple of W)
__host__ __device__ __forceinline__ int vwords(int n) { return (n >> 3) * GS; }

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

#ifdef __CUDACC__

// ------------------------------------------------------------------ limb products

// One chunk of a unit walk.  A unit q of the product A' * C (A' of M = (P+1)W
// limbs, C of Lp limbs kept as a cyclic vector of period M with zeros at
// [Lp, M)) owns columns qW..qW+W-1 of block 0 and the same columns plus M of
// block 1.  Walking the limbs of A' in chunks of W, chunk j pairs a_{jW+u}
// with c_{(qW + k - jW - u) mod M} in column k; chunks j <= q land in block
// 0 and chunks j > q in block 1 (the limbs that wrap into the zero padding
// between the two contribute nothing, so the split may be made per chunk).
// sA, sC are shared-memory addresses of A' and C; gA = j,
// gC0 = (q - j) mod (P+1), gC1 = (q - j - 1) mod (P+1) are limb groups.
__device__ __forceinline__ uint4 lds128(unsigned addr)
{
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(addr));
    return v;
}
__device__ __forceinline__ void chunk_mac(unsigned sA, unsigned sC, int gA, int gC0, int gC1,
                                          uint32_t (&c0)[W], uint32_t (&c1)[W], uint32_t (&c2)[W])
{
    const unsigned pa = sA + gA * GS * 4, pb = sC + gC0 * GS * 4, pn = sC + gC1 * GS * 4;
    const uint4 a_lo = lds128(pa), a_hi = lds128(pa + 16), b_lo = lds128(pb), b_hi = lds128(pb + 16);
    const uint4 n_lo = lds128(pn), n_hi = lds128(pn + 16);
    const uint32_t av[W] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
    const uint32_t bw[W] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
    const uint32_t bn[W] = {n_lo.x, n_lo.y, n_lo.z, n_lo.w, n_hi.x, n_hi.y, n_hi.z, n_hi.w};
#pragma unroll
    for (int u = 0; u < W; u++) {
#pragma unroll
        for (int k = W - 1; k >= 0; k--) {
            const uint32_t b = (k >= u) ? bw[k - u] : bn[W + k - u];
            mac_cc(av[u], b, c0[k], c1[k], c2[k]);
        }
    }
}
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// int64 digit t (t < W+2) of the 96-bit columns (c0, c1, c2)[k]: the column
// sums as sum_t digit_t 2^(32t)
__device__ __forceinline__ long long col_digit(const uint32_t (&c0)[W], const uint32_t (&c1)[W],
                                               const uint32_t (&c2)[W], int t)
{
    long long v = 0;
    if (t < W) v += c0[t];
    if (t >= 1 && t - 1 < W) v += c1[t - 1];
    if (t >= 2 && t - 2 < W) v += c2[t - 2];
    return v;
}

// ------------------------------------------------------------------ block reductions

__device__ __forceinline__ long long warp_min_ll(long long v)
{
    for (int o = 16; o; o >>= 1) {
        long long w = __shfl_xor_sync(FULL, v, o);
        v = w < v ? w : v;
    }
    return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v)
{
    for (int o = 16; o; o >>= 1) {
        long long w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// block-wide min (max) of v, returned in every thread; red holds >= NWARPS
// long longs; two __syncthreads.
// 32-bit warp min / max: one warp-reduction instruction (sm_80 and later)
__device__ __forceinline__ int warp_min_i(int v)
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
    return __reduce_min_sync(FULL, v);
#else
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
#endif
}
__device__ __forceinline__ int warp_max_i(int v)
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 800
    return __reduce_max_sync(FULL, v);
#else
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
    return v;
#endif
}

__device__ __forceinline__ long long block_min_ll(long long v, long long *red)
{
    v = warp_min_ll(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long r = red[0];
    for (int w = 1; w < NWARPS; w++) r = red[w] < r ? red[w] : r;
    __syncthreads();
    return r;
}
__device__ __forceinline__ long long block_max_ll(long long v, long long *red)
{
    v = warp_max_ll(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    long long r = red[0];
    for (int w = 1; w < NWARPS; w++) r = red[w] > r ? red[w] : r;
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------ close: normalise, divide

struct Norm {
    int neg;
    int top;  // index of the top non-zero digit, -1 for zero
};

// A carry map: the adjustment (-1, 0 or +1) that leaves a thread's digits
// for each adjustment that arrives from below.  Three 2-bit fields (value +
// 1) for arrivals -1, 0, +1.
__device__ __forceinline__ int cmap_apply(int f, int x) { return ((f >> (2 * (x + 1))) & 3) - 1; }
// g after f
__device__ __forceinline__ int cmap_compose(int g, int f)
{
    int r = 0;
#pragma unroll
    for (int x = -1; x <= 1; x++) r |= (cmap_apply(g, cmap_apply(f, x)) + 1) << (2 * (x + 1));
    return r;
}
constexpr int CMAP_ID = (0 << 0) | (1 << 2) | (2 << 4);

// carry out of adding cin to the digits dig[c0..c1) (c1 > c0); in {-1, 0, 1}
// when |cin| < 2^32
__device__ __forceinline__ int carry_through(const uint32_t *dig, int c0, int c1, long long cin)
{
    long long c = cin;
    for (int x = c0; x < c1 && c != 0; x++) {
        const long long v = (long long)dig[x] + c;
        c = v >> 32;
    }
    return (int)c;
}

constexpr int KMAX = 8;      // columns per thread the normalisation keeps in registers
constexpr int RED_LL = 96;   // long longs of scratch the block routines need

// Exact value of Wn int64 columns (sum col[c] 2^(32c), plain layout) as sign
// and magnitude digits dig[0..Wn), Wn <= KK PT.  Thread t owns columns
// [tKK, tKK+KK) and folds them into digits (kept in registers) and a local
// carry (|carry| < 2^31).  The carry of thread t-1 moves thread t's carry out
// by -1, 0 or +1 more, a function of what thread t-1 itself received, so these
// adjustments come from one scan of 3-entry carry maps (within each warp,
// then over the warps in warp 0, which also yields the sign), and are then
// applied.  One merged reduction gives the lowest non-zero digit and the top
// digit.  The magnitude is 2^(32 Wn) - D when the value is negative.  `red`
// holds RED_LL long longs.  Needs |V| < 2^(32 Wn) (else status DEV_INTERNAL).
// The columns read are left zero.
template <int KK>
__device__ Norm block_normalize_k(long long *col, uint32_t *dig, int Wn, long long *red,
                                  int *status)
{
    Norm r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c0 = min(tid * KK, Wn), nk = min(c0 + KK, Wn) - c0;
    uint32_t d[KK];
    long long lc = 0;
#pragma unroll
    for (int k = 0; k < KK; k++) {
        d[k] = 0u;
        if (k < nk) {
            const long long v = col[c0 + k] + lc;
            col[c0 + k] = 0;  // the window is left empty for its next use
            d[k] = (uint32_t)v;
            lc = v >> 32;
        }
    }
    long long *lcw = red;                  // [NWARPS] carries of lane 31
    int *mapw = (int *)(red + NWARPS);     // [NWARPS] warp maps
    int *pre = mapw + NWARPS;              // [NWARPS] maps of all lower warps
    long long *fin = red + 2 * NWARPS;     // [0] top thread's carry, [1] final carry, [2+3w..] z, t0, t1
    long long lprev = __shfl_up_sync(FULL, lc, 1);
    if (lane == 31) lcw[warp] = lc;
    if (nk > 0 && c0 + nk == Wn) fin[0] = lc;
    __syncthreads();
    if (lane == 0) lprev = warp ? lcw[warp - 1] : 0;
    int f = CMAP_ID;
    if (nk > 0) {
        f = 0;
#pragma unroll
        for (int x = -1; x <= 1; x++) {
            long long c = lprev + x;
#pragma unroll
            for (int k = 0; k < KK; k++)
                if (k < nk) c = ((long long)d[k] + c) >> 32;
            f |= ((int)c + 1) << (2 * (x + 1));
        }
    }
    int F = f;  // inclusive scan of maps, lowest thread first
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int G = __shfl_up_sync(FULL, F, o);
        if (lane >= o) F = cmap_compose(F, G);
    }
    if (lane == 31) mapw[warp] = F;
    __syncthreads();
    if (warp == 0) {
        int G = lane < NWARPS ? mapw[lane] : CMAP_ID;
#pragma unroll
        for (int o = 1; o < NWARPS; o <<= 1) {
            const int H = __shfl_up_sync(FULL, G, o);
            if (lane >= o) G = cmap_compose(G, H);
        }
        int E = __shfl_up_sync(FULL, G, 1);
        if (lane == 0) E = CMAP_ID;
        if (lane < NWARPS) pre[lane] = E;
        if (lane == NWARPS - 1) fin[1] = fin[0] + cmap_apply(G, 0);
    }
    __syncthreads();
    int ex = __shfl_up_sync(FULL, F, 1);
    if (lane == 0) ex = CMAP_ID;
    const int din = cmap_apply(cmap_compose(ex, pre[warp]), 0);
    long long cin = lprev + din;
    // column indices (< 2^31): lowest non-zero digit, top non-zero, top non-all-ones
    int z = INT_MAX, t0 = -1, t1 = -1;
#pragma unroll
    for (int k = 0; k < KK; k++) {
        if (k < nk) {
            const long long v = (long long)d[k] + cin;
            d[k] = (uint32_t)v;
            cin = v >> 32;
            dig[c0 + k] = d[k];
            if (d[k]) {
                z = min(z, c0 + k);
                t0 = c0 + k;
            }
            if (d[k] != 0xffffffffu) t1 = c0 + k;
        }
    }
    const long long topc = fin[1];
    z = warp_min_i(z);
    t0 = warp_max_i(t0);
    t1 = warp_max_i(t1);
    if (lane == 0) {
        fin[2 + 3 * warp] = z;
        fin[3 + 3 * warp] = t0;
        fin[4 + 3 * warp] = t1;
    }
    __syncthreads();
    {
        // the warps' values, reduced across lanes (lane w holds warp w's)
        int zz = INT_MAX, a0 = -1, a1 = -1;
        if (lane < NWARPS) {
            zz = (int)fin[2 + 3 * lane];
            a0 = (int)fin[3 + 3 * lane];
            a1 = (int)fin[4 + 3 * lane];
        }
        z = warp_min_i(zz);
        t0 = warp_max_i(a0);
        t1 = warp_max_i(a1);
    }
    if (topc != 0 && topc != -1 && tid == 0) atomicCAS(status, 0, DEV_INTERNAL);
    r.neg = topc < 0;
    r.top = r.neg ? (z == INT_MAX ? -1 : max(t1, z)) : t0;
    if (r.neg) {
        // |V| = 2^(32 Wn) - D: digits below the lowest non-zero one stay 0,
        // that one becomes 2^32 - d, the ones above are complemented
#pragma unroll
        for (int k = 0; k < KK; k++) {
            const int c = c0 + k;
            if (k < nk) {
                if (c > z) dig[c] = ~d[k];
                else if (c == z) dig[c] = 0u - d[k];
            }
        }
        __syncthreads();
    }
    return r;
}

__device__ Norm block_normalize(long long *col, uint32_t *dig, int Wn, long long *red,
                                int *status)
{
    if (Wn <= 0) {
        Norm r;
        r.neg = 0;
        r.top = -1;
        return r;
    }
    if (Wn <= PT) return block_normalize_k<1>(col, dig, Wn, red, status);
    if (Wn <= 2 * PT) return block_normalize_k<2>(col, dig, Wn, red, status);
    if (Wn <= 4 * PT) return block_normalize_k<4>(col, dig, Wn, red, status);
    return block_normalize_k<KMAX>(col, dig, Wn, red, status);
}

// trunc_L(|E| / d) for |E| = sum_c dig[c] 2^(32(base+c)) with top digit t:
// writes L limbs to out and returns the exponent.  Only limbs of |E| at or
// above the quotient's lowest kept position matter,
// floor(|E| / (d 2^(32 s))) = floor(floor(|E| / 2^(32 s)) / d); below the
// window's lowest limb they are zero.  The long division runs on all
// threads: each thread's chunk of digits (the top chunk in thread 0) is the
// affine map r -> (2^(32 len) r + chunk) mod d of the running remainder; the
// maps are composed with a scan within each warp and one over the warps (in
// warp 0), then every thread divides its chunk from its incoming remainder.
// d < 2^16; `red` holds >= 4 NWARPS ints.  Ends with __syncthreads (out is
// complete).  For d = 1 the limbs also go to out2 (when given) in the
// grouped operand layout of the limb products.
__device__ long long block_divide(const uint32_t *dig, int t, long long base, const Divisor &dv,
                                  int L, uint32_t *out, int *red, uint32_t *out2 = nullptr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long T = base + t + 1;
    const uint32_t d = dv.d;
    const long long eq = (dig[t] >= d) ? T : T - 1;
    const long long s = eq - L;
    const int nX = (int)(T - s);  // L or L+1 digits j = 0 .. nX-1, bottom up
    const int KX = (nX + PT - 1) / PT;
    const int jhi = max(nX - tid * KX, 0);  // this thread: digits [jlo, jhi)
    const int jlo = max(jhi - KX, 0);
    auto X = [&](int j) -> uint32_t {
        const long long idx = s + j - base;
        return idx >= 0 ? dig[idx] : 0u;
    };
    if (d == 1u) {
        for (int j = jhi - 1; j >= jlo; j--)
            if (j < L) {
                const uint32_t v = X(j);
                out[j] = v;
                if (out2) out2[gpos(j)] = v;
            }
        __syncthreads();
        return eq;
    }
    uint32_t t32 = 1;
    (void)divstep(t32, 0u, dv);  // 2^32 mod d
    uint32_t V = 0, Pm = 1;
    for (int j = jhi - 1; j >= jlo; j--) {
        (void)divstep(V, X(j), dv);
        Pm = mod_inv(Pm * t32, dv);
    }
    // inclusive scan: (P2, V2) after (P1, V1) = (P2 P1, P2 V1 + V2) mod d
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t Po = __shfl_up_sync(FULL, Pm, o);
        const uint32_t Vo = __shfl_up_sync(FULL, V, o);
        if (lane >= o) {
            V = mod_inv(Pm * Vo + V, dv);
            Pm = mod_inv(Pm * Po, dv);
        }
    }
    int *wP = red, *wV = red + NWARPS, *eV = red + 2 * NWARPS;
    if (lane == 31) {
        wP[warp] = (int)Pm;
        wV[warp] = (int)V;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t GP = lane < NWARPS ? (uint32_t)wP[lane] : 1u;
        uint32_t GV = lane < NWARPS ? (uint32_t)wV[lane] : 0u;
#pragma unroll
        for (int o = 1; o < NWARPS; o <<= 1) {
            const uint32_t Po = __shfl_up_sync(FULL, GP, o);
            const uint32_t Vo = __shfl_up_sync(FULL, GV, o);
            if (lane >= o) {
                GV = mod_inv(GP * Vo + GV, dv);
                GP = mod_inv(GP * Po, dv);
            }
        }
        uint32_t EV = __shfl_up_sync(FULL, GV, 1);  // remainder leaving all lower warps
        if (lane == 0) EV = 0;
        if (lane < NWARPS) eV[lane] = (int)EV;
    }
    __syncthreads();
    const uint32_t rin = (uint32_t)eV[warp];
    uint32_t Pe = __shfl_up_sync(FULL, Pm, 1), Ve = __shfl_up_sync(FULL, V, 1);
    if (lane == 0) {
        Pe = 1;
        Ve = 0;
    }
    uint32_t r = mod_inv(Pe * rin + Ve, dv);
    for (int j = jhi - 1; j >= jlo; j--) {
        const uint32_t qd = divstep(r, X(j), dv);
        if (j < L) out[j] = qd;
    }
    __syncthreads();
    return eq;
}

// Carries into each bit of a binary carry chain over 32 positions: generate
// mask g, propagate mask p (disjoint), carry cin into bit 0; bit 32 of the
// result is the carry out of bit 31.  The carries are those of the integer
// sum (g | p) + g + cin: a generating bit is 1 in both addends, a propagating
// bit in one, a killing bit in neither.
__device__ __forceinline__ unsigned long long chain_carries(unsigned g, unsigned p, unsigned cin)
{
    const unsigned long long A = (unsigned long long)(g | p), B = g;
    return (A + B + cin) ^ A ^ B;
}

// block_normalize for Wn <= PT (one column a thread) with carry lookahead
// instead of a scan of carry maps.  With v_t = d_t + 2^32 h_t (0 <= d_t <
// 2^32), the value is sum (d_t + h_{t-1}) 2^(32 t) + h_top 2^(32 Wn); split
// each h_{t-1} into its positive part p_t and negative part n_t (both below
// 2^31): first S = sum (d_t + p_t) 2^(32 t), a binary carry chain (a column
// generates a carry when d_t + p_t >= 2^32 and propagates one when it is
// 2^32 - 1), then S - sum n_t 2^(32 t), a binary borrow chain (a column
// generates a borrow when its digit of S is below n_t and propagates one when
// equal).  Each chain's carries come from one addition of ballot masks per
// warp, and across the warps from one more on the warps' summaries.  Same
// result and contract as block_normalize; `red` holds RED_LL long longs (ints
// [96, 182) used).
__device__ Norm block_normalize_2(long long *col, uint32_t *dig, int Wn, long long *red, int *status)
{
    Norm r;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int *ri = (int *)red;
    int *sw1 = ri + 150, *sw2 = ri + 166;  // [NWARPS] the warps' summaries of each chain
    long long *ftop = red + 48;            // ints 96, 97: what lies beyond the top column
    int *zt = ri + 100;                    // [3][NWARPS] lowest non-zero, top non-zero, top non-all-ones
    const bool own = tid < Wn;
    const long long v = own ? col[tid] : 0;
    const long long hp = (own && tid > 0) ? (col[tid - 1] >> 32) : 0;
    const uint32_t pp = hp > 0 ? (uint32_t)hp : 0u, np = hp < 0 ? (uint32_t)(-hp) : 0u;
    const unsigned long long u = (unsigned long long)(uint32_t)v + pp;  // below 2^32 + 2^31
    const uint32_t e = (uint32_t)u;
    // the carry chain of S
    const unsigned g1 = __ballot_sync(FULL, own && (u >> 32) != 0);
    const unsigned p1 = __ballot_sync(FULL, own && (u >> 32) == 0 && e == 0xffffffffu);
    if (lane == 0) {
        const int o0 = (int)(chain_carries(g1, p1, 0) >> 32), o1 = (int)(chain_carries(g1, p1, 1) >> 32);
        sw1[warp] = o0 | ((o1 & ~o0) << 1);
    }
    __syncthreads();
    int s = lane < NWARPS ? sw1[lane] : 0;
    unsigned x = (unsigned)(chain_carries(__ballot_sync(FULL, s & 1), __ballot_sync(FULL, s & 2), 0) >> warp) & 1u;
    const unsigned cin = (unsigned)(chain_carries(g1, p1, x) >> lane) & 1u;
    const uint32_t sd = e + cin;  // this column's digit of S
    // the borrow chain of S minus the negative parts
    const unsigned g2 = __ballot_sync(FULL, own && sd < np), p2 = __ballot_sync(FULL, own && sd == np);
    if (lane == 0) {
        const int o0 = (int)(chain_carries(g2, p2, 0) >> 32), o1 = (int)(chain_carries(g2, p2, 1) >> 32);
        sw2[warp] = o0 | ((o1 & ~o0) << 1);
    }
    __syncthreads();
    s = lane < NWARPS ? sw2[lane] : 0;
    x = (unsigned)(chain_carries(__ballot_sync(FULL, s & 1), __ballot_sync(FULL, s & 2), 0) >> warp) & 1u;
    const unsigned bin = (unsigned)(chain_carries(g2, p2, x) >> lane) & 1u;
    uint32_t dd = 0u;
    int z = INT_MAX, t0 = -1, t1 = -1;
    if (own) {
        const long long w = (long long)sd - np - bin;
        dd = (uint32_t)w;
        dig[tid] = dd;
        col[tid] = 0;  // every read of it was before the first barrier
        if (dd) {
            z = tid;
            t0 = tid;
        }
        if (dd != 0xffffffffu) t1 = tid;
        // the top column's own high part, the carry out of S, the borrow out
        if (tid == Wn - 1) *ftop = (v >> 32) + (long long)((u + cin) >> 32) - (w < 0 ? 1 : 0);
    }
    z = warp_min_i(z);
    t0 = warp_max_i(t0);
    t1 = warp_max_i(t1);
    if (lane == 0) {
        zt[warp] = z;
        zt[NWARPS + warp] = t0;
        zt[2 * NWARPS + warp] = t1;
    }
    __syncthreads();
    {
        int zz = INT_MAX, a0 = -1, a1 = -1;
        if (lane < NWARPS) {
            zz = zt[lane];
            a0 = zt[NWARPS + lane];
            a1 = zt[2 * NWARPS + lane];
        }
        z = warp_min_i(zz);
        t0 = warp_max_i(a0);
        t1 = warp_max_i(a1);
    }
    const long long topc = *ftop;
    if (topc != 0 && topc != -1 && tid == 0) atomicCAS(status, 0, DEV_INTERNAL);
    r.neg = topc < 0;
    r.top = r.neg ? (z == INT_MAX ? -1 : max(t1, z)) : t0;
    if (r.neg) {
        if (own) {
            if (tid > z) dig[tid] = ~dd;
            else if (tid == z) dig[tid] = 0u - dd;
        }
        __syncthreads();
    }
    return r;
}

// block_divide when the quotient has at most PT digits (one digit a thread,
// thread 0 the top one), with two barriers: every warp composes the warps'
// remainder maps itself.  Same result and contract as block_divide; `red`
// holds >= 2 NWARPS ints (ints [0, 32) used).
__device__ long long block_divide_1(const uint32_t *dig, int t, long long base, const Divisor &dv, int L,
                                    uint32_t *out, int *red, uint32_t *out2 = nullptr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long T = base + t + 1;
    const uint32_t d = dv.d;
    const long long eq = (dig[t] >= d) ? T : T - 1;
    const long long s = eq - L;
    const int nX = (int)(T - s);  // L or L+1 digits j = 0 .. nX-1, bottom up
    const int j = nX - 1 - tid;   // this thread's digit (j < 0: none)
    uint32_t X = 0u;
    if (j >= 0) {
        const long long idx = s + j - base;
        X = idx >= 0 ? dig[idx] : 0u;
    }
    if (d == 1u) {
        if (j >= 0 && j < L) {
            out[j] = X;
            if (out2) out2[gpos(j)] = X;
        }
        __syncthreads();
        return eq;
    }
    uint32_t t32 = 1;
    (void)divstep(t32, 0u, dv);  // 2^32 mod d
    // this digit's map r -> (2^32 r + X) mod d, identity without a digit
    uint32_t Pm = 1u, V = 0u;
    if (j >= 0) {
        Pm = t32;
        (void)divstep(V, X, dv);
    }
    // inclusive scan: (P2, V2) after (P1, V1) = (P2 P1, P2 V1 + V2) mod d
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t Po = __shfl_up_sync(FULL, Pm, o);
        const uint32_t Vo = __shfl_up_sync(FULL, V, o);
        if (lane >= o) {
            V = mod_inv(Pm * Vo + V, dv);
            Pm = mod_inv(Pm * Po, dv);
        }
    }
    int *wP = red, *wV = red + NWARPS;
    if (lane == 31) {
        wP[warp] = (int)Pm;
        wV[warp] = (int)V;
    }
    __syncthreads();
    uint32_t GP = lane < NWARPS ? (uint32_t)wP[lane] : 1u;
    uint32_t GV = lane < NWARPS ? (uint32_t)wV[lane] : 0u;
#pragma unroll
    for (int o = 1; o < NWARPS; o <<= 1) {
        const uint32_t Po = __shfl_up_sync(FULL, GP, o);
        const uint32_t Vo = __shfl_up_sync(FULL, GV, o);
        if (lane >= o) {
            GV = mod_inv(GP * Vo + GV, dv);
            GP = mod_inv(GP * Po, dv);
        }
    }
    uint32_t rin = __shfl_sync(FULL, GV, (warp + 31) & 31);  // the remainder leaving the warps above
    if (warp == 0) rin = 0u;
    uint32_t Pe = __shfl_up_sync(FULL, Pm, 1), Ve = __shfl_up_sync(FULL, V, 1);
    if (lane == 0) {
        Pe = 1u;
        Ve = 0u;
    }
    uint32_t rr = mod_inv(Pe * rin + Ve, dv);
    if (j >= 0) {
        const uint32_t qd = divstep(rr, X, dv);
        if (j < L) out[j] = qd;
    }
    __syncthreads();
    return eq;
}

// block_divide when the quotient has at most PT digits and d = d' 2^a > 1
// (d' odd), without a scan of remainder maps: with Y = floor(E / 2^a) (so
// floor(E / d) = floor(Y / d')), the remainder mod d' entering quotient digit
// j from the digits above it is W_{i-1} (sum over the higher digits i' < i of
// (Y_{i'} mod d') U_{i'}) mod d', where i counts digits from the top (thread
// i holds the digit with index i from the top), W_i = 2^(32 i) mod d' and U_i
// = 2^(-32 i) mod d' (2 is invertible mod an odd d').  The sum is a prefix
// sum of integers below 2^16, then every thread divides its digit.  ent is
// this thread's U_i | W_{i-1} << 16; dvo divides by d'.  Same result and
// contract as block_divide (d > 1); `red` holds >= NWARPS ints (ints [0, 16)).
__device__ long long block_divide_2(const uint32_t *dig, int t, long long base, uint32_t d, int a,
                                    const Divisor &dvo, int L, uint32_t *out, int *red, uint32_t ent)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long T = base + t + 1;
    const long long eq = (dig[t] >= d) ? T : T - 1;
    const long long s = eq - L;
    const int nX = (int)(T - s);  // L or L+1 digits j = 0 .. nX-1, bottom up
    const int j = nX - 1 - tid;   // this thread's digit (j < 0: none)
    uint32_t Y = 0u, term = 0u;
    if (j >= 0) {
        const long long idx = s + j - base;
        const uint32_t x0 = idx >= 0 ? dig[idx] : 0u;
        const uint32_t x1 = (j + 1 < nX && idx + 1 >= 0) ? dig[idx + 1] : 0u;
        Y = a ? ((x0 >> a) | (x1 << (32 - a))) : x0;
        term = mod_inv(mod_inv(Y, dvo) * (ent & 0xffffu), dvo);
    }
    uint32_t P = term;  // inclusive prefix sum from the top digit
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t q = __shfl_up_sync(FULL, P, o);
        if (lane >= o) P += q;
    }
    if (lane == 31) red[warp] = (int)P;
    __syncthreads();
    uint32_t above = 0u;
#pragma unroll
    for (int w = 0; w < NWARPS; w++)
        if (w < warp) above += (uint32_t)red[w];
    const uint32_t E = P - term + above;  // the higher digits' sum
    uint32_t r = tid == 0 ? 0u : mod_inv(mod_inv(E, dvo) * (ent >> 16), dvo);
    if (j >= 0) {
        const uint32_t qd = divstep(r, Y, dvo);
        if (j < L) out[j] = qd;
    }
    __syncthreads();
    return eq;
}

// ------------------------------------------------------------------ async copies

__device__ __forceinline__ void cp_async4(uint32_t *dst_smem, const uint32_t *src_gmem)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst_smem, const void *src_gmem)
{
    unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ flags

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned *p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_int(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

#endif  // __CUDACC__

}  // namespace mpt
