// mpt_pipe.cu -- pipelined multiple-precision Taylor step (Sec. 2 of Dimova
// et al., arXiv 1908.09301) for large L x N: one persistent cooperative
// launch, one CTA per SM, four roles.  Eq. (3)'s Cauchy sums of index m,
//     sum_{a=0}^{m} alpha_a gamma_{m-a},  sum_{a=0}^{m} alpha_a beta_{m-a},
// are split by the newest coefficient they need, so that each part starts as
// early as it can:
//
//  * Workers (CTAs 10 and up) take the middle pairs a = 2..m-2, which need
//    coefficients up to m-2 only, so they run while the bracket CTAs are
//    still finishing coefficients m-1 and m.  A worker takes a contiguous
//    range of one target's m-3 terms.  All of its terms are summed in one
//    frame: a term whose lowest limb lies d = 8 d_hi + d_lo limbs above the
//    window base has its first factor staged shifted up by d_lo limbs (and
//    complemented when the term is negative; the complement's correction is
//    added separately), so the terms with equal d_hi share columns and are
//    accumulated in the same registers.  Two warps of a worker (control)
//    wait, load, stage and flush while the other fourteen (compute) run the
//    products.
//  * The outer-pair CTAs 3 (beta') and 4 (gamma') take the pairs a = 1 and
//    a = m-1 as soon as coefficient m-1 is out.
//  * The edge CTAs 5..9 take the terms with coefficient m itself (the pairs
//    a = 0 and a = m, and products with a parameter of more than one limb,
//    such as b gamma_m), one term each, as soon as coefficient m is out.
//  * The bracket CTAs 0, 1, 2 own Eq. (3)'s brackets alpha', beta', gamma'.
//    Each adds its one-limb and lone terms and the other CTAs' sums,
//    normalises, divides by (m+1) and publishes its component of coefficient
//    m+1; the three exchange components through global memory.  After index
//    N-1 each runs the Horner chain of Eq. (2) for its component,
//    h_i = trunc_L(tau h_{i+1} + c_i).
//
// The non-bracket CTAs add their windows into a global window set (one part
// per kind) and count themselves done.
//
// Limb products use units: unit q of a product A' * C (A' of M = (P+1)W
// limbs, C of Lp limbs) owns columns qW..qW+W-1 of two blocks (block 1 is M
// columns up); a group of RS lanes of one warp shares a unit: lane r first
// takes chunk r of every term, then a contiguous share of the chunks RS..P
// of all terms, so the chunks a lane meets only increase and it switches
// blocks at most once.  The lanes' sums are combined by a reduce-scatter
// within the lane group, then added into the window one column per thread.
//
// Hand-over: a monotone "published" counter (release/acquire, 3 per
// coefficient) and per-set monotone completion counters; every wait is
// bounded and ends the launch with a status code when it expires.  Integer
// sums are exact and associative, so the result does not depend on the split.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "mpt_common.cuh"
#include "mpt_kernel.cuh"

namespace mpt {
namespace {

constexpr int NCL = 3;           // bracket CTAs
constexpr int NOUT = 2;          // outer-pair CTAs (one per target: beta', gamma')
constexpr int NEDGE = 5;         // edge CTAs (products with the newest coefficient)
constexpr int NFIX = NCL + NOUT + NEDGE;  // CTAs with fixed roles; workers follow
constexpr int NA = 2;            // A' slots of a bracket / edge CTA (Horner's h: slot 0)
constexpr int NC = 2;            // C slots (tau: slot 0)
constexpr int GIN_PARTS = 3;     // parts of a bracket's global window: middle, outer, edge
constexpr int TI = 8;            // ints of term info per slot
constexpr int TB_MAX = 32;       // worker slots per batch (one warp finds the groups)
// a worker CTA's two groups: control warps (waits, loads, staging, flushes)
// and compute warps (products), handing batches over through two buffers
constexpr int CW = 2;            // control warps
constexpr int CT = 32 * CW;      // control threads
constexpr int KT = PT - CT;      // compute threads
// named barriers: FULL + b (a batch in buffer b is ready), EMPTY + b (the
// compute group is through buffer b), the compute group's, the control group's
enum { BAR_FULL = 1, BAR_EMPTY = 3, BAR_KT = 5, BAR_CT = 6 };
// batch descriptor: exit flag, term groups, window parity, group starts and ends,
// the window column below which each target's sums are left out (shortened
// products; INT_MIN / 2: none)
enum { DS_EXIT = 0, DS_NRUN = 1, DS_PAR = 2, DS_RUN = 4, DS_RUNE = 4 + TB_MAX, DS_CUT = 4 + 2 * TB_MAX,
       DESC_INTS = 6 + 2 * TB_MAX };
constexpr int NO_CUT = INT_MIN / 2;

enum { P_SIGMA = 0, P_R = 1, P_B = 2, P_TAU = 3 };

enum {
    MS_STATUS = 0,  // CTA-uniform copy of the status word
    MS_NRUN = 1,    // bracket and Horner close: flags of the buffer digits of a shortened sum
    MS_NEWE = 2,    // [2] exponent and flags of this CTA's newest number
    MS_PSCAL = 8,   // [3][2] sigma, R, b: single non-zero limb index (or -1), value
    MS_WLO = 16,    // [4] long long window bases (ints 16..23)
    MS_WID = 24,    // [2][2] window widths by parity and target (workers); bracket CTAs:
                    // [4] long long workers-window table of the next index (ints 24..31, MS_IMID)
    MS_CUT = 28,    // [2][2] workers: window column of the cut by parity and target (NO_CUT: none)
    MS_IMID = 24,
    MS_BK = 32,     // [48] bracket setup (ints 32..79)
    MS_RED = 80,    // [RED_LL] long long scratch of the block routines (ints 80..271)
    MS_PARX = 272,  // [4][2] exponent and flags of sigma, R, b, tau (ints 272..279)
    MS_PROF = 336,  // [PROF_SLOTS] long long (ints 336..367)
    MS_CHUNKS = 368,  // long long: limb-product chunks this CTA executed
    MS_KDONE = 372,   // workers: batches the compute group is through (written by its thread 0)
    MISC_INTS = 376
};

// bracket setup (ints at MS_BK): lo (long long), width, simple parts, terms, the workers' sums
enum {
    BK_LO = 0,      // long long (2 ints)
    BK_WIDTH = 2,
    BK_NSIMPLE = 3,
    BK_SIMPLE = 4,  // [2][4]: kind (1 lone, 2 scaled), neg, offset, component
    BK_SV = 12,     // [2] scaled: the parameter's limb
    BK_INNER = 14,  // offset of the workers' sums (or -1)
    BK_IWIDTH = 15,
    BK_EINNER = 16, // offset of the edge-term sums (or -1)
    BK_EWIDTH = 17,
    BK_CUT = 18,    // long long (2 ints): the highest cut of the shortened parts, LLONG_MIN: none
    BK_OINNER = 28, // offset of the outer-pair sums (or -1)
    BK_OWIDTH = 29,
};

// Geometry of the unit walk (host and device)
struct Geo {
    int L, Lp, P, P1, M, VW, RS, RSW, WW, GW, N1;
    __host__ __device__ Geo(int L_, int Lp_, int N, int Wcap)
    {
        L = L_;
        Lp = Lp_;
        P = Lp / W;
        P1 = P + 1;
        M = P1 * W;
        VW = vwords(M);
        // lanes per unit of the few-term products (brackets, Horner) and of
        // the workers' batches: powers of two, units within warps
        RS = 8;
        while (RS > 2 && RS * P1 > PT) RS >>= 1;
        RSW = 16;
        while (RSW > 2 && RSW * P1 > KT) RSW >>= 1;
        WW = Wcap + 4 * W;
        GW = 2 * M + 2;
        N1 = N + 1;
    }
};

struct PSmem {
    int *expT, *flgT;  // [3][N+1]
    int *misc;         // [MISC_INTS]
    int *tinfo;        // [2][TB_MAX][TI] term info (by buffer)
    int *desc;         // [2][DESC_INTS] batch descriptors (workers)
    long long *win;    // [4][WW] windows (workers: by parity and target)
    uint32_t *dig;     // [WW] normalised digits
    // workers
    long long *stage;  // [P1 2][W+2] unit digit sums
    uint32_t *araw;    // [TB][Lp] first factors as loaded
    uint32_t *cc;      // [2][TB][VW] second factors (cyclic, zero above Lp)
    uint32_t *ash;     // [2][TB][VW] first factors shifted / complemented
    long long *cstage; // [KT][W+2] digit sums of one chunk each (shortened products)
    // bracket CTAs (same bytes as the workers' part)
    long long *bstage; // [P1 2][W+2] unit digit sums of the few-term products
    uint32_t *vA;      // [NA][VW]
    uint32_t *vC;      // [NC][VW]
    uint32_t *raw;     // [3][Lp] limbs of the current coefficient; [2] also Horner's h
    uint32_t *newc;    // [Lp] this CTA's newest number
    long long *bcstage;  // [PT][W+2] digit sums of one chunk each (shortened products)
    Divisor *divT;       // [N+1] bracket CTAs: the invariant divisors of 1..N+1 (entry m: m+1)
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t pipe_layout(const Geo &G, int N, int TB, PSmem *S,
                                              unsigned char *base)
{
    size_t o = 0;
    auto take = [&](size_t bytes) -> unsigned char * {
        size_t at = o;
        o = al16(o + bytes);
        return base ? base + at : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(int) * 3 * (N + 1));
    if (S) S->expT = (int *)p;
    p = take(sizeof(int) * 3 * (N + 1));
    if (S) S->flgT = (int *)p;
    p = take(sizeof(int) * MISC_INTS);
    if (S) S->misc = (int *)p;
    p = take(sizeof(int) * 2 * TB_MAX * TI);
    if (S) S->tinfo = (int *)p;
    p = take(sizeof(int) * 2 * DESC_INTS);
    if (S) S->desc = (int *)p;
    p = take(sizeof(long long) * 4 * (size_t)G.WW);
    if (S) S->win = (long long *)p;
    p = take(sizeof(uint32_t) * (size_t)G.WW);
    if (S) S->dig = (uint32_t *)p;
    const size_t u0 = o;
    p = take(sizeof(long long) * (size_t)G.P1 * 2 * (W + 2));
    if (S) S->stage = (long long *)p;
    p = take(sizeof(uint32_t) * (size_t)TB * G.Lp);
    if (S) S->araw = (uint32_t *)p;
    p = take(sizeof(uint32_t) * 2 * (size_t)TB * G.VW);
    if (S) S->cc = (uint32_t *)p;
    p = take(sizeof(uint32_t) * 2 * (size_t)TB * G.VW);
    if (S) S->ash = (uint32_t *)p;
    p = take(sizeof(long long) * (size_t)KT * (W + 2));
    if (S) S->cstage = (long long *)p;
    const size_t worker_end = o;
    o = u0;
    p = take(sizeof(long long) * (size_t)G.P1 * 2 * (W + 2));
    if (S) S->bstage = (long long *)p;
    p = take(sizeof(uint32_t) * NA * (size_t)G.VW);
    if (S) S->vA = (uint32_t *)p;
    p = take(sizeof(uint32_t) * NC * (size_t)G.VW);
    if (S) S->vC = (uint32_t *)p;
    p = take(sizeof(uint32_t) * 3 * (size_t)G.Lp);
    if (S) S->raw = (uint32_t *)p;
    p = take(sizeof(uint32_t) * (size_t)G.Lp);
    if (S) S->newc = (uint32_t *)p;
    p = take(sizeof(long long) * (size_t)PT * (W + 2));
    if (S) S->bcstage = (long long *)p;
    p = take(sizeof(Divisor) * (size_t)(N + 1));
    if (S) S->divT = (Divisor *)p;
    if (worker_end > o) o = worker_end;
    return o;
}

__device__ __forceinline__ long long &ll_at(int *misc, int slot) { return ((long long *)(misc + slot))[0]; }

// Per-phase cycle counters of one thread (`who`) of a CTA, accumulated in
// shared memory and written out at the end.
struct Prof {
    long long *p;
    long long t;
    __device__ Prof(const KArgs &a, bool on, int *misc, int who = 0)
    {
        p = nullptr;
        t = 0;
        if (a.prof && on && threadIdx.x == (unsigned)who) {
            p = (long long *)(misc + MS_PROF);
            t = clock64();
        }
    }
    __device__ __forceinline__ void mark(int slot)
    {
        if (p) {
            long long n = clock64();
            p[slot] += n - t;
            t = n;
        }
    }
};

// Per-index timeline (profiling only): global-timer stamp of index m of the
// launch's last step, set (tl_put) or raised to the latest of several CTAs
// (tl_max).
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void tl_put(const KArgs &a, int row, int m, long long step)
{
    if (a.timeline && step == a.nsteps - 1) a.timeline[(size_t)row * (MAX_N + 1) + m] = (long long)global_ns();
}
__device__ __forceinline__ void tl_max(const KArgs &a, int row, int m, long long step)
{
    if (a.timeline && step == a.nsteps - 1)
        atomicMax((unsigned long long *)&a.timeline[(size_t)row * (MAX_N + 1) + m], global_ns());
}

// One poll of a flag: the status word and the flag, both loads in flight
// together (the status load is issued first: an acquire load holds back only
// the memory operations that follow it).
__device__ __forceinline__ unsigned poll_flag(const unsigned *flag, const int *status, int &st, bool acquire)
{
    st = ld_relaxed_int(status);
    return acquire ? ld_acquire_u32(flag) : ld_relaxed_u32(flag);
}

// bounded wait (thread 0) until *flag >= target, the status word read with
// every poll; returns the status (0: go on).  Acquire on the flag.
__device__ __forceinline__ int poll_geq(const KArgs &a, const unsigned *flag, unsigned target)
{
    long long it = 0;
    for (;;) {
        int st;
        const unsigned v = poll_flag(flag, a.status, st, true);
        if (st) return st;
        if ((int)(v - target) >= 0) return 0;
        if (++it > a.spin_limit) {
            atomicCAS(a.status, 0, DEV_TIMEOUT);
            return DEV_TIMEOUT;
        }
        __nanosleep(20);
    }
}

// bounded wait until *flag >= target (thread 0), the status word checked on
// the way.  Returns false (CTA-uniform) when the launch must stop.
__device__ bool wait_geq(PSmem &S, const KArgs &a, const unsigned *flag, unsigned target)
{
    if (threadIdx.x == 0) S.misc[MS_STATUS] = poll_geq(a, flag, target);
    __syncthreads();
    return S.misc[MS_STATUS] == 0;
}

// ------------------------------------------------------------------ unit products

// The walk of lane r (of RS = 2^LOG) of unit q over the n terms in slots
// [s0, s0+n), in two phases: first chunk j = r of every term (a fixed chunk,
// so only the slot advances), then a contiguous share of the remaining
// chunks RS..P of all terms, chunk-major.  The chunks a lane meets only
// increase, so its block-0 part (chunks j <= q) is complete before its first
// chunk j > q; x keeps that part, a the whole sum.
template <int LOG>
__device__ __forceinline__ void unit_walk(const Geo &G, const uint32_t *Abase, const uint32_t *Cbase,
                                          int s0, int n, int q, int r, uint32_t (&a0)[W],
                                          uint32_t (&a1)[W], uint32_t (&a2)[W], uint32_t (&x0)[W],
                                          uint32_t (&x1)[W], uint32_t (&x2)[W])
{
    constexpr int RS = 1 << LOG;
    const unsigned slot = G.VW * 4;
    const unsigned sAb = smem_addr(Abase), sCb = smem_addr(Cbase);
    bool snap = false;  // x holds the block-0 part
    if (r <= G.P) {
        const int j = r;
        if (j > q) snap = true;  // all of this lane's chunks are in block 1: x stays 0
        int gc0 = q - j;
        if (gc0 < 0) gc0 += G.P1;
        const int gc1 = gc0 == 0 ? G.P : gc0 - 1;
        unsigned sA = sAb + s0 * slot, sC = sCb + s0 * slot;
        for (int t = 0; t < n; t++) {
            chunk_mac(sA, sC, j, gc0, gc1, a0, a1, a2);
            sA += slot;
            sC += slot;
        }
    }
    const int J2 = G.P1 - RS;
    if (J2 > 0) {
        const int I = J2 * n, i0 = I * r / RS, i1 = I * (r + 1) / RS;
        const int jj = i0 / n;
        int t = i0 - jj * n, j = RS + jj;
        for (int it = i0; it < i1; it++) {
            const bool sw = !snap && j > q;  // first chunk of block 1: keep block 0
            if (__any_sync(__activemask(), sw)) {
#pragma unroll
                for (int k = 0; k < W; k++) {
                    x0[k] = sw ? a0[k] : x0[k];
                    x1[k] = sw ? a1[k] : x1[k];
                    x2[k] = sw ? a2[k] : x2[k];
                }
            }
            snap = snap || sw;
            int gc0 = q - j;
            if (gc0 < 0) gc0 += G.P1;
            const int gc1 = gc0 == 0 ? G.P : gc0 - 1;
            const unsigned off = (unsigned)(s0 + t) * slot;
            chunk_mac(sAb + off, sCb + off, j, gc0, gc1, a0, a1, a2);
            t++;
            const bool wrap = t == n;
            t = wrap ? 0 : t;
            j += wrap ? 1 : 0;
        }
    }
    if (!snap) {
#pragma unroll
        for (int k = 0; k < W; k++) {
            x0[k] = a0[k];
            x1[k] = a1[k];
            x2[k] = a2[k];
        }
    }
}

// A thread group of the CTA: the whole CTA (bar 0, __syncthreads) or a set of
// whole warps synchronised by named barrier `bar`; t is the thread's index in
// the group, n the group's size.
struct Grp {
    int t, n, bar;
};
__device__ __forceinline__ void named_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void named_arrive(int id, int n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void grp_sync(const Grp &g)
{
    if (g.bar == 0) __syncthreads();
    else named_sync(g.bar, g.n);
}
__device__ __forceinline__ Grp whole_cta() { return Grp{(int)threadIdx.x, PT, 0}; }

// Reduce-scatter of NV values over the 2^LOG lanes r = 0.. of an aligned lane
// group: lane r ends with NV >> LOG sums, of the values base .. base +
// (NV >> LOG) - 1; returns base.  Each step swaps half of the values with
// the partner lane (xor offset) and keeps the other half.
template <int NV, int LOG>
__device__ __forceinline__ int reduce_scatter(long long (&v)[NV], int r)
{
    int base = 0;
#pragma unroll
    for (int k = 0; k < LOG; k++) {
        const int o = 1 << (LOG - 1 - k);
        const int half = NV >> (k + 1);
        const bool up = (r & o) != 0;  // keep the upper half
#pragma unroll
        for (int i = 0; i < NV / 2; i++) {
            if (i < half) {
                const long long send = up ? v[i] : v[half + i];
                const long long keep = up ? v[half + i] : v[i];
                v[i] = keep + __shfl_xor_sync(FULL, send, o);
            }
        }
        base += up ? half : 0;
    }
    return base;
}

// Sum over the n terms in slots [s0, s0+n) of A'_s * C_s (A'_s = Abase + s VW,
// C_s = Cbase + s VW), exact, added into win[coff + c], c < 2M+2.  With
// `tinfo`, slots flagged negative hold the complement of the shifted first
// factor over its Lp limbs, and the complement's correction
// (+C 2^(32 d) + ~C 2^(32 (d+Lp)) + 2^(32 (d+Lp)) - 2^(32 (d+2Lp))) is added
// as well.  neg_all negates the whole sum.  Every thread of group g calls
// this (its first thread is a warp's first).  RS = 2^LOG threads share a
// unit (RS (P+1) <= g.n), always
// inside one warp, so their shares are combined by a reduce-scatter of the
// unit's 2 (W+2) digits (block 0, block 1) and each lane stores its part;
// then one thread per window column adds the column (with the complement
// corrections).  Only the first RS (P+1) threads walk.  `stage` holds
// (P+1) 2 (W+2) long longs.  Starts and ends with a barrier of the group.
template <int LOG>
__device__ void small_products_t(const Geo &G, const Grp &gr, const uint32_t *Abase,
                                 const uint32_t *Cbase, int s0, int n, const int *tinfo,
                                 bool neg_all, long long *stage, long long *win, int coff)
{
    constexpr int ND = W + 2;
    constexpr int RS = 1 << LOG;
    constexpr int NV = ((2 * ND + RS - 1) / RS) * RS;  // the digits, padded to a multiple of RS
    const int tid = gr.t;
    grp_sync(gr);
    if (tid < ((G.P1 * RS + 31) & ~31) && n > 0) {
        uint32_t a0[W], a1[W], a2[W], x0[W], x1[W], x2[W];
#pragma unroll
        for (int k = 0; k < W; k++) a0[k] = a1[k] = a2[k] = x0[k] = x1[k] = x2[k] = 0u;
        const int q = tid >> LOG, r = tid & (RS - 1);
        if (q < G.P1) unit_walk<LOG>(G, Abase, Cbase, s0, n, q, r, a0, a1, a2, x0, x1, x2);
        long long v[NV];
#pragma unroll
        for (int t = 0; t < ND; t++) {
            const long long bx = col_digit(x0, x1, x2, t), ba = col_digit(a0, a1, a2, t);
            v[t] = bx;
            v[ND + t] = ba - bx;
        }
#pragma unroll
        for (int t = 2 * ND; t < NV; t++) v[t] = 0;
        const int base = reduce_scatter<NV, LOG>(v, r);
        if (q < G.P1) {
            long long *d = stage + (size_t)q * 2 * ND;
#pragma unroll
            for (int i = 0; i < NV / RS; i++)
                if (base + i < 2 * ND) d[base + i] = v[i];
        }
    }
    grp_sync(gr);
    if (n > 0) {
        for (int c = tid; c < G.GW; c += gr.n) {
            long long s = 0;
            if (c < G.M + 2) {
                const int u = c / W;
                if (u <= G.P) s += stage[(u * 2) * ND + c - u * W];
                if (u >= 1 && c - (u - 1) * W < ND) s += stage[((u - 1) * 2) * ND + c - (u - 1) * W];
            }
            const int c1 = c - G.M;
            if (c1 >= 0) {
                const int u = c1 / W;
                if (u <= G.P) s += stage[(u * 2 + 1) * ND + c1 - u * W];
                if (u >= 1 && c1 - (u - 1) * W < ND) s += stage[((u - 1) * 2 + 1) * ND + c1 - (u - 1) * W];
            }
            if (tinfo) {
                for (int sl = s0; sl < s0 + n; sl++) {
                    const int *ti = tinfo + sl * TI;
                    if (!ti[1]) continue;
                    const int y = c - ti[2];
                    const uint32_t *Cs = Cbase + (size_t)sl * G.VW;
                    if (y >= 0 && y < G.Lp) s += Cs[gpos(y)];
                    else if (y >= G.Lp && y < 2 * G.Lp) s += (uint32_t)~Cs[gpos(y - G.Lp)];
                    if (y == G.Lp) s += 1;
                    if (y == 2 * G.Lp) s -= 1;
                }
            }
            if (s) win[coff + c] += neg_all ? -s : s;
        }
    }
    grp_sync(gr);
}

// One product A'_s0 * C_s0 (a Horner step, an edge term) with the same
// result as small_products(n = 1), on the whole CTA, RS = 2^LOG lanes per
// unit: lane r of unit q takes the chunks j = r, r + RS, ... (increasing, so
// the block-0 part is complete before the first chunk j > q), at most NJ of
// them (NJ RS >= P+1), in one fully unrolled sequence, with none of the
// general walk's bookkeeping.
template <int LOG, int NJ>
__device__ void single_product_t(const Geo &G, const uint32_t *Abase, const uint32_t *Cbase, int s0,
                                 const int *tinfo, bool neg_all, long long *stage, long long *win,
                                 int coff)
{
    constexpr int ND = W + 2;
    constexpr int RS = 1 << LOG;
    constexpr int NV = ((2 * ND + RS - 1) / RS) * RS;
    const int tid = threadIdx.x;
    __syncthreads();
    if (tid < ((G.P1 * RS + 31) & ~31)) {
        uint32_t a0[W], a1[W], a2[W], x0[W], x1[W], x2[W];
#pragma unroll
        for (int k = 0; k < W; k++) a0[k] = a1[k] = a2[k] = x0[k] = x1[k] = x2[k] = 0u;
        const int q = tid >> LOG, r = tid & (RS - 1);
        const unsigned slot = G.VW * 4;
        const unsigned sA = smem_addr(Abase) + s0 * slot, sC = smem_addr(Cbase) + s0 * slot;
        if (q < G.P1) {
#pragma unroll
            for (int k = 0; k < NJ; k++) {
                const int j = r + k * RS;
                if (j <= G.P) {
                    if (j > q && j - RS <= q) {  // first chunk of block 1: keep block 0
#pragma unroll
                        for (int u = 0; u < W; u++) {
                            x0[u] = a0[u];
                            x1[u] = a1[u];
                            x2[u] = a2[u];
                        }
                    }
                    int gc0 = q - j;
                    if (gc0 < 0) gc0 += G.P1;
                    const int gc1 = gc0 == 0 ? G.P : gc0 - 1;
                    chunk_mac(sA, sC, j, gc0, gc1, a0, a1, a2);
                }
            }
            if (r + ((G.P - r) / RS) * RS <= q) {  // the lane's last chunk is in block 0
#pragma unroll
                for (int u = 0; u < W; u++) {
                    x0[u] = a0[u];
                    x1[u] = a1[u];
                    x2[u] = a2[u];
                }
            }
        }
        long long v[NV];
#pragma unroll
        for (int t = 0; t < ND; t++) {
            const long long bx = col_digit(x0, x1, x2, t), ba = col_digit(a0, a1, a2, t);
            v[t] = bx;
            v[ND + t] = ba - bx;
        }
#pragma unroll
        for (int t = 2 * ND; t < NV; t++) v[t] = 0;
        const int base = reduce_scatter<NV, LOG>(v, r);
        if (q < G.P1) {
            long long *d = stage + (size_t)q * 2 * ND;
#pragma unroll
            for (int i = 0; i < NV / RS; i++)
                if (base + i < 2 * ND) d[base + i] = v[i];
        }
    }
    __syncthreads();
    for (int c = tid; c < G.GW; c += PT) {
        long long s = 0;
        if (c < G.M + 2) {
            const int u = c / W;
            if (u <= G.P) s += stage[(u * 2) * ND + c - u * W];
            if (u >= 1 && c - (u - 1) * W < ND) s += stage[((u - 1) * 2) * ND + c - (u - 1) * W];
        }
        const int c1 = c - G.M;
        if (c1 >= 0) {
            const int u = c1 / W;
            if (u <= G.P) s += stage[(u * 2 + 1) * ND + c1 - u * W];
            if (u >= 1 && c1 - (u - 1) * W < ND) s += stage[((u - 1) * 2 + 1) * ND + c1 - (u - 1) * W];
        }
        if (tinfo && tinfo[s0 * TI + 1]) {  // complement correction of a negative term
            const int y = c - tinfo[s0 * TI + 2];
            const uint32_t *Cs = Cbase + (size_t)s0 * G.VW;
            if (y >= 0 && y < G.Lp) s += Cs[gpos(y)];
            else if (y >= G.Lp && y < 2 * G.Lp) s += (uint32_t)~Cs[gpos(y - G.Lp)];
            if (y == G.Lp) s += 1;
            if (y == 2 * G.Lp) s -= 1;
        }
        if (s) win[coff + c] += neg_all ? -s : s;
    }
    __syncthreads();
}

__device__ void small_products(const Geo &G, int RS, const Grp &gr, const uint32_t *Abase,
                               const uint32_t *Cbase, int s0, int n, const int *tinfo, bool neg_all,
                               long long *stage, long long *win, int coff);

// one variant (8 lanes, at most 4 chunks a lane: Lp <= 248), the general
// walk otherwise
__device__ void single_product(const Geo &G, const uint32_t *Abase, const uint32_t *Cbase, int s0,
                               const int *tinfo, bool neg_all, long long *stage, long long *win,
                               int coff)
{
    if (G.RS == 8 && G.P1 <= 32)
        single_product_t<3, 4>(G, Abase, Cbase, s0, tinfo, neg_all, stage, win, coff);
    else
        small_products(G, G.RS, whole_cta(), Abase, Cbase, s0, 1, tinfo, neg_all, stage, win, coff);
}

// RS threads per unit: a power of two from 2 to 16 with RS (P+1) <= gr.n
__device__ void small_products(const Geo &G, int RS, const Grp &gr, const uint32_t *Abase,
                               const uint32_t *Cbase, int s0, int n, const int *tinfo, bool neg_all,
                               long long *stage, long long *win, int coff)
{
    switch (RS) {
    case 16: small_products_t<4>(G, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, win, coff); break;
    case 8: small_products_t<3>(G, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, win, coff); break;
    case 4: small_products_t<2>(G, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, win, coff); break;
    default: small_products_t<1>(G, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, win, coff); break;
    }
}

// ------------------------------------------------------------------ shortened products

// largest q with q (q + 1) / 2 <= x (x < 2^24)
__device__ __forceinline__ int tri_root(int x)
{
    int q = (int)((sqrtf(8.0f * (float)x + 1.0f) - 1.0f) * 0.5f);
    while ((q + 1) * (q + 2) / 2 <= x) q++;
    while (q > 0 && q * (q + 1) / 2 > x) q--;
    return q;
}

// Window-relative column below which a part of a bracket (products only,
// window [lo, hi) with hi = its largest term top + 2Lp + 2 - 2L) leaves its
// columns out: c0 = T - L - 3 - CUT_GUARD with T the largest term top
// e_a + e_b; NO_CUT when the launch is exact or no block-0 unit of the
// part's lowest term would fall below c0.
__device__ __forceinline__ int part_cut(const KArgs &a, const Geo &G, long long lo, long long hi)
{
    if (a.exact || hi <= lo) return NO_CUT;
    const long long T = hi - 2LL * G.Lp - 2 + 2LL * G.L;
    const long long r = T - G.L - 3 - CUT_GUARD - lo;
    return r < W ? NO_CUT : (int)r;
}

// The column sums, for product columns >= kcut only, of the n terms in slots
// [s0, s0+n) (the same product layout as small_products), added into
// win[coff + c]; columns below kcut are left out altogether (see CUT_GUARD).
// Block 0 of unit q holds columns qW..qW+W-1 and is needed iff
// q >= Q0 = floor(kcut / W); block 1 of unit q (columns M + qW ..) iff
// q >= Q1 = floor((kcut - M) / W).  The needed chunks form a list -- block-0
// units q = Q0..P (chunks j = 0..q), then block-1 units q = P-1 down to Q1
// (chunks j = q+1..P) -- and in each round thread t of the group takes chunk
// t of the round's share of it, for all n terms, so every thread has the
// same work.  Each thread stores its chunk's W+2 digit sums in its own row
// of cstage ([group threads][W+2]); one thread per (unit, block, digit) adds
// up the rows of its unit's chunks into stage (the small_products layout,
// [P+1][2][W+2]); after the last round one thread per column adds the
// digits of the two units that reach the column (and the complement
// corrections of negative terms) into the window.  Every thread of group gr
// calls this; starts and ends with a barrier of the group.  Returns the
// chunks of one term.
__device__ int cut_products(const Geo &G, const Grp &gr, const uint32_t *Abase, const uint32_t *Cbase,
                            int s0, int n, const int *tinfo, bool neg_all, long long *stage,
                            long long *cstage, long long *win, int coff, int kcut)
{
    constexpr int ND = W + 2;
    const int P = G.P;
    // unit q's columns of block b are below kcut iff qW + W - 1 < kcut - bM
    const int Q0 = min(kcut > 0 ? kcut / W : 0, P + 1);
    const int Q1 = min(kcut > G.M ? (kcut - G.M) / W : 0, P);
    const int T0 = (P + 1) * (P + 2) / 2 - Q0 * (Q0 + 1) / 2;  // block-0 chunks
    const int n1 = P - Q1;                                       // block-1 units
    const int C = T0 + n1 * (n1 + 1) / 2;
    const int nseg0 = P + 1 - Q0, nseg = nseg0 + n1;            // (unit, block) segments
    const int tid = gr.t;
    const unsigned slot = G.VW * 4;
    const unsigned sAb = smem_addr(Abase) + s0 * slot, sCb = smem_addr(Cbase) + s0 * slot;
    grp_sync(gr);
    for (int r0 = 0; r0 < C; r0 += gr.n) {
        const int r1 = min(C, r0 + gr.n);
        const int c = r0 + tid;
        if (c < r1) {
            uint32_t a0[W], a1[W], a2[W];
#pragma unroll
            for (int k = 0; k < W; k++) a0[k] = a1[k] = a2[k] = 0u;
            int q, j;
            if (c < T0) {
                const int x = c + Q0 * (Q0 + 1) / 2;
                q = tri_root(x);
                j = x - q * (q + 1) / 2;
            } else {
                const int x = c - T0;
                const int qq = tri_root(x);
                q = P - 1 - qq;
                j = q + 1 + (x - qq * (qq + 1) / 2);
            }
            int gc0 = q - j;
            if (gc0 < 0) gc0 += G.P1;
            const int gc1 = gc0 == 0 ? P : gc0 - 1;
            unsigned sA = sAb, sC = sCb;
            for (int t = 0; t < n; t++) {
                chunk_mac(sA, sC, j, gc0, gc1, a0, a1, a2);
                sA += slot;
                sC += slot;
            }
            long long *row = cstage + (size_t)tid * ND;
#pragma unroll
            for (int t = 0; t < ND; t++) row[t] = col_digit(a0, a1, a2, t);
        }
        grp_sync(gr);
        // one thread per (segment, digit): the rows of the segment's chunks in this round
        for (int e = tid; e < nseg * ND; e += gr.n) {
            const int sg = e / ND, t = e - sg * ND;
            int q, blk, st, len;
            if (sg < nseg0) {
                q = Q0 + sg;
                blk = 0;
                st = q * (q + 1) / 2 - Q0 * (Q0 + 1) / 2;
                len = q + 1;
            } else {
                q = Q1 + (sg - nseg0);
                blk = 1;
                const int qq = P - 1 - q;
                st = T0 + qq * (qq + 1) / 2;
                len = qq + 1;
            }
            const int ka = max(st, r0) - r0, kb = min(st + len, r1) - r0;
            long long v0 = 0, v1 = 0, v2 = 0, v3 = 0;
            int k = ka;
            for (; k + 4 <= kb; k += 4) {
                v0 += cstage[(k + 0) * ND + t];
                v1 += cstage[(k + 1) * ND + t];
                v2 += cstage[(k + 2) * ND + t];
                v3 += cstage[(k + 3) * ND + t];
            }
            for (; k < kb; k++) v0 += cstage[k * ND + t];
            long long &d = stage[(q * 2 + blk) * ND + t];
            d = (r0 == 0 ? 0 : d) + (v0 + v1) + (v2 + v3);
        }
        grp_sync(gr);
    }
    // stage holds the digits of the needed (unit, block)s only
    for (int cc = max(kcut, 0) + tid; cc < G.GW; cc += gr.n) {
        long long sum = 0;
        if (cc < G.M + 2) {
            const int u = cc / W;
            if (u <= P && u >= Q0) sum += stage[(u * 2) * ND + cc - u * W];
            if (u >= 1 && u - 1 >= Q0 && cc - (u - 1) * W < ND) sum += stage[((u - 1) * 2) * ND + cc - (u - 1) * W];
        }
        const int c1 = cc - G.M;
        if (c1 >= 0) {
            const int u = c1 / W;
            if (u <= P - 1 && u >= Q1) sum += stage[(u * 2 + 1) * ND + c1 - u * W];
            if (u >= 1 && u - 1 <= P - 1 && u - 1 >= Q1 && c1 - (u - 1) * W < ND)
                sum += stage[((u - 1) * 2 + 1) * ND + c1 - (u - 1) * W];
        }
        if (tinfo) {
            for (int sl = s0; sl < s0 + n; sl++) {
                const int *ti = tinfo + sl * TI;
                if (!ti[1]) continue;
                const int y = cc - ti[2];
                const uint32_t *Cs = Cbase + (size_t)sl * G.VW;
                if (y >= 0 && y < G.Lp) sum += Cs[gpos(y)];
                else if (y >= G.Lp && y < 2 * G.Lp) sum += (uint32_t)~Cs[gpos(y - G.Lp)];
                if (y == G.Lp) sum += 1;
                if (y == 2 * G.Lp) sum -= 1;
            }
        }
        if (sum) win[coff + cc] += neg_all ? -sum : sum;
    }
    grp_sync(gr);
    return C;
}

// The products of the n terms in slots [s0, s0+n): shortened at product
// column kcut when kcut leaves out at least one block-0 unit (and the launch
// is not exact), else in full (RS lanes per unit); the executed chunks (per
// term) are added to *chunks (thread 0 of the group, when given).
__device__ void products(const Geo &G, int RS, const Grp &gr, const uint32_t *Abase,
                         const uint32_t *Cbase, int s0, int n, const int *tinfo, bool neg_all,
                         long long *stage, long long *cstage, long long *win, int coff, int kcut,
                         long long *chunks)
{
    int c;
    // shortened only where the full product takes more than one chunk per
    // thread of the group (below that the full walk's latency is no longer)
    if (kcut >= W && G.P1 * G.P1 > gr.n) {
        c = cut_products(G, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, cstage, win, coff, kcut);
    } else {
        if (n == 1 && gr.bar == 0)
            single_product(G, Abase, Cbase, s0, tinfo, neg_all, stage, win, coff);
        else
            small_products(G, RS, gr, Abase, Cbase, s0, n, tinfo, neg_all, stage, win, coff);
        c = G.P1 * G.P1;
    }
    if (chunks && gr.t == 0) *chunks += (long long)c * n;
}

// ------------------------------------------------------------------ workers

// Term t of index m for a CTA of role `role`.  Role 0, the workers: the
// middle pairs a = 2..m-2 of the Cauchy sums (coefficients up to m-2),
// 2(m-3) terms; Y (tg 0) for t < m-3 with a = t+2 and second factor
// gamma_{m-a}, Z (tg 1) after, a = t-(m-3)+2, beta_{m-a}.  Role 1 + tg, the
// outer-pair CTA of target tg: the pairs a = 1 and a = m-1 (coefficients up
// to m-1), one term when m = 2, else two.  Rows of coefL.
__device__ __forceinline__ void inner_term(int role, int m, int t, int N1, int &tg, int &arow,
                                           int &crow, int &a)
{
    if (role != 0) {
        tg = role - 1;
        a = t == 0 ? 1 : m - 1;
    } else if (t < m - 3) {
        tg = 0;
        a = t + 2;
    } else {
        tg = 1;
        a = t - (m - 3) + 2;
    }
    crow = (tg == 0 ? 2 : 1) * N1 + (m - a);
    arow = a;
}

// Window of the workers' part of index m (targets Y, Z): the pairs
// a = 3..m-3 come from the table filled with coefficient m-2's publication,
// the pairs a = 2 and a = m-2 (which involve coefficient m-2) are added here.
__device__ void inner_window(const KArgs &a, const long long mid[4], const int *expT,
                             const int *flgT, int m, long long lo[2], long long hi[2])
{
    const int N1 = a.N + 1;
    lo[0] = mid[0];
    hi[0] = mid[1];
    lo[1] = mid[2];
    hi[1] = mid[3];
    const int ends[2] = {2, m - 2};
    for (int e = 0; e < (m - 2 == 2 ? 1 : 2); e++) {
        const int aa = ends[e];
        for (int tg = 0; tg < 2; tg++) {
            const int crow = (tg == 0 ? 2 : 1) * N1 + (m - aa);
            if (!(flgT[aa] & F_NZ) || !(flgT[crow] & F_NZ)) continue;
            const long long lp = (long long)expT[aa] + expT[crow] - 2LL * a.L;
            lo[tg] = min(lo[tg], lp);
            hi[tg] = max(hi[tg], lp + 2LL * a.Lp + 2);
        }
    }
}

// Window of the outer pairs a = 1 and a = m-1 of index m >= 2 for target tg
// (0: Y, second factors gamma; 1: Z, beta); empty: lo > hi.
__device__ void outer_window(const KArgs &a, const int *expT, const int *flgT, int m, int tg,
                             long long &lo, long long &hi)
{
    const int N1 = a.N + 1;
    lo = LLONG_MAX;
    hi = LLONG_MIN;
    const int ends[2] = {1, m - 1};
    for (int e = 0; e < (m - 1 == 1 ? 1 : 2); e++) {
        const int aa = ends[e];
        const int crow = (tg == 0 ? 2 : 1) * N1 + (m - aa);
        if (!(flgT[aa] & F_NZ) || !(flgT[crow] & F_NZ)) continue;
        const long long lp = (long long)expT[aa] + expT[crow] - 2LL * a.L;
        lo = min(lo, lp);
        hi = max(hi, lp + 2LL * a.Lp + 2);
    }
}

// cp.async the factors of slots [0, nb) of the batch (m, tb0), 16 bytes a
// copy: the first factors plain into araw, the second factors into their
// cyclic layout in cc[buf] (a group of W limbs is two 16-byte pieces).
// Control group, one warp per slot.
__device__ void ctl_issue_loads(PSmem &S, const KArgs &a, const Geo &G, int TB, int buf, int role,
                                int m, int tb0, int nb, int ct)
{
    const int Lp = G.Lp, q4 = Lp / 4, lane = ct & 31;
    for (int sl = ct >> 5; sl < nb; sl += CW) {
        int tg, arow, crow, aa;
        inner_term(role, m, tb0 + sl, G.N1, tg, arow, crow, aa);
        uint32_t *ar = S.araw + (size_t)sl * Lp;
        uint32_t *cr = S.cc + ((size_t)buf * TB + sl) * G.VW;
        const uint32_t *ga = a.coefL + (size_t)arow * Lp, *gc = a.coefL + (size_t)crow * Lp;
        for (int x = lane; x < q4; x += 32) {
            cp_async16(ar + 4 * x, ga + 4 * x);
            const int g = x >> 1, h = x & 1;
            cp_async16(cr + g * GS + 4 * h, gc + 8 * g + 4 * h);
        }
    }
}

// Term info and term groups of the batch (control warp 0), then the first
// factors shifted by d_lo (complemented when negative) into ash[buf]; the
// batch's descriptor.  Window bases at MS_WLO.  Control group; the loads of
// the batch have landed.
__device__ void ctl_prepare(PSmem &S, const Geo &G, int TB, int buf, int role, int m, int tb0,
                            int nb, int par, int ct)
{
    int *desc = S.desc + buf * DESC_INTS;
    int *tinfo = S.tinfo + buf * TB_MAX * TI;
    if (ct < 32) {
        const long long *wlo = (const long long *)(S.misc + MS_WLO);
        const int lane = ct;
        int key = -1;
        if (lane < nb) {
            int tg, arow, crow, aa;
            inner_term(role, m, tb0 + lane, G.N1, tg, arow, crow, aa);
            const int fa = S.flgT[arow], fc = S.flgT[crow];
            const int neg = (tg == 0 ? 1 : 0) ^ (((fa ^ fc) & F_NEG) ? 1 : 0);
            int d = 0;
            if ((fa & F_NZ) && (fc & F_NZ)) {
                d = (int)((long long)S.expT[arow] + S.expT[crow] - 2LL * G.L - wlo[tg]);
                key = (tg << 20) | (d >> 3);
            }
            int *ti = tinfo + lane * TI;
            ti[0] = tg;
            ti[1] = neg;
            ti[2] = d & 7;
            ti[3] = d >> 3;
            ti[4] = key;
        }
        const int kprev = __shfl_up_sync(FULL, key, 1), knext = __shfl_down_sync(FULL, key, 1);
        const bool st = key >= 0 && (lane == 0 || kprev != key);
        const bool en = key >= 0 && (lane == 31 || knext != key);
        const unsigned Sm = __ballot_sync(FULL, st), Em = __ballot_sync(FULL, en);
        const unsigned lt = (1u << lane) - 1u;
        if (st) desc[DS_RUN + __popc(Sm & lt)] = lane;
        if (en) desc[DS_RUNE + __popc(Em & lt)] = lane + 1;
        if (lane == 0) {
            desc[DS_EXIT] = 0;
            desc[DS_NRUN] = __popc(Sm);
            desc[DS_PAR] = par;
            desc[DS_CUT] = S.misc[MS_CUT + 2 * par];
            desc[DS_CUT + 1] = S.misc[MS_CUT + 2 * par + 1];
        }
    }
    named_sync(BAR_CT, CT);
    for (int sl = ct >> 5; sl < nb; sl += CW) {  // one warp per slot
        const int *ti = tinfo + sl * TI;
        if (ti[4] < 0) continue;
        const int dl = ti[2];
        const uint32_t inv = ti[1] ? 0xffffffffu : 0u;
        const uint32_t *src = S.araw + (size_t)sl * G.Lp;
        uint32_t *dst = S.ash + ((size_t)buf * TB + sl) * G.VW;
        for (int x = ct & 31; x < G.M; x += 32) {
            const int y = x - dl;
            dst[gpos(x)] = (y >= 0 && y < G.Lp) ? (src[y] ^ inv) : 0u;
        }
    }
    named_sync(BAR_CT, CT);
}

// bounded wait of the control group until *flag >= target (its first thread
// polls); returns 0 when the flag is reached, -1 (group-uniform) when the
// launch must stop, and 1 as soon as the compute group is through batch
// `flush_at` - 1 (flush_at >= 0), so that the window of those batches can be
// flushed before the wait goes on.  The compute warps keep running
// meanwhile, so the poll is a relaxed load (an acquire load may invalidate
// the SM's L1 on every poll), made an acquire at the end by a fence.
__device__ int ctl_wait_geq(PSmem &S, const KArgs &a, const unsigned *flag, unsigned target, int ct,
                            long long flush_at = -1)
{
    if (ct == 0) {
        int st = 0, r = 0;
        long long it = 0;
        for (;;) {
            if ((int)(ld_relaxed_u32(flag) - target) >= 0) break;
            if ((it & 63) == 63) {  // the status word now and then (many CTAs poll here)
                st = ld_relaxed_int(a.status);
                if (st) break;
            }
            if (flush_at >= 0 && *(volatile int *)&S.misc[MS_KDONE] >= flush_at) {
                r = 1;
                break;
            }
            if (++it > a.spin_limit) {
                atomicCAS(a.status, 0, DEV_TIMEOUT);
                st = DEV_TIMEOUT;
                break;
            }
            __nanosleep(64);
        }
        // with the relaxed loads above, an acquire pattern (the flag; and the
        // compute group's count, published with a CTA fence)
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (!st && !r) st = ld_relaxed_int(a.status);
        S.misc[MS_STATUS] = st ? -1 : r;
    }
    named_sync(BAR_CT, CT);
    return S.misc[MS_STATUS];
}

// The control group of a worker or outer-pair CTA (roles 0 and 1 + target):
// per index it waits for the coefficient its terms need, places the window,
// loads and stages each batch of terms into the free buffer and hands it to
// the compute group, and once the compute group is through an index's last
// batch, adds that window into the global set and counts the CTA done.
// Consecutive indices with terms alternate between two windows, so that the
// flush of one overlaps the products of the next.
__device__ void worker_control(PSmem &S, const KArgs &a, const PArgs &pa, const Geo &G)
{
    const int ct = threadIdx.x - KT;
    const int N1 = G.N1, TB = pa.tb;
    const int role = blockIdx.x < (unsigned)(NCL + NOUT) ? 1 + (int)blockIdx.x - NCL : 0;
    const int nw = gridDim.x - NFIX;
    const int w = blockIdx.x - NFIX;
    // index m waits for coefficient m-2 (workers) or m-1 (outer pairs)
    const int lag = role ? 1 : 2;
    // with two workers or more, the first half takes the Y terms and the
    // rest the Z terms, so that no worker's range straddles the two targets
    const bool wsplit = nw >= 2;
    const int wtg = w < nw / 2 ? 0 : 1;
    const int wl = wtg ? w - nw / 2 : w, wn = wtg ? nw - nw / 2 : nw / 2;
    // this worker's terms [ta, tb) of index mm (mm >= 4); 32-bit arithmetic
    // (2 N * gridDim < 2^31), a 64-bit division being a long software routine
    auto range_of = [&](int mm, int &ta, int &tb) {
        const unsigned Tt = (unsigned)(mm - 3);  // terms per target
        if (wsplit) {
            ta = wtg * (int)Tt + (int)(Tt * (unsigned)wl / (unsigned)wn);
            tb = wtg * (int)Tt + (int)(Tt * (unsigned)(wl + 1) / (unsigned)wn);
        } else {
            ta = (int)(2u * Tt * (unsigned)w / (unsigned)nw);
            tb = (int)(2u * Tt * (unsigned)(w + 1) / (unsigned)nw);
        }
    };
    Prof pr(a, true, S.misc, KT);
    long long k = 0, kdone = 0;  // batches handed over; batches the compute group is through
    auto consumed = [&](long long upto) {
        while (kdone < upto) {
            named_sync(BAR_EMPTY + (int)(kdone & 1), PT);
            kdone++;
        }
    };
    auto flush = [&](int set, int par) {
        for (int tg = 0; tg < 2; tg++) {
            const int wd = S.misc[MS_WID + 2 * par + tg];
            long long *src = S.win + (size_t)(2 * par + tg) * G.WW;
            long long *dst = pa.gin + (((size_t)set * 3 + 1 + tg) * GIN_PARTS + (role ? 1 : 0)) * a.Wcap;
            for (int c = ct; c < wd; c += CT) {
                const long long v = src[c];
                if (v) {
                    atomicAdd((unsigned long long *)&dst[c], (unsigned long long)v);
                    src[c] = 0;
                }
            }
        }
        named_sync(BAR_CT, CT);
        if (ct == 0) {
            __threadfence();
            atomicAdd(&pa.done[set], 1u);
        }
    };
    bool pend = false;  // an index (global number pend_g) whose window awaits its flush
    int pend_set = 0, pend_par = 0, wpar = 0;
    long long pend_last = 0, pend_g = 0;
    auto flush_pending = [&]() {
        consumed(pend_last + 1);
        flush(pend_set, pend_par);
        if (ct == 0) tl_max(a, TL_WORK, (int)(pend_g % a.N), pend_g / a.N);
        pend = false;
        pr.mark(PR_CLOSE);
    };
    bool ok = true;
    for (long long step = 0; step < a.nsteps && ok; step++) {
        for (int m = 0; m < a.N; m++) {
            const long long g = step * a.N + m;
            const int set = (int)(g % PIPE_SETS);
            if (m < (role ? 2 : 4)) {  // no pairs; keep the completion counts uniform
                if (ct == 0) atomicAdd(&pa.done[set], 1u);
                continue;
            }
            // the coefficient awaited, m - lag, comes out of the brackets'
            // index g - lag - 1, which needs the windows of every index up to
            // that one: a pending one among them is flushed first
            if (pend && pend_g <= g - lag - 1) flush_pending();
            // every index waits for its coefficient, so that no CTA runs more
            // than a few indices ahead of the brackets (the sets are reused);
            // a pending window is flushed meanwhile as soon as the compute
            // group is through it
            int wr;
            while ((wr = ctl_wait_geq(S, a, pa.pub, (unsigned)(3 * (step * N1 + m + 1 - lag)), ct,
                                      pend ? pend_last + 1 : -1)) == 1)
                flush_pending();
            if (wr < 0) {
                ok = false;
                break;
            }
            pr.mark(PR_X1);
            int tA = 0, tB = m == 2 ? 1 : 2;  // outer pairs: all of them
            if (role == 0) range_of(m, tA, tB);
            // the exponents of the new coefficient, needed by later indices
            // even when this one has no terms here
            if (ct < 3) {
                const int idx = ct * N1 + m - lag;
                S.expT[idx] = __ldcg(&a.coefE[idx]);
                S.flgT[idx] = __ldcg(&a.coefF[idx]);
            } else if (role == 0 && ct >= 32 && ct < 36 && tB > tA) {
                ((long long *)(S.misc + MS_BK))[ct - 32] = __ldcg(&pa.imid[(size_t)set * 4 + ct - 32]);
            }
            if (tB <= tA) {  // no terms here: nothing to add
                if (ct == 0) atomicAdd(&pa.done[set], 1u);
                continue;
            }
            const int par = wpar;
            wpar ^= 1;
            named_sync(BAR_CT, CT);
            if (ct == 0) {
                long long lo[2], hi[2];
                if (role == 0) {
                    inner_window(a, (const long long *)(S.misc + MS_BK), S.expT, S.flgT, m, lo, hi);
                    if (wsplit) {  // only this worker's target
                        lo[1 - wtg] = 0;
                        hi[1 - wtg] = 0;
                    }
                } else {
                    const int tg = role - 1;
                    outer_window(a, S.expT, S.flgT, m, tg, lo[tg], hi[tg]);
                    lo[1 - tg] = 0;
                    hi[1 - tg] = 0;
                }
                for (int tg = 0; tg < 2; tg++) {
                    int width = 0;
                    if (hi[tg] > lo[tg]) {
                        if (hi[tg] - lo[tg] > a.Wcap) {
                            atomicCAS(a.status, 0, DEV_ERANGE);
                            S.misc[MS_STATUS] = DEV_ERANGE;
                        } else {
                            width = (int)(hi[tg] - lo[tg]);
                        }
                    }
                    ll_at(S.misc, MS_WLO + 2 * tg) = hi[tg] > lo[tg] ? lo[tg] : 0;
                    S.misc[MS_WID + 2 * par + tg] = width;
                    S.misc[MS_CUT + 2 * par + tg] =
                        width > 0 ? part_cut(a, G, lo[tg], hi[tg]) : NO_CUT;
                }
            }
            named_sync(BAR_CT, CT);
            pr.mark(PR_PLACE);
            if (S.misc[MS_STATUS] != 0) {
                ok = false;
                break;
            }
            bool first = true;
            for (int tb0 = tA; tb0 < tB; tb0 += TB) {
                const int nb = min(TB, tB - tb0);
                const int buf = (int)(k & 1);
                consumed(k - 1);  // the buffer's previous batch is through
                pr.mark(PR_STAGE);
                ctl_issue_loads(S, a, G, TB, buf, role, m, tb0, nb, ct);
                cp_async_commit();
                cp_async_wait<0>();
                named_sync(BAR_CT, CT);
                ctl_prepare(S, G, TB, buf, role, m, tb0, nb, par, ct);
                named_arrive(BAR_FULL + buf, PT);
                k++;
                pr.mark(PR_FLUSH);
                if (first && pend) flush_pending();  // the previous window (other parity)
                first = false;
            }
            pend = true;
            pend_set = set;
            pend_par = par;
            pend_last = k - 1;
            pend_g = g;
        }
    }
    if (ok && pend) flush_pending();
    // hand the compute group its exit
    consumed(k - 1);
    if (ct == 0) S.desc[(k & 1) * DESC_INTS + DS_EXIT] = 1;
    named_arrive(BAR_FULL + (int)(k & 1), PT);
    cp_async_wait<0>();
}

// The compute group: the products of each batch handed over, into the
// window of its parity.
__device__ void worker_compute(PSmem &S, const Geo &G, const PArgs &pa, const KArgs &a)
{
    const Grp gr{(int)threadIdx.x, KT, BAR_KT};
    const int TB = pa.tb;
    long long *chunks = a.chunks ? &ll_at(S.misc, MS_CHUNKS) : nullptr;
    Prof pr(a, true, S.misc, 0);
    for (long long k = 0;; k++) {
        const int b = (int)(k & 1);
        named_sync(BAR_FULL + b, PT);
        pr.mark(PR_BARRIER);
        const int *desc = S.desc + b * DESC_INTS;
        if (desc[DS_EXIT]) break;
        const int nrun = desc[DS_NRUN], par = desc[DS_PAR];
        const int *tinfo = S.tinfo + b * TB_MAX * TI;
        if (pr.p) {  // counts: term groups (slot PR_X2)
            pr.p[PR_X2] += nrun;
        }
        for (int rr = 0; rr < nrun; rr++) {
            const int rs = desc[DS_RUN + rr], re = desc[DS_RUNE + rr];
            const int *ti = tinfo + rs * TI;
            if (pr.p) pr.p[PR_X6] += re - rs;
            const int cw = desc[DS_CUT + ti[0]];
            products(G, G.RSW, gr, S.ash + (size_t)b * TB * G.VW, S.cc + (size_t)b * TB * G.VW, rs,
                     re - rs, tinfo, false, S.stage, S.cstage, S.win + (size_t)(2 * par + ti[0]) * G.WW,
                     ti[3] * W, cw == NO_CUT ? 0 : cw - ti[3] * W, chunks);
        }
        named_arrive(BAR_EMPTY + b, PT);
        if (threadIdx.x == 0) {
            // every compute thread's window sums are in (the products end
            // with a barrier of the group): tell the control group
            __threadfence_block();
            *(volatile int *)&S.misc[MS_KDONE] = (int)(k + 1);
        }
        pr.mark(PR_MAC);
    }
}

__device__ void worker_loop(PSmem &S, const KArgs &a, const PArgs &pa, const Geo &G)
{
    // zero padding of the second factors stays zero; windows start empty
    for (int e = threadIdx.x; e < 2 * pa.tb * G.M; e += PT) {
        const int s = e / G.M, x = e - s * G.M;
        if (x >= G.Lp) S.cc[(size_t)s * G.VW + gpos(x)] = 0u;
    }
    for (int e = threadIdx.x; e < 4 * G.WW; e += PT) S.win[e] = 0;
    __syncthreads();
    if (threadIdx.x < (unsigned)KT)
        worker_compute(S, G, pa, a);
    else
        worker_control(S, a, pa, G);
}

// raw limbs -> operand slot (the zero padding above Lp is never written)
__device__ __forceinline__ void to_slot(uint32_t *dst, const uint32_t *src, int Lp)
{
    for (int x = threadIdx.x; x < Lp; x += PT) dst[gpos(x)] = src[x];
}

// single non-zero limb of sigma, R, b (index and value at MS_PSCAL, index
// -1 otherwise) and the parameters' exponents and flags (MS_PARX); whole
// CTA, ends with __syncthreads
__device__ void scan_one_limb_params(PSmem &S, const KArgs &a, const Geo &G)
{
    if (threadIdx.x < 3) {
        const int p = threadIdx.x;
        int cnt = 0, i0 = -1;
        uint32_t v = 0;
        for (int x = 0; x < G.Lp; x++) {
            const uint32_t l = __ldg(&a.parL[(size_t)p * G.Lp + x]);
            if (l) {
                cnt++;
                i0 = x;
                v = l;
            }
        }
        S.misc[MS_PSCAL + 2 * p] = cnt == 1 ? i0 : -1;
        S.misc[MS_PSCAL + 2 * p + 1] = (int)v;
    } else if (threadIdx.x >= 32 && threadIdx.x < 36) {
        const int p = threadIdx.x - 32;
        S.misc[MS_PARX + 2 * p] = __ldg(&a.parE[p]);
        S.misc[MS_PARX + 2 * p + 1] = __ldg(&a.parF[p]);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ edge terms

// The edge terms of index m: a component of coefficient m times a number
// fixed for the step, i.e. the pairs a = 0 and a = m of Eq. (3)'s Cauchy
// sums and the parameter products whose parameter has more than one non-zero
// limb (a one-limb parameter's product stays a simple part of its bracket).
// They need coefficient m itself, so they sit on the chain from coefficient m
// to coefficient m+1; edge CTA e computes EDGE_T[e][0..1] as soon as m is
// out, in parallel with the others.
struct EdgeTerm {
    int tgt;   // bracket (0 alpha', 1 beta', 2 gamma'), -1 none
    int comp;  // component of coefficient m
    int fix;   // fixed factor: 0..2 component of coefficient 0, 3 + p parameter p
    int neg;   // the term enters negated
    int mpos;  // only for m > 0 (the pair a = m is the pair a = 0 at m = 0)
};
__device__ constexpr EdgeTerm EDGE_T[NEDGE][2] = {
    {{1, 0, 2, 1, 0}, {0, 1, 3 + P_SIGMA, 0, 0}},  // -alpha_m gamma_0;  +sigma beta_m
    {{1, 2, 0, 1, 1}, {0, 0, 3 + P_SIGMA, 1, 0}},  // -gamma_m alpha_0;  -sigma alpha_m
    {{2, 0, 1, 0, 0}, {1, 0, 3 + P_R, 0, 0}},      // +alpha_m beta_0;   +R alpha_m
    {{2, 1, 0, 0, 1}, {-1, 0, 0, 0, 0}},           // +beta_m alpha_0
    {{2, 2, 3 + P_B, 1, 0}, {-1, 0, 0, 0, 0}},     // -gamma_m b
};

// term T at index m: present?  Its lowest limb lp (relative to the base of
// the exact sum) and its sign.  expT/flgT hold coefficients 0 and m; the
// one-limb parameters are marked at MS_PSCAL.
__device__ bool edge_term(const PSmem &S, const KArgs &a, const Geo &G, const EdgeTerm &T, int m,
                          long long &lp, int &neg)
{
    if (T.tgt < 0 || (T.mpos && m == 0)) return false;
    const int eA = S.expT[T.comp * G.N1 + m], fA = S.flgT[T.comp * G.N1 + m];
    int eF, fF;
    if (T.fix < 3) {
        eF = S.expT[T.fix * G.N1];
        fF = S.flgT[T.fix * G.N1];
    } else {
        const int p = T.fix - 3;
        if (S.misc[MS_PSCAL + 2 * p] >= 0) return false;  // one limb: a simple part
        eF = S.misc[MS_PARX + 2 * p];
        fF = S.misc[MS_PARX + 2 * p + 1];
    }
    if (!(fA & F_NZ) || !(fF & F_NZ)) return false;
    lp = (long long)eA + eF - 2LL * G.L;
    neg = T.neg ^ (((fA ^ fF) & F_NEG) ? 1 : 0);
    return true;
}

// window of bracket c's edge terms at index m (empty: lo > hi)
__device__ void edge_window(const PSmem &S, const KArgs &a, const Geo &G, int c, int m, long long &lo,
                            long long &hi)
{
    lo = LLONG_MAX;
    hi = LLONG_MIN;
#pragma unroll
    for (int e = 0; e < NEDGE; e++)
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const EdgeTerm T = EDGE_T[e][k];
            long long lp;
            int neg;
            if (T.tgt != c || !edge_term(S, a, G, T, m, lp, neg)) continue;
            lo = min(lo, lp);
            hi = max(hi, lp + 2LL * G.Lp + 2);
        }
}

// Edge CTA e: at each index m, once coefficient m is out, its terms
// EDGE_T[e] (a component of coefficient m times a number fixed for the step)
// into the edge part of their brackets' global windows; then it counts
// itself done.
__device__ void edge_loop(PSmem &S, const KArgs &a, const PArgs &pa, const Geo &G)
{
    const int e = blockIdx.x - (NCL + NOUT);
    const int N1 = G.N1, Lp = G.Lp;
    long long *chunks = a.chunks ? &ll_at(S.misc, MS_CHUNKS) : nullptr;
    for (int i = threadIdx.x; i < NA * G.VW; i += PT) S.vA[i] = 0u;
    for (int i = threadIdx.x; i < NC * G.VW; i += PT) S.vC[i] = 0u;
    for (int i = threadIdx.x; i < 2 * G.WW; i += PT) S.win[i] = 0;
    scan_one_limb_params(S, a, G);
    for (long long step = 0; step < a.nsteps; step++) {
        for (int m = 0; m < a.N; m++) {
            Prof pr(a, true, S.misc);
            const long long g = step * a.N + m;
            const int set = (int)(g % PIPE_SETS);
            // thread 0 waits for coefficient m; then, in one round trip, its
            // exponents and the limbs of this CTA's components of it
            if (threadIdx.x == 0) S.misc[MS_STATUS] = poll_geq(a, pa.pub, (unsigned)(3 * (step * N1 + m + 1)));
            __syncthreads();
            if (S.misc[MS_STATUS]) return;
            pr.mark(PR_BARRIER);
            if (threadIdx.x == 0) tl_max(a, TL_E_SEEN, m, step);
            if (threadIdx.x >= 32) {
                // warps 1..: the limbs of this CTA's components of coefficient m
                for (int x = threadIdx.x - 32; x < 2 * Lp; x += PT - 32) {
                    const int k = x >= Lp ? 1 : 0, y = x - k * Lp;
                    const EdgeTerm T = EDGE_T[e][k];
                    if (T.tgt >= 0) S.raw[x] = __ldcg(&a.coefL[((size_t)T.comp * N1 + m) * Lp + y]);
                }
                if (m == 0) {
                    // the fixed factors of this CTA's terms: coefficient 0 or a parameter
                    for (int x = threadIdx.x - 32; x < 2 * Lp; x += PT - 32) {
                        const int k = x >= Lp ? 1 : 0, y = x - k * Lp;
                        const EdgeTerm T = EDGE_T[e][k];
                        if (T.tgt < 0) continue;
                        const uint32_t *src = T.fix < 3 ? a.coefL + (size_t)T.fix * N1 * Lp
                                                        : a.parL + (size_t)(T.fix - 3) * Lp;
                        S.vC[(size_t)k * G.VW + gpos(y)] = __ldcg(&src[y]);
                    }
                }
            } else if (threadIdx.x == 0) {
                // thread 0: the exponents of coefficient m (one round trip, in
                // step with the limbs), then the placement of the terms
                int ev[3], fv[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    ev[k] = __ldcg(&a.coefE[k * N1 + m]);
                    fv[k] = __ldcg(&a.coefF[k * N1 + m]);
                }
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    S.expT[k * N1 + m] = ev[k];
                    S.flgT[k * N1 + m] = fv[k];
                }
#pragma unroll
                for (int k = 0; k < 2; k++) {
                    const EdgeTerm T = EDGE_T[e][k];
                    long long lp, lo, hi;
                    int neg = 0, on = 0, d = 0, width = 0, cut = NO_CUT;
                    if (T.tgt >= 0 && edge_term(S, a, G, T, m, lp, neg)) {
                        edge_window(S, a, G, T.tgt, m, lo, hi);
                        if (hi - lo > a.Wcap) {
                            atomicCAS(a.status, 0, DEV_ERANGE);
                        } else {
                            on = 1;
                            d = (int)(lp - lo);
                            width = (int)(hi - lo);
                            cut = part_cut(a, G, lo, hi);
                        }
                    }
                    int *ti = S.tinfo + k * TI;
                    ti[0] = on;
                    ti[1] = neg;
                    ti[2] = d & 7;
                    ti[3] = d >> 3;
                    ti[4] = width;
                    // product column of the cut (0: in full)
                    ti[5] = cut == NO_CUT ? 0 : cut - (d >> 3) * W;
                }
            }
            __syncthreads();
            pr.mark(PR_PLACE);
            // first factors: the component shifted by d_lo, complemented when negative
            for (int k = 0; k < 2; k++) {
                const int *ti = S.tinfo + k * TI;
                if (!ti[0]) continue;
                const uint32_t *src = S.raw + (size_t)k * Lp;
                const uint32_t inv = ti[1] ? 0xffffffffu : 0u;
                const int dl = ti[2];
                uint32_t *dst = S.vA + (size_t)k * G.VW;
                for (int x = threadIdx.x; x < G.M; x += PT) {
                    const int y = x - dl;
                    dst[gpos(x)] = (y >= 0 && y < Lp) ? (src[y] ^ inv) : 0u;
                }
            }
            pr.mark(PR_STAGE);
            if (threadIdx.x == 0) tl_max(a, TL_E_MAC, m, step);
            for (int k = 0; k < 2; k++) {
                const int *ti = S.tinfo + k * TI;
                if (!ti[0]) continue;
                products(G, G.RS, whole_cta(), S.vA, S.vC, k, 1, S.tinfo, false, S.bstage, S.bcstage,
                         S.win + (size_t)k * G.WW, ti[3] * W, ti[5], chunks);
            }
            if (threadIdx.x == 0) tl_max(a, TL_E_MACD, m, step);
            pr.mark(PR_MAC);
            for (int k = 0; k < 2; k++) {
                const int *ti = S.tinfo + k * TI;
                if (!ti[0]) continue;
                const EdgeTerm T = EDGE_T[e][k];
                long long *src = S.win + (size_t)k * G.WW;
                long long *dst = pa.gin + (((size_t)set * 3 + T.tgt) * GIN_PARTS + 2) * a.Wcap;
                for (int c = threadIdx.x; c < ti[4]; c += PT) {
                    const long long v = src[c];
                    if (v) {
                        atomicAdd((unsigned long long *)&dst[c], (unsigned long long)v);
                        src[c] = 0;
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&pa.done[set], 1u);
                tl_max(a, TL_EDGE, m, step);
            }
            pr.mark(PR_FLUSH);
        }
    }
}

// ------------------------------------------------------------------ bracket CTAs

// Setup of bracket c at index m (thread 0): the simple parts (a lone number,
// a number times a one-limb parameter); the windows of the parts the other
// CTAs add (edge terms, outer pairs, middle pairs); the bracket's window
// (base, width) and each part's offset in it.  Returns false (status set)
// when the window is wider than Wcap.
__device__ bool bracket_setup(PSmem &S, const KArgs &a, const PArgs &pa, const Geo &G, int c, int m,
                              int set)
{
    (void)pa;
    (void)set;
    const int N1 = G.N1, L = G.L, Lp = G.Lp;
    int *bk = S.misc + MS_BK;
    const int eA = S.expT[m], fA = S.flgT[m];
    const int eB = S.expT[N1 + m], fB = S.flgT[N1 + m];
    int sk[2] = {0, 0}, sneg[2] = {0, 0}, scomp[2] = {0, 0};
    uint32_t sv[2] = {0u, 0u};
    long long slp[2] = {0, 0};
    int ns = 0;
    // one-limb parameter p times component comp of coefficient m (exponent e, flags f)
    auto param = [&](int p, int comp, int e, int f, int neg) {
        const int pe = S.misc[MS_PARX + 2 * p], pf = S.misc[MS_PARX + 2 * p + 1];
        const int i0 = S.misc[MS_PSCAL + 2 * p];
        if (!(pf & F_NZ) || !(f & F_NZ) || i0 < 0) return;
        sk[ns] = 2;
        sneg[ns] = neg ^ (((pf ^ f) & F_NEG) ? 1 : 0);
        scomp[ns] = comp;
        sv[ns] = (uint32_t)S.misc[MS_PSCAL + 2 * p + 1];
        slp[ns] = (long long)pe - L + i0 + (long long)e - L;
        ns++;
    };
    if (c == 0) {
        param(P_SIGMA, 1, eB, fB, 0);  // + sigma beta_m
        param(P_SIGMA, 0, eA, fA, 1);  // - sigma alpha_m
    } else if (c == 1) {
        param(P_R, 0, eA, fA, 0);      // + R alpha_m
        if (fB & F_NZ) {               // - beta_m
            sk[ns] = 1;
            sneg[ns] = 1 ^ ((fB & F_NEG) ? 1 : 0);
            scomp[ns] = 1;
            slp[ns] = (long long)eB - L;
            ns++;
        }
    } else {
        const int eG = S.expT[2 * N1 + m], fG = S.flgT[2 * N1 + m];
        param(P_B, 2, eG, fG, 1);      // - b gamma_m
    }
    long long lo = LLONG_MAX, hi = LLONG_MIN;
    for (int k = 0; k < ns; k++) {
        lo = min(lo, slp[k]);
        hi = max(hi, slp[k] + Lp + 2);
    }
    // the edge terms (edge CTAs), the middle pairs (workers) and the outer
    // pairs (outer-pair CTAs)
    long long elo, ehi, ilo = 0, ihi = 0, olo = 0, ohi = 0;
    edge_window(S, a, G, c, m, elo, ehi);
    if (ehi > elo) {
        lo = min(lo, elo);
        hi = max(hi, ehi);
    }
    if (c > 0 && m >= 4) {
        long long l2[2], h2[2];
        inner_window(a, (const long long *)(S.misc + MS_IMID), S.expT, S.flgT, m, l2, h2);
        ilo = l2[c - 1];
        ihi = h2[c - 1];
        if (ihi > ilo) {
            lo = min(lo, ilo);
            hi = max(hi, ihi);
        }
    }
    if (c > 0 && m >= 2) {
        outer_window(a, S.expT, S.flgT, m, c - 1, olo, ohi);
        if (ohi > olo) {
            lo = min(lo, olo);
            hi = max(hi, ohi);
        }
    }
    int width = 0;
    if (hi > lo) {
        if (hi - lo > a.Wcap) {
            atomicCAS(a.status, 0, DEV_ERANGE);
            return false;
        }
        width = (int)(hi - lo);
    } else {
        lo = 0;
    }
    ((long long *)(bk + BK_LO))[0] = lo;
    bk[BK_WIDTH] = width;
    bk[BK_NSIMPLE] = ns;
    for (int k = 0; k < ns; k++) {
        bk[BK_SIMPLE + 4 * k] = sk[k];
        bk[BK_SIMPLE + 4 * k + 1] = sneg[k];
        bk[BK_SIMPLE + 4 * k + 2] = (int)(slp[k] - lo);
        bk[BK_SIMPLE + 4 * k + 3] = scomp[k];
        bk[BK_SV + k] = (int)sv[k];
    }
    const bool edge = ehi > elo;
    bk[BK_EINNER] = edge ? (int)(elo - lo) : -1;
    bk[BK_EWIDTH] = edge ? (int)(ehi - elo) : 0;
    const bool inner = c > 0 && m >= 4 && ihi > ilo;
    bk[BK_INNER] = inner ? (int)(ilo - lo) : -1;
    bk[BK_IWIDTH] = inner ? (int)(ihi - ilo) : 0;
    const bool outer = c > 0 && m >= 2 && ohi > olo;
    bk[BK_OINNER] = outer ? (int)(olo - lo) : -1;
    bk[BK_OWIDTH] = outer ? (int)(ohi - olo) : 0;
    // the cuts the other CTAs take in these parts (the same windows, the same rule)
    long long cut = LLONG_MIN;
    const bool present[3] = {edge, inner, outer};
    const long long plo[3] = {elo, ilo, olo}, phi[3] = {ehi, ihi, ohi};
    for (int k = 0; k < 3; k++) {
        if (!present[k]) continue;
        const int r = part_cut(a, G, plo[k], phi[k]);
        if (r != NO_CUT) cut = max(cut, plo[k] + r);
    }
    ((long long *)(bk + BK_CUT))[0] = cut;
    return true;
}

// the bracket's lone and one-limb-parameter parts into win (thread t owns
// columns t mod PT)
__device__ void add_simple_parts(const PSmem &S, const Geo &G, long long *win, int width)
{
    const int *bk = S.misc + MS_BK;
    const int ns = bk[BK_NSIMPLE];
    for (int cc = threadIdx.x; cc < width; cc += PT) {
        long long s = 0;
        for (int k = 0; k < ns; k++) {
            const int kind = bk[BK_SIMPLE + 4 * k], neg = bk[BK_SIMPLE + 4 * k + 1];
            const int y = cc - bk[BK_SIMPLE + 4 * k + 2];
            const uint32_t *X = S.raw + (size_t)bk[BK_SIMPLE + 4 * k + 3] * G.Lp;
            long long v = 0;
            if (kind == 1) {
                if (y >= 0 && y < G.Lp) v = X[y];
            } else {
                const uint32_t pv = (uint32_t)bk[BK_SV + k];
                if (y >= 0 && y < G.Lp) v += (uint32_t)((uint64_t)pv * X[y]);
                if (y >= 1 && y <= G.Lp) v += (long long)(((uint64_t)pv * X[y - 1]) >> 32);
            }
            s += neg ? -v : v;
        }
        if (s) win[cc] += s;
    }
}

// normalise win[0..width) (base lo) and divide by dv.d into L limbs of out;
// zero the window.  Exponent and flags via e, f; false on a range error
// (status set).  `cut` (absolute limb position; LLONG_MIN: none) is the
// highest column below which some part of the sum was left out: the digits
// from cut + 2 up to the quotient's lowest kept limb must then be neither all
// zero nor all ones, or the sum may differ from the exact one in what the
// truncated quotient keeps, and the launch ends with DEV_INEXACT.
// Divisor d with its division-table entry for this thread (DivT::ent, the
// table row of d) and the odd part of d (dvo, shift a), when the table is used.
struct DivT {
    uint32_t ent;
    int a;
    Divisor dvo;
    bool on;
};
// divT: divisors of 1, 2, 3, ... (entry k: k + 1) covering d, or null
__device__ __forceinline__ DivT div_entry(const KArgs &a, int row, uint32_t d, const Divisor *divT = nullptr)
{
    DivT r;
    r.on = a.divtab != nullptr && d > 1u;
    r.ent = 0u;
    r.a = 0;
    if (r.on) {
        r.a = __ffs(d) - 1;
        r.dvo = divT ? divT[(d >> r.a) - 1] : make_divisor(d >> r.a);
        if ((int)threadIdx.x < a.divtab_rl) r.ent = __ldg(&a.divtab[(size_t)row * a.divtab_rl + threadIdx.x]);
    }
    return r;
}

__device__ bool close_bracket(PSmem &S, const KArgs &a, const Geo &G, long long *win, int width,
                              long long lo, const Divisor &dv, uint32_t *out, int &e, int &f,
                              uint32_t *out2 = nullptr, long long cut = LLONG_MIN, const DivT *dt = nullptr)
{
    e = 0;
    f = 0;
    bool ok = true;
    int top = -1, neg = 0;
    if (threadIdx.x == 0) S.misc[MS_NRUN] = 0;  // the buffer-digit flags (ordered by the barriers below)
    if (width > 0) {
        long long *red = (long long *)(S.misc + MS_RED);
        const Norm nr = width <= PT ? block_normalize_2(win, S.dig, width, red, a.status)
                                    : block_normalize(win, S.dig, width, red, a.status);
        top = nr.top;
        neg = nr.neg;
    }
    if (cut != LLONG_MIN && top >= 0) {
        // the buffer digits [cut + 2, s), s = eq - L the quotient's lowest kept
        // limb (eq as block_divide takes it): bit 0 = one is non-zero, bit 1 =
        // one is not all ones; gathered while the division runs
        const long long T = lo + top + 1;
        const long long eq = (S.dig[top] >= dv.d) ? T : T - 1;
        const long long b0 = max(cut + 2 - lo, 0LL), b1 = eq - G.L - lo;
        int bits = 0;
        for (long long x = b0 + threadIdx.x; x < b1; x += PT) {
            const uint32_t v = S.dig[x];
            bits |= (v != 0u ? 1 : 0) | (v != 0xffffffffu ? 2 : 0);
        }
        if (bits) atomicOr(&S.misc[MS_NRUN], bits);
    }
    if (top >= 0) {
        const long long eq =
            (dt && dt->on && G.L < PT) ? block_divide_2(S.dig, top, lo, dv.d, dt->a, dt->dvo, G.L, out, S.misc + MS_RED, dt->ent)
            : G.L < PT                 ? block_divide_1(S.dig, top, lo, dv, G.L, out, S.misc + MS_RED, out2)
                                       : block_divide(S.dig, top, lo, dv, G.L, out, S.misc + MS_RED, out2);
        if (eq > (1LL << 30) || eq < -(1LL << 30)) {
            if (threadIdx.x == 0) atomicCAS(a.status, 0, DEV_ERANGE);
            ok = false;
        } else {
            e = (int)eq;
            f = F_NZ | (neg ? F_NEG : 0);
        }
    }
    if (!(f & F_NZ)) {
        for (int x = threadIdx.x; x < G.L; x += PT) out[x] = 0u;
        __syncthreads();
    }
    if (cut != LLONG_MIN && S.misc[MS_NRUN] != 3) {
        // the left-out part could reach the kept limbs: the launch is rerun in full
        __syncthreads();
        if (threadIdx.x == 0) atomicCAS(a.status, 0, DEV_INEXACT);
        return false;
    }
    return ok;
}

// One Horner chain of Eq. (2) for component c on this CTA: h_N = c_N,
// h_i = trunc_L(tau h_{i+1} + c_i) for i = N-1 .. 0, then the new state (and
// a record).  h_N is this CTA's newest number.
__device__ bool horner_component(PSmem &S, const KArgs &a, const Geo &G, int c, long long step,
                                 Prof &pr)
{
    const int N1 = G.N1, Lp = G.Lp, L = G.L;
    long long *chunks = a.chunks ? &ll_at(S.misc, MS_CHUNKS) : nullptr;
    uint32_t *hA = S.vA;         // h as first factor (slot 0)
    const uint32_t *tauC = S.vC; // tau (slot 0)
    uint32_t *hp = S.raw + 2 * (size_t)Lp;     // h, plain limbs
    long long *win = S.win;
    const int tauE = __ldg(&a.parE[P_TAU]), tauF = __ldg(&a.parF[P_TAU]);
    const uint32_t *cN = S.newc;
    int he = S.misc[MS_NEWE], hf = S.misc[MS_NEWE + 1];
    for (int x = threadIdx.x; x < Lp; x += PT) {
        hp[x] = cN[x];
        hA[gpos(x)] = cN[x];
    }
    const Divisor one = make_divisor(1u);
    constexpr int CR = MAX_L / PT;
    uint32_t cur[CR], nxt[CR];
#pragma unroll
    for (int r = 0; r < CR; r++) {
        const int x = threadIdx.x + r * PT;
        cur[r] = (x < Lp && a.N >= 1) ? __ldcg(&a.coefL[((size_t)c * N1 + a.N - 1) * Lp + x]) : 0u;
    }
    __syncthreads();
    bool ok = true;
    for (int i = a.N - 1; i >= 0; i--) {
#pragma unroll
        for (int r = 0; r < CR; r++) {
            const int x = threadIdx.x + r * PT;
            nxt[r] = (i > 0 && x < Lp) ? __ldcg(&a.coefL[((size_t)c * N1 + i - 1) * Lp + x]) : 0u;
        }
        const int ce = S.expT[c * N1 + i], cf = S.flgT[c * N1 + i];
        const bool prod = (hf & F_NZ) && (tauF & F_NZ);
        const bool lone = (cf & F_NZ) != 0;
        const long long lpp = (long long)tauE + he - 2LL * L, lpa = (long long)ce - L;
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        if (prod) {
            lo = min(lo, lpp);
            hi = max(hi, lpp + 2LL * Lp + 2);
        }
        if (lone) {
            lo = min(lo, lpa);
            hi = max(hi, lpa + Lp + 2);
        }
        int width = 0;
        if (hi > lo) {
            if (hi - lo > a.Wcap) {
                if (threadIdx.x == 0) atomicCAS(a.status, 0, DEV_ERANGE);
                ok = false;
                break;  // uniform: every thread computed the same width
            }
            width = (int)(hi - lo);
        }
        // the product's columns below c0 = T - L - 3 - CUT_GUARD (T: the larger
        // top of tau h and c_i) are left out when that drops a block-0 unit
        long long cut = LLONG_MIN;
        int kcut = 0;
        if (prod && !a.exact) {
            const long long T = max((long long)tauE + he, lone ? (long long)ce : LLONG_MIN);
            const long long c0 = T - L - 3 - CUT_GUARD;
            if (c0 - lpp >= W) {
                cut = c0;
                kcut = (int)(c0 - lpp);
            }
        }
        if (prod)
            products(G, G.RS, whole_cta(), hA, tauC, 0, 1, nullptr, ((hf ^ tauF) & F_NEG) != 0, S.bstage,
                     S.bcstage, win, (int)(lpp - lo), kcut, chunks);
        pr.mark(PR_HMAC);
        if (lone) {
            const int offa = (int)(lpa - lo);
#pragma unroll
            for (int r = 0; r < CR; r++) {
                const int x = threadIdx.x + r * PT;
                if (x < Lp && cur[r]) win[offa + x] += (cf & F_NEG) ? -(long long)cur[r] : (long long)cur[r];
            }
        }
        __syncthreads();
        int e, f;
        // h for the next step, plain (hp) and as the product's first factor
        // (hA; when h is zero, the next step has no product)
        if (!close_bracket(S, a, G, win, width, lo, one, hp, e, f, hA, cut)) {
            ok = false;
            break;
        }
        he = e;
        hf = f;
#pragma unroll
        for (int r = 0; r < CR; r++) cur[r] = nxt[r];
        pr.mark(PR_HCLOSE);
    }
    if (!ok) return false;
    const long long rec = (a.record_every > 0 && ((step + 1) % a.record_every) == 0)
                              ? (step + 1) / a.record_every - 1 : -1;
    for (int x = threadIdx.x; x < Lp; x += PT) {
        const uint32_t v = x < L ? hp[x] : 0u;
        a.stL[(size_t)c * Lp + x] = v;
        if (rec >= 0 && x < L) a.recL[((size_t)rec * 3 + c) * L + x] = v;
    }
    if (threadIdx.x == 0) {
        a.stE[c] = he;
        a.stF[c] = hf;
        if (rec >= 0) {
            a.recS[rec * 3 + c] = (hf & F_NEG) ? 1 : 0;
            a.recE[rec * 3 + c] = he;
        }
    }
    __threadfence();
    return true;
}


// One Horner chain of Eq. (2) when tau = trunc_L(p/q) with small p, q: then
// tau h = (p h - r h 2^(-32 shift)) / q exactly (r = p 2^(32 shift) mod q), so
// h_i = trunc_L(tau h_{i+1} + c_i) = trunc_L(E / q) with the exact
//   E = +-(p h_{i+1} - r h_{i+1} 2^(-32 shift)) + q c_i,
// three one-limb multiples of numbers instead of an L x L product: the window
// gets them column by column, then the close divides by q.  Same bits as
// horner_component.
__device__ bool horner_ratio(PSmem &S, const KArgs &a, const Geo &G, int c, long long step, Prof &pr)
{
    const int N1 = G.N1, Lp = G.Lp, L = G.L;
    uint32_t *hp = S.raw + 2 * (size_t)Lp;  // h, plain limbs
    uint32_t *ci = S.raw;                    // c_i, plain limbs
    long long *win = S.win;
    const uint32_t tp = a.tau_p, tq = a.tau_q, tr = a.tau_r;
    const int sh = a.tau_shift;
    const Divisor dq = make_divisor(tq);
    const DivT dth = div_entry(a, 0, tq);  // row 0: tau's q
    int he = S.misc[MS_NEWE], hf = S.misc[MS_NEWE + 1];
    constexpr int CR = MAX_L / PT;
    uint32_t nxt[CR];
    for (int x = threadIdx.x; x < Lp; x += PT) {
        hp[x] = S.newc[x];
        ci[x] = a.N >= 1 ? __ldcg(&a.coefL[((size_t)c * N1 + a.N - 1) * Lp + x]) : 0u;
    }
    __syncthreads();
    bool ok = true;
    for (int i = a.N - 1; i >= 0; i--) {
#pragma unroll
        for (int r = 0; r < CR; r++) {
            const int x = threadIdx.x + r * PT;
            nxt[r] = (i > 0 && x < Lp) ? __ldcg(&a.coefL[((size_t)c * N1 + i - 1) * Lp + x]) : 0u;
        }
        const int ce = S.expT[c * N1 + i], cf = S.flgT[c * N1 + i];
        const bool prod = (hf & F_NZ) != 0;
        const bool lone = (cf & F_NZ) != 0;
        const long long lph = (long long)he - L, lpr = lph - sh, lpc = (long long)ce - L;
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        if (prod) {
            lo = min(lo, tr ? lpr : lph);
            hi = max(hi, lph + Lp + 2);
        }
        if (lone) {
            lo = min(lo, lpc);
            hi = max(hi, lpc + Lp + 2);
        }
        int width = 0;
        if (hi > lo) {
            if (hi - lo > a.Wcap) {
                if (threadIdx.x == 0) atomicCAS(a.status, 0, DEV_ERANGE);
                ok = false;
                break;  // uniform
            }
            width = (int)(hi - lo);
        }
        const bool hneg = ((hf & F_NEG) != 0) != (a.tau_neg != 0), cneg = (cf & F_NEG) != 0;
        const int oh = (int)(lph - lo), orr = (int)(lpr - lo), oc = (int)(lpc - lo);
        // column cc of v X placed at offset o: low half of v x_y plus high half of v x_{y-1}
        auto scaled = [&](const uint32_t *X, uint32_t v, int y) -> long long {
            long long t = 0;
            if (y >= 0 && y < Lp) t += (uint32_t)((uint64_t)v * X[y]);
            if (y >= 1 && y <= Lp) t += (long long)(((uint64_t)v * X[y - 1]) >> 32);
            return t;
        };
        for (int cc = threadIdx.x; cc < width; cc += PT) {
            long long s = 0;
            if (prod) {
                const long long th = scaled(hp, tp, cc - oh) - (tr ? scaled(hp, tr, cc - orr) : 0);
                s += hneg ? -th : th;
            }
            if (lone) {
                const long long tc = scaled(ci, tq, cc - oc);
                s += cneg ? -tc : tc;
            }
            if (s) win[cc] += s;
        }
        __syncthreads();
        pr.mark(PR_HMAC);
        int e, f;
        if (!close_bracket(S, a, G, win, width, lo, dq, hp, e, f, nullptr, LLONG_MIN, &dth)) {
            ok = false;
            break;
        }
        he = e;
        hf = f;
        // c_{i-1} for the next step (every thread is past the column loop)
#pragma unroll
        for (int r = 0; r < CR; r++) {
            const int x = threadIdx.x + r * PT;
            if (x < Lp) ci[x] = nxt[r];
        }
        __syncthreads();
        pr.mark(PR_HCLOSE);
    }
    if (!ok) return false;
    const long long rec = (a.record_every > 0 && ((step + 1) % a.record_every) == 0)
                              ? (step + 1) / a.record_every - 1 : -1;
    for (int x = threadIdx.x; x < Lp; x += PT) {
        const uint32_t v = x < L ? hp[x] : 0u;
        a.stL[(size_t)c * Lp + x] = v;
        if (rec >= 0 && x < L) a.recL[((size_t)rec * 3 + c) * L + x] = v;
    }
    if (threadIdx.x == 0) {
        a.stE[c] = he;
        a.stF[c] = hf;
        if (rec >= 0) {
            a.recS[rec * 3 + c] = (hf & F_NEG) ? 1 : 0;
            a.recE[rec * 3 + c] = he;
        }
    }
    __threadfence();
    return true;
}

// Bracket CTA c: coefficient component c of every index, then Horner.
__device__ void closer_loop(PSmem &S, const KArgs &a, const PArgs &pa, const Geo &G)
{
    const int c = blockIdx.x;
    const int N1 = G.N1, Lp = G.Lp;
    const bool prof_on = true;
    for (int e = threadIdx.x; e < NA * G.VW; e += PT) S.vA[e] = 0u;
    for (int e = threadIdx.x; e < NC * G.VW; e += PT) S.vC[e] = 0u;
    for (int e = threadIdx.x; e < 3 * Lp; e += PT) S.raw[e] = 0u;
    for (int e = threadIdx.x; e < Lp; e += PT) S.newc[e] = 0u;
    for (int e = threadIdx.x; e < 2 * G.WW; e += PT) S.win[e] = 0;
    for (int m = threadIdx.x; m <= a.N; m += PT) S.divT[m] = make_divisor((uint32_t)(m + 1));
    scan_one_limb_params(S, a, G);
    // tau (Horner's fixed factor)
    to_slot(S.vC, a.parL + (size_t)P_TAU * Lp, Lp);
    __syncthreads();
    for (long long step = 0; step < a.nsteps; step++) {
        // the state is coefficient 0 (Sec. 2): publish this CTA's component,
        // then take all three
        for (int x = threadIdx.x; x < Lp; x += PT)
            a.coefL[(size_t)c * N1 * Lp + x] = __ldcg(&a.stL[(size_t)c * Lp + x]);
        if (threadIdx.x == 0) {
            a.coefE[c * N1] = __ldcg(&a.stE[c]);
            a.coefF[c * N1] = __ldcg(&a.stF[c]);
        }
        __syncthreads();
        if (threadIdx.x == 0) red_release_add_u32(pa.pub, 1u);
        if (!wait_geq(S, a, pa.pub, (unsigned)(3 * (step * N1 + 1)))) return;
        if (threadIdx.x < 3) {
            S.expT[threadIdx.x * N1] = __ldcg(&a.coefE[threadIdx.x * N1]);
            S.flgT[threadIdx.x * N1] = __ldcg(&a.coefF[threadIdx.x * N1]);
        }
        for (int e = threadIdx.x; e < 3 * Lp; e += PT) {
            const int comp = e / Lp, x = e - comp * Lp;
            S.raw[e] = __ldcg(&a.coefL[((size_t)comp * N1) * Lp + x]);
        }
        __syncthreads();
        for (int m = 0; m < a.N; m++) {
            Prof pr(a, prof_on, S.misc);
            const long long g = step * a.N + m;
            const int set = (int)(g % PIPE_SETS);
            const Divisor dvm = S.divT[m];
            const DivT dtm = div_entry(a, m + 1, (uint32_t)(m + 1), S.divT);  // read now, used at the close
            if (c == 1 && threadIdx.x == 0) tl_put(a, TL_B_START, m, step);
            if (threadIdx.x == 0) S.misc[MS_STATUS] = bracket_setup(S, a, pa, G, c, m, set) ? 0 : 1;
            __syncthreads();
            pr.mark(PR_X1);
            if (S.misc[MS_STATUS]) return;
            const int *bk = S.misc + MS_BK;
            const long long lo = ((const long long *)(bk + BK_LO))[0];
            const int width = bk[BK_WIDTH];
            long long *win = S.win;
            add_simple_parts(S, G, win, width);
            pr.mark(PR_PLACE);
            if (bk[BK_INNER] >= 0 || bk[BK_OINNER] >= 0 || bk[BK_EINNER] >= 0) {
                // every other CTA has added its sums of index m
                const unsigned target = (unsigned)((g / PIPE_SETS + 1) * (long long)(gridDim.x - NCL));
                if (!wait_geq(S, a, pa.done + set, target)) return;
                if (c == 1 && threadIdx.x == 0) tl_put(a, TL_B_WAITED, m, step);
                pr.mark(PR_BARRIER);
                // the three parts of this bracket (middle pairs, outer pairs,
                // edge terms); a thread owns window columns cc = threadIdx.x mod PT
                long long *gp = pa.gin + ((size_t)set * 3 + c) * 3 * a.Wcap;
                int off[3], wd[3];
                off[0] = bk[BK_INNER];
                wd[0] = bk[BK_IWIDTH];
                off[1] = bk[BK_OINNER];
                wd[1] = bk[BK_OWIDTH];
                off[2] = bk[BK_EINNER];
                wd[2] = bk[BK_EWIDTH];
                for (int cc = threadIdx.x; cc < width; cc += PT) {
                    // the three loads first (one round trip), then the zeroing
                    long long u[3];
                    long long *q[3];
#pragma unroll
                    for (int part = 0; part < 3; part++) {
                        const int y = cc - off[part];
                        q[part] = nullptr;
                        u[part] = 0;
                        if (off[part] >= 0 && y >= 0 && y < wd[part]) {
                            q[part] = gp + (size_t)part * a.Wcap + y;
                            u[part] = __ldcg(q[part]);
                        }
                    }
                    long long v = 0;
#pragma unroll
                    for (int part = 0; part < 3; part++) {
                        if (u[part]) {
                            v += u[part];
                            *q[part] = 0;
                        }
                    }
                    if (v) win[cc] += v;
                }
                pr.mark(PR_STAGE);
            }
            __syncthreads();
            int e, f;
            const bool ok = close_bracket(S, a, G, win, width, lo, dvm, S.newc, e, f, nullptr,
                                          ((const long long *)(bk + BK_CUT))[0], &dtm);
            pr.mark(PR_CLOSE);
            if (!ok) return;
            if (threadIdx.x == 0) {
                S.misc[MS_NEWE] = e;
                S.misc[MS_NEWE + 1] = f;
            }
            for (int x = threadIdx.x; x < Lp; x += PT) a.coefL[((size_t)c * N1 + m + 1) * Lp + x] = S.newc[x];
            if (c == 0 && m + 3 < a.N) {
                // window table of the workers' part of index m+3 without its
                // two newest pairs: pairs (a, m+3-a), a = 3..m
                long long lo3[2] = {LLONG_MAX, LLONG_MAX}, hi3[2] = {LLONG_MIN, LLONG_MIN};
                for (int aa = 3 + threadIdx.x; aa <= m; aa += PT) {
                    const int b = m + 3 - aa;
                    if (!(S.flgT[aa] & F_NZ)) continue;
                    for (int tg = 0; tg < 2; tg++) {
                        const int crow = (tg == 0 ? 2 : 1) * N1 + b;
                        if (!(S.flgT[crow] & F_NZ)) continue;
                        const long long lp = (long long)S.expT[aa] + S.expT[crow] - 2LL * G.L;
                        lo3[tg] = min(lo3[tg], lp);
                        hi3[tg] = max(hi3[tg], lp + 2LL * Lp + 2);
                    }
                }
                long long *red = (long long *)(S.misc + MS_RED);
                const long long r0 = block_min_ll(lo3[0], red), r1 = block_max_ll(hi3[0], red);
                const long long r2 = block_min_ll(lo3[1], red), r3 = block_max_ll(hi3[1], red);
                if (threadIdx.x == 0) {
                    long long *mid = pa.imid + (size_t)((g + 3) % PIPE_SETS) * 4;
                    mid[0] = r0;
                    mid[1] = r1;
                    mid[2] = r2;
                    mid[3] = r3;
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                a.coefE[c * N1 + m + 1] = e;
                a.coefF[c * N1 + m + 1] = f;
                red_release_add_u32(pa.pub, 1u);
                if (c == 1) tl_put(a, TL_B_PUB, m, step);
                if (c == 2) tl_put(a, TL_G_PUB, m, step);
            }
            pr.mark(PR_X3);
            // coefficient m+1: all three components
            if (!wait_geq(S, a, pa.pub, (unsigned)(3 * (step * N1 + m + 2)))) return;
            pr.mark(PR_X4);
            if (threadIdx.x < 3) {
                const int idx = threadIdx.x * N1 + m + 1;
                S.expT[idx] = __ldcg(&a.coefE[idx]);
                S.flgT[idx] = __ldcg(&a.coefF[idx]);
            }
            if (threadIdx.x >= 32 && threadIdx.x < 36 && m + 1 >= 4 && m + 1 < a.N) {
                // window table of the workers' part of index m+1 (written with
                // coefficient m-1)
                ((long long *)(S.misc + MS_IMID))[threadIdx.x - 32] =
                    __ldcg(&pa.imid[(size_t)((g + 1) % PIPE_SETS) * 4 + threadIdx.x - 32]);
            }
            for (int e2 = threadIdx.x; e2 < 3 * Lp; e2 += PT) {
                const int comp = e2 / Lp, x = e2 - comp * Lp;
                S.raw[e2] = comp == c ? S.newc[x] : __ldcg(&a.coefL[((size_t)comp * N1 + m + 1) * Lp + x]);
            }
            __syncthreads();
            pr.mark(PR_X5);
        }
        // Horner (Eq. (2)) for this CTA's component
        Prof ph(a, prof_on, S.misc);
        if (!(a.tau_q ? horner_ratio(S, a, G, c, step, ph) : horner_component(S, a, G, c, step, ph)))
            return;
        __syncthreads();
        ph.mark(PR_HORNER);
    }
}

__global__ void __launch_bounds__(PT, 1) pipe_kernel(KArgs a, PArgs pa)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Geo G(a.L, a.Lp, a.N, a.Wcap);
    PSmem S;
    pipe_layout(G, a.N, pa.tb, &S, smem_raw);
    const bool prof_cta = true;
    if (threadIdx.x < PROF_SLOTS) ((long long *)(S.misc + MS_PROF))[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        S.misc[MS_STATUS] = 0;
        S.misc[MS_KDONE] = 0;
        ll_at(S.misc, MS_CHUNKS) = 0;
    }
    __syncthreads();
    Prof tot(a, prof_cta, S.misc);
    if (blockIdx.x < (unsigned)NCL)
        closer_loop(S, a, pa, G);
    else if (blockIdx.x < (unsigned)(NCL + NOUT) || blockIdx.x >= (unsigned)NFIX)
        worker_loop(S, a, pa, G);
    else
        edge_loop(S, a, pa, G);
    __syncthreads();
    tot.mark(PR_TOTAL);
    if (a.chunks && threadIdx.x == 0)
        atomicAdd(a.chunks, (unsigned long long)ll_at(S.misc, MS_CHUNKS));
    if (a.prof && threadIdx.x == 0) {
        // rows 0 and 1: the beta' bracket CTA and the last worker; then one row per CTA
        const long long *src = (const long long *)(S.misc + MS_PROF);
        long long *row = a.prof + (size_t)(2 + blockIdx.x) * PROF_SLOTS;
        for (int k = 0; k < PROF_SLOTS; k++) row[k] += src[k];
        if (blockIdx.x == 1 || blockIdx.x == gridDim.x - 1) {
            long long *dst = a.prof + (blockIdx.x == 1 ? 0 : PROF_SLOTS);
            for (int k = 0; k < PROF_SLOTS; k++) dst[k] += src[k];
        }
    }
}

}  // namespace

size_t pipe_smem_bytes(int L, int Lp, int N, int Wcap, int tb)
{
    const Geo G(L, Lp, N, Wcap);
    return pipe_layout(G, N, tb, nullptr, nullptr);
}

int pipe_tb_max() { return TB_MAX; }
int pipe_fixed_ctas() { return NFIX; }

int pipe_max_ctas(size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pipe_kernel, PT, smem) != cudaSuccess)
        return 0;
    return per * sms;
}

cudaError_t launch_pipe(const KArgs &a, const PArgs &pa, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    KArgs ca = a;
    PArgs cpa = pa;
    void *args[] = {&ca, &cpa};
    return cudaLaunchCooperativeKernel((const void *)pipe_kernel, dim3(grid), dim3(PT), args, smem, st);
}

}  // namespace mpt
