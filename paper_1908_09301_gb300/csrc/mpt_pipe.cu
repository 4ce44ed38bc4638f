// mpt_pipe.cu -- pipelined multiple-precision Taylor step (Sec. 2 of Dimova
// et al., arXiv 1908.09301) for large L x N: one persistent launch, two roles.
//
//  * The critical path (one CTA cluster, "closer"): for each index m it forms
//    the terms of Eq. (3)'s brackets that involve the newest coefficient m --
//    the "outer" Cauchy products alpha_m gamma_0, alpha_0 gamma_m,
//    alpha_m beta_0, alpha_0 beta_m and the linear terms sigma beta_m,
//    sigma alpha_m, R alpha_m, b gamma_m, beta_m -- split over the cluster's
//    CTAs, reduces them through distributed shared memory, adds the "inner"
//    sums computed by the workers, normalises, divides by (m+1) and
//    publishes coefficient m+1.  After index N-1 it runs the three Horner
//    chains of Eq. (2), h_i = trunc_L(tau h_{i+1} + c_i), the same way.
//  * The bulk ("workers", every other CTA): the inner part of the Cauchy
//    sums, sum_{a=1}^{m-1} alpha_a gamma_{m-a} and alpha_a beta_{m-a}, which
//    needs only coefficients up to m-1, so it is computed while the closer
//    is still finishing index m-1.  Each worker takes a contiguous slice of
//    the (product, chunk, column pair) units, accumulates exact int64 column
//    windows in shared memory, adds them into a global window set and counts
//    itself done.
//
// Hand-over: a monotone "published" counter (release/acquire) and per-set
// monotone completion counters; every wait is bounded and ends the launch
// with a status code when it expires.  Integer sums are exact and
// associative, so the result does not depend on the split.
#include <climits>
#include <cstdint>
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "mpt_common.cuh"
#include "mpt_kernel.cuh"

namespace cg = cooperative_groups;

namespace mpt {
namespace {

constexpr int CP_C = 8;                               // CTAs of the closer cluster
constexpr int NA = 8;                                 // A-layout vector slots of the closer
constexpr int NC = 8;                                 // C-layout vector slots of the closer
constexpr int HU = NT;                                // Horner units per step (one per thread)

// closer vector slots
enum { A_SIGMA = 0, A_R, A_B, A_TAU, A_ALPHA0, A_ALPHAM, A_BETAM, A_CI };
enum { C_GAMMA0 = 0, C_BETA0, C_GAMMAM, C_BETAM, C_ALPHAM, C_H0, C_H1, C_H2 };
enum { P_SIGMA = 0, P_R = 1, P_B = 2, P_TAU = 3 };

struct PSmem {
    int *expT, *flgT;    // [3][N+1]
    int *tinfo;          // [max(tb, 64)][4]
    int *misc;           // [MISC_INTS]
    // closer CTAs
    long long *win;      // [3][wsz] outer-term accumulators
    long long *comb;     // [3][wsz] CTA 0: combined windows
    uint32_t *dig;       // [3][Wcap]
    uint32_t *newc;      // [3][Lp] plain limbs of the newest number (CTA 0)
    uint32_t *vec;       // [NA][AV] then [NC][CV]
    long long *hstage;   // [2 (W+2)][HU + 1] Horner unit results
    // worker CTAs (same bytes as the closer's part)
    uint32_t *wvec;      // [tb][AV + CV]
    long long *stage;    // [2 (W+2)][umax + 1] unit results (odd row stride: no bank conflicts)
    long long *wwin;     // [2][wsz] inner-sum windows (beta, gamma)
    int AV, CV, M, wsz;
};

enum {
    MS_BASE = 0,     // [3] long long: window base of each target (ints 0..5)
    MS_WIDTH = 8,    // [3]
    MS_OBASE = 12,   // [3] long long: outer-terms base (ints 12..17)
    MS_OWIDTH = 20,  // [3]
    MS_IBASE = 24,   // [3] long long: inner-terms base (ints 24..29)
    MS_IWIDTH = 32,  // [3]
    MS_NTERM = 36,   // number of outer terms
    MS_ERR_A = 37,   // closer: stop flag set before barrier #1 (read by the whole cluster)
    MS_ERR_C = 38,   // closer: stop flag set before barrier #3
    MS_PSCAL = 40,   // [3][2] parameter sigma, R, b: single non-zero limb index (or -1), value
    MS_UNITS = 48,   // unit bookkeeping
    MS_HE = 52,      // [3] Horner exponents
    MS_HF = 56,      // [3] Horner flags
    MS_RED = 64,     // [8 warps][6] long long reduction scratch: ints 64..159
    MS_STATUS = 160, // CTA-uniform copy of the status word
    MS_HERR = 161,   // Horner of this CTA failed
    MISC_INTS = 256
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline void psizes(int Lp, int Wcap, int &AV, int &CV, int &M, int &wsz)
{
    M = Lp + W;
    AV = phys(Lp - 1) + 2;
    CV = phys(M - 1) + 2;
    wsz = wsize(Wcap);
}

__host__ __device__ inline size_t pipe_layout(int Lp, int N, int Wcap, int tb, int umax, PSmem *S,
                                              unsigned char *base)
{
    int AV, CV, M, wsz;
    psizes(Lp, Wcap, AV, CV, M, wsz);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = al16(o + bytes);
        return base ? base + at : nullptr;
    };
    unsigned char *p;
    p = take(sizeof(int) * 3 * (N + 1));
    if (S) S->expT = (int *)p;
    p = take(sizeof(int) * 3 * (N + 1));
    if (S) S->flgT = (int *)p;
    p = take(sizeof(int) * 4 * (tb > 64 ? tb : 64));
    if (S) S->tinfo = (int *)p;
    p = take(sizeof(int) * MISC_INTS);
    if (S) S->misc = (int *)p;
    const size_t u0 = o;
    // closer part
    p = take(sizeof(long long) * 3 * wsz);
    if (S) S->win = (long long *)p;
    p = take(sizeof(long long) * 3 * wsz);
    if (S) S->comb = (long long *)p;
    p = take(sizeof(uint32_t) * 3 * Wcap);
    if (S) S->dig = (uint32_t *)p;
    p = take(sizeof(uint32_t) * 3 * Lp);
    if (S) S->newc = (uint32_t *)p;
    p = take(sizeof(uint32_t) * (size_t)(NA * AV + NC * CV));
    if (S) S->vec = (uint32_t *)p;
    p = take(sizeof(long long) * 2 * (W + 2) * (size_t)(HU + 1));
    if (S) S->hstage = (long long *)p;
    const size_t closer_end = o;
    // worker part, over the same bytes
    o = u0;
    p = take(sizeof(uint32_t) * (size_t)tb * (AV + CV));
    if (S) S->wvec = (uint32_t *)p;
    p = take(sizeof(long long) * 2 * (W + 2) * (size_t)(umax + 1));
    if (S) S->stage = (long long *)p;
    p = take(sizeof(long long) * 2 * wsz);
    if (S) S->wwin = (long long *)p;
    if (closer_end > o) o = closer_end;
    if (S) {
        S->AV = AV;
        S->CV = CV;
        S->M = M;
        S->wsz = wsz;
    }
    return o;
}

__device__ __forceinline__ long long &ll_at(int *misc, int slot) { return ((long long *)(misc + slot))[0]; }

// --------------------------------------------------------------- small helpers

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

// block min/max of lo[t], hi[t] for t < 3 -> misc[base_slot + 2t] (ll), misc[width_slot + t];
// width > Wcap sets the status word (ERANGE) and width 0
__device__ void block_window(PSmem &S, const KArgs &a, long long lo[3], long long hi[3],
                             int base_slot, int width_slot)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long *red = (long long *)(S.misc + MS_RED);
    for (int t = 0; t < 3; t++) {
        long long l = warp_min_ll(lo[t]), h = warp_max_ll(hi[t]);
        if (lane == 0) {
            red[warp * 6 + t] = l;
            red[warp * 6 + 3 + t] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        const int t = threadIdx.x;
        long long l = red[t], h = red[3 + t];
        for (int w = 1; w < NT / 32; w++) {
            l = min(l, red[w * 6 + t]);
            h = max(h, red[w * 6 + 3 + t]);
        }
        int width = 0;
        if (h > l) {
            if (h - l > a.Wcap) {
                atomicCAS(a.status, 0, DEV_ERANGE);
                S.misc[MS_STATUS] = DEV_ERANGE;
            } else {
                width = (int)(h - l);
            }
        }
        ((long long *)(S.misc + base_slot))[t] = (h > l) ? l : 0;
        S.misc[width_slot + t] = width;
    }
    __syncthreads();
}

// Per-phase cycle counters of thread 0 of the closer's CTA 0 and of the last
// worker, accumulated in shared memory and written out at the end.
constexpr int MS_PROF = 192;  // [PROF_SLOTS] long long: ints 192..223

struct Prof {
    long long *p;
    long long t;
    __device__ Prof(const KArgs &a, bool on, int *misc)
    {
        p = nullptr;
        t = 0;
        if (a.prof && on && threadIdx.x == 0) {
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

// bounded wait until *flag >= target (thread 0); status checked on the way.
// Returns false (CTA-uniform) when the launch must stop.
__device__ bool wait_geq(PSmem &S, const KArgs &a, const unsigned *flag, unsigned target)
{
    if (threadIdx.x == 0) {
        int st = 0;
        long long it = 0;
        while ((int)(ld_acquire_u32(flag) - target) < 0) {
            if (++it > a.spin_limit) {
                atomicCAS(a.status, 0, DEV_TIMEOUT);
                st = DEV_TIMEOUT;
                break;
            }
            if ((it & 63) == 0) {
                st = ld_relaxed_int(a.status);
                if (st) break;
            }
            __nanosleep(20);
        }
        if (!st) st = ld_relaxed_int(a.status);
        S.misc[MS_STATUS] = st;
    }
    __syncthreads();
    return S.misc[MS_STATUS] == 0;
}

// --------------------------------------------------------------- workers

// inner Cauchy terms of index m: t < m-1 -> Y: -alpha_a gamma_{m-a}, a = t+1;
// otherwise Z: +alpha_a beta_{m-a}, a = t-(m-1)+1
__device__ __forceinline__ void inner_term(int m, int t, int &tg, int &neg, int &acomp, int &aidx,
                                           int &bcomp, int &bidx)
{
    if (t < m - 1) {
        tg = 1;
        neg = 1;
        acomp = 0;
        aidx = t + 1;
        bcomp = 2;
        bidx = m - aidx;
    } else {
        tg = 2;
        neg = 0;
        acomp = 0;
        aidx = t - (m - 1) + 1;
        bcomp = 1;
        bidx = m - aidx;
    }
}

// window placement of the inner terms of index m (targets 1 = Y, 2 = Z)
__device__ void inner_windows(PSmem &S, const KArgs &a, int m, int base_slot, int width_slot)
{
    const int N1 = a.N + 1;
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
    long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    const int T = 2 * (m - 1);
    for (int t = threadIdx.x; t < T; t += NT) {
        int tg, neg, ac, ai, bc, bi;
        inner_term(m, t, tg, neg, ac, ai, bc, bi);
        int fa = S.flgT[ac * N1 + ai], fb = S.flgT[bc * N1 + bi];
        if (!(fa & F_NZ) || !(fb & F_NZ)) continue;
        long long lp = (long long)S.expT[ac * N1 + ai] + S.expT[bc * N1 + bi] - 2LL * a.L;
        lo[tg] = min(lo[tg], lp);
        hi[tg] = max(hi[tg], lp + 2LL * a.Lp + 2);
    }
    block_window(S, a, lo, hi, base_slot, width_slot);
}

struct Chunking {
    int H;   // chunks per column pair
    int CL;  // steps per chunk (multiple of W)
};

__device__ __forceinline__ Chunking chunking(long long pairs, long long threads, int P)
{
    // enough units that every thread has about one and a half
    long long want = (3 * threads + 2 * pairs - 1) / (2 * pairs);
    int H = (int)min((long long)(P + 1), max(1LL, want));
    Chunking c;
    c.CL = ((P + 1 + H - 1) / H) * W;
    c.H = ((P + 1) * W + c.CL - 1) / c.CL;
    return c;
}

// Chunks per column pair for nt terms on NT threads: the H in 1..4 whose
// units fill the threads' rounds best (a unit per thread per round), a little
// biased toward fewer, longer units; units of one batch must fit `umax`.
__device__ __forceinline__ Chunking worker_chunking(int nt, int P, int umax)
{
    int best = 1;
    double best_score = -1.0;
    for (int H = 1; H <= 4; H++) {
        const int CL = ((P + 1 + H - 1) / H) * W;
        const int He = ((P + 1) * W + CL - 1) / CL;
        const long long U = (long long)nt * P * He;
        if (H > 1 && U > umax) break;
        const double x = (double)U / NT;
        const double rounds = ceil(x);
        const double score = x / rounds - 0.03 * (He - 1);
        if (score > best_score + 1e-9) {
            best_score = score;
            best = H;
        }
    }
    Chunking c;
    c.CL = ((P + 1 + best - 1) / best) * W;
    c.H = ((P + 1) * W + c.CL - 1) / c.CL;
    return c;
}

// Workers: the inner Cauchy sums of index m (pairs a = 1..m-1, which need
// coefficients up to m-1 only).  Each worker takes a contiguous range of
// whole products; inside a CTA the units are ordered (chunk, pair, product),
// so a warp holds few distinct column pairs.  Units write their column
// digits to a private staging slot; a column reduction then adds each
// window column once into the global accumulator set.
__device__ void worker_loop(PSmem &S, const KArgs &a, const PArgs &pa)
{
    const int N1 = a.N + 1, Lp = a.Lp, P = a.P;
    const int nw = gridDim.x - CP_C;
    const int w = blockIdx.x - CP_C;
    const int SL = S.AV + S.CV;
    const int umax = pa.umax;
    const int ustride = umax + 1;
    const bool prof_on = (blockIdx.x == gridDim.x - 1);
    // C padding of every slot stays zero; windows start empty
    for (int e = threadIdx.x; e < a.tb * S.M; e += NT) {
        int slot = e / S.M, x = e - slot * S.M;
        if (x >= Lp) S.wvec[(size_t)slot * SL + S.AV + phys(x)] = 0u;
    }
    for (int e = threadIdx.x; e < 2 * S.wsz; e += NT) S.wwin[e] = 0;
    __syncthreads();
    for (long long step = 0; step < a.nsteps; step++) {
        for (int m = 0; m < a.N; m++) {
            const long long g = step * a.N + m;
            const int set = (int)(g % PIPE_SETS);
            if (m < 2) {  // no inner terms; keep the completion counts uniform
                if (threadIdx.x == 0) atomicAdd(&pa.done[set], 1u);
                continue;
            }
            Prof pr(a, prof_on, S.misc);
            if (!wait_geq(S, a, pa.pub, (unsigned)(step * N1 + m))) return;
            pr.mark(PR_BARRIER);
            // exponent / flag of coefficient m-1 (published with it)
            if (threadIdx.x < 3) {
                const int idx = threadIdx.x * N1 + m - 1;
                S.expT[idx] = __ldcg(&a.coefE[idx]);
                S.flgT[idx] = __ldcg(&a.coefF[idx]);
            }
            __syncthreads();
            inner_windows(S, a, m, MS_IBASE, MS_IWIDTH);
            pr.mark(PR_PLACE);
            if (S.misc[MS_STATUS] != 0) return;  // window too wide: status set, stop
            const int T = 2 * (m - 1);
            const int tA = (int)((long long)T * w / nw), tB = (int)((long long)T * (w + 1) / nw);
            long long *gset = pa.gin + (size_t)set * 2 * a.Wcap;
            const Chunking ck = worker_chunking(tB - tA, P, umax);
            const int per_term = ck.H * P;
            const int tbw = max(1, min(a.tb, umax / per_term));
            for (int tb0 = tA; tb0 < tB; tb0 += tbw) {
                const int nt = min(tbw, tB - tb0);
                const int U = nt * per_term;
                // per-slot term info and source rows
                if (threadIdx.x < nt) {
                    int tg, neg, ac, ai, bc, bi;
                    inner_term(m, tb0 + threadIdx.x, tg, neg, ac, ai, bc, bi);
                    int fa = S.flgT[ac * N1 + ai], fb = S.flgT[bc * N1 + bi];
                    bool skip = !(fa & F_NZ) || !(fb & F_NZ);
                    int off = 0;
                    if (!skip) {
                        long long lp = (long long)S.expT[ac * N1 + ai] + S.expT[bc * N1 + bi] - 2LL * a.L;
                        off = (int)(lp - ((long long *)(S.misc + MS_IBASE))[tg]);
                    }
                    int sgn = neg ^ (fa & F_NEG) ^ (fb & F_NEG);
                    S.tinfo[4 * threadIdx.x] = off;
                    S.tinfo[4 * threadIdx.x + 1] = (skip ? 4 : 0) | (sgn ? 1 : 0) | (tg << 4);
                    S.tinfo[4 * threadIdx.x + 2] = ac * N1 + ai;
                    S.tinfo[4 * threadIdx.x + 3] = bc * N1 + bi;
                }
                __syncthreads();
                // stage alpha_a (A layout) and gamma/beta_{m-a} (C layout): all
                // loads of a thread are issued before its stores
                {
                    const int total = nt * 2 * Lp;
                    for (int e0 = 0; e0 < total; e0 += NT * 8) {
                        uint32_t v[8];
                        int dst[8];
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            const int e = e0 + k * NT + threadIdx.x;
                            dst[k] = -1;
                            v[k] = 0u;
                            if (e < total) {
                                const int slot = e / (2 * Lp), r = e - slot * 2 * Lp;
                                const int which = r >= Lp, x = r - which * Lp;
                                const int row = S.tinfo[4 * slot + 2 + which];
                                v[k] = __ldcg(&a.coefL[(size_t)row * Lp + x]);
                                dst[k] = slot * SL + (which ? S.AV : 0) + phys(x);
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 8; k++)
                            if (dst[k] >= 0) S.wvec[dst[k]] = v[k];
                    }
                }
                __syncthreads();
                pr.mark(PR_STAGE);
                // units (chunk h, pair q, product tl): u = (h P + q) nt + tl
                for (int u = threadIdx.x; u < U; u += NT) {
                    const int tl = u % nt;
                    const int hq = u / nt;
                    const int h = hq / P, q = hq - h * P;
                    const int fl = S.tinfo[4 * tl + 1];
                    long long v1[W + 2], v2[W + 2];
                    if (fl & 4) {
#pragma unroll
                        for (int t = 0; t < W + 2; t++) v1[t] = v2[t] = 0;
                    } else {
                        const int s0 = h * ck.CL, s1 = min(s0 + ck.CL, (P + 1) * W);
                        const uint32_t *Av = S.wvec + (size_t)tl * SL;
                        mac_unit_vals<false>(Av, Av + S.AV, q, s0, s1, Lp, S.M, v1, v2);
                        if (fl & 1) {
#pragma unroll
                            for (int t = 0; t < W + 2; t++) {
                                v1[t] = -v1[t];
                                v2[t] = -v2[t];
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < W + 2; t++) {
                        S.stage[(size_t)t * ustride + u] = v1[t];
                        S.stage[(size_t)(W + 2 + t) * ustride + u] = v2[t];
                    }
                }
                __syncthreads();
                pr.mark(PR_MAC);
                // reduction: every (pair q, block b, digit k) sums the chunks
                // of each product with the same target and offset and adds the
                // sum at column off + b Lp + q W + k of the shared window
                for (int cb = threadIdx.x; cb < P * 2 * (W + 2); cb += NT) {
                    const int q = cb / (2 * (W + 2)), r = cb - q * 2 * (W + 2);
                    const int b = r / (W + 2), k = r - b * (W + 2);
                    const long long *st = S.stage + (size_t)r * ustride + (size_t)q * nt;
                    long long sum = 0;
                    int cur_tg = -1, cur_off = 0;
                    for (int tl = 0; tl < nt; tl++) {
                        const int fl = S.tinfo[4 * tl + 1];
                        if (fl & 4) continue;
                        const int tg = (fl >> 4) & 3, off = S.tinfo[4 * tl];
                        if (tg != cur_tg || off != cur_off) {
                            if (sum)
                                atomicAdd((unsigned long long *)&S.wwin[(size_t)(cur_tg - 1) * S.wsz +
                                                                      wphys(cur_off + b * Lp + q * W + k)],
                                          (unsigned long long)sum);
                            sum = 0;
                            cur_tg = tg;
                            cur_off = off;
                        }
                        for (int h = 0; h < ck.H; h++) sum += st[(size_t)h * P * nt + tl];
                    }
                    if (sum)
                        atomicAdd((unsigned long long *)&S.wwin[(size_t)(cur_tg - 1) * S.wsz +
                                                              wphys(cur_off + b * Lp + q * W + k)],
                                  (unsigned long long)sum);
                }
                __syncthreads();
                pr.mark(PR_FLUSH);
            }
            // the shared windows into the global set
            for (int tg = 1; tg <= 2; tg++) {
                const int wd = S.misc[MS_IWIDTH + tg];
                long long *src = S.wwin + (size_t)(tg - 1) * S.wsz;
                for (int c = threadIdx.x; c < wd; c += NT) {
                    const long long v = src[wphys(c)];
                    if (v) {
                        atomicAdd((unsigned long long *)&gset[(size_t)(tg - 1) * a.Wcap + c],
                                  (unsigned long long)v);
                        src[wphys(c)] = 0;
                    }
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&pa.done[set], 1u);
            }
        }
    }
}

// --------------------------------------------------------------- closer (cluster)

struct OTerm {
    int kind;   // 0 dense product, 1 one-limb parameter times a number, 2 lone number
    int tg, neg;
    int aslot, bslot;  // A slot (product / scaled source / lone number), C slot (product)
    long long lp;      // lowest limb position of the term
    uint32_t v;        // one-limb multiplier
};

// The terms of Eq. (3)'s brackets at index m that involve coefficient m
// (all of them for m = 0).  Operands are in the closer's slots.
__device__ int outer_terms(PSmem &S, const KArgs &a, int m, OTerm *ot)
{
    const int N1 = a.N + 1;
    const int eA0 = S.expT[0 * N1], fA0 = S.flgT[0 * N1];
    const int eB0 = S.expT[1 * N1], fB0 = S.flgT[1 * N1];
    const int eG0 = S.expT[2 * N1], fG0 = S.flgT[2 * N1];
    const int eAm = S.expT[0 * N1 + m], fAm = S.flgT[0 * N1 + m];
    const int eBm = S.expT[1 * N1 + m], fBm = S.flgT[1 * N1 + m];
    const int eGm = S.expT[2 * N1 + m], fGm = S.flgT[2 * N1 + m];
    int n = 0;
    auto prod = [&](int tg, int neg, int aslot, int ea, int fa, int bslot, int eb, int fb) {
        if (!(fa & F_NZ) || !(fb & F_NZ)) return;
        OTerm t;
        t.kind = 0;
        t.tg = tg;
        t.neg = neg ^ (fa & F_NEG) ^ (fb & F_NEG);
        t.aslot = aslot;
        t.bslot = bslot;
        t.lp = (long long)ea + eb - 2LL * a.L;
        t.v = 0;
        ot[n++] = t;
    };
    auto param = [&](int tg, int neg, int p, int aslot_p, int src_aslot, int src_cslot, int ec,
                     int fc) {
        const int pe = __ldg(&a.parE[p]), pf = __ldg(&a.parF[p]);
        if (!(pf & F_NZ) || !(fc & F_NZ)) return;
        const int i0 = S.misc[MS_PSCAL + 2 * p];
        if (i0 >= 0) {  // one non-zero limb v at index i0: v * c shifted
            OTerm t;
            t.kind = 1;
            t.tg = tg;
            t.neg = neg ^ (pf & F_NEG) ^ (fc & F_NEG);
            t.aslot = src_aslot;
            t.bslot = -1;
            t.lp = (long long)pe - a.L + i0 + (long long)ec - a.L;
            t.v = (uint32_t)S.misc[MS_PSCAL + 2 * p + 1];
            ot[n++] = t;
        } else {
            prod(tg, neg, aslot_p, pe, pf, src_cslot, ec, fc);
        }
    };
    if (m == 0) {
        prod(1, 1, A_ALPHA0, eA0, fA0, C_GAMMA0, eG0, fG0);
        prod(2, 0, A_ALPHA0, eA0, fA0, C_BETA0, eB0, fB0);
    } else {
        prod(1, 1, A_ALPHAM, eAm, fAm, C_GAMMA0, eG0, fG0);
        prod(1, 1, A_ALPHA0, eA0, fA0, C_GAMMAM, eGm, fGm);
        prod(2, 0, A_ALPHAM, eAm, fAm, C_BETA0, eB0, fB0);
        prod(2, 0, A_ALPHA0, eA0, fA0, C_BETAM, eBm, fBm);
    }
    {
        const int pe = __ldg(&a.parE[P_B]), pf = __ldg(&a.parF[P_B]);
        prod(2, 1, A_B, pe, pf, C_GAMMAM, eGm, fGm);
    }
    param(0, 0, P_SIGMA, A_SIGMA, A_BETAM, C_BETAM, eBm, fBm);
    param(0, 1, P_SIGMA, A_SIGMA, A_ALPHAM, C_ALPHAM, eAm, fAm);
    param(1, 0, P_R, A_R, A_ALPHAM, C_ALPHAM, eAm, fAm);
    if (fBm & F_NZ) {
        OTerm t;
        t.kind = 2;
        t.tg = 1;
        t.neg = 1 ^ (fBm & F_NEG);
        t.aslot = A_BETAM;
        t.bslot = -1;
        t.lp = (long long)eBm - a.L;
        t.v = 0;
        ot[n++] = t;
    }
    return n;
}

__device__ __forceinline__ long long term_top(const OTerm &t, int Lp)
{
    return t.kind == 0 ? t.lp + 2LL * Lp + 2 : t.lp + Lp + 2;
}

// outer units of the cluster CTAs 1..C-1 (CTA 0 only combines)
__device__ void outer_units(PSmem &S, const KArgs &a, const OTerm *ot, int nterm, int rank, int C)
{
    const int P = a.P, Lp = a.Lp;
    int nd = 0;
    for (int k = 0; k < nterm; k++) nd += ot[k].kind == 0;
    const Chunking ck = chunking((long long)max(nd, 1) * P, (long long)(C - 1) * NT, P);
    const long long Ud = (long long)nd * ck.H * P;
    const long long U = Ud + (long long)(nterm - nd) * P;
    const long long u0 = U * (rank - 1) / (C - 1), u1 = U * rank / (C - 1);
    for (long long u = u0 + threadIdx.x; u < u1; u += NT) {
        int k, h = 0, q;
        if (u < Ud) {
            int di = (int)(u / ((long long)ck.H * P));
            int rem = (int)(u - (long long)di * ck.H * P);
            h = rem / P;
            q = rem - h * P;
            // di-th dense term
            k = 0;
            for (int c = 0;; k++)
                if (ot[k].kind == 0 && c++ == di) break;
        } else {
            int si = (int)((u - Ud) / P);
            q = (int)(u - Ud - (long long)si * P);
            k = 0;
            for (int c = 0;; k++)
                if (ot[k].kind != 0 && c++ == si) break;
        }
        const OTerm &t = ot[k];
        long long *win = S.win + (size_t)t.tg * S.wsz;
        const int off = (int)(t.lp - ll_at(S.misc, MS_OBASE + 2 * t.tg));
        const uint32_t *Av = S.vec + (size_t)t.aslot * S.AV;
        if (t.kind == 0) {
            const uint32_t *Cv = S.vec + (size_t)NA * S.AV + (size_t)t.bslot * S.CV;
            const int s0 = h * ck.CL, s1 = min(s0 + ck.CL, (P + 1) * W);
            mac_unit<false>(Av, Cv, q, s0, s1, Lp, S.M, win, off, t.neg);
        } else if (t.kind == 1) {
            scaled_unit(t.v, Av, q, win, off, t.neg);
        } else {
            add_unit(Av, q, win, off, t.neg);
        }
    }
}

// combined window of each target from the outer and the inner bases
__device__ void combine_bases(PSmem &S, const KArgs &a, bool have_inner)
{
    if (threadIdx.x < 3) {
        const int t = threadIdx.x;
        const int ow = S.misc[MS_OWIDTH + t], iw = have_inner ? S.misc[MS_IWIDTH + t] : 0;
        const long long ob = ll_at(S.misc, MS_OBASE + 2 * t), ib = ll_at(S.misc, MS_IBASE + 2 * t);
        long long lo = LLONG_MAX, hi = LLONG_MIN;
        if (ow) {
            lo = min(lo, ob);
            hi = max(hi, ob + ow);
        }
        if (iw) {
            lo = min(lo, ib);
            hi = max(hi, ib + iw);
        }
        int width = 0;
        if (hi > lo) {
            if (hi - lo > a.Wcap) {
                atomicCAS(a.status, 0, DEV_ERANGE);
                S.misc[MS_STATUS] = DEV_ERANGE;
            } else {
                width = (int)(hi - lo);
            }
        }
        ll_at(S.misc, MS_BASE + 2 * t) = (hi > lo) ? lo : 0;
        S.misc[MS_WIDTH + t] = width;
    }
}

// Sum the outer windows of CTAs 1..C-1 into CTA 0's combined windows; every
// CTA of the cluster takes a slice of the columns.
__device__ void reduce_outer(PSmem &S, const KArgs &a, cg::cluster_group &cl, int rank, int C)
{
    int *misc0 = cl.map_shared_rank(S.misc, 0);
    long long *comb0 = cl.map_shared_rank(S.comb, 0);
    for (int t = 0; t < 3; t++) {
        const int ow = S.misc[MS_OWIDTH + t];
        if (!ow) continue;
        const long long shift = ll_at(S.misc, MS_OBASE + 2 * t) - ll_at(misc0, MS_BASE + 2 * t);
        const int c0 = ow * rank / C, c1 = ow * (rank + 1) / C;
        for (int c = c0 + threadIdx.x; c < c1; c += NT) {
            long long v = 0;
#pragma unroll
            for (int r = 1; r < CP_C; r++) {
                long long *wr = cl.map_shared_rank(S.win, r);
                v += wr[(size_t)t * S.wsz + wphys(c)];
            }
            if (v) {
                long long *dst = comb0 + (size_t)t * S.wsz + wphys((int)(c + shift));
                *dst += v;
            }
        }
    }
}

// close the three brackets in CTA 0 (warps 0..2): normalise, divide by d
// (d = 1 truncates), write limbs to newc[t], return via misc exps/flags
__device__ void close_three(PSmem &S, const KArgs &a, uint32_t d, int *outE, int *outF)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp < 3) {
        const int t = warp;
        const int wd = S.misc[MS_WIDTH + t];
        uint32_t *out = S.newc + (size_t)t * a.Lp;
        int e = 0, f = 0;
        if (wd > 0) {
            uint32_t *dig = S.dig + (size_t)t * a.Wcap;
            long long *col = S.comb + (size_t)t * S.wsz;
            Norm nr = warp_normalize(col, dig, wd, a.status);
            for (int c = lane; c < wd; c += 32) col[wphys(c)] = 0;
            if (nr.top >= 0) {
                long long eq = warp_divide(dig, nr.top, ll_at(S.misc, MS_BASE + 2 * t), d, a.L, out);
                if (eq > (1LL << 30) || eq < -(1LL << 30)) {
                    if (lane == 0) atomicCAS(a.status, 0, DEV_ERANGE);
                    eq = 0;
                }
                e = (int)eq;
                f = F_NZ | (nr.neg ? F_NEG : 0);
            }
        }
        if (!(f & F_NZ))
            for (int x = lane; x < a.L; x += 32) out[x] = 0u;
        for (int x = a.L + lane; x < a.Lp; x += 32) out[x] = 0u;
        __syncwarp();
        if (lane == 0) {
            outE[t] = e;
            outF[t] = f;
        }
    }
}

// copy the newest number (3 components, plain limbs in CTA 0's newc) into
// this CTA's slots in A and C layout
__device__ void pull_newest(PSmem &S, const KArgs &a, cg::cluster_group &cl, bool coefficient)
{
    const uint32_t *src = cl.map_shared_rank(S.newc, 0);
    const int Lp = a.Lp;
    uint32_t *A = S.vec, *Cb = S.vec + (size_t)NA * S.AV;
    for (int e = threadIdx.x; e < 3 * Lp; e += NT) {
        const int comp = e / Lp, x = e - comp * Lp;
        const uint32_t v = src[e];
        if (coefficient) {
            if (comp == 0) {
                A[(size_t)A_ALPHAM * S.AV + phys(x)] = v;
                Cb[(size_t)C_ALPHAM * S.CV + phys(x)] = v;
            } else if (comp == 1) {
                A[(size_t)A_BETAM * S.AV + phys(x)] = v;
                Cb[(size_t)C_BETAM * S.CV + phys(x)] = v;
            } else {
                Cb[(size_t)C_GAMMAM * S.CV + phys(x)] = v;
            }
        } else {
            Cb[(size_t)(C_H0 + comp) * S.CV + phys(x)] = v;
        }
    }
}

// One Horner chain of Eq. (2) for component c, in one CTA: h_N = c_N,
// h_i = trunc_L(tau h_{i+1} + c_i) for i = N-1 .. 0, then the new state (and
// a record).  The product tau h is split into (chunk, pair) units, one per
// thread; their column digits are staged and summed per (pair, block, digit)
// into the window, c_i (prefetched from global one step ahead) is added, and
// warp 0 normalises and truncates.
__device__ void horner_component(PSmem &S, const KArgs &a, int c, long long step, Prof &pr)
{
    const int N1 = a.N + 1, Lp = a.Lp, L = a.L, P = a.P;
    const int cslot = c == 0 ? C_ALPHAM : (c == 1 ? C_BETAM : C_GAMMAM);
    uint32_t *hC = S.vec + (size_t)NA * S.AV + (size_t)cslot * S.CV;  // h in C layout
    const uint32_t *tauA = S.vec + (size_t)A_TAU * S.AV;
    uint32_t *hp = S.newc + (size_t)c * Lp;                           // h, plain limbs
    long long *win = S.win;
    const int tauE = __ldg(&a.parE[P_TAU]), tauF = __ldg(&a.parF[P_TAU]);
    // chunks: at most one unit per thread
    int He = HU / P;
    if (He < 1) He = 1;
    if (He > P + 1) He = P + 1;
    const int CL = ((P + 1 + He - 1) / He) * W;
    He = ((P + 1) * W + CL - 1) / CL;
    const int U = P * He;
    int *hE = S.misc + MS_HE + c, *hF = S.misc + MS_HF + c;
    if (threadIdx.x == 0) {
        *hE = S.expT[c * N1 + a.N];
        *hF = S.flgT[c * N1 + a.N];
    }
    for (int x = threadIdx.x; x < Lp; x += NT) hp[x] = hC[phys(x)];
    uint32_t cur[4], nxt[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int x = threadIdx.x + r * NT;
        cur[r] = (x < Lp && a.N >= 1) ? __ldcg(&a.coefL[((size_t)c * N1 + a.N - 1) * Lp + x]) : 0u;
    }
    __syncthreads();
    for (int i = a.N - 1; i >= 0; i--) {
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int x = threadIdx.x + r * NT;
            nxt[r] = (i > 0 && x < Lp) ? __ldcg(&a.coefL[((size_t)c * N1 + i - 1) * Lp + x]) : 0u;
        }
        // window: the product tau h and the lone c_i
        const int he = *hE, hf = *hF;
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
                if (threadIdx.x == 0) {
                    atomicCAS(a.status, 0, DEV_ERANGE);
                    S.misc[MS_HERR] = 1;
                }
                break;  // uniform: every thread computed the same width
            }
            width = (int)(hi - lo);
        }
        const int offp = (int)(lpp - lo), offa = (int)(lpa - lo);
        const bool pneg = ((hf ^ tauF) & F_NEG) != 0;
        if (prod && threadIdx.x < U) {
            const int h = threadIdx.x / P, q = threadIdx.x - h * P;
            const int s0 = h * CL, s1 = min(s0 + CL, (P + 1) * W);
            long long v1[W + 2], v2[W + 2];
            mac_unit_vals<false>(tauA, hC, q, s0, s1, Lp, S.M, v1, v2);
#pragma unroll
            for (int t = 0; t < W + 2; t++) {
                S.hstage[(size_t)t * (HU + 1) + threadIdx.x] = pneg ? -v1[t] : v1[t];
                S.hstage[(size_t)(W + 2 + t) * (HU + 1) + threadIdx.x] = pneg ? -v2[t] : v2[t];
            }
        }
        __syncthreads();
        pr.mark(PR_HMAC);
        if (prod) {
            for (int cb = threadIdx.x; cb < P * 2 * (W + 2); cb += NT) {
                const int q = cb / (2 * (W + 2)), r = cb - q * 2 * (W + 2);
                const int b = r / (W + 2), k = r - b * (W + 2);
                long long sum = 0;
                for (int h = 0; h < He; h++) sum += S.hstage[(size_t)r * (HU + 1) + h * P + q];
                if (sum)
                    atomicAdd((unsigned long long *)&win[wphys(offp + b * Lp + q * W + k)],
                              (unsigned long long)sum);
            }
        }
        if (lone) {
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int x = threadIdx.x + r * NT;
                if (x < Lp && cur[r]) {
                    const long long v = (cf & F_NEG) ? -(long long)cur[r] : (long long)cur[r];
                    atomicAdd((unsigned long long *)&win[wphys(offa + x)], (unsigned long long)v);
                }
            }
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int e = 0, f = 0;
            if (width > 0) {
                Norm nr = warp_normalize(win, S.dig, width, a.status);
                for (int cc = lane; cc < width; cc += 32) win[wphys(cc)] = 0;
                if (nr.top >= 0) {
                    long long eq = warp_divide(S.dig, nr.top, lo, 1u, L, hp);
                    if (eq > (1LL << 30) || eq < -(1LL << 30)) {
                        if (lane == 0) {
                            atomicCAS(a.status, 0, DEV_ERANGE);
                            S.misc[MS_HERR] = 1;
                        }
                        eq = 0;
                    }
                    e = (int)eq;
                    f = F_NZ | (nr.neg ? F_NEG : 0);
                }
            }
            if (!(f & F_NZ))
                for (int x = lane; x < L; x += 32) hp[x] = 0u;
            __syncwarp();
            for (int x = lane; x < Lp; x += 32) hC[phys(x)] = x < L ? hp[x] : 0u;
            if (lane == 0) {
                *hE = e;
                *hF = f;
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) cur[r] = nxt[r];
        __syncthreads();
        pr.mark(PR_HCLOSE);
        if (S.misc[MS_HERR]) break;
    }
    // the new state and, when due, a record
    const long long rec = (a.record_every > 0 && ((step + 1) % a.record_every) == 0)
                              ? (step + 1) / a.record_every - 1 : -1;
    for (int x = threadIdx.x; x < Lp; x += NT) {
        a.stL[(size_t)c * Lp + x] = hp[x];
        if (rec >= 0 && x < L) a.recL[((size_t)rec * 3 + c) * L + x] = hp[x];
    }
    if (threadIdx.x == 0) {
        a.stE[c] = *hE;
        a.stF[c] = *hF;
        if (rec >= 0) {
            a.recS[rec * 3 + c] = (*hF & F_NEG) ? 1 : 0;
            a.recE[rec * 3 + c] = *hE;
        }
    }
    __threadfence();
}

__device__ void closer_loop(PSmem &S, const KArgs &a, const PArgs &pa)
{
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int C = CP_C;
    const int N1 = a.N + 1, Lp = a.Lp, L = a.L;
    uint32_t *A = S.vec, *Cb = S.vec + (size_t)NA * S.AV;
    OTerm *ot = (OTerm *)(S.tinfo);  // up to 10 terms (tinfo holds >= 64 x 4 ints)
    const bool prof_on = (rank == 0);
    int *misc0 = cl.map_shared_rank(S.misc, 0);
    // zero windows and C padding; parameters into A slots
    for (int e = threadIdx.x; e < 3 * S.wsz; e += NT) {
        S.win[e] = 0;
        S.comb[e] = 0;
    }
    for (int e = threadIdx.x; e < NC * S.M; e += NT) {
        int slot = e / S.M, x = e - slot * S.M;
        if (x >= Lp) Cb[(size_t)slot * S.CV + phys(x)] = 0u;
    }
    for (int e = threadIdx.x; e < 4 * Lp; e += NT) {
        int p = e / Lp, x = e - p * Lp;
        A[(size_t)p * S.AV + phys(x)] = __ldg(&a.parL[(size_t)p * Lp + x]);  // A_SIGMA.. = P_*
    }
    if (threadIdx.x < 3) {
        // single non-zero limb of sigma, R, b (else -1)
        const int p = threadIdx.x;
        int cnt = 0, i0 = -1;
        uint32_t v = 0;
        for (int x = 0; x < Lp; x++) {
            uint32_t l = __ldg(&a.parL[(size_t)p * Lp + x]);
            if (l) {
                cnt++;
                i0 = x;
                v = l;
            }
        }
        S.misc[MS_PSCAL + 2 * p] = cnt == 1 ? i0 : -1;
        S.misc[MS_PSCAL + 2 * p + 1] = (int)v;
    }
    if (rank == 0 && threadIdx.x == 0) {
        S.misc[MS_ERR_A] = 0;
        S.misc[MS_ERR_C] = 0;
    }
    cl.sync();
    // stop: the cluster-wide decision to end the launch.  It is only ever read
    // from CTA 0's shared memory between two cluster barriers, so every CTA of
    // the cluster takes the same branch, and the launch leaves through one
    // final cluster barrier: no CTA exits while a peer may still read its
    // shared memory.
    bool stop = false;
    for (long long step = 0; step < a.nsteps && !stop; step++) {
        // the state is coefficient 0 (Sec. 2): into every CTA's slots and tables
        for (int e = threadIdx.x; e < 3 * Lp; e += NT) {
            const int comp = e / Lp, x = e - comp * Lp;
            const uint32_t v = __ldcg(&a.stL[e]);
            if (comp == 0) {
                A[(size_t)A_ALPHA0 * S.AV + phys(x)] = v;
                A[(size_t)A_ALPHAM * S.AV + phys(x)] = v;
                Cb[(size_t)C_ALPHAM * S.CV + phys(x)] = v;
            } else if (comp == 1) {
                Cb[(size_t)C_BETA0 * S.CV + phys(x)] = v;
                A[(size_t)A_BETAM * S.AV + phys(x)] = v;
                Cb[(size_t)C_BETAM * S.CV + phys(x)] = v;
            } else {
                Cb[(size_t)C_GAMMA0 * S.CV + phys(x)] = v;
                Cb[(size_t)C_GAMMAM * S.CV + phys(x)] = v;
            }
            if (rank == 0) a.coefL[(size_t)comp * N1 * Lp + x] = v;
        }
        if (threadIdx.x < 3) {
            const int e = __ldcg(&a.stE[threadIdx.x]), f = __ldcg(&a.stF[threadIdx.x]);
            S.expT[threadIdx.x * N1] = e;
            S.flgT[threadIdx.x * N1] = f;
            if (rank == 0) {
                a.coefE[threadIdx.x * N1] = e;
                a.coefF[threadIdx.x * N1] = f;
            }
        }
        __syncthreads();
        for (int m = 0; m < a.N; m++) {
            Prof pr(a, prof_on, S.misc);
            const long long g = step * a.N + m;
            const int set = (int)(g % PIPE_SETS);
            const bool have_inner = m >= 2;
            // (A) outer terms and their windows; CTA 0 also places the inner
            // windows and fetches the workers' inner sums
            if (threadIdx.x == 0) {
                S.misc[MS_NTERM] = outer_terms(S, a, m, ot);
                S.misc[MS_STATUS] = 0;
            }
            __syncthreads();
            const int nterm = S.misc[MS_NTERM];
            {
                long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
                long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
                if (threadIdx.x == 0)
                    for (int k = 0; k < nterm; k++) {
                        lo[ot[k].tg] = min(lo[ot[k].tg], ot[k].lp);
                        hi[ot[k].tg] = max(hi[ot[k].tg], term_top(ot[k], Lp));
                    }
                block_window(S, a, lo, hi, MS_OBASE, MS_OWIDTH);
            }
            if (rank == 0) {
                if (have_inner) inner_windows(S, a, m, MS_IBASE, MS_IWIDTH);
                combine_bases(S, a, have_inner);
                __syncthreads();
                pr.mark(PR_PLACE);
                const bool bad = S.misc[MS_STATUS] != 0;
                if (have_inner && !bad) {
                    // every worker has added its inner sums of index m
                    const unsigned target =
                        (unsigned)((g / PIPE_SETS + 1) * (long long)(gridDim.x - CP_C));
                    const bool ok = wait_geq(S, a, pa.done + set, target);
                    pr.mark(PR_BARRIER);
                    if (ok) {
                        const long long *gs = pa.gin + (size_t)set * 2 * a.Wcap;
                        for (int t = 1; t <= 2; t++) {
                            const int iw = S.misc[MS_IWIDTH + t];
                            const long long shift =
                                ll_at(S.misc, MS_IBASE + 2 * t) - ll_at(S.misc, MS_BASE + 2 * t);
                            long long *gg = (long long *)gs + (size_t)(t - 1) * a.Wcap;
                            for (int c0 = 0; c0 < iw; c0 += 4 * NT) {
                                long long v[4];
#pragma unroll
                                for (int k = 0; k < 4; k++) {
                                    const int c = c0 + k * NT + threadIdx.x;
                                    v[k] = c < iw ? __ldcg(&gg[c]) : 0;
                                }
#pragma unroll
                                for (int k = 0; k < 4; k++) {
                                    const int c = c0 + k * NT + threadIdx.x;
                                    if (v[k]) {
                                        S.comb[(size_t)t * S.wsz + wphys((int)(c + shift))] += v[k];
                                        gg[c] = 0;
                                    }
                                }
                            }
                        }
                    }
                    pr.mark(PR_STAGE);
                }
                if (threadIdx.x == 0) S.misc[MS_ERR_A] = bad || ld_relaxed_int(a.status) != 0;
            } else if (S.misc[MS_STATUS] == 0) {
                outer_units(S, a, ot, nterm, rank, C);
            }
            cl.sync();  // #1: outer partial windows and the inner sums are in place
            pr.mark(PR_MAC);
            stop = misc0[MS_ERR_A] != 0;
            if (!stop) reduce_outer(S, a, cl, rank, C);
            pr.mark(PR_X1);
            cl.sync();  // #2: CTA 0 holds the full brackets
            pr.mark(PR_X2);
            if (stop) break;
            for (int e = threadIdx.x; e < 3 * S.wsz; e += NT) S.win[e] = 0;
            pr.mark(PR_FLUSH);
            if (rank == 0) {
                int *eo = S.misc + MS_HE, *fo = S.misc + MS_HF;
                close_three(S, a, (uint32_t)(m + 1), eo, fo);
                __syncthreads();
                pr.mark(PR_X5);
                if (threadIdx.x < 3) {
                    S.expT[threadIdx.x * N1 + m + 1] = eo[threadIdx.x];
                    S.flgT[threadIdx.x * N1 + m + 1] = fo[threadIdx.x];
                    a.coefE[threadIdx.x * N1 + m + 1] = eo[threadIdx.x];
                    a.coefF[threadIdx.x * N1 + m + 1] = fo[threadIdx.x];
                }
                for (int e = threadIdx.x; e < 3 * Lp; e += NT) {
                    const int comp = e / Lp, x = e - comp * Lp;
                    a.coefL[((size_t)comp * N1 + m + 1) * Lp + x] = S.newc[e];
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    __threadfence();
                    st_release_u32(pa.pub, (unsigned)(step * N1 + m + 2));
                    S.misc[MS_ERR_C] = ld_relaxed_int(a.status) != 0;
                }
            }
            pr.mark(PR_CLOSE);
            cl.sync();  // #3: coefficient m+1 is in CTA 0's newc
            pr.mark(PR_X3);
            stop = misc0[MS_ERR_C] != 0;
            if (stop) break;
            pull_newest(S, a, cl, true);
            if (threadIdx.x < 3 && rank != 0) {
                S.expT[threadIdx.x * N1 + m + 1] = misc0[MS_HE + threadIdx.x];
                S.flgT[threadIdx.x * N1 + m + 1] = misc0[MS_HF + threadIdx.x];
            }
            __syncthreads();
            pr.mark(PR_X4);
        }
        if (stop) break;
        // Horner (Eq. (2)), one component per CTA (ranks 0..2), no cluster
        // barrier inside: h_N = c_N, h_i = trunc_L(tau h_{i+1} + c_i)
        Prof ph(a, prof_on, S.misc);
        if (threadIdx.x == 0) S.misc[MS_HERR] = 0;
        __syncthreads();
        if (rank < 3) horner_component(S, a, rank, step, ph);
        __syncthreads();
        ph.mark(PR_HORNER);
        cl.sync();  // the new state is in global memory
        {
            // stop if any component failed (each CTA reads the same three flags)
            int bad = 0;
            for (int r = 0; r < 3; r++) bad |= cl.map_shared_rank(S.misc, r)[MS_HERR];
            stop = bad != 0;
        }
        cl.sync();  // flags read; the next step may reuse them
    }
    cl.sync();  // the only way out of the closer
}

__global__ void __launch_bounds__(NT, 1) pipe_kernel(KArgs a, PArgs pa)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PSmem S;
    pipe_layout(a.Lp, a.N, a.Wcap, a.tb, pa.umax, &S, smem_raw);
    const bool prof_cta = blockIdx.x == 0 || blockIdx.x == gridDim.x - 1;
    if (threadIdx.x < PROF_SLOTS) ((long long *)(S.misc + MS_PROF))[threadIdx.x] = 0;
    __syncthreads();
    Prof tot(a, prof_cta, S.misc);
    if (blockIdx.x < (unsigned)CP_C)
        closer_loop(S, a, pa);
    else
        worker_loop(S, a, pa);
    tot.mark(PR_TOTAL);
    if (a.prof && prof_cta && threadIdx.x == 0) {
        long long *dst = a.prof + (blockIdx.x == 0 ? 0 : PROF_SLOTS);
        for (int k = 0; k < PROF_SLOTS; k++) dst[k] += ((long long *)(S.misc + MS_PROF))[k];
    }
}

}  // namespace

size_t pipe_smem_bytes(int Lp, int N, int Wcap, int tb, int umax)
{
    return pipe_layout(Lp, N, Wcap, tb, umax, nullptr, nullptr);
}

static cudaLaunchConfig_t pipe_config(int grid, int C, size_t smem, cudaStream_t st,
                                      cudaLaunchAttribute *attrs, bool coop)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attrs[0].id = cudaLaunchAttributeClusterDimension;
    attrs[0].val.clusterDim.x = C;
    attrs[0].val.clusterDim.y = 1;
    attrs[0].val.clusterDim.z = 1;
    cfg.attrs = attrs;
    cfg.numAttrs = 1;
    if (coop) {
        attrs[1].id = cudaLaunchAttributeCooperative;
        attrs[1].val.cooperative = 1;
        cfg.numAttrs = 2;
    }
    return cfg;
}

int pipe_max_clusters(int C, size_t smem)
{
    if (cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    if (C > 8 &&
        cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess)
        return 0;
    cudaLaunchAttribute attrs[2];
    cudaLaunchConfig_t cfg = pipe_config(C, C, smem, 0, attrs, false);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (void *)pipe_kernel, &cfg) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_pipe(const KArgs &a, const PArgs &pa, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(pipe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attrs[2];
    cudaLaunchConfig_t cfg = pipe_config(grid, pa.C, smem, st, attrs, true);
    e = cudaLaunchKernelEx(&cfg, pipe_kernel, a, pa);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        // clusters without the cooperative guarantee: the grid is sized to the
        // device's active-cluster limit, and every wait is bounded
        cfg = pipe_config(grid, pa.C, smem, st, attrs, false);
        e = cudaLaunchKernelEx(&cfg, pipe_kernel, a, pa);
    }
    return e;
}

}  // namespace mpt
