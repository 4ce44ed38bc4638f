// mpt_step.cu -- the multiple-precision Taylor step for the Lorenz system on
// sm_103a: Eq. (3)'s coefficient recursion with its Cauchy sums, the
// division by (i+1), and Eq. (2) evaluated by Horner's rule (Sec. 2 of
// Dimova et al., arXiv 1908.09301).
//
// Layout and method (one persistent launch runs nsteps steps):
//  * Numbers are L 32-bit limbs (padded with zero limbs to Lp, a multiple of
//    W), an exponent in limbs and a flag word (sign, non-zero).  The
//    coefficients of the running step live in global memory (they stay in
//    L2); every CTA keeps the exponent and flag tables in shared memory.
//  * Coefficient index m (Eq. (3) with i = m) is a set of "terms": the
//    products of Eq. (3)'s brackets (sigma*beta_m, sigma*alpha_m, R*alpha_m,
//    b*gamma_m and the 2(m+1) Cauchy products alpha_{m-k}gamma_k,
//    alpha_{m-k}beta_k) plus the lone -beta_m.  Each term is an exact L x L
//    limb product added into one of three exact accumulators (X, Y, Z for
//    alpha, beta, gamma): int64 columns on the absolute 2^32 grid, with the
//    window placed from the terms' exponents.  The Cauchy-sum reduction the
//    paper parallelises over k with OpenMP (Sec. 3-4) is split here over
//    CTAs (contiguous term ranges), threads (column pairs of a product) and
//    registers (8-column Comba tiles with mad.lo.cc / madc.hi.cc / addc).
//    Integer addition is associative, so partial sums of any split add up to
//    the same exact value.
//  * After all CTAs have added their partial windows into global memory, a
//    grid barrier, then every CTA closes the three brackets redundantly:
//    carry-normalise the window (warp-level carry resolution), take sign and
//    magnitude, and divide by (m+1) with a warp-parallel long division (the
//    remainder passes from chunk to chunk as an affine map mod (m+1), composed
//    with a shuffle scan), truncating to L limbs.
//  * Horner: h_N = c_N, h_i = trunc_L(tau*h_{i+1} + c_i): the same exact
//    accumulator with a division by one, one CTA per component.
#include <cstdint>
#include <cuda_runtime.h>

#include "mpt_divisor.cuh"
#include "mpt_kernel.cuh"

namespace mpt {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ int phys(int x) { return x + (x >> 3); }

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

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *(volatile const int *)p;
}

__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// the grid the kernel runs as: the launch's, or one CTA per trajectory (batch)
__device__ __forceinline__ int vgrid(const KArgs &a) { return a.vG ? a.vG : (int)gridDim.x; }
__device__ __forceinline__ int vrank(const KArgs &a) { return a.vG ? a.vg : (int)blockIdx.x; }

// per-phase cycle counters (thread 0 of the first and the last CTA)
struct Prof {
    long long *p;
    long long t;
    __device__ Prof(const KArgs &a)
    {
        p = nullptr;
        t = 0;
        if (a.prof && threadIdx.x == 0 && (blockIdx.x == 0 || blockIdx.x == gridDim.x - 1))
            p = a.prof + (blockIdx.x == 0 ? 0 : PROF_SLOTS);
        if (p) t = clock64();
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

// ------------------------------------------------------------------ smem

struct Smem {
    long long *win;   // [3][Wcap]
    uint32_t *dig;    // [3][Wcap]
    int *expT;        // [3][N+1]
    int *flgT;        // [3][N+1]
    uint32_t *newc;   // [3][Lp]
    uint32_t *slots;  // [tb][AV + CV]
    int *tinfo;       // [tb][2]
    int *srcs;        // [tb][2] operand sources of the staged terms
    int *misc;        // [MISC_INTS]
    int *fexpT, *fflgT;  // reverse sweep: [3][N+1] the forward coefficients of the step
    int *pexpT, *pflgT;  // reverse sweep: [N+1] the powers of tau
    int AV, CV, M;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline void vec_sizes(int Lp, int &AV, int &CV, int &M)
{
    M = Lp + W;
    AV = Lp + Lp / 8 + 1;
    CV = M + M / 8 + 1;
}

// misc slots
enum {
    MS_BASE = 0,    // [3] long long window base (lowest limb position) per target: ints 0..5
    MS_WIDTH = 8,   // [3] window width (0 = no non-zero term)
    MS_RED = 16,    // [8 warps][6] long long reduction scratch -> ints 16..111
    MS_HE = 112,    // [3] Horner: exponent of h per local component
    MS_HF = 116,    // [3] Horner: flags of h
    MS_ERR = 120,   // status snapshot shared by the CTA
    MS_PNZ = 124,   // [SYS_MAX_PAR] non-zero limb count of each parameter
    MS_FWDOFF = MS_PNZ + SYS_MAX_PAR,  // long long (2 ints): limb offset of the step in fwdL
    MISC_INTS = MS_FWDOFF + 2,
};

// what an index of the lock-step body computes: Eq. (3) (forward); in the
// reverse sweep: a power of tau, an adjoint index, the parameter adjoints
enum { MODE_FWD = 0, MODE_POW = 1, MODE_ADJ = 2, MODE_PAR = 3 };

// The status word as one value for the whole CTA, so that every thread takes
// the same branch after it (a per-thread read could differ while another CTA
// is writing it).
__device__ __forceinline__ bool cta_ok(const Smem &S, const KArgs &a)
{
    __syncthreads();
    if (threadIdx.x == 0) S.misc[MS_ERR] = *(volatile const int *)a.status;
    __syncthreads();
    return S.misc[MS_ERR] == 0;
}

__device__ __forceinline__ int nwin_of(const KArgs &a) { return a.nwin > 1 ? a.nwin : 1; }

__device__ Smem carve(unsigned char *base, const KArgs &a)
{
    Smem S;
    vec_sizes(a.Lp, S.AV, S.CV, S.M);
    size_t o = 0;
    S.win = (long long *)(base + o);
    o = align16(o + sizeof(long long) * 3 * (size_t)nwin_of(a) * a.Wcap);
    S.dig = (uint32_t *)(base + o);
    o = align16(o + sizeof(uint32_t) * 3 * a.Wcap);
    S.expT = (int *)(base + o);
    o = align16(o + sizeof(int) * 3 * (a.N + 1));
    S.flgT = (int *)(base + o);
    o = align16(o + sizeof(int) * 3 * (a.N + 1));
    S.newc = (uint32_t *)(base + o);
    o = align16(o + sizeof(uint32_t) * 3 * a.Lp);
    S.slots = (uint32_t *)(base + o);
    o = align16(o + sizeof(uint32_t) * (size_t)a.tb * (S.AV + S.CV));
    S.tinfo = (int *)(base + o);
    o = align16(o + sizeof(int) * 2 * a.tb);
    S.srcs = (int *)(base + o);
    o = align16(o + sizeof(int) * 2 * a.tb);
    S.misc = (int *)(base + o);
    o = align16(o + sizeof(int) * MISC_INTS);
    S.fexpT = S.fflgT = S.pexpT = S.pflgT = nullptr;
    if (a.adj) {
        S.fexpT = (int *)(base + o);
        o = align16(o + sizeof(int) * 3 * (a.N + 1));
        S.fflgT = (int *)(base + o);
        o = align16(o + sizeof(int) * 3 * (a.N + 1));
        S.pexpT = (int *)(base + o);
        o = align16(o + sizeof(int) * (a.N + 1));
        S.pflgT = (int *)(base + o);
    }
    return S;
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

// ------------------------------------------------------------------ grid barrier

// Sense-free generation barrier over all CTAs of a cooperative launch.  The
// wait is bounded: on expiry the status word is set and every CTA unwinds.
__device__ bool grid_barrier(const Smem &S, const KArgs &a)
{
    Prof pr(a);
    __syncthreads();
    if (vgrid(a) > 1) {
        if (threadIdx.x == 0) {
            unsigned gen = ld_acquire(&a.bar[1]);
            __threadfence();
            unsigned arrived = atomicAdd(&a.bar[0], 1u);
            if (arrived == (unsigned)vgrid(a) - 1) {
                atomicExch(&a.bar[0], 0u);
                __threadfence();
                atomicAdd(&a.bar[1], 1u);
            } else {
                long long it = 0;
                while (ld_acquire(&a.bar[1]) == gen) {
                    if (++it > a.spin_limit) {
                        set_status(a.status, DEV_TIMEOUT);
                        break;
                    }
                    if ((it & 255) == 0 && ld_volatile_int(a.status) != 0) break;
                    __nanosleep(32);
                }
            }
        }
    }
    bool ok = cta_ok(S, a);
    pr.mark(PR_BARRIER);
    return ok;
}

// ------------------------------------------------------------------ terms of Eq. (3)

// source of an operand: >= 0 coefficient (comp * (N+1) + index); < 0 parameter -1-p
enum { P_SIGMA = 0, P_R = 1, P_B = 2, P_TAU = 3 };
enum { T_X = 0, T_Y = 1, T_Z = 2 };

struct Term {
    int target;  // 0 X (alpha), 1 Y (beta), 2 Z (gamma)
    int neg;     // the bracket subtracts this term
    int add;     // lone number (no product): c = bsrc
    int asrc, bsrc;
    int skip;    // no term at this index (a constant of the right-hand side, m > 0)
};

// Terms of the brackets of Eq. (3) at i = m (T = 2m + 7 of them):
//   X: +sigma beta_m, -sigma alpha_m
//   Y: +R alpha_m, -beta_m, -sum_{k=0}^{m} alpha_{m-k} gamma_k
//   Z: -b gamma_m, +sum_{k=0}^{m} alpha_{m-k} beta_k
__device__ __forceinline__ Term lorenz_term(int m, int t, int N1)
{
    Term r;
    r.add = 0;
    r.skip = 0;
    if (t == 0) { r.target = T_X; r.neg = 0; r.asrc = -1 - P_SIGMA; r.bsrc = 1 * N1 + m; }
    else if (t == 1) { r.target = T_X; r.neg = 1; r.asrc = -1 - P_SIGMA; r.bsrc = 0 * N1 + m; }
    else if (t == 2) { r.target = T_Y; r.neg = 0; r.asrc = -1 - P_R; r.bsrc = 0 * N1 + m; }
    else if (t == 3) { r.target = T_Y; r.neg = 1; r.add = 1; r.asrc = 0; r.bsrc = 1 * N1 + m; }
    else if (t == 4) { r.target = T_Z; r.neg = 1; r.asrc = -1 - P_B; r.bsrc = 2 * N1 + m; }
    else if (t <= 5 + m) {
        int k = t - 5;
        r.target = T_Y; r.neg = 1; r.asrc = 0 * N1 + (m - k); r.bsrc = 2 * N1 + k;
    } else {
        int k = t - 6 - m;
        r.target = T_Z; r.neg = 0; r.asrc = 0 * N1 + (m - k); r.bsrc = 1 * N1 + k;
    }
    return r;
}

// Terms of a general three-component quadratic system (the AD reading of
// Eq. (3), Sec. 2 after Fig. 1) at index m: the fixed terms first, each
// {target, neg, p, j} = p x_j (p >= 0, j >= 0), the lone x_j (p < 0) or the
// constant p (j < 0; index 0 only); then per Cauchy product {target, neg,
// i, j} its m+1 terms x_i[m-l] x_j[l], l = 0..m.  T = NF + NQ (m+1).
// operand sources of the reverse sweep beyond the coefficient (here: adjoint
// series) rows: the step's forward coefficients and the powers of tau
constexpr int SRC_FWD = 1 << 24, SRC_POW = 2 << 24;

// Terms of the reverse sweep (the adjoint of Eq. (3) and Eq. (2)).  The
// adjoint series is y_X[r] = Ebar_X,{N-1-r} for r < N (Ebar_X,i: the
// adjoint of the bracket of Eq. (3) that gives coefficient i+1) and y_X[N]
// the adjoint of the step's starting state; with j = N - m, index m is
//   y_x[m] = ( gbar_x P_j - sigma y_x[m-1] + R y_y[m-1]
//              + sum_{l<m} (-y_y[m-1-l] gamma_l + y_z[m-1-l] beta_l) ) / j
//   y_y[m] = ( gbar_y P_j + sigma y_x[m-1] - y_y[m-1] + sum_{l<m} y_z[m-1-l] alpha_l ) / j
//   y_z[m] = ( gbar_z P_j - b y_z[m-1] - sum_{l<m} y_y[m-1-l] alpha_l ) / j
// (divisor 1 at m = N; no y[m-1] terms at m = 0), the Cauchy sums of the
// brackets E_i, i >= j, read through their factor of index j.  MODE_POW:
// P_m = P_{m-1} tau.  MODE_PAR: thbar_sigma + sum_i Ebar_x,i (beta_i -
// alpha_i), thbar_R + sum_i Ebar_y,i alpha_i, thbar_b - sum_i Ebar_z,i gamma_i.
__device__ __forceinline__ Term adjoint_term(const KArgs &a, int mode, int m, int t, int N1)
{
    const int N = a.N;
    Term r;
    r.add = 0;
    r.skip = 0;
    r.neg = 0;
    if (mode == MODE_POW) {
        r.target = 0;
        r.asrc = SRC_POW + m - 1;
        r.bsrc = -1 - P_TAU;
        return r;
    }
    if (mode == MODE_PAR) {
        if (t < 3) {  // the running parameter adjoints
            r.target = t;
            r.add = 1;
            r.asrc = 0;
            r.bsrc = -1 - (ADJ_THBAR + t);
            return r;
        }
        const int u = t - 3, i = u >> 2, k = u & 3;
        const int yr = N - 1 - i;  // Ebar_i
        if (k == 0) { r.target = 0; r.asrc = 0 * N1 + yr; r.bsrc = SRC_FWD + 1 * N1 + i; }
        else if (k == 1) { r.target = 0; r.neg = 1; r.asrc = 0 * N1 + yr; r.bsrc = SRC_FWD + 0 * N1 + i; }
        else if (k == 2) { r.target = 1; r.asrc = 1 * N1 + yr; r.bsrc = SRC_FWD + 0 * N1 + i; }
        else { r.target = 2; r.neg = 1; r.asrc = 2 * N1 + yr; r.bsrc = SRC_FWD + 2 * N1 + i; }
        return r;
    }
    // MODE_ADJ
    if (t < 3) {  // Eq. (2): gbar_X P_j
        r.target = t;
        r.asrc = -1 - (ADJ_GBAR + t);
        r.bsrc = SRC_POW + (N - m);
        return r;
    }
    if (t < 8) {  // the linear terms of the brackets E_j
        const int k = m - 1;
        switch (t) {
        case 3: r.target = 0; r.neg = 1; r.asrc = -1 - P_SIGMA; r.bsrc = 0 * N1 + k; break;
        case 4: r.target = 0; r.asrc = -1 - P_R; r.bsrc = 1 * N1 + k; break;
        case 5: r.target = 1; r.asrc = -1 - P_SIGMA; r.bsrc = 0 * N1 + k; break;
        case 6: r.target = 1; r.neg = 1; r.add = 1; r.asrc = 0; r.bsrc = 1 * N1 + k; break;
        default: r.target = 2; r.neg = 1; r.asrc = -1 - P_B; r.bsrc = 2 * N1 + k; break;
        }
        return r;
    }
    const int u = t - 8, l = u >> 2, k = u & 3, yr = m - 1 - l;
    if (k == 0) { r.target = 0; r.neg = 1; r.asrc = 1 * N1 + yr; r.bsrc = SRC_FWD + 2 * N1 + l; }
    else if (k == 1) { r.target = 0; r.asrc = 2 * N1 + yr; r.bsrc = SRC_FWD + 1 * N1 + l; }
    else if (k == 2) { r.target = 1; r.asrc = 2 * N1 + yr; r.bsrc = SRC_FWD + 0 * N1 + l; }
    else { r.target = 2; r.neg = 1; r.asrc = 1 * N1 + yr; r.bsrc = SRC_FWD + 0 * N1 + l; }
    return r;
}

__device__ __forceinline__ Term term_of(const KArgs &a, int m, int t, int N1, int mode = MODE_FWD)
{
    if (mode != MODE_FWD) return adjoint_term(a, mode, m, t, N1);
    if (!a.sysT) return lorenz_term(m, t, N1);
    Term r;
    r.add = 0;
    r.skip = 0;
    r.asrc = 0;
    if (t < a.sysNF) {
        const int *e = a.sysT + 4 * t;
        const int p = __ldg(e + 2), j = __ldg(e + 3);
        r.target = __ldg(e);
        r.neg = __ldg(e + 1);
        if (j >= 0) {
            r.bsrc = j * N1 + m;
            if (p >= 0) r.asrc = -1 - p;
            else r.add = 1;
        } else {
            r.add = 1;
            r.bsrc = -1 - p;
            r.skip = m != 0;
        }
    } else {
        const int u = t - a.sysNF, q = u / (m + 1), l = u - q * (m + 1);
        const int *e = a.sysT + 4 * (a.sysNF + q);
        r.target = __ldg(e);
        r.neg = __ldg(e + 1);
        r.asrc = __ldg(e + 2) * N1 + (m - l);
        r.bsrc = __ldg(e + 3) * N1 + l;
    }
    return r;
}

// terms of index m
__device__ __forceinline__ int nterms(const KArgs &a, int m, int mode = MODE_FWD)
{
    if (mode == MODE_POW) return 1;
    if (mode == MODE_ADJ) return m >= 1 ? 8 + 4 * m : 3;
    if (mode == MODE_PAR) return 3 + 4 * a.N;
    return a.sysT ? a.sysNF + a.sysNQ * (m + 1) : 2 * m + 7;
}

struct Meta {
    int e, f;
};

__device__ __forceinline__ Meta meta_of(const Smem &S, const KArgs &a, int src)
{
    Meta r;
    if (src >= SRC_POW) {
        r.e = S.pexpT[src - SRC_POW];
        r.f = S.pflgT[src - SRC_POW];
    } else if (src >= SRC_FWD) {
        r.e = S.fexpT[src - SRC_FWD];
        r.f = S.fflgT[src - SRC_FWD];
    } else if (src >= 0) {
        r.e = S.expT[src];
        r.f = S.flgT[src];
    } else if (-1 - src < 4) {
        r.e = __ldg(&a.parE[-1 - src]);
        r.f = __ldg(&a.parF[-1 - src]);
    } else {  // reverse sweep: gbar and the parameter adjoints change during the launch
        r.e = __ldcg(&a.parE[-1 - src]);
        r.f = __ldcg(&a.parF[-1 - src]);
    }
    return r;
}

// ------------------------------------------------------------------ the limb-product tile

// Columns of the exact product A*B (Lp x Lp limbs): column c = sum_i a_i b_{c-i}.
// A thread owns the column pair block1 = [qW, qW+W) and block2 = [qW+Lp, qW+Lp+W);
// together they hold exactly W*Lp products, so every pair costs the same.  It
// walks s = 0 .. Lp+W-1: block1 for s < (q+1)W (i = s), block2 after it
// (i = s - W).  The window of W b-limbs slides down one limb per step through
// a cyclic copy C of B padded with W zeros (C[x] = b_x for x < Lp, 0 for
// Lp <= x < Lp+W), which makes the hand-over from block1 to block2 seamless;
// the block1 sums are saved at the hand-over (a predicated copy, so the warp
// never diverges) and block2 = final - saved.
// The walk of unit q over the limbs of A: a = the sums of all its columns'
// products, s = those of block 1 (saved at the hand-over).
template <bool SPARSE>
__device__ __forceinline__ void unit_sums(const uint32_t *A, const uint32_t *C, int q, int P, int M,
                                          uint32_t (&a0)[W], uint32_t (&a1)[W], uint32_t (&a2)[W],
                                          uint32_t (&s0)[W], uint32_t (&s1)[W], uint32_t (&s2)[W])
{
    uint32_t bw[W];
#pragma unroll
    for (int k = 0; k < W; k++) bw[k] = C[phys(q * W + k)];
    for (int j = 0; j <= P; j++) {
        const bool snap = (j == q + 1);
#pragma unroll
        for (int k = 0; k < W; k++) {
            s0[k] = snap ? a0[k] : s0[k];
            s1[k] = snap ? a1[k] : s1[k];
            s2[k] = snap ? a2[k] : s2[k];
        }
        const int ib = (j <= q) ? j * W : (j - 1) * W;
        const uint32_t *Ap = A + phys(ib);
        int xg = (q - j - 1) * W;
        if (xg < 0) xg += M;
        const uint32_t *Cp = C + phys(xg);
#pragma unroll
        for (int u = 0; u < W; u++) {
            const uint32_t av = Ap[u];
            if (!SPARSE || av != 0u) {
#pragma unroll
                for (int k = 0; k < W; k++) mac_cc(av, bw[k], a0[k], a1[k], a2[k]);
            }
#pragma unroll
            for (int k = W - 1; k > 0; k--) bw[k] = bw[k - 1];
            bw[0] = Cp[W - 1 - u];
        }
    }
}

// column t of block 1 (v1) and of block 2 (v2) of a unit's sums
__device__ __forceinline__ void unit_digit(const uint32_t (&a0)[W], const uint32_t (&a1)[W],
                                           const uint32_t (&a2)[W], const uint32_t (&s0)[W],
                                           const uint32_t (&s1)[W], const uint32_t (&s2)[W], int t,
                                           long long &v1, long long &v2)
{
    v1 = 0;
    v2 = 0;
    if (t < W) {
        v1 += s0[t];
        v2 += (long long)a0[t] - s0[t];
    }
    if (t >= 1 && t - 1 < W) {
        v1 += s1[t - 1];
        v2 += (long long)a1[t - 1] - s1[t - 1];
    }
    if (t >= 2 && t - 2 < W) {
        v1 += s2[t - 2];
        v2 += (long long)a2[t - 2] - s2[t - 2];
    }
}

template <bool SPARSE>
__device__ void mac_pair(const uint32_t *A, const uint32_t *C, int q, int P, int Lp, int M,
                         long long *win, int off, bool neg)
{
    uint32_t a0[W], a1[W], a2[W], s0[W], s1[W], s2[W];
#pragma unroll
    for (int k = 0; k < W; k++) a0[k] = a1[k] = a2[k] = s0[k] = s1[k] = s2[k] = 0u;
    unit_sums<SPARSE>(A, C, q, P, M, a0, a1, a2, s0, s1, s2);
    // block1 = saved sums at columns qW + t, block2 = final - saved at qW + Lp + t
    long long *w1 = win + off + q * W;
    long long *w2 = w1 + Lp;
#pragma unroll
    for (int t = 0; t < W + 2; t++) {
        long long v1, v2;
        unit_digit(a0, a1, a2, s0, s1, s2, t, v1, v2);
        if (neg) {
            v1 = -v1;
            v2 = -v2;
        }
        if (v1) atomicAdd((unsigned long long *)&w1[t], (unsigned long long)v1);
        if (v2) atomicAdd((unsigned long long *)&w2[t], (unsigned long long)v2);
    }
}

// A unit of the term phase, called by all 32 lanes of a warp together
// (`prod` false: no work for this lane).  The lanes hold units of
// consecutive terms with the same q, so lanes whose sums go to the same
// columns (same window, offset and q) are neighbours: each run of them is
// summed by shuffles into its first lane, which alone adds into the window.
__device__ void mac_unit_warp(const uint32_t *A, const uint32_t *C, int q, int P, int Lp, int M,
                              long long *win, int off, bool neg, bool prod, bool sparse)
{
    const int lane = threadIdx.x & 31;
    uint32_t a0[W], a1[W], a2[W], s0[W], s1[W], s2[W];
#pragma unroll
    for (int k = 0; k < W; k++) a0[k] = a1[k] = a2[k] = s0[k] = s1[k] = s2[k] = 0u;
    if (prod) {
        if (sparse) unit_sums<true>(A, C, q, P, M, a0, a1, a2, s0, s1, s2);
        else unit_sums<false>(A, C, q, P, M, a0, a1, a2, s0, s1, s2);
    }
    __syncwarp();
    long long *w1 = win + off + q * W;
    const long long key = prod ? (long long)(size_t)w1 : -1 - (long long)lane;
    const long long prev = __shfl_up_sync(FULL, key, 1);
    const bool head = lane == 0 || prev != key;
    const unsigned heads = __ballot_sync(FULL, head);
    const unsigned above = heads & ~((2u << lane) - 1u);
    const int seg_end = above ? __ffs(above) - 2 : 31;
    long long v1[W + 2], v2[W + 2];
#pragma unroll
    for (int t = 0; t < W + 2; t++) {
        unit_digit(a0, a1, a2, s0, s1, s2, t, v1[t], v2[t]);
        if (neg) {
            v1[t] = -v1[t];
            v2[t] = -v2[t];
        }
    }
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const bool take = lane + d <= seg_end;
#pragma unroll
        for (int t = 0; t < W + 2; t++) {
            const long long o1 = __shfl_down_sync(FULL, v1[t], d);
            const long long o2 = __shfl_down_sync(FULL, v2[t], d);
            if (take) {
                v1[t] += o1;
                v2[t] += o2;
            }
        }
    }
    if (prod && head) {
        long long *w2 = w1 + Lp;
#pragma unroll
        for (int t = 0; t < W + 2; t++) {
            if (v1[t]) atomicAdd((unsigned long long *)&w1[t], (unsigned long long)v1[t]);
            if (v2[t]) atomicAdd((unsigned long long *)&w2[t], (unsigned long long)v2[t]);
        }
    }
}

// a lone number +-c: limbs [qW, qW+W) of c (staged in A layout) into the window
__device__ void add_unit(const uint32_t *A, int q, long long *win, int off, bool neg)
{
#pragma unroll
    for (int k = 0; k < W; k++) {
        long long v = A[phys(q * W + k)];
        if (v) atomicAdd((unsigned long long *)&win[off + q * W + k],
                         (unsigned long long)(neg ? -v : v));
    }
}

// ------------------------------------------------------------------ close: normalise, divide

struct Norm {
    int neg;
    int top;  // index of the top non-zero digit, -1 for zero
};

// Exact value of Wn int64 columns (sum col[c] 2^(32c)) as sign and magnitude
// digits.  One warp; lane l owns columns [lK, lK+K).  Local carries first,
// then the carries that cross lanes ride up one lane per round until none is
// left (any carry is absorbed or passed on, so 32 rounds always suffice).
__device__ Norm warp_normalize(const long long *col, bool from_global, uint32_t *dig, int Wn,
                               int *status)
{
    const int lane = threadIdx.x & 31;
    const int K = (Wn + 31) >> 5;
    const int c0 = lane * K;
    const int c1 = min(c0 + K, Wn);
    long long carry = 0;
    for (int c = c0; c < c1; c++) {
        long long v = (from_global ? __ldcg(&col[c]) : col[c]) + carry;
        dig[c] = (uint32_t)v;
        carry = v >> 32;
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
    if (!settled && lane == 0) set_status(status, DEV_INTERNAL);
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
// writes L limbs to out (lanes write their own chunks) and returns the exponent.
// Only limbs of |E| at or above the quotient's lowest kept position matter
// (floor(|E| / (d 2^(32 s))) = floor(floor(|E| / 2^(32 s)) / d)); below the
// window's lowest limb they are zero.
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
    // this lane's chunk as an affine map r -> (Pm r + V) mod d; the divisions
    // by d with a multiplier (invariant-divisor method)
    const Divisor dv = make_divisor16(d);
    uint32_t V = 0, Pm = 1;
    uint32_t t32 = 1;
    (void)divstep(t32, 0u, dv);  // 2^32 mod d
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

// ------------------------------------------------------------------ phases

__device__ void init_slots(const Smem &S, const KArgs &a)
{
    // C-layout padding (x in [Lp, M)) stays zero for the whole launch
    for (int e = threadIdx.x; e < a.tb * S.M; e += NT) {
        int slot = e / S.M, x = e - slot * S.M;
        uint32_t *Cv = S.slots + (size_t)slot * (S.AV + S.CV) + S.AV;
        if (x >= a.Lp) Cv[phys(x)] = 0u;
    }
    for (int e = threadIdx.x; e < 3 * nwin_of(a) * a.Wcap; e += NT) S.win[e] = 0;
}

// block-wide min (lo) / max (hi) for three targets; returns in S.misc
__device__ void reduce_windows(const Smem &S, const KArgs &a, long long lo[3], long long hi[3])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    long long *red = (long long *)(S.misc + MS_RED);  // [8][6] long long = 96 ints
    for (int tg = 0; tg < 3; tg++) {
        long long l = warp_min_ll(lo[tg]), h = warp_max_ll(hi[tg]);
        if (lane == 0) {
            red[warp * 6 + tg] = l;
            red[warp * 6 + 3 + tg] = h;
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        int tg = threadIdx.x;
        long long l = red[tg], h = red[3 + tg];
        for (int w = 1; w < NT / 32; w++) {
            l = min(l, red[w * 6 + tg]);
            h = max(h, red[w * 6 + 3 + tg]);
        }
        int width = 0;
        if (h > l) {
            if (h - l > a.Wcap) {
                set_status(a.status, DEV_ERANGE);
            } else {
                width = (int)(h - l);
            }
        }
        ((long long *)(S.misc + MS_BASE))[tg] = l;
        S.misc[MS_WIDTH + tg] = width;
    }
    __syncthreads();
}

__device__ __forceinline__ long long win_base(const Smem &S, int tg)
{
    return ((const long long *)(S.misc + MS_BASE))[tg];
}

// window placement for coefficient index m: lowest limb position over the
// non-zero terms of each bracket and the highest position the exact sum can
// reach (product: 2Lp columns plus two carry limbs of the 96-bit column sums
// and of the sum's growth; lone number: Lp limbs plus two).
__device__ void place_windows(const Smem &S, const KArgs &a, int m, int mode = MODE_FWD)
{
    const int T = nterms(a, m, mode);
    const int N1 = a.N + 1;
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX};
    long long hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int t = threadIdx.x; t < T; t += NT) {
        Term tm = term_of(a, m, t, N1, mode);
        if (tm.skip) continue;
        Meta mb = meta_of(S, a, tm.bsrc);
        if (!(mb.f & F_NZ)) continue;
        long long lp, top;
        if (tm.add) {
            lp = (long long)mb.e - a.L;
            top = lp + a.Lp + 2;
        } else {
            Meta ma = meta_of(S, a, tm.asrc);
            if (!(ma.f & F_NZ)) continue;
            lp = (long long)ma.e - a.L + (long long)mb.e - a.L;
            top = lp + 2 * a.Lp + 2;
        }
        lo[tm.target] = min(lo[tm.target], lp);
        hi[tm.target] = max(hi[tm.target], top);
    }
    reduce_windows(S, a, lo, hi);
}

// where a staged operand comes from: a row of the coefficient table (>= 0),
// parameter p (-1 - p), the newest coefficient of component c in shared memory
// (SRC_NEWC - c), or nothing
enum { SRC_NEWC = -100, SRC_NONE = -1000 };

__device__ __forceinline__ int src_code(int src, int m, int N1)
{
    if (src < 0 || src >= SRC_FWD) return src;
    const int comp = src / N1, idx = src - comp * N1;
    return idx == m ? SRC_NEWC - comp : src;
}

// stage terms [t0, t0 + nt) of index m into slots; record offset and flags.
// One thread per slot places the term and records where its operands come
// from; then all threads copy the operands' limbs, element by element over
// the whole batch, with no per-element term lookup.
__device__ void stage_terms(const Smem &S, const KArgs &a, int m, int t0, int nt, int mode = MODE_FWD)
{
    const int N1 = a.N + 1;
    const int Lp = a.Lp;
    // the row held in S.newc: coefficient m (forward), adjoint m - 1 (reverse sweep)
    const int newest = mode == MODE_FWD ? m : (mode == MODE_ADJ ? m - 1 : -1);
    for (int slot = threadIdx.x; slot < nt; slot += NT) {
        Term tm = term_of(a, m, t0 + slot, N1, mode);
        Meta mb = meta_of(S, a, tm.bsrc);
        int flags = 0, off = 0;
        bool skip = tm.skip || !(mb.f & F_NZ);
        long long lp = 0;
        int neg = tm.neg ^ (mb.f & F_NEG);
        if (tm.add) {
            lp = (long long)mb.e - a.L;
            flags |= 2;
        } else {
            Meta ma = meta_of(S, a, tm.asrc);
            skip = skip || !(ma.f & F_NZ);
            neg ^= (ma.f & F_NEG);
            lp = (long long)ma.e - a.L + (long long)mb.e - a.L;
            if (tm.asrc < 0 && S.misc[MS_PNZ + (-1 - tm.asrc)] * 8 <= Lp) flags |= 8;  // sparse
        }
        if (skip) flags |= 4;
        if (!skip) off = (int)(lp - win_base(S, tm.target));
        flags |= neg ? 1 : 0;
        flags |= tm.target << 4;
        S.tinfo[2 * slot] = off;
        S.tinfo[2 * slot + 1] = flags;
        int ca = SRC_NONE, cb = SRC_NONE;
        if (!skip) {
            if (tm.add) {
                ca = src_code(tm.bsrc, newest, N1);  // a lone number goes to the A layout
            } else {
                ca = src_code(tm.asrc, newest, N1);
                cb = src_code(tm.bsrc, newest, N1);
            }
        }
        S.srcs[2 * slot] = ca;
        S.srcs[2 * slot + 1] = cb;
    }
    __syncthreads();
    // element e of slot s: operand e / Lp (0 A, 1 B), limb e mod Lp; each
    // thread takes elements NT apart, four at a time (loads before stores, so
    // that their latencies overlap)
    constexpr int U = 4;
    const int E = 2 * Lp;
    int slot = threadIdx.x / E, r = threadIdx.x - slot * E;
    const int dslot = NT / E, dr = NT - dslot * E;
    while (slot < nt) {
        int dst[U];
        uint32_t v[U];
#pragma unroll
        for (int k = 0; k < U; k++) {
            dst[k] = -1;
            v[k] = 0u;
            if (slot < nt) {
                const int which = r >= Lp ? 1 : 0;
                const int x = r - which * Lp;
                const int code = S.srcs[2 * slot + which];
                if (code != SRC_NONE) {
                    if (code >= SRC_POW) v[k] = __ldcg(&a.powL[(size_t)(code - SRC_POW) * Lp + x]);
                    else if (code >= SRC_FWD)
                        v[k] = __ldcg(&a.fwdL[((const long long *)(S.misc + MS_FWDOFF))[0] +
                                              (size_t)(code - SRC_FWD) * Lp + x]);
                    else if (code >= 0) v[k] = __ldcg(&a.coefL[(size_t)code * Lp + x]);
                    else if (code <= SRC_NEWC) v[k] = S.newc[(SRC_NEWC - code) * Lp + x];
                    else if (-1 - code < 4) v[k] = __ldg(&a.parL[(size_t)(-1 - code) * Lp + x]);
                    else v[k] = __ldcg(&a.parL[(size_t)(-1 - code) * Lp + x]);
                    dst[k] = slot * (S.AV + S.CV) + (which ? S.AV + phys(x) : phys(x));
                }
            }
            slot += dslot;
            r += dr;
            if (r >= E) {
                r -= E;
                slot++;
            }
        }
#pragma unroll
        for (int k = 0; k < U; k++)
            if (dst[k] >= 0) S.slots[dst[k]] = v[k];
    }
}

// unit q of the term in `slot`, added into window copy `copy`
__device__ void run_unit(const Smem &S, const KArgs &a, int slot, int q, int copy)
{
    const int off = S.tinfo[2 * slot];
    const int flags = S.tinfo[2 * slot + 1];
    if (flags & 4) return;
    const int tg = (flags >> 4) & 3;
    const bool neg = flags & 1;
    const uint32_t *A = S.slots + (size_t)slot * (S.AV + S.CV);
    long long *win = S.win + ((size_t)copy * 3 + tg) * a.Wcap;
    if (flags & 2) {
        add_unit(A, q, win, off, neg);
    } else if (flags & 8) {
        mac_pair<true>(A, A + S.AV, q, a.P, a.Lp, S.M, win, off, neg);
    } else {
        mac_pair<false>(A, A + S.AV, q, a.P, a.Lp, S.M, win, off, neg);
    }
}

// run_unit for all lanes of a warp (slot < 0: nothing for this lane); lone
// numbers are added directly, products through mac_unit_warp
__device__ void run_unit_warp(const Smem &S, const KArgs &a, int slot, int q, int copy)
{
    int off = 0, flags = 4;
    if (slot >= 0) {
        off = S.tinfo[2 * slot];
        flags = S.tinfo[2 * slot + 1];
    }
    const bool live = !(flags & 4);
    const int tg = (flags >> 4) & 3;
    const bool neg = flags & 1;
    const uint32_t *A = S.slots + (size_t)(slot >= 0 ? slot : 0) * (S.AV + S.CV);
    long long *win = S.win + ((size_t)copy * 3 + tg) * a.Wcap;
    if (live && (flags & 2)) add_unit(A, q, win, off, neg);
    mac_unit_warp(A, A + S.AV, q, a.P, a.Lp, S.M, win, off, neg, live && !(flags & 2), (flags & 8) != 0);
}

// this CTA's share of the products of index m, added into the shared windows
// and then into the global accumulators
// ONE_CTA: compiled for a grid of one CTA only (the batch)
template <bool ONE_CTA>
__device__ void term_phase(const Smem &S, const KArgs &a, int m, int set, int mode = MODE_FWD)
{
    const int G = vgrid(a), g = vrank(a);
    Prof pr(a);
    place_windows(S, a, m, mode);
    if (!cta_ok(S, a)) return;
    pr.mark(PR_PLACE);
    if (G > 1) {
        // clear the accumulator set that the next index will use (last read
        // by the close two indices back, which every CTA finished before the
        // previous barrier); sets rotate over the running index of the launch
        long long *nxt = a.gwin + (size_t)((set + 1) % 3) * 3 * a.Wcap;
        for (int e = g * NT + threadIdx.x; e < 3 * a.Wcap; e += G * NT) nxt[e] = 0;
    }
    const long long T = nterms(a, m, mode);
    const long long U = T * a.P;
    const long long u0 = U * g / G, u1 = U * (g + 1) / G;
    if (u0 < u1) {
        const int tA = (int)(u0 / a.P), tB = (int)((u1 - 1) / a.P);
        for (int tb0 = tA; tb0 <= tB; tb0 += a.tb) {
            const int nt = min(a.tb, tB - tb0 + 1);
            stage_terms(S, a, m, tb0, nt, mode);
            __syncthreads();
            pr.mark(PR_STAGE);
            const long long ua = max(u0, (long long)tb0 * a.P);
            const long long ub = min(u1, (long long)(tb0 + nt) * a.P);
            // the column sums of many terms land on the same columns: each warp
            // adds into a window copy of its own, so that the shared-memory
            // atomics of different warps do not queue on the same words
            const int copy = (int)(threadIdx.x >> 5) % nwin_of(a);
            if (ONE_CTA || G == 1) {
                // one CTA takes every term: units (slot, q), slot fastest, a
                // warp's 32 lanes at a time (every lane of a warp makes the same
                // number of passes), so that many lanes share destinations and
                // combine before the atomics
                const int total = nt * a.P, lane = threadIdx.x & 31;
                for (int base = threadIdx.x - lane; base < total; base += NT) {
                    const int i = base + lane;
                    int slot = -1, q = 0;
                    if (i < total) {
                        q = i / nt;
                        slot = i - q * nt;
                        const long long u = (long long)(tb0 + slot) * a.P + q;
                        if (u < ua || u >= ub) slot = -1;
                    }
                    run_unit_warp(S, a, slot, q, copy);
                }
            } else {
                // a share of the units of many CTAs: q fastest, few lanes share
                // destinations
                for (long long u = ua + threadIdx.x; u < ub; u += NT) {
                    const int t = (int)(u / a.P);
                    run_unit(S, a, t - tb0, (int)(u - (long long)t * a.P), copy);
                }
            }
            __syncthreads();
            pr.mark(PR_MAC);
        }
    }
    if (nwin_of(a) > 1) {  // the copies into copy 0 (and emptied)
        for (int tg = 0; tg < 3; tg++) {
            const int wd = S.misc[MS_WIDTH + tg];
            for (int c = threadIdx.x; c < wd; c += NT) {
                long long v = 0;
                for (int k = 1; k < nwin_of(a); k++) {
                    long long *w = S.win + ((size_t)k * 3 + tg) * a.Wcap + c;
                    v += *w;
                    *w = 0;
                }
                if (v) S.win[tg * a.Wcap + c] += v;
            }
        }
        __syncthreads();
    }
    if (G > 1) {
        long long *dst = a.gwin + (size_t)set * 3 * a.Wcap;
        for (int tg = 0; tg < 3; tg++) {
            const int wd = S.misc[MS_WIDTH + tg];
            for (int c = threadIdx.x; c < wd; c += NT) {
                long long v = S.win[tg * a.Wcap + c];
                if (v) {
                    atomicAdd((unsigned long long *)&dst[tg * a.Wcap + c], (unsigned long long)v);
                    S.win[tg * a.Wcap + c] = 0;
                }
            }
        }
        __syncthreads();
        pr.mark(PR_FLUSH);
    }
}

// the three brackets of index m -> coefficients m+1 (every CTA, redundantly)
__device__ void close_phase(const Smem &S, const KArgs &a, int m, int set)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = vgrid(a);
    const int N1 = a.N + 1;
    Prof pr(a);
    if (G > 1) {
        // the three windows of the global set into shared memory, every thread
        // taking a share (one round trip, not one per column a lane)
        for (int tg = 0; tg < 3; tg++) {
            const int wd = S.misc[MS_WIDTH + tg];
            const long long *src = a.gwin + ((size_t)set * 3 + tg) * a.Wcap;
            for (int c = threadIdx.x; c < wd; c += NT) S.win[(size_t)tg * a.Wcap + c] = __ldcg(&src[c]);
        }
        __syncthreads();
    }
    if (warp < 3) {
        const int tg = warp;  // 0 alpha, 1 beta, 2 gamma
        const int wd = S.misc[MS_WIDTH + tg];
        uint32_t *out = S.newc + tg * a.Lp;
        int e = 0, f = 0;
        if (wd > 0) {
            const long long *src = S.win + (size_t)tg * a.Wcap;
            uint32_t *dig = S.dig + (size_t)tg * a.Wcap;
            Norm nr = warp_normalize(src, false, dig, wd, a.status);
            for (int c = lane; c < wd; c += 32) S.win[tg * a.Wcap + c] = 0;
            if (nr.top >= 0) {
                long long eq = warp_divide(dig, nr.top, win_base(S, tg), (uint32_t)(m + 1), a.L, out);
                if (eq > (1LL << 30) || eq < -(1LL << 30)) {
                    if (lane == 0) set_status(a.status, DEV_ERANGE);
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
            S.expT[tg * N1 + m + 1] = e;
            S.flgT[tg * N1 + m + 1] = f;
        }
        if (vrank(a) == 0) {
            uint32_t *g = a.coefL + ((size_t)tg * N1 + m + 1) * a.Lp;
            for (int x = lane; x < a.Lp; x += 32) g[x] = out[x];
            if (lane == 0) {
                a.coefE[tg * N1 + m + 1] = e;
                a.coefF[tg * N1 + m + 1] = f;
            }
        }
    }
    __syncthreads();
    pr.mark(PR_CLOSE);
}

// Horner for the components this CTA owns: h_N = c_N,
// h_i = trunc_L(tau*h_{i+1} + c_i), i = N-1 .. 0.  Slot layout:
// slot 2j: tau (A layout) and h_j (C layout); slot 2j+1: c_i (A layout).
__device__ void horner_phase(const Smem &S, const KArgs &a, int step)
{
    const int G = vgrid(a), g = vrank(a);
    const int ptau = a.sysT ? a.ptau : P_TAU;
    int c_first, nc;
    if (G >= 3) {
        if (g >= 3) return;
        c_first = g;
        nc = 1;
    } else {
        if (g != 0) return;
        c_first = 0;
        nc = 3;
    }
    const int N1 = a.N + 1, Lp = a.Lp, N = a.N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int SL = S.AV + S.CV;
    // h meta per local component in misc: e at 32+j, f at 36+j
    int *hE = S.misc + MS_HE, *hF = S.misc + MS_HF;
    // stage tau and h = c_N, c_{N-1}
    for (int j = 0; j < nc; j++) {
        const int comp = c_first + j;
        uint32_t *s0 = S.slots + (size_t)(2 * j) * SL;
        uint32_t *s1 = S.slots + (size_t)(2 * j + 1) * SL;
        for (int x = threadIdx.x; x < Lp; x += NT) {
            s0[phys(x)] = __ldg(&a.parL[(size_t)ptau * Lp + x]);
            s0[S.AV + phys(x)] = S.newc[comp * Lp + x];  // coefficient N
            s1[phys(x)] = __ldcg(&a.coefL[((size_t)comp * N1 + N - 1) * Lp + x]);
        }
        if (threadIdx.x == 0) {
            hE[j] = S.expT[comp * N1 + N];
            hF[j] = S.flgT[comp * N1 + N];
        }
    }
    const int tauE = __ldg(&a.parE[ptau]), tauF = __ldg(&a.parF[ptau]);
    __syncthreads();
    Prof pr(a);
    for (int i = N - 1; i >= 0; i--) {
        // prefetch c_{i-1} into registers while the products of step i run
        uint32_t pre[3][4];
        if (i > 0) {
            for (int j = 0; j < nc; j++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    int x = threadIdx.x + r * NT;
                    pre[j][r] = x < Lp
                        ? __ldcg(&a.coefL[((size_t)(c_first + j) * N1 + i - 1) * Lp + x]) : 0u;
                }
        }
        // window placement and term info
        if (a.tau_q && threadIdx.x < nc) {
            // tau = trunc_L(p/q): h_i = trunc_L(E / q), E = +-(p h - r h 2^(-32 shift)) + q c_i
            const int j = threadIdx.x, comp = c_first + j;
            const int ce = S.expT[comp * N1 + i], cf = S.flgT[comp * N1 + i];
            const bool prod = (hF[j] & F_NZ) != 0, lone = (cf & F_NZ) != 0;
            const long long lph = (long long)hE[j] - a.L, lpr = lph - a.tau_shift, lpc = (long long)ce - a.L;
            long long lo = LLONG_MAX, hi = LLONG_MIN;
            if (prod) {
                lo = min(lo, a.tau_r ? lpr : lph);
                hi = max(hi, lph + Lp + 2);
            }
            if (lone) {
                lo = min(lo, lpc);
                hi = max(hi, lpc + Lp + 2);
            }
            int width = 0;
            if (hi > lo) {
                if (hi - lo > a.Wcap) set_status(a.status, DEV_ERANGE);
                else width = (int)(hi - lo);
            }
            S.tinfo[2 * (2 * j)] = prod ? (int)(lph - lo) : 0;
            S.tinfo[2 * (2 * j) + 1] = (prod ? 1 : 0) | ((((hF[j] & F_NEG) != 0) != (a.tau_neg != 0)) ? 2 : 0);
            S.tinfo[2 * (2 * j + 1)] = lone ? (int)(lpc - lo) : 0;
            S.tinfo[2 * (2 * j + 1) + 1] = (lone ? 1 : 0) | ((cf & F_NEG) ? 2 : 0);
            ((long long *)(S.misc + MS_BASE))[j] = lo;
            S.misc[MS_WIDTH + j] = width;
        } else if (!a.tau_q && threadIdx.x < nc) {
            const int j = threadIdx.x, comp = c_first + j;
            const int ce = S.expT[comp * N1 + i], cf = S.flgT[comp * N1 + i];
            long long lo = LLONG_MAX, hi = LLONG_MIN;
            int off0 = 0, off1 = 0, fl0 = 4, fl1 = 4 | 2;
            long long lp0 = 0, lp1 = 0;
            if ((hF[j] & F_NZ) && (tauF & F_NZ)) {
                lp0 = (long long)hE[j] - a.L + (long long)tauE - a.L;
                lo = min(lo, lp0);
                hi = max(hi, lp0 + 2 * Lp + 2);
                fl0 = ((hF[j] ^ tauF) & F_NEG) ? 1 : 0;
            }
            if (cf & F_NZ) {
                lp1 = (long long)ce - a.L;
                lo = min(lo, lp1);
                hi = max(hi, lp1 + Lp + 2);
                fl1 = 2 | ((cf & F_NEG) ? 1 : 0);
            }
            int width = 0;
            if (hi > lo) {
                if (hi - lo > a.Wcap) set_status(a.status, DEV_ERANGE);
                else width = (int)(hi - lo);
            }
            if (!(fl0 & 4)) off0 = (int)(lp0 - lo);
            if (!(fl1 & 4)) off1 = (int)(lp1 - lo);
            S.tinfo[2 * (2 * j)] = off0;
            S.tinfo[2 * (2 * j) + 1] = fl0 | (j << 4);
            S.tinfo[2 * (2 * j + 1)] = off1;
            S.tinfo[2 * (2 * j + 1) + 1] = fl1 | (j << 4);
            ((long long *)(S.misc + MS_BASE))[j] = lo;
            S.misc[MS_WIDTH + j] = width;
        }
        if (!cta_ok(S, a)) return;
        if (a.tau_q) {
            // the window of E column by column: low half of v x_y plus high half of v x_{y-1}
            for (int j = 0; j < nc; j++) {
                const int wd = S.misc[MS_WIDTH + j];
                const int oh = S.tinfo[2 * (2 * j)], fh = S.tinfo[2 * (2 * j) + 1];
                const int oc = S.tinfo[2 * (2 * j + 1)], fc = S.tinfo[2 * (2 * j + 1) + 1];
                const uint32_t *hp = S.newc + (size_t)(c_first + j) * Lp;
                const uint32_t *cs = S.slots + (size_t)(2 * j + 1) * SL;  // c_i, A layout
                for (int cc = threadIdx.x; cc < wd; cc += NT) {
                    long long sum = 0;
                    if (fh & 1) {
                        const int y = cc - oh, yr = y + a.tau_shift;
                        long long t = 0;
                        if (y >= 0 && y < Lp) t += (uint32_t)((uint64_t)a.tau_p * hp[y]);
                        if (y >= 1 && y <= Lp) t += (long long)(((uint64_t)a.tau_p * hp[y - 1]) >> 32);
                        if (yr >= 0 && yr < Lp) t -= (uint32_t)((uint64_t)a.tau_r * hp[yr]);
                        if (yr >= 1 && yr <= Lp) t -= (long long)(((uint64_t)a.tau_r * hp[yr - 1]) >> 32);
                        sum += (fh & 2) ? -t : t;
                    }
                    if (fc & 1) {
                        const int y = cc - oc;
                        long long t = 0;
                        if (y >= 0 && y < Lp) t += (uint32_t)((uint64_t)a.tau_q * cs[phys(y)]);
                        if (y >= 1 && y <= Lp) t += (long long)(((uint64_t)a.tau_q * cs[phys(y - 1)]) >> 32);
                        sum += (fc & 2) ? -t : t;
                    }
                    if (sum) S.win[(size_t)j * a.Wcap + cc] += sum;
                }
            }
        } else {
            const int units = 2 * nc * a.P;
            for (int u = threadIdx.x; u < units; u += NT) {
                const int slot = u / a.P;
                run_unit(S, a, slot, u - slot * a.P, 0);
            }
        }
        __syncthreads();
        pr.mark(PR_HMAC);
        // close: h_i for each component (division by one = truncation)
        if (warp < nc) {
            const int j = warp;
            const int wd = S.misc[MS_WIDTH + j];
            uint32_t *hC = S.slots + (size_t)(2 * j) * SL + S.AV;
            uint32_t *hp = S.newc + (size_t)(c_first + j) * Lp;  // plain copy of h
            int e = 0, f = 0;
            if (wd > 0) {
                uint32_t *dig = S.dig + (size_t)j * a.Wcap;
                Norm nr = warp_normalize(S.win + (size_t)j * a.Wcap, false, dig, wd, a.status);
                for (int c = lane; c < wd; c += 32) S.win[j * a.Wcap + c] = 0;
                if (nr.top >= 0) {
                    long long eq = warp_divide(dig, nr.top, win_base(S, j), a.tau_q ? a.tau_q : 1u, a.L, hp);
                    if (eq > (1LL << 30) || eq < -(1LL << 30)) {
                        if (lane == 0) set_status(a.status, DEV_ERANGE);
                        eq = 0;
                    }
                    e = (int)eq;
                    f = F_NZ | (nr.neg ? F_NEG : 0);
                }
            }
            if (!(f & F_NZ))
                for (int x = lane; x < a.L; x += 32) hp[x] = 0u;
            __syncwarp();
            for (int x = lane; x < Lp; x += 32) hC[phys(x)] = x < a.L ? hp[x] : 0u;
            if (lane == 0) {
                hE[j] = e;
                hF[j] = f;
            }
        }
        // c_{i-1} into the lone-number slots
        if (i > 0) {
            for (int j = 0; j < nc; j++)
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    int x = threadIdx.x + r * NT;
                    if (x < Lp) S.slots[(size_t)(2 * j + 1) * SL + phys(x)] = pre[j][r];
                }
        }
        __syncthreads();
        pr.mark(PR_HCLOSE);
    }
    // the new state and, when due, a record
    const long long rec = (a.record_every > 0 && ((step + 1) % a.record_every) == 0)
                              ? (step + 1) / a.record_every - 1 : -1;
    for (int j = 0; j < nc; j++) {
        const int comp = c_first + j;
        const uint32_t *hp = S.newc + (size_t)comp * Lp;
        for (int x = threadIdx.x; x < Lp; x += NT) a.stL[comp * Lp + x] = hp[x];
        if (rec >= 0)
            for (int x = threadIdx.x; x < a.L; x += NT)
                a.recL[((size_t)rec * 3 + comp) * a.L + x] = hp[x];
        if (threadIdx.x == 0) {
            a.stE[comp] = hE[j];
            a.stF[comp] = hF[j];
            if (rec >= 0) {
                a.recS[rec * 3 + comp] = (hF[j] & F_NEG) ? 1 : 0;
                a.recE[rec * 3 + comp] = hE[j];
            }
        }
    }
}

// ------------------------------------------------------------------ reverse sweep

// The brackets of one index of the reverse sweep, on one CTA (the windows in
// shared memory): normalise each target's window, divide by d, truncate to L
// limbs into S.newc (component = target), and store the result -- a power of
// tau (MODE_POW, index m), adjoint m (MODE_ADJ), or the parameter adjoints
// (MODE_PAR).
__device__ void adj_close(const Smem &S, const KArgs &a, int mode, int m, uint32_t d)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int N1 = a.N + 1, Lp = a.Lp;
    const int ntg = mode == MODE_POW ? 1 : 3;
    if (warp < ntg) {
        const int tg = warp;
        const int wd = S.misc[MS_WIDTH + tg];
        uint32_t *out = S.newc + tg * Lp;
        int e = 0, f = 0;
        if (wd > 0) {
            uint32_t *dig = S.dig + (size_t)tg * a.Wcap;
            Norm nr = warp_normalize(S.win + (size_t)tg * a.Wcap, false, dig, wd, a.status);
            for (int c = lane; c < wd; c += 32) S.win[tg * a.Wcap + c] = 0;
            if (nr.top >= 0) {
                long long eq = warp_divide(dig, nr.top, win_base(S, tg), d, a.L, out);
                if (eq > (1LL << 30) || eq < -(1LL << 30)) {
                    if (lane == 0) set_status(a.status, DEV_ERANGE);
                    eq = 0;
                }
                e = (int)eq;
                f = F_NZ | (nr.neg ? F_NEG : 0);
            }
        }
        if (!(f & F_NZ))
            for (int x = lane; x < a.L; x += 32) out[x] = 0u;
        for (int x = a.L + lane; x < Lp; x += 32) out[x] = 0u;
        __syncwarp();
        uint32_t *gl;
        int32_t *ge, *gf;
        int *se = nullptr, *sf = nullptr;
        if (mode == MODE_POW) {
            gl = a.powL + (size_t)m * Lp;
            ge = a.powE + m;
            gf = a.powF + m;
            se = S.pexpT + m;
            sf = S.pflgT + m;
        } else if (mode == MODE_ADJ) {
            const int row = tg * N1 + m;
            gl = a.coefL + (size_t)row * Lp;
            ge = a.coefE + row;
            gf = a.coefF + row;
            se = S.expT + row;
            sf = S.flgT + row;
        } else {
            const int p = ADJ_THBAR + tg;
            gl = (uint32_t *)a.parL + (size_t)p * Lp;
            ge = (int32_t *)a.parE + p;
            gf = (int32_t *)a.parF + p;
        }
        for (int x = lane; x < Lp; x += 32) gl[x] = out[x];
        if (lane == 0) {
            *ge = e;
            *gf = f;
            if (se) {
                *se = e;
                *sf = f;
            }
        }
    }
    __syncthreads();
}

// The reverse sweep over the launch's nsteps steps, last step first (one CTA,
// one item: a trajectory's forward coefficients and one adjoint gbar): the
// powers of tau P_0 = 1, P_j = trunc_L(P_{j-1} tau); then per step the
// adjoint indices m = 0..N (the division by j = N - m, by 1 at m = N; y[N]
// becomes gbar of the step before) and the parameter adjoints.
__device__ void adjoint_body(const Smem &S, const KArgs &a)
{
    const int N = a.N, N1 = N + 1, Lp = a.Lp;
    for (int x = threadIdx.x; x < Lp; x += NT) a.powL[x] = x == a.L - 1 ? 1u : 0u;
    if (threadIdx.x == 0) {
        a.powE[0] = 1;  // 1 = 1 * 2^(32 (1 - L + L - 1))
        a.powF[0] = F_NZ;
        S.pexpT[0] = 1;
        S.pflgT[0] = F_NZ;
    }
    __syncthreads();
    for (int j = 1; j <= N; j++) {
        term_phase<true>(S, a, j, 0, MODE_POW);
        if (!cta_ok(S, a)) return;
        adj_close(S, a, MODE_POW, j, 1u);
    }
    if (!cta_ok(S, a)) return;
    const size_t nc = 3 * (size_t)N1;
    for (long long s = a.nsteps - 1; s >= 0; s--) {
        for (int e = threadIdx.x; e < 3 * N1; e += NT) {
            S.fexpT[e] = __ldcg(&a.fwdE[(size_t)s * nc + e]);
            S.fflgT[e] = __ldcg(&a.fwdF[(size_t)s * nc + e]);
        }
        if (threadIdx.x == 0) ((long long *)(S.misc + MS_FWDOFF))[0] = s * (long long)nc * Lp;
        __syncthreads();
        for (int m = 0; m <= N; m++) {
            term_phase<true>(S, a, m, 0, MODE_ADJ);
            if (!cta_ok(S, a)) return;
            adj_close(S, a, MODE_ADJ, m, m < N ? (uint32_t)(N - m) : 1u);
        }
        if (!cta_ok(S, a)) return;
        // the adjoint of the step's starting state (y[N], in S.newc) is gbar of the step before
        for (int e = threadIdx.x; e < 3 * Lp; e += NT)
            ((uint32_t *)a.parL)[(size_t)ADJ_GBAR * Lp + e] = S.newc[e];
        if (threadIdx.x < 3) {
            ((int32_t *)a.parE)[ADJ_GBAR + threadIdx.x] = S.expT[threadIdx.x * N1 + N];
            ((int32_t *)a.parF)[ADJ_GBAR + threadIdx.x] = S.flgT[threadIdx.x * N1 + N];
        }
        __syncthreads();
        term_phase<true>(S, a, 0, 0, MODE_PAR);
        if (!cta_ok(S, a)) return;
        adj_close(S, a, MODE_PAR, 0, 1u);
        if (!cta_ok(S, a)) return;
    }
}

template <bool ONE_CTA>
__device__ void taylor_body(const KArgs &a, unsigned char *smem_raw)
{
    Smem S = carve(smem_raw, a);
    const int N1 = a.N + 1;
    Prof tot(a);
    if (threadIdx.x < (a.adj ? ADJ_NPAR : (a.sysT ? a.npar : 4))) {
        int nz = 0;
        for (int x = 0; x < a.Lp; x++) nz += __ldg(&a.parL[(size_t)threadIdx.x * a.Lp + x]) != 0u;
        S.misc[MS_PNZ + threadIdx.x] = nz;
    }
    init_slots(S, a);
    __syncthreads();
    if (ONE_CTA && a.adj) {
        adjoint_body(S, a);
        __syncthreads();
        tot.mark(PR_TOTAL);
        return;
    }
    for (long long step = 0; step < a.nsteps; step++) {
        // alpha_0, beta_0, gamma_0 = the state (Sec. 2)
        for (int e = threadIdx.x; e < 3 * a.Lp; e += NT) {
            uint32_t v = __ldcg(&a.stL[e]);
            S.newc[e] = v;
            if (vrank(a) == 0) {
                int comp = e / a.Lp, x = e - comp * a.Lp;
                a.coefL[(size_t)comp * N1 * a.Lp + x] = v;
            }
        }
        if (threadIdx.x < 3) {
            int e = __ldcg(&a.stE[threadIdx.x]), f = __ldcg(&a.stF[threadIdx.x]);
            S.expT[threadIdx.x * N1] = e;
            S.flgT[threadIdx.x * N1] = f;
            if (vrank(a) == 0) {
                a.coefE[threadIdx.x * N1] = e;
                a.coefF[threadIdx.x * N1] = f;
            }
        }
        __syncthreads();
        bool ok = true;
        for (int m = 0; m < a.N && ok; m++) {
            const int set = (int)((step * a.N + m) % 3);
            term_phase<ONE_CTA>(S, a, m, set);
            ok = grid_barrier(S, a);
            if (!ok) break;
            close_phase(S, a, m, set);
            ok = cta_ok(S, a);
        }
        if (!ok) break;
        if (!grid_barrier(S, a)) break;
        {
            Prof ph(a);
            horner_phase(S, a, (int)step);
            __syncthreads();
            ph.mark(PR_HORNER);
        }
        if (ONE_CTA && a.histL) {
            // the step's coefficients, kept for a reverse sweep
            const size_t nc = 3 * (size_t)N1;
            uint32_t *hl = a.histL + (size_t)step * nc * a.Lp;
            for (size_t e = threadIdx.x; e < nc * a.Lp; e += NT) hl[e] = __ldcg(&a.coefL[e]);
            for (int e = threadIdx.x; e < (int)nc; e += NT) {
                a.histE[(size_t)step * nc + e] = __ldcg(&a.coefE[e]);
                a.histF[(size_t)step * nc + e] = __ldcg(&a.coefF[e]);
            }
            __syncthreads();
        }
        if (!grid_barrier(S, a)) break;
    }
    __syncthreads();
    tot.mark(PR_TOTAL);
}

__global__ void __launch_bounds__(NT, 1) taylor_kernel(KArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    taylor_body<false>(a, smem_raw);
}

// one trajectory per CTA: its own argument block, a grid of one; registers
// capped so that two CTAs share an SM
__global__ void __launch_bounds__(NT, 2) taylor_batch_kernel(const KArgs *args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KArgs a;
    if (threadIdx.x == 0) a = args[blockIdx.x];
    __syncthreads();
    taylor_body<true>(a, smem_raw);
}

// the same without the register cap (one CTA an SM, no spills)
__global__ void __launch_bounds__(NT, 1) taylor_batch_kernel_wide(const KArgs *args)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ KArgs a;
    if (threadIdx.x == 0) a = args[blockIdx.x];
    __syncthreads();
    taylor_body<true>(a, smem_raw);
}

}  // namespace

size_t smem_bytes(int L, int Lp, int N, int Wcap, int tb, int nwin, bool adj)
{
    (void)L;
    int AV, CV, M;
    vec_sizes(Lp, AV, CV, M);
    size_t o = 0;
    o = align16(o + sizeof(long long) * 3 * (size_t)(nwin > 1 ? nwin : 1) * Wcap);
    o = align16(o + sizeof(uint32_t) * 3 * Wcap);
    o = align16(o + sizeof(int) * 3 * (N + 1));
    o = align16(o + sizeof(int) * 3 * (N + 1));
    o = align16(o + sizeof(uint32_t) * 3 * Lp);
    o = align16(o + sizeof(uint32_t) * (size_t)tb * (AV + CV));
    o = align16(o + sizeof(int) * 2 * tb);
    o = align16(o + sizeof(int) * 2 * tb);
    o = align16(o + sizeof(int) * MISC_INTS);
    if (adj) {
        o = align16(o + sizeof(int) * 3 * (N + 1));
        o = align16(o + sizeof(int) * 3 * (N + 1));
        o = align16(o + sizeof(int) * (N + 1));
        o = align16(o + sizeof(int) * (N + 1));
    }
    return o;
}

int max_coresident_ctas(size_t smem)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(taylor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, taylor_kernel, NT, smem) != cudaSuccess)
        return 0;
    return per * sms;
}

cudaError_t launch_batch(const KArgs *args, int B, size_t smem, cudaStream_t st, int variant)
{
    if (variant == 1) {
        cudaError_t e = cudaFuncSetAttribute(taylor_batch_kernel_wide,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        taylor_batch_kernel_wide<<<B, NT, smem, st>>>(args);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(taylor_batch_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    taylor_batch_kernel<<<B, NT, smem, st>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_integrate(const KArgs &a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(taylor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    KArgs copy = a;
    if (grid <= 1) {
        taylor_kernel<<<1, NT, smem, st>>>(copy);
        return cudaGetLastError();
    }
    void *args[] = {&copy};
    return cudaLaunchCooperativeKernel((const void *)taylor_kernel, dim3(grid), dim3(NT), args,
                                       smem, st);
}

}  // namespace mpt
