// mpt_kernel.cuh -- shared declarations between the host side of libmpt and
// the Taylor-step kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpt {

constexpr int W = 8;         // columns per limb-product block (register tile)
constexpr int NT = 256;      // threads per CTA of the lock-step kernel
constexpr int PT = 512;      // threads per CTA of the pipelined kernel
constexpr int MAX_L = 1024;  // limbs per number
constexpr int MAX_N = 4096;  // Taylor order (exponent tables live in shared memory)

// status word values written by the device (0 = fine)
constexpr int DEV_ERANGE = 1;    // exponent range or accumulator window exceeded
constexpr int DEV_TIMEOUT = 2;   // a bounded wait expired
constexpr int DEV_INTERNAL = 3;  // an internal invariant failed (carry did not settle)
constexpr int DEV_INEXACT = 4;   // a shortened sum could not be shown to give the exact
                                 // truncated result: the host reruns the launch in full

// Shortened products (pipelined kernel).  Of an exact bracket sum E only the
// top L + 1 limbs of |E| reach the truncated quotient (division by a small
// integer, then truncation to L limbs), so each part of a sum computes only
// the columns at or above  c0 = T - L - 3 - CUT_GUARD  (T: the part's largest
// term top, e_a + e_b) and drops the rest.  What is dropped is below
// 2^(32 (c0 + 2)) in magnitude (fewer than 2^31 limb pairs below the cut,
// each below 2^64), so if the digits of the computed |E'| between limb c0 + 2
// and the quotient's lowest kept limb are neither all zero nor all ones, E
// and E' give the same sign, exponent and limbs.  Otherwise the launch ends
// with DEV_INEXACT and the host runs it again with every column.
constexpr int CUT_GUARD = 2;

// flag bits of a stored number
constexpr int F_NEG = 1;
constexpr int F_NZ = 2;

struct KArgs {
    int L, Lp, P, N, Wcap;  // limbs, padded limbs (multiple of W), Lp / W, order, window
    int tb;                 // terms per staging batch
    uint32_t *coefL;        // [3][N+1][Lp]   coefficients of the current step
    int32_t *coefE;         // [3][N+1]
    int32_t *coefF;         // [3][N+1]
    const uint32_t *parL;   // [4][Lp]        sigma, R, b, tau
    const int32_t *parE;    // [4]
    const int32_t *parF;    // [4]
    uint32_t *stL;          // [3][Lp]        state (x, y, z)
    int32_t *stE;           // [3]
    int32_t *stF;           // [3]
    long long *gwin;        // [3 sets][3 targets][Wcap] cross-CTA accumulators
    unsigned *bar;          // [2] grid barrier: arrival count, generation
    int *status;            // [1]
    int32_t *recS;          // [nrec][3]      records in the interchange layout
    int32_t *recE;          // [nrec][3]
    uint32_t *recL;         // [nrec][3][L]
    long long nsteps;
    long long record_every;
    long long *prof;        // [2][PROF_SLOTS] per-phase SM cycles of CTAs 0 and G-1, or null
    long long *timeline;    // pipelined kernel, profiling: [TL_ROWS][MAX_N + 1] global-timer
                            // stamps of each index of the launch's last step (or null)
    long long spin_limit;   // polls before a device-side wait gives up
    int vG, vg;             // lock-step kernel: grid size and CTA index it runs as
                            // (vG = 0: the launch's own grid); a batch runs each
                            // trajectory on one CTA (vG = 1, vg = 0)
    // lock-step kernel: a general three-component quadratic system instead of
    // Lorenz (null: the Lorenz brackets of Eq. (3), parameters sigma, R, b, tau)
    const int *sysT;        // [sysNF][4] fixed terms, then [sysNQ][4] Cauchy products
    int sysNF, sysNQ;
    int npar, ptau;         // parameters in parL, tau's index among them
    int nwin;               // lock-step kernel: copies of the three windows the term
                            // phase adds into (warp w uses copy w mod nwin; 0 = 1)
    // batch kernel: after each step, a copy of the step's coefficient table to
    // histL + step 3 (N+1) Lp and histE/F + step 3 (N+1) (null: none)
    uint32_t *histL;
    int32_t *histE, *histF;
    // batch kernel, reverse sweep (the adjoint of Eq. (3) and Eq. (2)): adj = 1;
    // the forward coefficients of the launch's steps (as histL above); the powers
    // of tau [N+1][Lp] the launch computes; parL holds sigma, R, b, tau, then the
    // adjoint gbar of the state (3 rows, replaced step by step) and the
    // parameter adjoints (3 rows, accumulated); coefL holds the adjoint series
    int adj;
    const uint32_t *fwdL;
    const int32_t *fwdE, *fwdF;
    uint32_t *powL;
    int32_t *powE, *powF;
    // tau = trunc_L(p/q) with small p, q (tau_q = 0: not): tau h =
    // (p h - r h 2^(-32 shift)) / q exactly, so a Horner step of Eq. (2) is
    // trunc_L((+-(p h - r h 2^(-32 shift)) + q c_i) / q) with no limb product
    uint32_t tau_p, tau_q, tau_r;
    int tau_shift, tau_neg;
    int exact;              // pipelined kernel: 1 = every product in full (no shortened sums)
    unsigned long long *chunks;  // pipelined kernel: executed 8 x 8 limb-product chunks of
                                 // the launch are added here (null: not counted)
    // pipelined kernel, L < PT: for each divisor d (row d = 1..N: the brackets'
    // m + 1; row 0: tau's q, or 1) and i < L + 2, with d' the odd part of d,
    // 2^(-32 i) mod d' | (2^(32 (i-1)) mod d') << 16 (null: not used)
    const uint32_t *divtab;
    int divtab_rl;  // entries a row (L + 2)
};

// limits of a general system
constexpr int SYS_MAX_PAR = 16;    // parameters, tau included
// rows of parL in a reverse sweep: sigma, R, b, tau, gbar (x, y, z), thbar (sigma, R, b)
constexpr int ADJ_GBAR = 4, ADJ_THBAR = 7, ADJ_NPAR = 10;
constexpr int SYS_MAX_FIXED = 32;  // fixed terms (linear and constant)
constexpr int SYS_MAX_QUAD = 16;   // Cauchy products

constexpr long long DEFAULT_SPIN_LIMIT = 20LL * 1000 * 1000;

// rows of the per-index timeline (global timer, ns) of the pipelined kernel:
// the beta' bracket at the start of index m, after its wait for the other
// CTAs' sums, after publishing; the last edge CTA and the last worker (or
// outer-pair CTA) to count index m done; the gamma' bracket after publishing;
// the last edge CTA to see coefficient m, to start its products, to end them
enum { TL_B_START = 0, TL_B_WAITED = 1, TL_B_PUB = 2, TL_EDGE = 3, TL_WORK = 4, TL_G_PUB = 5,
       TL_E_SEEN = 6, TL_E_MAC = 7, TL_E_MACD = 8, TL_ROWS = 9 };

// phases of the per-phase cycle profile
enum ProfSlot {
    PR_PLACE = 0,   // window placement for an index
    PR_STAGE,       // operand staging
    PR_MAC,         // limb products
    PR_FLUSH,       // shared -> global accumulator flush
    PR_BARRIER,     // grid barrier wait
    PR_CLOSE,       // normalise + divide
    PR_HORNER,      // Horner chains (all of it)
    PR_HMAC,        // Horner products
    PR_HCLOSE,      // Horner normalise + truncate
    PR_TOTAL,       // whole launch
    PR_X1,          // finer marks of the pipelined closer
    PR_X2,
    PR_X3,
    PR_X4,
    PR_X5,
    PR_X6,
    PROF_SLOTS = 16
};

// pipelined kernel: bracket, outer-pair and edge CTAs, and workers
constexpr int PIPE_SETS = 8;  // rotating global accumulator sets / completion counters

struct PArgs {
    unsigned *pub;    // [1] component publications of the launch (monotone, 3 per coefficient)
    unsigned *done;   // [PIPE_SETS] non-bracket CTAs finished with an index (monotone)
    long long *gin;   // [PIPE_SETS][3 brackets][3 parts][Wcap] sums the other CTAs add to the
                      // brackets alpha', beta', gamma' (parts: middle pairs, outer pairs, edge terms)
    long long *imid;  // [PIPE_SETS][4] middle-pair windows without their two newest pairs
    int C;            // CTAs with fixed roles (pipe_fixed_ctas())
    int tb;           // worker term slots per batch (<= pipe_tb_max())
};

size_t pipe_smem_bytes(int L, int Lp, int N, int Wcap, int tb);
int pipe_tb_max();
// CTAs with fixed roles (brackets, outer pairs, edge terms); a launch needs at least one more
int pipe_fixed_ctas();
// co-resident CTAs of the pipelined kernel (one per SM at most; 0 on error)
int pipe_max_ctas(size_t smem);
cudaError_t launch_pipe(const KArgs &a, const PArgs &pa, int grid, size_t smem, cudaStream_t st);

// dynamic shared memory bytes for a configuration (adj: the reverse sweep's tables too)
size_t smem_bytes(int L, int Lp, int N, int Wcap, int tb, int nwin = 1, bool adj = false);
// launch nsteps steps on `grid` CTAs (cooperative when grid > 1)
cudaError_t launch_integrate(const KArgs &a, int grid, size_t smem, cudaStream_t st);
// largest co-resident grid for this smem size (0 on error)
int max_coresident_ctas(size_t smem);
// independent trajectories: CTA j runs the lock-step kernel for args[j] (device
// array of B argument blocks, each with vG = 1, vg = 0); variant 0 caps the
// registers so that two CTAs share an SM, variant 1 does not (one CTA an SM)
cudaError_t launch_batch(const KArgs *args, int B, size_t smem, cudaStream_t st, int variant = 0);

}  // namespace mpt
