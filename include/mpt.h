/*
 * mpt.h -- C ABI of the GB300 multiple-precision Taylor integrator for the
 * Lorenz system (Dimova et al., "OpenMP parallelization of multiple precision
 * Taylor series method", arXiv 1908.09301).
 *
 * The library computes, on one GPU and entirely in its own CUDA kernels, the
 * Taylor step of Sec. 2:
 *   - Eq. (1)  dx/dt = -sigma x + sigma y, dy/dt = R x - y - x z, dz/dt = x y - b z;
 *   - Eq. (3)  the recursion for the normalized Taylor coefficients
 *              alpha_i, beta_i, gamma_i (i = 0..N), whose Cauchy sums
 *              sum_{k=0}^{i} alpha_{i-k} gamma_k and sum_{k=0}^{i} alpha_{i-k} beta_k
 *              are the reductions Sec. 2 and Sec. 4 parallelise;
 *   - Eq. (2)  x_{n+1} = x_n + sum_{i=1}^{N} alpha_i tau^i (same for y, z),
 *              evaluated by Horner's rule as the complexity remark of Sec. 2 says.
 *
 * Number format.  A number with L 32-bit limbs is (sign, exp, limb[L]) with
 *   value = (-1)^sign * sum_{j<L} limb[j] * 2^(32*(exp-L+j)),
 * limb[0] least significant, limb[L-1] != 0, sign in {0, 1}; zero is
 * sign = 0, exp = 0, all limbs 0.  |exp| <= 2^30.  Arrays of numbers are SoA:
 * signs[n], exps[n], limbs[n][L].
 *
 * Arithmetic.  trunc_L(v) keeps the top L limbs of |v| counted from its top
 * non-zero limb on the absolute 2^32 grid and drops the rest (toward zero).
 * Every bracket of Eq. (3) is formed exactly from the stored coefficients and
 * parameters and then coefficient_{i+1} = trunc_L(bracket / (i+1)); every
 * Horner step is h_i = trunc_L(h_{i+1} * tau + c_i) with an exact product and
 * sum, starting from h_N = c_N.  Results do not depend on how the GPU splits
 * the sums, so they are bit-identical across launch shapes.
 *
 * Errors.  Every int-returning call returns MPT_OK (0) or a negative code and
 * never throws; mpt_last_error() gives a message for the calling thread.
 * Device-side conditions (exponent range, a bounded wait that expired) are
 * reported by the call that launched the work, which waits for it.
 *
 * Threads.  A context may be used by one host thread at a time.
 */
#ifndef MPT_H
#define MPT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MPT_OK 0
#define MPT_EINVAL (-1)    /* bad argument: sizes, a malformed number string, a null pointer */
#define MPT_ENOMEM (-2)    /* a host or device allocation failed */
#define MPT_ERANGE (-3)    /* an exponent left |exp| <= 2^30, or the terms of one exact sum
                              span more limbs than the accumulator holds */
#define MPT_ETIMEDOUT (-4) /* a bounded device-side wait expired; the context stays usable */
#define MPT_ECUDA (-5)     /* a CUDA runtime call failed (message in mpt_last_error) */

typedef struct mpt_ctx mpt_ctx;

/* Number of 32-bit limbs for K decimal digits: ceil(K * log2(10) / 32). */
int mpt_limbs_for_digits(int K_digits);

/*
 * Create a context for the Taylor method of order N (Sec. 2, Eq. (2)) with
 * L-limb numbers.  L_limbs == 0 takes L = mpt_limbs_for_digits(K_digits).
 * tau, sigma, R, b are decimal ("0.01", "-1.5e-3") or rational ("8/3")
 * strings; each becomes trunc_L of its exact value (Sec. 2 gives
 * sigma = 10, R = 28, b = 8/3; Sec. 5 takes tau = 0.01).  cuda_stream is a
 * cudaStream_t (0 = the legacy default stream) on which all work of this
 * context is queued; it must belong to the current device.  The context owns
 * all the device memory it needs.  Limits: 1 <= L <= 1024, 1 <= N <= 4096, and
 * the per-CTA tables for (L, N) must fit in shared memory (else MPT_EINVAL).
 * The state starts at (0, 0, 0).
 */
int mpt_init(mpt_ctx **ctx, int K_digits, int N_order, int L_limbs, const char *tau,
             const char *sigma, const char *R, const char *b, uint64_t cuda_stream);

/*
 * trunc_L of the exact value of a decimal ("-15.8", "1e-20") or rational
 * ("8/3", "-1.5/0.25") string, as one number in the interchange layout
 * (host memory, L limbs).  Host only; no device is needed.  MPT_EINVAL for
 * a malformed string or zero denominator, MPT_ERANGE for |exp| > 2^30.
 */
int mpt_parse_number(const char *str, int L, int32_t *sign, int32_t *exp, uint32_t *limbs);

/* Release the context and its device memory (null is accepted). */
void mpt_destroy(mpt_ctx *ctx);

/* L and N of the context. */
int mpt_get_dims(const mpt_ctx *ctx, int *L, int *N);

/*
 * Set the state (x_n, y_n, z_n) = (alpha_0, beta_0, gamma_0) of Sec. 2 from
 * decimal or rational strings, each truncated to L limbs (Sec. 5's benchmark
 * point is "-15.8", "-17.48", "35.64").
 */
int mpt_set_state(mpt_ctx *ctx, const char *x0, const char *y0, const char *z0);

/*
 * Set / read the state as 3 numbers (x, y, z) in the interchange layout:
 * signs[3], exps[3], limbs[3][L], all HOST memory owned by the caller.
 * set_state_raw rejects non-normalised numbers with MPT_EINVAL.  get_state
 * waits for the context's queued work.
 */
int mpt_set_state_raw(mpt_ctx *ctx, const int32_t *signs, const int32_t *exps,
                      const uint32_t *limbs);
int mpt_get_state(mpt_ctx *ctx, int32_t *signs, int32_t *exps, uint32_t *limbs);

/* The truncated parameters (sigma, R, b, tau) as 4 numbers, host memory. */
int mpt_get_params(mpt_ctx *ctx, int32_t *signs, int32_t *exps, uint32_t *limbs);

/* One Taylor step (Eq. (3) for i = 0..N-1, then Eq. (2) by Horner). */
int mpt_step(mpt_ctx *ctx);

/*
 * nsteps Taylor steps in one device launch.  If record_every > 0 the state
 * after every record_every-th step is written to rec_* (nsteps / record_every
 * records of 3 numbers, layout [record][component] for signs and exps and
 * [record][component][L] for limbs).  The rec_* pointers may be host or
 * device memory (CUDA unified addressing tells them apart); they may be null
 * when record_every <= 0.  The call returns when the work is done.
 */
int mpt_integrate(mpt_ctx *ctx, int64_t nsteps, int64_t record_every, int32_t *rec_signs,
                  int32_t *rec_exps, uint32_t *rec_limbs);

/*
 * Queue nsteps steps on the context's stream and return at once (no records).
 * Finish with mpt_wait, which reports device-side errors; until then the
 * context accepts no other launch, and the calls that read or set the state
 * wait first.  On an error the state is put back to where the launch began.
 */
int mpt_launch(mpt_ctx *ctx, int64_t nsteps);
int mpt_wait(mpt_ctx *ctx);

/*
 * Shortened sums (pipelined kernel; results are identical either way).  Each
 * bracket of Eq. (3) and each Horner step of Eq. (2) keeps only the top L
 * limbs of an exact sum, so by default the products of a sum leave out the
 * columns more than L + 3 + 2 limbs below the sum's largest term.  The
 * dropped part is below 2^(32 (c0 + 2)) (c0: the lowest column kept); when
 * the digits of the computed sum between that bound and the result's lowest
 * kept limb are all zero or all ones (exact cancellation, special data such
 * as a fixed point), the launch stops and the library runs it again from the
 * same state with every product in full, so the result is always the exact
 * one.  mpt_set_exact(ctx, 1) makes every launch full from the start
 * (0 restores the default).
 *
 * mpt_get_counters: the number of such full reruns since the context was
 * made, and the 8 x 8 limb-product chunks (64 limb multiply-adds each) the
 * last launch executed in the pipelined kernel (its rerun included; 0 for
 * the lock-step kernel, which does not count).  Waits for queued work.
 * (Not part of the paper.)
 */
int mpt_set_exact(mpt_ctx *ctx, int on);
int mpt_get_counters(mpt_ctx *ctx, int64_t *exact_reruns, int64_t *chunks);

/*
 * The Taylor coefficients of the most recent step: 3*(N+1) numbers,
 * component-major (alpha_0..alpha_N, beta_0..beta_N, gamma_0..gamma_N;
 * index 0 is the state the step started from), host memory.
 */
int mpt_get_coefficients(mpt_ctx *ctx, int32_t *signs, int32_t *exps, uint32_t *limbs);

/*
 * Launch shape.  ctas = 0 lets the library choose; otherwise the coefficient
 * phase runs on exactly that many CTAs (1 .. number of SMs).  Results do not
 * depend on it.
 */
int mpt_set_launch(mpt_ctx *ctx, int ctas);
int mpt_get_launch(const mpt_ctx *ctx, int *ctas);

/*
 * Terms a worker CTA of the pipelined kernel stages per batch (1 .. the
 * largest that fits in shared memory; 0 = that largest, the default).
 * Results do not depend on it; the autotuner searches it with the CTA count.
 */
int mpt_set_pipe_batch(mpt_ctx *ctx, int tb);

/*
 * Kernel organisation (results are identical): 1 = lock-step (every CTA
 * takes a share of each index's products, grid barrier, every CTA closes the
 * brackets); 2 = pipelined (a CTA cluster closes the brackets and runs
 * Horner while the other CTAs compute the next index's inner Cauchy sums);
 * 0 = the library's choice (pipelined for large L x N).  mpt_get_kernel
 * reports the organisation the next launch uses.
 */
int mpt_set_kernel(mpt_ctx *ctx, int kind);
int mpt_get_kernel(const mpt_ctx *ctx, int *kind);

/*
 * A general three-component quadratic system instead of Lorenz.  The paper
 * notes (Sec. 2, after Fig. 1) that the recursion of Eq. (3) is automatic
 * differentiation, so any right-hand side built from sums and products gives
 * Cauchy sums of the same form.  For
 *     x_k' = sum A x_j + sum s x_i x_j + c_k        (k = 0, 1, 2)
 * the coefficients are x_k[m+1] = trunc_L(bracket / (m+1)) with the exact
 * bracket  sum A x_j[m] + sum s sum_{l=0}^{m} x_i[m-l] x_j[l] + c_k [m = 0],
 * and the step is Eq. (2) by Horner's rule with the context's tau.
 *   params[npar]:   parameter strings (decimal or a/b), parsed exactly and
 *                   truncated to L limbs; npar <= 15.
 *   fixed[nfixed][4] {target, neg, p, j}: the term p * x_j (p >= 0, j >= 0),
 *                   the lone x_j (p = -1) or the constant p (j = -1; index 0
 *                   only); neg 1 subtracts it; nfixed <= 32.
 *   quad[nquad][4] {target, neg, i, j}: the Cauchy product x_i * x_j;
 *                   nquad <= 16.
 * Host arrays, copied; targets and components are 0, 1, 2.  Malformed
 * input: MPT_EINVAL, the context unchanged.  From then on the context runs
 * the lock-step kernel (mpt_set_kernel(2) is refused) and mpt_get_params is
 * refused; the state is kept.  Synchronous on the context's stream.
 */
int mpt_set_system(mpt_ctx *ctx, int npar, const char *const *params, int nfixed,
                   const int32_t *fixed, int nquad, const int32_t *quad);

/*
 * Bound of every device-side wait (grid barrier, hand-over flags), in polls;
 * 0 restores the default (tens of millions, seconds).  When a wait runs out
 * the launch stops, the call returns MPT_ETIMEDOUT and the state is put back
 * to where the launch began; the context stays usable.  A small bound is the
 * way to exercise that path on purpose.  (Not part of the paper.)
 */
int mpt_set_wait_limit(mpt_ctx *ctx, int64_t polls);

/*
 * Per-phase cycle profile (a device-side stats block; not part of the
 * paper).  With profiling on, every launch accumulates SM clock cycles per
 * phase; mpt_get_profile copies up to n counters of the last launch.
 * Layout: rows of 16 slots (0 window placement, 1 operand staging, 2 limb
 * products, 3 accumulator flush, 4 wait, 5 close (normalise + divide),
 * 6 Horner, 7 Horner products, 8 Horner close, 9 whole launch, 10-15 finer
 * marks of the pipelined kernel).  Row 0 is the first CTA (the pipelined
 * kernel: its beta' bracket CTA), row 1 the last CTA; the pipelined kernel
 * adds one row per CTA of the launch (row 2 + CTA index), up to 2 + the
 * device's SM count rows in all.  After those rows (at (2 + SM count) * 16)
 * the pipelined kernel writes a per-index timeline of the launch's last step:
 * 9 rows of 4097 global-timer stamps in ns (row r, index m at r * 4097 + m):
 * the beta' bracket at the start of index m, after its wait for the other
 * CTAs' sums, after publishing; the last edge CTA and the last worker to
 * finish index m; the gamma' bracket after publishing; the last edge CTA to
 * see coefficient m, to start its products, to end them.  Off by default.
 */
int mpt_set_profiling(mpt_ctx *ctx, int on);
int mpt_get_profile(mpt_ctx *ctx, int64_t *cycles, int n);

/*
 * INT32 multiply-add throughput probe (sets the roofline of the limb
 * products).  Runs instruction-form `variant` (0 mad.lo.u32, 1 mad.hi.u32,
 * 2 mad.wide.u32, 3 limb product with mad.lo.cc/madc.hi.cc/addc, 4 two
 * mad.wide.u32 on 16-bit halves, 5 mad.wide.u32 plus a wide carry word,
 * 6 mad.lo.cc+addc and mad.hi.cc+addc, 7 mad.lo+mad.hi, 8 mul.wide plus
 * add.cc chains, 9 a row of 8 limb products with the carries along the row:
 * one madc.lo.cc chain, one madc.hi.cc chain, two addc) on one CTA of `threads` threads (multiple of 32, <= 1024)
 * per SM, 8 independent chains per thread, `iters` rounds.  Outputs: mean
 * loop cycles of a CTA, kernel time in ms, number of distinct SMs used, grid
 * size.  Allocates its own scratch buffers.  Returns 0 or a cudaError_t
 * value.  (Not part of the paper: a measurement aid.)
 */
int mpt_int_peak_run(int variant, int threads, int iters, double *mean_cycles, double *ms,
                     int *distinct_sms, int *grid_out);

/*
 * Batch of independent trajectories (an ensemble of the problem of Sec. 2:
 * B initial points, each with its own precision L_j and order N_j; the
 * paper integrates one trajectory at a time).  Every trajectory takes
 * nsteps steps of exactly the arithmetic of mpt_integrate (bit-identical
 * to a single-trajectory run with the same L, N, parameters and state); the
 * trajectories run concurrently, one CTA each.
 *
 * Arguments: B >= 1; Ls[B], Ns[B] as the L and N of mpt_init (L <= 1024,
 * N <= 4096); the parameters as decimal or rational strings, converted to
 * each trajectory's L (as mpt_init does); the states in host memory, in the
 * interchange layout, packed: signs[3B] and exps[3B] (trajectory j's x, y,
 * z at 3j..3j+2) and limbs (trajectory j's three numbers of L_j limbs each
 * at offset 3 (L_0 + ... + L_{j-1})).  They are read at the start and, on
 * success, overwritten with the states after nsteps steps.  Work is queued
 * on cuda_stream (0 = legacy default stream); the call allocates its device
 * buffers, returns when the steps are done and frees them.
 *
 * Errors: MPT_EINVAL for a size outside the limits, a null pointer or a
 * malformed number (the message names the trajectory), MPT_ERANGE for an
 * exponent or accumulator window out of range in any trajectory, MPT_ENOMEM
 * or MPT_ECUDA from the device.  On any error the states are left as they
 * were.  (Not part of the paper.)
 */
int mpt_integrate_batch(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps,
                        const char *tau, const char *sigma, const char *R, const char *b,
                        int32_t *signs, int32_t *exps, uint32_t *limbs, uint64_t cuda_stream);

/*
 * The same batch with a launch shape of the caller's choosing (results are
 * identical for every shape: the sums are exact).  shape[3] (host; null =
 * the library's choice): the kernel variant (0: registers capped so that two
 * trajectories share an SM; 1: not capped, one trajectory an SM), the terms
 * staged per batch (0: as many as fit, up to 64; else 1..256), the copies of
 * the accumulator windows the products add into (0: as many as fit, up to
 * 8; else 1..8).  MPT_EINVAL for a value outside these ranges or a shape
 * whose shared memory does not fit.  The project's autotuner picks shapes
 * per workload with it (paper_1908_09301_gb300/autotune.py).
 */
int mpt_integrate_batch_shape(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps,
                              const char *tau, const char *sigma, const char *R, const char *b,
                              int32_t *signs, int32_t *exps, uint32_t *limbs, const int32_t *shape,
                              uint64_t cuda_stream);

/*
 * The same batch with parameters of each trajectory's own: sigma[j], R[j],
 * b[j] (B strings each, host) for trajectory j; tau is common.  Trajectories
 * with equal L and equal strings share one parse.  Used for the derivatives
 * of the flow with respect to the parameters (runs at sigma +- h, ...).
 * Errors and layouts as mpt_integrate_batch.
 */
int mpt_integrate_batch_params(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps,
                               const char *tau, const char *const *sigma, const char *const *R,
                               const char *const *b, int32_t *signs, int32_t *exps,
                               uint32_t *limbs, uint64_t cuda_stream);

/*
 * Derivatives of the n-step map (x0, y0, z0, sigma, R, b) -> (x, y, z) after
 * nsteps steps of Eq. (3) and Eq. (2) (Sec. 2; the paper has no derivatives,
 * this is the differentiation of its flow) by a reverse sweep in the same
 * L-limb format.  It is the derivative of the exact-arithmetic order-N map,
 * evaluated at the stored (truncated) coefficients: going j = N .. 0 through
 * each step, the adjoint of coefficient j is the exact sum of gbar tau^j
 * (Eq. (2)), the linear terms of the brackets E_j of Eq. (3) and the Cauchy
 * sums of the brackets E_i, i >= j, through their factor of index j; the
 * adjoint of bracket E_{j-1} is that sum divided by j and truncated once, the
 * adjoint of the step's starting state is the sum at j = 0 truncated, the
 * parameter adjoints gain sum_i Ebar_i dE_i/d(sigma, R, b) per step (one
 * truncation each), and tau^j is P_j = trunc_L(P_{j-1} tau).  The state is
 * checkpointed every `checkpoint_every` steps (0: 50) and the coefficients of
 * a segment's steps are recomputed before its sweep, so the cost is about
 * four forward runs per adjoint vector.
 *
 * mpt_backward_raw: B trajectories with a common L and N, G adjoint vectors
 * per trajectory (item j*G + g belongs to trajectory j); all arrays host
 * memory in the interchange layout.  par: sigma, R, b, tau (4 numbers);
 * st: the initial states (3B numbers); g: in, the adjoints of the final
 * states (3 B G numbers), out, the adjoints of the initial states; th: out,
 * the adjoints of (sigma, R, b) of every item (3 B G numbers).  MPT_EINVAL
 * for sizes outside those of mpt_init or a malformed number; MPT_ERANGE /
 * MPT_ENOMEM / MPT_ECUDA from the device.  Synchronous on cuda_stream.
 */
int mpt_backward_raw(int B, int G, int L, int N, int64_t nsteps, int checkpoint_every,
                     const int32_t *par_signs, const int32_t *par_exps, const uint32_t *par_limbs,
                     const int32_t *st_signs, const int32_t *st_exps, const uint32_t *st_limbs,
                     int32_t *g_signs, int32_t *g_exps, uint32_t *g_limbs, int32_t *th_signs,
                     int32_t *th_exps, uint32_t *th_limbs, uint64_t cuda_stream);

/*
 * The same in float64 for B initial points given as strings (x0[B * 3],
 * point-major, as mpt_set_state) and parameters as strings (as mpt_init):
 *   g[B * 3]:        the upstream gradient of each final state (exact doubles);
 *   g_x0[B * 3]:     out, g^T J with respect to each point's x0, y0, z0;
 *   g_params[3]:     out, g^T J with respect to sigma, R, b, summed over points;
 *   jac[B * 3 * 6]:  out (nullable), J per point, [output][input]; when given,
 *                    three sweeps per point (gbar = e_x, e_y, e_z) and g_x0,
 *                    g_params formed from J in double.
 * Every number is rounded once to the nearest double.
 */
int mpt_backward(int B, int L, int N, int64_t nsteps, const char *tau, const char *sigma,
                 const char *R, const char *b, const char *const *x0, const double *g,
                 int checkpoint_every, double *g_x0, double *g_params, double *jac,
                 uint64_t cuda_stream);

/*
 * The 3 x 6 Jacobians of the same map by central differences of bit-exact
 * runs: J[:, i] = (F(u + h e_i) - F(u - h e_i)) / (2h), h = 10^(-h_digits)
 * (0: 100), each difference formed exactly and rounded once to double; its
 * error is about |F'''| h^2 + 2^(-32 (L-1)) |F| / h.  The 12 B runs go to one
 * batch launch.  A check of mpt_backward that needs no adjoint.
 * jac[B * 3 * 6], [output][input]; errors as mpt_integrate_batch, MPT_EINVAL
 * for h_digits outside 1..10000.
 */
int mpt_jacobian_fd(int B, int L, int N, int64_t nsteps, const char *tau, const char *sigma,
                    const char *R, const char *b, const char *const *x0, int h_digits, double *jac,
                    uint64_t cuda_stream);

/*
 * Allocation-free stepping (the paper has no counterpart; it is a service of
 * this library).  Some callers cannot call cudaMalloc when they step: code
 * whose device memory belongs to a pool it may not grow, a plug-in of a
 * runtime that forbids allocation after start-up, or code that must not
 * synchronise with the allocator.  mpt_integrate_noalloc runs nsteps Taylor
 * steps (the same arithmetic as mpt_integrate, bit-identical results) with
 * all working memory in one static device array of
 * MPT_NOALLOC_SCRATCH_BYTES (4 MiB) that every GPU loading this library
 * holds until the process exits; it calls no allocating routine.
 *
 * Arguments: L limbs and order N as for mpt_init; the parameters sigma, R,
 * b, tau as 4 numbers (par_signs[4], par_exps[4], par_limbs[4][L]); the
 * state x, y, z as 3 numbers (signs[3], exps[3], limbs[3][L]), read at the
 * start and overwritten with the state after nsteps steps.  All six arrays
 * are in the interchange layout and must be memory the current device can
 * read and write (device, managed or registered host memory); they stay the
 * caller's.  Work is queued on cuda_stream (0 = legacy default stream) and
 * the call returns when it is done.
 *
 * Limits and errors: MPT_EINVAL for sizes outside those of mpt_init, for a
 * null or unreachable pointer, for a malformed number, and when L and N need
 * more scratch than the array holds (about 12 (N+1) L bytes plus a few
 * kilobytes: L <= 64 fits every N, L = 208 (2000 digits) fits N <= 1641,
 * L = 1024 fits N <= 319); the message gives the bytes needed.  On any error
 * the caller's state is left as it was.
 *
 * The first call on a device takes the array's device address and queries
 * the device (with that device current); make that first call before any
 * stream capture.  Every call on a device shares the one array and clears
 * the parts that must start at zero itself; calls that overlap on the GPU
 * (two host threads, or two streams at once) race on it and must be
 * serialised by the caller.
 */
#define MPT_NOALLOC_SCRATCH_BYTES 4194304u
int mpt_integrate_noalloc(int L, int N, int64_t nsteps, const int32_t *par_signs,
                          const int32_t *par_exps, const uint32_t *par_limbs, int32_t *signs,
                          int32_t *exps, uint32_t *limbs, uint64_t cuda_stream);

/* Message for an error code; message of the calling thread's last error. */
const char *mpt_strerror(int code);
const char *mpt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MPT_H */
