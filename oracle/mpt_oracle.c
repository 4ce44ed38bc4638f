/*
 * mpt_oracle.c -- plain, slow, exact CPU oracle for one multiple-precision
 * Taylor step of the Lorenz system (Dimova et al., "OpenMP parallelization of
 * multiple precision Taylor series method", arXiv 1908.09301).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product path (the CUDA
 * library) shares no code with it and must never call it.
 *
 * What it computes (all names follow the paper):
 *   Sec. 2, Eq. (1): dx/dt = -sigma x + sigma y, dy/dt = R x - y - x z,
 *                    dz/dt = x y - b z.
 *   Sec. 2, first coefficients: alpha_0 = x_n, beta_0 = y_n, gamma_0 = z_n.
 *   Sec. 2, Eq. (3): for i = 0..N-1
 *       alpha_{i+1} = ( -sigma alpha_i + sigma beta_i ) / (i+1)
 *       beta_{i+1}  = ( R alpha_i - beta_i - sum_{k=0}^{i} alpha_{i-k} gamma_k ) / (i+1)
 *       gamma_{i+1} = ( sum_{k=0}^{i} alpha_{i-k} beta_k - b gamma_i ) / (i+1)
 *   Sec. 2, Eq. (2) evaluated with Horner's rule (Sec. 2, complexity remark):
 *       h_N = alpha_N,  h_i = h_{i+1} tau + alpha_i,  x_{n+1} = h_0.
 *
 * Number format (the paper uses GMP floats with a precision in bits, Sec. 4-5;
 * the exact format is this project's reading):
 *   value = (-1)^sign * sum_{j<L} limb[j] * 2^(32*(exp-L+j)), limb[L-1] != 0,
 *   zero = (sign 0, exp 0, all limbs 0).
 *   trunc_L(v): keep the top L limbs of |v| counted from its top non-zero limb
 *   on the absolute 2^32 grid, drop the rest (toward zero), keep the sign.
 *
 * Rounding reading: every bracket of Eq. (3) is formed EXACTLY from the stored
 * (already truncated) coefficients and parameters, then divided by (i+1) and
 * truncated once; every Horner step is an exact h*tau + alpha_i followed by
 * one truncation.  The exact sums make the result independent of summation
 * order, so the serial path and the OpenMP path (Sec. 4's per-thread
 * containers sum[2*tid], sum[2*tid+1] folded by the master) agree bit for bit.
 *
 * The adjoint (reverse sweep, orc_adjoint_step / orc_backward): the derivative
 * of the exact-arithmetic order-N step map -- Eq. (3) and Eq. (2) read as
 * exact operations -- with respect to the state and (sigma, R, b), evaluated
 * at the stored coefficients.  With E_i the bracket of Eq. (3) that gives
 * coefficient i+1 and Ebar_i = d(out)/d(E_i), going j = N down to 0:
 *   S_x(j) = gbar_x P_j - sigma Ebar_x,j + R Ebar_y,j
 *            + sum_{i=j}^{N-1} ( -Ebar_y,i gamma_{i-j} + Ebar_z,i beta_{i-j} )
 *   S_y(j) = gbar_y P_j + sigma Ebar_x,j - Ebar_y,j + sum_{i=j}^{N-1} Ebar_z,i alpha_{i-j}
 *   S_z(j) = gbar_z P_j - b Ebar_z,j - sum_{i=j}^{N-1} Ebar_y,i alpha_{i-j}
 * (the terms with Ebar_j are absent at j = N); Ebar_{j-1} = trunc_L(S(j)/j)
 * for j >= 1 and the state's adjoint is trunc_L(S(0)).  P_0 = 1,
 * P_j = trunc_L(P_{j-1} tau) (d(out)/d(c_j) = tau^j by Eq. (2)).  Every S is
 * formed exactly from stored numbers and truncated once.  Per step the
 * parameter adjoints become trunc_L(old + sum_i Ebar_x,i (beta_i - alpha_i)),
 * trunc_L(old + sum_i Ebar_y,i alpha_i), trunc_L(old - sum_i Ebar_z,i gamma_i).
 *
 * Parity status: pinned (closed-form coefficients, exact-fraction brute force,
 * closed-form special case, exact fixed point, symmetry, (K,N) vs larger (K,N),
 * double-precision RK4; the adjoint against exact dual-number derivatives of
 * the order-N map and against central differences of runs) -- see the tests.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ERANGE (-3)

/* largest exponent magnitude (in limbs) a stored number may have */
#define ORC_EXP_MAX (1LL << 30)

/* An L-limb number of the format above; limb points at L words. */
typedef struct {
    int32_t sign;
    int32_t exp;
    uint32_t *limb;
} mpnum;

/* An exact signed dyadic number: (-1)^neg * sum_{j<n} mag[j] * 2^(32*(low+j)).
 * n == 0 means zero.  mag is heap memory owned by the value. */
typedef struct {
    int neg;
    int64_t low;
    int n;
    uint32_t *mag;
} dyadic;

static int g_err; /* sticky error of the current call (per thread below) */
#ifdef _OPENMP
#pragma omp threadprivate(g_err)
#endif

static void *xcalloc(size_t n, size_t sz)
{
    void *p = calloc(n ? n : 1, sz);
    if (!p) g_err = ORC_ENOMEM;
    return p;
}

static dyadic dy_zero(void)
{
    dyadic z = {0, 0, 0, NULL};
    return z;
}

static void dy_free(dyadic *x)
{
    free(x->mag);
    *x = dy_zero();
}

/* drop leading zero limbs so that mag[n-1] != 0 (or n == 0) */
static void dy_trim(dyadic *x)
{
    while (x->n > 0 && x->mag[x->n - 1] == 0) x->n--;
    if (x->n == 0) {
        free(x->mag);
        *x = dy_zero();
    }
}

static int mp_is_zero(const mpnum *a, int L)
{
    for (int j = 0; j < L; j++)
        if (a->limb[j]) return 0;
    return 1;
}

/* the exact value of an L-limb number */
static dyadic dy_from_mp(const mpnum *a, int L)
{
    if (mp_is_zero(a, L)) return dy_zero();
    dyadic r;
    r.neg = a->sign != 0;
    r.low = (int64_t)a->exp - L;
    r.n = L;
    r.mag = xcalloc((size_t)L, sizeof(uint32_t));
    if (!r.mag) return dy_zero();
    memcpy(r.mag, a->limb, (size_t)L * sizeof(uint32_t));
    return r;
}

/* exact product of two L-limb numbers: schoolbook, 2L limbs */
static dyadic dy_mul(const mpnum *a, const mpnum *b, int L)
{
    if (mp_is_zero(a, L) || mp_is_zero(b, L)) return dy_zero();
    dyadic r;
    r.neg = (a->sign != 0) != (b->sign != 0);
    r.low = ((int64_t)a->exp - L) + ((int64_t)b->exp - L);
    r.n = 2 * L;
    r.mag = xcalloc((size_t)(2 * L), sizeof(uint32_t));
    if (!r.mag) return dy_zero();
    for (int i = 0; i < L; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < L; j++) {
            uint64_t t = (uint64_t)a->limb[i] * b->limb[j] + r.mag[i + j] + carry;
            r.mag[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        r.mag[i + L] = (uint32_t)carry;
    }
    dy_trim(&r);
    return r;
}

/* compare magnitudes of two aligned limb vectors of length n */
static int mag_cmp(const uint32_t *x, const uint32_t *y, int n)
{
    for (int j = n - 1; j >= 0; j--) {
        if (x[j] != y[j]) return x[j] > y[j] ? 1 : -1;
    }
    return 0;
}

/* exact signed sum x + y (neither argument is consumed) */
static dyadic dy_add(const dyadic *x, const dyadic *y)
{
    if (y->n == 0) {
        dyadic r = *x;
        if (x->n) {
            r.mag = xcalloc((size_t)x->n, sizeof(uint32_t));
            if (!r.mag) return dy_zero();
            memcpy(r.mag, x->mag, (size_t)x->n * sizeof(uint32_t));
        }
        return r;
    }
    if (x->n == 0) return dy_add(y, x);
    int64_t low = x->low < y->low ? x->low : y->low;
    int64_t topx = x->low + x->n, topy = y->low + y->n;
    int64_t top = (topx > topy ? topx : topy) + 1;
    int n = (int)(top - low);
    uint32_t *ax = xcalloc((size_t)n, sizeof(uint32_t));
    uint32_t *ay = xcalloc((size_t)n, sizeof(uint32_t));
    dyadic r = dy_zero();
    if (!ax || !ay) goto out;
    memcpy(ax + (x->low - low), x->mag, (size_t)x->n * sizeof(uint32_t));
    memcpy(ay + (y->low - low), y->mag, (size_t)y->n * sizeof(uint32_t));
    r.low = low;
    r.n = n;
    r.mag = xcalloc((size_t)n, sizeof(uint32_t));
    if (!r.mag) { r = dy_zero(); goto out; }
    if (x->neg == y->neg) {
        uint64_t carry = 0;
        for (int j = 0; j < n; j++) {
            uint64_t t = (uint64_t)ax[j] + ay[j] + carry;
            r.mag[j] = (uint32_t)t;
            carry = t >> 32;
        }
        r.neg = x->neg;
    } else {
        /* subtract the smaller magnitude from the larger one */
        int c = mag_cmp(ax, ay, n);
        const uint32_t *big = c >= 0 ? ax : ay, *small = c >= 0 ? ay : ax;
        uint64_t borrow = 0;
        for (int j = 0; j < n; j++) {
            uint64_t t = (uint64_t)big[j] - small[j] - borrow;
            r.mag[j] = (uint32_t)t;
            borrow = (t >> 32) & 1;
        }
        r.neg = c >= 0 ? x->neg : y->neg;
    }
    dy_trim(&r);
out:
    free(ax);
    free(ay);
    return r;
}

/* x += y, replacing x */
static void dy_accumulate(dyadic *x, const dyadic *y)
{
    dyadic s = dy_add(x, y);
    dy_free(x);
    *x = s;
}

static dyadic dy_neg(dyadic x)
{
    if (x.n) x.neg = !x.neg;
    return x;
}

static void mp_set_zero(mpnum *out, int L)
{
    out->sign = 0;
    out->exp = 0;
    memset(out->limb, 0, (size_t)L * sizeof(uint32_t));
}

static int check_exp(int64_t e)
{
    if (e > ORC_EXP_MAX || e < -ORC_EXP_MAX) {
        g_err = ORC_ERANGE;
        return 0;
    }
    return 1;
}

/* out = trunc_L(x) */
static void dy_trunc(const dyadic *x, int L, mpnum *out)
{
    if (x->n == 0) { mp_set_zero(out, L); return; }
    int t = x->n - 1; /* x is trimmed: mag[t] != 0 */
    int64_t e = x->low + t + 1;
    if (!check_exp(e)) { mp_set_zero(out, L); return; }
    for (int j = 0; j < L; j++) {
        int src = t - (L - 1) + j;
        out->limb[j] = src >= 0 ? x->mag[src] : 0u;
    }
    out->exp = (int32_t)e;
    out->sign = x->neg;
}

/* out = trunc_L(x / d) for an integer d >= 1: exact long division from the top.
 * floor(|x| / (d 2^(32 s))) = floor(floor(|x| / 2^(32 s)) / d), so only the
 * limbs of |x| at or above position s matter; positions below x's lowest
 * limb are zero. */
static void dy_div_trunc(const dyadic *x, uint32_t d, int L, mpnum *out)
{
    if (x->n == 0) { mp_set_zero(out, L); return; }
    int t = x->n - 1;
    int64_t T = x->low + t + 1;              /* 2^(32(T-1)) <= |x| < 2^(32T) */
    int64_t eq = x->mag[t] >= d ? T : T - 1; /* exponent of |x|/d */
    int64_t s = eq - L;                      /* lowest limb position kept */
    int nX = (int)(T - s);                   /* L or L+1 */
    uint32_t *X = xcalloc((size_t)nX, sizeof(uint32_t));
    uint32_t *Q = xcalloc((size_t)nX, sizeof(uint32_t));
    if (!X || !Q) { free(X); free(Q); mp_set_zero(out, L); return; }
    for (int j = 0; j < nX; j++) {
        int64_t src = s + j - x->low;
        X[j] = (src >= 0 && src < x->n) ? x->mag[src] : 0u;
    }
    uint64_t r = 0;
    for (int j = nX - 1; j >= 0; j--) {
        uint64_t num = (r << 32) | X[j];
        Q[j] = (uint32_t)(num / d);
        r = num % d;
    }
    /* the quotient has exactly L significant limbs: Q[L-1] != 0 and, when
     * nX == L+1, Q[L] == 0 */
    if (!check_exp(eq)) { mp_set_zero(out, L); goto out; }
    for (int j = 0; j < L; j++) out->limb[j] = Q[j];
    out->exp = (int32_t)eq;
    out->sign = x->neg;
out:
    free(X);
    free(Q);
}

/* ----------------------------------------------------------------------- */
/* Eq. (3): the two Leibniz/Cauchy sums s1 = sum_k alpha_{i-k} gamma_k and
 * s2 = sum_k alpha_{i-k} beta_k.  With nthreads > 1 this is Sec. 4's manual
 * OpenMP reduction: thread tid keeps its part of s1 in sum[2*tid] and its part
 * of s2 in sum[2*tid+1], the k-loop is split into near-equal static chunks,
 * and after the implicit barrier the master folds the containers. */
static void cauchy_sums(int i, int L, const mpnum *al, const mpnum *be,
                        const mpnum *ga, int nthreads, dyadic *s1, dyadic *s2)
{
    *s1 = dy_zero();
    *s2 = dy_zero();
    if (nthreads <= 1) {
        for (int k = 0; k <= i; k++) {
            dyadic p1 = dy_mul(&al[i - k], &ga[k], L);
            dyadic p2 = dy_mul(&al[i - k], &be[k], L);
            dy_accumulate(s1, &p1);
            dy_accumulate(s2, &p2);
            dy_free(&p1);
            dy_free(&p2);
        }
        return;
    }
#ifdef _OPENMP
    dyadic *sum = calloc((size_t)(2 * nthreads), sizeof(dyadic));
    int errs = 0;
    if (!sum) { g_err = ORC_ENOMEM; return; }
#pragma omp parallel num_threads(nthreads) reduction(| : errs)
    {
        int tid = omp_get_thread_num();
        g_err = 0;
#pragma omp for schedule(static)
        for (int k = 0; k <= i; k++) {
            dyadic p1 = dy_mul(&al[i - k], &ga[k], L);
            dyadic p2 = dy_mul(&al[i - k], &be[k], L);
            dy_accumulate(&sum[2 * tid], &p1);
            dy_accumulate(&sum[2 * tid + 1], &p2);
            dy_free(&p1);
            dy_free(&p2);
        }
        errs |= g_err;
    }
    if (errs) g_err = errs;
    for (int t = 0; t < nthreads; t++) {
        dy_accumulate(s1, &sum[2 * t]);
        dy_accumulate(s2, &sum[2 * t + 1]);
        dy_free(&sum[2 * t]);
        dy_free(&sum[2 * t + 1]);
    }
    free(sum);
#else
    cauchy_sums(i, L, al, be, ga, 1, s1, s2);
#endif
}

/* Eq. (3) for i = 0..N-1: al/be/ga hold N+1 numbers each; index 0 is the
 * state (Sec. 2: alpha_0 = x_n, beta_0 = y_n, gamma_0 = z_n). */
static void taylor_coefficients(int L, int N, const mpnum par[4], mpnum *al,
                                mpnum *be, mpnum *ga, int nthreads)
{
    const mpnum *sigma = &par[0], *R = &par[1], *b = &par[2];
    for (int i = 0; i < N && !g_err; i++) {
        dyadic s1, s2;
        cauchy_sums(i, L, al, be, ga, nthreads, &s1, &s2);

        /* E_x = -sigma alpha_i + sigma beta_i */
        dyadic t1 = dy_neg(dy_mul(sigma, &al[i], L));
        dyadic t2 = dy_mul(sigma, &be[i], L);
        dyadic Ex = dy_add(&t1, &t2);
        dy_free(&t1);
        dy_free(&t2);

        /* E_y = R alpha_i - beta_i - s1 */
        dyadic u1 = dy_mul(R, &al[i], L);
        dyadic u2 = dy_neg(dy_from_mp(&be[i], L));
        dyadic u3 = dy_neg(s1);
        dyadic Ey = dy_add(&u1, &u2);
        dy_accumulate(&Ey, &u3);
        dy_free(&u1);
        dy_free(&u2);
        dy_free(&u3);

        /* E_z = s2 - b gamma_i */
        dyadic v1 = dy_neg(dy_mul(b, &ga[i], L));
        dyadic Ez = dy_add(&s2, &v1);
        dy_free(&v1);
        dy_free(&s2);

        uint32_t d = (uint32_t)(i + 1);
        dy_div_trunc(&Ex, d, L, &al[i + 1]);
        dy_div_trunc(&Ey, d, L, &be[i + 1]);
        dy_div_trunc(&Ez, d, L, &ga[i + 1]);
        dy_free(&Ex);
        dy_free(&Ey);
        dy_free(&Ez);
    }
}

/* Eq. (2) with Horner's rule: h_N = c_N, h_i = trunc_L(h_{i+1} tau + c_i). */
static void horner(int L, int N, const mpnum *tau, const mpnum *c, mpnum *out,
                   uint32_t *scratch)
{
    mpnum h = {c[N].sign, c[N].exp, scratch};
    memcpy(h.limb, c[N].limb, (size_t)L * sizeof(uint32_t));
    for (int i = N - 1; i >= 0 && !g_err; i--) {
        dyadic p = dy_mul(&h, tau, L);
        dyadic a = dy_from_mp(&c[i], L);
        dyadic s = dy_add(&p, &a);
        dy_trunc(&s, L, &h);
        dy_free(&p);
        dy_free(&a);
        dy_free(&s);
    }
    out->sign = h.sign;
    out->exp = h.exp;
    memcpy(out->limb, h.limb, (size_t)L * sizeof(uint32_t));
}

/* ----------------------------------------------------------------------- */
/* flat-array interface (SoA: signs[n], exps[n], limbs[n][L]) */

static int valid_number(int32_t sign, int32_t exp, const uint32_t *limb, int L)
{
    int zero = 1;
    for (int j = 0; j < L; j++)
        if (limb[j]) zero = 0;
    if (zero) return sign == 0 && exp == 0;
    if (sign != 0 && sign != 1) return 0;
    if (limb[L - 1] == 0) return 0;
    return exp <= ORC_EXP_MAX && exp >= -ORC_EXP_MAX;
}

static void wrap(mpnum *m, const int32_t *s, const int32_t *e, uint32_t *l, int n, int L)
{
    for (int j = 0; j < n; j++) {
        m[j].sign = s[j];
        m[j].exp = e[j];
        m[j].limb = l + (size_t)j * L;
    }
}

/* All Taylor coefficients of one step.
 * par: 4 numbers (sigma, R, b, tau); st: 3 numbers (x, y, z);
 * out: 3*(N+1) numbers, component-major: alpha_0..alpha_N, beta_0.., gamma_0.. */
int orc_coefficients(int L, int N, const int32_t *par_s, const int32_t *par_e,
                     const uint32_t *par_l, const int32_t *st_s, const int32_t *st_e,
                     const uint32_t *st_l, int32_t *out_s, int32_t *out_e,
                     uint32_t *out_l, int nthreads)
{
    if (L < 1 || N < 1) return ORC_EINVAL;
    for (int j = 0; j < 4; j++)
        if (!valid_number(par_s[j], par_e[j], par_l + (size_t)j * L, L)) return ORC_EINVAL;
    for (int j = 0; j < 3; j++)
        if (!valid_number(st_s[j], st_e[j], st_l + (size_t)j * L, L)) return ORC_EINVAL;
    g_err = 0;
    mpnum par[4];
    uint32_t *pl = malloc((size_t)4 * L * sizeof(uint32_t));
    if (!pl) return ORC_ENOMEM;
    memcpy(pl, par_l, (size_t)4 * L * sizeof(uint32_t));
    int32_t ps[4], pe[4];
    memcpy(ps, par_s, sizeof ps);
    memcpy(pe, par_e, sizeof pe);
    wrap(par, ps, pe, pl, 4, L);
    mpnum *c = malloc((size_t)3 * (N + 1) * sizeof(mpnum));
    if (!c) { free(pl); return ORC_ENOMEM; }
    wrap(c, out_s, out_e, out_l, 3 * (N + 1), L);
    for (int comp = 0; comp < 3; comp++) {
        mpnum *c0 = &c[comp * (N + 1)];
        c0->sign = st_s[comp];
        c0->exp = st_e[comp];
        memcpy(c0->limb, st_l + (size_t)comp * L, (size_t)L * sizeof(uint32_t));
    }
    taylor_coefficients(L, N, par, c, c + (N + 1), c + 2 * (N + 1), nthreads);
    for (int j = 0; j < 3 * (N + 1); j++) {
        out_s[j] = c[j].sign;
        out_e[j] = c[j].exp;
    }
    free(c);
    free(pl);
    return g_err;
}

/* nsteps Taylor steps from st (overwritten with the final state).  When
 * record_every > 0 the state after every record_every-th step is appended to
 * rec_* (capacity nsteps / record_every numbers of each component, laid out
 * [record][component]). */
int orc_integrate(int L, int N, int64_t nsteps, const int32_t *par_s,
                  const int32_t *par_e, const uint32_t *par_l, int32_t *st_s,
                  int32_t *st_e, uint32_t *st_l, int64_t record_every,
                  int32_t *rec_s, int32_t *rec_e, uint32_t *rec_l, int nthreads)
{
    if (L < 1 || N < 1 || nsteps < 0) return ORC_EINVAL;
    size_t nc = (size_t)3 * (N + 1);
    int32_t *cs = malloc(nc * sizeof(int32_t));
    int32_t *ce = malloc(nc * sizeof(int32_t));
    uint32_t *cl = malloc(nc * (size_t)L * sizeof(uint32_t));
    uint32_t *scratch = malloc((size_t)L * sizeof(uint32_t));
    int rc = ORC_OK;
    if (!cs || !ce || !cl || !scratch) { rc = ORC_ENOMEM; goto out; }
    mpnum par[4];
    int32_t ps[4], pe[4];
    uint32_t *pl = malloc((size_t)4 * L * sizeof(uint32_t));
    if (!pl) { rc = ORC_ENOMEM; goto out; }
    memcpy(ps, par_s, sizeof ps);
    memcpy(pe, par_e, sizeof pe);
    memcpy(pl, par_l, (size_t)4 * L * sizeof(uint32_t));
    wrap(par, ps, pe, pl, 4, L);
    int64_t nrec = 0;
    for (int64_t step = 0; step < nsteps && rc == ORC_OK; step++) {
        rc = orc_coefficients(L, N, par_s, par_e, par_l, st_s, st_e, st_l, cs, ce, cl,
                              nthreads);
        if (rc) break;
        mpnum *coef = malloc(nc * sizeof(mpnum));
        if (!coef) { rc = ORC_ENOMEM; break; }
        wrap(coef, cs, ce, cl, (int)nc, L);
        g_err = 0;
        for (int comp = 0; comp < 3; comp++) {
            mpnum out = {0, 0, st_l + (size_t)comp * L};
            horner(L, N, &par[3], &coef[comp * (N + 1)], &out, scratch);
            st_s[comp] = out.sign;
            st_e[comp] = out.exp;
        }
        free(coef);
        rc = g_err;
        if (rc == ORC_OK && record_every > 0 && (step + 1) % record_every == 0) {
            for (int comp = 0; comp < 3; comp++) {
                rec_s[nrec * 3 + comp] = st_s[comp];
                rec_e[nrec * 3 + comp] = st_e[comp];
                memcpy(rec_l + ((size_t)nrec * 3 + comp) * L, st_l + (size_t)comp * L,
                       (size_t)L * sizeof(uint32_t));
            }
            nrec++;
        }
    }
    free(pl);
out:
    free(cs);
    free(ce);
    free(cl);
    free(scratch);
    return rc;
}

/* Single operations, exposed so the tests can pin them one by one. */

/* out = trunc_L(a*b + c) with a, b, c L-limb numbers (one Horner step) */
int orc_fma_trunc(int L, const int32_t *s, const int32_t *e, const uint32_t *l,
                  int32_t *out_s, int32_t *out_e, uint32_t *out_l)
{
    mpnum v[3];
    int32_t ss[3], ee[3];
    memcpy(ss, s, sizeof ss);
    memcpy(ee, e, sizeof ee);
    for (int j = 0; j < 3; j++)
        if (!valid_number(s[j], e[j], l + (size_t)j * L, L)) return ORC_EINVAL;
    g_err = 0;
    wrap(v, ss, ee, (uint32_t *)l, 3, L);
    dyadic p = dy_mul(&v[0], &v[1], L);
    dyadic c = dy_from_mp(&v[2], L);
    dyadic sum = dy_add(&p, &c);
    mpnum out = {0, 0, out_l};
    dy_trunc(&sum, L, &out);
    *out_s = out.sign;
    *out_e = out.exp;
    dy_free(&p);
    dy_free(&c);
    dy_free(&sum);
    return g_err;
}

/* ----------------------------------------------------------------------- */
/* The adjoint of the step (see the header). */

/* P_0 = 1, P_j = trunc_L(P_{j-1} tau), j = 1..N: d(x_{n+1})/d(alpha_j) = tau^j
 * by Eq. (2). */
static void tau_powers(int L, int N, const mpnum *tau, mpnum *P)
{
    mp_set_zero(&P[0], L);
    P[0].limb[L - 1] = 1u; /* 1 = 1 * 2^(32 (exp - 1)) with exp = 1 */
    P[0].exp = 1;
    for (int j = 1; j <= N && !g_err; j++) {
        dyadic p = dy_mul(&P[j - 1], tau, L);
        dy_trunc(&p, L, &P[j]);
        dy_free(&p);
    }
}

/* s += sg * a * b */
static void acc_prod(dyadic *s, int sg, const mpnum *a, const mpnum *b, int L)
{
    dyadic p = dy_mul(a, b, L);
    if (sg < 0) p = dy_neg(p);
    dy_accumulate(s, &p);
    dy_free(&p);
}

/* s += sg * a */
static void acc_lone(dyadic *s, int sg, const mpnum *a, int L)
{
    dyadic p = dy_from_mp(a, L);
    if (sg < 0) p = dy_neg(p);
    dy_accumulate(s, &p);
    dy_free(&p);
}

/* One step backwards.  al/be/ga: the step's coefficients (N+1 each); P: the
 * powers of tau; gb[3]: the adjoint of the step's result, replaced by the
 * adjoint of the step's starting state; th[3]: the running adjoints of
 * sigma, R, b; Ea/Eb/Eg: N numbers each of scratch (Ebar_x, Ebar_y, Ebar_z). */
static void adjoint_step(int L, int N, const mpnum par[4], const mpnum *al, const mpnum *be,
                         const mpnum *ga, const mpnum *P, mpnum *gb, mpnum *th, mpnum *Ea,
                         mpnum *Eb, mpnum *Eg)
{
    const mpnum *sigma = &par[0], *R = &par[1], *b = &par[2];
    for (int j = N; j >= 0 && !g_err; j--) {
        dyadic Sx = dy_zero(), Sy = dy_zero(), Sz = dy_zero();
        /* Eq. (2): x_{n+1} = sum_j alpha_j tau^j */
        acc_prod(&Sx, 1, &gb[0], &P[j], L);
        acc_prod(&Sy, 1, &gb[1], &P[j], L);
        acc_prod(&Sz, 1, &gb[2], &P[j], L);
        if (j <= N - 1) {
            /* the linear terms of the brackets E_j of Eq. (3) */
            acc_prod(&Sx, -1, sigma, &Ea[j], L);
            acc_prod(&Sx, 1, R, &Eb[j], L);
            acc_prod(&Sy, 1, sigma, &Ea[j], L);
            acc_lone(&Sy, -1, &Eb[j], L);
            acc_prod(&Sz, -1, b, &Eg[j], L);
        }
        /* the Cauchy sums of the brackets E_i, i >= j, through their factor of index j */
        for (int i = j; i <= N - 1; i++) {
            acc_prod(&Sx, -1, &Eb[i], &ga[i - j], L);
            acc_prod(&Sx, 1, &Eg[i], &be[i - j], L);
            acc_prod(&Sy, 1, &Eg[i], &al[i - j], L);
            acc_prod(&Sz, -1, &Eb[i], &al[i - j], L);
        }
        if (j >= 1) {
            /* alpha_j = E_{j-1} / j */
            dy_div_trunc(&Sx, (uint32_t)j, L, &Ea[j - 1]);
            dy_div_trunc(&Sy, (uint32_t)j, L, &Eb[j - 1]);
            dy_div_trunc(&Sz, (uint32_t)j, L, &Eg[j - 1]);
        } else {
            /* alpha_0 = x_n: the state's adjoint */
            dy_trunc(&Sx, L, &gb[0]);
            dy_trunc(&Sy, L, &gb[1]);
            dy_trunc(&Sz, L, &gb[2]);
        }
        dy_free(&Sx);
        dy_free(&Sy);
        dy_free(&Sz);
    }
    /* dE_x,i/dsigma = beta_i - alpha_i, dE_y,i/dR = alpha_i, dE_z,i/db = -gamma_i */
    dyadic ts = dy_from_mp(&th[0], L), tr = dy_from_mp(&th[1], L), tb = dy_from_mp(&th[2], L);
    for (int i = 0; i <= N - 1; i++) {
        acc_prod(&ts, 1, &Ea[i], &be[i], L);
        acc_prod(&ts, -1, &Ea[i], &al[i], L);
        acc_prod(&tr, 1, &Eb[i], &al[i], L);
        acc_prod(&tb, -1, &Eg[i], &ga[i], L);
    }
    dy_trunc(&ts, L, &th[0]);
    dy_trunc(&tr, L, &th[1]);
    dy_trunc(&tb, L, &th[2]);
    dy_free(&ts);
    dy_free(&tr);
    dy_free(&tb);
}

static mpnum *mp_array(int n, int L, uint32_t **store)
{
    mpnum *m = malloc((size_t)(n ? n : 1) * sizeof(mpnum));
    *store = calloc((size_t)(n ? n : 1) * L, sizeof(uint32_t));
    if (!m || !*store) {
        free(m);
        free(*store);
        *store = NULL;
        g_err = ORC_ENOMEM;
        return NULL;
    }
    for (int j = 0; j < n; j++) {
        m[j].sign = 0;
        m[j].exp = 0;
        m[j].limb = *store + (size_t)j * L;
    }
    return m;
}

/* One reverse step from a step's coefficients (3*(N+1) numbers,
 * component-major, as orc_coefficients gives them): gb[3] in/out, th[3]
 * in/out (see adjoint_step). */
int orc_adjoint_step(int L, int N, const int32_t *par_s, const int32_t *par_e, const uint32_t *par_l,
                     const int32_t *c_s, const int32_t *c_e, const uint32_t *c_l, int32_t *gb_s,
                     int32_t *gb_e, uint32_t *gb_l, int32_t *th_s, int32_t *th_e, uint32_t *th_l)
{
    if (L < 1 || N < 1) return ORC_EINVAL;
    g_err = 0;
    int32_t ps[4], pe[4];
    memcpy(ps, par_s, sizeof ps);
    memcpy(pe, par_e, sizeof pe);
    mpnum par[4], gb[3], th[3];
    wrap(par, ps, pe, (uint32_t *)par_l, 4, L);
    wrap(gb, gb_s, gb_e, gb_l, 3, L);
    wrap(th, th_s, th_e, th_l, 3, L);
    int32_t *cs = malloc((size_t)3 * (N + 1) * sizeof(int32_t));
    int32_t *ce = malloc((size_t)3 * (N + 1) * sizeof(int32_t));
    mpnum *c = malloc((size_t)3 * (N + 1) * sizeof(mpnum));
    uint32_t *Pst = NULL, *Est = NULL;
    mpnum *P = mp_array(N + 1, L, &Pst), *E = mp_array(3 * N, L, &Est);
    if (!cs || !ce || !c || !P || !E) g_err = ORC_ENOMEM;
    if (!g_err) {
        memcpy(cs, c_s, (size_t)3 * (N + 1) * sizeof(int32_t));
        memcpy(ce, c_e, (size_t)3 * (N + 1) * sizeof(int32_t));
        wrap(c, cs, ce, (uint32_t *)c_l, 3 * (N + 1), L);
        tau_powers(L, N, &par[3], P);
        adjoint_step(L, N, par, c, c + (N + 1), c + 2 * (N + 1), P, gb, th, E, E + N, E + 2 * N);
        for (int k = 0; k < 3; k++) {
            gb_s[k] = gb[k].sign;
            gb_e[k] = gb[k].exp;
            th_s[k] = th[k].sign;
            th_e[k] = th[k].exp;
        }
    }
    free(cs);
    free(ce);
    free(c);
    free(P);
    free(Pst);
    free(E);
    free(Est);
    return g_err;
}

/* nsteps steps from st, then the reverse sweep: gb[3] (in: the adjoint of
 * the final state; out: of the initial state) and th[3] (out: the adjoints
 * of sigma, R, b, starting from zero).  The coefficients of every step are
 * kept (the library recomputes them from checkpoints instead: the same
 * numbers).  nthreads as orc_integrate (forward sums only). */
int orc_backward(int L, int N, int64_t nsteps, const int32_t *par_s, const int32_t *par_e,
                 const uint32_t *par_l, const int32_t *st_s, const int32_t *st_e,
                 const uint32_t *st_l, int32_t *gb_s, int32_t *gb_e, uint32_t *gb_l, int32_t *th_s,
                 int32_t *th_e, uint32_t *th_l, int nthreads)
{
    if (L < 1 || N < 1 || nsteps < 0) return ORC_EINVAL;
    const size_t nc = (size_t)3 * (N + 1);
    int32_t *hs = malloc((size_t)(nsteps ? nsteps : 1) * nc * sizeof(int32_t));
    int32_t *he = malloc((size_t)(nsteps ? nsteps : 1) * nc * sizeof(int32_t));
    uint32_t *hl = malloc((size_t)(nsteps ? nsteps : 1) * nc * L * sizeof(uint32_t));
    int32_t ss[3], se[3];
    uint32_t *sl = malloc((size_t)3 * L * sizeof(uint32_t));
    uint32_t *scratch = malloc((size_t)L * sizeof(uint32_t));
    int rc = ORC_OK;
    if (!hs || !he || !hl || !sl || !scratch) rc = ORC_ENOMEM;
    if (rc == ORC_OK) {
        memcpy(ss, st_s, sizeof ss);
        memcpy(se, st_e, sizeof se);
        memcpy(sl, st_l, (size_t)3 * L * sizeof(uint32_t));
    }
    int32_t ps[4], pe[4];
    memcpy(ps, par_s, sizeof ps);
    memcpy(pe, par_e, sizeof pe);
    mpnum par[4];
    wrap(par, ps, pe, (uint32_t *)par_l, 4, L);
    for (int64_t n = 0; n < nsteps && rc == ORC_OK; n++) {
        int32_t *cs = hs + n * nc, *ce = he + n * nc;
        uint32_t *cl = hl + (size_t)n * nc * L;
        rc = orc_coefficients(L, N, par_s, par_e, par_l, ss, se, sl, cs, ce, cl, nthreads);
        if (rc) break;
        mpnum *coef = malloc(nc * sizeof(mpnum));
        if (!coef) { rc = ORC_ENOMEM; break; }
        wrap(coef, cs, ce, cl, (int)nc, L);
        g_err = 0;
        for (int comp = 0; comp < 3; comp++) {
            mpnum out = {0, 0, sl + (size_t)comp * L};
            horner(L, N, &par[3], &coef[comp * (N + 1)], &out, scratch);
            ss[comp] = out.sign;
            se[comp] = out.exp;
        }
        free(coef);
        rc = g_err;
    }
    if (rc == ORC_OK) {
        for (int k = 0; k < 3; k++) {
            th_s[k] = 0;
            th_e[k] = 0;
        }
        memset(th_l, 0, (size_t)3 * L * sizeof(uint32_t));
        for (int64_t n = nsteps - 1; n >= 0 && rc == ORC_OK; n--)
            rc = orc_adjoint_step(L, N, par_s, par_e, par_l, hs + n * nc, he + n * nc,
                                  hl + (size_t)n * nc * L, gb_s, gb_e, gb_l, th_s, th_e, th_l);
    }
    free(hs);
    free(he);
    free(hl);
    free(sl);
    free(scratch);
    return rc;
}

int orc_omp_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
