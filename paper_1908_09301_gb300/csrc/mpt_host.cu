// mpt_host.cu -- the C ABI of libmpt (declared in include/mpt.h): contexts,
// device buffers, parameter and state conversion, launches and error codes.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mpt.h"
#include "host_parse.h"
#include "mpt_kernel.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(MPT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// restores the caller's current device on scope exit
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

namespace mpt {
// sets the calling thread's mpt_last_error() message from another translation unit
int record_error(int code, const char *msg)
{
    g_last_error = msg;
    return code;
}
}  // namespace mpt

struct mpt_ctx {
    int L = 0, Lp = 0, P = 0, N = 0, Wcap = 0, tb = 0, nwin = 1;
    int dev = 0, sms = 0;
    cudaStream_t st = nullptr;
    int ctas_req = 0;
    size_t smem = 0;
    int max_grid = 0;
    // device buffers
    uint32_t *coefL = nullptr;
    int32_t *coefE = nullptr, *coefF = nullptr;
    uint32_t *parL = nullptr;
    int32_t *parE = nullptr, *parF = nullptr;
    uint32_t *stL = nullptr, *stBackL = nullptr;
    int32_t *stE = nullptr, *stF = nullptr, *stBackEF = nullptr;
    long long *gwin = nullptr;
    unsigned *bar = nullptr;
    int *status = nullptr;
    int32_t *recS = nullptr, *recE = nullptr;
    uint32_t *recL = nullptr;
    long long rec_cap = 0;
    bool have_coefficients = false;
    bool pending = false;  // steps queued by mpt_launch, not yet waited for
    long long *prof = nullptr;  // per-phase cycle counters when profiling is on
    long long spin_limit = mpt::DEFAULT_SPIN_LIMIT;
    // pipelined kernel (bracket and outer-pair CTAs + workers)
    int kind_req = 0;           // 0 auto, 1 lockstep, 2 pipelined
    int pipe_C = 10;            // CTAs with fixed roles in the pipelined kernel (fixed by the kernel)
    int pipe_max_grid = 0;      // co-resident CTAs of the pipelined kernel
    int pipe_tb = 0;
    int pipe_tb_fit = 0;        // the largest worker batch that fits (mpt_set_pipe_batch 0)
    size_t pipe_smem = 0;
    unsigned *pub = nullptr, *done = nullptr;
    long long *gin = nullptr;
    long long *imid = nullptr;
    // parameters in the interchange layout (host)
    int32_t par_s[4] = {0, 0, 0, 0}, par_e[4] = {0, 0, 0, 0};
    std::vector<uint32_t> par_l;
    // a general quadratic system (mpt_set_system): its term table on the
    // device, its parameters (tau last) in parL
    int *sysT = nullptr;
    int sysNF = 0, sysNQ = 0, sys_npar = 0;
    // the last launch (for an exact rerun of a launch whose shortened sums
    // could not be shown exact) and the counters of mpt_get_counters
    long long last_nsteps = 0, last_nrec = 0, last_every = 0;
    bool last_exact = false;
    bool force_exact = false;      // mpt_set_exact: every launch in full
    long long exact_reruns = 0;
    // tau as a small ratio p/q (tau_q = 0: not), for Horner steps without a limb product
    uint32_t tau_p = 0, tau_q = 0, tau_r = 0;
    int tau_shift = 0, tau_neg = 0;
    unsigned long long *chunks = nullptr;  // executed limb-product chunks of the last launch
    uint32_t *divtab = nullptr;            // pipelined kernel: powers of 2^32 modulo the divisors
    int divtab_rl = 0;
};

namespace {

// profile counters: the first and the last CTA, then one row per SM, then the
// pipelined kernel's per-index timeline
size_t prof_rows_len(const mpt_ctx *c) { return (size_t)(2 + c->sms) * mpt::PROF_SLOTS; }
size_t prof_len(const mpt_ctx *c)
{
    return prof_rows_len(c) + (size_t)mpt::TL_ROWS * (mpt::MAX_N + 1);
}

// which kernel runs a launch: the pipelined one for large L x N, when the
// device fits its fixed-role CTAs and at least one worker
int kind_for(const mpt_ctx *c)
{
    if (c->kind_req == 1 || c->sysT) return 1;  // the pipelined kernel is Lorenz's own
    bool pipe_ok = c->pipe_max_grid >= c->pipe_C + 1 && c->N >= 3;
    if (c->kind_req == 2) return pipe_ok ? 2 : 1;
    double work = (double)c->N * c->Lp * c->Lp;
    return (pipe_ok && work >= 5e5) ? 2 : 1;
}

int pipe_grid_for(const mpt_ctx *c)
{
    int g = c->pipe_max_grid;
    if (g > c->sms) g = c->sms;
    if (c->ctas_req > 0) {
        int r = c->ctas_req;
        if (r < c->pipe_C + 1) r = c->pipe_C + 1;
        if (r < g) g = r;
    }
    return g;
}

int grid_for(const mpt_ctx *c)
{
    int g = c->ctas_req;
    if (g <= 0) {
        // enough CTAs that the per-index work outweighs a grid barrier
        double work = (double)c->N * c->Lp * c->Lp;
        g = (int)std::lround(work / 50000.0);
    }
    if (g < 1) g = 1;
    if (g > c->sms) g = c->sms;
    if (g > c->max_grid) g = c->max_grid;
    return g;
}


// interchange (sign, exp, L limbs) -> device layout (flags, exp, Lp limbs)
int to_device_layout(const mpt_ctx *c, const int32_t *s, const int32_t *e, const uint32_t *l, int n,
                     std::vector<uint32_t> &dl, std::vector<int32_t> &de, std::vector<int32_t> &df)
{
    dl.assign((size_t)n * c->Lp, 0u);
    de.assign(n, 0);
    df.assign(n, 0);
    for (int j = 0; j < n; j++) {
        const uint32_t *lj = l + (size_t)j * c->L;
        bool zero = true;
        for (int x = 0; x < c->L; x++) zero = zero && lj[x] == 0;
        if (zero) {
            if (s[j] != 0 || e[j] != 0)
                return fail(MPT_EINVAL, "number %d: zero must have sign 0 and exp 0", j);
            continue;
        }
        if (s[j] != 0 && s[j] != 1) return fail(MPT_EINVAL, "number %d: sign must be 0 or 1", j);
        if (lj[c->L - 1] == 0) return fail(MPT_EINVAL, "number %d: top limb is zero", j);
        if (e[j] > (1 << 30) || e[j] < -(1 << 30))
            return fail(MPT_ERANGE, "number %d: exponent %d out of range", j, e[j]);
        std::memcpy(&dl[(size_t)j * c->Lp], lj, sizeof(uint32_t) * c->L);
        de[j] = e[j];
        df[j] = mpt::F_NZ | (s[j] ? mpt::F_NEG : 0);
    }
    return MPT_OK;
}

void from_device_layout(const mpt_ctx *c, const std::vector<uint32_t> &dl,
                        const std::vector<int32_t> &de, const std::vector<int32_t> &df, int n,
                        int32_t *s, int32_t *e, uint32_t *l)
{
    for (int j = 0; j < n; j++) {
        s[j] = (df[j] & mpt::F_NEG) ? 1 : 0;
        e[j] = de[j];
        std::memcpy(l + (size_t)j * c->L, &dl[(size_t)j * c->Lp], sizeof(uint32_t) * c->L);
    }
}

int wait_steps(mpt_ctx *c);

int upload_state(mpt_ctx *c, const int32_t *s, const int32_t *e, const uint32_t *l)
{
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    std::vector<uint32_t> dl;
    std::vector<int32_t> de, df;
    int rc = to_device_layout(c, s, e, l, 3, dl, de, df);
    if (rc) return rc;
    DeviceGuard g(c->dev);
    cudaError_t ce = cudaMemcpyAsync(c->stL, dl.data(), sizeof(uint32_t) * 3 * c->Lp,
                                     cudaMemcpyHostToDevice, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->stE, de.data(), sizeof(int32_t) * 3, cudaMemcpyHostToDevice, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->stF, df.data(), sizeof(int32_t) * 3, cudaMemcpyHostToDevice, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "state upload");
    return MPT_OK;
}

void free_all(mpt_ctx *c)
{
    if (c->sysT) cudaFree(c->sysT);
    c->sysT = nullptr;
    void *ptrs[] = {c->coefL, c->coefE, c->coefF, c->parL, c->parE, c->parF, c->stL, c->stBackL,
                    c->stE, c->stF, c->stBackEF, c->gwin, c->bar, c->status, c->recS, c->recE,
                    c->recL, c->prof, c->pub, c->done, c->gin, c->imid, c->chunks, c->divtab};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    const cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
    // a refused allocation is not sticky, but it stays the runtime's "last
    // error", which the launch paths read after a kernel launch: clear it
    if (e != cudaSuccess) {
        *p = nullptr;
        (void)cudaGetLastError();
    }
    return e;
}

}  // namespace

extern "C" {

int mpt_limbs_for_digits(int K)
{
    if (K < 1) return fail(MPT_EINVAL, "K_digits must be >= 1");
    return (int)std::ceil((double)K * 3.321928094887362 / 32.0);
}

const char *mpt_strerror(int code)
{
    switch (code) {
        case MPT_OK: return "ok";
        case MPT_EINVAL: return "invalid argument";
        case MPT_ENOMEM: return "out of memory";
        case MPT_ERANGE: return "exponent or accumulator range exceeded";
        case MPT_ETIMEDOUT: return "a bounded device wait expired";
        case MPT_ECUDA: return "CUDA error";
        default: return "unknown error";
    }
}

const char *mpt_last_error(void) { return g_last_error.c_str(); }

int mpt_parse_number(const char *str, int L, int32_t *sign, int32_t *exp, uint32_t *limbs)
{
    if (!str || !sign || !exp || !limbs) return fail(MPT_EINVAL, "null argument");
    if (L < 1 || L > mpt::MAX_L) return fail(MPT_EINVAL, "L = %d outside 1..%d", L, mpt::MAX_L);
    int rc = mpt_host::parse_number(str, L, sign, exp, limbs);
    if (rc == -3) return fail(MPT_ERANGE, "exponent of \"%s\" out of range", str);
    if (rc) return fail(MPT_EINVAL, "malformed number \"%s\"", str);
    return MPT_OK;
}



int mpt_init(mpt_ctx **out, int K_digits, int N_order, int L_limbs, const char *tau,
             const char *sigma, const char *R, const char *b, uint64_t cuda_stream)
{
    if (!out) return fail(MPT_EINVAL, "ctx pointer is null");
    *out = nullptr;
    int L = L_limbs;
    if (L == 0) {
        L = mpt_limbs_for_digits(K_digits);
        if (L < 0) return L;
    }
    if (L < 1 || L > mpt::MAX_L) return fail(MPT_EINVAL, "L = %d outside 1..%d", L, mpt::MAX_L);
    if (N_order < 1 || N_order > mpt::MAX_N)
        return fail(MPT_EINVAL, "N = %d outside 1..%d", N_order, mpt::MAX_N);
    mpt_ctx *c = new (std::nothrow) mpt_ctx();
    if (!c) return fail(MPT_ENOMEM, "host allocation");
    c->L = L;
    c->Lp = (L + mpt::W - 1) / mpt::W * mpt::W;
    c->P = c->Lp / mpt::W;
    c->N = N_order;
    int spread = c->Lp > 64 ? c->Lp : 64;
    c->Wcap = (2 * c->Lp + 2 + spread + 31) / 32 * 32;
    c->st = (cudaStream_t)(uintptr_t)cuda_stream;
    // parameters: sigma, R, b, tau
    const char *strs[4] = {sigma, R, b, tau};
    const char *names[4] = {"sigma", "R", "b", "tau"};
    c->par_l.assign((size_t)4 * L, 0u);
    for (int j = 0; j < 4; j++) {
        if (!strs[j]) {
            delete c;
            return fail(MPT_EINVAL, "%s is null", names[j]);
        }
        int rc = mpt_host::parse_number(strs[j], L, &c->par_s[j], &c->par_e[j],
                                        &c->par_l[(size_t)j * L]);
        if (rc) {
            delete c;
            return fail(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use %s = \"%s\"", names[j],
                        strs[j]);
        }
    }
    if (mpt_host::small_ratio(tau, L, &c->tau_p, &c->tau_q, &c->tau_r, &c->tau_shift, &c->tau_neg))
        c->tau_q = 0;
    cudaError_t ce = cudaGetDevice(&c->dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
    int smem_optin = 0;
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    if (ce != cudaSuccess) {
        delete c;
        return cuda_fail(ce, "device query");
    }
    // staging batch: as many terms as fit next to the fixed shared-memory parts
    int tb = 64;
    while (tb > 8 && mpt::smem_bytes(L, c->Lp, c->N, c->Wcap, tb) > (size_t)smem_optin) tb /= 2;
    c->tb = tb;
    // window copies for the lock-step term phase, as many (up to 8) as fit
    int nwin = 8;
    while (nwin > 1 && mpt::smem_bytes(L, c->Lp, c->N, c->Wcap, tb, nwin) > (size_t)smem_optin) nwin /= 2;
    c->nwin = nwin;
    c->smem = mpt::smem_bytes(L, c->Lp, c->N, c->Wcap, tb, nwin);
    if (c->smem > (size_t)smem_optin) {
        delete c;
        return fail(MPT_EINVAL, "L = %d, N = %d need %zu bytes of shared memory (device has %d)", L,
                    N_order, c->smem, smem_optin);
    }
    c->max_grid = mpt::max_coresident_ctas(c->smem);
    if (c->max_grid < 1) {
        delete c;
        return fail(MPT_ECUDA, "kernel does not fit on the device");
    }
    {
        // worker term slots: as many as fit (at most pipe_tb_max())
        int ptb = mpt::pipe_tb_max();
        while (ptb > 1 && mpt::pipe_smem_bytes(L, c->Lp, c->N, c->Wcap, ptb) > (size_t)smem_optin)
            ptb--;
        c->pipe_tb = ptb;
        c->pipe_tb_fit = ptb;
        c->pipe_smem = mpt::pipe_smem_bytes(L, c->Lp, c->N, c->Wcap, ptb);
        c->pipe_C = mpt::pipe_fixed_ctas();
        c->pipe_max_grid = 0;
        if (c->pipe_smem <= (size_t)smem_optin) {
            c->pipe_max_grid = mpt::pipe_max_ctas(c->pipe_smem);
            (void)cudaGetLastError();
        }
    }
    const size_t N1 = (size_t)c->N + 1;
    ce = dalloc(&c->coefL, 3 * N1 * c->Lp);
    if (ce == cudaSuccess) ce = dalloc(&c->coefE, 3 * N1);
    if (ce == cudaSuccess) ce = dalloc(&c->coefF, 3 * N1);
    if (ce == cudaSuccess) ce = dalloc(&c->parL, (size_t)mpt::SYS_MAX_PAR * c->Lp);
    if (ce == cudaSuccess) ce = dalloc(&c->parE, mpt::SYS_MAX_PAR);
    if (ce == cudaSuccess) ce = dalloc(&c->parF, mpt::SYS_MAX_PAR);
    if (ce == cudaSuccess) ce = dalloc(&c->stL, (size_t)3 * c->Lp);
    if (ce == cudaSuccess) ce = dalloc(&c->stBackL, (size_t)3 * c->Lp);
    if (ce == cudaSuccess) ce = dalloc(&c->stE, 3);
    if (ce == cudaSuccess) ce = dalloc(&c->stF, 3);
    if (ce == cudaSuccess) ce = dalloc(&c->stBackEF, 6);
    if (ce == cudaSuccess) ce = dalloc(&c->gwin, (size_t)9 * c->Wcap);
    if (ce == cudaSuccess) ce = dalloc(&c->bar, 2);
    if (ce == cudaSuccess) ce = dalloc(&c->status, 1);
    if (ce == cudaSuccess) ce = dalloc(&c->pub, 1);
    if (ce == cudaSuccess) ce = dalloc(&c->done, mpt::PIPE_SETS);
    if (ce == cudaSuccess) ce = dalloc(&c->gin, (size_t)mpt::PIPE_SETS * 9 * c->Wcap);
    if (ce == cudaSuccess) ce = dalloc(&c->imid, (size_t)mpt::PIPE_SETS * 4);
    if (ce == cudaSuccess) ce = dalloc(&c->chunks, 1);
    if (ce == cudaSuccess && L + 1 < mpt::PT) {
        c->divtab_rl = L + 2;
        ce = dalloc(&c->divtab, (size_t)(N_order + 1) * c->divtab_rl);
        if (ce == cudaSuccess) {
            const std::vector<uint32_t> t = mpt_host::division_table(N_order, c->divtab_rl, c->tau_q);
            ce = cudaMemcpy(c->divtab, t.data(), sizeof(uint32_t) * t.size(), cudaMemcpyHostToDevice);
        }
    }
    if (ce != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(ce == cudaErrorMemoryAllocation ? MPT_ENOMEM : MPT_ECUDA, "device allocation: %s",
                    cudaGetErrorString(ce));
    }
    std::vector<uint32_t> dl;
    std::vector<int32_t> de, df;
    int rc = to_device_layout(c, c->par_s, c->par_e, c->par_l.data(), 4, dl, de, df);
    if (rc) {
        free_all(c);
        delete c;
        return rc;
    }
    ce = cudaMemcpy(c->parL, dl.data(), sizeof(uint32_t) * 4 * c->Lp, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->parE, de.data(), sizeof(int32_t) * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->parF, df.data(), sizeof(int32_t) * 4, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(c->gwin, 0, sizeof(long long) * 9 * c->Wcap);
    if (ce == cudaSuccess) ce = cudaMemset(c->status, 0, sizeof(int));
    if (ce == cudaSuccess) ce = cudaMemset(c->bar, 0, sizeof(unsigned) * 2);
    if (ce == cudaSuccess) ce = cudaMemset(c->stL, 0, sizeof(uint32_t) * 3 * c->Lp);
    if (ce == cudaSuccess) ce = cudaMemset(c->stE, 0, sizeof(int32_t) * 3);
    if (ce == cudaSuccess) ce = cudaMemset(c->stF, 0, sizeof(int32_t) * 3);
    if (ce == cudaSuccess) ce = cudaMemset(c->coefL, 0, sizeof(uint32_t) * 3 * N1 * c->Lp);
    if (ce == cudaSuccess) ce = cudaMemset(c->coefE, 0, sizeof(int32_t) * 3 * N1);
    if (ce == cudaSuccess) ce = cudaMemset(c->coefF, 0, sizeof(int32_t) * 3 * N1);
    if (ce == cudaSuccess) ce = cudaMemset(c->chunks, 0, sizeof(unsigned long long));
    if (ce != cudaSuccess) {
        free_all(c);
        delete c;
        return cuda_fail(ce, "device initialisation");
    }
    *out = c;
    return MPT_OK;
}

void mpt_destroy(mpt_ctx *c)
{
    if (!c) return;
    {
        DeviceGuard g(c->dev);
        cudaStreamSynchronize(c->st);
        free_all(c);
    }
    delete c;
}

int mpt_get_dims(const mpt_ctx *c, int *L, int *N)
{
    if (!c || !L || !N) return fail(MPT_EINVAL, "null argument");
    *L = c->L;
    *N = c->N;
    return MPT_OK;
}

int mpt_set_state(mpt_ctx *c, const char *x0, const char *y0, const char *z0)
{
    if (!c || !x0 || !y0 || !z0) return fail(MPT_EINVAL, "null argument");
    int32_t s[3], e[3];
    std::vector<uint32_t> l((size_t)3 * c->L);
    const char *strs[3] = {x0, y0, z0};
    for (int j = 0; j < 3; j++) {
        int rc = mpt_host::parse_number(strs[j], c->L, &s[j], &e[j], &l[(size_t)j * c->L]);
        if (rc)
            return fail(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use state \"%s\"", strs[j]);
    }
    return upload_state(c, s, e, l.data());
}

int mpt_set_state_raw(mpt_ctx *c, const int32_t *s, const int32_t *e, const uint32_t *l)
{
    if (!c || !s || !e || !l) return fail(MPT_EINVAL, "null argument");
    return upload_state(c, s, e, l);
}

int mpt_get_state(mpt_ctx *c, int32_t *s, int32_t *e, uint32_t *l)
{
    if (!c || !s || !e || !l) return fail(MPT_EINVAL, "null argument");
    DeviceGuard g(c->dev);
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    std::vector<uint32_t> dl((size_t)3 * c->Lp);
    std::vector<int32_t> de(3), df(3);
    cudaError_t ce = cudaMemcpyAsync(dl.data(), c->stL, sizeof(uint32_t) * 3 * c->Lp,
                                     cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(de.data(), c->stE, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(df.data(), c->stF, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "state download");
    from_device_layout(c, dl, de, df, 3, s, e, l);
    return MPT_OK;
}

int mpt_get_params(mpt_ctx *c, int32_t *s, int32_t *e, uint32_t *l)
{
    if (!c || !s || !e || !l) return fail(MPT_EINVAL, "null argument");
    if (c->sysT) return fail(MPT_EINVAL, "the context runs a general system (no sigma, R, b)");
    for (int j = 0; j < 4; j++) {
        s[j] = c->par_s[j];
        e[j] = c->par_e[j];
    }
    std::memcpy(l, c->par_l.data(), sizeof(uint32_t) * 4 * c->L);
    return MPT_OK;
}

int mpt_set_launch(mpt_ctx *c, int ctas)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (ctas < 0 || ctas > c->sms)
        return fail(MPT_EINVAL, "ctas = %d outside 0..%d", ctas, c->sms);
    c->ctas_req = ctas;
    return MPT_OK;
}

int mpt_set_pipe_batch(mpt_ctx *c, int tb)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (tb < 0 || tb > c->pipe_tb_fit)
        return fail(MPT_EINVAL, "worker batch %d outside 0..%d", tb, c->pipe_tb_fit);
    const int t = tb ? tb : c->pipe_tb_fit;
    const size_t sm = mpt::pipe_smem_bytes(c->L, c->Lp, c->N, c->Wcap, t);
    DeviceGuard g(c->dev);
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    const int grid = mpt::pipe_max_ctas(sm);
    (void)cudaGetLastError();
    if (grid < c->pipe_C + 1) return fail(MPT_EINVAL, "worker batch %d leaves too few co-resident CTAs", tb);
    c->pipe_tb = t;
    c->pipe_smem = sm;
    c->pipe_max_grid = grid;
    return MPT_OK;
}

int mpt_get_launch(const mpt_ctx *c, int *ctas)
{
    if (!c || !ctas) return fail(MPT_EINVAL, "null argument");
    *ctas = kind_for(c) == 2 ? pipe_grid_for(c) : grid_for(c);
    return MPT_OK;
}

int mpt_set_kernel(mpt_ctx *c, int kind)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (kind < 0 || kind > 2) return fail(MPT_EINVAL, "kernel kind %d outside 0..2", kind);
    if (kind == 2 && c->sysT) return fail(MPT_EINVAL, "the pipelined kernel runs Lorenz only");
    c->kind_req = kind;
    return MPT_OK;
}

int mpt_get_kernel(const mpt_ctx *c, int *kind)
{
    if (!c || !kind) return fail(MPT_EINVAL, "null argument");
    *kind = kind_for(c);
    return MPT_OK;
}

int mpt_set_system(mpt_ctx *c, int npar, const char *const *params, int nfixed, const int32_t *fixed,
                   int nquad, const int32_t *quad)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (npar < 0 || npar > mpt::SYS_MAX_PAR - 1)
        return fail(MPT_EINVAL, "npar = %d outside 0..%d", npar, mpt::SYS_MAX_PAR - 1);
    if (nfixed < 0 || nfixed > mpt::SYS_MAX_FIXED)
        return fail(MPT_EINVAL, "nfixed = %d outside 0..%d", nfixed, mpt::SYS_MAX_FIXED);
    if (nquad < 0 || nquad > mpt::SYS_MAX_QUAD)
        return fail(MPT_EINVAL, "nquad = %d outside 0..%d", nquad, mpt::SYS_MAX_QUAD);
    if ((npar > 0 && !params) || (nfixed > 0 && !fixed) || (nquad > 0 && !quad))
        return fail(MPT_EINVAL, "null argument");
    for (int t = 0; t < nfixed; t++) {
        const int32_t *f = fixed + 4 * t;
        const bool ok = f[0] >= 0 && f[0] < 3 && (f[1] == 0 || f[1] == 1) && f[2] >= -1 && f[2] < npar &&
                        f[3] >= -1 && f[3] < 3 && (f[2] >= 0 || f[3] >= 0);
        if (!ok) return fail(MPT_EINVAL, "fixed term %d = {%d, %d, %d, %d} is malformed", t, f[0], f[1], f[2], f[3]);
    }
    for (int t = 0; t < nquad; t++) {
        const int32_t *q = quad + 4 * t;
        const bool ok = q[0] >= 0 && q[0] < 3 && (q[1] == 0 || q[1] == 1) && q[2] >= 0 && q[2] < 3 &&
                        q[3] >= 0 && q[3] < 3;
        if (!ok) return fail(MPT_EINVAL, "Cauchy product %d = {%d, %d, %d, %d} is malformed", t, q[0], q[1], q[2], q[3]);
    }
    // the parameters, then tau (kept from mpt_init), in the interchange layout
    const int L = c->L, np = npar + 1;
    std::vector<int32_t> ps(np), pe(np);
    std::vector<uint32_t> pl((size_t)np * L, 0u);
    for (int j = 0; j < npar; j++) {
        if (!params[j]) return fail(MPT_EINVAL, "parameter %d is null", j);
        int rc = mpt_host::parse_number(params[j], L, &ps[j], &pe[j], &pl[(size_t)j * L]);
        if (rc) return fail(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use parameter %d = \"%s\"", j, params[j]);
    }
    ps[npar] = c->par_s[3];
    pe[npar] = c->par_e[3];
    std::memcpy(&pl[(size_t)npar * L], &c->par_l[(size_t)3 * L], sizeof(uint32_t) * L);
    std::vector<uint32_t> dl;
    std::vector<int32_t> de, df;
    int rc = to_device_layout(c, ps.data(), pe.data(), pl.data(), np, dl, de, df);
    if (rc) return rc;
    rc = wait_steps(c);
    if (rc) return rc;
    cudaError_t ce = cudaSuccess;
    if (!c->sysT) ce = dalloc(&c->sysT, (size_t)4 * (mpt::SYS_MAX_FIXED + mpt::SYS_MAX_QUAD));
    std::vector<int32_t> tab((size_t)4 * (nfixed + nquad));
    if (nfixed) std::memcpy(tab.data(), fixed, sizeof(int32_t) * 4 * nfixed);
    if (nquad) std::memcpy(tab.data() + 4 * nfixed, quad, sizeof(int32_t) * 4 * nquad);
    if (ce == cudaSuccess && !tab.empty())
        ce = cudaMemcpy(c->sysT, tab.data(), sizeof(int32_t) * tab.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->parL, dl.data(), sizeof(uint32_t) * np * c->Lp, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->parE, de.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(c->parF, df.data(), sizeof(int32_t) * np, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return cuda_fail(ce, "system upload");
    c->sysNF = nfixed;
    c->sysNQ = nquad;
    c->sys_npar = npar;
    c->have_coefficients = false;
    return MPT_OK;
}

}  // extern "C"

namespace {

// queue nsteps steps on the context's stream; records go to the device buffers
// exact: every product in full (a rerun, or mpt_set_exact); rerun: keep the
// chunk counter of the launch being repeated
int launch_steps(mpt_ctx *c, int64_t nsteps, long long nrec, int64_t record_every,
                 bool exact = false, bool rerun = false)
{
    exact = exact || c->force_exact;
    c->last_nsteps = nsteps;
    c->last_nrec = nrec;
    c->last_every = record_every;
    c->last_exact = exact;
    cudaError_t ce = cudaSuccess;
    if (nrec > c->rec_cap) {
        ce = cudaStreamSynchronize(c->st);
        if (ce != cudaSuccess) return cuda_fail(ce, "stream synchronisation");
        if (c->recS) cudaFree(c->recS);
        if (c->recE) cudaFree(c->recE);
        if (c->recL) cudaFree(c->recL);
        c->recS = c->recE = nullptr;
        c->recL = nullptr;
        c->rec_cap = 0;
        ce = dalloc(&c->recS, (size_t)nrec * 3);
        if (ce == cudaSuccess) ce = dalloc(&c->recE, (size_t)nrec * 3);
        if (ce == cudaSuccess) ce = dalloc(&c->recL, (size_t)nrec * 3 * c->L);
        if (ce != cudaSuccess)
            return fail(ce == cudaErrorMemoryAllocation ? MPT_ENOMEM : MPT_ECUDA,
                        "record buffer: %s", cudaGetErrorString(ce));
        c->rec_cap = nrec;
    }
    // keep the starting state so that a failed launch leaves it unchanged
    ce = cudaMemcpyAsync(c->stBackL, c->stL, sizeof(uint32_t) * 3 * c->Lp, cudaMemcpyDeviceToDevice, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->stBackEF, c->stE, sizeof(int32_t) * 3, cudaMemcpyDeviceToDevice, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(c->stBackEF + 3, c->stF, sizeof(int32_t) * 3, cudaMemcpyDeviceToDevice, c->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->bar, 0, sizeof(unsigned) * 2, c->st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(c->gwin, 0, sizeof(long long) * 9 * c->Wcap, c->st);
    if (ce == cudaSuccess && !rerun)
        ce = cudaMemsetAsync(c->chunks, 0, sizeof(unsigned long long), c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "launch preparation");
    mpt::KArgs a{};  // value-initialised: vG = 0 (the launch's own grid)
    a.L = c->L;
    a.Lp = c->Lp;
    a.P = c->P;
    a.N = c->N;
    a.Wcap = c->Wcap;
    a.tb = c->tb;
    a.nwin = c->nwin;
    a.coefL = c->coefL;
    a.coefE = c->coefE;
    a.coefF = c->coefF;
    a.parL = c->parL;
    a.parE = c->parE;
    a.parF = c->parF;
    a.stL = c->stL;
    a.stE = c->stE;
    a.stF = c->stF;
    a.gwin = c->gwin;
    a.bar = c->bar;
    a.status = c->status;
    a.recS = c->recS;
    a.recE = c->recE;
    a.recL = c->recL;
    a.nsteps = nsteps;
    a.record_every = nrec > 0 ? record_every : 0;
    a.prof = c->prof;
    a.timeline = c->prof ? c->prof + prof_rows_len(c) : nullptr;
    a.spin_limit = c->spin_limit;
    a.sysT = c->sysT;
    a.sysNF = c->sysNF;
    a.sysNQ = c->sysNQ;
    a.npar = c->sysT ? c->sys_npar + 1 : 4;
    a.ptau = c->sysT ? c->sys_npar : 3;
    a.exact = exact ? 1 : 0;
    a.chunks = c->chunks;
    a.divtab = c->divtab;
    a.divtab_rl = c->divtab_rl;
    a.tau_p = c->tau_p;
    a.tau_q = c->tau_q;
    a.tau_r = c->tau_r;
    a.tau_shift = c->tau_shift;
    a.tau_neg = c->tau_neg;
    if (c->prof) {
        ce = cudaMemsetAsync(c->prof, 0, sizeof(long long) * prof_len(c), c->st);
        if (ce != cudaSuccess) return cuda_fail(ce, "profile reset");
    }
    if (kind_for(c) == 2) {
        mpt::PArgs pa;
        pa.pub = c->pub;
        pa.done = c->done;
        pa.gin = c->gin;
        pa.C = c->pipe_C;
        pa.imid = c->imid;
        pa.tb = c->pipe_tb;
        ce = cudaMemsetAsync(c->pub, 0, sizeof(unsigned), c->st);
        if (ce == cudaSuccess) ce = cudaMemsetAsync(c->done, 0, sizeof(unsigned) * mpt::PIPE_SETS, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemsetAsync(c->gin, 0, sizeof(long long) * mpt::PIPE_SETS * 9 * c->Wcap, c->st);
        if (ce == cudaSuccess) ce = mpt::launch_pipe(a, pa, pipe_grid_for(c), c->pipe_smem, c->st);
    } else {
        ce = mpt::launch_integrate(a, grid_for(c), c->smem, c->st);
    }
    if (ce != cudaSuccess) return cuda_fail(ce, "kernel launch");
    c->pending = true;
    return MPT_OK;
}

// wait for queued steps; on a device-side error put the starting state back
int wait_steps(mpt_ctx *c)
{
    int status = 0;
    cudaError_t ce = cudaMemcpyAsync(&status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "kernel execution");
    if (!c->pending) return MPT_OK;
    c->pending = false;
    c->have_coefficients = true;
    if (status != 0) {
        cudaMemcpyAsync(c->stL, c->stBackL, sizeof(uint32_t) * 3 * c->Lp, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->stE, c->stBackEF, sizeof(int32_t) * 3, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->stF, c->stBackEF + 3, sizeof(int32_t) * 3, cudaMemcpyDeviceToDevice, c->st);
        cudaMemsetAsync(c->status, 0, sizeof(int), c->st);
        cudaStreamSynchronize(c->st);
        c->have_coefficients = false;
        if (status == mpt::DEV_INEXACT && !c->last_exact) {
            // a shortened sum could not be shown exact: the same launch again,
            // from the same state, with every product in full
            c->exact_reruns++;
            int rc = launch_steps(c, c->last_nsteps, c->last_nrec, c->last_every, true, true);
            if (rc) return rc;
            return wait_steps(c);
        }
        if (status == mpt::DEV_ERANGE)
            return fail(MPT_ERANGE, "exponent out of range, or an exact sum spans more than %d limbs",
                        c->Wcap);
        if (status == mpt::DEV_TIMEOUT) return fail(MPT_ETIMEDOUT, "a grid barrier wait expired");
        return fail(MPT_ECUDA, "device invariant failed (status %d)", status);
    }
    return MPT_OK;
}

}  // namespace

extern "C" {

int mpt_integrate(mpt_ctx *c, int64_t nsteps, int64_t record_every, int32_t *rs, int32_t *re,
                  uint32_t *rl)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (nsteps < 0) return fail(MPT_EINVAL, "nsteps < 0");
    long long nrec = record_every > 0 ? nsteps / record_every : 0;
    if (nrec > 0 && (!rs || !re || !rl)) return fail(MPT_EINVAL, "record pointers are null");
    if (nsteps == 0) return MPT_OK;
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(MPT_ECUDA, "cannot select the context's device");
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    int rc = launch_steps(c, nsteps, nrec, record_every);
    if (rc) return rc;
    rc = wait_steps(c);
    if (rc) return rc;
    if (nrec > 0) {
        cudaError_t ce = cudaMemcpyAsync(rs, c->recS, sizeof(int32_t) * nrec * 3, cudaMemcpyDefault, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(re, c->recE, sizeof(int32_t) * nrec * 3, cudaMemcpyDefault, c->st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(rl, c->recL, sizeof(uint32_t) * nrec * 3 * c->L, cudaMemcpyDefault,
                                 c->st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
        if (ce != cudaSuccess) return cuda_fail(ce, "record copy");
    }
    return MPT_OK;
}

int mpt_set_wait_limit(mpt_ctx *c, int64_t polls)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (polls < 0) return fail(MPT_EINVAL, "polls < 0");
    c->spin_limit = polls == 0 ? mpt::DEFAULT_SPIN_LIMIT : polls;
    return MPT_OK;
}

int mpt_set_profiling(mpt_ctx *c, int on)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    DeviceGuard g(c->dev);
    if (on && !c->prof) {
        cudaError_t ce = dalloc(&c->prof, prof_len(c));
        if (ce == cudaSuccess) ce = cudaMemset(c->prof, 0, sizeof(long long) * prof_len(c));
        if (ce != cudaSuccess) return cuda_fail(ce, "profile buffer");
    } else if (!on && c->prof) {
        cudaStreamSynchronize(c->st);
        cudaFree(c->prof);
        c->prof = nullptr;
    }
    return MPT_OK;
}

int mpt_get_profile(mpt_ctx *c, int64_t *cycles, int n)
{
    if (!c || !cycles) return fail(MPT_EINVAL, "null argument");
    if (!c->prof) return fail(MPT_EINVAL, "profiling is off");
    DeviceGuard g(c->dev);
    const size_t len = prof_len(c);
    std::vector<long long> h(len);
    cudaError_t ce = cudaMemcpyAsync(h.data(), c->prof, sizeof(long long) * len,
                                     cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "profile download");
    for (int i = 0; i < n && (size_t)i < len; i++) cycles[i] = h[i];
    return MPT_OK;
}

int mpt_launch(mpt_ctx *c, int64_t nsteps)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (nsteps < 0) return fail(MPT_EINVAL, "nsteps < 0");
    if (nsteps == 0) return MPT_OK;
    if (c->pending) return fail(MPT_EINVAL, "steps already queued: call mpt_wait first");
    DeviceGuard g(c->dev);
    if (!g.ok) return fail(MPT_ECUDA, "cannot select the context's device");
    return launch_steps(c, nsteps, 0, 0);
}

int mpt_wait(mpt_ctx *c)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    DeviceGuard g(c->dev);
    return wait_steps(c);
}

int mpt_set_exact(mpt_ctx *c, int on)
{
    if (!c) return fail(MPT_EINVAL, "null context");
    if (on != 0 && on != 1) return fail(MPT_EINVAL, "on = %d is neither 0 nor 1", on);
    c->force_exact = on != 0;
    return MPT_OK;
}

int mpt_get_counters(mpt_ctx *c, int64_t *exact_reruns, int64_t *chunks)
{
    if (!c || !exact_reruns || !chunks) return fail(MPT_EINVAL, "null argument");
    DeviceGuard g(c->dev);
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    unsigned long long h = 0;
    cudaError_t ce = cudaMemcpyAsync(&h, c->chunks, sizeof h, cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "counter download");
    *exact_reruns = c->exact_reruns;
    *chunks = (int64_t)h;
    return MPT_OK;
}

int mpt_step(mpt_ctx *c) { return mpt_integrate(c, 1, 0, nullptr, nullptr, nullptr); }

int mpt_get_coefficients(mpt_ctx *c, int32_t *s, int32_t *e, uint32_t *l)
{
    if (!c || !s || !e || !l) return fail(MPT_EINVAL, "null argument");
    DeviceGuard g(c->dev);
    if (c->pending) {
        int rc = wait_steps(c);
        if (rc) return rc;
    }
    if (!c->have_coefficients) return fail(MPT_EINVAL, "no step has completed yet");
    const size_t n = (size_t)3 * (c->N + 1);
    std::vector<uint32_t> dl(n * c->Lp);
    std::vector<int32_t> de(n), df(n);
    cudaError_t ce = cudaMemcpyAsync(dl.data(), c->coefL, sizeof(uint32_t) * n * c->Lp,
                                     cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(de.data(), c->coefE, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(df.data(), c->coefF, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->st);
    if (ce != cudaSuccess) return cuda_fail(ce, "coefficient download");
    from_device_layout(c, dl, de, df, (int)n, s, e, l);
    return MPT_OK;
}

}  // extern "C"

namespace {

// the batch, with the parameters (sigma, R, b) of trajectory j at sig[j * per],
// Rr[j * per], bb[j * per] (per = 0: one set for all)
// shape (nullable): {kernel variant (0: registers capped, two CTAs an SM; 1:
// not), terms per staging batch (0: as many as fit, up to 64), window copies
// (0: as many as fit, up to 8)}
int batch_impl(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps, const char *tau,
               const char *const *sig, const char *const *Rr, const char *const *bb, int per,
               int32_t *signs, int32_t *exps, uint32_t *limbs, uint64_t cuda_stream,
               const int32_t *shape = nullptr)
{
    const int variant = shape ? shape[0] : 0, tb_req = shape ? shape[1] : 0, nwin_req = shape ? shape[2] : 0;
    if (variant < 0 || variant > 1) return fail(MPT_EINVAL, "kernel variant %d is neither 0 nor 1", variant);
    if (tb_req < 0 || tb_req > 256) return fail(MPT_EINVAL, "staging batch %d outside 0..256", tb_req);
    if (nwin_req < 0 || nwin_req > 8) return fail(MPT_EINVAL, "window copies %d outside 0..8", nwin_req);
    if (B < 1) return fail(MPT_EINVAL, "batch size %d < 1", B);
    if (!Ls || !Ns || !signs || !exps || !limbs || !sig || !Rr || !bb)
        return fail(MPT_EINVAL, "null argument");
    if (nsteps < 0) return fail(MPT_EINVAL, "nsteps = %lld < 0", (long long)nsteps);
    const char *names[4] = {"sigma", "R", "b", "tau"};
    if (!tau) return fail(MPT_EINVAL, "tau is null");
    for (int j = 0; j < (per ? B : 1); j++)
        if (!sig[j] || !Rr[j] || !bb[j]) return fail(MPT_EINVAL, "trajectory %d: a parameter is null", j);
    // per trajectory: sizes, staging batch, shared memory; offsets in the packed arrays
    struct Traj {
        int L, Lp, P, N, Wcap, tb, nwin;
        size_t off_limbs, off_coef, off_coefEF, off_par, off_st;
        double work;
    };
    std::vector<Traj> T(B);
    size_t n_limbs = 0, n_coef = 0, n_coefEF = 0, n_par = 0, n_st = 0, smem = 0;
    for (int j = 0; j < B; j++) {
        Traj &t = T[j];
        t.L = Ls[j];
        t.N = Ns[j];
        if (t.L < 1 || t.L > mpt::MAX_L) return fail(MPT_EINVAL, "trajectory %d: L = %d outside 1..%d", j, t.L, mpt::MAX_L);
        if (t.N < 1 || t.N > mpt::MAX_N) return fail(MPT_EINVAL, "trajectory %d: N = %d outside 1..%d", j, t.N, mpt::MAX_N);
        t.Lp = (t.L + mpt::W - 1) / mpt::W * mpt::W;
        t.P = t.Lp / mpt::W;
        const int spread = t.Lp > 64 ? t.Lp : 64;
        t.Wcap = (2 * t.Lp + 2 + spread + 31) / 32 * 32;
        t.off_limbs = n_limbs;
        n_limbs += (size_t)3 * t.L;
        t.off_coef = n_coef;
        n_coef += (size_t)3 * (t.N + 1) * t.Lp;
        t.off_coefEF = n_coefEF;
        n_coefEF += (size_t)3 * (t.N + 1);
        t.off_par = n_par;
        n_par += (size_t)4 * t.Lp;
        t.off_st = n_st;
        n_st += (size_t)3 * t.Lp;
        t.work = (double)t.L * t.L * ((double)t.N * (t.N + 1) + 7.0 * t.N);
    }
    // host layouts: parameters (parsed once per L and parameter set) and states
    std::vector<uint32_t> hparL(n_par, 0u), hstL(n_st, 0u);
    std::vector<int32_t> hparE(4 * (size_t)B), hparF(4 * (size_t)B), hstE(3 * (size_t)B), hstF(3 * (size_t)B);
    std::vector<int> done_L;
    std::vector<int> done_j;  // a trajectory with that parameter set
    std::vector<std::vector<uint32_t>> parsed_l;
    std::vector<std::vector<int32_t>> parsed_s, parsed_e;
    for (int j = 0; j < B; j++) {
        const Traj &t = T[j];
        const int jp = j * per;
        const char *strs[4] = {sig[jp], Rr[jp], bb[jp], tau};
        int k = -1;
        for (size_t i = 0; i < done_L.size() && k < 0; i++) {
            const int q = done_j[i] * per;
            if (done_L[i] == t.L && std::strcmp(sig[q], strs[0]) == 0 && std::strcmp(Rr[q], strs[1]) == 0 &&
                std::strcmp(bb[q], strs[2]) == 0)
                k = (int)i;
        }
        if (k < 0) {
            std::vector<uint32_t> l((size_t)4 * t.L, 0u);
            std::vector<int32_t> ps(4), pe(4);
            for (int q = 0; q < 4; q++) {
                const int rc = mpt_host::parse_number(strs[q], t.L, &ps[q], &pe[q], &l[(size_t)q * t.L]);
                if (rc)
                    return fail(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "trajectory %d: cannot use %s = \"%s\"",
                                j, names[q], strs[q]);
            }
            done_L.push_back(t.L);
            done_j.push_back(j);
            parsed_l.push_back(l);
            parsed_s.push_back(ps);
            parsed_e.push_back(pe);
            k = (int)done_L.size() - 1;
        }
        mpt_ctx tmp;
        tmp.L = t.L;
        tmp.Lp = t.Lp;
        std::vector<uint32_t> dl;
        std::vector<int32_t> de, df;
        int rc = to_device_layout(&tmp, parsed_s[k].data(), parsed_e[k].data(), parsed_l[k].data(), 4,
                                  dl, de, df);
        if (rc) return rc;
        std::memcpy(&hparL[t.off_par], dl.data(), sizeof(uint32_t) * 4 * t.Lp);
        for (int q = 0; q < 4; q++) {
            hparE[4 * (size_t)j + q] = de[q];
            hparF[4 * (size_t)j + q] = df[q];
        }
        rc = to_device_layout(&tmp, signs + 3 * (size_t)j, exps + 3 * (size_t)j, limbs + t.off_limbs, 3,
                              dl, de, df);
        if (rc) return fail(rc, "trajectory %d: %s", j, mpt_last_error());
        std::memcpy(&hstL[t.off_st], dl.data(), sizeof(uint32_t) * 3 * t.Lp);
        for (int q = 0; q < 3; q++) {
            hstE[3 * (size_t)j + q] = de[q];
            hstF[3 * (size_t)j + q] = df[q];
        }
    }
    if (nsteps == 0) return MPT_OK;
    // staging batches and shared memory on this device
    int dev = 0, smem_optin = 0, smem_sm = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ce == cudaSuccess)
        ce = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (ce != cudaSuccess) return cuda_fail(ce, "device query");
    for (int j = 0; j < B; j++) {
        Traj &t = T[j];
        int tb = tb_req ? tb_req : 64;
        if (!tb_req)
            while (tb > 8 && mpt::smem_bytes(t.L, t.Lp, t.N, t.Wcap, tb) > (size_t)smem_optin) tb /= 2;
        t.tb = tb;
        // window copies (up to 8) while two CTAs still share an SM (the capped
        // variant) or while one fits (the other)
        const size_t two = smem_sm > 2048 ? (size_t)smem_sm / 2 - 1024 : 0;
        const size_t budget = variant == 1 ? (size_t)smem_optin : two;
        int nwin = nwin_req ? nwin_req : 8;
        if (!nwin_req)
            while (nwin > 1 && mpt::smem_bytes(t.L, t.Lp, t.N, t.Wcap, tb, nwin) > budget) nwin /= 2;
        t.nwin = nwin;
        const size_t sm = mpt::smem_bytes(t.L, t.Lp, t.N, t.Wcap, tb, nwin);
        if (sm > (size_t)smem_optin)
            return fail(MPT_EINVAL, "trajectory %d: L = %d, N = %d need %zu bytes of shared memory", j,
                        t.L, t.N, sm);
        if (sm > smem) smem = sm;
    }
    cudaStream_t st = (cudaStream_t)(uintptr_t)cuda_stream;
    uint32_t *coefL = nullptr, *parL = nullptr, *stL = nullptr;
    int32_t *coefE = nullptr, *coefF = nullptr, *parE = nullptr, *parF = nullptr, *stE = nullptr, *stF = nullptr;
    int *status = nullptr;
    unsigned *bar = nullptr;
    long long *gwin = nullptr;
    mpt::KArgs *dargs = nullptr;
    ce = dalloc(&coefL, n_coef);
    if (ce == cudaSuccess) ce = dalloc(&coefE, n_coefEF);
    if (ce == cudaSuccess) ce = dalloc(&coefF, n_coefEF);
    if (ce == cudaSuccess) ce = dalloc(&parL, n_par);
    if (ce == cudaSuccess) ce = dalloc(&parE, 4 * (size_t)B);
    if (ce == cudaSuccess) ce = dalloc(&parF, 4 * (size_t)B);
    if (ce == cudaSuccess) ce = dalloc(&stL, n_st);
    if (ce == cudaSuccess) ce = dalloc(&stE, 3 * (size_t)B);
    if (ce == cudaSuccess) ce = dalloc(&stF, 3 * (size_t)B);
    if (ce == cudaSuccess) ce = dalloc(&status, 1);
    if (ce == cudaSuccess) ce = dalloc(&bar, 2);
    if (ce == cudaSuccess) ce = dalloc(&gwin, 1);
    if (ce == cudaSuccess) ce = dalloc(&dargs, (size_t)B);
    auto release = [&]() {
        cudaFree(coefL);
        cudaFree(coefE);
        cudaFree(coefF);
        cudaFree(parL);
        cudaFree(parE);
        cudaFree(parF);
        cudaFree(stL);
        cudaFree(stE);
        cudaFree(stF);
        cudaFree(status);
        cudaFree(bar);
        cudaFree(gwin);
        cudaFree(dargs);
    };
    if (ce != cudaSuccess) {
        release();
        return fail(ce == cudaErrorMemoryAllocation ? MPT_ENOMEM : MPT_ECUDA, "batch buffers: %s",
                    cudaGetErrorString(ce));
    }
    // tau as a small ratio p/q at each L (Horner steps without a limb product)
    struct TauRatio {
        int L;
        uint32_t p, q, r;
        int shift, neg;
    };
    std::vector<TauRatio> ratios;
    auto ratio_for = [&](int L) -> const TauRatio & {
        for (const TauRatio &t : ratios)
            if (t.L == L) return t;
        TauRatio t{L, 0, 0, 0, 0, 0};
        if (mpt_host::small_ratio(tau, L, &t.p, &t.q, &t.r, &t.shift, &t.neg)) t.q = 0;
        ratios.push_back(t);
        return ratios.back();
    };
    // argument blocks, heaviest trajectories first (CTAs start in index order)
    std::vector<int> order(B);
    for (int j = 0; j < B; j++) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return T[x].work > T[y].work; });
    std::vector<mpt::KArgs> hargs(B);
    for (int i = 0; i < B; i++) {
        const int j = order[i];
        const Traj &t = T[j];
        mpt::KArgs a{};
        a.L = t.L;
        a.Lp = t.Lp;
        a.P = t.P;
        a.N = t.N;
        a.Wcap = t.Wcap;
        a.tb = t.tb;
        a.nwin = t.nwin;
        a.coefL = coefL + t.off_coef;
        a.coefE = coefE + t.off_coefEF;
        a.coefF = coefF + t.off_coefEF;
        a.parL = parL + t.off_par;
        a.parE = parE + 4 * (size_t)j;
        a.parF = parF + 4 * (size_t)j;
        a.stL = stL + t.off_st;
        a.stE = stE + 3 * (size_t)j;
        a.stF = stF + 3 * (size_t)j;
        a.gwin = gwin;
        a.bar = bar;
        a.status = status;
        a.nsteps = nsteps;
        a.record_every = 0;
        a.spin_limit = mpt::DEFAULT_SPIN_LIMIT;
        a.vG = 1;
        a.vg = 0;
        const TauRatio tr = ratio_for(t.L);
        a.tau_p = tr.p;
        a.tau_q = tr.q;
        a.tau_r = tr.r;
        a.tau_shift = tr.shift;
        a.tau_neg = tr.neg;
        hargs[i] = a;
    }
    ce = cudaMemcpyAsync(parL, hparL.data(), sizeof(uint32_t) * n_par, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(parE, hparE.data(), sizeof(int32_t) * 4 * B, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(parF, hparF.data(), sizeof(int32_t) * 4 * B, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(stL, hstL.data(), sizeof(uint32_t) * n_st, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(stE, hstE.data(), sizeof(int32_t) * 3 * B, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(stF, hstF.data(), sizeof(int32_t) * 3 * B, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2, st);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(dargs, hargs.data(), sizeof(mpt::KArgs) * B, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = mpt::launch_batch(dargs, B, smem, st, variant);
    int hstatus = 0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&hstatus, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hstL.data(), stL, sizeof(uint32_t) * n_st, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hstE.data(), stE, sizeof(int32_t) * 3 * B, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(hstF.data(), stF, sizeof(int32_t) * 3 * B, cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    release();
    if (ce != cudaSuccess) return cuda_fail(ce, "batch launch");
    if (hstatus == mpt::DEV_ERANGE) return fail(MPT_ERANGE, "exponent or window range exceeded in the batch");
    if (hstatus != 0) return fail(MPT_ECUDA, "batch kernel status %d", hstatus);
    // the new states, in the caller's order and layout
    for (int j = 0; j < B; j++) {
        const Traj &t = T[j];
        mpt_ctx tmp;
        tmp.L = t.L;
        tmp.Lp = t.Lp;
        std::vector<uint32_t> dl(hstL.begin() + t.off_st, hstL.begin() + t.off_st + 3 * (size_t)t.Lp);
        std::vector<int32_t> de(hstE.begin() + 3 * (size_t)j, hstE.begin() + 3 * (size_t)j + 3);
        std::vector<int32_t> df(hstF.begin() + 3 * (size_t)j, hstF.begin() + 3 * (size_t)j + 3);
        from_device_layout(&tmp, dl, de, df, 3, signs + 3 * (size_t)j, exps + 3 * (size_t)j, limbs + t.off_limbs);
    }
    return MPT_OK;
}

}  // namespace

extern "C" {

int mpt_integrate_batch(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps, const char *tau,
                        const char *sigma, const char *R, const char *b, int32_t *signs,
                        int32_t *exps, uint32_t *limbs, uint64_t cuda_stream)
{
    return batch_impl(B, Ls, Ns, nsteps, tau, &sigma, &R, &b, 0, signs, exps, limbs, cuda_stream);
}

int mpt_integrate_batch_shape(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps,
                              const char *tau, const char *sigma, const char *R, const char *b,
                              int32_t *signs, int32_t *exps, uint32_t *limbs, const int32_t *shape,
                              uint64_t cuda_stream)
{
    return batch_impl(B, Ls, Ns, nsteps, tau, &sigma, &R, &b, 0, signs, exps, limbs, cuda_stream, shape);
}

int mpt_integrate_batch_params(int B, const int32_t *Ls, const int32_t *Ns, int64_t nsteps,
                               const char *tau, const char *const *sigma, const char *const *R,
                               const char *const *b, int32_t *signs, int32_t *exps, uint32_t *limbs,
                               uint64_t cuda_stream)
{
    return batch_impl(B, Ls, Ns, nsteps, tau, sigma, R, b, 1, signs, exps, limbs, cuda_stream);
}

int mpt_jacobian_fd(int B, int L, int N, int64_t nsteps, const char *tau, const char *sigma,
                    const char *R, const char *b, const char *const *x0, int h_digits, double *jac,
                    uint64_t cuda_stream)
{
    if (B < 1) return fail(MPT_EINVAL, "batch size %d < 1", B);
    if (!tau || !sigma || !R || !b || !x0 || !jac) return fail(MPT_EINVAL, "null argument");
    if (h_digits == 0) h_digits = 100;
    if (h_digits < 1 || h_digits > 10000) return fail(MPT_EINVAL, "h_digits = %d outside 1..10000", h_digits);
    if (L < 1 || L > mpt::MAX_L) return fail(MPT_EINVAL, "L = %d outside 1..%d", L, mpt::MAX_L);
    for (int j = 0; j < 3 * B; j++)
        if (!x0[j]) return fail(MPT_EINVAL, "initial value %d is null", j);
    // runs: per point j and input i (x0, y0, z0, sigma, R, b), u + h e_i then u - h e_i
    const int runs = 12 * B;
    const char *par[3] = {sigma, R, b};
    std::vector<std::string> pstr((size_t)runs * 3);
    std::vector<int32_t> ss((size_t)runs * 3), se((size_t)runs * 3), Ls(runs, L), Ns(runs, N);
    std::vector<uint32_t> sl((size_t)runs * 3 * L);
    for (int j = 0; j < B; j++)
        for (int i = 0; i < 6; i++)
            for (int t = 0; t < 2; t++) {
                const int run = (j * 6 + i) * 2 + t, sg = t == 0 ? 1 : -1;
                for (int k = 0; k < 3; k++) {
                    std::string v = x0[3 * j + k];
                    if (i == k && mpt_host::perturbed_string(x0[3 * j + k], h_digits, sg, v))
                        return fail(MPT_EINVAL, "cannot use initial value \"%s\"", x0[3 * j + k]);
                    const size_t q = (size_t)run * 3 + k;
                    const int rc = mpt_host::parse_number(v.c_str(), L, &ss[q], &se[q], &sl[q * L]);
                    if (rc) return fail(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use initial value \"%s\"",
                                        x0[3 * j + k]);
                    std::string pv = par[k];
                    if (i == 3 + k && mpt_host::perturbed_string(par[k], h_digits, sg, pv))
                        return fail(MPT_EINVAL, "cannot use parameter \"%s\"", par[k]);
                    pstr[q] = pv;
                }
            }
    std::vector<const char *> ps[3];
    for (int k = 0; k < 3; k++) {
        ps[k].resize(runs);
        for (int r = 0; r < runs; r++) ps[k][r] = pstr[(size_t)r * 3 + k].c_str();
    }
    const int rc = batch_impl(runs, Ls.data(), Ns.data(), nsteps, tau, ps[0].data(), ps[1].data(),
                              ps[2].data(), 1, ss.data(), se.data(), sl.data(), cuda_stream);
    if (rc) return rc;
    for (int j = 0; j < B; j++)
        for (int i = 0; i < 6; i++)
            for (int o = 0; o < 3; o++) {
                const size_t a = ((size_t)(j * 6 + i) * 2) * 3 + o, c = a + 3;
                jac[((size_t)j * 3 + o) * 6 + i] =
                    mpt_host::diff_over_2h(L, ss[a], se[a], &sl[a * L], ss[c], se[c], &sl[c * L], h_digits);
            }
    return MPT_OK;
}

}  // extern "C"
