// mpt_adjoint.cu -- the reverse sweep of the Taylor method (derivatives of
// the n-step map of Eq. (3) and Eq. (2), Sec. 2, with respect to the initial
// state and sigma, R, b): host orchestration of mpt_backward_raw and
// mpt_backward (include/mpt.h).
//
// Plan of one call (B trajectories of one L and N; G adjoint vectors each):
//  1. forward in segments of `every` steps from the initial states, the
//     state after each segment kept as a checkpoint (one batch launch a
//     segment, one CTA a trajectory);
//  2. last segment first: the segment's steps again from its checkpoint,
//     every step's coefficient table kept (the batch kernel's history), then
//     one launch of the reverse sweep over those steps (one CTA an adjoint
//     vector), which carries gbar and the parameter adjoints on to the
//     segment before.
// So the derivatives cost about four forward runs (one forward pass, one
// recomputation, and a sweep with twice the products of a forward step) for
// G = 1, and 2 + 2G for G vectors.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/mpt.h"
#include "host_parse.h"
#include "mpt_kernel.cuh"

namespace mpt {
int record_error(int code, const char *msg);  // sets mpt_last_error() (mpt_host.cu)
}

namespace {

using namespace mpt;

int failf(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return record_error(code, buf);
}

int cuda_failf(cudaError_t e, const char *what)
{
    return failf(MPT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// device buffers of one call, freed on scope exit
struct Buffers {
    std::vector<void *> ptrs;
    ~Buffers()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t get(T **p, size_t count)
    {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (count ? count : 1));
        if (e != cudaSuccess) {
            *p = nullptr;
            (void)cudaGetLastError();
            return e;
        }
        ptrs.push_back(*p);
        return e;
    }
};

// interchange (sign, exp, L limbs) -> the kernel's (Lp limbs, exp, flags); false if malformed
bool to_dev(int L, int Lp, int32_t s, int32_t e, const uint32_t *l, uint32_t *dl, int32_t *de, int32_t *df)
{
    bool zero = true;
    for (int x = 0; x < L; x++) zero = zero && l[x] == 0;
    std::memset(dl, 0, sizeof(uint32_t) * Lp);
    if (zero) {
        *de = 0;
        *df = 0;
        return s == 0 && e == 0;
    }
    if ((s != 0 && s != 1) || l[L - 1] == 0 || e > (1 << 30) || e < -(1 << 30)) return false;
    std::memcpy(dl, l, sizeof(uint32_t) * L);
    *de = e;
    *df = F_NZ | (s ? F_NEG : 0);
    return true;
}

void from_dev(int L, const uint32_t *dl, int32_t de, int32_t df, int32_t *s, int32_t *e, uint32_t *l)
{
    *s = (df & F_NEG) ? 1 : 0;
    *e = de;
    std::memcpy(l, dl, sizeof(uint32_t) * L);
}

int status_error(int st)
{
    if (st == DEV_ERANGE) return failf(MPT_ERANGE, "exponent or window range exceeded in the reverse sweep");
    if (st == DEV_TIMEOUT) return failf(MPT_ETIMEDOUT, "a bounded device wait expired");
    return failf(MPT_ECUDA, "device status %d in the reverse sweep", st);
}

// tau as a small ratio p/q (q = 0: not known to be one), for the forward
// recomputation's Horner steps without a limb product
struct TauRatio {
    uint32_t p = 0, q = 0, r = 0;
    int shift = 0, neg = 0;
};

int backward_impl(int B, int G, int L, int N, int64_t nsteps, int checkpoint_every,
                  const int32_t *par_signs, const int32_t *par_exps, const uint32_t *par_limbs,
                  const int32_t *st_signs, const int32_t *st_exps, const uint32_t *st_limbs,
                  int32_t *g_signs, int32_t *g_exps, uint32_t *g_limbs, int32_t *th_signs,
                  int32_t *th_exps, uint32_t *th_limbs, uint64_t cuda_stream, const TauRatio &tr)
{
    if (B < 1 || G < 1) return failf(MPT_EINVAL, "B = %d and G = %d must be >= 1", B, G);
    if ((long long)B * G > (1LL << 24)) return failf(MPT_EINVAL, "B * G = %lld is too large", (long long)B * G);
    if (L < 1 || L > MAX_L) return failf(MPT_EINVAL, "L = %d outside 1..%d", L, MAX_L);
    if (N < 1 || N > MAX_N) return failf(MPT_EINVAL, "N = %d outside 1..%d", N, MAX_N);
    if (nsteps < 0) return failf(MPT_EINVAL, "nsteps = %lld < 0", (long long)nsteps);
    if (checkpoint_every < 0) return failf(MPT_EINVAL, "checkpoint_every = %d < 0", checkpoint_every);
    if (!par_signs || !par_exps || !par_limbs || !st_signs || !st_exps || !st_limbs || !g_signs ||
        !g_exps || !g_limbs || !th_signs || !th_exps || !th_limbs)
        return failf(MPT_EINVAL, "null argument");
    const int every = checkpoint_every == 0 ? 50 : checkpoint_every;
    const int items = B * G;
    const int Lp = (L + W - 1) / W * W, P = Lp / W, N1 = N + 1;
    const int spread = Lp > 64 ? Lp : 64;
    const int Wcap = (2 * Lp + 2 + spread + 31) / 32 * 32;
    const size_t nc = 3 * (size_t)N1;  // numbers of a coefficient table
    // inputs in the kernel's layout: parameters (sigma, R, b, tau), states, gbar
    std::vector<uint32_t> hpar((size_t)4 * Lp), hst((size_t)B * 3 * Lp), hgb((size_t)items * 3 * Lp);
    std::vector<int32_t> hparE(4), hparF(4), hstE((size_t)B * 3), hstF((size_t)B * 3), hgE((size_t)items * 3),
        hgF((size_t)items * 3);
    const char *pname[4] = {"sigma", "R", "b", "tau"};
    for (int p = 0; p < 4; p++)
        if (!to_dev(L, Lp, par_signs[p], par_exps[p], par_limbs + (size_t)p * L, &hpar[(size_t)p * Lp],
                    &hparE[p], &hparF[p]))
            return failf(MPT_EINVAL, "%s: malformed number", pname[p]);
    for (int k = 0; k < 3 * B; k++)
        if (!to_dev(L, Lp, st_signs[k], st_exps[k], st_limbs + (size_t)k * L, &hst[(size_t)k * Lp], &hstE[k],
                    &hstF[k]))
            return failf(MPT_EINVAL, "state %d of trajectory %d: malformed number", k % 3, k / 3);
    for (int k = 0; k < 3 * items; k++)
        if (!to_dev(L, Lp, g_signs[k], g_exps[k], g_limbs + (size_t)k * L, &hgb[(size_t)k * Lp], &hgE[k],
                    &hgF[k]))
            return failf(MPT_EINVAL, "gbar %d of item %d: malformed number", k % 3, k / 3);
    if (nsteps == 0) {
        for (int k = 0; k < 3 * items; k++) {
            th_signs[k] = 0;
            th_exps[k] = 0;
        }
        std::memset(th_limbs, 0, sizeof(uint32_t) * 3 * (size_t)items * L);
        return MPT_OK;
    }
    // shared memory, staging batch and window copies as the batch kernel takes them
    int dev = 0, smem_optin = 0, smem_sm = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (ce != cudaSuccess) return cuda_failf(ce, "device query");
    int tb = 64;
    while (tb > 8 && smem_bytes(L, Lp, N, Wcap, tb, 1, true) > (size_t)smem_optin) tb /= 2;
    const size_t two = smem_sm > 2048 ? (size_t)smem_sm / 2 - 1024 : 0;
    int nwin = 8;
    while (nwin > 1 && smem_bytes(L, Lp, N, Wcap, tb, nwin, true) > two) nwin /= 2;
    const size_t smem = smem_bytes(L, Lp, N, Wcap, tb, nwin, true);
    if (smem > (size_t)smem_optin)
        return failf(MPT_EINVAL, "L = %d, N = %d need %zu bytes of shared memory", L, N, smem);
    const long long nseg = (nsteps + every - 1) / every;
    // device buffers
    Buffers db;
    uint32_t *parL, *stL, *ckL, *coefL, *histL, *ycoefL, *aparL, *powL;
    int32_t *parE, *parF, *stE, *stF, *ckE, *ckF, *coefE, *coefF, *histE, *histF, *ycoefE, *ycoefF, *aparE,
        *aparF, *powE, *powF;
    int *status;
    unsigned *bar;
    long long *gwin;
    KArgs *fargs, *aargs;
    ce = db.get(&parL, (size_t)4 * Lp);
    if (ce == cudaSuccess) ce = db.get(&parE, 4);
    if (ce == cudaSuccess) ce = db.get(&parF, 4);
    if (ce == cudaSuccess) ce = db.get(&stL, (size_t)B * 3 * Lp);
    if (ce == cudaSuccess) ce = db.get(&stE, (size_t)B * 3);
    if (ce == cudaSuccess) ce = db.get(&stF, (size_t)B * 3);
    if (ce == cudaSuccess) ce = db.get(&ckL, (size_t)(nseg + 1) * B * 3 * Lp);
    if (ce == cudaSuccess) ce = db.get(&ckE, (size_t)(nseg + 1) * B * 3);
    if (ce == cudaSuccess) ce = db.get(&ckF, (size_t)(nseg + 1) * B * 3);
    if (ce == cudaSuccess) ce = db.get(&coefL, (size_t)B * nc * Lp);
    if (ce == cudaSuccess) ce = db.get(&coefE, (size_t)B * nc);
    if (ce == cudaSuccess) ce = db.get(&coefF, (size_t)B * nc);
    if (ce == cudaSuccess) ce = db.get(&histL, (size_t)B * every * nc * Lp);
    if (ce == cudaSuccess) ce = db.get(&histE, (size_t)B * every * nc);
    if (ce == cudaSuccess) ce = db.get(&histF, (size_t)B * every * nc);
    if (ce == cudaSuccess) ce = db.get(&ycoefL, (size_t)items * nc * Lp);
    if (ce == cudaSuccess) ce = db.get(&ycoefE, (size_t)items * nc);
    if (ce == cudaSuccess) ce = db.get(&ycoefF, (size_t)items * nc);
    if (ce == cudaSuccess) ce = db.get(&aparL, (size_t)items * ADJ_NPAR * Lp);
    if (ce == cudaSuccess) ce = db.get(&aparE, (size_t)items * ADJ_NPAR);
    if (ce == cudaSuccess) ce = db.get(&aparF, (size_t)items * ADJ_NPAR);
    if (ce == cudaSuccess) ce = db.get(&powL, (size_t)items * N1 * Lp);
    if (ce == cudaSuccess) ce = db.get(&powE, (size_t)items * N1);
    if (ce == cudaSuccess) ce = db.get(&powF, (size_t)items * N1);
    if (ce == cudaSuccess) ce = db.get(&status, 1);
    if (ce == cudaSuccess) ce = db.get(&bar, 2);
    if (ce == cudaSuccess) ce = db.get(&gwin, 1);
    if (ce == cudaSuccess) ce = db.get(&fargs, (size_t)B);
    if (ce == cudaSuccess) ce = db.get(&aargs, (size_t)items);
    if (ce != cudaSuccess)
        return failf(ce == cudaErrorMemoryAllocation ? MPT_ENOMEM : MPT_ECUDA, "reverse-sweep buffers: %s",
                     cudaGetErrorString(ce));
    cudaStream_t st = (cudaStream_t)(uintptr_t)cuda_stream;
    // the adjoint items' parameter rows: sigma, R, b, tau, gbar, zero parameter adjoints
    std::vector<uint32_t> hapar((size_t)items * ADJ_NPAR * Lp, 0u);
    std::vector<int32_t> haparE((size_t)items * ADJ_NPAR, 0), haparF((size_t)items * ADJ_NPAR, 0);
    for (int it = 0; it < items; it++) {
        uint32_t *row = &hapar[(size_t)it * ADJ_NPAR * Lp];
        std::memcpy(row, hpar.data(), sizeof(uint32_t) * 4 * Lp);
        std::memcpy(row + (size_t)ADJ_GBAR * Lp, &hgb[(size_t)it * 3 * Lp], sizeof(uint32_t) * 3 * Lp);
        for (int p = 0; p < 4; p++) {
            haparE[(size_t)it * ADJ_NPAR + p] = hparE[p];
            haparF[(size_t)it * ADJ_NPAR + p] = hparF[p];
        }
        for (int k = 0; k < 3; k++) {
            haparE[(size_t)it * ADJ_NPAR + ADJ_GBAR + k] = hgE[(size_t)it * 3 + k];
            haparF[(size_t)it * ADJ_NPAR + ADJ_GBAR + k] = hgF[(size_t)it * 3 + k];
        }
    }
    ce = cudaMemcpyAsync(parL, hpar.data(), sizeof(uint32_t) * 4 * Lp, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(parE, hparE.data(), sizeof(int32_t) * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(parF, hparF.data(), sizeof(int32_t) * 4, cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(ckL, hst.data(), sizeof(uint32_t) * hst.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(ckE, hstE.data(), sizeof(int32_t) * hstE.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(ckF, hstF.data(), sizeof(int32_t) * hstF.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(aparL, hapar.data(), sizeof(uint32_t) * hapar.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(aparE, haparE.data(), sizeof(int32_t) * haparE.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(aparF, haparF.data(), sizeof(int32_t) * haparF.size(), cudaMemcpyHostToDevice, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(status, 0, sizeof(int), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2, st);
    if (ce != cudaSuccess) return cuda_failf(ce, "reverse-sweep uploads");
    // argument blocks: trajectory b's forward (one per trajectory), item (b, g)'s sweep
    auto forward_args = [&](long long n, bool hist) {
        std::vector<KArgs> h(B);
        for (int b = 0; b < B; b++) {
            KArgs a{};
            a.L = L;
            a.Lp = Lp;
            a.P = P;
            a.N = N;
            a.Wcap = Wcap;
            a.tb = tb;
            a.nwin = nwin;
            a.coefL = coefL + (size_t)b * nc * Lp;
            a.coefE = coefE + (size_t)b * nc;
            a.coefF = coefF + (size_t)b * nc;
            a.parL = parL;
            a.parE = parE;
            a.parF = parF;
            a.stL = stL + (size_t)b * 3 * Lp;
            a.stE = stE + (size_t)b * 3;
            a.stF = stF + (size_t)b * 3;
            a.gwin = gwin;
            a.bar = bar;
            a.status = status;
            a.nsteps = n;
            a.spin_limit = DEFAULT_SPIN_LIMIT;
            a.vG = 1;
            a.vg = 0;
            a.npar = 4;
            a.ptau = 3;
            a.tau_p = tr.p;
            a.tau_q = tr.q;
            a.tau_r = tr.r;
            a.tau_shift = tr.shift;
            a.tau_neg = tr.neg;
            if (hist) {
                a.histL = histL + (size_t)b * every * nc * Lp;
                a.histE = histE + (size_t)b * every * nc;
                a.histF = histF + (size_t)b * every * nc;
            }
            h[b] = a;
        }
        return h;
    };
    std::vector<KArgs> hadj(items);
    for (int it = 0; it < items; it++) {
        const int b = it / G;
        KArgs a{};
        a.L = L;
        a.Lp = Lp;
        a.P = P;
        a.N = N;
        a.Wcap = Wcap;
        a.tb = tb;
        a.nwin = nwin;
        a.coefL = ycoefL + (size_t)it * nc * Lp;
        a.coefE = ycoefE + (size_t)it * nc;
        a.coefF = ycoefF + (size_t)it * nc;
        a.parL = aparL + (size_t)it * ADJ_NPAR * Lp;
        a.parE = aparE + (size_t)it * ADJ_NPAR;
        a.parF = aparF + (size_t)it * ADJ_NPAR;
        a.gwin = gwin;
        a.bar = bar;
        a.status = status;
        a.spin_limit = DEFAULT_SPIN_LIMIT;
        a.vG = 1;
        a.vg = 0;
        a.npar = ADJ_NPAR;
        a.ptau = 3;
        a.adj = 1;
        a.fwdL = histL + (size_t)b * every * nc * Lp;
        a.fwdE = histE + (size_t)b * every * nc;
        a.fwdF = histF + (size_t)b * every * nc;
        a.powL = powL + (size_t)it * N1 * Lp;
        a.powE = powE + (size_t)it * N1;
        a.powF = powF + (size_t)it * N1;
        hadj[it] = a;
    }
    const size_t fsmem = smem_bytes(L, Lp, N, Wcap, tb, nwin, false);
    auto set_state = [&](long long seg) {
        cudaError_t e = cudaMemcpyAsync(stL, ckL + (size_t)seg * B * 3 * Lp, sizeof(uint32_t) * B * 3 * Lp,
                                        cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stE, ckE + (size_t)seg * B * 3, sizeof(int32_t) * B * 3, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(stF, ckF + (size_t)seg * B * 3, sizeof(int32_t) * B * 3, cudaMemcpyDeviceToDevice, st);
        return e;
    };
    auto run_forward = [&](long long n, bool hist) {
        const std::vector<KArgs> h = forward_args(n, hist);
        cudaError_t e = cudaMemcpyAsync(fargs, h.data(), sizeof(KArgs) * B, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_batch(fargs, B, fsmem, st);
        // the host vector must outlive the copy
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        return e;
    };
    auto check_status = [&]() -> int {
        int hs = 0;
        cudaError_t e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_failf(e, "reverse-sweep launch");
        return hs ? status_error(hs) : MPT_OK;
    };
    // 1. forward in segments, a checkpoint after each
    for (long long seg = 0; seg < nseg; seg++) {
        const long long n = std::min<long long>(every, nsteps - seg * every);
        ce = set_state(seg);
        if (ce == cudaSuccess) ce = run_forward(n, false);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(ckL + (size_t)(seg + 1) * B * 3 * Lp, stL, sizeof(uint32_t) * B * 3 * Lp,
                                 cudaMemcpyDeviceToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(ckE + (size_t)(seg + 1) * B * 3, stE, sizeof(int32_t) * B * 3,
                                 cudaMemcpyDeviceToDevice, st);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(ckF + (size_t)(seg + 1) * B * 3, stF, sizeof(int32_t) * B * 3,
                                 cudaMemcpyDeviceToDevice, st);
        if (ce != cudaSuccess) return cuda_failf(ce, "forward segment");
        int rc = check_status();
        if (rc) return rc;
    }
    // 2. last segment first: recompute with the coefficient history, then sweep
    for (long long seg = nseg - 1; seg >= 0; seg--) {
        const long long n = std::min<long long>(every, nsteps - seg * every);
        ce = set_state(seg);
        if (ce == cudaSuccess) ce = run_forward(n, true);
        if (ce != cudaSuccess) return cuda_failf(ce, "segment recomputation");
        for (int it = 0; it < items; it++) hadj[it].nsteps = n;
        ce = cudaMemcpyAsync(aargs, hadj.data(), sizeof(KArgs) * items, cudaMemcpyHostToDevice, st);
        if (ce == cudaSuccess) ce = launch_batch(aargs, items, smem, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) return cuda_failf(ce, "reverse sweep");
        int rc = check_status();
        if (rc) return rc;
    }
    // gbar (now the adjoint of the initial state) and the parameter adjoints
    ce = cudaMemcpyAsync(hapar.data(), aparL, sizeof(uint32_t) * hapar.size(), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(haparE.data(), aparE, sizeof(int32_t) * haparE.size(), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(haparF.data(), aparF, sizeof(int32_t) * haparF.size(), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_failf(ce, "reverse-sweep results");
    for (int it = 0; it < items; it++)
        for (int k = 0; k < 3; k++) {
            const size_t r = (size_t)it * ADJ_NPAR;
            from_dev(L, &hapar[(r + ADJ_GBAR + k) * Lp], haparE[r + ADJ_GBAR + k], haparF[r + ADJ_GBAR + k],
                     &g_signs[it * 3 + k], &g_exps[it * 3 + k], &g_limbs[((size_t)it * 3 + k) * L]);
            from_dev(L, &hapar[(r + ADJ_THBAR + k) * Lp], haparE[r + ADJ_THBAR + k], haparF[r + ADJ_THBAR + k],
                     &th_signs[it * 3 + k], &th_exps[it * 3 + k], &th_limbs[((size_t)it * 3 + k) * L]);
        }
    return MPT_OK;
}

}  // namespace

extern "C" int mpt_backward_raw(int B, int G, int L, int N, int64_t nsteps, int checkpoint_every,
                                const int32_t *par_signs, const int32_t *par_exps,
                                const uint32_t *par_limbs, const int32_t *st_signs,
                                const int32_t *st_exps, const uint32_t *st_limbs, int32_t *g_signs,
                                int32_t *g_exps, uint32_t *g_limbs, int32_t *th_signs,
                                int32_t *th_exps, uint32_t *th_limbs, uint64_t cuda_stream)
{
    return backward_impl(B, G, L, N, nsteps, checkpoint_every, par_signs, par_exps, par_limbs, st_signs,
                         st_exps, st_limbs, g_signs, g_exps, g_limbs, th_signs, th_exps, th_limbs,
                         cuda_stream, TauRatio{});
}

extern "C" int mpt_backward(int B, int L, int N, int64_t nsteps, const char *tau, const char *sigma,
                            const char *R, const char *b, const char *const *x0, const double *g,
                            int checkpoint_every, double *g_x0, double *g_params, double *jac,
                            uint64_t cuda_stream)
{
    if (B < 1) return failf(MPT_EINVAL, "batch size %d < 1", B);
    if (!tau || !sigma || !R || !b || !x0 || !g || !g_x0 || !g_params)
        return failf(MPT_EINVAL, "null argument");
    if (L < 1 || L > MAX_L) return failf(MPT_EINVAL, "L = %d outside 1..%d", L, MAX_L);
    const char *ps[4] = {sigma, R, b, tau};
    const char *pname[4] = {"sigma", "R", "b", "tau"};
    std::vector<int32_t> pS(4), pE(4), sS((size_t)3 * B), sE((size_t)3 * B);
    std::vector<uint32_t> pLm((size_t)4 * L), sLm((size_t)3 * B * L);
    for (int p = 0; p < 4; p++) {
        const int rc = mpt_host::parse_number(ps[p], L, &pS[p], &pE[p], &pLm[(size_t)p * L]);
        if (rc) return failf(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use %s = \"%s\"", pname[p], ps[p]);
    }
    for (int k = 0; k < 3 * B; k++) {
        if (!x0[k]) return failf(MPT_EINVAL, "initial value %d is null", k);
        const int rc = mpt_host::parse_number(x0[k], L, &sS[k], &sE[k], &sLm[(size_t)k * L]);
        if (rc) return failf(rc == -3 ? MPT_ERANGE : MPT_EINVAL, "cannot use initial value \"%s\"", x0[k]);
    }
    // jac: one sweep per output component (gbar = e_x, e_y, e_z); else one from g
    const int G = jac ? 3 : 1, items = B * G;
    std::vector<int32_t> gS((size_t)3 * items), gE((size_t)3 * items), tS((size_t)3 * items), tE((size_t)3 * items);
    std::vector<uint32_t> gLm((size_t)3 * items * L), tLm((size_t)3 * items * L);
    for (int it = 0; it < items; it++)
        for (int k = 0; k < 3; k++) {
            const double v = jac ? (it % 3 == k ? 1.0 : 0.0) : g[3 * it + k];
            if (mpt_host::from_double(v, L, &gS[3 * it + k], &gE[3 * it + k], &gLm[((size_t)3 * it + k) * L]))
                return failf(MPT_EINVAL, "g[%d] is not finite", 3 * it + k);
        }
    TauRatio tr;
    if (mpt_host::small_ratio(tau, L, &tr.p, &tr.q, &tr.r, &tr.shift, &tr.neg)) tr = TauRatio{};
    const int rc = backward_impl(B, G, L, N, nsteps, checkpoint_every, pS.data(), pE.data(), pLm.data(),
                                 sS.data(), sE.data(), sLm.data(), gS.data(), gE.data(), gLm.data(), tS.data(),
                                 tE.data(), tLm.data(), cuda_stream, tr);
    if (rc) return rc;
    auto dbl = [&](const std::vector<int32_t> &s, const std::vector<int32_t> &e, const std::vector<uint32_t> &l,
                   size_t k) { return mpt_host::to_double(L, s[k], e[k], &l[k * L]); };
    for (int p = 0; p < 3; p++) g_params[p] = 0.0;
    for (int j = 0; j < B; j++) {
        if (jac) {
            // rows: output component o; columns x0, y0, z0, sigma, R, b
            for (int o = 0; o < 3; o++)
                for (int i = 0; i < 6; i++) {
                    const size_t k = (size_t)3 * (3 * j + o) + (i % 3);
                    jac[((size_t)j * 3 + o) * 6 + i] = i < 3 ? dbl(gS, gE, gLm, k) : dbl(tS, tE, tLm, k);
                }
            for (int i = 0; i < 6; i++) {
                double v = 0.0;
                for (int o = 0; o < 3; o++) v += g[3 * j + o] * jac[((size_t)j * 3 + o) * 6 + i];
                if (i < 3) g_x0[3 * j + i] = v;
                else g_params[i - 3] += v;
            }
        } else {
            for (int i = 0; i < 3; i++) {
                g_x0[3 * j + i] = dbl(gS, gE, gLm, (size_t)3 * j + i);
                g_params[i] += dbl(tS, tE, tLm, (size_t)3 * j + i);
            }
        }
    }
    return MPT_OK;
}
