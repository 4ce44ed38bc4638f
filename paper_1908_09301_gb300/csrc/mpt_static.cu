// mpt_static.cu -- mpt_integrate_noalloc: Taylor steps for callers that must
// not allocate device memory.
//
// Some host programs cannot call cudaMalloc at the point where they step the
// integrator: a caller whose memory is owned by a pool it may not grow, a
// plugin inside a runtime that forbids allocation after start-up, or code
// that must not synchronise with the allocator.  For them this file keeps all
// working memory of the lock-step Taylor kernel -- the coefficient table, the
// padded parameter and state copies, the cross-CTA accumulator windows, the
// grid-barrier words and the status word -- in one file-scope device array
// of fixed size.  The caller passes only its inputs and outputs.
//
// The array is a `static __device__` symbol.  Host code cannot use its name
// as an address (on the host the name denotes a host-side stand-in), so at
// set-up, once per device and with that device current, the device address
// is taken with cudaGetSymbolAddress and handed to the kernels as a plain
// pointer.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/mpt.h"
#include "mpt_kernel.cuh"

namespace mpt {
int record_error(int code, const char *msg);  // sets mpt_last_error() (mpt_host.cu)
}

namespace {

using namespace mpt;

constexpr size_t SCRATCH_BYTES = MPT_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;

// The working memory of every mpt_integrate_noalloc call on a device.  It is
// held by each GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// status codes of the input check (the kernel's own codes are 1..3)
constexpr int BAD_NUMBER = 0x100;  // + index: malformed number (zero form, sign, top limb)
constexpr int BAD_EXP = 0x200;     // + index: |exp| > 2^30

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_scratch
    int sms = 0;
    int smem_optin = 0;
};

std::mutex g_setup_lock;
DeviceSetup g_setup[MAX_DEVICES];

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

// Offsets of the kernel's buffers inside the scratch array, each on a
// 256-byte boundary.
struct Layout {
    int L, Lp, P, N, Wcap;
    size_t coefL, coefE, coefF, parL, parE, parF, stL, stE, stF, gwin, bar, status, total;

    Layout(int L_, int N_) : L(L_), N(N_)
    {
        Lp = (L + W - 1) / W * W;
        P = Lp / W;
        const int spread = Lp > 64 ? Lp : 64;
        Wcap = (2 * Lp + 2 + spread + 31) / 32 * 32;
        const size_t N1 = (size_t)N + 1;
        size_t o = 0;
        auto take = [&o](size_t bytes) {
            size_t at = o;
            o = (o + bytes + 255) / 256 * 256;
            return at;
        };
        coefL = take(sizeof(uint32_t) * 3 * N1 * Lp);
        coefE = take(sizeof(int32_t) * 3 * N1);
        coefF = take(sizeof(int32_t) * 3 * N1);
        parL = take(sizeof(uint32_t) * 4 * Lp);
        parE = take(sizeof(int32_t) * 4);
        parF = take(sizeof(int32_t) * 4);
        stL = take(sizeof(uint32_t) * 3 * Lp);
        stE = take(sizeof(int32_t) * 3);
        stF = take(sizeof(int32_t) * 3);
        gwin = take(sizeof(long long) * 9 * Wcap);
        bar = take(sizeof(unsigned) * 2);
        status = take(sizeof(int));
        total = o;
    }
};

// Interchange layout -> the kernel's layout (Lp limbs, flags), with the
// checks the context path makes on the host.  Block j < 4 converts parameter
// j (sigma, R, b, tau), block 4 + j state component j.
__global__ void pack_inputs(int L, int Lp, const int32_t *ps, const int32_t *pe, const uint32_t *pl,
                            const int32_t *ss, const int32_t *se, const uint32_t *sl,
                            uint32_t *parL, int32_t *parE, int32_t *parF, uint32_t *stL,
                            int32_t *stE, int32_t *stF, int *status)
{
    const int j = blockIdx.x;
    const bool is_par = j < 4;
    const int k = is_par ? j : j - 4;
    const int32_t s = is_par ? ps[k] : ss[k];
    const int32_t e = is_par ? pe[k] : se[k];
    const uint32_t *src = (is_par ? pl : sl) + (size_t)k * L;
    uint32_t *dst = (is_par ? parL : stL) + (size_t)k * Lp;
    int nz = 0;
    for (int x = threadIdx.x; x < Lp; x += blockDim.x) {
        const uint32_t v = x < L ? src[x] : 0u;
        dst[x] = v;
        nz |= v != 0u;
    }
    nz = __syncthreads_or(nz);
    if (threadIdx.x != 0) return;
    int code = 0, flags = 0, exp = 0;
    if (!nz) {
        if (s != 0 || e != 0) code = BAD_NUMBER + j;
    } else if ((s != 0 && s != 1) || src[L - 1] == 0u) {
        code = BAD_NUMBER + j;
    } else if (e > (1 << 30) || e < -(1 << 30)) {
        code = BAD_EXP + j;
    } else {
        flags = F_NZ | (s ? F_NEG : 0);
        exp = e;
    }
    if (code) atomicCAS(status, 0, code);
    (is_par ? parE : stE)[k] = exp;
    (is_par ? parF : stF)[k] = flags;
}

// The kernel's state -> the caller's output, only when every step succeeded.
__global__ void unpack_state(int L, int Lp, const uint32_t *stL, const int32_t *stE,
                             const int32_t *stF, const int *status, int32_t *ss, int32_t *se,
                             uint32_t *sl)
{
    if (*(volatile const int *)status != 0) return;
    const int k = blockIdx.x;
    for (int x = threadIdx.x; x < L; x += blockDim.x)
        sl[(size_t)k * L + x] = stL[(size_t)k * Lp + x];
    if (threadIdx.x == 0) {
        ss[k] = (stF[k] & F_NEG) ? 1 : 0;
        se[k] = stE[k];
    }
}

// the current device's set-up (made on first use) and its index
int device_setup(DeviceSetup **out, int *dev_out)
{
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_failf(ce, "current device");
    if (dev < 0 || dev >= MAX_DEVICES)
        return failf(MPT_EINVAL, "device %d: at most %d devices are supported", dev, MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_setup_lock);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *p = nullptr;
        ce = cudaGetSymbolAddress(&p, g_scratch);
        if (ce != cudaSuccess) return cuda_failf(ce, "address of the static scratch array");
        ce = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (ce == cudaSuccess)
            ce = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (ce != cudaSuccess) return cuda_failf(ce, "device query");
        d.scratch = (unsigned char *)p;
        d.ready = true;
    }
    *out = &d;
    *dev_out = dev;
    return MPT_OK;
}

// A pointer the kernels can dereference: device, managed or registered host memory.
int check_pointer(const void *p, const char *name, int dev)
{
    if (!p) return failf(MPT_EINVAL, "%s is null", name);
    cudaPointerAttributes at;
    cudaError_t ce = cudaPointerGetAttributes(&at, p);
    if (ce != cudaSuccess) return cuda_failf(ce, name);
    if (at.type == cudaMemoryTypeUnregistered)
        return failf(MPT_EINVAL, "%s is not device-accessible memory", name);
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return failf(MPT_EINVAL, "%s lives on device %d, the current device is %d", name, at.device, dev);
    return MPT_OK;
}

int read_status(cudaStream_t st, const int *dstatus, int *out)
{
    cudaError_t ce = cudaMemcpyAsync(out, dstatus, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return cuda_failf(ce, "kernel execution");
    return MPT_OK;
}

const char *number_name(int j)
{
    static const char *names[7] = {"sigma", "R", "b", "tau", "x", "y", "z"};
    return (j >= 0 && j < 7) ? names[j] : "?";
}

}  // namespace

extern "C" int mpt_integrate_noalloc(int L, int N, int64_t nsteps, const int32_t *par_signs,
                                     const int32_t *par_exps, const uint32_t *par_limbs,
                                     int32_t *signs, int32_t *exps, uint32_t *limbs,
                                     uint64_t cuda_stream)
{
    if (L < 1 || L > MAX_L) return failf(MPT_EINVAL, "L = %d outside 1..%d", L, MAX_L);
    if (N < 1 || N > MAX_N) return failf(MPT_EINVAL, "N = %d outside 1..%d", N, MAX_N);
    if (nsteps < 0) return failf(MPT_EINVAL, "nsteps = %lld is negative", (long long)nsteps);
    const Layout lay(L, N);
    if (lay.total > SCRATCH_BYTES)
        return failf(MPT_EINVAL,
                     "L = %d, N = %d need %zu bytes of scratch; the static scratch array holds %zu",
                     L, N, lay.total, SCRATCH_BYTES);
    DeviceSetup *d = nullptr;
    int dev = 0;
    int rc = device_setup(&d, &dev);
    if (rc) return rc;
    const void *ptrs[6] = {par_signs, par_exps, par_limbs, signs, exps, limbs};
    const char *names[6] = {"par_signs", "par_exps", "par_limbs", "signs", "exps", "limbs"};
    for (int i = 0; i < 6; i++)
        if ((rc = check_pointer(ptrs[i], names[i], dev))) return rc;
    if (nsteps == 0) return MPT_OK;

    // shared memory and grid as the context path chooses them for the lock-step kernel
    int tb = 64;
    while (tb > 8 && smem_bytes(L, lay.Lp, N, lay.Wcap, tb) > (size_t)d->smem_optin) tb /= 2;
    const size_t smem = smem_bytes(L, lay.Lp, N, lay.Wcap, tb);
    if (smem > (size_t)d->smem_optin)
        return failf(MPT_EINVAL, "L = %d, N = %d need %zu bytes of shared memory (device has %d)", L,
                     N, smem, d->smem_optin);
    const int max_grid = max_coresident_ctas(smem);
    if (max_grid < 1) return failf(MPT_ECUDA, "kernel does not fit on the device");
    int grid = (int)std::lround((double)N * lay.Lp * lay.Lp / 50000.0);
    if (grid < 1) grid = 1;
    if (grid > d->sms) grid = d->sms;
    if (grid > max_grid) grid = max_grid;

    unsigned char *s = d->scratch;
    cudaStream_t st = (cudaStream_t)(uintptr_t)cuda_stream;
    KArgs a{};  // value-initialised: vG = 0 (the launch's own grid)
    a.L = L;
    a.Lp = lay.Lp;
    a.P = lay.P;
    a.N = N;
    a.Wcap = lay.Wcap;
    a.tb = tb;
    a.coefL = (uint32_t *)(s + lay.coefL);
    a.coefE = (int32_t *)(s + lay.coefE);
    a.coefF = (int32_t *)(s + lay.coefF);
    a.parL = (const uint32_t *)(s + lay.parL);
    a.parE = (const int32_t *)(s + lay.parE);
    a.parF = (const int32_t *)(s + lay.parF);
    a.stL = (uint32_t *)(s + lay.stL);
    a.stE = (int32_t *)(s + lay.stE);
    a.stF = (int32_t *)(s + lay.stF);
    a.gwin = (long long *)(s + lay.gwin);
    a.bar = (unsigned *)(s + lay.bar);
    a.status = (int *)(s + lay.status);
    a.recS = nullptr;
    a.recE = nullptr;
    a.recL = nullptr;
    a.nsteps = nsteps;
    a.record_every = 0;
    a.prof = nullptr;
    a.spin_limit = DEFAULT_SPIN_LIMIT;

    // The array keeps whatever the previous call left: the accumulator
    // windows, the barrier words and the status must start at zero.  The
    // coefficient table and the copies of the inputs are written before they
    // are read.
    cudaError_t ce = cudaMemsetAsync(a.status, 0, sizeof(int), st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a.bar, 0, sizeof(unsigned) * 2, st);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(a.gwin, 0, sizeof(long long) * 9 * lay.Wcap, st);
    if (ce != cudaSuccess) return cuda_failf(ce, "clearing the scratch array");

    pack_inputs<<<7, 128, 0, st>>>(L, lay.Lp, par_signs, par_exps, par_limbs, signs, exps, limbs,
                                   (uint32_t *)a.parL, (int32_t *)a.parE, (int32_t *)a.parF, a.stL,
                                   a.stE, a.stF, a.status);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_failf(ce, "input conversion launch");
    int status = 0;
    if ((rc = read_status(st, a.status, &status))) return rc;
    if (status >= BAD_EXP)
        return failf(MPT_ERANGE, "%s: exponent out of range", number_name(status - BAD_EXP));
    if (status >= BAD_NUMBER)
        return failf(MPT_EINVAL, "%s: malformed number (zero must be sign 0, exp 0; sign 0 or 1; "
                     "top limb non-zero)", number_name(status - BAD_NUMBER));

    ce = launch_integrate(a, grid, smem, st);
    if (ce != cudaSuccess) return cuda_failf(ce, "kernel launch");
    unpack_state<<<3, 128, 0, st>>>(L, lay.Lp, a.stL, a.stE, a.stF, a.status, signs, exps, limbs);
    ce = cudaGetLastError();
    if (ce != cudaSuccess) return cuda_failf(ce, "state conversion launch");
    if ((rc = read_status(st, a.status, &status))) return rc;
    if (status == DEV_ERANGE)
        return failf(MPT_ERANGE, "exponent out of range, or an exact sum spans more than %d limbs",
                     lay.Wcap);
    if (status == DEV_TIMEOUT) return failf(MPT_ETIMEDOUT, "a grid barrier wait expired");
    if (status != 0) return failf(MPT_ECUDA, "device invariant failed (status %d)", status);
    return MPT_OK;
}
