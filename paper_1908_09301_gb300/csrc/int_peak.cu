// int_peak.cu -- INT32 multiply-add throughput microbenchmark.
//
// The Taylor step's hot loop is made of 32x32->64-bit limb products added into
// exact column sums (Eq. (3)'s Cauchy sums over multiple-precision numbers).
// Its roofline is the SM's integer multiply-add rate, which no vendor table
// states for this chip with certainty, so it is measured here: each variant
// runs register-resident chains of one instruction form and reports how many
// results (or limb products) one SM retires per clock.
//
// Variants (all operands in registers, 8 independent chains per thread):
//   0  mad.lo.u32                          one 32-bit multiply-add per result
//   1  mad.hi.u32                          high half of a 32x32 product
//   2  mad.wide.u32                        full 64-bit product plus 64-bit addend
//   3  limb product, carry chain:          mad.lo.cc / madc.hi.cc / addc (96-bit column)
//   4  limb product, two wide half-limbs:  2x mad.wide.u32 with a 16-bit operand
//   5  limb product, wide + low word:      t = a*b + c0 (wide), c12 += t.hi (wide by 1)
//   6  limb product, lo/hi separately:     mad.lo.cc+addc, mad.hi.cc+addc
//   7  mad.lo.u32 + mad.hi.u32 pair, no carries (two 32-bit column sums)
//   8  limb product, wide + carry adds:    mul.wide, add.cc/addc.cc/addc
//   9  limb products of a row, carries along the row: one limb a times 8
//      limbs b_j into columns 0..8, low halves in one mad.lo.cc/madc.lo.cc
//      chain over columns 0..7 and high halves in one mad.hi.cc/madc.hi.cc
//      chain over columns 1..8, each chain's carry out into a counter word
//      (8 products, 16 multiply-adds, 2 addc)
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int W = 8;  // independent chains per thread

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint32_t mad_hi(uint32_t a, uint32_t b, uint32_t c)
{
    uint32_t d;
    asm volatile("mad.hi.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ uint64_t mad_wide(uint32_t a, uint32_t b, uint64_t c)
{
    uint64_t d;
    asm volatile("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// one limb product into a 96-bit column accumulator with the carry flag
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

__device__ __forceinline__ void mac_wide_add(uint32_t a, uint32_t b, uint32_t &c0, uint32_t &c1,
                                             uint32_t &c2)
{
    asm volatile(
        "{.reg .u64 t; .reg .u32 tl, th;\n\t"
        "mul.wide.u32 t, %3, %4;\n\t"
        "mov.b64 {tl, th}, t;\n\t"
        "add.cc.u32 %0, %0, tl;\n\t"
        "addc.cc.u32 %1, %1, th;\n\t"
        "addc.u32 %2, %2, 0;}"
        : "+r"(c0), "+r"(c1), "+r"(c2)
        : "r"(a), "r"(b));
}

__device__ __forceinline__ void mac_lohi(uint32_t a, uint32_t b, uint32_t &l0, uint32_t &l1,
                                         uint32_t &h0, uint32_t &h1)
{
    asm volatile(
        "mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
        "addc.u32 %1, %1, 0;\n\t"
        "mad.hi.cc.u32 %2, %4, %5, %2;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(l0), "+r"(l1), "+r"(h0), "+r"(h1)
        : "r"(a), "r"(b));
}

// a times the row b[0..7] added into the columns acc[0..8] with carries along
// the row; the low chain's carry out goes to k[0], the high chain's to k[1]
__device__ __forceinline__ void mac_row(uint32_t a, const uint32_t (&b)[W], uint32_t (&acc)[W + 1],
                                        uint32_t (&k)[2])
{
    asm volatile(
        "mad.lo.cc.u32  %0, %11, %12, %0;\n\t"
        "madc.lo.cc.u32 %1, %11, %13, %1;\n\t"
        "madc.lo.cc.u32 %2, %11, %14, %2;\n\t"
        "madc.lo.cc.u32 %3, %11, %15, %3;\n\t"
        "madc.lo.cc.u32 %4, %11, %16, %4;\n\t"
        "madc.lo.cc.u32 %5, %11, %17, %5;\n\t"
        "madc.lo.cc.u32 %6, %11, %18, %6;\n\t"
        "madc.lo.cc.u32 %7, %11, %19, %7;\n\t"
        "addc.u32       %9, %9, 0;\n\t"
        "mad.hi.cc.u32  %1, %11, %12, %1;\n\t"
        "madc.hi.cc.u32 %2, %11, %13, %2;\n\t"
        "madc.hi.cc.u32 %3, %11, %14, %3;\n\t"
        "madc.hi.cc.u32 %4, %11, %15, %4;\n\t"
        "madc.hi.cc.u32 %5, %11, %16, %5;\n\t"
        "madc.hi.cc.u32 %6, %11, %17, %6;\n\t"
        "madc.hi.cc.u32 %7, %11, %18, %7;\n\t"
        "madc.hi.cc.u32 %8, %11, %19, %8;\n\t"
        "addc.u32       %10, %10, 0;"
        : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2]), "+r"(acc[3]), "+r"(acc[4]), "+r"(acc[5]),
          "+r"(acc[6]), "+r"(acc[7]), "+r"(acc[8]), "+r"(k[0]), "+r"(k[1])
        : "r"(a), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]),
          "r"(b[7]));
}

template <int V>
__global__ void __launch_bounds__(1024) peak_kernel(int iters, uint32_t seed, uint64_t *sink,
                                                       long long *cycles, int *smid)
{
    uint32_t a = seed ^ (threadIdx.x * 2654435761u);
    uint32_t b[W];
#pragma unroll
    for (int k = 0; k < W; k++) b[k] = a * (2 * k + 1) + k;
    uint32_t c0[W], c1[W], c2[W];
    uint64_t w0[W], w1[W];
#pragma unroll
    for (int k = 0; k < W; k++) {
        c0[k] = c1[k] = c2[k] = 0;
        w0[k] = w1[k] = 0;
    }
    uint32_t acc[W + 1], kc[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k <= W; k++) acc[k] = 0;
    __syncthreads();
    long long t0 = clock64();
    for (int it = 0; it < iters; it++) {
        if (V == 9) mac_row(a, b, acc, kc);  // W limb products a round, as the chains below
#pragma unroll
        for (int k = 0; k < W; k++) {
            if (V == 0) c0[k] = mad_lo(c0[k], b[k], a);
            if (V == 1) c0[k] = mad_hi(c0[k] | 1u, b[k], a);
            if (V == 2) w0[k] = mad_wide((uint32_t)w0[k] | b[k], a, w0[k]);
            if (V == 3) mac_cc(a, b[k], c0[k], c1[k], c2[k]);
            if (V == 4) {
                w0[k] = mad_wide(a, b[k] & 0xFFFFu, w0[k]);
                w1[k] = mad_wide(a, b[k] >> 16, w1[k]);
            }
            if (V == 5) {
                uint64_t t = mad_wide(a, b[k], (uint64_t)c0[k]);
                c0[k] = (uint32_t)t;
                w1[k] = mad_wide((uint32_t)(t >> 32), 1u, w1[k]);
            }
            if (V == 6) mac_lohi(a, b[k], c0[k], c1[k], c2[k], b[k]);
            if (V == 7) {
                c0[k] = mad_lo(a, b[k], c0[k]);
                c1[k] = mad_hi(a, b[k], c1[k]);
            }
            if (V == 8) mac_wide_add(a, b[k], c0[k], c1[k], c2[k]);
        }
        // the broadcast operand changes every round, as a_i does in the real loop
        a = a * 0x9E3779B1u + (uint32_t)it;
    }
    long long t1 = clock64();
    uint64_t s = 0;
#pragma unroll
    for (int k = 0; k < W; k++) s += c0[k] + c1[k] + c2[k] + w0[k] + w1[k] + b[k] + acc[k];
    s += acc[W] + kc[0] + kc[1];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (threadIdx.x == 0) {
        cycles[blockIdx.x] = t1 - t0;
        uint32_t id;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
        smid[blockIdx.x] = (int)id;
    }
}

constexpr int MAX_THREADS = 1024;
int g_threads = MAX_THREADS;

template <int V>
void launch(int grid, int iters, uint64_t *sink, long long *cycles, int *smid, cudaStream_t st)
{
    peak_kernel<V><<<grid, g_threads, 0, st>>>(iters, 12345u, sink, cycles, smid);
}

}  // namespace

// Runs variant `variant` on one CTA of `threads` threads (a multiple of 32,
// at most 1024) per SM (grid = SM count) for `iters` rounds of 8 chains per
// thread.  Writes the mean loop cycles of a CTA to *mean_cycles, the kernel's
// wall time to *ms, and the number of distinct SMs the CTAs ran on to
// *distinct_sms.  Allocates and frees its own small buffers.  Returns 0, or
// the CUDA error code.
extern "C" int mpt_int_peak_run(int variant, int threads, int iters, double *mean_cycles,
                                double *ms, int *distinct_sms, int *grid_out)
{
    if (threads < 32 || threads > MAX_THREADS || threads % 32) return (int)cudaErrorInvalidValue;
    g_threads = threads;
    int dev = 0, grid = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&grid, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    *grid_out = grid;
    uint64_t *sink = nullptr;
    long long *cycles = nullptr;
    int *smid = nullptr;
    e = cudaMalloc(&sink, (size_t)grid * MAX_THREADS * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&cycles, (size_t)grid * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&smid, (size_t)grid * sizeof(int));
    cudaEvent_t a = nullptr, b = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
        cudaEventRecord(a, 0);
        switch (variant) {
            case 0: launch<0>(grid, iters, sink, cycles, smid, 0); break;
            case 1: launch<1>(grid, iters, sink, cycles, smid, 0); break;
            case 2: launch<2>(grid, iters, sink, cycles, smid, 0); break;
            case 3: launch<3>(grid, iters, sink, cycles, smid, 0); break;
            case 4: launch<4>(grid, iters, sink, cycles, smid, 0); break;
            case 5: launch<5>(grid, iters, sink, cycles, smid, 0); break;
            case 6: launch<6>(grid, iters, sink, cycles, smid, 0); break;
            case 7: launch<7>(grid, iters, sink, cycles, smid, 0); break;
            case 8: launch<8>(grid, iters, sink, cycles, smid, 0); break;
            case 9: launch<9>(grid, iters, sink, cycles, smid, 0); break;
            default: e = cudaErrorInvalidValue;
        }
        cudaEventRecord(b, 0);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
    }
    if (e == cudaSuccess) {
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        *ms = t;
        long long *h = new long long[grid];
        int *hs = new int[grid];
        e = cudaMemcpy(h, cycles, (size_t)grid * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(hs, smid, (size_t)grid * sizeof(int), cudaMemcpyDeviceToHost);
        double s = 0;
        for (int i = 0; i < grid; i++) s += (double)h[i];
        *mean_cycles = s / grid;
        int distinct = 0;
        for (int i = 0; i < grid; i++) {
            bool seen = false;
            for (int j = 0; j < i; j++) seen = seen || hs[j] == hs[i];
            distinct += !seen;
        }
        *distinct_sms = distinct;
        delete[] h;
        delete[] hs;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(sink);
    cudaFree(cycles);
    cudaFree(smid);
    return (int)e;
}
