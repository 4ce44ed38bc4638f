// Host-side check of the invariant-divisor division used by the device code:
// for every d in [1, 2^16) and a set of numerators, div_inv and divstep must
// agree with the plain integer quotient and remainder, and make_divisor16 must
// give make_divisor's multiplier and shifts.
#include <cstdio>
#include <cstdint>
#include "../../paper_1908_09301_gb300/csrc/mpt_common.cuh"

int main()
{
    uint64_t state = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        state ^= state << 13;
        state ^= state >> 7;
        state ^= state << 17;
        return (uint32_t)state;
    };
    long long checks = 0;
    for (uint32_t d = 1; d < 65536u; d++) {
        mpt::Divisor v = mpt::make_divisor(d);
        const mpt::Divisor w = mpt::make_divisor16(d);
        if (w.d != v.d || w.m != v.m || w.s1 != v.s1 || w.s2 != v.s2) {
            printf("FAIL make_divisor16 d=%u\n", d);
            return 1;
        }
        uint32_t ns[12] = {0u, 1u, d - 1u, d, d + 1u, 0xffffffffu, 0xfffffffeu, 0x80000000u,
                           0x7fffffffu, (uint32_t)(d * 65535u), next(), next()};
        for (uint32_t n : ns) {
            if (mpt::div_inv(n, v) != n / d || mpt::mod_inv(n, v) != n % d) {
                printf("FAIL div d=%u n=%u\n", d, n);
                return 1;
            }
            checks++;
        }
        for (int k = 0; k < 4; k++) {
            uint32_t r = next() % d, x = next();
            uint32_t r0 = r;
            uint64_t num = ((uint64_t)r0 << 32) | x;
            uint32_t q = mpt::divstep(r, x, v);
            if (q != (uint32_t)(num / d) || r != (uint32_t)(num % d)) {
                printf("FAIL divstep d=%u r=%u x=%u\n", d, r0, x);
                return 1;
            }
            checks++;
        }
    }
    printf("OK %lld\n", checks);
    return 0;
}
