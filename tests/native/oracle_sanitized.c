/* The oracle under AddressSanitizer and UndefinedBehaviorSanitizer: reads
 * L, N, nsteps, the parameters (sigma, R, b, tau) and the state (x, y, z) as
 * interchange numbers (sign exp limb_0 .. limb_{L-1}) from stdin, runs
 * orc_coefficients and orc_integrate, and prints the final state and a
 * checksum of the coefficients in the same form.  Built and run by
 * tests/test_oracle_sanitized.py. */
#include "../../oracle/mpt_oracle.c"

#include <stdio.h>

static int read_numbers(int n, int L, int32_t *s, int32_t *e, uint32_t *l)
{
    for (int j = 0; j < n; j++) {
        if (scanf("%d %d", &s[j], &e[j]) != 2) return 0;
        for (int x = 0; x < L; x++)
            if (scanf("%u", &l[(size_t)j * L + x]) != 1) return 0;
    }
    return 1;
}

int main(void)
{
    int L, N;
    long long nsteps;
    if (scanf("%d %d %lld", &L, &N, &nsteps) != 3 || L < 1 || N < 1 || nsteps < 0) return 2;
    int32_t ps[4], pe[4], ss[3], se[3];
    uint32_t *pl = malloc((size_t)4 * L * sizeof(uint32_t));
    uint32_t *sl = malloc((size_t)3 * L * sizeof(uint32_t));
    size_t nc = (size_t)3 * (N + 1);
    int32_t *cs = malloc(nc * sizeof(int32_t)), *ce = malloc(nc * sizeof(int32_t));
    uint32_t *cl = malloc(nc * L * sizeof(uint32_t));
    if (!pl || !sl || !cs || !ce || !cl) return 3;
    if (!read_numbers(4, L, ps, pe, pl) || !read_numbers(3, L, ss, se, sl)) return 2;
    int rc = orc_coefficients(L, N, ps, pe, pl, ss, se, sl, cs, ce, cl, 1);
    unsigned long long sum = 0;
    for (size_t j = 0; j < nc; j++) {
        sum = sum * 1000003ull + (unsigned)cs[j] * 7ull + (unsigned)ce[j];
        for (int x = 0; x < L; x++) sum = sum * 1000003ull + cl[j * L + x];
    }
    if (rc == 0) rc = orc_integrate(L, N, nsteps, ps, pe, pl, ss, se, sl, 0, NULL, NULL, NULL, 1);
    printf("%d %llu\n", rc, sum);
    for (int j = 0; j < 3; j++) {
        printf("%d %d", ss[j], se[j]);
        for (int x = 0; x < L; x++) printf(" %u", sl[(size_t)j * L + x]);
        printf("\n");
    }
    free(pl);
    free(sl);
    free(cs);
    free(ce);
    free(cl);
    return 0;
}
