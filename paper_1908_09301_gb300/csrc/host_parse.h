// host_parse.h -- exact decimal / rational string -> L-limb number (host).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mpt_host {
// trunc_L of the exact value of `str` (decimal such as "-15.8", "1e-20", or a
// rational "p/q" of two decimals).  Returns 0, -1 for a malformed string or a
// zero denominator, -3 for an exponent outside |exp| <= 2^30.
int parse_number(const char *str, int L, int32_t *sign, int32_t *exp, uint32_t *limbs);
// the exact x + sgn 10^(-h_digits) as "p/q"; 0, or -1 for a malformed x
int perturbed_string(const char *x, int h_digits, int sgn, std::string &out);
// (v1 - v2) / (2 10^(-h_digits)) of two L-limb interchange numbers, rounded
// once to the nearest double
double diff_over_2h(int L, int32_t s1, int32_t e1, const uint32_t *l1, int32_t s2, int32_t e2,
                    const uint32_t *l2, int h_digits);
// the L-limb interchange number rounded once to the nearest double (ties to even)
double to_double(int L, int32_t s, int32_t e, const uint32_t *l);
// trunc_L of the exact value of a finite double; 0, or -1 for inf / nan
int from_double(double v, int L, int32_t *sign, int32_t *exp, uint32_t *limbs);
// tau = trunc_L(p/q) with p/q in lowest terms, 0 < p < 2^32, 1 <= q < 2^16:
// then its limbs are M = (p 2^k - r) / q, k = 32 shift, r = p 2^k mod q, and
// tau h = (p h - r h 2^-k) / q exactly.  0 with (p, q, r, shift, neg), else -1.
int small_ratio(const char *str, int L, uint32_t *p, uint32_t *q, uint32_t *r, int *shift, int *neg);
// The division table of the pipelined kernel's closes: rows d = 0..N (row 0
// for q0, or 1 when q0 = 0), rl entries a row; with d' the odd part of d,
// entry i holds 2^(-32 i) mod d' in its low 16 bits and 2^(32 (i-1)) mod d'
// (0 for i = 0) in its high 16 bits.  Every entry is 0 where d' = 1.
std::vector<uint32_t> division_table(int N, int rl, uint32_t q0);
}  // namespace mpt_host
