// host_parse.h -- exact decimal / rational string -> L-limb number (host).
#pragma once
#include <cstdint>

namespace mpt_host {
// trunc_L of the exact value of `str` (decimal such as "-15.8", "1e-20", or a
// rational "p/q" of two decimals).  Returns 0, -1 for a malformed string or a
// zero denominator, -3 for an exponent outside |exp| <= 2^30.
int parse_number(const char *str, int L, int32_t *sign, int32_t *exp, uint32_t *limbs);
}  // namespace mpt_host
