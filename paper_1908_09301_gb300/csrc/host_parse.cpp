// host_parse.cpp -- exact parsing of decimal / rational strings into L-limb
// numbers (trunc_L of the exact value), on the host.
//
// The paper's constants (sigma = 10, R = 28, b = 8/3 after Eq. (1); tau = 0.01
// and x(0) = -15.8, y(0) = -17.48, z(0) = 35.64 in Sec. 5) are not all binary
// fractions, so each one enters the method as trunc_L of its exact rational
// value.  This file holds a small unsigned big integer with exactly the
// operations that needs: decimal digits in, shifts, comparison, subtraction
// and long division.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "host_parse.h"

namespace mpt_host {
namespace {

struct BigU {
    std::vector<uint32_t> w;  // little-endian limbs, no leading zeros

    void trim()
    {
        while (!w.empty() && w.back() == 0) w.pop_back();
    }
    bool zero() const { return w.empty(); }
    int bits() const
    {
        if (w.empty()) return 0;
        uint32_t t = w.back();
        int b = 0;
        while (t) {
            b++;
            t >>= 1;
        }
        return (int)(w.size() - 1) * 32 + b;
    }
    void mul_small(uint32_t m)
    {
        uint64_t c = 0;
        for (auto &x : w) {
            uint64_t t = (uint64_t)x * m + c;
            x = (uint32_t)t;
            c = t >> 32;
        }
        if (c) w.push_back((uint32_t)c);
    }
    void add_small(uint32_t a)
    {
        uint64_t c = a;
        for (size_t i = 0; i < w.size() && c; i++) {
            uint64_t t = (uint64_t)w[i] + c;
            w[i] = (uint32_t)t;
            c = t >> 32;
        }
        if (c) w.push_back((uint32_t)c);
    }
    void shl(int64_t s)  // s >= 0 bits
    {
        if (w.empty() || s == 0) return;
        size_t limbs = (size_t)(s / 32);
        int r = (int)(s % 32);
        std::vector<uint32_t> o(w.size() + limbs + 1, 0);
        for (size_t i = 0; i < w.size(); i++) {
            uint64_t v = (uint64_t)w[i] << r;
            o[i + limbs] |= (uint32_t)v;
            o[i + limbs + 1] |= (uint32_t)(v >> 32);
        }
        w.swap(o);
        trim();
    }
    int bit(int64_t i) const
    {
        size_t l = (size_t)(i / 32);
        if (l >= w.size()) return 0;
        return (w[l] >> (i % 32)) & 1;
    }
};

int cmp(const BigU &a, const BigU &b)
{
    if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
    for (size_t i = a.w.size(); i-- > 0;)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    return 0;
}

void sub_inplace(BigU &a, const BigU &b)  // a -= b, requires a >= b
{
    int64_t borrow = 0;
    for (size_t i = 0; i < a.w.size(); i++) {
        int64_t t = (int64_t)a.w[i] - (i < b.w.size() ? b.w[i] : 0) - borrow;
        borrow = t < 0;
        a.w[i] = (uint32_t)(t + (borrow ? ((int64_t)1 << 32) : 0));
    }
    a.trim();
}

// floor(a / b), b != 0: restoring binary long division
BigU divide(const BigU &a, const BigU &b)
{
    BigU q, r;
    int nb = a.bits();
    q.w.assign((size_t)nb / 32 + 1, 0);
    for (int i = nb - 1; i >= 0; i--) {
        r.shl(1);
        if (a.bit(i)) {
            if (r.w.empty()) r.w.push_back(0);
            r.w[0] |= 1;
        }
        if (cmp(r, b) >= 0) {
            sub_inplace(r, b);
            q.w[(size_t)i / 32] |= 1u << (i % 32);
        }
    }
    q.trim();
    return q;
}

BigU pow10(int e)
{
    BigU p;
    p.w.push_back(1);
    for (int i = 0; i < e; i++) p.mul_small(10);
    return p;
}

struct Rat {
    bool neg = false;
    BigU num, den;
};

const int kMaxDecimalExponent = 100000;

bool parse_decimal(const char *&s, Rat &out)
{
    while (*s == ' ' || *s == '\t') s++;
    bool neg = false;
    if (*s == '+' || *s == '-') {
        neg = *s == '-';
        s++;
    }
    BigU digits;
    int ndig = 0, frac = 0;
    bool seen_point = false;
    for (;; s++) {
        if (*s >= '0' && *s <= '9') {
            digits.mul_small(10);
            digits.add_small((uint32_t)(*s - '0'));
            digits.trim();
            ndig++;
            if (seen_point) frac++;
        } else if (*s == '.' && !seen_point) {
            seen_point = true;
        } else {
            break;
        }
    }
    if (ndig == 0) return false;
    long long e = 0;
    if (*s == 'e' || *s == 'E') {
        s++;
        bool eneg = false;
        if (*s == '+' || *s == '-') {
            eneg = *s == '-';
            s++;
        }
        int ed = 0;
        while (*s >= '0' && *s <= '9') {
            e = e * 10 + (*s - '0');
            if (e > kMaxDecimalExponent) return false;
            s++;
            ed++;
        }
        if (ed == 0) return false;
        if (eneg) e = -e;
    }
    long long scale = e - frac;
    if (scale > kMaxDecimalExponent || scale < -kMaxDecimalExponent) return false;
    out.neg = neg;
    out.num = digits;
    out.den.w.assign(1, 1);
    if (scale >= 0) {
        BigU p = pow10((int)scale);
        // num *= 10^scale
        BigU r;
        r.w.assign(out.num.w.size() + p.w.size() + 1, 0);
        for (size_t i = 0; i < out.num.w.size(); i++) {
            uint64_t c = 0;
            for (size_t j = 0; j < p.w.size(); j++) {
                uint64_t t = (uint64_t)out.num.w[i] * p.w[j] + r.w[i + j] + c;
                r.w[i + j] = (uint32_t)t;
                c = t >> 32;
            }
            r.w[i + p.w.size()] += (uint32_t)c;
        }
        r.trim();
        out.num = r;
    } else {
        out.den = pow10((int)-scale);
    }
    while (*s == ' ' || *s == '\t') s++;
    return true;
}

BigU mul(const BigU &a, const BigU &b)
{
    BigU r;
    if (a.zero() || b.zero()) return r;
    r.w.assign(a.w.size() + b.w.size(), 0);
    for (size_t i = 0; i < a.w.size(); i++) {
        uint64_t c = 0;
        for (size_t j = 0; j < b.w.size(); j++) {
            uint64_t t = (uint64_t)a.w[i] * b.w[j] + r.w[i + j] + c;
            r.w[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        r.w[i + b.w.size()] = (uint32_t)c;
    }
    r.trim();
    return r;
}

bool parse_rational(const char *s, Rat &out)
{
    if (!s) return false;
    Rat p;
    if (!parse_decimal(s, p)) return false;
    if (*s == '/') {
        s++;
        Rat q;
        if (!parse_decimal(s, q)) return false;
        if (q.num.zero()) return false;
        out.neg = p.neg != q.neg;
        out.num = mul(p.num, q.den);
        out.den = mul(p.den, q.num);
    } else {
        out = p;
    }
    if (*s != '\0') return false;
    if (out.num.zero()) out.neg = false;
    return true;
}

// a / d for a small d, a replaced by the quotient; returns the remainder
uint32_t div_small(BigU &a, uint32_t d)
{
    uint64_t r = 0;
    for (size_t i = a.w.size(); i-- > 0;) {
        const uint64_t cur = (r << 32) | a.w[i];
        a.w[i] = (uint32_t)(cur / d);
        r = cur % d;
    }
    a.trim();
    return (uint32_t)r;
}

std::string to_decimal(BigU a)
{
    if (a.zero()) return "0";
    std::vector<uint32_t> parts;  // base 10^9, least significant first
    while (!a.zero()) parts.push_back(div_small(a, 1000000000u));
    std::string out = std::to_string(parts.back());
    char buf[16];
    for (size_t i = parts.size() - 1; i-- > 0;) {
        std::snprintf(buf, sizeof buf, "%09u", parts[i]);
        out += buf;
    }
    return out;
}

// M 2^(32 sh) of an L-limb magnitude, sh >= 0
BigU magnitude(const uint32_t *l, int L, long long sh)
{
    BigU m;
    m.w.assign(l, l + L);
    m.trim();
    m.shl(32 * sh);
    return m;
}

}  // namespace

// The exact rational x + sgn 10^(-h_digits) of a decimal or rational string,
// written as "p/q".  Returns 0, or -1 for a malformed x.
// Y 2^k (Y a non-zero magnitude), negated when neg, rounded once to the
// nearest double (ties to even)
static double rounded(const BigU &y, long long k, bool neg)
{
    const int nb = y.bits();
    double r;
    if (nb <= 53) {
        uint64_t v = 0;
        for (size_t i = y.w.size(); i-- > 0;) v = (v << 32) | y.w[i];
        r = std::ldexp((double)v, (int)k);
    } else {
        const int drop = nb - 53;
        uint64_t q = 0;
        for (int i = nb - 1; i >= drop; i--) q = (q << 1) | (uint64_t)y.bit(i);
        const int half = y.bit(drop - 1);
        bool sticky = false;
        for (int i = drop - 2; i >= 0 && !sticky; i--) sticky = y.bit(i) != 0;
        if (half && (sticky || (q & 1))) q++;
        r = std::ldexp((double)q, (int)(k + drop));
    }
    return neg ? -r : r;
}

int perturbed_string(const char *x, int h_digits, int sgn, std::string &out)
{
    Rat r;
    if (!parse_rational(x, r) || h_digits < 0 || h_digits > kMaxDecimalExponent) return -1;
    // (+-num 10^h + sgn den) / (den 10^h)
    const BigU p = pow10(h_digits);
    BigU a = mul(r.num, p);
    const BigU &b = r.den;
    const bool aneg = r.neg, bneg = sgn < 0;
    bool neg;
    BigU n;
    if (aneg == bneg) {  // same signs: add
        n = a;
        BigU t = b;
        n.w.resize(std::max(n.w.size(), t.w.size()) + 1, 0);
        uint64_t c = 0;
        for (size_t i = 0; i < n.w.size(); i++) {
            const uint64_t v = (uint64_t)n.w[i] + (i < t.w.size() ? t.w[i] : 0) + c;
            n.w[i] = (uint32_t)v;
            c = v >> 32;
        }
        n.trim();
        neg = aneg;
    } else if (cmp(a, b) >= 0) {
        n = a;
        sub_inplace(n, b);
        neg = aneg;
    } else {
        n = b;
        sub_inplace(n, a);
        neg = bneg;
    }
    const BigU q = mul(r.den, p);
    out = (neg && !n.zero() ? "-" : "") + to_decimal(n) + "/" + to_decimal(q);
    return 0;
}

// (v1 - v2) / (2 10^(-h_digits)) of two L-limb numbers in the interchange
// layout, rounded once to the nearest double (ties to even).
double diff_over_2h(int L, int32_t s1, int32_t e1, const uint32_t *l1, int32_t s2, int32_t e2,
                    const uint32_t *l2, int h_digits)
{
    bool z1 = true, z2 = true;
    for (int j = 0; j < L; j++) {
        z1 = z1 && l1[j] == 0;
        z2 = z2 && l2[j] == 0;
    }
    if (z1 && z2) return 0.0;
    const long long emin = z1 ? e2 : (z2 ? e1 : std::min(e1, e2));
    BigU a = z1 ? BigU() : magnitude(l1, L, (long long)e1 - emin);
    BigU b = z2 ? BigU() : magnitude(l2, L, (long long)e2 - emin);
    const bool aneg = s1 != 0, bneg = s2 == 0;  // v1 - v2 = v1 + (-v2)
    bool neg;
    BigU d;
    if (aneg == bneg) {
        d = a;
        d.w.resize(std::max(d.w.size(), b.w.size()) + 1, 0);
        uint64_t c = 0;
        for (size_t i = 0; i < d.w.size(); i++) {
            const uint64_t v = (uint64_t)d.w[i] + (i < b.w.size() ? b.w[i] : 0) + c;
            d.w[i] = (uint32_t)v;
            c = v >> 32;
        }
        d.trim();
        neg = aneg;
    } else if (cmp(a, b) >= 0) {
        d = a;
        sub_inplace(d, b);
        neg = aneg;
    } else {
        d = b;
        sub_inplace(d, a);
        neg = bneg;
    }
    if (d.zero()) return 0.0;
    // |result| = Y 2^k, Y = |d| 10^h, k = 32 (emin - L) - 1
    return rounded(mul(d, pow10(h_digits)), 32LL * (emin - L) - 1, neg);
}

// the L-limb interchange number, rounded once to the nearest double
double to_double(int L, int32_t s, int32_t e, const uint32_t *l)
{
    bool z = true;
    for (int j = 0; j < L; j++) z = z && l[j] == 0;
    if (z) return 0.0;
    return rounded(magnitude(l, L, 0), 32LL * ((long long)e - L), s != 0);
}

// trunc_L of the exact value of a finite double; 0, or -1 for inf / nan
int from_double(double v, int L, int32_t *sign, int32_t *exp, uint32_t *limbs)
{
    if (!std::isfinite(v)) return -1;
    int x = 0;
    const double f = std::frexp(std::fabs(v), &x);  // |v| = f 2^x, 1/2 <= f < 1
    const uint64_t m = (uint64_t)std::ldexp(f, 53);  // exact: |v| = m 2^(x - 53)
    BigU num;
    num.w = {(uint32_t)m, (uint32_t)(m >> 32)};
    num.trim();
    std::string str = (v < 0 ? "-" : "");
    if (x - 53 >= 0) {
        num.shl(x - 53);
        str += to_decimal(num);
    } else {
        BigU den;
        den.w = {1u};
        den.shl(53 - x);
        str += to_decimal(num) + "/" + to_decimal(den);
    }
    return parse_number(str.c_str(), L, sign, exp, limbs);
}

// tau = trunc_L(p/q) with p/q in lowest terms, 0 < p < 2^32, 1 <= q < 2^16:
// its limbs M = floor(p 2^k / q), k = 32 shift (shift = L - exp), so
// M = (p 2^k - r) / q with r = p 2^k mod q.  Returns 0 with (p, q, r, shift,
// neg), or -1 when tau is not such a ratio (or M differs, which cannot happen).
int small_ratio(const char *str, int L, uint32_t *p, uint32_t *q, uint32_t *r, int *shift, int *neg)
{
    Rat t;
    if (!parse_rational(str, t) || t.num.zero() || t.num.bits() > 64 || t.den.bits() > 64) return -1;
    auto u64 = [](const BigU &a) {
        uint64_t v = 0;
        for (size_t i = a.w.size(); i-- > 0;) v = (v << 32) | a.w[i];
        return v;
    };
    uint64_t a = u64(t.num), b = u64(t.den);
    uint64_t x = a, y = b;
    while (y) {
        const uint64_t z = x % y;
        x = y;
        y = z;
    }
    a /= x;
    b /= x;
    if (a >= (1ull << 32) || b >= (1ull << 16)) return -1;
    int32_t s = 0, e = 0;
    std::vector<uint32_t> limbs((size_t)L);
    if (parse_number(str, L, &s, &e, limbs.data())) return -1;
    const long long sh = (long long)L - e;
    if (sh < 0 || sh > (1LL << 20)) return -1;
    uint64_t rem = a % b;
    for (long long i = 0; i < sh; i++) rem = (rem << 32) % b;
    // check M = (a 2^k - rem) / b limb for limb
    BigU X;
    X.w = {(uint32_t)a};
    X.trim();
    X.shl(32 * sh);
    BigU R;
    R.w = {(uint32_t)rem};
    R.trim();
    sub_inplace(X, R);
    BigU D;
    D.w = {(uint32_t)b};
    const BigU M = divide(X, D);
    if ((int)M.w.size() != L) return -1;
    for (int j = 0; j < L; j++)
        if (M.w[(size_t)j] != limbs[(size_t)j]) return -1;
    *p = (uint32_t)a;
    *q = (uint32_t)b;
    *r = (uint32_t)rem;
    *shift = (int)sh;
    *neg = t.neg ? 1 : 0;
    return 0;
}

// trunc_L of an exact decimal or rational string.  Returns 0, or -1 for a
// malformed string, -3 for an exponent outside |exp| <= 2^30.
int parse_number(const char *str, int L, int32_t *sign, int32_t *exp, uint32_t *limbs)
{
    Rat r;
    if (!parse_rational(str, r)) return -1;
    std::memset(limbs, 0, sizeof(uint32_t) * (size_t)L);
    if (r.num.zero()) {
        *sign = 0;
        *exp = 0;
        return 0;
    }
    // e with 2^(32(e-1)) <= num/den < 2^(32e)
    long long e = ((long long)r.num.bits() - (long long)r.den.bits()) / 32;
    auto ge_pow = [&](long long k) {  // num/den >= 2^(32k) ?
        BigU a = r.num, b = r.den;
        if (k >= 0)
            b.shl(32 * k);
        else
            a.shl(-32 * k);
        return cmp(a, b) >= 0;
    };
    while (ge_pow(e)) e++;
    while (!ge_pow(e - 1)) e--;
    if (e > (1LL << 30) || e < -(1LL << 30)) return -3;
    // M = floor(num * 2^(32(L-e)) / den)
    BigU a = r.num, b = r.den;
    long long sh = 32LL * (L - e);
    if (sh >= 0)
        a.shl(sh);
    else
        b.shl(-sh);
    BigU M = divide(a, b);
    if ((int)M.w.size() != L || M.w[(size_t)L - 1] == 0) return -1;  // cannot happen
    for (int j = 0; j < L; j++) limbs[j] = M.w[(size_t)j];
    *sign = r.neg ? 1 : 0;
    *exp = (int32_t)e;
    return 0;
}

// The division table of the pipelined kernel's closes (KArgs::divtab): row
// d (row 0 for q0) holds, for the odd part d' of d and i < rl,
// 2^(-32 i) mod d' in the low half and 2^(32 (i-1)) mod d' in the high half.
std::vector<uint32_t> division_table(int N, int rl, uint32_t q0)
{
    std::vector<uint32_t> t((size_t)(N + 1) * rl, 0u);
    for (int row = 0; row <= N; row++) {
        uint32_t d = row == 0 ? (q0 ? q0 : 1u) : (uint32_t)row;
        while (d % 2 == 0) d /= 2;
        if (d == 1) continue;  // every power is 0 mod 1
        const uint64_t w1 = (1ull << 32) % d;
        // inverse of w1 mod d (d odd, so it exists): extended Euclid
        int64_t r0 = d, r1 = (int64_t)w1, s0 = 0, s1 = 1;
        while (r1) {
            const int64_t qq = r0 / r1, r2 = r0 - qq * r1, s2 = s0 - qq * s1;
            r0 = r1;
            r1 = r2;
            s0 = s1;
            s1 = s2;
        }
        const uint64_t u1 = (uint64_t)((s0 % (int64_t)d + d) % d);
        uint64_t W = 1 % d, U = 1 % d, Wprev = 0;
        for (int i = 0; i < rl; i++) {
            t[(size_t)row * rl + i] = (uint32_t)U | ((uint32_t)Wprev << 16);
            Wprev = W;
            W = W * w1 % d;
            U = U * u1 % d;
        }
    }
    return t;
}

}  // namespace mpt_host
