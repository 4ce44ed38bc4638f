// Driver for tests/test_host_parse.py: the host's exact perturbation strings
// and rounded differences, one case per input line.
//   P x h sgn                      -> the string x + sgn 10^-h
//   D L h s1 e1 l1.. s2 e2 l2..    -> (v1 - v2) / (2 10^-h) as %.17g
//   T N rl q0                      -> the division table, (N+1) rl entries
#include <cstdio>
#include <iostream>
#include <string>
#include <vector>

#include "../../paper_1908_09301_gb300/csrc/host_parse.h"

int main()
{
    std::string op;
    while (std::cin >> op) {
        if (op == "P") {
            std::string x;
            int h, sg;
            std::cin >> x >> h >> sg;
            std::string out;
            const int rc = mpt_host::perturbed_string(x.c_str(), h, sg, out);
            std::cout << rc << " " << (rc ? "-" : out) << "\n";
        } else if (op == "D") {
            int L, h;
            std::cin >> L >> h;
            int32_t s[2], e[2];
            std::vector<uint32_t> l[2];
            for (int k = 0; k < 2; k++) {
                std::cin >> s[k] >> e[k];
                l[k].resize(L);
                for (int x = 0; x < L; x++) std::cin >> l[k][x];
            }
            const double d = mpt_host::diff_over_2h(L, s[0], e[0], l[0].data(), s[1], e[1], l[1].data(), h);
            char buf[64];
            std::snprintf(buf, sizeof buf, "%.17g", d);
            std::cout << buf << "\n";
        } else if (op == "T") {
            int N, rl;
            uint32_t q0;
            std::cin >> N >> rl >> q0;
            const std::vector<uint32_t> t = mpt_host::division_table(N, rl, q0);
            for (size_t i = 0; i < t.size(); i++) std::cout << t[i] << (i + 1 < t.size() ? " " : "\n");
        }
    }
    return 0;
}
