// Test harness for the library's host number theory (plan construction):
// reads one command per line on stdin and prints one result line each, so
// that tests/test_host_nt_cpu.py can compare them with the oracle and with
// exact integer arithmetic, without a GPU.
//
//   prime n            -> 1 / 0
//   order m            -> ord_m(2) if a power of two, else 0
//   pow a e m          -> a^e mod m
//   powers count m     -> 2^k mod m, k = 0 .. count-1 (space separated)
//   shoupq z m B       -> floor(z 2^B / m)
//   shl x B m          -> (x 2^B) mod m
//   invpow2 m B        -> m^-1 mod 2^B
//   brv i bits         -> i with its low `bits` bits reversed
#include <cstdio>
#include <cstring>
#include <iostream>
#include <sstream>
#include <string>

#include "../paper_1005_1497_gb300/csrc/nt_host.h"

int main()
{
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string cmd;
        in >> cmd;
        unsigned long long a = 0, b = 0, c = 0;
        if (cmd == "prime") {
            in >> a;
            std::printf("%d\n", nt::is_prime(a) ? 1 : 0);
        } else if (cmd == "order") {
            in >> a;
            std::printf("%llu\n", (unsigned long long)nt::order_of_two_pow2(a));
        } else if (cmd == "pow") {
            in >> a >> b >> c;
            std::printf("%llu\n", (unsigned long long)nt::pow_mod(a, b, c));
        } else if (cmd == "powers") {
            in >> a >> b;
            const std::vector<uint64_t> p = nt::powers_of_two_by_doubling(a, b);
            for (unsigned long long k = 0; k < a; ++k) std::printf(k ? " %llu" : "%llu", (unsigned long long)p[k]);
            std::printf("\n");
        } else if (cmd == "shoupq") {
            in >> a >> b >> c;
            std::printf("%llu\n", (unsigned long long)nt::shoup_quot(a, b, (int)c));
        } else if (cmd == "shl") {
            in >> a >> b >> c;
            std::printf("%llu\n", (unsigned long long)nt::shl_mod(a, (int)b, c));
        } else if (cmd == "invpow2") {
            in >> a >> b;
            std::printf("%llu\n", (unsigned long long)nt::inv_pow2(a, (int)b));
        } else if (cmd == "brv") {
            in >> a >> b;
            std::printf("%llu\n", (unsigned long long)nt::bit_reverse(a, (int)b));
        } else {
            std::printf("?\n");
        }
    }
    return 0;
}
