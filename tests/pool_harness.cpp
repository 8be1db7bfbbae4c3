// Test harness for the convolution server's device-memory pool: reads
// commands on stdin and prints one result line each, so that
// tests/test_serve_pool_cpu.py can drive it without a GPU.
//
//   init bytes        -> ok
//   alloc bytes       -> offset, or -1 when no free block is large enough
//   free off bytes    -> ok
//   peak              -> the largest number of bytes in use so far
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>

#include "../paper_1005_1497_gb300/csrc/serve_pool.h"

int main()
{
    ntt::Pool pool;
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string cmd;
        unsigned long long a = 0, b = 0;
        in >> cmd;
        if (cmd == "init") {
            in >> a;
            pool.init(a);
            std::printf("ok\n");
        } else if (cmd == "alloc") {
            in >> a;
            size_t off = 0;
            if (pool.alloc(a, &off)) std::printf("%llu\n", (unsigned long long)off);
            else std::printf("-1\n");
        } else if (cmd == "free") {
            in >> a >> b;
            pool.release(a, b);
            std::printf("ok\n");
        } else if (cmd == "peak") {
            std::printf("%llu\n", (unsigned long long)pool.peak());
        } else {
            std::printf("?\n");
        }
    }
    return 0;
}
