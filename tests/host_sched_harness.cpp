// Test harness for the library's host scheduling rules (host_sched.h): reads
// one command per line on stdin and prints one result line each, so that
// tests/test_host_sched_cpu.py can check them without a GPU.
//
//   small L rw word_bytes nsm        -> small_batch_max
//   chunkpairs seq_bytes split batch -> host_chunk_pairs
//   chunks pairs chunk shrink        -> host_chunk_sizes (space separated; "-" when empty)
#include <iostream>
#include <sstream>
#include <string>

#include "../paper_1005_1497_gb300/csrc/host_sched.h"

int main()
{
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        std::string cmd;
        in >> cmd;
        if (cmd == "small") {
            int L = 0, rw = 0, wb = 0, nsm = 0;
            in >> L >> rw >> wb >> nsm;
            std::cout << ntt::small_batch_max(L, rw, wb, nsm) << "\n";
        } else if (cmd == "chunkpairs") {
            unsigned long long seq = 0, batch = 0;
            int split = 0;
            in >> seq >> split >> batch;
            std::cout << ntt::host_chunk_pairs((size_t)seq, split != 0, (size_t)batch) << "\n";
        } else if (cmd == "chunks") {
            unsigned long long pairs = 0, chunk = 0;
            int shrink = 0;
            in >> pairs >> chunk >> shrink;
            const auto v = ntt::host_chunk_sizes((size_t)pairs, (size_t)chunk, shrink != 0);
            if (v.empty()) std::cout << "-";
            for (size_t i = 0; i < v.size(); ++i) std::cout << (i ? " " : "") << v[i];
            std::cout << "\n";
        } else {
            std::cout << "?\n";
        }
    }
    return 0;
}
