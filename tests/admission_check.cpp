// Drives the serving loop's admission policy (csrc/admission.h) without a GPU:
// reads commands from stdin and prints each decision.
//   cap <budget> <free> <held>        -> prints the cap
//   admit <in_use> <cap> <max_jobs> <jobs:est> ...   -> prints "<count> <est>"
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "admission.h"

int main() {
    char cmd[32];
    while (std::scanf("%31s", cmd) == 1) {
        if (!std::strcmp(cmd, "cap")) {
            unsigned long long b, f, h;
            if (std::scanf("%llu %llu %llu", &b, &f, &h) != 3) return 2;
            std::printf("%llu\n", (unsigned long long)sa::admission_cap(b, f, h));
        } else if (!std::strcmp(cmd, "admit")) {
            unsigned long long in_use, cap, max_jobs, n;
            if (std::scanf("%llu %llu %llu %llu", &in_use, &cap, &max_jobs, &n) != 4) return 2;
            std::vector<std::pair<uint64_t, uint64_t>> q(n);
            for (auto& r : q) {
                unsigned long long j, e;
                if (std::scanf("%llu %llu", &j, &e) != 2) return 2;
                r = {j, e};
            }
            uint64_t est = 0;
            const size_t k = sa::admit_front(q, [](const std::pair<uint64_t, uint64_t>& r) { return r; },
                                             in_use, cap, max_jobs, &est);
            std::printf("%zu %llu\n", k, (unsigned long long)est);
        } else {
            return 3;
        }
    }
    return 0;
}
