// Drives chem::Arena (paper_2008_08483_gb300/csrc/chem_arena.h) from stdin for
// tests/test_serve_arena.py: "init N", "alloc B" (prints the offset or -1), "free OFF B",
// "state" (prints in_use, peak, largest free block, then each free block as offset:length).
#include <stdio.h>
#include <string.h>

#include "chem_arena.h"

int main()
{
    chem::Arena a;
    char op[16];
    unsigned long long x, y;
    while (scanf("%15s", op) == 1) {
        if (!strcmp(op, "init") && scanf("%llu", &x) == 1) {
            a.init((size_t)x);
        } else if (!strcmp(op, "alloc") && scanf("%llu", &x) == 1) {
            size_t off = 0;
            if (a.alloc((size_t)x, off))
                printf("%llu\n", (unsigned long long)off);
            else
                printf("-1\n");
        } else if (!strcmp(op, "free") && scanf("%llu %llu", &x, &y) == 2) {
            a.release((size_t)x, (size_t)y);
        } else if (!strcmp(op, "state")) {
            printf("%llu %llu %llu", (unsigned long long)a.in_use, (unsigned long long)a.peak,
                   (unsigned long long)a.largest_free());
            for (auto &kv : a.free_) printf(" %llu:%llu", (unsigned long long)kv.first, (unsigned long long)kv.second);
            printf("\n");
        }
    }
    return 0;
}
