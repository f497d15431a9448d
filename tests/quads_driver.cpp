// Drives chem::plan_quads (paper_2008_08483_gb300/csrc/chem_quads.h) for
// tests/test_f32t_quads.py.  Input: n_types n_reactions, then per reaction its type, the
// count of its net species and their indices.  Output: the slots of each quad, one quad per
// line as "type disjoint s0 s1 s2 s3".
#include <stdio.h>

#include "chem_quads.h"

int main()
{
    int ntypes = 0, nr = 0;
    if (scanf("%d %d", &ntypes, &nr) != 2) return 1;
    std::vector<int> type_of(nr);
    std::vector<std::vector<int>> net(nr);
    for (int j = 0; j < nr; ++j) {
        int c = 0;
        if (scanf("%d %d", &type_of[j], &c) != 2) return 1;
        net[j].resize(c);
        for (int i = 0; i < c; ++i)
            if (scanf("%d", &net[j][i]) != 1) return 1;
    }
    const chem::QuadPlan p = chem::plan_quads(ntypes, type_of, net);
    for (size_t q = 0; q < p.type.size(); ++q)
        printf("%d %d %d %d %d %d\n", p.type[q], p.disjoint[q] ? 1 : 0, p.slot[4 * q],
               p.slot[4 * q + 1], p.slot[4 * q + 2], p.slot[4 * q + 3]);
    return 0;
}
