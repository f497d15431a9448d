// chem_quads.h -- host-side order of the reactions for the thread-per-cell FP32 kernel
// (kern_f32t.cu), which takes them four at a time ("quads") with one code path per type.
//
// Within each type, in type order, reactions are packed greedily, in reaction order, into the
// first open quad whose net species (nu''_k != nu'_k) are disjoint from its members' (a quad
// is closed at four).  Full quads keep that order and are flagged disjoint: their omega
// entries can be read once and written once.  The reactions of the quads left incomplete
// follow in order, four to a quad, each quad flagged disjoint only if it is; the last quad of
// a type is padded with zero-rate slots (-1).
#pragma once

#include <vector>

namespace chem {

struct QuadPlan {
    std::vector<int> slot;        // reaction per slot (4 per quad), -1 for a padding slot
    std::vector<int> type;        // per quad
    std::vector<bool> disjoint;   // per quad: net species of its reactions pairwise distinct
};

inline QuadPlan plan_quads(int ntypes, const std::vector<int> &type_of,
                           const std::vector<std::vector<int>> &net, int quad = 4)
{
    QuadPlan plan;
    const int nr = (int)type_of.size();
    auto clash = [&](const std::vector<int> &a, const std::vector<int> &b) {
        for (int x : a)
            for (int y : b)
                if (x == y) return true;
        return false;
    };
    for (int g = 0; g < ntypes; ++g) {
        std::vector<std::vector<int>> open;     // members of each greedy quad
        std::vector<std::vector<int>> used;     // their net species
        for (int j = 0; j < nr; ++j) {
            if (type_of[j] != g) continue;
            size_t q = 0;
            for (; q < open.size(); ++q)
                if ((int)open[q].size() < quad && !clash(used[q], net[j])) break;
            if (q == open.size()) {
                open.emplace_back();
                used.emplace_back();
            }
            open[q].push_back(j);
            used[q].insert(used[q].end(), net[j].begin(), net[j].end());
        }
        std::vector<int> rest;
        for (size_t q = 0; q < open.size(); ++q) {
            if ((int)open[q].size() == quad) {
                plan.slot.insert(plan.slot.end(), open[q].begin(), open[q].end());
                plan.type.push_back(g);
                plan.disjoint.push_back(true);
            } else {
                rest.insert(rest.end(), open[q].begin(), open[q].end());
            }
        }
        for (size_t a = 0; a < rest.size(); a += quad) {
            std::vector<int> seen;
            bool dis = true;
            for (size_t b = a; b < a + quad; ++b) {
                if (b < rest.size()) {
                    const int j = rest[b];
                    dis = dis && !clash(seen, net[j]);
                    seen.insert(seen.end(), net[j].begin(), net[j].end());
                    plan.slot.push_back(j);
                } else {
                    plan.slot.push_back(-1);
                }
            }
            plan.type.push_back(g);
            plan.disjoint.push_back(dis);
        }
    }
    return plan;
}

}  // namespace chem
