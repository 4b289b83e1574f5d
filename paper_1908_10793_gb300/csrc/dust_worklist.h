// Work list of the batched persistent kernel (host side): the work items of
// each phase of an instance and the layout of all tasks of a call, checked on
// the CPU by tests/host/worklist_check.cpp.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "dust_internal.h"

namespace dust {

// Work items of phase p of a step of instance I (sorted: the step sorts
// first).
inline int64_t phase_items(const BatchInst &I, int p, bool sorted)
{
    auto items = [](int64_t chunks) { return (chunks + kBatchChunks - 1) / kBatchChunks; };
    const int64_t nscan = (I.nkeys + 2 + kBatchScanChunk - 1) / kBatchScanChunk;
    switch (p) {
    case BPH_SCANA: return sorted ? items(nscan) : 0;
    case BPH_SCANB: return sorted ? 1 : 0;
    case BPH_SCANC: return sorted ? items(nscan) : 0;
    case BPH_SCATTER: return sorted ? items((I.n + kBatchScatterChunk - 1) / kBatchScatterChunk) : 0;
    case BPH_SEG: return sorted ? items((I.nkeys + 1 + kBatchSegChunk - 1) / kBatchSegChunk) : 0;
    case BPH_ZERO:
        return items((std::max(I.ncell * 4, I.nkeys + 2) + kBatchZeroChunk - 1) / kBatchZeroChunk) +
               (sorted ? kBatchBigItems : 0);
    case BPH_TILE: return I.ntiles;
    default: return items((I.ncell + kBatchFbChunk - 1) / kBatchFbChunk);
    }
}

// The work list of nsteps steps of the n instances (batch_persistent_kernel):
// the instances dealt, most grains first, into groups of about equal work;
// group g's phase p of step s in round s * period + g + p, so that the
// groups run different phases side by side; inside a round by phase; tasks
// without items left out, each task depending on its group's previous one.
// Fills the table and the shape fields of d; false if the items overflow.
inline bool work_list(const BatchInst *inst, size_t n, int nsteps, int K, std::vector<int> &tab, BatchDev &d)
{
    const int G = (int)std::min<size_t>(n, BPH_N);
    const int W = std::max(G, (int)BPH_N);
    std::vector<int> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return inst[x].n > inst[y].n; });
    std::vector<std::vector<int>> members(G);
    for (size_t j = 0; j < n; ++j) members[j % G].push_back(order[j]);
    int gmax = 0;
    for (auto &m : members) gmax = std::max(gmax, (int)m.size());
    // prefix sums of the members' items per (sorted, phase, group)
    std::vector<int64_t> gpre((size_t)2 * BPH_N * G * (gmax + 1), 0);
    for (int so = 0; so < 2; ++so)
        for (int p = 0; p < BPH_N; ++p)
            for (int g = 0; g < G; ++g) {
                int64_t *q = &gpre[((size_t)(so * BPH_N + p) * G + g) * (gmax + 1)];
                for (size_t k = 0; k < members[g].size(); ++k)
                    q[k + 1] = q[k] + phase_items(inst[members[g][k]], p, so != 0);
                for (int k = (int)members[g].size(); k < gmax; ++k) q[k + 1] = q[k];
            }
    struct Slot {
        int64_t round;
        int p, s, g;
    };
    std::vector<Slot> slots;
    slots.reserve((size_t)nsteps * G * BPH_N);
    for (int s = 0; s < nsteps; ++s)
        for (int g = 0; g < G; ++g)
            for (int p = 0; p < BPH_N; ++p) slots.push_back({(int64_t)s * W + g + p, p, s, g});
    std::stable_sort(slots.begin(), slots.end(), [](const Slot &x, const Slot &y) {
        return x.round != y.round ? x.round < y.round : x.p < y.p;
    });
    std::vector<BatchTask> tasks;
    std::vector<int> last(G, -1);
    int64_t begin = 0;
    for (const Slot &sl : slots) {
        const int so = (sl.s % K) == 0 ? 1 : 0;
        const int64_t items = gpre[((size_t)(so * BPH_N + sl.p) * G + sl.g) * (gmax + 1) + members[sl.g].size()];
        if (items == 0) continue;
        if (begin + items >= ((int64_t)1 << 31)) return false;
        tasks.push_back({sl.s, sl.g, sl.p, (int)begin, (int)items, last[sl.g]});
        last[sl.g] = (int)tasks.size() - 1;
        begin += items;
    }
    static_assert(sizeof(BatchTask) == 6 * sizeof(int), "task layout");
    d.off_tasks = 0;
    d.off_members = (int)(tasks.size() * 6);
    d.off_gcount = d.off_members + G * gmax;
    d.off_gpre = d.off_gcount + G;
    d.nstatic = d.off_gpre + (int)gpre.size();
    tab.assign((size_t)d.nstatic, 0);
    std::memcpy(tab.data(), tasks.data(), tasks.size() * sizeof(BatchTask));
    for (int g = 0; g < G; ++g) {
        for (size_t k = 0; k < members[g].size(); ++k) tab[d.off_members + g * gmax + k] = members[g][k];
        tab[d.off_gcount + g] = (int)members[g].size();
    }
    for (size_t k = 0; k < gpre.size(); ++k) tab[d.off_gpre + k] = (int)gpre[k];
    d.ntasks = (int)tasks.size();
    d.nitems = (int)begin;
    d.ngroups = G;
    d.gmax = gmax;
    d.nsteps = nsteps;
    d.sort_interval = K;
    return true;
}

}  // namespace dust
