// CPU check of the batched persistent kernel's work list (dust_worklist.h):
// for random batches, every (step, instance, phase) receives exactly its
// work items, each task depends only on the same group's previous task
// (which comes earlier in the list, so the in-order item counter can never
// wait on a task whose items are not all taken), groups partition the
// instances, and the item -> (task, instance, local item) decode the kernel
// performs finds every item once.  Prints "ok" or the first failure.
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "dust_worklist.h"

using namespace dust;

static int fail(const char *what, int a, int b)
{
    std::printf("fail: %s (%d, %d)\n", what, a, b);
    return 1;
}

static int check(const std::vector<BatchInst> &inst, int nsteps, int K)
{
    std::vector<int> tab;
    BatchDev d{};
    if (!work_list(inst.data(), inst.size(), nsteps, K, tab, d)) return fail("overflow", 0, 0);
    const int n = (int)inst.size();
    const BatchTask *tasks = reinterpret_cast<const BatchTask *>(tab.data() + d.off_tasks);
    const int *members = tab.data() + d.off_members;
    const int *gcount = tab.data() + d.off_gcount;
    const int *gpre = tab.data() + d.off_gpre;
    // groups partition the instances
    std::vector<int> seen(n, 0);
    for (int g = 0; g < d.ngroups; ++g)
        for (int k = 0; k < gcount[g]; ++k) seen[members[g * d.gmax + k]]++;
    for (int i = 0; i < n; ++i)
        if (seen[i] != 1) return fail("instance not in exactly one group", i, seen[i]);
    // tasks: consecutive items, dependencies on the group's previous task
    std::vector<int> last(d.ngroups, -1);
    int64_t begin = 0;
    for (int t = 0; t < d.ntasks; ++t) {
        const BatchTask &T = tasks[t];
        if (T.begin != begin || T.items <= 0) return fail("task items", t, T.begin);
        if (T.dep != last[T.g]) return fail("dependency", t, T.dep);
        if (T.dep >= t) return fail("dependency not earlier", t, T.dep);
        if (T.dep >= 0) {
            const BatchTask &P = tasks[T.dep];
            if (!(P.s < T.s || (P.s == T.s && P.p < T.p))) return fail("chain order", t, T.dep);
        }
        last[T.g] = t;
        begin += T.items;
    }
    if (begin != d.nitems) return fail("item total", (int)begin, d.nitems);
    // decode every item as the kernel does and count per (step, instance, phase)
    std::vector<int64_t> got((size_t)nsteps * n * BPH_N, 0);
    for (int w = 0; w < d.nitems; ++w) {
        int lo = 0, hi = d.ntasks;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tasks[mid].begin <= w) lo = mid;
            else hi = mid;
        }
        const BatchTask &T = tasks[lo];
        const int l = w - T.begin;
        const bool sorted = (T.s % K) == 0;
        const int *pre = gpre + ((size_t)((sorted ? 1 : 0) * BPH_N + T.p) * d.ngroups + T.g) * (d.gmax + 1);
        int a = 0, b = gcount[T.g];
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (pre[mid] <= l) a = mid;
            else b = mid;
        }
        const int i = members[T.g * d.gmax + a];
        const int li = l - pre[a];
        if (li < 0 || li >= phase_items(inst[i], T.p, sorted)) return fail("local item", w, li);
        got[((size_t)T.s * n + i) * BPH_N + T.p]++;
    }
    for (int s = 0; s < nsteps; ++s)
        for (int i = 0; i < n; ++i)
            for (int p = 0; p < BPH_N; ++p)
                if (got[((size_t)s * n + i) * BPH_N + p] != phase_items(inst[i], p, (s % K) == 0))
                    return fail("items of (step, instance)", s, i * BPH_N + p);
    return 0;
}

int main()
{
    std::mt19937_64 rng(1234);
    for (int trial = 0; trial < 300; ++trial) {
        const int n = 1 + (int)(rng() % 70);
        std::vector<BatchInst> inst(n);
        for (auto &I : inst) {
            I = BatchInst{};
            const int side = 8 << (rng() % 6);
            const int flat = (int)(rng() % 2);
            I.ncell = (int64_t)side * side * (flat ? 1 : (1 + (int64_t)(rng() % 4)));
            I.nkeys = I.ncell + (int64_t)(rng() % 64);
            I.n = (rng() % 10 == 0) ? 0 : (int64_t)(rng() % 17) * I.ncell / 4;
            I.ntiles = (int)std::max<int64_t>(1, I.ncell / 256);
        }
        const int nsteps = 1 + (int)(rng() % 7);
        const int K = 1 + (int)(rng() % 3);
        if (check(inst, nsteps, K)) {
            std::printf("trial %d n %d steps %d K %d\n", trial, n, nsteps, K);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
