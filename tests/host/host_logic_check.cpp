// Host-side checks of two helpers the kernels share with the host code
// (csrc/dust_internal.h): order_key, the integer image of a double used for
// the zone-edge comparisons, and zone_key, the sort key of a zone in the
// tile layout.  Prints "ok" or the first failure and exits non-zero.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <random>
#include <set>
#include <vector>

#include "dust_internal.h"

using dust::GridDev;
using dust::order_key;
using dust::zone_key;

static int fail(const char *what, double a, double b)
{
    std::printf("FAIL %s: %.17g %.17g\n", what, a, b);
    return 1;
}

static int check_order_key()
{
    std::mt19937_64 rng(12345);
    std::vector<double> v = {0.0, -0.0, DBL_MIN, -DBL_MIN, DBL_TRUE_MIN, -DBL_TRUE_MIN,
                             DBL_MAX, -DBL_MAX, 1.0, -1.0, 0.5, -0.5, 1e-300, -1e-300};
    const size_t nspecial = v.size();
    for (size_t i = 0; i < nspecial; ++i)  // every pair of the special values
        for (size_t j = 0; j < nspecial; ++j) {
            const double a = v[i], b = v[j];
            if ((order_key(a) < order_key(b)) != (a < b)) return fail("order_key < special", a, b);
            if ((order_key(a) == order_key(b)) != (a == b)) return fail("order_key == special", a, b);
        }
    std::uniform_real_distribution<double> u(-1e3, 1e3);
    for (int i = 0; i < 20000; ++i) v.push_back(u(rng));
    for (int i = 0; i < 20000; ++i) {  // any finite bit pattern
        uint64_t b = rng();
        double d;
        std::memcpy(&d, &b, 8);
        if (std::isfinite(d)) v.push_back(d);
    }
    for (int i = 0; i < 2000; ++i) {  // neighbours one ulp apart
        const double d = u(rng);
        v.push_back(d);
        v.push_back(std::nextafter(d, INFINITY));
        v.push_back(std::nextafter(d, -INFINITY));
    }
    std::uniform_int_distribution<size_t> pick(0, v.size() - 1);
    for (int i = 0; i < 400000; ++i) {
        const double a = v[pick(rng)], b = v[pick(rng)];
        const long long ka = order_key(a), kb = order_key(b);
        if ((ka < kb) != (a < b)) return fail("order_key <", a, b);
        if ((ka == kb) != (a == b)) return fail("order_key ==", a, b);
    }
    for (size_t i = 0; i + 2 < v.size(); i += 3) {
        const double a = v[i], b = v[i + 1];
        if ((order_key(a) < order_key(b)) != (a < b)) return fail("order_key ulp", a, b);
    }
    return 0;
}

static int check_zone_key(int n0, int n1, int n2, int t0, int t1, int t2)
{
    GridDev g;
    std::memset(&g, 0, sizeof g);
    const int n[3] = {n0, n1, n2}, t[3] = {t0, t1, t2};
    g.tvol = 1;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = n[d];
        g.T[d] = t[d];
        g.nt[d] = (n[d] + t[d] - 1) / t[d];
        g.tvol *= t[d];
    }
    g.nkeys = (int64_t)g.nt[0] * g.nt[1] * g.nt[2] * g.tvol;
    std::set<int64_t> seen;
    for (int k = 0; k < n2; ++k)
        for (int j = 0; j < n1; ++j)
            for (int i = 0; i < n0; ++i) {
                const int64_t key = zone_key(g, i, j, k);
                if (key < 0 || key >= g.nkeys) return fail("zone_key range", i, (double)key);
                if (!seen.insert(key).second) return fail("zone_key not injective", i, (double)key);
                // the zone's tile owns the key range [tile * tvol, (tile + 1) * tvol)
                const int64_t tile = (i / t0) + (int64_t)g.nt[0] * ((j / t1) + (int64_t)g.nt[1] * (k / t2));
                if (key / g.tvol != tile) return fail("zone_key tile", i, (double)key);
                // the slab kernel's decode of the key inside the tile (x fastest)
                const int r = (int)(key % g.tvol);
                const int kx = r % t0, ky = (r / t0) % t1, kz = r / (t0 * t1);
                if (kx != i % t0 || ky != j % t1 || kz != k % t2) return fail("zone_key decode", i, (double)r);
            }
    return 0;
}

int main()
{
    if (check_order_key()) return 1;
    const int cases[][6] = {{16, 16, 16, 8, 8, 8}, {20, 13, 9, 8, 8, 8}, {64, 1, 64, 16, 1, 16},
                            {37, 1, 29, 8, 1, 8}, {24, 32, 8, 8, 2, 4}, {100, 1, 1, 256, 1, 1},
                            {12, 10, 7, 4, 4, 2}};
    for (const auto &c : cases)
        if (check_zone_key(c[0], c[1], c[2], c[3] > c[0] ? c[0] : c[3], c[4] > c[1] ? c[1] : c[4],
                           c[5] > c[2] ? c[2] : c[5]))
            return 1;
    std::printf("ok\n");
    return 0;
}
