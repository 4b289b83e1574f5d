// Shared-memory budget of the slab tile function for the tile shapes that
// have compiled copies: two blocks per SM must fit, since the step kernel's
// speed rests on 16 resident warps per SM (registers allow two blocks too).
// Host code only: no kernel is instantiated and no CUDA call is made.
#include <cstdio>

#include "dust_slab.cuh"

int main()
{
    using namespace dust;
    struct Case {
        int T[3], n[3];
    };
    // 8^3 tiles of a 3-D grid; 32 x 16 and 16 x 16 x-z tiles of 2-D boxes
    const Case cases[] = {{{8, 8, 8}, {128, 128, 128}}, {{32, 1, 16}, {512, 1, 512}}, {{16, 1, 16}, {256, 1, 256}}};
    // GB300: 228 KB of shared memory per SM, 1 KB of it reserved per block
    const size_t per_sm = 228 * 1024, reserved = 1024;
    for (const Case &c : cases) {
        GridDev g{};
        for (int d = 0; d < 3; ++d) {
            g.T[d] = c.T[d];
            g.n[d] = c.n[d];
        }
        g.tvol = c.T[0] * c.T[1] * c.T[2];
        const size_t b = slab_smem_bytes(g);
        if (2 * (b + reserved) > per_sm) {
            std::printf("tile %dx%dx%d: %zu bytes per block, two blocks do not fit\n", c.T[0], c.T[1], c.T[2], b);
            return 1;
        }
    }
    std::printf("ok\n");
    return 0;
}
