// Slab-group step kernel (mixed precision).  One CTA per tile of zones, the
// tile's gas stencil staged in shared memory.  A warp takes an equal range of
// the tile's sort keys (zones), whose grains are contiguous in the store, and
// walks it in passes of up to kSlabCap grains.
// Push: one grain per lane over the whole pass (coalesced loads and stores,
// no per-zone imbalance); the 27-node gather reads the staged gas box (grains
// of one zone read the same nodes, so the loads broadcast); each grain leaves
// a record (weights, deposit impulse) in the warp's shared buffer.  Deposit,
// ten zones of the pass at a time:
// three lanes own one zone; lane a keeps, in registers, the accumulators of
// the nine stencil nodes at x-offset a - 1 and sums the zone's records into
// them.  A zone's deposit (its run: the grains sorted into it whose half-step
// host is the zone itself), cut into chunks of kSlabCap grains by rank, is
// quantised once per chunk and node and added to the shared deposit box; the
// host node receives the remainder of the chunk's quantised total.  Grains
// are stored in id order inside a zone (see the sort), so the summation
// order, hence the integers, is reproducible and independent of the tile
// shape.  Grains whose host is not their key zone (stale sort) use the
// per-grain rule.
//
// The push runs relative to the key zone: each coordinate's offset from the
// zone centre is formed once in double precision and rounded to single;
// the half drifts, the weights, the metric factors and the kick then work on
// these offsets in single precision, and the coordinate is updated once, in
// double precision, by the step's summed increment.  This keeps the narrow
// double-precision pipe to four operations per coordinate.
#pragma once

#include "dust_tiled.cuh"

namespace dust {

constexpr int kSlabThreads = 256;
constexpr int kSlabCap = 128;  // grains per warp record pass
// Record slots: a grain of the pass's zone zp (counted from the pass's first
// zone) at pass position s uses slot s + min(zp, 15), so the owner lanes of
// neighbouring zones, which read their zones' grains in step, fall on
// different shared-memory banks; the stagger never decreases along the pass,
// so slots are unique.
constexpr int kRecStride = kSlabCap + 16;
constexpr int kRecFields = 13;  // 3 x 3 weights, 4 deposit channels

template <int FLAT>
struct SlabShape {
    // FLAT: 0 = three gridded directions, 1 = y not gridded, 2 = z not gridded
    static constexpr int NB = FLAT == 1 ? 1 : 3;
    static constexpr int NC = FLAT == 2 ? 1 : 3;
    static constexpr int BC = NB == 3 ? 1 : 0;   // index of the host node in y
    static constexpr int CC = NC == 3 ? 1 : 0;   // index of the host node in z
};

// Hint: move the line holding p into L2 (no register result, no wait).
template <typename T>
__device__ __forceinline__ void prefetch_l2(const T *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// The grain columns a push reads at store position src, prefetched into L2
// one push iteration (or one pass) before they are read.
template <typename Store>
__device__ __forceinline__ void prefetch_grain(const Store &S, int src)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        prefetch_l2(S.q[d] + src);
        prefetch_l2(S.p[d] + src);
    }
    if (S.species) prefetch_l2(S.species + src);
}

// A deposit piece too large for the split form of the shared deposit box
// (below), or from a tile too dense for it: added to the global deposit at
// the zone of box position lin (x fastest, box of B0 x B1 x ..., origin o).
static __device__ __noinline__ void box_piece_to_global(const GridDev &g, unsigned long long *dep, int o0, int o1,
                                                 int o2, int B0, int B1, int lin, int ch, long long v)
{
    const int bx = lin % B0, by = (lin / B0) % B1, bz = lin / (B0 * B1);
    const int i = map_zone(o0 + bx, g.n[0], g.bc[0]);
    const int j = map_zone(o1 + by, g.n[1], g.bc[1]);
    const int k = map_zone(o2 + bz, g.n[2], g.bc[2]);
    atomicAdd(&dep[4 * (i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k)) + ch], (unsigned long long)v);
}

__device__ __forceinline__ float sel3(const float v[3], int i)
{
    return i == 0 ? v[0] : (i == 1 ? v[1] : v[2]);
}

// The per-grain fixed-point rule (see deposit_fixed) for a grain whose
// stencil leaves the staged box: global atomics, the same nodes and order,
// in a rolled loop.
template <int NB, int NC>
__device__ __forceinline__ void deposit_fixed_rolled(const GridDev &g, unsigned long long *dep,
                                                     const int host[3], const float w[3][3],
                                                     const float Dq[4], unsigned int *status)
{
    long long rest[4];
    bool big = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        big |= !(fabsf(Dq[c]) < 4.5e15f);
        rest[c] = rround(Dq[c]);
    }
    if (big) atomicOr(&status[ST_FLAGS], DUST_FLAG_OVERFLOW);
#pragma unroll 1
    for (int nd = 0; nd < 27; ++nd) {
        const int a = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
        if ((NB == 1 && b != 1) || (NC == 1 && c3 != 1) || nd == 13) continue;
        const float W = sel3(w[0], a) * (sel3(w[1], b) * sel3(w[2], c3));
        const int ix = node_of(host[0], a - 1, g.n[0], g.bc[0]);
        const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
        const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
        const int64_t idx = ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long piece = rround(W * Dq[c]);
            if (piece != 0) {
                atomicAdd(&dep[4 * idx + c], (unsigned long long)piece);
                rest[c] -= piece;
            }
        }
    }
    const int64_t hidx = node_of(host[0], 0, g.n[0], g.bc[0]) +
                         (int64_t)g.n[0] * (node_of(host[1], 0, g.n[1], g.bc[1]) +
                                            (int64_t)g.n[1] * node_of(host[2], 0, g.n[2], g.bc[2]));
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (rest[c] != 0) atomicAdd(&dep[4 * hidx + c], (unsigned long long)rest[c]);
}

// Tile-local key -> zone offsets (x | y << 10 | z << 20) of a TX x TY x TZ
// tile.
template <int TX, int TY>
__device__ __forceinline__ int kdec_shape(int k)
{
    if constexpr (TX > 0 && TY > 0)
        return (k % TX) | (((k / TX) % TY) << 10) | ((k / (TX * TY)) << 20);
    else
        return 0;
}

// 27-node gather (Eq. Delta_vp) from the staged gas box around box
// position lb, channels in pairs on the packed single-precision FMA (each
// lane rounded once, as a scalar FMA), nodes x fastest.
template <int NB, int NC>
__device__ __forceinline__ void gather_box(const float *sgas, const int lb[3], int B0, int B1,
                                           const float w[3][3], float G[4])
{
    float2 G01 = make_float2(0.f, 0.f), G23 = make_float2(0.f, 0.f);
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        if (NC == 1 && c3 != 1) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (NB == 1 && b != 1) continue;
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                const float W = w[0][aa] * (w[1][b] * w[2][c3]);
                const float4 fv = reinterpret_cast<const float4 *>(sgas)[
                    (lb[0] + aa - 1) + B0 * ((lb[1] + b - 1) + B1 * (lb[2] + c3 - 1))];
                const float2 W2 = make_float2(W, W);
                G01 = __ffma2_rn(W2, make_float2(fv.x, fv.y), G01);
                G23 = __ffma2_rn(W2, make_float2(fv.z, fv.w), G23);
            }
        }
    }
    G[0] = G01.x; G[1] = G01.y; G[2] = G23.x; G[3] = G23.y;
}

// The same nodes in the same order from global memory, for a grain whose
// stencil leaves the staged box (rolled loop: a rare path).
template <int NB, int NC>
__device__ __forceinline__ void gather_global(const GridDev &g, const float *gas, const int host[3],
                                              const float w[3][3], float G[4])
{
#pragma unroll 1
    for (int nd = 0; nd < 27; ++nd) {
        const int aa = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
        if ((NB == 1 && b != 1) || (NC == 1 && c3 != 1)) continue;
        const float W = sel3(w[0], aa) * (sel3(w[1], b) * sel3(w[2], c3));
        const int ix = node_of(host[0], aa - 1, g.n[0], g.bc[0]);
        const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
        const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
        float fv[4];
        load_gas<float>(gas, ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz), fv);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) G[ch] += W * fv[ch];
    }
}

// The per-grain fixed-point rule into the shared deposit box (stencil
// inside the box around lb): rint(W D) for the other nodes, the host the
// remainder of rint(D).  Returns whether a channel was out of range.
template <int NB, int NC, class Add>
__device__ __forceinline__ bool deposit_box_per_grain(Add box_add, const int lb[3], int B0, int B1,
                                                      const float w[3][3], const float D[4])
{
    long long rest[4];
    bool big = false;
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        big |= !(fabsf(D[ch]) < 4.5e15f);
        rest[ch] = rround(D[ch]);
    }
    const int hl = lb[0] + B0 * (lb[1] + B1 * lb[2]);
#pragma unroll 1
    for (int nd = 0; nd < 27; ++nd) {
        const int aa = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
        if ((NB == 1 && b != 1) || (NC == 1 && c3 != 1) || nd == 13) continue;
        const float W = sel3(w[0], aa) * (sel3(w[1], b) * sel3(w[2], c3));
        const int lin = hl + (aa - 1) + B0 * ((b - 1) + B1 * (c3 - 1));
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const long long piece = rround(W * D[ch]);
            if (piece != 0) {
                box_add(ch, lin, piece);
                rest[ch] -= piece;
            }
        }
    }
#pragma unroll
    for (int ch = 0; ch < 4; ++ch)
        if (rest[ch] != 0) box_add(ch, hl, rest[ch]);
    return big;
}

// Out-of-line rare paths.  They work on copies (their addresses are taken
// here, not the hot loop's registers); the kernel argument is a grid
// constant, so the geometry structures are passed by reference to it.

// A grain that left its key zone in the first half drift: exact drift,
// boundaries, zone search and weights.  Returns false if it left the grid.
struct SlabExact {
    double q[3];
    float p[3], inc[3], w[3][3], iw[3], qf[3];
    int host[3];
};

// wk: the weighting (0 CIC, 1 TSC, 2 volume weighting).
template <int GEOM>
__device__ __noinline__ bool slab_exact_first_half(const GridDev &g, const PhysDev &ph, double shift,
                                                   int wk, float h, SlabExact &e)
{
#pragma unroll
    for (int d = 0; d < 3; ++d) e.inc[d] = 0.f;
    drift<float, GEOM>(ph, e.q, e.q, e.p, h, false, e.inc);
    if (!apply_bc<float, GEOM>(g, ph, shift, e.q, e.p)) return false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        zone_weights<float, GEOM>(g, d, wk, e.q[d], e.host[d], e.w[d], e.iw[d]);
        e.qf[d] = (float)e.q[d];
    }
    return true;
}

// Key of the next sort for a grain the in-zone prediction cannot place.
template <int GEOM>
__device__ __noinline__ int32_t slab_predict_key(const GridDev &g, const PhysDev &ph, double q[3],
                                                 const float p[3], float h)
{
    return predict_key<float, GEOM>(g, ph, q, p, h);
}

// MODE 0: the pusher and the shearing-box frame as the context has them;
// MODE > 0 fixes the exponential-midpoint pusher and, in the shearing box,
// the frame (1: orbital advection, 2: standard) at compile time, which
// drops the other branches from the hot code.
//
// One tile (tile index `tile` of `ntile` tiles; blocks of kSlabThreads
// threads, smem_raw the dynamic shared memory of slab_smem_bytes) as a
// device function: the step kernel below runs one tile per block, the
// batched persistent kernel runs tiles of many instances in turn.
// reuse: the block processes further tiles after this one (the batched
// persistent kernel): the tile ends with a block barrier and invalidates its
// copy barrier, so that the shared memory can be reused.
// TX > 0: the copy compiled for a TX x TY x TZ tile with TSC weights.  PRED: the gas
// predictor instead of the step: the same passes, chunks and deposit into
// TA.s.dep, from the grains' drag impulse at x^n (nothing is moved).
// Returns false when the wait for the gas box ran out (DUST_FLAG_TIMEOUT).
template <int GEOM, int FLAT, int MODE, int TX = 0, int TY = 0, int TZ = 0, bool PRED = false>
__device__ __forceinline__ bool slab_tile(const TiledArgs<float> &TA, const int tile, const int ntile,
                                          unsigned char *smem_raw, const bool reuse)
{
    using Sh = SlabShape<FLAT>;
    constexpr int NB = Sh::NB, NC = Sh::NC;
    const StepArgs<float> &A = TA.s;
    const GridDev &g = A.g;
    // tile extents: compile-time constants in a copy for one tile shape
    // (TX > 0; the flat pattern fixes the gridded directions), else the grid's
    constexpr bool FIX = TX > 0;
    const int T0 = FIX ? TX : g.T[0], T1 = FIX ? TY : g.T[1], T2 = FIX ? TZ : g.T[2];
    const int tvol = FIX ? TX * TY * TZ : g.tvol;
    auto Td = [&](int d) { return d == 0 ? T0 : (d == 1 ? T1 : T2); };
    // gridded directions, and the weights (the shape copies run TSC)
    auto gd = [&](int d) { return FIX ? (d == 0 || (d == 1 ? FLAT != 1 : FLAT != 2)) : g.n[d] > 1; };
    const int tsc = FIX ? 1 : TA.tsc;
    const bool vol = FIX ? false : TA.vol != 0;
    // the inline push reads ph; the rare out-of-line paths read the kernel
    // argument (the same values)
    PhysDev ph = A.ph;
    if (MODE > 0) ph.pusher = DUST_PUSHER_EM;
    if (GEOM == GEOM_SB && MODE == 1) ph.fargo = 1;
    if (GEOM == GEOM_SB && MODE == 2) ph.fargo = 0;
    const unsigned FULL = 0xffffffffu;

    // grains are read from S and written to O (the other store when the
    // sort's gather is fused into this kernel)
    const StoreDev<float> &S = A.s;
    const StoreDev<float> &O = TA.perm ? TA.dst : A.s;
    if (!PRED && (TA.emit_keys || TA.perm)) {
        // grains removed before the last sort sit after every zone's segment:
        // they keep the removed-grain key and are moved as they are
        const int D0 = TA.key_off[g.nkeys], D1 = (int)A.s.n;
        for (int gi = D0 + tile * blockDim.x + threadIdx.x; gi < D1; gi += ntile * blockDim.x) {
            if (TA.emit_keys) TA.key_out[gi] = (int32_t)g.nkeys;
            if (TA.perm) {
                const int src = TA.perm[gi];
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    O.q[d][gi] = S.q[d][src];
                    O.p[d][gi] = S.p[d][src];
                }
                O.id[gi] = TA.perm_id[gi];
                if (S.species) O.species[gi] = S.species[src];
                if (S.param) O.param[gi] = S.param[src];
            }
        }
        if (TA.emit_keys && tile == 0 && threadIdx.x == 0 && D1 > D0)
            atomicAdd(&TA.count_out[g.nkeys], (int32_t)(D1 - D0));
    }
    const int64_t kbase = (int64_t)tile * tvol;
    if (TA.key_off[kbase + tvol] <= TA.key_off[kbase]) return true;

    int B[3], o[3], tc[3];
    tc[0] = tile % g.nt[0];
    tc[1] = (tile / g.nt[0]) % g.nt[1];
    tc[2] = tile / (g.nt[0] * g.nt[1]);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int H = gd(d) ? 1 : 0;
        B[d] = Td(d) + 2 * H;
        o[d] = tc[d] * Td(d) - H;
    }
    const int bvol = B[0] * B[1] * B[2];
    // gas box first (128-byte aligned for the bulk tensor copy), then the
    // deposit box
    float *sgas = reinterpret_cast<float *>(smem_raw);
    unsigned long long *sdep = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)bvol * 4 * sizeof(float));
    // tile-local key -> zone offsets (x | y << 10 | z << 20), no runtime division
    int *kdec = reinterpret_cast<int *>(sdep + (size_t)bvol * 4);
    // the tile's zone offsets in the store, key_off[kbase .. kbase + tvol]
    int *skoff = kdec + ((tvol + 31) & ~31);
    // per warp: the zone (offset from the pass's first zone) of each grain of a pass
    unsigned short *sztab = reinterpret_cast<unsigned short *>(skoff + ((tvol + 32) & ~31));
    float *srec = reinterpret_cast<float *>(sztab + (kSlabThreads / 32) * kSlabCap);  // [warps][13][kRecStride]
    // the tile's zone geometry, per direction d at toff[d]: centre (double and
    // float) and inverse width; radial centre / width; polar lower edges
    const int toff[3] = {0, T0, T0 + T1};
    const int tsum = T0 + T1 + T2;
    double *szcd = reinterpret_cast<double *>(srec + (kSlabThreads / 32) * kRecFields * kRecStride);
    float *szcf = reinterpret_cast<float *>(szcd + tsum);
    float *szif = szcf + tsum;
    float *sznu = szif + tsum;          // [T0]
    float *szlo = sznu + T0;        // [T1 + 1]
    // volume weighting: inverse shell volumes to the lower and upper
    // neighbouring nodes, radial zones then polar zones ([2 (T0 + T1)])
    float *szvl = szlo + T1 + 1, *szvh = szvl + T0 + T1;
    unsigned long long *sbar = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(szvh + T0 + T1) + 7) & ~(uintptr_t)7);
    // the gas box by one bulk tensor copy, overlapping the tables below
    gas_box_begin<float>(TA.gas_tmap, sgas, o, bvol, sbar, TA.wait_extra_tx);
    for (int t = threadIdx.x; t < tsum + T1 + 1; t += blockDim.x) {
        if (t < tsum) {
            const int d = t < toff[1] ? 0 : (t < toff[2] ? 1 : 2);
            const int z = tc[d] * Td(d) + (t - toff[d]);
            const bool ok = gd(d) && z < g.n[d];
            szcd[t] = ok ? g.zc[d][z] : 0.0;
            szcf[t] = ok ? g.zc_f[d][z] : 0.f;
            szif[t] = ok ? g.ziw_f[d][z] : 0.f;
            if (d == 0 && (GEOM == GEOM_CYL || GEOM == GEOM_SPH)) sznu[t] = ok ? g.znu_f[0][z] : 0.f;
        } else if (GEOM == GEOM_SPH) {
            const int z = tc[1] * T1 + (t - tsum);
            szlo[t - tsum] = (g.n[1] > 1 && z <= g.n[1]) ? g.zlo_f[1][z] : 0.f;
        }
    }
    if ((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && vol) {
        for (int t = threadIdx.x; t < T0 + (GEOM == GEOM_SPH ? T1 : 0); t += blockDim.x) {
            const int d = t < T0 ? 0 : 1;
            const int z = d == 0 ? tc[0] * T0 + t : tc[1] * T1 + (t - T0);
            float vl = 0.f, vh = 0.f;
            if (z < g.n[d]) {
                const double c = g.zc[d][z];
                vl = (float)(1.0 / vol_shell<GEOM>(d, vol_node(g, d, z - 1), c));
                vh = (float)(1.0 / vol_shell<GEOM>(d, c, vol_node(g, d, z + 1)));
            }
            szvl[t] = vl;
            szvh[t] = vh;
        }
    }
    for (int k = threadIdx.x; k < tvol; k += blockDim.x) {
        const int kx = k % T0, ky = (k / T0) % T1, kz = k / (T0 * T1);
        kdec[k] = kx | (ky << 10) | (kz << 20);
    }
    // store positions fit in 32 bits (fewer than 2^31 grains)
    for (int k = threadIdx.x; k <= tvol; k += blockDim.x) skoff[k] = TA.key_off[kbase + k];

    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 4; ++c) sdep[c * bvol + lin] = 0ull;
    }
    __syncthreads();
    if (!gas_box_finish<float>(g, A.gas, TA.gas_tmap, sgas, o, B, sbar, A.status, TA.wait_ns)) return false;

    // The deposit box.  In a tile of at most 65535 grains each word of the box
    // takes at most one piece per grain, so a piece v with |v| < 2^31 is
    // added exactly as two 32-bit counters that need no carry: the sum of
    // the pieces' low 16 bits (unsigned, below 2^32) and of v >> 16 (signed,
    // below 2^31 in size); the word is 65536 * high + low.  Both adds return
    // nothing, so no lane waits for the shared-memory round trip.  Larger
    // pieces go to the global deposit directly.  A denser tile keeps the box
    // as int64 words added as two 32-bit atomics with the carry.
    unsigned *blo = reinterpret_cast<unsigned *>(sdep);
    int *bhi = reinterpret_cast<int *>(blo + 4 * bvol);
    // Measured: the split form pays in the 3-D tiles (27 nodes per zone); the
    // 2-D tiles of the batched x-z boxes ran 9% slower with it than with the
    // int64 words, so the 2-D copies keep those.
    const bool split = FLAT == 0 && skoff[tvol] - skoff[0] <= 65535;
    auto box_add_split = [&](int ch, int lin, int v) {
        atomicAdd(&blo[ch * bvol + lin], (unsigned)v & 0xffffu);
        atomicAdd(&bhi[ch * bvol + lin], v >> 16);
    };
    auto box_add = [&](int ch, int lin, long long v) {
        if (!split) {
            shared_add_i64(&sdep[ch * bvol + lin], v);
        } else if (v >= -2147483647LL && v <= 2147483647LL) {
            box_add_split(ch, lin, (int)v);
        } else {
            box_piece_to_global(g, A.dep, o[0], o[1], o[2], B[0], B[1], lin, ch, v);
        }
    };

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int a = lane % 3, kq = lane / 3;
    const int base = lane - a;
    const float h = (float)(0.5 * A.dt), dt = (float)A.dt;
    int nremoved = 0;
    float moved = 0.f;
    bool big = false;

    // Each warp takes an equal range [zw0, zw1) of the tile's zones (keys)
    // and walks its grains, contiguous in the store, in passes of at most
    // kSlabCap grains that end on chunk boundaries (a zone's end, or its
    // start plus a multiple of kSlabCap), so each zone's part of a pass is
    // one whole chunk of its run and is quantised in that pass: nothing is
    // carried between passes.  A pass spans as many zones as its grains
    // fill; its owner phase takes them ten at a time.
    const int zw0 = (warp * tvol) / nwarps, zw1 = ((warp + 1) * tvol) / nwarps;
    const int Gend = skoff[zw1];
    float *rb = srec + warp * (kRecFields * kRecStride);
    unsigned short *zt = sztab + warp * kSlabCap;
    int zc = zw0;  // the zone holding grain P0: skoff[zc] <= P0 < skoff[zc + 1]
    for (int P0 = skoff[zw0], P1; P0 < Gend; P0 = P1) {
        // skip the zones that end at or before P0 (32 at a time; offsets are
        // nondecreasing, so the ballot is a prefix)
        for (;;) {
            const int z = zc + 1 + lane;
            const int c = __popc(__ballot_sync(FULL, z <= zw1 && skoff[z] <= P0));
            zc += c;
            if (c < 32) break;
        }
        // the pass [P0, P1) over the zones [zc, zc + nz)
        int nz = 1;
        if (skoff[zc + 1] > P0 + kSlabCap) {
            P1 = P0 + kSlabCap;  // one chunk of a dense zone
        } else {
            // the last zone boundary at most kSlabCap grains from P0
            const int lim = P0 + kSlabCap;
            int zb = zc + 1;
            for (;;) {
                const int z = zb + 1 + lane;
                const int c = __popc(__ballot_sync(FULL, z <= zw1 && skoff[z] <= lim));
                zb += c;
                if (c < 32) break;
            }
            P1 = skoff[zb];
            nz = zb - zc;
        }
        // zone of each grain of the pass, as its offset from zc
        for (int zp = lane; zp < nz; zp += 32) {
            const int s0 = max(skoff[zc + zp], P0) - P0, s1 = min(skoff[zc + zp + 1], P1) - P0;
            for (int t = s0; t < s1; ++t) zt[t] = (unsigned short)zp;
        }
        __syncwarp();
        // the source positions of the first grains of the next pass; their
        // columns are prefetched after the push, ahead of that pass's loads
        int src_g = -1;
        if (P1 + lane < Gend) src_g = TA.perm ? TA.perm[P1 + lane] : P1 + lane;
        {
            // ---- push: one grain per lane, consecutive grains on consecutive
            // lanes (coalesced), each relative to its own key zone.  Source
            // positions two iterations ahead: the next iteration's grain
            // columns are prefetched into L2 while this one runs, and the
            // permutation load is off the grain loads' dependency chain
            int src_next = (TA.perm && P0 + lane < P1) ? TA.perm[P0 + lane] : 0;
            int src_nx2 = (TA.perm && P0 + lane + 32 < P1) ? TA.perm[P0 + lane + 32] : 0;
            for (int gi = P0 + lane; gi < P1; gi += 32) {
                const int src = TA.perm ? src_next : gi;
                if (gi + 32 < P1) prefetch_grain(S, TA.perm ? src_nx2 : gi + 32);
                if (TA.perm) {
                    src_next = src_nx2;
                    if (gi + 64 < P1) src_nx2 = TA.perm[gi + 64];
                }
                const int zp = zt[gi - P0];
                // the records of a zone start min(zp, 15) slots after its
                // grains' positions in the pass (staggers the owner lanes of
                // neighbouring zones across banks); never decreasing with zp,
                // so no two grains of a pass share a slot
                const int kq2 = min(zp, 15);
                const int kd = FIX ? kdec_shape<TX, TY>(zc + zp) : kdec[zc + zp];
                const int lx = kd & 1023, ly = (kd >> 10) & 1023, lz = kd >> 20;
                const int zx = tc[0] * T0 + lx, zy = tc[1] * T1 + ly, zz = tc[2] * T2 + lz;
                const int hx = lx + 1, hy = ly + (NB == 3 ? 1 : 0), hz = lz + (NC == 3 ? 1 : 0);
                const int lid[3] = {toff[0] + lx, toff[1] + ly, toff[2] + lz};
                double zcd[3];
                float zcf[3], zif[3];
                float znu = 0.f, zlo = 0.f, zhi = 0.f, zhw = 0.f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    zcd[d] = szcd[lid[d]];
                    zcf[d] = szcf[lid[d]];
                    zif[d] = szif[lid[d]];
                }
                float zvl[2] = {0.f, 0.f}, zvh[2] = {0.f, 0.f};
                if (GEOM == GEOM_CYL || GEOM == GEOM_SPH) {
                    znu = sznu[lx];
                    if (vol) {
                        zvl[0] = szvl[lx];
                        zvh[0] = szvh[lx];
                        if (GEOM == GEOM_SPH) {
                            zvl[1] = szvl[T0 + ly];
                            zvh[1] = szvh[T0 + ly];
                        }
                    }
                }
                if (GEOM == GEOM_SPH) {
                    zlo = szlo[ly];
                    zhi = szlo[ly + 1];
                    zhw = 0.5f / zif[1];
                }
                // the grain's weights and deposit impulse for the zone's
                // owners (zero impulse: the grain deposits by itself)
                float w[3][3] = {{0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 1.f, 0.f}};
                float D[4] = {0.f, 0.f, 0.f, 0.f};
                bool grp_ok = false;
                if constexpr (PRED) {
                    // ---- gas predictor (Sec. 3.1): the drag impulse over half
                    // a step, dt/2 m (v - v_g) / max(tau, dt), of the grain at
                    // x^n, gathered and deposited at x^n.  Grains whose x^n
                    // lies in their key zone go to the zone's chunks; the
                    // others take the exact zone search and the per-grain rule.
                    const double q[3] = {S.q[0][src], S.q[1][src], S.q[2][src]};
                    if ((__double_as_longlong(q[0]) & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll) {
                        const float pn[3] = {S.p[0][src], S.p[1][src], S.p[2][src]};
                        const int sp = S.species ? S.species[src] : 0;
                        float u[3] = {0.f, 0.f, 0.f}, qf[3], dl[3];
                        bool here = true;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            float zc3 = (float)q[d];
                            if (gd(d)) {
                                u[d] = __double2float_rn(q[d] - zcd[d]);
                                zc3 = zcf[d];
                            }
                            qf[d] = zc3 + u[d];
                            dl[d] = u[d] * zif[d];
                            if (gd(d)) here &= fabsf(dl[d]) <= 0.50001f;
                        }
                        int host[3] = {zx, zy, zz};
                        int lb[3] = {hx, hy, hz};
                        bool inbox = true;
                        if (here) {
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                if (!gd(d)) continue;
                                if ((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && d == 0) {
                                    if (vol) w_vol_f<GEOM>(0, u[0], zcf[0], zvl[0], zvh[0], w[0]);
                                    else if (GEOM == GEOM_CYL) w_cyl<float>(tsc, dl[0], znu, w[0]);
                                    else w_sphr<float>(tsc, dl[0], znu, w[0]);
                                } else if (GEOM == GEOM_SPH && d == 1) {
                                    if (vol) w_vol_f<GEOM>(1, u[1], zcf[1], zvl[1], zvh[1], w[1]);
                                    else w_theta<float>(tsc, qf[1], zlo, zhi, u[1], zhw, w[1]);
                                } else {
                                    w_cart<float>(tsc, dl[d], w[d]);
                                }
                            }
                        } else {
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                float iwd;
                                zone_weights<float, GEOM>(g, d, vol ? 2 : (tsc & 1), q[d], host[d], w[d], iwd);
                                qf[d] = (float)q[d];
                                int l = host[d] - o[d];
                                if (gd(d) && g.bc[d] == DUST_BC_PERIODIC) {
                                    if (l < 0) l += g.n[d];
                                    else if (l >= B[d]) l -= g.n[d];
                                }
                                lb[d] = l;
                                if (gd(d)) inbox &= (l >= 1) && (l <= B[d] - 2);
                            }
                        }
                        float G[4] = {0.f, 0.f, 0.f, 0.f};
                        if (inbox) gather_box<NB, NC>(sgas, lb, B[0], B[1], w, G);
                        else gather_global<NB, NC>(g, A.gas, host, w, G);
                        const float value = S.param ? S.param[src] : A.sp.tau_f[sp];
                        const float tau = stopping_time<float, GEOM>(ph, A.sp.mode[sp], value, qf, G[0]);
                        const float taup = fmaxf(tau, fabsf(dt));
                        const float coef = 0.5f * dt * A.sp.mqf[sp] / taup;
                        const float Dq[4] = {coef * (pn[0] - G[1]), coef * (pn[1] - G[2]), coef * (pn[2] - G[3]),
                                             0.f};
                        if (here) {
#pragma unroll
                            for (int c = 0; c < 4; ++c) D[c] = Dq[c];
                            grp_ok = true;
                        } else if (inbox) {
                            big |= deposit_box_per_grain<NB, NC>(box_add, lb, B[0], B[1], w, Dq);
                        } else {
                            deposit_fixed_rolled<NB, NC>(g, A.dep, host, w, Dq, A.status);
                        }
                    }
                } else {
                // ---- own grain: first half drift and weights, relative to the
                // key zone (fast); grains that left it take the exact path
                double q[3] = {0.0, 0.0, 0.0};
                float pn[3] = {0.f, 0.f, 0.f};
                float iw[3] = {0.f, 0.f, 0.f};
                float inc1[3] = {0.f, 0.f, 0.f};
                float qf[3] = {0.f, 0.f, 0.f};  // half-step coordinates
                float u[3] = {0.f, 0.f, 0.f}, zc3[3] = {0.f, 0.f, 0.f};
                int32_t nkey = (int32_t)g.nkeys;   // next sort key (removed: nkeys)
                int host[3] = {0, 0, 0};
                int sp = 0;
                bool live = false, ingroup = false, gone = false;
                {
                    q[0] = S.q[0][src]; q[1] = S.q[1][src]; q[2] = S.q[2][src];
                    live = !isnan(q[0]);
                    if (live) {
                        pn[0] = S.p[0][src]; pn[1] = S.p[1][src]; pn[2] = S.p[2][src];
                        sp = S.species ? S.species[src] : 0;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (gd(d)) { u[d] = __double2float_rn(q[d] - zcd[d]); zc3[d] = zcf[d]; }
                            else { u[d] = 0.f; zc3[d] = (float)q[d]; }
                        }
                        // first half drift (Eq. exp_midpoint; Eq. drift1_cylindrical;
                        // spherical r, theta, phi in turn)
                        if (GEOM == GEOM_CYL) {
                            inc1[0] = h * pn[0]; u[0] += inc1[0];
                            const float R = zc3[0] + u[0];
                            inc1[1] = h * pn[1] / (R * R); u[1] += inc1[1];
                            inc1[2] = h * pn[2]; u[2] += inc1[2];
                        } else if (GEOM == GEOM_SPH) {
                            inc1[0] = h * pn[0]; u[0] += inc1[0];
                            const float r = zc3[0] + u[0];
                            inc1[1] = h * pn[1] / (r * r); u[1] += inc1[1];
                            const float st = sinf(zc3[1] + u[1]);
                            inc1[2] = h * pn[2] / (r * r * st * st); u[2] += inc1[2];
                        } else if (GEOM == GEOM_SB) {
                            inc1[0] = h * pn[0]; u[0] += inc1[0];
                            inc1[1] = ph.fargo ? h * (pn[1] - ph.q_om_f * (zc3[0] + u[0])) : h * pn[1];
                            u[1] += inc1[1];
                            inc1[2] = h * pn[2]; u[2] += inc1[2];
                        } else {
#pragma unroll
                            for (int d = 0; d < 3; ++d) { inc1[d] = h * pn[d]; u[d] += inc1[d]; }
                        }
                        float dl[3];
                        ingroup = true;
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            qf[d] = zc3[d] + u[d];
                            dl[d] = u[d] * zif[d];
                            if (gd(d)) ingroup &= fabsf(dl[d]) <= 0.50001f;
                        }
                        if (ingroup) {
                            host[0] = zx; host[1] = zy; host[2] = zz;
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                iw[d] = zif[d];
                                if (!gd(d)) continue;
                                if ((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && d == 0) {
                                    if (vol) w_vol_f<GEOM>(0, u[0], zcf[0], zvl[0], zvh[0], w[0]);
                                    else if (GEOM == GEOM_CYL) w_cyl<float>(tsc, dl[0], znu, w[0]);
                                    else w_sphr<float>(tsc, dl[0], znu, w[0]);
                                } else if (GEOM == GEOM_SPH && d == 1) {
                                    if (vol) w_vol_f<GEOM>(1, u[1], zcf[1], zvl[1], zvh[1], w[1]);
                                    else w_theta<float>(tsc, qf[1], zlo, zhi, u[1], zhw, w[1]);
                                } else {
                                    w_cart<float>(tsc, dl[d], w[d]);
                                }
                            }
                        } else {
                            // exact path: double-precision half drift, boundaries
                            // and zone search (out of line)
                            SlabExact ex;
#pragma unroll
                            for (int d = 0; d < 3; ++d) { ex.q[d] = q[d]; ex.p[d] = pn[d]; }
                            const bool in = slab_exact_first_half<GEOM>(g, A.ph, shift_mid_of(A), vol ? 2 : (tsc & 1),
                                                                        h, ex);
#pragma unroll
                            for (int d = 0; d < 3; ++d) { q[d] = ex.q[d]; pn[d] = ex.p[d]; inc1[d] = ex.inc[d]; }
                            if (!in) {
                                q[0] = __longlong_as_double(0x7ff8000000000000LL);
                                if (!TA.perm) S.q[0][gi] = q[0];
                                ++nremoved;
                                live = false;
                                gone = true;
                            } else {
#pragma unroll
                                for (int d = 0; d < 3; ++d) {
                                    host[d] = ex.host[d];
                                    iw[d] = ex.iw[d];
                                    qf[d] = ex.qf[d];
#pragma unroll
                                    for (int k = 0; k < 3; ++k) w[d][k] = ex.w[d][k];
                                }
                            }
                        }
                    }
                }
                grp_ok = live && ingroup;
                float G[4] = {0.f, 0.f, 0.f, 0.f};
                // ---- own grain: kick, second half drift, deposit impulse
                if (live) {
                    int lb[3] = {hx, hy, hz};
                    bool inbox = true;
                    if (!ingroup) {
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            int l = host[d] - o[d];
                            if (gd(d) && g.bc[d] == DUST_BC_PERIODIC) {
                                if (l < 0) l += g.n[d];
                                else if (l >= B[d]) l -= g.n[d];
                            }
                            lb[d] = l;
                            if (gd(d)) inbox &= (l >= 1) && (l <= B[d] - 2);
                        }
                    }
                    // 27-node gather (Eq. Delta_vp) from the staged gas box; the
                    // grains of one zone read the same nodes (broadcast loads)
                    if (inbox) {
                        // channels in pairs on the packed single-precision
                        // FMA (each lane rounded once, as a scalar FMA)
                        float2 G01 = make_float2(0.f, 0.f), G23 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c3 = 0; c3 < 3; ++c3) {
                            if (NC == 1 && c3 != 1) continue;
#pragma unroll
                            for (int b = 0; b < 3; ++b) {
                                if (NB == 1 && b != 1) continue;
#pragma unroll
                                for (int aa = 0; aa < 3; ++aa) {
                                    const float W = w[0][aa] * (w[1][b] * w[2][c3]);
                                    const float4 fv = reinterpret_cast<const float4 *>(sgas)[
                                        (lb[0] + aa - 1) + B[0] * ((lb[1] + b - 1) + B[1] * (lb[2] + c3 - 1))];
                                    const float2 W2 = make_float2(W, W);
                                    G01 = __ffma2_rn(W2, make_float2(fv.x, fv.y), G01);
                                    G23 = __ffma2_rn(W2, make_float2(fv.z, fv.w), G23);
                                }
                            }
                        }
                        G[0] = G01.x; G[1] = G01.y; G[2] = G23.x; G[3] = G23.y;
                    } else {
                        // rare: the stencil leaves the staged box; the same
                        // nodes in the same order from global memory, in a
                        // rolled loop (keeps the hot code small)
#pragma unroll 1
                        for (int nd = 0; nd < 27; ++nd) {
                            const int aa = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
                            if ((NB == 1 && b != 1) || (NC == 1 && c3 != 1)) continue;
                            const float W = sel3(w[0], aa) * (sel3(w[1], b) * sel3(w[2], c3));
                            const int ix = node_of(host[0], aa - 1, g.n[0], g.bc[0]);
                            const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
                            const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
                            float fv[4];
                            load_gas<float>(A.gas, ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz), fv);
#pragma unroll
                            for (int ch = 0; ch < 4; ++ch) G[ch] += W * fv[ch];
                        }
                    }
                    float tau, E, cg, h1;
                    if (!S.param && ((A.sp.coef_const >> sp) & 1u)) {
                        // the species' propagators for this dt (host, once)
                        tau = A.sp.tau_eff_f[sp];
                        E = A.sp.E_f[sp];
                        cg = A.sp.cg_f[sp];
                        h1 = A.sp.h1_f[sp];
                    } else {
                        const float value = S.param ? S.param[src] : A.sp.tau_f[sp];
                        tau = stopping_time<float, GEOM>(ph, A.sp.mode[sp], value, qf, G[0]);
                        const float x = dt / tau;
                        E = expf(-x);
                        cg = -expm1f(-x);
                        h1 = (x == 0.f) ? dt : dt * cg / x;
                    }
                    const float vg[3] = {G[1], G[2], G[3]};
                    float pp[3], acc3[3], dH[3], inc2[3];
                    kick_any<float, GEOM>(ph, qf, pn, vg, tau, dt, E, cg, h1, pp, acc3, dH);
                    if (ingroup) {
                        // second half drift with the half-step metric factors, then
                        // one double-precision update by the summed increment
                        if (GEOM == GEOM_CYL) {
                            inc2[0] = h * pp[0];
                            inc2[1] = h * pp[1] / (qf[0] * qf[0]);
                            inc2[2] = h * pp[2];
                        } else if (GEOM == GEOM_SPH) {
                            const float st = sinf(qf[1]);
                            inc2[0] = h * pp[0];
                            inc2[1] = h * pp[1] / (qf[0] * qf[0]);
                            inc2[2] = h * pp[2] / (qf[0] * qf[0] * st * st);
                        } else if (GEOM == GEOM_SB) {
                            inc2[0] = h * pp[0];
                            inc2[1] = ph.fargo ? h * (pp[1] - ph.q_om_f * qf[0]) : h * pp[1];
                            inc2[2] = h * pp[2];
                        } else {
#pragma unroll
                            for (int d = 0; d < 3; ++d) inc2[d] = h * pp[d];
                        }
#pragma unroll
                        for (int d = 0; d < 3; ++d) q[d] += (double)(inc1[d] + inc2[d]);
                    } else {
                        const double qm[3] = {q[0], q[1], q[2]};
                        drift<float, GEOM>(ph, q, qm, pp, h, true, inc2);
                    }
                    float pnew[3] = {pp[0], pp[1], pp[2]};
                    // certainly inside the grid, judged from the single-
                    // precision end offset from the key zone's centre (error
                    // ~1e-7 zones): still inside the key zone (margin 1e-3),
                    // or, on a uniform direction, less than two zones from a
                    // key zone at least two zones from the edges; otherwise
                    // the exact boundary treatment
                    bool inner = ingroup;
                    if (inner) {
                        const int zk[3] = {zx, zy, zz};
#pragma unroll
                        for (int d = 0; d < 3; ++d) {
                            if (gd(d)) {
                                const float te = fabsf((u[d] + inc2[d]) * zif[d]);
                                inner &= te < 0.499f ||
                                         (g.edge_kind[d] == EDGE_UNIFORM && te < 1.999f && zk[d] >= 2 &&
                                          zk[d] < g.n[d] - 2);
                            } else {
                                inner &= inside(g, d, q[d]);
                            }
                        }
                    }
                    const bool alive = inner || apply_bc<float, GEOM>(g, ph, shift_end_of(A), q, pnew);
                    const float mq = A.sp.mqf[sp];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        D[c] = -mq * ((pp[c] - pn[c]) - dt * acc3[c]);
                        D[3] += D[c] * dH[c];
                    }
                    if (!(isfinite(pp[0]) && isfinite(pp[1]) && isfinite(pp[2])))
                        atomicOr(&A.status[ST_FLAGS], DUST_FLAG_NAN);
#pragma unroll
                    for (int d = 0; d < 3; ++d) moved = fmaxf(moved, fabsf(inc1[d] + inc2[d]) * iw[d]);
                    if (!ingroup) {
                        // per-grain fixed-point rule for a grain outside its key zone
                        if (inbox) {
                            long long rest[4];
#pragma unroll
                            for (int ch = 0; ch < 4; ++ch) rest[ch] = rround(D[ch]);
                            const int hl = lb[0] + B[0] * (lb[1] + B[1] * lb[2]);
#pragma unroll 1
                            for (int nd = 0; nd < 27; ++nd) {
                                const int aa = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
                                if ((NB == 1 && b != 1) || (NC == 1 && c3 != 1) || nd == 13) continue;
                                const float W = sel3(w[0], aa) * (sel3(w[1], b) * sel3(w[2], c3));
                                const int lin = hl + (aa - 1) + B[0] * ((b - 1) + B[1] * (c3 - 1));
#pragma unroll
                                for (int ch = 0; ch < 4; ++ch) {
                                    const long long piece = rround(W * D[ch]);
                                    if (piece != 0) {
                                        box_add(ch, lin, piece);
                                        rest[ch] -= piece;
                                    }
                                }
                            }
#pragma unroll
                            for (int ch = 0; ch < 4; ++ch)
                                if (rest[ch] != 0) box_add(ch, hl, rest[ch]);
                        } else {
                            deposit_fixed_rolled<NB, NC>(g, A.dep, host, w, D, A.status);
                        }
                    }
                    if (!alive) {
                        q[0] = __longlong_as_double(0x7ff8000000000000LL);
                        ++nremoved;
                    }
                    O.q[0][gi] = q[0]; O.q[1][gi] = q[1]; O.q[2][gi] = q[2];
                    O.p[0][gi] = pnew[0]; O.p[1][gi] = pnew[1]; O.p[2][gi] = pnew[2];
                    if (TA.emit_keys && alive) {
                        // key for the next sort: the zone of the next step's
                        // half-step position (same dt), relative to this key
                        // zone in single precision; the exact prediction when
                        // the grain moves more than one zone or crosses the grid
                        bool fast = ingroup;
                        int zn[3] = {zx, zy, zz}, kk[3] = {0, 0, 0};
                        if (fast) {
                            float un[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) un[d] = u[d] + inc2[d];
                            if (GEOM == GEOM_CYL) {
                                un[0] += h * pnew[0];
                                const float R = zc3[0] + un[0];
                                un[1] += h * pnew[1] / (R * R);
                                un[2] += h * pnew[2];
                            } else if (GEOM == GEOM_SPH) {
                                un[0] += h * pnew[0];
                                const float r = zc3[0] + un[0];
                                un[1] += h * pnew[1] / (r * r);
                                const float st = sinf(zc3[1] + un[1]);
                                un[2] += h * pnew[2] / (r * r * st * st);
                            } else if (GEOM == GEOM_SB) {
                                un[0] += h * pnew[0];
                                un[1] += ph.fargo ? h * (pnew[1] - ph.q_om_f * (zc3[0] + un[0])) : h * pnew[1];
                                un[2] += h * pnew[2];
                            } else {
#pragma unroll
                                for (int d = 0; d < 3; ++d) un[d] += h * pnew[d];
                            }
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                if (!gd(d)) continue;
                                // zone offset floor(t + 1/2) for |t| < 3/2, by comparisons
                                const float t = un[d] * zif[d];
                                const int k = (t >= 0.5f ? 1 : 0) - (t < -0.5f ? 1 : 0);
                                zn[d] += k;
                                kk[d] = k;
                                fast &= fabsf(t) < 1.5f && zn[d] >= 0 && zn[d] < g.n[d];
                            }
                        }
                        if (fast) {
                            // key of the neighbouring zone from this tile's
                            // coordinates (no division)
                            const int lloc[3] = {lx, ly, lz};
                            int tt[3], ll[3];
#pragma unroll
                            for (int d = 0; d < 3; ++d) {
                                int l = lloc[d] + kk[d], t = tc[d];
                                if (l < 0) { l += Td(d); --t; }
                                else if (l >= Td(d)) { l -= Td(d); ++t; }
                                ll[d] = l;
                                tt[d] = t;
                            }
                            nkey = (tt[0] + g.nt[0] * (tt[1] + g.nt[1] * tt[2])) * tvol +
                                   ll[0] + T0 * (ll[1] + T1 * ll[2]);
                        } else {
                            double qk[3] = {q[0], q[1], q[2]};
                            const float pk[3] = {pnew[0], pnew[1], pnew[2]};
                            nkey = slab_predict_key<GEOM>(g, A.ph, qk, pk, h);
                        }
                    }
                }
                if (TA.perm) {
                    // the rest of the gather: a grain removed in the first
                    // half drift, and the columns the step does not change
                    if (gone) {
                        O.q[0][gi] = q[0]; O.q[1][gi] = q[1]; O.q[2][gi] = q[2];
                        O.p[0][gi] = pn[0]; O.p[1][gi] = pn[1]; O.p[2][gi] = pn[2];
                    }
                    O.id[gi] = TA.perm_id[gi];
                    if (S.species) O.species[gi] = S.species[src];
                    if (S.param) O.param[gi] = S.param[src];
                }
                if (TA.emit_keys) {
                    TA.key_out[gi] = nkey;
                    // count runs of equal keys on consecutive lanes (the lanes
                    // of this pass iteration are 0 .. m-1): one atomic per run
                    const int m = min(32, P1 - (gi - lane));
                    const unsigned pm = m == 32 ? FULL : ((1u << m) - 1u);
                    const int prev = __shfl_up_sync(pm, nkey, 1);
                    const bool start = lane == 0 || prev != nkey;
                    const unsigned starts = __ballot_sync(pm, start);
                    if (start) {
                        const unsigned later = starts & ~((2u << lane) - 1u);
                        const int end = later ? __ffs(later) - 1 : m;
                        atomicAdd(&TA.count_out[nkey], end - lane);
                    }
                }
                }  // step
                // record for the zone's deposit owners (grains outside their
                // key zone, and removed ones, carry a zero impulse)
                const int slot = gi - P0 + kq2;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    rb[k * kRecStride + slot] = w[0][k];
                    rb[(3 + k) * kRecStride + slot] = w[1][k];
                    rb[(6 + k) * kRecStride + slot] = w[2][k];
                }
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) rb[(9 + ch) * kRecStride + slot] = grp_ok ? D[ch] : 0.f;
            }
            if (src_g >= 0) prefetch_grain(S, src_g);
            __syncwarp();
            // ---- deposit, ten zones of the pass at a time: the three owner
            // lanes of a zone accumulate its chunk in this pass (id order)
            // into their x slabs
            for (int z0 = zc; z0 < zc + nz; z0 += 10) {
                const int zl = z0 + kq;
                const bool kok = lane < 30 && zl < zc + nz;
                int za = 0, zb = 0;
                if (kok) {
                    za = max(skoff[zl], P0);
                    zb = min(skoff[zl + 1], P1);
                }
                const bool own = kok && zb > za;
                if (!__any_sync(FULL, own)) continue;
                // owner zone's position in the tile box
                const int okd = own ? (FIX ? kdec_shape<TX, TY>(zl) : kdec[zl]) : 0;
                const int ohx = (okd & 1023) + 1, ohy = ((okd >> 10) & 1023) + (NB == 3 ? 1 : 0),
                          ohz = (okd >> 20) + (NC == 3 ? 1 : 0);
                // channels in pairs (0, 1) and (2, 3) on the packed single-precision
                // FMA and add (each lane rounded once, as the scalar operations)
                float2 acc[NB][NC][2];
                float2 S2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
#pragma unroll
                for (int b = 0; b < NB; ++b)
#pragma unroll
                    for (int c = 0; c < NC; ++c)
#pragma unroll
                        for (int hc = 0; hc < 2; ++hc) acc[b][c][hc] = make_float2(0.f, 0.f);
                float Sabs = 0.f;  // sum over the chunk of the largest |channel| of each grain
                if (own) {
                    const int sk = min(zl - zc, 15);
                    const int s0 = za - P0 + sk, s1 = zb - P0 + sk;
                    const float *rx = rb + a * kRecStride;
                    auto one = [&](int sl) {
                        const float wx = rx[sl];
                        const float2 De01 = make_float2(rb[9 * kRecStride + sl], rb[10 * kRecStride + sl]);
                        const float2 De23 = make_float2(rb[11 * kRecStride + sl], rb[12 * kRecStride + sl]);
#pragma unroll
                        for (int b = 0; b < NB; ++b) {
                            const float wxy = wx * rb[(3 + (NB == 3 ? b : 1)) * kRecStride + sl];
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                const float W = wxy * rb[(6 + (NC == 3 ? c : 1)) * kRecStride + sl];
                                const float2 W2 = make_float2(W, W);
                                acc[b][c][0] = __ffma2_rn(W2, De01, acc[b][c][0]);
                                acc[b][c][1] = __ffma2_rn(W2, De23, acc[b][c][1]);
                            }
                        }
                        S2[0] = __fadd2_rn(S2[0], De01);
                        S2[1] = __fadd2_rn(S2[1], De23);
                        Sabs += fmaxf(fmaxf(fabsf(De01.x), fabsf(De01.y)), fmaxf(fabsf(De23.x), fabsf(De23.y)));
                    };
                    int sl = s0;
                    for (; sl + 1 < s1; sl += 2) {
                        one(sl);
                        one(sl + 1);
                    }
                    if (sl < s1) one(sl);
                }
                __syncwarp();

                // ---- quantise the chunk and add it to the deposit box (the
                // predictor's impulse has no energy channel)
                constexpr int NCH = PRED ? 3 : 4;
                long long ps[4] = {0, 0, 0, 0};
                // every chunk sum of a channel is at most the sum of the grains'
                // |impulse| in it (the weights lie in [0, 1]); below 2^31 (with a
                // margin for the sums' rounding) the 32-bit rounding instruction
                // gives the same integer as the 64-bit one, at a fraction of its
                // cost on this GPU.  Decided for the whole warp, so that its
                // lanes never run both forms.
                const bool narrow = __all_sync(FULL, !own || Sabs < 2147000000.f);
                auto quantise = [&](auto round_piece, auto add_piece) {
#pragma unroll
                    for (int b = 0; b < NB; ++b)
#pragma unroll
                        for (int c = 0; c < NC; ++c) {
                            if (a == 1 && b == Sh::BC && c == Sh::CC) continue;  // host: remainder
                            const int lin = (ohx + a - 1) + B[0] * ((ohy + b - Sh::BC) + B[1] * (ohz + c - Sh::CC));
#pragma unroll
                            for (int ch = 0; ch < NCH; ++ch) {
                                const float v = (ch & 1) ? acc[b][c][ch >> 1].y : acc[b][c][ch >> 1].x;
                                const long long piece = round_piece(v);
                                // no test for zero: a chunk sum is rarely exactly
                                // zero, and the test cost more than the adds it saved
                                add_piece(ch, lin, piece);
                                ps[ch] += piece;
                            }
                        }
                };
                if (own) {
                    if (narrow && split) {
                        // the common form: 32-bit roundings, carry-free adds, and
                        // 32-bit sums of the pieces (their sizes add up to at most
                        // the chunk's bound, below 2^31)
                        int ps32[4] = {0, 0, 0, 0};
#pragma unroll
                        for (int b = 0; b < NB; ++b)
#pragma unroll
                            for (int c = 0; c < NC; ++c) {
                                if (a == 1 && b == Sh::BC && c == Sh::CC) continue;  // host: remainder
                                const int lin =
                                    (ohx + a - 1) + B[0] * ((ohy + b - Sh::BC) + B[1] * (ohz + c - Sh::CC));
#pragma unroll
                                for (int ch = 0; ch < NCH; ++ch) {
                                    const float v = (ch & 1) ? acc[b][c][ch >> 1].y : acc[b][c][ch >> 1].x;
                                    const int piece = __float2int_rn(v);
                                    box_add_split(ch, lin, piece);
                                    ps32[ch] += piece;
                                }
                            }
#pragma unroll
                        for (int ch = 0; ch < 4; ++ch) ps[ch] = ps32[ch];
                    } else if (FLAT != 0 && narrow) {
                        // 2-D tiles: 32-bit roundings into the int64 words
                        quantise([](float v) { return (long long)__float2int_rn(v); },
                                 [&](int ch, int lin, long long v) {
                                     shared_add_i64_always(&sdep[ch * bvol + lin], v);
                                 });
                    } else {
                        // wide chunk sums, or a tile too dense for the split box
                        quantise([&](float v) {
                            big |= !(fabsf(v) < 4.5e15f);
                            return rround(v);
                        }, box_add);
                    }
                }
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const long long s1 = __shfl_sync(FULL, ps[ch], base + 0);
                    const long long s2 = __shfl_sync(FULL, ps[ch], base + 2);
                    if (a == 1 && own) {
                        const float Sc = (ch & 1) ? S2[ch >> 1].y : S2[ch >> 1].x;
                        big |= !(fabsf(Sc) < 4.5e15f);
                        const long long rest = (narrow ? (long long)__float2int_rn(Sc) : rround(Sc)) - (ps[ch] + s1 + s2);
                        if (rest != 0) box_add(ch, ohx + B[0] * (ohy + B[1] * ohz), rest);
                    }
                }
            }
        }
    }
    if (big) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_OVERFLOW);
    __syncthreads();

    // ---- flush the deposit box
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        const int64_t gz = i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const long long v = split ? (long long)bhi[c * bvol + lin] * 65536 + (long long)blo[c * bvol + lin]
                                      : (long long)sdep[c * bvol + lin];
            if (v != 0) atomicAdd(&A.dep[4 * gz + c], (unsigned long long)v);
        }
    }
    const unsigned mv = __reduce_max_sync(FULL, __float_as_uint(moved));
    const unsigned nr = __reduce_add_sync(FULL, (unsigned)nremoved);
    if (lane == 0) {
        if (mv) atomicMax(&A.status[ST_MAXMOVE], mv);
        if (nr) atomicAdd(reinterpret_cast<unsigned long long *>(&A.status[ST_REMOVED_LO]),
                          (unsigned long long)nr);
    }
    if (reuse) {
        __syncthreads();
        if (threadIdx.x == 0 && TA.gas_tmap) tma_barrier_inval(sbar);
    }
    return true;
}

template <int GEOM, int FLAT, int MODE, int TX = 0, int TY = 0, int TZ = 0>
__global__ void __launch_bounds__(kSlabThreads, 2)
step_slab_kernel(const __grid_constant__ TiledArgs<float> TA)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    slab_tile<GEOM, FLAT, MODE, TX, TY, TZ>(TA, blockIdx.x, gridDim.x, smem_raw, false);
}

// Gas predictor on the slab layout (Sec. 3.1): one tile per block, the
// chunk rule for grains whose x^n lies in their key zone, the per-grain rule
// for the others.
template <int GEOM, int FLAT, int TX = 0, int TY = 0, int TZ = 0>
__global__ void __launch_bounds__(kSlabThreads, 2)
predict_slab_kernel(const __grid_constant__ TiledArgs<float> TA)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    slab_tile<GEOM, FLAT, 1, TX, TY, TZ, true>(TA, blockIdx.x, gridDim.x, smem_raw, false);
}

using SlabKernel = void (*)(TiledArgs<float>);

// The step kernel's copy for this tile shape (slab_shape_id).
template <int GEOM, int FLAT, int MODE>
SlabKernel step_slab_pick(int shape)
{
    if constexpr (MODE == 1 && FLAT == 0) {
        if (shape == SHAPE_8C) return step_slab_kernel<GEOM, FLAT, MODE, 8, 8, 8>;
    } else if constexpr (MODE == 1 && FLAT == 1) {
        if (shape == SHAPE_32X16) return step_slab_kernel<GEOM, FLAT, MODE, 32, 1, 16>;
        if (shape == SHAPE_16X16) return step_slab_kernel<GEOM, FLAT, MODE, 16, 1, 16>;
    }
    return step_slab_kernel<GEOM, FLAT, MODE>;
}

inline size_t slab_smem_bytes(const GridDev &g)
{
    size_t bvol = 1;
    for (int d = 0; d < 3; ++d) bvol *= (size_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
    const size_t tsum = (size_t)g.T[0] + g.T[1] + g.T[2];
    return bvol * (4 * sizeof(float) + 4 * sizeof(long long)) +
           (size_t)((g.tvol + 31) & ~31) * sizeof(int) + (size_t)((g.tvol + 32) & ~31) * sizeof(int) +
           (size_t)(kSlabThreads / 32) * kSlabCap * sizeof(unsigned short) +
           (size_t)(kSlabThreads / 32) * kRecFields * kRecStride * sizeof(float) +
           tsum * (sizeof(double) + 2 * sizeof(float)) + ((size_t)g.T[0] + g.T[1] + 1) * sizeof(float) +
           2 * ((size_t)g.T[0] + g.T[1]) * sizeof(float) +
           16;  // the bulk copy's transaction barrier (8-byte aligned)
}

template <int GEOM, int FLAT, int MODE>
cudaError_t launch_step_slab(const TiledArgs<float> &a, cudaStream_t s)
{
    const GridDev &g = a.s.g;
    const int ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    const size_t smem = slab_smem_bytes(g);
    // the default tiles (TSC, exponential midpoint) run copies compiled for
    // their shape
    const SlabKernel kern = step_slab_pick<GEOM, FLAT, MODE>(slab_shape_id(g, FLAT, a.tsc, MODE));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kSlabThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int GEOM, int FLAT>
cudaError_t launch_predict_slab(const TiledArgs<float> &a, cudaStream_t s)
{
    const GridDev &g = a.s.g;
    const int ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    const size_t smem = slab_smem_bytes(g);
    SlabKernel kern = predict_slab_kernel<GEOM, FLAT>;
    if constexpr (FLAT == 0)
        if (slab_shape_id(g, FLAT, a.tsc, 1) == SHAPE_8C) kern = predict_slab_kernel<GEOM, FLAT, 8, 8, 8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kSlabThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dust
