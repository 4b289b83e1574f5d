// Tiled fused step kernel: one CTA per tile of zones.  The tile's gas
// stencil (tile + one halo zone) is staged in shared memory, every grain
// sorted into the tile is pushed with the same arithmetic as the per-grain
// kernel, its fixed-point deposit pieces are accumulated with shared-memory
// 64-bit atomics, and the tile box is flushed to the global deposit once.
// Grains whose half-step zone left the tile (stale sort) take the global
// gather / global atomic path, so results never depend on the tiling.
#pragma once

#include "dust_step_kernels.cuh"

namespace dust {

constexpr int kTiledThreads = 256;  // threads per CTA = grains per chunk

// Index of zone k (possibly one beyond the grid) in a direction of n zones.
__device__ __forceinline__ int map_zone(int k, int n, int bc)
{
    if (n <= 1) return 0;
    if (k < 0) return bc == DUST_BC_PERIODIC ? k + n : 0;
    if (k >= n) return bc == DUST_BC_PERIODIC ? k - n : n - 1;
    return k;
}

template <typename Real>
__device__ __forceinline__ void smem_gas_store(Real *s, int lin, const Real v[4]);
template <>
__device__ __forceinline__ void smem_gas_store<float>(float *s, int lin, const float v[4])
{
    reinterpret_cast<float4 *>(s)[lin] = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void smem_gas_store<double>(double *s, int lin, const double v[4])
{
    reinterpret_cast<double2 *>(s)[2 * lin] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(s)[2 * lin + 1] = make_double2(v[2], v[3]);
}
template <typename Real>
__device__ __forceinline__ void smem_gas_load(const Real *s, int lin, Real v[4]);
template <>
__device__ __forceinline__ void smem_gas_load<float>(const float *s, int lin, float v[4])
{
    const float4 a = reinterpret_cast<const float4 *>(s)[lin];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <>
__device__ __forceinline__ void smem_gas_load<double>(const double *s, int lin, double v[4])
{
    const double2 a = reinterpret_cast<const double2 *>(s)[2 * lin];
    const double2 b = reinterpret_cast<const double2 *>(s)[2 * lin + 1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}


// Adds v to the 64-bit integer at p (shared memory) with two 32-bit atomics:
// the low word's carry goes into the high word, so the sum is exact modulo
// 2^64 and mixes freely with 64-bit atomic adds to the same word.  On this
// GPU 32-bit shared atomics are much cheaper than 64-bit ones.
__device__ __forceinline__ void shared_add_i64(unsigned long long *p, long long v)
{
    unsigned *w = reinterpret_cast<unsigned *>(p);
    const unsigned lo = (unsigned)(unsigned long long)v;
    const unsigned hi = (unsigned)((unsigned long long)v >> 32);
    const unsigned old = atomicAdd(w, lo);
    const unsigned up = hi + ((old + lo < old) ? 1u : 0u);
    if (up != 0u) atomicAdd(w + 1, up);
}

// The same, with the high word's add issued unconditionally (no branch on
// the carried value): for the many pieces of a chunk, where the branch costs
// more than the adds of zero it saves.
__device__ __forceinline__ void shared_add_i64_always(unsigned long long *p, long long v)
{
    unsigned *w = reinterpret_cast<unsigned *>(p);
    const unsigned lo = (unsigned)(unsigned long long)v;
    const unsigned hi = (unsigned)((unsigned long long)v >> 32);
    const unsigned old = atomicAdd(w, lo);
    atomicAdd(w + 1, hi + ((old + lo < old) ? 1u : 0u));
}

// How long a block waits for its gas box before it gives up
// (DUST_FLAG_TIMEOUT): one second; the copy of a few tens of KB takes
// microseconds.
constexpr unsigned long long kTmaWaitNs = 1000000000ull;

// ---- bulk tensor copy (TMA) of the gas box into shared memory

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// One thread: initialise the transaction barrier and make it visible to the
// copy engine.
__device__ __forceinline__ void tma_barrier_init(unsigned long long *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread, after every thread's wait on it has returned: invalidate the
// barrier, so that the same shared memory can hold the next tile's barrier
// (a block that processes several tiles in turn).
__device__ __forceinline__ void tma_barrier_inval(unsigned long long *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One thread: expect `bytes` and start the 4-D tile copy of the box at
// coordinates (0, x, y, z) of the tensor map into dst.
__device__ __forceinline__ void tma_load_box(void *dst, const void *tmap, int x, int y, int z,
                                             unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(smem_u32(dst)), "l"(tmap), "r"(0), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every thread: wait for phase 0 of the barrier, at most limit_ns.
__device__ __forceinline__ bool tma_wait(unsigned long long *bar, unsigned long long limit_ns)
{
    const unsigned long long t0 = global_ns();
    for (;;) {
        unsigned done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(smem_u32(bar)) : "memory");
        if (done) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// Staging of a tile's gas box (the tile plus its halo: origin o, B zones per
// direction, bvol = B0 B1 B2 zones of 4 channels) into shared memory.
// Begin: with a tensor map of the gas, thread 0 starts one bulk copy.
// extra_tx > 0 (testing the timeout path only) makes the barrier expect
// more bytes than the copy delivers, so that the wait runs out.
template <typename Real>
__device__ __forceinline__ void gas_box_begin(const void *tmap, Real *sgas, const int o[3], int bvol,
                                              unsigned long long *bar, unsigned extra_tx)
{
    if (tmap && threadIdx.x == 0) {
        tma_barrier_init(bar);
        tma_load_box(sgas, tmap, o[0], o[1], o[2], bar, (unsigned)(bvol * 4 * sizeof(Real)) + extra_tx);
    }
}

// Finish (every thread, after a __syncthreads that follows gas_box_begin):
// without a tensor map, load the box zone by zone; with one, wait for the
// copy (bounded: on a timeout every thread waits once more for the copy in
// flight, DUST_FLAG_TIMEOUT is raised and false returned, and the block
// must return) and replace the zones outside the grid, which the copy
// zero-fills, by their periodic images or outflow ghosts.
template <typename Real>
__device__ bool gas_box_finish(const GridDev &g, const Real *gas, const void *tmap, Real *sgas,
                               const int o[3], const int B[3], unsigned long long *bar,
                               unsigned int *status, unsigned long long wait_ns)
{
    const int bvol = B[0] * B[1] * B[2];
    bool edge = !tmap;
    if (tmap) {
        const unsigned long long lim = wait_ns ? wait_ns : kTmaWaitNs;
        const bool late = !tma_wait(bar, lim);
        if (__syncthreads_or(late)) {
            if (late) tma_wait(bar, lim);
            if (threadIdx.x == 0) atomicOr(&status[ST_FLAGS], DUST_FLAG_TIMEOUT);
            return false;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) edge |= g.n[d] > 1 && (o[d] < 0 || o[d] + B[d] > g.n[d]);
    }
    if (edge) {
        for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
            const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
            const int x = o[0] + bx, y = o[1] + by, z = o[2] + bz;
            if (tmap && x >= 0 && x < g.n[0] && y >= 0 && y < g.n[1] && z >= 0 && z < g.n[2]) continue;
            const int i = map_zone(x, g.n[0], g.bc[0]);
            const int j = map_zone(y, g.n[1], g.bc[1]);
            const int k = map_zone(z, g.n[2], g.bc[2]);
            Real v[4];
            load_gas<Real>(gas, i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k), v);
            smem_gas_store<Real>(sgas, lin, v);
        }
        __syncthreads();
    }
    return true;
}

constexpr int kChunk = kTiledThreads;

// Shared memory of one CTA: deposit box (channel major), run tables, gas
// box, and the per-grain records of one chunk.
template <typename Real>
__host__ __device__ inline size_t tiled_smem_bytes(const GridDev &g)
{
    size_t bvol = 1;
    for (int d = 0; d < 3; ++d) bvol *= (size_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
    const size_t ch = kChunk;
    // + 64: the three control words and the bulk copy's barrier (8-byte aligned)
    return bvol * (4 * sizeof(Real) + 4 * sizeof(long long)) +
           ch * (8 * sizeof(long long) + 13 * sizeof(Real) + 7 * sizeof(int)) + 64;
}

// Tiled step.  Grains of a tile are processed in chunks of whole sort keys
// (at most kChunk grains).  The deposit of a chunk is formed per run: the
// grains of one sort key that share their half-step host zone.  A run's node
// contributions are summed in registers in grain-id order, each node
// receives rint(sum / quantum), and the host zone receives the remainder
// rint(sum of D / quantum) - (other nodes), so a run deposits exactly its
// quantised total.  Runs are sets fixed by the sort keys, so the integer
// grid depends neither on the tile shape nor on the order of the scatter or
// of the threads.  Keys holding more than kChunk grains use the per-grain
// rule.
template <typename Real, int GEOM, int WEIGHT>
__global__ void __launch_bounds__(kTiledThreads)
step_tiled_kernel(const TiledArgs<Real> TA)
{
    const StepArgs<Real> &A = TA.s;
    const GridDev &g = A.g;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int CH = kChunk;

    const int tile = blockIdx.x;
    const int64_t kbase = (int64_t)tile * g.tvol;
    const int64_t g0 = TA.key_off[kbase];
    const int64_t g1 = TA.key_off[kbase + g.tvol];
    if (g1 <= g0) return;  // no grains: nothing to deposit

    int B[3], o[3];
    {
        const int t = tile;
        const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int H = g.n[d] > 1 ? 1 : 0;
            B[d] = g.T[d] + 2 * H;
            o[d] = tc[d] * g.T[d] - H;
        }
    }
    const int bvol = B[0] * B[1] * B[2];
    unsigned char *ptr = smem_raw;
    Real *sgas = reinterpret_cast<Real *>(ptr);     // first: 128-byte aligned for the bulk copy
    ptr += (size_t)bvol * 4 * sizeof(Real);
    unsigned long long *sdep = reinterpret_cast<unsigned long long *>(ptr);
    ptr += (size_t)bvol * 4 * sizeof(long long);
    unsigned long long *run_sum = reinterpret_cast<unsigned long long *>(ptr);   // [4][CH]
    ptr += (size_t)CH * 4 * sizeof(long long);
    long long *run_q = reinterpret_cast<long long *>(ptr);                       // [4][CH]
    ptr += (size_t)CH * 4 * sizeof(long long);
    Real *rec_w = reinterpret_cast<Real *>(ptr);                                 // [9][CH]
    ptr += (size_t)CH * 9 * sizeof(Real);
    Real *rec_d = reinterpret_cast<Real *>(ptr);                                 // [4][CH]
    ptr += (size_t)CH * 4 * sizeof(Real);
    int *rec_host = reinterpret_cast<int *>(ptr);                                // [CH]
    ptr += (size_t)CH * sizeof(int);
    int *rec_id = reinterpret_cast<int *>(ptr);                                  // [CH]
    ptr += (size_t)CH * sizeof(int);
    int *rec_order = reinterpret_cast<int *>(ptr);                               // [CH]
    ptr += (size_t)CH * sizeof(int);
    int *run_start = reinterpret_cast<int *>(ptr);                               // [CH]
    ptr += (size_t)CH * sizeof(int);
    int *key_start = reinterpret_cast<int *>(ptr);                               // [CH] 1 = slot starts a key
    ptr += (size_t)CH * sizeof(int);
    int *seg_lo = reinterpret_cast<int *>(ptr);                                  // [CH] key segment of a slot
    ptr += (size_t)CH * sizeof(int);
    int *seg_hi = reinterpret_cast<int *>(ptr);                                  // [CH]
    ptr += (size_t)CH * sizeof(int);
    int *ctl = reinterpret_cast<int *>(ptr);  // [0] runs, [1] chunk end key, [2] chunk grains
    unsigned long long *sbar = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(ctl + 3) + 7) & ~(uintptr_t)7);

    // ---- stage the gas box, clear the deposit box and the run sums
    gas_box_begin<Real>(TA.gas_tmap, sgas, o, bvol, sbar, TA.wait_extra_tx);
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 4; ++c) sdep[c * bvol + lin] = 0ull;
    }
    for (int k = threadIdx.x; k < 4 * CH; k += blockDim.x) run_sum[k] = 0ull;
    __syncthreads();
    if (!gas_box_finish<Real>(g, A.gas, TA.gas_tmap, sgas, o, B, sbar, A.status, TA.wait_ns)) return;

    int nremoved = 0;
    float moved = 0.f;
    const int lane = threadIdx.x & 31;
    const int na = g.n[0] > 1 ? 3 : 1, nb = g.n[1] > 1 ? 3 : 1, nc = g.n[2] > 1 ? 3 : 1;
    const int ntask = na * nb;
    const Real h = (Real)(0.5 * A.dt);
    const Real dt = (Real)A.dt;

    int kcur = 0;          // first key (relative to the tile) of the chunk
    int64_t split = 0;     // grains of an oversized key already processed
    while (kcur < g.tvol) {
        // ---- choose the chunk: whole keys with at most CH grains, or the
        // next CH grains of one oversized key (per-grain rule)
        if (threadIdx.x == 0) {
            const int64_t base = TA.key_off[kbase + kcur] + split;
            int lo = kcur, hi = g.tvol;  // largest end with key_off[end] - base <= CH
            while (hi - lo > 0) {
                const int mid = (lo + hi + 1) >> 1;
                if (TA.key_off[kbase + mid] - base <= CH) lo = mid; else hi = mid - 1;
            }
            ctl[0] = 0;
            if (lo > kcur && split == 0) {
                ctl[1] = lo;
                ctl[2] = (int)(TA.key_off[kbase + lo] - base);
            } else {  // key kcur alone has more than CH grains left
                ctl[1] = -1;
                ctl[2] = (int)min((int64_t)CH, TA.key_off[kbase + kcur + 1] - base);
            }
        }
        __syncthreads();  // gas box ready; previous chunk's records consumed
        const int kend = ctl[1];
        const int cn = ctl[2];
        const bool per_grain = kend < 0;
        const int64_t cb = TA.key_off[kbase + kcur] + split;
        key_start[threadIdx.x] = 0;

        // ---- phase A: one grain per thread
        const int slot = threadIdx.x;
        const int64_t gi = cb + slot;
        int hl = -1;
        if (slot < cn) {
            double q[3] = {A.s.q[0][gi], A.s.q[1][gi], A.s.q[2][gi]};
            if (!isnan(q[0])) {
                Real pn[3] = {A.s.p[0][gi], A.s.p[1][gi], A.s.p[2][gi]};
                const int sp = A.s.species ? A.s.species[gi] : 0;
                Real inc1[3], inc2[3];
                drift<Real, GEOM>(A.ph, q, q, pn, h, false, inc1);
                if (!apply_bc<Real, GEOM>(g, A.ph, shift_mid_of(A), q, pn)) {
                    A.s.q[0][gi] = __longlong_as_double(0x7ff8000000000000LL);
                    ++nremoved;
                } else {
                    const double qm[3] = {q[0], q[1], q[2]};
                    int host[3];
                    Real w[3][3];
                    float iw[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        zone_weights<Real, GEOM>(g, d, WEIGHT, qm[d], host[d], w[d], iw[d]);
                    int lb[3];
                    bool inbox = true;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        int l = host[d] - o[d];
                        if (g.n[d] > 1 && g.bc[d] == DUST_BC_PERIODIC) {
                            if (l < 0) l += g.n[d];
                            else if (l >= B[d]) l -= g.n[d];
                        }
                        lb[d] = l;
                        if (g.n[d] > 1) inbox &= (l >= 1) && (l <= B[d] - 2);
                    }
                    // gather (Eq. Delta_vp)
                    Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        if (nc == 1 && c3 != 1) continue;
#pragma unroll
                        for (int b = 0; b < 3; ++b) {
                            if (nb == 1 && b != 1) continue;
                            const Real wyz = w[1][b] * w[2][c3];
#pragma unroll
                            for (int a = 0; a < 3; ++a) {
                                if (na == 1 && a != 1) continue;
                                const Real W = w[0][a] * wyz;
                                Real f[4];
                                if (inbox) {
                                    smem_gas_load<Real>(sgas, (lb[0] + a - 1) + B[0] * ((lb[1] + b - 1) + B[1] * (lb[2] + c3 - 1)), f);
                                } else {
                                    const int ix = node_of(host[0], a - 1, g.n[0], g.bc[0]);
                                    const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
                                    const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
                                    load_gas<Real>(A.gas, ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz), f);
                                }
#pragma unroll
                                for (int c = 0; c < 4; ++c) acc[c] += W * f[c];
                            }
                        }
                    }
                    const Real value = A.s.param ? A.s.param[gi] : (Real)A.sp.tau[sp];
                    const Real tau = stopping_time<Real, GEOM>(A.ph, A.sp.mode[sp], value, qm, acc[0]);
                    const Real x = dt / tau;
                    const Real E = rexp(-x);
                    const Real cg = -rexpm1(-x);
                    const Real h1 = (x == Real(0)) ? dt : dt * cg / x;
                    const Real vg[3] = {acc[1], acc[2], acc[3]};
                    Real pp[3], a[3], dH[3];
                    kick_any<Real, GEOM>(A.ph, qm, pn, vg, tau, dt, E, cg, h1, pp, a, dH);
                    drift<Real, GEOM>(A.ph, q, qm, pp, h, true, inc2);
                    Real pnew[3] = {pp[0], pp[1], pp[2]};
                    const bool alive = apply_bc<Real, GEOM>(g, A.ph, shift_end_of(A), q, pnew);
                    const Real mq = sizeof(Real) == 4 ? (Real)A.sp.mqf[sp] : (Real)A.sp.mq[sp];
                    Real Dq[4];
                    Dq[3] = Real(0);
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        Dq[c] = -mq * ((pp[c] - pn[c]) - dt * a[c]);
                        Dq[3] += Dq[c] * dH[c];
                    }
                    if (!(isfinite(pp[0]) && isfinite(pp[1]) && isfinite(pp[2])))
                        atomicOr(&A.status[ST_FLAGS], DUST_FLAG_NAN);
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        moved = fmaxf(moved, fabsf((float)(inc1[d] + inc2[d])) * iw[d]);
                    if (inbox && !per_grain) {
                        hl = lb[0] + B[0] * (lb[1] + B[1] * lb[2]);
#pragma unroll
                        for (int d = 0; d < 3; ++d)
#pragma unroll
                            for (int k = 0; k < 3; ++k) rec_w[(3 * d + k) * CH + slot] = w[d][k];
#pragma unroll
                        for (int c = 0; c < 4; ++c) rec_d[c * CH + slot] = Dq[c];
                        rec_id[slot] = A.s.id[gi];
                    } else {
                        deposit_fixed<Real>(g, A.dep, host, w, Dq, A.status);
                    }
                    if (!alive) {
                        q[0] = __longlong_as_double(0x7ff8000000000000LL);
                        ++nremoved;
                    }
                    A.s.q[0][gi] = q[0]; A.s.q[1][gi] = q[1]; A.s.q[2][gi] = q[2];
                    A.s.p[0][gi] = pnew[0]; A.s.p[1][gi] = pnew[1]; A.s.p[2][gi] = pnew[2];
                }
            }
        }
        rec_host[slot] = hl;
        // key boundaries inside the chunk
        if (!per_grain)
            for (int k = kcur + threadIdx.x; k < kend; k += blockDim.x) {
                const int s = (int)(TA.key_off[kbase + k] - cb);
                if (s >= 0 && s < cn) key_start[s] = 1;
            }
        __syncthreads();

        if (!per_grain) {
            // ---- each key segment listed in grain-id order (one thread per
            // key, insertion sort of its few slots)
            if (slot < cn && (slot == 0 || key_start[slot])) {
                int e = slot + 1;
                while (e < cn && !key_start[e]) ++e;
                for (int u = slot; u < e; ++u) {
                    const int id = rec_host[u] >= 0 ? rec_id[u] : 0x7fffffff;
                    int j = u - 1;
                    while (j >= slot) {
                        const int sj = rec_order[j];
                        const int idj = rec_host[sj] >= 0 ? rec_id[sj] : 0x7fffffff;
                        if (idj <= id) break;
                        rec_order[j + 1] = sj;
                        --j;
                    }
                    rec_order[j + 1] = u;
                    seg_lo[u] = slot;
                    seg_hi[u] = e;
                }
            }
            __syncthreads();
            // ---- runs: the grains of one key sharing a host zone; a run
            // starts at its first grain in id order
            if (slot < cn) {
                const int hs = rec_host[rec_order[slot]];
                bool first = hs >= 0;
                for (int u = seg_lo[slot]; u < slot && first; ++u) first = rec_host[rec_order[u]] != hs;
                if (first) run_start[atomicAdd(&ctl[0], 1)] = slot;
            }
            __syncthreads();

            // ---- phase B: one task per (run, x node, y node); z nodes and
            // the four channels are summed in registers over the run
            const int R = ctl[0];
            bool big = false;
            for (int t = threadIdx.x; t < R * ntask; t += blockDim.x) {
                const int r = t / ntask, ab = t - r * ntask;
                const int a = na == 3 ? ab % 3 : 1;
                const int b = nb == 3 ? ab / na : 1;
                const bool htask = a == 1 && b == 1;
                const int u0 = run_start[r];
                const int hlin = rec_host[rec_order[u0]];
                const int u1 = seg_hi[u0];
                Real sum[3][4], S[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    S[c] = Real(0);
#pragma unroll
                    for (int z = 0; z < 3; ++z) sum[z][c] = Real(0);
                }
                for (int u = u0; u < u1; ++u) {
                    const int s = rec_order[u];
                    if (rec_host[s] != hlin) continue;
                    const Real wab = rec_w[a * CH + s] * rec_w[(3 + b) * CH + s];
                    Real D[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) D[c] = rec_d[c * CH + s];
#pragma unroll
                    for (int z = 0; z < 3; ++z) {
                        if (nc == 1 && z != 1) continue;
                        const Real W = wab * rec_w[(6 + z) * CH + s];
#pragma unroll
                        for (int c = 0; c < 4; ++c) sum[z][c] += W * D[c];
                    }
                    if (htask) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) S[c] += D[c];
                    }
                }
                long long ps[4] = {0, 0, 0, 0};
#pragma unroll
                for (int z = 0; z < 3; ++z) {
                    if (nc == 1 && z != 1) continue;
                    if (htask && z == 1) continue;  // the host node takes the remainder
                    const int lin = hlin + (a - 1) + B[0] * ((b - 1) + B[1] * (z - 1));
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        big |= !(fabs(sum[z][c]) < Real(4.5e15));
                        const long long piece = rround(sum[z][c]);
                        if (piece != 0) {
                            shared_add_i64(&sdep[c * bvol + lin], piece);
                            ps[c] += piece;
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (ps[c] != 0) shared_add_i64(&run_sum[c * CH + r], ps[c]);
                    if (htask) {
                        big |= !(fabs(S[c]) < Real(4.5e15));
                        run_q[c * CH + r] = rround(S[c]);
                    }
                }
            }
            if (big) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_OVERFLOW);
            __syncthreads();

            // ---- host remainders
            for (int r = threadIdx.x; r < R; r += blockDim.x) {
                const int hlin = rec_host[rec_order[run_start[r]]];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long rest = run_q[c * CH + r] - (long long)run_sum[c * CH + r];
                    run_sum[c * CH + r] = 0ull;
                    if (rest != 0) shared_add_i64(&sdep[c * bvol + hlin], rest);
                }
            }
            kcur = kend;
            split = 0;
        } else {
            split += cn;
            if (TA.key_off[kbase + kcur] + split >= TA.key_off[kbase + kcur + 1]) {
                ++kcur;
                split = 0;
            }
        }
        // skip keys without grains
        __syncthreads();
    }

    // ---- flush the deposit box
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        const int64_t gz = i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const unsigned long long v = sdep[c * bvol + lin];
            if (v != 0ull) atomicAdd(&A.dep[4 * gz + c], v);
        }
    }
    // removed-grain count and largest displacement (warp aggregated)
    const unsigned mv = __reduce_max_sync(0xffffffffu, __float_as_uint(moved));
    const unsigned nr = __reduce_add_sync(0xffffffffu, (unsigned)nremoved);
    if (lane == 0) {
        if (mv) atomicMax(&A.status[ST_MAXMOVE], mv);
        if (nr) atomicAdd(reinterpret_cast<unsigned long long *>(&A.status[ST_REMOVED_LO]),
                          (unsigned long long)nr);
    }
}

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_step_tiled(const TiledArgs<Real> &a, cudaStream_t s)
{
    const GridDev &g = a.s.g;
    const int ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    const size_t smem = tiled_smem_bytes<Real>(g);
    auto kern = step_tiled_kernel<Real, GEOM, WEIGHT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kTiledThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dust

namespace dust {

// Tiled gas half-step predictor (same arithmetic and fixed-point rule as
// predict_gas_kernel): one block per tile of zones stages the tile's gas box
// and an int64 impulse box in shared memory, takes the grains sorted into the
// tile (through the sort's permutation when the step kernel will finish the
// sort), gathers at x^n from the box and adds each grain's pieces to the box
// with 32-bit atomics; grains whose stencil at x^n leaves the box use global
// memory.  The per-grain rule makes the integers independent of the order.
template <typename Real, int GEOM, int WEIGHT>
__global__ void __launch_bounds__(kTiledThreads)
predict_tiled_kernel(const __grid_constant__ TiledArgs<Real> TA)
{
    const StepArgs<Real> &A = TA.s;
    const GridDev &g = A.g;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tile = blockIdx.x;
    const int64_t kbase = (int64_t)tile * g.tvol;
    const int g0 = TA.key_off[kbase], g1 = TA.key_off[kbase + g.tvol];
    if (g1 <= g0) return;
    int B[3], o[3];
    {
        const int tc[3] = {tile % g.nt[0], (tile / g.nt[0]) % g.nt[1], tile / (g.nt[0] * g.nt[1])};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int H = g.n[d] > 1 ? 1 : 0;
            B[d] = g.T[d] + 2 * H;
            o[d] = tc[d] * g.T[d] - H;
        }
    }
    const int bvol = B[0] * B[1] * B[2];
    Real *sgas = reinterpret_cast<Real *>(smem_raw);   // first: 128-byte aligned for the bulk copy
    unsigned long long *simp = reinterpret_cast<unsigned long long *>(smem_raw + (size_t)bvol * 4 * sizeof(Real));   // [3][bvol]
    unsigned long long *sbar = simp + (size_t)3 * bvol;
    gas_box_begin<Real>(TA.gas_tmap, sgas, o, bvol, sbar, TA.wait_extra_tx);
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) simp[c * bvol + lin] = 0ull;
    }
    __syncthreads();
    if (!gas_box_finish<Real>(g, A.gas, TA.gas_tmap, sgas, o, B, sbar, A.status, TA.wait_ns)) return;
    const Real dt = (Real)A.dt;
    for (int gi = g0 + threadIdx.x; gi < g1; gi += blockDim.x) {
        const int src = TA.perm ? TA.perm[gi] : gi;
        const double q[3] = {A.s.q[0][src], A.s.q[1][src], A.s.q[2][src]};
        if (isnan(q[0])) continue;
        const Real pn[3] = {A.s.p[0][src], A.s.p[1][src], A.s.p[2][src]};
        const int sp = A.s.species ? A.s.species[src] : 0;
        int host[3];
        Real w[3][3];
        float iw[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) zone_weights<Real, GEOM>(g, d, WEIGHT, q[d], host[d], w[d], iw[d]);
        int lb[3];
        bool inbox = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            int l = host[d] - o[d];
            if (g.n[d] > 1 && g.bc[d] == DUST_BC_PERIODIC) {
                if (l < 0) l += g.n[d];
                else if (l >= B[d]) l -= g.n[d];
            }
            lb[d] = l;
            if (g.n[d] > 1) inbox &= (l >= 1) && (l <= B[d] - 2);
        }
        Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
#pragma unroll 1
        for (int nd = 0; nd < 27; ++nd) {
            const int a = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
            if ((g.n[0] <= 1 && a != 1) || (g.n[1] <= 1 && b != 1) || (g.n[2] <= 1 && c3 != 1)) continue;
            const Real W = w[0][a] * (w[1][b] * w[2][c3]);
            Real f[4];
            if (inbox) {
                smem_gas_load<Real>(sgas, (lb[0] + a - 1) + B[0] * ((lb[1] + b - 1) + B[1] * (lb[2] + c3 - 1)), f);
            } else {
                const int ix = node_of(host[0], a - 1, g.n[0], g.bc[0]);
                const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
                const int iz = node_of(host[2], c3 - 1, g.n[2], g.bc[2]);
                load_gas<Real>(A.gas, ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz), f);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += W * f[c];
        }
        const Real value = A.s.param ? A.s.param[src] : (Real)A.sp.tau[sp];
        const Real tau = stopping_time<Real, GEOM>(A.ph, A.sp.mode[sp], value, q, acc[0]);
        const Real taup = fmax(tau, fabs(dt));
        // mass / quantum, precomputed per species in both precisions
        const Real mq = sizeof(Real) == 4 ? (Real)A.sp.mqf[sp] : (Real)A.sp.mq[sp];
        const Real coef = Real(0.5) * dt * mq / taup;
        Real Dq[4];
#pragma unroll
        for (int c = 0; c < 3; ++c) Dq[c] = coef * (pn[c] - acc[1 + c]);
        Dq[3] = Real(0);
        if (!inbox) {
            deposit_fixed<Real>(g, A.dep, host, w, Dq, A.status);
            continue;
        }
        // per-grain rule into the shared box: pieces for the other nodes,
        // the host takes the remainder
        long long rest[3];
        bool big = false;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            big |= !(fabs(Dq[c]) < Real(4.5e15));  // in the working precision
            rest[c] = rround(Dq[c]);
        }
        if (big) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_OVERFLOW);
        const int hl = lb[0] + B[0] * (lb[1] + B[1] * lb[2]);
#pragma unroll 1
        for (int nd = 0; nd < 27; ++nd) {
            const int a = nd % 3, b = (nd / 3) % 3, c3 = nd / 9;
            if (nd == 13 || (g.n[0] <= 1 && a != 1) || (g.n[1] <= 1 && b != 1) ||
                (g.n[2] <= 1 && c3 != 1))
                continue;
            const Real W = w[0][a] * (w[1][b] * w[2][c3]);
            const int lin = hl + (a - 1) + B[0] * ((b - 1) + B[1] * (c3 - 1));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const long long piece = rround(W * Dq[c]);
                if (piece != 0) {
                    shared_add_i64(&simp[c * bvol + lin], piece);
                    rest[c] -= piece;
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (rest[c] != 0) shared_add_i64(&simp[c * bvol + hl], rest[c]);
    }
    __syncthreads();
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        const int64_t gz = i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const unsigned long long v = simp[c * bvol + lin];
            if (v != 0ull) atomicAdd(&A.dep[4 * gz + c], v);
        }
    }
}

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_predict_tiled(const TiledArgs<Real> &a, cudaStream_t s)
{
    const GridDev &g = a.s.g;
    const int ntiles = g.nt[0] * g.nt[1] * g.nt[2];
    size_t bvol = 1;
    for (int d = 0; d < 3; ++d) bvol *= (size_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
    const size_t smem = bvol * (3 * sizeof(long long) + 4 * sizeof(Real)) + 16;  // + the barrier
    auto kern = predict_tiled_kernel<Real, GEOM, WEIGHT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<ntiles, kTiledThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dust
