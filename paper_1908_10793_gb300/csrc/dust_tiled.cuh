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

constexpr int kTiledThreads = 256;

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

template <typename Real>
__host__ __device__ inline size_t tiled_smem_bytes(const GridDev &g)
{
    size_t bvol = 1;
    for (int d = 0; d < 3; ++d) bvol *= (size_t)(g.T[d] + (g.n[d] > 1 ? 2 : 0));
    return bvol * (4 * sizeof(Real) + 4 * sizeof(long long));
}

template <typename Real, int GEOM, int WEIGHT>
__global__ void __launch_bounds__(kTiledThreads)
step_tiled_kernel(const TiledArgs<Real> TA)
{
    const StepArgs<Real> &A = TA.s;
    const GridDev &g = A.g;
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const int tile = blockIdx.x;
    const int64_t g0 = TA.key_off[(int64_t)tile * g.tvol];
    const int64_t g1 = TA.key_off[(int64_t)(tile + 1) * g.tvol];
    if (g1 <= g0) return;  // no grains: nothing to deposit

    int H[3], B[3], o[3];
    {
        int t = tile;
        const int tc[3] = {t % g.nt[0], (t / g.nt[0]) % g.nt[1], t / (g.nt[0] * g.nt[1])};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            H[d] = g.n[d] > 1 ? 1 : 0;
            B[d] = g.T[d] + 2 * H[d];
            o[d] = tc[d] * g.T[d] - H[d];
        }
    }
    const int bvol = B[0] * B[1] * B[2];
    Real *sgas = reinterpret_cast<Real *>(smem_raw);
    unsigned long long *sdep =
        reinterpret_cast<unsigned long long *>(smem_raw + (size_t)bvol * 4 * sizeof(Real));

    // ---- stage the gas box, clear the deposit box
    for (int lin = threadIdx.x; lin < bvol; lin += blockDim.x) {
        const int bx = lin % B[0], by = (lin / B[0]) % B[1], bz = lin / (B[0] * B[1]);
        const int i = map_zone(o[0] + bx, g.n[0], g.bc[0]);
        const int j = map_zone(o[1] + by, g.n[1], g.bc[1]);
        const int k = map_zone(o[2] + bz, g.n[2], g.bc[2]);
        Real v[4];
        load_gas<Real>(A.gas, i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k), v);
        smem_gas_store<Real>(sgas, lin, v);
#pragma unroll
        for (int c = 0; c < 4; ++c) sdep[4 * lin + c] = 0ull;
    }
    __syncthreads();

    int nremoved = 0;
    float moved = 0.f;
    const int lane = threadIdx.x & 31;
    for (int64_t gi = g0 + threadIdx.x; gi < g1; gi += blockDim.x) {
        double q[3] = {A.s.q[0][gi], A.s.q[1][gi], A.s.q[2][gi]};
        if (isnan(q[0])) continue;
        Real pn[3] = {A.s.p[0][gi], A.s.p[1][gi], A.s.p[2][gi]};
        const int sp = A.s.species ? A.s.species[gi] : 0;
        const Real h = (Real)(0.5 * A.dt);
        Real inc1[3], inc2[3];
        drift<Real, GEOM>(A.ph, q, q, pn, h, false, inc1);
        if (!apply_bc<Real, GEOM>(g, A.ph, A.ph.shift_mid, q, pn)) {
            A.s.q[0][gi] = __longlong_as_double(0x7ff8000000000000LL);
            ++nremoved;
            continue;
        }
        const double qm[3] = {q[0], q[1], q[2]};
        int host[3];
        Real w[3][3];
        float iw[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) zone_weights<Real, GEOM>(g, d, WEIGHT, qm[d], host[d], w[d], iw[d]);

        // host position inside the tile box (periodic images folded back)
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
            if (g.n[2] <= 1 && c3 != 1) continue;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (g.n[1] <= 1 && b != 1) continue;
                const Real wyz = w[1][b] * w[2][c3];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (g.n[0] <= 1 && a != 1) continue;
                    const Real W = w[0][a] * wyz;
                    Real f[4];
                    if (inbox) {
                        const int lin = (lb[0] + a - 1) + B[0] * ((lb[1] + b - 1) + B[1] * (lb[2] + c3 - 1));
                        smem_gas_load<Real>(sgas, lin, f);
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
        const Real dt = (Real)A.dt;
        const Real x = dt / tau;
        const Real E = rexp(-x);
        const Real cg = -rexpm1(-x);
        const Real h1 = (x == Real(0)) ? dt : dt * cg / x;
        const Real vg[3] = {acc[1], acc[2], acc[3]};
        Real pp[3], a[3], dH[3];
        kick<Real, GEOM>(A.ph, qm, pn, vg, E, cg, h1, pp, a, dH);
        drift<Real, GEOM>(A.ph, q, qm, pp, h, true, inc2);
        Real pnew[3] = {pp[0], pp[1], pp[2]};
        const bool alive = apply_bc<Real, GEOM>(g, A.ph, A.ph.shift_end, q, pnew);

        const Real mq = (Real)(A.sp.mass[sp] * A.inv_quantum);
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
        for (int d = 0; d < 3; ++d) moved = fmaxf(moved, fabsf((float)(inc1[d] + inc2[d])) * iw[d]);

        if (inbox) {
            // per-grain fixed-point rule into the shared box; lanes start at
            // different stencil nodes so that grains of one zone do not hit
            // the same shared word in the same instruction
            long long rest[4];
            bool big = false;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                big |= !(fabs((double)Dq[c]) < 4.5e15);
                rest[c] = rround(Dq[c]);
            }
            if (big) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_OVERFLOW);
            for (int k = 0; k < 27; ++k) {
                int nidx = k + lane;
                nidx -= 27 * (nidx >= 27);
                nidx -= 27 * (nidx >= 27);
                const int na = nidx % 3, nb = (nidx / 3) % 3, nc = nidx / 9;
                if (nidx == 13) continue;  // host node: remainder below
                if ((g.n[0] <= 1 && na != 1) || (g.n[1] <= 1 && nb != 1) || (g.n[2] <= 1 && nc != 1))
                    continue;
                const Real wa = na == 0 ? w[0][0] : (na == 1 ? w[0][1] : w[0][2]);
                const Real wb = nb == 0 ? w[1][0] : (nb == 1 ? w[1][1] : w[1][2]);
                const Real wc = nc == 0 ? w[2][0] : (nc == 1 ? w[2][1] : w[2][2]);
                const Real W = wa * (wb * wc);
                const int lin = (lb[0] + na - 1) + B[0] * ((lb[1] + nb - 1) + B[1] * (lb[2] + nc - 1));
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long piece = rround(W * Dq[c]);
                    if (piece != 0) {
                        atomicAdd(&sdep[4 * lin + c], (unsigned long long)piece);
                        rest[c] -= piece;
                    }
                }
            }
            const int hl = lb[0] + B[0] * (lb[1] + B[1] * lb[2]);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (rest[c] != 0) atomicAdd(&sdep[4 * hl + c], (unsigned long long)rest[c]);
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
            const unsigned long long v = sdep[4 * lin + c];
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
