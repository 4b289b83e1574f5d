// Step and sort kernels, templated on precision, geometry and weight order.
// Instantiated by the per-geometry translation units.
#pragma once

#include "dust_device.cuh"

namespace dust {

constexpr int kStepThreads = 256;

// Per-grain fixed-point deposit rule: for every channel c the grain's total
// Q_c = rint(D_c / quantum) is split over the stencil; every node other than
// the host gets rint(W_j D_c / quantum) and the host gets the remainder, so
// sum over zones = sum over grains of Q_c exactly (integer addition is
// order independent, so the grid does not depend on thread order).
template <typename Real>
__device__ __forceinline__ void deposit_fixed(const GridDev &g, unsigned long long *dep,
                                              const int host[3], const Real w[3][3],
                                              const Real Dq[4], unsigned int *status)
{
    long long rest[4];
    bool big = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        big |= !(fabs(Dq[c]) < Real(4.5e15));  // in the working precision
        rest[c] = rround(Dq[c]);
    }
    if (big) atomicOr(&status[ST_FLAGS], DUST_FLAG_OVERFLOW);
    const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
    int ix[3], iy[3], iz[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        ix[o] = node_of(host[0], o - 1, n0, g.bc[0]);
        iy[o] = node_of(host[1], o - 1, n1, g.bc[1]);
        iz[o] = node_of(host[2], o - 1, n2, g.bc[2]);
    }
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        if (n2 <= 1 && c3 != 1) continue;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (n1 <= 1 && b != 1) continue;
            const Real wyz = w[1][b] * w[2][c3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (n0 <= 1 && a != 1) continue;
                if (a == 1 && b == 1 && c3 == 1) continue;
                const Real W = w[0][a] * wyz;
                const int64_t idx = ix[a] + (int64_t)n0 * (iy[b] + (int64_t)n1 * iz[c3]);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long piece = rround(W * Dq[c]);
                    if (piece != 0) {
                        atomicAdd(&dep[4 * idx + c], (unsigned long long)piece);
                        rest[c] -= piece;
                    }
                }
            }
        }
    }
    const int64_t hidx = ix[1] + (int64_t)n0 * (iy[1] + (int64_t)n1 * iz[1]);
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (rest[c] != 0) atomicAdd(&dep[4 * hidx + c], (unsigned long long)rest[c]);
}

template <typename Real>
__device__ __forceinline__ void load_gas(const Real *gas, int64_t idx, Real out[4]);

template <>
__device__ __forceinline__ void load_gas<float>(const float *gas, int64_t idx, float out[4])
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(gas) + idx);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}

template <>
__device__ __forceinline__ void load_gas<double>(const double *gas, int64_t idx, double out[4])
{
    const double2 *p = reinterpret_cast<const double2 *>(gas) + 2 * idx;
    const double2 a = __ldg(p), b = __ldg(p + 1);
    out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
}

// One thread per grain: half drift, weights, gather, kick, half drift,
// boundaries, fixed-point deposit through global 64-bit atomics.
template <typename Real, int GEOM, int WEIGHT>
__global__ void __launch_bounds__(kStepThreads)
step_per_grain_kernel(const StepArgs<Real> A)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool removed = false;
    float moved = 0.f;
    if (gi < A.s.n) {
        double q[3] = {A.s.q[0][gi], A.s.q[1][gi], A.s.q[2][gi]};
        const int sp = A.s.species ? A.s.species[gi] : 0;
        // a species index the species table does not hold (possible only
        // where the caller owns the store): flagged, the grain left as it is
        const bool sp_ok = sp < A.sp.n;
        if (!sp_ok && !isnan(q[0])) atomicOr(&A.status[ST_FLAGS], DUST_FLAG_SPECIES);
        if (!isnan(q[0]) && sp_ok) {
            Real pn[3] = {A.s.p[0][gi], A.s.p[1][gi], A.s.p[2][gi]};
            const Real h = (Real)(0.5 * A.dt);
            Real inc1[3], inc2[3];
            drift<Real, GEOM>(A.ph, q, q, pn, h, false, inc1);
            if (!apply_bc<Real, GEOM>(A.g, A.ph, shift_mid_of(A), q, pn)) {
                removed = true;
            } else {
                const double qm[3] = {q[0], q[1], q[2]};
                int host[3];
                Real w[3][3];
                float iw[3];
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    zone_weights<Real, GEOM>(A.g, d, WEIGHT, qm[d], host[d], w[d], iw[d]);
                // gather (Eq. Delta_vp)
                Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
                const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
#pragma unroll
                for (int c3 = 0; c3 < 3; ++c3) {
                    if (n2 <= 1 && c3 != 1) continue;
                    const int iz = node_of(host[2], c3 - 1, n2, A.g.bc[2]);
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        if (n1 <= 1 && b != 1) continue;
                        const int iy = node_of(host[1], b - 1, n1, A.g.bc[1]);
                        const Real wyz = w[1][b] * w[2][c3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            if (n0 <= 1 && a != 1) continue;
                            const int ix = node_of(host[0], a - 1, n0, A.g.bc[0]);
                            const Real W = w[0][a] * wyz;
                            Real f[4];
                            load_gas<Real>(A.gas, ix + (int64_t)n0 * (iy + (int64_t)n1 * iz), f);
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
                kick_any<Real, GEOM>(A.ph, qm, pn, vg, tau, dt, E, cg, h1, pp, a, dH);
                drift<Real, GEOM>(A.ph, q, qm, pp, h, true, inc2);
                Real pnew[3] = {pp[0], pp[1], pp[2]};
                const bool alive = apply_bc<Real, GEOM>(A.g, A.ph, shift_end_of(A), q, pnew);
                // deposit: -m (dp - dt a), energy sum_c of that times dH/dp_c
                const Real mq = (Real)(A.sp.mass[sp] * A.inv_quantum);
                Real Dq[4];
                Dq[3] = Real(0);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    Dq[c] = -mq * ((pp[c] - pn[c]) - dt * a[c]);
                    Dq[3] += Dq[c] * dH[c];
                }
                deposit_fixed<Real>(A.g, A.dep, host, w, Dq, A.status);
                if (!(isfinite(pp[0]) && isfinite(pp[1]) && isfinite(pp[2])))
                    atomicOr(&A.status[ST_FLAGS], DUST_FLAG_NAN);
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    moved = fmaxf(moved, fabsf((float)(inc1[d] + inc2[d])) * iw[d]);
                if (!alive) {
                    removed = true;
                    q[0] = __longlong_as_double(0x7ff8000000000000LL);
                }
                A.s.q[0][gi] = q[0]; A.s.q[1][gi] = q[1]; A.s.q[2][gi] = q[2];
                A.s.p[0][gi] = pnew[0]; A.s.p[1][gi] = pnew[1]; A.s.p[2][gi] = pnew[2];
            }
            if (removed && !(isnan(A.s.q[0][gi]))) A.s.q[0][gi] = __longlong_as_double(0x7ff8000000000000LL);
        }
    }
    // warp-aggregated status updates
    const unsigned mask = __ballot_sync(0xffffffffu, removed);
    const unsigned mv = __reduce_max_sync(0xffffffffu, __float_as_uint(moved));
    if ((threadIdx.x & 31) == 0) {
        if (mask) atomicAdd(reinterpret_cast<unsigned long long *>(&A.status[ST_REMOVED_LO]),
                            (unsigned long long)__popc(mask));
        if (mv) atomicMax(&A.status[ST_MAXMOVE], mv);
    }
}

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_step_per_grain(const StepArgs<Real> &a, cudaStream_t s)
{
    if (a.s.n == 0) return cudaSuccess;
    const int64_t blocks = (a.s.n + kStepThreads - 1) / kStepThreads;
    step_per_grain_kernel<Real, GEOM, WEIGHT><<<(unsigned)blocks, kStepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------- predictor ----
// Gas half-step drag predictor (Sec. 3.1, Eqs. Delta_vp and f_D, with
// tau_s <- max(tau_s, |dt|) against the predictor's stiffness): one thread per
// grain gathers the gas at the grain's position x^n (weights of Sec. 3.4),
// and deposits the impulse dt/2 (m/tau') W (v_p - v_g(x^n)) per zone with the
// per-grain fixed-point rule into A.dep (three momentum-like channels).
template <typename Real, int GEOM, int WEIGHT>
__global__ void __launch_bounds__(kStepThreads)
predict_gas_kernel(const StepArgs<Real> A)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= A.s.n) return;
    const double q[3] = {A.s.q[0][gi], A.s.q[1][gi], A.s.q[2][gi]};
    if (isnan(q[0])) return;
    const Real pn[3] = {A.s.p[0][gi], A.s.p[1][gi], A.s.p[2][gi]};
    const int sp = A.s.species ? A.s.species[gi] : 0;
    int host[3];
    Real w[3][3];
    float iw[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) zone_weights<Real, GEOM>(A.g, d, WEIGHT, q[d], host[d], w[d], iw[d]);
    Real acc[4] = {Real(0), Real(0), Real(0), Real(0)};
    const int n0 = A.g.n[0], n1 = A.g.n[1], n2 = A.g.n[2];
#pragma unroll
    for (int c3 = 0; c3 < 3; ++c3) {
        if (n2 <= 1 && c3 != 1) continue;
        const int iz = node_of(host[2], c3 - 1, n2, A.g.bc[2]);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (n1 <= 1 && b != 1) continue;
            const int iy = node_of(host[1], b - 1, n1, A.g.bc[1]);
            const Real wyz = w[1][b] * w[2][c3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (n0 <= 1 && a != 1) continue;
                const int ix = node_of(host[0], a - 1, n0, A.g.bc[0]);
                const Real W = w[0][a] * wyz;
                Real f[4];
                load_gas<Real>(A.gas, ix + (int64_t)n0 * (iy + (int64_t)n1 * iz), f);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] += W * f[c];
            }
        }
    }
    const Real value = A.s.param ? A.s.param[gi] : (Real)A.sp.tau[sp];
    const Real tau = stopping_time<Real, GEOM>(A.ph, A.sp.mode[sp], value, q, acc[0]);
    const Real dt = (Real)A.dt;
    const Real taup = fmax(tau, fabs(dt));
    // mass / quantum, precomputed per species in both precisions
    const Real mq = sizeof(Real) == 4 ? (Real)A.sp.mqf[sp] : (Real)A.sp.mq[sp];
    const Real coef = Real(0.5) * dt * mq / taup;
    Real Dq[4];
#pragma unroll
    for (int c = 0; c < 3; ++c) Dq[c] = coef * (pn[c] - acc[1 + c]);
    Dq[3] = Real(0);
    deposit_fixed<Real>(A.g, A.dep, host, w, Dq, A.status);
}

template <typename Real, int GEOM, int WEIGHT>
cudaError_t launch_predict_gas(const StepArgs<Real> &a, cudaStream_t s)
{
    if (a.s.n == 0) return cudaSuccess;
    const int64_t blocks = (a.s.n + kStepThreads - 1) / kStepThreads;
    predict_gas_kernel<Real, GEOM, WEIGHT><<<(unsigned)blocks, kStepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- sort ----
// Sort key of a grain for a step of half length h: the zone of its predicted
// half-step position (first half drift, periodic wrap, clamped onto the grid
// otherwise).  q is overwritten.
template <typename Real, int GEOM>
__device__ __forceinline__ int32_t predict_key(const GridDev &g, const PhysDev &ph, double q[3],
                                               const Real p[3], Real h)
{
    Real inc[3];
    drift<Real, GEOM>(ph, q, q, p, h, false, inc);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (!inside(g, d, q[d])) {
            if (g.bc[d] == DUST_BC_PERIODIC) q[d] = wrap_once(q[d], g.lo[d], g.hi[d]);
            if (q[d] < g.lo[d]) q[d] = g.lo[d];
            if (q[d] >= g.hi[d]) q[d] = g.edges[d][g.n[d] - 1];
        }
    }
    const int i = locate(g, 0, q[0]), j = locate(g, 1, q[1]), k = locate(g, 2, q[2]);
    return (int32_t)zone_key(g, i, j, k);
}

// Key of a grain = zone of its predicted half-step position for the next
// step (the zone the step kernel will gather from); removed grains get
// key ncell and sort to the end.
template <typename Real, int GEOM>
__global__ void sort_keys_kernel(const SortArgs<Real> A)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < A.src.n;
    int32_t key = valid ? (int32_t)A.g.nkeys : -1;
    double q[3] = {0.0, 0.0, 0.0};
    if (valid) {
        q[0] = A.src.q[0][gi]; q[1] = A.src.q[1][gi]; q[2] = A.src.q[2][gi];
    }
    if (valid && !isnan(q[0])) {
        Real p[3] = {A.src.p[0][gi], A.src.p[1][gi], A.src.p[2][gi]};
        key = predict_key<Real, GEOM>(A.g, A.ph, q, p, (Real)(0.5 * A.dt));
    }
    if (valid) A.key[gi] = key;
    // consecutive grains mostly share a key: one atomic per distinct key in
    // the warp
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&A.count[key], __popc(peers));
}

// Dust mass per zone (Eq. deposition with q_p = m_p) in int64 fixed point,
// with the per-grain rule of the drag deposit: each grain gives the pieces
// rint(W m / quantum) to the non-host nodes of its stencil and the host the
// rest of rint(m / quantum), so the zone sum is the grain sum exactly and
// independent of the order.  The weights (weighting wk: CIC, TSC or volume)
// are evaluated in double precision at the stored positions.
template <int GEOM>
__global__ void deposit_mass_kernel(GridDev g, SpeciesDev sp, int wk, int64_t n, const double *q0,
                                    const double *q1, const double *q2, const uint8_t *species,
                                    unsigned long long *out, unsigned int *status)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double q[3] = {q0[k], q1[k], q2[k]};
    if (isnan(q[0])) return;  // removed grain
    int host[3];
    double w[3][3];
    float iw[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) zone_weights<double, GEOM>(g, d, wk, q[d], host[d], w[d], iw[d]);
    const double M = sp.mq[species ? species[k] : 0];
    if (!(fabs(M) < 4.5e15)) atomicOr(&status[ST_FLAGS], DUST_FLAG_OVERFLOW);
    long long rest = rround(M);
#pragma unroll 1
    for (int nd = 0; nd < 27; ++nd) {
        const int a = nd % 3, b = (nd / 3) % 3, c = nd / 9;
        if (nd == 13 || (g.n[0] <= 1 && a != 1) || (g.n[1] <= 1 && b != 1) || (g.n[2] <= 1 && c != 1))
            continue;
        const long long piece = rround(w[0][a] * w[1][b] * w[2][c] * M);
        if (piece == 0) continue;
        const int ix = node_of(host[0], a - 1, g.n[0], g.bc[0]);
        const int iy = node_of(host[1], b - 1, g.n[1], g.bc[1]);
        const int iz = node_of(host[2], c - 1, g.n[2], g.bc[2]);
        atomicAdd(&out[ix + (int64_t)g.n[0] * (iy + (int64_t)g.n[1] * iz)], (unsigned long long)piece);
        rest -= piece;
    }
    const int64_t h = node_of(host[0], 0, g.n[0], g.bc[0]) +
                      (int64_t)g.n[0] * (node_of(host[1], 0, g.n[1], g.bc[1]) +
                                         (int64_t)g.n[1] * node_of(host[2], 0, g.n[2], g.bc[2]));
    if (rest != 0) atomicAdd(&out[h], (unsigned long long)rest);
}

template <int GEOM>
cudaError_t launch_deposit_mass(const GridDev &g, const SpeciesDev &sp, int wk, int64_t n,
                                const double *const q[3], const uint8_t *species,
                                unsigned long long *out, unsigned int *status, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    deposit_mass_kernel<GEOM><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, sp, wk, n, q[0], q[1], q[2],
                                                                           species, out, status);
    return cudaGetLastError();
}

// Single-precision estimate of a double from its bit fields (the mantissa
// truncated; magnitudes outside the single range clamped): no
// double-precision instruction.  Only an estimate: zone_at corrects it with
// exact comparisons of integer order keys.
__device__ __forceinline__ float float_estimate(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)((unsigned long long)b >> 32);
    const int e = (int)((hi >> 20) & 0x7ff) - 1023 + 127;
    const unsigned sign = hi & 0x80000000u;
    if (e <= 0) return __int_as_float((int)sign);
    if (e >= 255) return __int_as_float((int)(sign | 0x7f7fffffu));
    const unsigned m = (unsigned)((unsigned long long)b >> 29) & 0x7fffffu;
    return __int_as_float((int)(sign | ((unsigned)e << 23) | m));
}

// Zone of x in direction d, exactly as locate() finds it, with the estimate
// taken from float_estimate.
__device__ __forceinline__ int zone_at(const GridDev &g, int d, double x)
{
    const int n = g.n[d];
    if (n <= 1) return 0;
    const long long *ek = g.ekey[d];
    const long long kx = order_key(x);
    int i;
    if (g.edge_kind[d] == EDGE_UNIFORM) {
        i = (int)floorf((float_estimate(x) - (float)g.lo[d]) * g.inv_df[d]);
    } else if (g.edge_kind[d] == EDGE_LOG) {
        i = (int)floorf((logf(float_estimate(x)) - g.log_lo_f[d]) * g.inv_df[d]);
    } else {
        int lo = 0, hi = n;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (ek[mid] <= kx) lo = mid; else hi = mid;
        }
        return lo;
    }
    i = i < 0 ? 0 : (i > n - 1 ? n - 1 : i);
    for (int it = 0; it < 8 && i > 0 && kx < ek[i]; ++it) --i;
    for (int it = 0; it < 8 && i < n - 1 && kx >= ek[i + 1]; ++it) ++i;
    // the bounded walk could stop short only for an estimate far off, which
    // the truncation does not produce for a coordinate inside the grid;
    // fall back to the exact search if it did
    if ((i > 0 && kx < ek[i]) || (i < n - 1 && kx >= ek[i + 1])) return locate(g, d, x);
    return i;
}

// Keys of the zones at x^n (the gas predictor's sort): the key kernel with
// no drift, without double-precision arithmetic for grains inside the grid.
// Grains outside the grid take predict_key with no drift (the same clamping
// and wrapping); the keys equal predict_key's for every grain.
template <int GEOM>
__global__ void zone_keys_kernel(const SortArgs<float> A)
{
    const int64_t gi = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gi < A.src.n;
    int32_t key = valid ? (int32_t)A.g.nkeys : -1;
    double q[3] = {0.0, 0.0, 0.0};
    if (valid) {
        q[0] = A.src.q[0][gi]; q[1] = A.src.q[1][gi]; q[2] = A.src.q[2][gi];
    }
    if (valid && (__double_as_longlong(q[0]) & 0x7fffffffffffffffll) <= 0x7ff0000000000000ll) {
        // -0 as +0, as the no-drift update q + 0 leaves it in predict_key
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (__double_as_longlong(q[d]) == (long long)0x8000000000000000ull) q[d] = 0.0;
        if (inside(A.g, 0, q[0]) && inside(A.g, 1, q[1]) && inside(A.g, 2, q[2])) {
            key = (int32_t)zone_key(A.g, zone_at(A.g, 0, q[0]), zone_at(A.g, 1, q[1]), zone_at(A.g, 2, q[2]));
        } else {
            const float p[3] = {0.f, 0.f, 0.f};
            key = predict_key<float, GEOM>(A.g, A.ph, q, p, 0.f);
        }
    }
    if (valid) A.key[gi] = key;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&A.count[key], __popc(peers));
}

template <int GEOM>
cudaError_t launch_zone_keys(const SortArgs<float> &a, cudaStream_t s)
{
    if (a.src.n == 0) return cudaSuccess;
    const int64_t blocks = (a.src.n + 255) / 256;
    zone_keys_kernel<GEOM><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename Real, int GEOM>
cudaError_t launch_sort_keys(const SortArgs<Real> &a, cudaStream_t s)
{
    if (a.src.n == 0) return cudaSuccess;
    const int64_t blocks = (a.src.n + 255) / 256;
    sort_keys_kernel<Real, GEOM><<<(unsigned)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace dust
