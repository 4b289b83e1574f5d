// Device-side arithmetic of the dust step: locate, weights, drift, kick,
// boundaries.  Templated on the precision of the momentum-like variables
// (Real = float for the mixed path, double for the FP64 path); coordinates
// are always double.
#pragma once

#include <math.h>
#include <stdint.h>

#include "dust_internal.h"

namespace dust {

// ---------------------------------------------------------------- math ----
__device__ __forceinline__ float rexp(float x) { return expf(x); }
__device__ __forceinline__ double rexp(double x) { return exp(x); }
__device__ __forceinline__ float rexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double rexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float rsin(float x) { return sinf(x); }
__device__ __forceinline__ double rsin(double x) { return sin(x); }
__device__ __forceinline__ float rcos(float x) { return cosf(x); }
__device__ __forceinline__ double rcos(double x) { return cos(x); }
__device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ long long rround(float x) { return __float2ll_rn(x); }
__device__ __forceinline__ long long rround(double x) { return __double2ll_rn(x); }

// Shear-periodic shifts of the step at its half and full time: from the
// kernel arguments, or from device memory for steps replayed from a graph.
template <typename Real>
__device__ __forceinline__ double shift_mid_of(const StepArgs<Real> &A)
{
    return A.tdev ? A.tdev[1] : A.ph.shift_mid;
}
template <typename Real>
__device__ __forceinline__ double shift_end_of(const StepArgs<Real> &A)
{
    return A.tdev ? A.tdev[2] : A.ph.shift_end;
}

// A uniform parameter in the working precision (single-precision copies are
// prepared on the host, so the mixed path converts nothing per grain).
template <typename Real>
__device__ __forceinline__ Real pick(double d, float f);
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }

// e - sin(e), without cancellation for small e (Taylor series, |e| < 0.5).
template <typename R>
__device__ __forceinline__ R e_minus_sin(R e)
{
    R s = e * e;
    if (fabs(e) < R(0.5))
        return e * s * (R(1) / R(6)) *
               (R(1) - s * (R(1) / R(20)) * (R(1) - s * (R(1) / R(42)) * (R(1) - s * (R(1) / R(72)))));
    return e - rsin(e);
}

// -------------------------------------------------------------- grid ------
// Zone of direction d containing x (zones are half open [e_i, e_{i+1})).
// A single-precision estimate is corrected against the stored double edges,
// so the chosen zone is the exact one.
__device__ __forceinline__ int locate(const GridDev &g, int d, double x)
{
    const int n = g.n[d];
    if (n <= 1) return 0;
    const long long *ek = g.ekey[d];
    const long long kx = order_key(x);
    int i;
    if (g.edge_kind[d] == EDGE_UNIFORM) {
        i = (int)floorf(((float)x - (float)g.lo[d]) * g.inv_df[d]);
    } else if (g.edge_kind[d] == EDGE_LOG) {
        i = (int)floorf((logf((float)x) - g.log_lo_f[d]) * g.inv_df[d]);
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
    return i;
}

// Stencil node i + o: periodic directions wrap, outflow directions fold onto
// the edge zone (zero-gradient gas, conservative deposit).
__device__ __forceinline__ int node_of(int i, int o, int n, int bc)
{
    if (n <= 1) return 0;
    int k = i + o;
    if (k < 0) return bc == DUST_BC_PERIODIC ? k + n : 0;
    if (k >= n) return bc == DUST_BC_PERIODIC ? k - n : n - 1;
    return k;
}

// ------------------------------------------------------------ weights -----
// 1-D weights of zones (i-1, i, i+1), Sec. 3.4 and App. C.  d = (x - x_i)/dx
// in [-1/2, 1/2), nu = x_i / dx.
template <typename R>
__device__ __forceinline__ void w_cart(int tsc, R d, R w[3])
{
    if (tsc) {  // b1 spline (TSC)
        R a = R(0.5) - d, b = R(0.5) + d;
        w[0] = R(0.5) * a * a;
        w[1] = R(0.75) - d * d;
        w[2] = R(0.5) * b * b;
    } else {    // b0 spline (CIC)
        w[0] = d < R(0) ? -d : R(0);
        w[2] = d > R(0) ? d : R(0);
        w[1] = R(1) - w[0] - w[2];
    }
}

// Eqs. CIC_cylindrical, TSC_cylindrical (measure R dR).
template <typename R>
__device__ __forceinline__ void w_cyl(int tsc, R d, R nu, R w[3])
{
    if (tsc) {
        R inv = R(1) / (R(3) * (d + nu));
        R base = d + R(3) * nu;
        R a = R(0.5) - d, b = R(0.5) + d;
        w[0] = (base - R(2)) * inv * R(0.5) * a * a;
        w[2] = (base + R(2)) * inv * R(0.5) * b * b;
        w[1] = base * inv * (R(0.75) - d * d);
    } else {
        R inv = R(1) / (R(2) * (d + nu));
        R base = d + R(2) * nu;
        R ad = fabs(d);
        w[0] = (base - R(1)) * inv * R(0.5) * (ad - d);
        w[2] = (base + R(1)) * inv * R(0.5) * (ad + d);
        w[1] = base * inv * (R(1) - ad);
    }
}

// Eqs. CIC_spherical_r, TSC_spherical_r (measure r^2 dr).
template <typename R>
__device__ __forceinline__ void w_sphr(int tsc, R d, R nu, R w[3])
{
    R s = d + nu;
    if (tsc) {
        R inv = R(1) / (R(6) * s * s + R(1));
        R a = R(0.5) - d, b = R(0.5) + d;
        R c0 = R(6) * nu * nu + R(2.75) + d * d + R(4) * nu * d;
        R odd = R(8) * nu + R(3) * d;
        w[0] = (c0 - odd) * inv * R(0.5) * a * a;
        w[2] = (c0 + odd) * inv * R(0.5) * b * b;
        R t = d + R(2) * nu;
        w[1] = ((t * t + R(2) * nu * nu + R(0.75)) * (R(0.75) - d * d) - R(0.25)) * inv;
    } else {
        R inv = R(1) / (R(12) * s * s + R(1));
        R ad = fabs(d);
        R base = R(2) * d + R(3) * nu;
        R p = base + R(1.5), m = base - R(1.5);
        R np_ = nu + R(0.5), nm = nu - R(0.5);
        w[0] = (m * m + R(3) * nm * nm) * inv * R(0.5) * (ad - d);
        w[2] = (p * p + R(3) * np_ * np_) * inv * R(0.5) * (ad + d);
        R t = d + R(2) * nu, u = ad - R(1);
        w[1] = (R(3) * t * t + u * u) * inv * (R(1) - ad);
    }
}

// Polar angle (measure sin(theta) dtheta).  CIC: Eq. CIC_spherical_theta
// with the differences of cosines written as products of sines.  TSC: the
// defining integral of the b1 shape in closed form (not printed in the
// paper).  th = theta_p, lo/hi = host zone edges, dr = theta_p - theta_i.
template <typename R>
__device__ __forceinline__ void w_theta(int tsc, R th, R lo, R hi, R dr, R hw, R w[3])
{
    // hw = half the zone width, passed in accurately (hi - lo in single
    // precision would lose digits)
    R sh = rsin(hw);
    if (tsc) {
        R N = R(4) * rsin(th) * sh * sh;
        R ep = hw + dr, em = hw - dr;
        R sp = rsin(R(0.5) * ep), sm = rsin(R(0.5) * em);
        w[2] = (rcos(hi) * e_minus_sin(ep) + R(2) * sp * sp * rsin(hi)) / N;
        w[0] = (R(2) * sm * sm * rsin(lo) - rcos(lo) * e_minus_sin(em)) / N;
    } else {
        R D = R(2) * rsin(th) * sh;
        R s2 = rsin(R(0.5) * dr);
        w[2] = dr > R(0) ? R(2) * rsin(hi + R(0.5) * dr) * s2 / D : R(0);
        w[0] = dr < R(0) ? -R(2) * rsin(lo + R(0.5) * dr) * s2 / D : R(0);
    }
    w[1] = R(1) - w[0] - w[2];
}

// Traditional volume weighting, Eq. CIC_vol: the CIC rule in the volume
// coordinate, i.e. linear interpolation in V = R^2 (cylindrical radius),
// r^3 (spherical radius) or -cos(theta) (polar angle) between the centres of
// the two zones around x.  The nodes are the zones' own centres, with a ghost
// centre one edge-zone width beyond each end of the grid; a difference of V
// is the shell volume |dV| between the two points, so it stays positive when
// a ghost centre lies across the axis or a pole.  Evaluated in double
// precision from the edge tables in both precisions: this is the paper's
// comparison weighting, not a fast path.
__device__ __forceinline__ double vol_node(const GridDev &g, int d, int k)
{
    const int n = g.n[d];
    const double *e = g.edges[d];
    if (k < 0) return g.zc[d][0] - (e[1] - e[0]);
    if (k >= n) return g.zc[d][n - 1] + (e[n] - e[n - 1]);
    return g.zc[d][k];
}

// |cos u - cos v| for u <= v on one side of a pole, as a product of sines.
__device__ __forceinline__ double polar_piece(double u, double v)
{
    return fabs(2.0 * sin(0.5 * (u + v)) * sin(0.5 * (v - u)));
}

// Shell volume between b <= a (per unit of the other coordinates, up to the
// direction's constant factor).
template <int GEOM>
__device__ __forceinline__ double vol_shell(int d, double b, double a)
{
    if (GEOM == GEOM_CYL || d == 0) {
        if (GEOM == GEOM_SPH) return (a - b) * (a * a + a * b + b * b);  // a^3 - b^3
        return (b >= 0.0 || a <= 0.0) ? fabs((a - b) * (a + b)) : a * a + b * b;
    }
    // polar angle: |sin| integrated over [b, a], split at 0 and pi
    const double kPi = 3.14159265358979323846;
    double s = 0.0, u = b;
    if (u < 0.0) {
        const double v = fmin(a, 0.0);
        s += polar_piece(u, v);
        u = v;
    }
    if (u < kPi && a > u) {
        const double v = fmin(a, kPi);
        s += polar_piece(u, v);
        u = v;
    }
    if (a > u) s += polar_piece(u, a);
    return s;
}

template <typename R, int GEOM>
__device__ __forceinline__ void w_volume(const GridDev &g, int d, double x, int i, R w[3])
{
    const double c = g.zc[d][i];
    double lo = 0.0, hi = 0.0;
    if (x >= c) hi = vol_shell<GEOM>(d, c, x) / vol_shell<GEOM>(d, c, vol_node(g, d, i + 1));
    else lo = vol_shell<GEOM>(d, x, c) / vol_shell<GEOM>(d, vol_node(g, d, i - 1), c);
    w[0] = (R)lo;
    w[2] = (R)hi;
    w[1] = (R)(1.0 - lo - hi);
}

// Eq. CIC_vol in single precision relative to the host zone's centre c, for
// a coordinate x = c + u inside the zone: the shell volume between c and x
// (written so that it stays accurate for small u) times the inverse shell
// volume between c and the neighbouring node on that side (ivl, ivh, from
// vol_shell and vol_node in double precision).  d = 0: the radius
// (cylindrical R^2, spherical r^3); d = 1: the spherical polar angle.
template <int GEOM>
__device__ __forceinline__ void w_vol_f(int d, float u, float c, float ivl, float ivh, float w[3])
{
    float num;
    if (GEOM == GEOM_SPH && d == 1) num = 2.f * sinf(c + 0.5f * u) * sinf(0.5f * fabsf(u));
    else if (GEOM == GEOM_SPH) num = fabsf(u) * (3.f * c * c + 3.f * c * u + u * u);
    else num = fabsf(u) * (2.f * c + u);
    w[0] = u < 0.f ? num * ivl : 0.f;
    w[2] = u > 0.f ? num * ivh : 0.f;
    w[1] = 1.f - w[0] - w[2];
}

// Host zone and weights of direction d for coordinate x.  wk: 0 CIC, 1 TSC,
// 2 volume weighting (plain CIC in the directions whose volume coordinate
// is the coordinate itself).
template <typename R, int GEOM>
__device__ __forceinline__ void zone_weights(const GridDev &g, int d, int wk, double x, int &i,
                                             R w[3], float &inv_width)
{
    const int tsc = wk == 1;
    if (g.n[d] <= 1) {
        i = 0; w[0] = R(0); w[1] = R(1); w[2] = R(0);
        inv_width = 0.f;
        return;
    }
    i = locate(g, d, x);
    // offset from the zone centre, scaled by the stored inverse width (no
    // double-precision division on the device)
    const double off = x - g.zc[d][i];
    inv_width = g.ziw_f[d][i];
    const bool single = sizeof(R) == 4;
    const R dd = single ? (R)((float)off * g.ziw_f[d][i]) : (R)(off * g.ziw[d][i]);
    if (wk == 2 && (((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && d == 0) || (GEOM == GEOM_SPH && d == 1))) {
        w_volume<R, GEOM>(g, d, x, i, w);
    } else if ((GEOM == GEOM_CYL || GEOM == GEOM_SPH) && d == 0) {
        const R nu = single ? (R)g.znu_f[d][i] : (R)(g.zc[d][i] * g.ziw[d][i]);
        if (GEOM == GEOM_CYL) w_cyl<R>(tsc, dd, nu, w);
        else w_sphr<R>(tsc, dd, nu, w);
    } else if (GEOM == GEOM_SPH && d == 1) {
        const R lo = single ? (R)g.zlo_f[d][i] : (R)g.edges[d][i];
        const R hi = single ? (R)g.zlo_f[d][i + 1] : (R)g.edges[d][i + 1];
        const R hw = single ? (R)(0.5f / g.ziw_f[d][i]) : (R)(0.5 * (g.edges[d][i + 1] - g.edges[d][i]));
        w_theta<R>(tsc, (R)x, lo, hi, (R)off, hw, w);
    } else {
        w_cart<R>(tsc, dd, w);
    }
}

// ---------------------------------------------------------- boundaries ----
__device__ __forceinline__ double wrap_once(double x, double lo, double hi)
{
    const double L = hi - lo;
    if (x >= hi) { x -= L; if (x < lo) x = lo; }
    else if (x < lo) { x += L; if (x >= hi) x = lo; }
    return x;
}

// Boundary conditions after a half drift.  Returns false when the grain left
// through an outflow boundary (or moved more than a period).  Shearing-box x
// is shear-periodic: y shifts by +-shift and, in the standard frame, v_y by
// +-q Omega Lx.
__device__ __forceinline__ bool inside(const GridDev &g, int d, double x)
{
    const long long k = order_key(x);
    return k >= g.lo_key[d] && k < g.hi_key[d];
}

template <typename Real, int GEOM>
__device__ __forceinline__ bool apply_bc(const GridDev &g, const PhysDev &ph, double shift,
                                         double q[3], Real p[3])
{
    // common case first: every coordinate inside its range
    if (inside(g, 0, q[0]) && inside(g, 1, q[1]) && inside(g, 2, q[2])) return true;
    bool ok = true;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double lo = g.lo[d], hi = g.hi[d];
        if (inside(g, d, q[d])) continue;
        if (g.bc[d] == DUST_BC_OUTFLOW) return false;
        if (GEOM == GEOM_SB && d == 0) {
            if (q[0] >= hi) {
                q[1] += shift;
                if (!ph.fargo) p[1] += pick<Real>(ph.jump_v, ph.jump_v_f);
            } else {
                q[1] -= shift;
                if (!ph.fargo) p[1] -= pick<Real>(ph.jump_v, ph.jump_v_f);
            }
            q[0] = wrap_once(q[0], lo, hi);
            q[1] = wrap_once(q[1], g.lo[1], g.hi[1]);
        } else {
            q[d] = wrap_once(q[d], lo, hi);
        }
        if (q[d] < lo || q[d] >= hi) ok = false;
    }
    if (!ok) return false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (q[d] < g.lo[d] || q[d] >= g.hi[d]) {
            if (g.bc[d] == DUST_BC_OUTFLOW) return false;
            q[d] = wrap_once(q[d], g.lo[d], g.hi[d]);
        }
    }
    return true;
}

// --------------------------------------------------------------- drift ----
// Half drift (Eq. exp_midpoint; Eqs. drift1/drift2_cylindrical; App. B.2.2).
// First half (second == false): metric factors from the coordinates just
// updated; second half: metric factors frozen at the midpoint qm.  inc[]
// receives the coordinate increments (for the displacement diagnostic).
template <typename Real, int GEOM>
__device__ __forceinline__ void drift(const PhysDev &ph, double q[3], const double qm[3],
                                      const Real p[3], Real h, bool second, Real inc[3])
{
    if (GEOM == GEOM_CYL) {
        inc[0] = h * p[0];
        q[0] += (double)inc[0];
        const Real R = (Real)(second ? qm[0] : q[0]);
        inc[1] = h * p[1] / (R * R);
        q[1] += (double)inc[1];
        inc[2] = h * p[2];
        q[2] += (double)inc[2];
    } else if (GEOM == GEOM_SPH) {
        inc[0] = h * p[0];
        q[0] += (double)inc[0];
        const Real r = (Real)(second ? qm[0] : q[0]);
        inc[1] = h * p[1] / (r * r);
        q[1] += (double)inc[1];
        const Real s = rsin((Real)(second ? qm[1] : q[1]));
        inc[2] = h * p[2] / (r * r * s * s);
        q[2] += (double)inc[2];
    } else if (GEOM == GEOM_SB) {
        inc[0] = h * p[0];
        q[0] += (double)inc[0];
        if (ph.fargo) inc[1] = h * (p[1] - pick<Real>(ph.q_om, ph.q_om_f) * (Real)(second ? qm[0] : q[0]));
        else inc[1] = h * p[1];
        q[1] += (double)inc[1];
        inc[2] = h * p[2];
        q[2] += (double)inc[2];
    } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            inc[d] = h * p[d];
            q[d] += (double)inc[d];
        }
    }
}

// ------------------------------------------------------ stopping time -----
// qm: half-step coordinates, in double or in the working precision.
template <typename Real, int GEOM, typename QT>
__device__ __forceinline__ Real stopping_time(const PhysDev &ph, int mode, Real value,
                                              const QT qm[3], Real rho_g)
{
    if (mode == DUST_TAU_CONST) return value;
    if (mode == DUST_TAU_EPSTEIN) return value / rho_g;
    if (GEOM == GEOM_CYL || GEOM == GEOM_SPH) {
        Real R = (Real)qm[0];
        if (GEOM == GEOM_SPH) R *= rsin((Real)qm[1]);
        return value * rsqrt_(R * R * R / pick<Real>(ph.gm, ph.gm_f));
    }
    return value / pick<Real>(ph.omega, ph.omega_f);
}

// ------------------------------------------------------ semi-implicit ----
// Semi-implicit kick (Sec. 3.2.1, Eqs. semi-implicit, a_linear, Lambda):
// v^{n+1} = v^n + Lambda^{-1} dt a_tot(x^{n+1/2}, v^n, v_g), Lambda =
// I - (dt/2) d a_tot / d v, with the drag -(v - v_g)/tau giving b = dt/(2 tau)
// on the diagonal and the shearing-box Coriolis (standard frame) or
// orbital-advection terms off it.  Cartesian and shearing-box geometries;
// it = 1/tau (0 for tau = infinity).  Returns the same quantities as kick().
template <typename Real, int GEOM, typename QT>
__device__ __forceinline__ void kick_si(const PhysDev &ph, const QT qm[3], const Real pn[3],
                                        const Real vg[3], Real it, Real dt, Real pp[3],
                                        Real a[3], Real dH[3])
{
    const Real b = Real(0.5) * dt * it;
    const Real l00 = Real(1) + b;
    Real at[3] = {Real(0), Real(0), Real(0)};
    Real l01 = Real(0), l10 = Real(0), Om = Real(0), q = Real(0), az = Real(0);
    if (GEOM == GEOM_SB) {
        Om = pick<Real>(ph.omega, ph.omega_f);
        q = pick<Real>(ph.qshear, ph.qshear_f);
        az = ph.vgrav ? -Om * Om * (Real)qm[2] : Real(0);
        if (ph.fargo) {
            at[0] = Real(2) * Om * pn[1];
            at[1] = (q - Real(2)) * Om * pn[0];
            l10 = (Real(1) - Real(0.5) * q) * Om * dt;
        } else {
            at[0] = Real(2) * Om * (pn[1] + q * Om * (Real)qm[0]);
            at[1] = -Real(2) * Om * pn[0];
            l10 = Om * dt;
        }
        l01 = -Om * dt;
        at[2] = az;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) at[d] += (vg[d] - pn[d]) * it;
    const Real det = l00 * l00 - l01 * l10;
    const Real r0 = dt * at[0], r1 = dt * at[1];
    pp[0] = pn[0] + (l00 * r0 - l01 * r1) / det;
    pp[1] = pn[1] + (-l10 * r0 + l00 * r1) / det;
    pp[2] = pn[2] + dt * at[2] / l00;
    const Real vx = Real(0.5) * (pn[0] + pp[0]);
    const Real vy = Real(0.5) * (pn[1] + pp[1]);
    const Real vz = Real(0.5) * (pn[2] + pp[2]);
    if (GEOM == GEOM_SB) {
        if (ph.fargo) {
            a[0] = Real(2) * Om * vy;
            a[1] = (q - Real(2)) * Om * vx;
        } else {
            a[0] = Real(2) * Om * (vy + q * Om * (Real)qm[0]);
            a[1] = -Real(2) * Om * vx;
        }
        a[2] = az;
    } else {
        a[0] = a[1] = a[2] = Real(0);
    }
    dH[0] = vx;
    dH[1] = vy;
    dH[2] = vz;
}

// ---------------------------------------------------------------- kick ----
// Kick with E = exp(-dt/tau), cg = 1 - E = h1/tau, h1 = dt phi1(-dt/tau)
// (Eqs. phi1, h1); returns the new p, the non-frictional acceleration a at
// (q^{n+1/2}, p^{n+1/2}) and dH/dp at the half step.
template <typename Real, int GEOM, typename QT>
__device__ __forceinline__ void kick(const PhysDev &ph, const QT qm[3], const Real pn[3],
                                     const Real vg[3], Real E, Real cg, Real h1, Real pp[3],
                                     Real a[3], Real dH[3])
{
    if (GEOM == GEOM_SB) {
        // App. B.1: R v^{n+1} = E v^n + h1 G(x^{n+1/2}, v^n/2, v_g^{n+1/2})
        const Real Om = pick<Real>(ph.omega, ph.omega_f), q = pick<Real>(ph.qshear, ph.qshear_f);
        const Real az = ph.vgrav ? -Om * Om * (Real)qm[2] : Real(0);
        const Real Om1 = Om * h1;
        Real G0, G1;
        if (ph.fargo) {
            G0 = Om * pn[1];
            G1 = Real(0.5) * (q - Real(2)) * Om * pn[0];
        } else {
            G0 = Om * pn[1] + Real(2) * q * Om * Om * (Real)qm[0];
            G1 = -Om * pn[0];
        }
        const Real r0 = E * pn[0] + h1 * G0 + cg * vg[0];
        const Real r1 = E * pn[1] + h1 * G1 + cg * vg[1];
        pp[2] = E * pn[2] + h1 * az + cg * vg[2];
        const Real Om2 = ph.fargo ? Om1 * (Real(1) - Real(0.5) * q) : Om1;
        const Real inv = Real(1) / (Real(1) + Om1 * Om2);
        pp[0] = inv * (r0 + Om1 * r1);
        pp[1] = inv * (r1 - Om2 * r0);
        const Real vx = Real(0.5) * (pn[0] + pp[0]);
        const Real vy = Real(0.5) * (pn[1] + pp[1]);
        if (ph.fargo) {
            a[0] = Real(2) * Om * vy;
            a[1] = (q - Real(2)) * Om * vx;
        } else {
            a[0] = Real(2) * Om * (vy + q * Om * (Real)qm[0]);
            a[1] = -Real(2) * Om * vx;
        }
        a[2] = az;
        dH[0] = vx;
        dH[1] = vy;
        dH[2] = Real(0.5) * (pn[2] + pp[2]);
    } else if (GEOM == GEOM_CYL) {
        // App. B.2.1: v_z, l_phi, then v_R with (l^2)^{n+1/2}
        const Real R = (Real)qm[0];
        Real gR = Real(0), gz = Real(0);
        if (ph.gm != 0.0) {
            if (ph.vgrav) {
                const Real z = (Real)qm[2];
                const Real r2 = R * R + z * z;
                const Real ir3 = Real(1) / (r2 * rsqrt_(r2));
                gR = -pick<Real>(ph.gm, ph.gm_f) * R * ir3;
                gz = -pick<Real>(ph.gm, ph.gm_f) * z * ir3;
            } else {
                gR = -pick<Real>(ph.gm, ph.gm_f) / (R * R);
            }
        }
        pp[2] = E * pn[2] + h1 * gz + cg * vg[2];
        pp[1] = E * pn[1] + cg * vg[1];
        const Real l2 = Real(0.5) * (pn[1] * pn[1] + pp[1] * pp[1]);
        const Real aR = l2 / (R * R * R) + gR;
        pp[0] = E * pn[0] + h1 * aR + cg * vg[0];
        a[0] = aR; a[1] = Real(0); a[2] = gz;
        dH[0] = Real(0.5) * (pn[0] + pp[0]);
        dH[1] = Real(0.5) * (pn[1] + pp[1]) / (R * R);
        dH[2] = Real(0.5) * (pn[2] + pp[2]);
    } else if (GEOM == GEOM_SPH) {
        // App. B.2.2: l_phi, l_theta, then v_r, averaged squares
        const Real r = (Real)qm[0];
        const Real th = (Real)qm[1];
        const Real st = rsin(th), ct = rcos(th);
        const Real gr = ph.gm != 0.0 ? -pick<Real>(ph.gm, ph.gm_f) / (r * r) : Real(0);
        pp[2] = E * pn[2] + cg * vg[2];
        const Real lp2 = Real(0.5) * (pn[2] * pn[2] + pp[2] * pp[2]);
        const Real ath = lp2 * ct / (r * r * st * st * st);
        pp[1] = E * pn[1] + h1 * ath + cg * vg[1];
        const Real lt2 = Real(0.5) * (pn[1] * pn[1] + pp[1] * pp[1]);
        const Real ar = (lt2 + lp2 / (st * st)) / (r * r * r) + gr;
        pp[0] = E * pn[0] + h1 * ar + cg * vg[0];
        a[0] = ar; a[1] = ath; a[2] = Real(0);
        dH[0] = Real(0.5) * (pn[0] + pp[0]);
        dH[1] = Real(0.5) * (pn[1] + pp[1]) / (r * r);
        dH[2] = Real(0.5) * (pn[2] + pp[2]) / (r * r * st * st);
    } else {
        // Eq. kick_modified: drag only
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            pp[d] = E * pn[d] + cg * vg[d];
            a[d] = Real(0);
            dH[d] = Real(0.5) * (pn[d] + pp[d]);
        }
    }
}

// The configured pusher: semi-implicit (Cartesian and shearing box only) or
// exponential midpoint.
template <typename Real, int GEOM, typename QT>
__device__ __forceinline__ void kick_any(const PhysDev &ph, const QT qm[3], const Real pn[3],
                                         const Real vg[3], Real tau, Real dt, Real E, Real cg,
                                         Real h1, Real pp[3], Real a[3], Real dH[3])
{
    if ((GEOM == GEOM_CART || GEOM == GEOM_SB) && ph.pusher == DUST_PUSHER_SEMI_IMPLICIT)
        kick_si<Real, GEOM>(ph, qm, pn, vg, Real(1) / tau, dt, pp, a, dH);
    else
        kick<Real, GEOM>(ph, qm, pn, vg, E, cg, h1, pp, a, dH);
}

}  // namespace dust
