/*
 * Oracle for the dust drag-coupling step of Mignone, Flock & Vaidya,
 * "A Particle Module for the PLUTO Code: III - Dust" (arXiv:1908.10793).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, double-precision
 * CPU restatement of the method, used by the tests, by the smoke check and
 * by the CPU-baseline leg of the benchmark.  Nothing on the product path
 * links, loads or calls it, and it shares no code, header or table with the
 * CUDA library.
 *
 * One call of oracle_step() advances every active grain by one exponential
 * midpoint (EM) drift-kick-drift step (Sec. 3.2.2, Eq. exp_midpoint; App. B)
 * and deposits the drag back-reaction on the grid (Eq. dust_feedback_final),
 * grain by grain, in the order the paper states the algorithm:
 *
 *   1. half drift of the coordinates          (Eq. exp_midpoint; Eqs. B.1 drift)
 *   2. host zone and 1-D weights at x^{n+1/2}  (Sec. 3.4, Eqs. weight, b0, b1,
 *                                              CIC/TSC_cylindrical, App. C;
 *                                              or the volume weights of Eq.
 *                                              CIC_vol)
 *   3. gather of gas rho and momentum-like velocity (Eq. Delta_vp)
 *   4. E = exp(-dt/tau), h1 = tau (1 - exp(-dt/tau))   (Eqs. phi1, h1)
 *   5. kick, per geometry                      (Eq. kick_modified; App. B.1, B.2)
 *   6. second half drift with the midpoint metric factors
 *   7. boundaries (periodic, shear-periodic, outflow)
 *   8. deposit  -m W (dp - dt a)  and its energy   (Eq. dust_feedback_final)
 *
 * The deposit is accumulated densely in double precision; the optional
 * feedback update of the gas momentum (corrector term of the RK2 step,
 * Sec. 3.1) is applied after all grains.
 *
 * Readings of points the paper leaves open are listed in the design notes and
 * are repeated where they are used below.
 *
 * Parity status: every part is pinned by a reference built outside this
 * file.  The weights on non-uniform radial grids and the theta-TSC weights,
 * which the paper does not print, follow stated readings (see the notes at
 * each function) and are pinned by quadrature of their defining integral.
 * The deposit channels are pinned by the drag impulse and drag work of an
 * independently integrated trajectory in the shearing box (both frames),
 * and the energy channel in the curvilinear geometries by the grain's
 * mechanical-energy change, to third order per step; the Epstein stopping
 * time by the relaxation of a grain with the TSC-gathered density; the
 * fixed-point rule by integer identities and a closed-form case; the
 * shear-periodic boundary by the sheared image of a wider box.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OG_CARTESIAN 0
#define OG_SHEARING_BOX 1
#define OG_CYLINDRICAL 2
#define OG_SPHERICAL 3

#define OB_PERIODIC 0
#define OB_OUTFLOW 1

#define OW_CIC 0
#define OW_TSC 1
#define OW_VOLUME 2  /* traditional volume weighting, Eq. CIC_vol (comparator) */

#define OP_EM 0             /* exponential midpoint, Sec. 3.2.2                */
#define OP_SEMI_IMPLICIT 1  /* semi-implicit drift-kick-drift, Sec. 3.2.1       */

#define OT_CONST 0   /* tau_s given directly                                  */
#define OT_STOKES 1  /* St given: tau_s = St / Omega_K at the grain           */
#define OT_EPSTEIN 2 /* tau_s = value / rho_gathered  (Sec. 2, tau_s ~ 1/rho) */

/* 1-D weight kinds (which formula of Sec. 3.4 / App. C is used). */
#define W1_CART_CIC 0
#define W1_CART_TSC 1
#define W1_CYL_R_CIC 2
#define W1_CYL_R_TSC 3
#define W1_SPH_R_CIC 4
#define W1_SPH_R_TSC 5
#define W1_SPH_TH_CIC 6
#define W1_SPH_TH_TSC 7
#define W1_CYL_R_VOL 8   /* linear interpolation in R^2 between zone centres   */
#define W1_SPH_R_VOL 9   /* ... in r^3                                          */
#define W1_SPH_TH_VOL 10 /* ... in the polar-angle volume coordinate -cos(th)  */

typedef struct {
    int geom;             /* OG_*                                             */
    int fargo;            /* shearing box: 1 = orbital-advection residual form */
    double omega, q;      /* shearing box Omega and shear parameter q         */
    double gm;            /* point-mass GM (cylindrical / spherical)          */
    int vertical_gravity; /* SB: -Omega^2 z; cylindrical: z part of GM gravity */
    int n[3];             /* zones per direction (1 = direction not gridded)  */
    const double *edges[3]; /* n[d]+1 increasing zone edges per direction     */
    int bc[3];            /* OB_* per direction                               */
    int weight;           /* OW_CIC, OW_TSC or OW_VOLUME                      */
    int n_species;
    const double *sp_mass;
    const int *sp_tau_mode;
    const double *sp_tau;
    int feedback_apply;   /* 1: add the deposit to the gas momentum           */
    int pusher;           /* OP_EM or OP_SEMI_IMPLICIT (Cartesian, shearing box) */
} oracle_problem;

/* ------------------------------------------------------------------------- */
/* Grid helpers                                                               */
/* ------------------------------------------------------------------------- */

/* Zone containing x: largest i with edges[i] <= x (zones are [lo, hi)). */
int oracle_locate(const double *edges, int n, double x)
{
    if (n <= 1) return 0;
    if (x < edges[0]) return 0;
    if (x >= edges[n]) return n - 1;
    int lo = 0, hi = n; /* edges[lo] <= x < edges[hi] */
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (edges[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

/* Index of stencil node i+o in a direction with n zones.  Periodic
 * directions wrap; outflow directions fold onto the edge zone (zero-gradient
 * ghost for the gather, fold-back for the deposit, which keeps the deposit
 * conservative).  Reading: the paper does not state the non-periodic case. */
static int node_index(int i, int o, int n, int bc)
{
    int k = i + o;
    if (n <= 1) return 0;
    if (k < 0) return bc == OB_PERIODIC ? k + n : 0;
    if (k >= n) return bc == OB_PERIODIC ? k - n : n - 1;
    return k;
}

/* ------------------------------------------------------------------------- */
/* 1-D weights, Sec. 3.4 and App. C.                                          */
/* w[0], w[1], w[2] are the weights of zones i-1, i, i+1 where i hosts x and  */
/* [lo, hi) are the edges of zone i.                                          */
/* ------------------------------------------------------------------------- */

/* Cylindrical radial CIC, Eq. CIC_cylindrical: delta=(R_p-R_i)/dR,
 * nu = R_i/dR.  On non-uniform grids the host zone's own width and centre
 * are used (reading: the formula is the defining integral with the three
 * stencil nodes taking the shape below, inside and above the host zone). */
static void w_cyl_r_cic(double d, double nu, double w[3])
{
    double den = 2.0 * d + 2.0 * nu;
    w[1] = (d + 2.0 * nu) / den * (1.0 - fabs(d));
    w[2] = (d + 2.0 * nu + 1.0) / den * (fabs(d) + d) / 2.0;
    w[0] = (d + 2.0 * nu - 1.0) / den * (fabs(d) - d) / 2.0;
}

/* Cylindrical radial TSC, Eq. TSC_cylindrical. */
static void w_cyl_r_tsc(double d, double nu, double w[3])
{
    double den = 3.0 * d + 3.0 * nu;
    w[1] = (d + 3.0 * nu) / den * (0.75 - d * d);
    w[2] = (d + 3.0 * nu + 2.0) / den * 0.5 * (0.5 + d) * (0.5 + d);
    w[0] = (d + 3.0 * nu - 2.0) / den * 0.5 * (0.5 - d) * (0.5 - d);
}

/* Spherical radial CIC, Eq. CIC_spherical_r. */
static void w_sph_r_cic(double d, double nu, double w[3])
{
    double den = 12.0 * (d + nu) * (d + nu) + 1.0;
    double a = d + 2.0 * nu, b = fabs(d) - 1.0;
    w[1] = (3.0 * a * a + b * b) / den * (1.0 - fabs(d));
    double cp = 2.0 * d + 3.0 * nu + 1.5, cm = 2.0 * d + 3.0 * nu - 1.5;
    w[2] = (cp * cp + 3.0 * (nu + 0.5) * (nu + 0.5)) / den * (fabs(d) + d) / 2.0;
    w[0] = (cm * cm + 3.0 * (nu - 0.5) * (nu - 0.5)) / den * (fabs(d) - d) / 2.0;
}

/* Spherical radial TSC, Eq. TSC_spherical_r. */
static void w_sph_r_tsc(double d, double nu, double w[3])
{
    double den = 6.0 * (d + nu) * (d + nu) + 1.0;
    double a = d + 2.0 * nu;
    w[1] = ((a * a + 2.0 * nu * nu + 0.75) * (0.75 - d * d) - 0.25) / den;
    w[2] = (d * d + (4.0 * nu + 3.0) * d + 6.0 * nu * nu + 8.0 * nu + 2.75) / den
           * 0.5 * (0.5 + d) * (0.5 + d);
    w[0] = (d * d + (4.0 * nu - 3.0) * d + 6.0 * nu * nu - 8.0 * nu + 2.75) / den
           * 0.5 * (0.5 - d) * (0.5 - d);
}

/* Spherical theta CIC, Eq. CIC_spherical_theta with delta = theta_p - theta_i
 * in radians.  Reading: the printed W_{i-1} has a sign garble; the integral of
 * sin(theta) over the overlap gives W_{i+-1} = +-[cos x_{i+-1/2} -
 * cos(x_{i+-1/2} + delta)] / D * H(+-delta). */
static void w_sph_th_cic(double th, double lo, double hi, double w[3])
{
    double tc = 0.5 * (lo + hi);
    double d = th - tc;
    double D = cos(lo + d) - cos(hi + d);
    w[0] = 0.0; w[2] = 0.0;
    if (d > 0.0) w[2] = (cos(hi) - cos(hi + d)) / D;
    if (d < 0.0) w[0] = -(cos(lo) - cos(lo + d)) / D;
    w[1] = 1.0 - w[0] - w[2];
}

/* Spherical theta TSC.  Not printed in the paper (App. C gives theta-CIC
 * only).  Reading: the defining integral, Eq. weight with Eq. shape_curv,
 * b1 of half-width h = dtheta centred on theta_p = t and measure sin(theta).
 * Integrating (1 - |u|/h) sin(t+u) by parts over the part of the shape that
 * lies in zone i+1 (an interval of width e = h/2 + delta starting at angle c)
 * gives  [cos(c) (e - sin e) + 2 sin^2(e/2) sin(c)] / h,  over zone i-1
 * (width e = h/2 - delta ending at angle c)  [-cos(c) (e - sin e) +
 * 2 sin^2(e/2) sin(c)] / h, and over the whole shape 4 sin(t) sin^2(h/2) / h.
 * These are the plain antiderivative differences rearranged so that no O(1)
 * terms cancel. */
static void w_sph_th_tsc(double th, double lo, double hi, double w[3])
{
    double h = hi - lo;
    double d = th - 0.5 * (lo + hi);
    double sh = sin(0.5 * h);
    double N = 4.0 * sin(th) * sh * sh;
    double ep = 0.5 * h + d, cp = hi;          /* zone i+1: [hi, th + h]     */
    double em = 0.5 * h - d, cm = lo;          /* zone i-1: [th - h, lo]     */
    double sp = sin(0.5 * ep), sm = sin(0.5 * em);
    w[2] = (cos(cp) * (ep - sin(ep)) + 2.0 * sp * sp * sin(cp)) / N;
    w[0] = (-cos(cm) * (em - sin(em)) + 2.0 * sm * sm * sin(cm)) / N;
    w[1] = 1.0 - w[0] - w[2];
}

void oracle_weights_1d(int kind, double x, double lo, double hi, double w[3])
{
    double dx = hi - lo;
    double xc = 0.5 * (lo + hi);
    double d = (x - xc) / dx;
    double nu = xc / dx;
    switch (kind) {
    case W1_CART_CIC: /* b0 spline: nu -> infinity limit of Eq. CIC_cylindrical */
        w[0] = d < 0.0 ? -d : 0.0;
        w[1] = 1.0 - fabs(d);
        w[2] = d > 0.0 ? d : 0.0;
        break;
    case W1_CART_TSC: /* b1 spline: nu -> infinity limit of Eq. TSC_cylindrical */
        w[0] = 0.5 * (0.5 - d) * (0.5 - d);
        w[1] = 0.75 - d * d;
        w[2] = 0.5 * (0.5 + d) * (0.5 + d);
        break;
    case W1_CYL_R_CIC: w_cyl_r_cic(d, nu, w); break;
    case W1_CYL_R_TSC: w_cyl_r_tsc(d, nu, w); break;
    case W1_SPH_R_CIC: w_sph_r_cic(d, nu, w); break;
    case W1_SPH_R_TSC: w_sph_r_tsc(d, nu, w); break;
    case W1_SPH_TH_CIC: w_sph_th_cic(x, lo, hi, w); break;
    case W1_SPH_TH_TSC: w_sph_th_tsc(x, lo, hi, w); break;
    default: w[0] = 0.0; w[1] = 1.0; w[2] = 0.0;
    }
}

/* ------------------------------------------------------------------------- */
/* Traditional volume weighting, Eq. CIC_vol (Sec. 3.4): the Cartesian CIC  */
/* rule with the linear coordinate replaced by the volume coordinate, i.e.  */
/* linear interpolation in V between the centres of the two zones around x. */
/* The paper prints the cylindrical radial case, V = R^2; the same          */
/* statement gives V = r^3 for the spherical radius and V = -cos(theta) for */
/* the polar angle (the volume element is R dR, r^2 dr, sin(theta) dtheta). */
/* Readings: the two nodes are the actual zone centres (on a non-uniform    */
/* grid the neighbours' own centres), with a ghost centre one edge-zone     */
/* width beyond each end of the grid; the volume-coordinate difference of   */
/* two points is the volume of the shell between them, |dV| integrated from */
/* one to the other, which stays positive when a ghost centre lies across   */
/* the axis (R < 0) or a pole (theta < 0 or theta > pi).                     */
/* ------------------------------------------------------------------------- */

/* Volume (per unit of the other coordinates, up to a constant factor) of
 * the shell between coordinates b <= a for a volume-weight kind. */
static double shell_volume(int kind, double b, double a)
{
    if (kind == W1_CYL_R_VOL) {
        /* int_b^a 2|R| dR: a^2 - b^2 on each side of the axis */
        if (b >= 0.0 || a <= 0.0) return fabs((a - b) * (a + b));
        return a * a + b * b;
    }
    if (kind == W1_SPH_R_VOL) {
        /* int_b^a 3 r^2 dr = a^3 - b^3 */
        return (a - b) * (a * a + a * b + b * b);
    }
    /* polar angle: int_b^a |sin t| dt, split where sin changes sign; on a
     * piece [u, v] of one sign it is |cos u - cos v| = |2 sin((u+v)/2)
     * sin((v-u)/2)| */
    double cuts[4] = {b, 0.0, 3.14159265358979323846, a};
    double total = 0.0;
    double u = b;
    for (int k = 1; k < 4; k++) {
        double v = k < 3 ? cuts[k] : a;
        if (v <= u) continue;
        if (v > a) v = a;
        total += fabs(2.0 * sin(0.5 * (u + v)) * sin(0.5 * (v - u)));
        u = v;
    }
    return total;
}

/* Centre of zone k of a direction with n zones; ghost centres one edge-zone
 * width beyond the ends. */
static double zone_centre(const double *edges, int n, int k)
{
    if (k < 0) return 0.5 * (edges[0] + edges[1]) - (edges[1] - edges[0]);
    if (k >= n) return 0.5 * (edges[n - 1] + edges[n]) + (edges[n] - edges[n - 1]);
    return 0.5 * (edges[k] + edges[k + 1]);
}

/* Weights of zones (i-1, i, i+1) for a grain at x hosted by zone i. */
void oracle_weights_vol(int kind, double x, const double *edges, int n, int i, double w[3])
{
    double c = zone_centre(edges, n, i);
    w[0] = 0.0;
    w[2] = 0.0;
    if (x >= c) {
        /* Eq. CIC_vol with R_i = c, R_{i+1} = the next centre */
        double cp = zone_centre(edges, n, i + 1);
        w[2] = shell_volume(kind, c, x) / shell_volume(kind, c, cp);
        w[1] = 1.0 - w[2];
    } else {
        /* Eq. CIC_vol with R_i = the previous centre, R_{i+1} = c */
        double cm = zone_centre(edges, n, i - 1);
        w[0] = shell_volume(kind, x, c) / shell_volume(kind, cm, c);
        w[1] = 1.0 - w[0];
    }
}

/* Which 1-D weight formula each direction uses (Sec. 3.4: the product of
 * three 1-D factors, W = W(x1) W(x2) W(x3)). */
static int weight_kind(const oracle_problem *P, int d)
{
    if (P->weight == OW_VOLUME) {
        /* the volume coordinate of a Cartesian-like direction is the
         * coordinate itself: plain CIC there */
        if (P->geom == OG_CYLINDRICAL && d == 0) return W1_CYL_R_VOL;
        if (P->geom == OG_SPHERICAL && d == 0) return W1_SPH_R_VOL;
        if (P->geom == OG_SPHERICAL && d == 1) return W1_SPH_TH_VOL;
        return W1_CART_CIC;
    }
    int tsc = P->weight == OW_TSC;
    if (P->geom == OG_CYLINDRICAL && d == 0) return tsc ? W1_CYL_R_TSC : W1_CYL_R_CIC;
    if (P->geom == OG_SPHERICAL && d == 0) return tsc ? W1_SPH_R_TSC : W1_SPH_R_CIC;
    if (P->geom == OG_SPHERICAL && d == 1) return tsc ? W1_SPH_TH_TSC : W1_SPH_TH_CIC;
    return tsc ? W1_CART_TSC : W1_CART_CIC;
}

/* 1-D weights of direction d for a grain at x hosted by zone i. */
static void direction_weights(const oracle_problem *P, int d, int kind, double x, int i,
                              double w[3])
{
    if (kind >= W1_CYL_R_VOL)
        oracle_weights_vol(kind, x, P->edges[d], P->n[d], i, w);
    else
        oracle_weights_1d(kind, x, P->edges[d][i], P->edges[d][i + 1], w);
}

/* ------------------------------------------------------------------------- */
/* Boundaries                                                                  */
/* ------------------------------------------------------------------------- */

/* One periodic wrap of x into [lo, hi). */
static double wrap_once(double x, double lo, double hi)
{
    double L = hi - lo;
    if (x >= hi) { x -= L; if (x < lo) x = lo; }
    else if (x < lo) { x += L; if (x >= hi) x = lo; }
    return x;
}

/* Apply the boundary conditions to a grain at time t.  Returns 0 if the
 * grain left through an outflow boundary.  Shearing box x-boundaries are
 * shear-periodic: leaving through +x the grain re-enters at -x with
 * y += q Omega Lx t (mod Ly); the standard-frame v_y gains q Omega Lx, the
 * residual velocity of the orbital-advection frame is unchanged (Sec. 2.1). */
static int apply_bc(const oracle_problem *P, double q[3], double p[3], double t)
{
    for (int d = 0; d < 3; d++) {
        double lo = P->edges[d][0], hi = P->edges[d][P->n[d]];
        if (q[d] >= lo && q[d] < hi) continue;
        if (P->bc[d] == OB_OUTFLOW) return 0;
        if (P->geom == OG_SHEARING_BOX && d == 0) {
            double Lx = hi - lo;
            double ylo = P->edges[1][0], yhi = P->edges[1][P->n[1]];
            double shift = fmod(P->q * P->omega * Lx * t, yhi - ylo);
            if (q[0] >= hi) {
                q[1] += shift;
                if (!P->fargo) p[1] += P->q * P->omega * Lx;
            } else {
                q[1] -= shift;
                if (!P->fargo) p[1] -= P->q * P->omega * Lx;
            }
            q[0] = wrap_once(q[0], lo, hi);
            q[1] = wrap_once(q[1], ylo, yhi);
        } else {
            q[d] = wrap_once(q[d], lo, hi);
        }
        if (q[d] < lo || q[d] >= hi) return 0; /* moved more than a period */
    }
    /* the y-shift above may have pushed y out of range once more */
    for (int d = 0; d < 3; d++) {
        double lo = P->edges[d][0], hi = P->edges[d][P->n[d]];
        if (q[d] < lo || q[d] >= hi) {
            if (P->bc[d] == OB_OUTFLOW) return 0;
            q[d] = wrap_once(q[d], lo, hi);
        }
    }
    return 1;
}

/* ------------------------------------------------------------------------- */
/* Drifts (Eq. exp_midpoint; Eqs. drift1/drift2_cylindrical; App. B.2.2).     */
/* qm[] receives the metric quantities used by both half drifts.              */
/* ------------------------------------------------------------------------- */

/* First half drift.  Shearing box with orbital advection: dy/dt includes the
 * mean shear -q Omega x, evaluated at the drifted x (reading, by analogy with
 * the midpoint R^2 of the cylindrical drift). */
static void drift_first(const oracle_problem *P, double q[3], const double p[3], double h)
{
    switch (P->geom) {
    case OG_CYLINDRICAL: {
        q[0] = q[0] + h * p[0];
        q[1] = q[1] + h * p[1] / (q[0] * q[0]);
        q[2] = q[2] + h * p[2];
        break;
    }
    case OG_SPHERICAL: {
        q[0] = q[0] + h * p[0];
        q[1] = q[1] + h * p[1] / (q[0] * q[0]);
        double s = sin(q[1]);
        q[2] = q[2] + h * p[2] / (q[0] * q[0] * s * s);
        break;
    }
    case OG_SHEARING_BOX:
        q[0] = q[0] + h * p[0];
        if (P->fargo) q[1] = q[1] + h * (p[1] - P->q * P->omega * q[0]);
        else q[1] = q[1] + h * p[1];
        q[2] = q[2] + h * p[2];
        break;
    default:
        q[0] += h * p[0]; q[1] += h * p[1]; q[2] += h * p[2];
    }
}

/* Second half drift: the metric factors (R^2, r^2, r^2 sin^2 theta, and the
 * shear term's x) stay at their midpoint values qm[]. */
static void drift_second(const oracle_problem *P, double q[3], const double qm[3],
                         const double p[3], double h)
{
    switch (P->geom) {
    case OG_CYLINDRICAL:
        q[0] = q[0] + h * p[0];
        q[1] = q[1] + h * p[1] / (qm[0] * qm[0]);
        q[2] = q[2] + h * p[2];
        break;
    case OG_SPHERICAL: {
        double s = sin(qm[1]);
        q[0] = q[0] + h * p[0];
        q[1] = q[1] + h * p[1] / (qm[0] * qm[0]);
        q[2] = q[2] + h * p[2] / (qm[0] * qm[0] * s * s);
        break;
    }
    case OG_SHEARING_BOX:
        q[0] = q[0] + h * p[0];
        if (P->fargo) q[1] = q[1] + h * (p[1] - P->q * P->omega * qm[0]);
        else q[1] = q[1] + h * p[1];
        q[2] = q[2] + h * p[2];
        break;
    default:
        q[0] += h * p[0]; q[1] += h * p[1]; q[2] += h * p[2];
    }
}

/* ------------------------------------------------------------------------- */
/* External (non-drag) forces                                                 */
/* ------------------------------------------------------------------------- */

/* Point-mass gravity at the midpoint, in the components the kick needs:
 * cylindrical (g_R, g_phi, g_z), spherical (g_r, g_theta, g_phi). */
static void gravity(const oracle_problem *P, const double qm[3], double g[3])
{
    g[0] = g[1] = g[2] = 0.0;
    if (P->gm == 0.0) return;
    if (P->geom == OG_CYLINDRICAL) {
        double R = qm[0], z = qm[2];
        if (P->vertical_gravity) {
            double r2 = R * R + z * z;
            double r3 = r2 * sqrt(r2);
            g[0] = -P->gm * R / r3;
            g[2] = -P->gm * z / r3;
        } else {
            g[0] = -P->gm / (R * R);
        }
    } else if (P->geom == OG_SPHERICAL) {
        g[0] = -P->gm / (qm[0] * qm[0]);
    }
}

/* Stopping time of a grain (Sec. 2, Epstein regime; constant Stokes number
 * as in Secs. 4.5-4.6: tau_s = St / Omega_K with Omega_K = sqrt(GM/R^3) at
 * the cylindrical radius of the midpoint; shearing box: St / Omega). */
static double stopping_time(const oracle_problem *P, int mode, double value,
                            const double qm[3], double rho_g)
{
    if (mode == OT_CONST) return value;
    if (mode == OT_EPSTEIN) return value / rho_g;
    /* OT_STOKES */
    if (P->geom == OG_CYLINDRICAL || P->geom == OG_SPHERICAL) {
        double R = P->geom == OG_CYLINDRICAL ? qm[0] : qm[0] * sin(qm[1]);
        return value * sqrt(R * R * R / P->gm);
    }
    return value / P->omega;
}

/* ------------------------------------------------------------------------- */
/* Fixed-point deposit rule                                                    */
/* ------------------------------------------------------------------------- */

/*
 * Integer deposit of one grain's impulse D[4] (Eq. dust_feedback_final, one
 * grain's term) with the stencil weights w[d][0..2] of host zone host[].
 * Reading (the paper deposits in floating point; the integer form is this
 * project's, so that the deposited grid does not depend on the order in
 * which grains are summed): in units of the quantum, per channel c,
 *   Q      = nearest integer to D[c] / quantum,
 *   piece  = nearest integer to W_j D[c] / quantum   for every node j other
 *            than the host zone (W_j the product of the three 1-D weights),
 *   host  += Q - (sum of the pieces),
 * so the zones receive exactly Q in total.  Ties round to even (the IEEE
 * default rounding).  Nodes beyond an outflow boundary fold onto the edge
 * zone, as in the dense deposit.
 */
static void deposit_fixed_point(const oracle_problem *P, const int host[3],
                                double w[3][3], const double D[4], double quantum,
                                int64_t *fixed)
{
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    int64_t hidx = node_index(host[0], 0, n0, P->bc[0])
        + (int64_t)n0 * (node_index(host[1], 0, n1, P->bc[1])
        + (int64_t)n1 * node_index(host[2], 0, n2, P->bc[2]));
    for (int ch = 0; ch < 4; ch++) {
        int64_t rest = (int64_t)llrint(D[ch] / quantum);
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    if (a == 1 && b == 1 && c == 1) continue;
                    double W = w[0][a] * w[1][b] * w[2][c];
                    if (W == 0.0) continue;
                    int64_t idx = node_index(host[0], a - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    int64_t piece = (int64_t)llrint(W * D[ch] / quantum);
                    fixed[4 * idx + ch] += piece;
                    rest -= piece;
                }
        fixed[4 * hidx + ch] += rest;
    }
}

/* ------------------------------------------------------------------------- */
/* The step                                                                    */
/* ------------------------------------------------------------------------- */

/*
 * Advance n grains by one step of size dt starting at time t.
 *   q0..q2, p0..p2 : coordinates and momentum-like variables (updated)
 *                    Cartesian / shearing box: (x,y,z), (vx,vy,vz) (residual
 *                    velocity in the orbital-advection frame);
 *                    cylindrical: (R,phi,z), (v_R, l_phi = R v_phi, v_z);
 *                    spherical: (r,theta,phi), (v_r, l_theta = r v_theta,
 *                    l_phi = r sin(theta) v_phi)
 *   species, param : per-grain species index and stopping-time value
 *                    (either may be NULL: species 0 / the species value)
 *   active         : 1 = in the domain; set to 0 when a grain leaves through
 *                    an outflow boundary
 *   rho, pg0..pg2  : gas density and momentum-like velocity per zone,
 *                    zone index i + n0 (j + n1 k); pg updated when
 *                    feedback_apply is set
 *   dep            : out, [ncell][4] dense deposit: momentum-like channels
 *                    0..2 (Eq. dust_feedback_final times the zone volume and
 *                    dt, i.e. the impulse given to the gas) and energy (3)
 * Returns the number of grains removed in this step.
 */
static int64_t step_grains(const oracle_problem *P,
                           double *q0, double *q1, double *q2,
                           double *p0, double *p1, double *p2,
                           const uint8_t *species, const double *param,
                           uint8_t *active, int64_t n, double t, double dt,
                           const double *rho, double *pg0, double *pg1, double *pg2,
                           double *dep, int64_t *fixed, double quantum)
{
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    const int64_t ncell = (int64_t)n0 * n1 * n2;
    const double h = 0.5 * dt;
    int64_t removed = 0;
    int wk[3];
    for (int d = 0; d < 3; d++) wk[d] = weight_kind(P, d);
    memset(dep, 0, sizeof(double) * 4 * ncell);
    if (fixed) memset(fixed, 0, sizeof(int64_t) * 4 * ncell);

    for (int64_t g = 0; g < n; g++) {
        if (!active[g]) continue;
        int sp = species ? species[g] : 0;
        double m = P->sp_mass[sp];
        double q[3] = {q0[g], q1[g], q2[g]};
        double pn[3] = {p0[g], p1[g], p2[g]};

        /* 1. first half drift and boundaries at t + dt/2 */
        drift_first(P, q, pn, h);
        if (!apply_bc(P, q, pn, t + h)) { active[g] = 0; removed++; continue; }
        double qm[3] = {q[0], q[1], q[2]};

        /* 2. host zone and weights at x^{n+1/2} */
        int host[3];
        double w[3][3];
        for (int d = 0; d < 3; d++) {
            if (P->n[d] <= 1) {
                host[d] = 0; w[d][0] = 0.0; w[d][1] = 1.0; w[d][2] = 0.0;
                continue;
            }
            host[d] = oracle_locate(P->edges[d], P->n[d], qm[d]);
            direction_weights(P, d, wk[d], qm[d], host[d], w[d]);
        }

        /* 3. gather (Eq. Delta_vp) */
        double rg = 0.0, vg[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    double W = w[0][a] * w[1][b] * w[2][c];
                    int64_t idx = node_index(host[0], a - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    rg += W * rho[idx];
                    vg[0] += W * pg0[idx];
                    vg[1] += W * pg1[idx];
                    vg[2] += W * pg2[idx];
                }

        /* 4. propagators: E = e^{-dt/tau}, cg = h1/tau = 1 - E, h1 = dt phi1 */
        int mode = P->sp_tau_mode[sp];
        double value = param ? param[g] : P->sp_tau[sp];
        double tau = stopping_time(P, mode, value, qm, rg);
        double x = dt / tau;
        double E = exp(-x);
        double cg = -expm1(-x);
        double h1 = (x == 0.0) ? dt : dt * cg / x;

        /* 5. kick */
        double pp[3], a[3], dHdp[3];
        if (P->pusher == OP_SEMI_IMPLICIT) {
            /* Sec. 3.2.1: v^{n+1} = v^n + Lambda^{-1} dt a_tot(x^{n+1/2}, v^n, v_g)
             * with Lambda = I - (dt/2) d a_tot / d v (Eqs. semi-implicit,
             * a_linear, Lambda); drag -(v - v_g)/tau gives b = dt / (2 tau). */
            double it = 1.0 / tau;            /* 0 for tau = infinity */
            double b = 0.5 * dt * it;
            double at[3], l00 = 1.0 + b, l01 = 0.0, l10 = 0.0;
            if (P->geom == OG_SHEARING_BOX) {
                double Om = P->omega, qq = P->q;
                double zf = P->vertical_gravity ? -Om * Om * qm[2] : 0.0;
                if (!P->fargo) {        /* standard frame, Eq. standard_SB_g */
                    at[0] = 2.0 * Om * (pn[1] + qq * Om * qm[0]);
                    at[1] = -2.0 * Om * pn[0];
                    l01 = -Om * dt;
                    l10 = Om * dt;
                } else {                /* orbital advection, residual velocity */
                    at[0] = 2.0 * Om * pn[1];
                    at[1] = (qq - 2.0) * Om * pn[0];
                    l01 = -Om * dt;
                    l10 = (1.0 - 0.5 * qq) * Om * dt;
                }
                at[2] = zf;
            } else {
                at[0] = at[1] = at[2] = 0.0;
            }
            for (int d = 0; d < 3; d++) at[d] += (vg[d] - pn[d]) * it;
            /* solve the 2x2 (x, y) block and the diagonal z entry */
            double det = l00 * l00 - l01 * l10;
            double r0 = dt * at[0], r1 = dt * at[1];
            pp[0] = pn[0] + (l00 * r0 - l01 * r1) / det;
            pp[1] = pn[1] + (-l10 * r0 + l00 * r1) / det;
            pp[2] = pn[2] + dt * at[2] / l00;
            /* non-frictional acceleration at (x^{n+1/2}, v^{n+1/2}) */
            double vh[3] = {0.5 * (pn[0] + pp[0]), 0.5 * (pn[1] + pp[1]), 0.5 * (pn[2] + pp[2])};
            if (P->geom == OG_SHEARING_BOX) {
                double Om = P->omega, qq = P->q;
                if (!P->fargo) {
                    a[0] = 2.0 * Om * (vh[1] + qq * Om * qm[0]);
                    a[1] = -2.0 * Om * vh[0];
                } else {
                    a[0] = 2.0 * Om * vh[1];
                    a[1] = (qq - 2.0) * Om * vh[0];
                }
                a[2] = P->vertical_gravity ? -Om * Om * qm[2] : 0.0;
            } else {
                a[0] = a[1] = a[2] = 0.0;
            }
            dHdp[0] = vh[0]; dHdp[1] = vh[1]; dHdp[2] = vh[2];
        } else if (P->geom == OG_SHEARING_BOX) {
            /* App. B.1: R v^{n+1} = E v^n + h1 G(x^{n+1/2}, v^n/2, v_g) */
            double Om = P->omega, qq = P->q;
            double zf = P->vertical_gravity ? -Om * Om * qm[2] : 0.0;
            double Om1 = Om * h1;
            double r[3];
            if (!P->fargo) {
                double G0 = 2.0 * Om * (0.5 * pn[1] + qq * Om * qm[0]);
                double G1 = -2.0 * (0.5 * pn[0]) * Om;
                r[0] = E * pn[0] + h1 * G0 + cg * vg[0];
                r[1] = E * pn[1] + h1 * G1 + cg * vg[1];
                r[2] = E * pn[2] + h1 * zf + cg * vg[2];
                double inv = 1.0 / (1.0 + Om1 * Om1);
                pp[0] = inv * (r[0] + Om1 * r[1]);
                pp[1] = inv * (-Om1 * r[0] + r[1]);
                pp[2] = r[2];
            } else {
                double Om2 = Om1 * (1.0 - 0.5 * qq);
                double G0 = 2.0 * Om * (0.5 * pn[1]);
                double G1 = (0.5 * pn[0]) * Om * (qq - 2.0);
                r[0] = E * pn[0] + h1 * G0 + cg * vg[0];
                r[1] = E * pn[1] + h1 * G1 + cg * vg[1];
                r[2] = E * pn[2] + h1 * zf + cg * vg[2];
                double inv = 1.0 / (1.0 + Om1 * Om2);
                pp[0] = inv * (r[0] + Om1 * r[1]);
                pp[1] = inv * (-Om2 * r[0] + r[1]);
                pp[2] = r[2];
            }
            /* non-frictional acceleration at (x^{n+1/2}, v^{n+1/2}) */
            double vh[3] = {0.5 * (pn[0] + pp[0]), 0.5 * (pn[1] + pp[1]), 0.5 * (pn[2] + pp[2])};
            if (!P->fargo) {
                a[0] = 2.0 * Om * (vh[1] + qq * Om * qm[0]);
                a[1] = -2.0 * Om * vh[0];
            } else {
                a[0] = 2.0 * Om * vh[1];
                a[1] = (qq - 2.0) * Om * vh[0];
            }
            a[2] = zf;
            dHdp[0] = vh[0]; dHdp[1] = vh[1]; dHdp[2] = vh[2];
        } else if (P->geom == OG_CYLINDRICAL) {
            /* App. B.2.1: v_z, then l_phi, then v_R with (l^2)^{n+1/2} */
            double g[3];
            gravity(P, qm, g);
            double R = qm[0];
            pp[2] = E * pn[2] + h1 * g[2] + cg * vg[2];
            pp[1] = E * pn[1] + h1 * g[1] * R + cg * vg[1];
            double l2 = 0.5 * (pn[1] * pn[1] + pp[1] * pp[1]);
            double aR = l2 / (R * R * R) + g[0];
            pp[0] = E * pn[0] + h1 * aR + cg * vg[0];
            a[0] = aR; a[1] = g[1] * R; a[2] = g[2];
            dHdp[0] = 0.5 * (pn[0] + pp[0]);
            dHdp[1] = 0.5 * (pn[1] + pp[1]) / (R * R);
            dHdp[2] = 0.5 * (pn[2] + pp[2]);
        } else if (P->geom == OG_SPHERICAL) {
            /* App. B.2.2: l_phi, then l_theta, then v_r; the second averaged
             * square is (l_theta^2)^{n+1/2} (the printed formula repeats
             * l_phi, a typo). */
            double g[3];
            gravity(P, qm, g);
            double r = qm[0], st = sin(qm[1]), ct = cos(qm[1]);
            pp[2] = E * pn[2] + h1 * g[2] * r * st + cg * vg[2];
            double lp2 = 0.5 * (pn[2] * pn[2] + pp[2] * pp[2]);
            double ath = lp2 * ct / (r * r * st * st * st) + r * g[1];
            pp[1] = E * pn[1] + h1 * ath + cg * vg[1];
            double lt2 = 0.5 * (pn[1] * pn[1] + pp[1] * pp[1]);
            double ar = lt2 / (r * r * r) + lp2 / (r * r * r * st * st) + g[0];
            pp[0] = E * pn[0] + h1 * ar + cg * vg[0];
            a[0] = ar; a[1] = ath; a[2] = g[2] * r * st;
            dHdp[0] = 0.5 * (pn[0] + pp[0]);
            dHdp[1] = 0.5 * (pn[1] + pp[1]) / (r * r);
            dHdp[2] = 0.5 * (pn[2] + pp[2]) / (r * r * st * st);
        } else {
            /* Eq. kick_modified: v^{n+1} = E v^n + h1 v_g / tau */
            for (int d = 0; d < 3; d++) {
                pp[d] = E * pn[d] + cg * vg[d];
                a[d] = 0.0;
                dHdp[d] = 0.5 * (pn[d] + pp[d]);
            }
        }

        /* 6. second half drift with the midpoint metric, 7. boundaries */
        double qn[3] = {qm[0], qm[1], qm[2]};
        drift_second(P, qn, qm, pp, h);
        double pnew[3] = {pp[0], pp[1], pp[2]};
        int alive = apply_bc(P, qn, pnew, t + dt);

        /* 8. deposit at x^{n+1/2}: -m W (dp - dt a), energy = sum dP dH/dp */
        double D[4];
        D[3] = 0.0;
        for (int c = 0; c < 3; c++) {
            D[c] = -m * ((pp[c] - pn[c]) - dt * a[c]);
            D[3] += D[c] * dHdp[c];
        }
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int aa = 0; aa < 3; aa++) {
                    double W = w[0][aa] * w[1][b] * w[2][c];
                    if (W == 0.0) continue;
                    int64_t idx = node_index(host[0], aa - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    for (int ch = 0; ch < 4; ch++) dep[4 * idx + ch] += W * D[ch];
                }
        if (fixed) deposit_fixed_point(P, host, w, D, quantum, fixed);

        q0[g] = qn[0]; q1[g] = qn[1]; q2[g] = qn[2];
        p0[g] = pnew[0]; p1[g] = pnew[1]; p2[g] = pnew[2];
        if (!alive) { active[g] = 0; removed++; }
    }

    /* feedback on the gas momentum: rho v_i += dP_i / dV_i */
    if (P->feedback_apply) {
        for (int k = 0; k < n2; k++)
            for (int j = 0; j < n1; j++)
                for (int i = 0; i < n0; i++) {
                    int64_t idx = i + (int64_t)n0 * (j + (int64_t)n1 * k);
                    double a0 = P->edges[0][i], a1 = P->edges[0][i + 1];
                    double b0 = P->edges[1][j], b1 = P->edges[1][j + 1];
                    double c0 = P->edges[2][k], c1 = P->edges[2][k + 1];
                    double dV;
                    if (P->geom == OG_CYLINDRICAL)
                        dV = 0.5 * (a1 * a1 - a0 * a0) * (b1 - b0) * (c1 - c0);
                    else if (P->geom == OG_SPHERICAL)
                        dV = (a1 * a1 * a1 - a0 * a0 * a0) / 3.0 * (cos(b0) - cos(b1)) * (c1 - c0);
                    else
                        dV = (a1 - a0) * (b1 - b0) * (c1 - c0);
                    double s = 1.0 / (rho[idx] * dV);
                    pg0[idx] += dep[4 * idx + 0] * s;
                    pg1[idx] += dep[4 * idx + 1] * s;
                    pg2[idx] += dep[4 * idx + 2] * s;
                }
    }
    return removed;
}

/* One step with the deposit accumulated densely in double precision only. */
int64_t oracle_step(const oracle_problem *P,
                    double *q0, double *q1, double *q2,
                    double *p0, double *p1, double *p2,
                    const uint8_t *species, const double *param,
                    uint8_t *active, int64_t n, double t, double dt,
                    const double *rho, double *pg0, double *pg1, double *pg2,
                    double *dep)
{
    return step_grains(P, q0, q1, q2, p0, p1, p2, species, param, active, n, t, dt,
                       rho, pg0, pg1, pg2, dep, NULL, 0.0);
}

/* The same step, with the deposit also given in fixed point: fixed[ncell][4]
 * receives the integers of the per-grain rule (deposit_fixed_point) in units
 * of quantum.  The dense deposit dep and the feedback are as in
 * oracle_step (the feedback uses the dense deposit). */
int64_t oracle_step_fixed(const oracle_problem *P,
                          double *q0, double *q1, double *q2,
                          double *p0, double *p1, double *p2,
                          const uint8_t *species, const double *param,
                          uint8_t *active, int64_t n, double t, double dt,
                          const double *rho, double *pg0, double *pg1, double *pg2,
                          double *dep, int64_t *fixed, double quantum)
{
    return step_grains(P, q0, q1, q2, p0, p1, p2, species, param, active, n, t, dt,
                       rho, pg0, pg1, pg2, dep, fixed, quantum);
}

/* Volume of zone (i, j, k): dR dphi dz R-weighted in cylindrical, r^2 dr
 * sin(theta) dtheta dphi in spherical coordinates (Sec. 3.4). */
static double zone_volume(const oracle_problem *P, int i, int j, int k)
{
    double a0 = P->edges[0][i], a1 = P->edges[0][i + 1];
    double b0 = P->edges[1][j], b1 = P->edges[1][j + 1];
    double c0 = P->edges[2][k], c1 = P->edges[2][k + 1];
    if (P->geom == OG_CYLINDRICAL) return 0.5 * (a1 * a1 - a0 * a0) * (b1 - b0) * (c1 - c0);
    if (P->geom == OG_SPHERICAL)
        return (a1 * a1 * a1 - a0 * a0 * a0) / 3.0 * (cos(b0) - cos(b1)) * (c1 - c0);
    return (a1 - a0) * (b1 - b0) * (c1 - c0);
}

/*
 * Gas half-step predictor of the drag coupling (Sec. 3.1, Eqs. Delta_vp and
 * f_D, with tau_s replaced by max(tau_s, dt) against the predictor's
 * stiffness, as the paper adopts from BS10).  Every active grain gathers the
 * gas at its position x^n (weights of Sec. 3.4 at x^n, stopping time from the
 * gas gathered there) and the drag force density
 *     f_D,i = (1/dV_i) sum_p (m_p / tau') W(x^n_p - x_i) (v_p - v_g(x^n_p))
 * advances the gas by half a step:  (rho v)_i^{n+1/2} = (rho v)_i^n + dt/2 f_D,i.
 * imp [ncell][3] receives the impulse dt/2 sum_p (...) per zone (FP64, dense),
 * ph0..ph2 the half-step momentum-like gas velocity pg + imp / (rho dV).
 * Reading: the predictor acts on the momentum-like channels of the deposit
 * (l_phi = R v_phi etc.), like the corrector.
 */
void oracle_gas_predictor(const oracle_problem *P,
                          const double *q0, const double *q1, const double *q2,
                          const double *p0, const double *p1, const double *p2,
                          const uint8_t *species, const double *param,
                          const uint8_t *active, int64_t n, double dt,
                          const double *rho, const double *pg0, const double *pg1,
                          const double *pg2, double *imp,
                          double *ph0, double *ph1, double *ph2)
{
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    const int64_t ncell = (int64_t)n0 * n1 * n2;
    int wk[3];
    for (int d = 0; d < 3; d++) wk[d] = weight_kind(P, d);
    memset(imp, 0, sizeof(double) * 3 * ncell);
    for (int64_t g = 0; g < n; g++) {
        if (!active[g]) continue;
        int sp = species ? species[g] : 0;
        double q[3] = {q0[g], q1[g], q2[g]};
        double pn[3] = {p0[g], p1[g], p2[g]};
        int host[3];
        double w[3][3];
        for (int d = 0; d < 3; d++) {
            if (P->n[d] <= 1) {
                host[d] = 0; w[d][0] = 0.0; w[d][1] = 1.0; w[d][2] = 0.0;
                continue;
            }
            host[d] = oracle_locate(P->edges[d], P->n[d], q[d]);
            direction_weights(P, d, wk[d], q[d], host[d], w[d]);
        }
        double rg = 0.0, vg[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    double W = w[0][a] * w[1][b] * w[2][c];
                    int64_t idx = node_index(host[0], a - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    rg += W * rho[idx];
                    vg[0] += W * pg0[idx];
                    vg[1] += W * pg1[idx];
                    vg[2] += W * pg2[idx];
                }
        double value = param ? param[g] : P->sp_tau[sp];
        double tau = stopping_time(P, P->sp_tau_mode[sp], value, q, rg);
        double taup = fmax(tau, fabs(dt));
        double coef = 0.5 * dt * P->sp_mass[sp] / taup;   /* 0 for tau = infinity */
        double J[3];
        for (int c = 0; c < 3; c++) J[c] = coef * (pn[c] - vg[c]);
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    double W = w[0][a] * w[1][b] * w[2][c];
                    if (W == 0.0) continue;
                    int64_t idx = node_index(host[0], a - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    for (int ch = 0; ch < 3; ch++) imp[3 * idx + ch] += W * J[ch];
                }
    }
    for (int k = 0; k < n2; k++)
        for (int j = 0; j < n1; j++)
            for (int i = 0; i < n0; i++) {
                int64_t idx = i + (int64_t)n0 * (j + (int64_t)n1 * k);
                double s = 1.0 / (rho[idx] * zone_volume(P, i, j, k));
                ph0[idx] = pg0[idx] + imp[3 * idx + 0] * s;
                ph1[idx] = pg1[idx] + imp[3 * idx + 1] * s;
                ph2[idx] = pg2[idx] + imp[3 * idx + 2] * s;
            }
}

/* Dust mass per zone (Sec. 3.4, Eq. deposition with q_p = m_p): every active
 * grain adds m_p W to the zones of its stencil at its position, with the
 * weights of the problem's weighting (CIC, TSC or volume weighting); nodes
 * beyond an outflow boundary fold onto the edge zone, as the deposit does.
 * mass[ncell] is overwritten; dividing by the zone volume gives rho_d. */
void oracle_deposit_mass(const oracle_problem *P,
                         const double *q0, const double *q1, const double *q2,
                         const uint8_t *species, const uint8_t *active, int64_t n,
                         double *mass)
{
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    int wk[3];
    for (int d = 0; d < 3; d++) wk[d] = weight_kind(P, d);
    memset(mass, 0, sizeof(double) * (size_t)n0 * n1 * n2);
    for (int64_t g = 0; g < n; g++) {
        if (!active[g]) continue;
        double m = P->sp_mass[species ? species[g] : 0];
        double q[3] = {q0[g], q1[g], q2[g]};
        int host[3];
        double w[3][3];
        for (int d = 0; d < 3; d++) {
            if (P->n[d] <= 1) {
                host[d] = 0; w[d][0] = 0.0; w[d][1] = 1.0; w[d][2] = 0.0;
                continue;
            }
            host[d] = oracle_locate(P->edges[d], P->n[d], q[d]);
            direction_weights(P, d, wk[d], q[d], host[d], w[d]);
        }
        for (int c = 0; c < 3; c++)
            for (int b = 0; b < 3; b++)
                for (int a = 0; a < 3; a++) {
                    int64_t idx = node_index(host[0], a - 1, n0, P->bc[0])
                        + (int64_t)n0 * (node_index(host[1], b - 1, n1, P->bc[1])
                        + (int64_t)n1 * node_index(host[2], c - 1, n2, P->bc[2]));
                    mass[idx] += m * (w[0][a] * w[1][b] * w[2][c]);
                }
    }
}

/* Gas momentum-like velocity per zone from physical velocity components
 * (Sec. 2.2: l_phi = R v_phi; spherical l_theta = r v_theta, l_phi = r
 * sin(theta) v_phi), evaluated at the zone centres (reading: the gathered
 * angular quantity is the zone's own angular momentum per unit mass). */
void oracle_gas_momentum(const oracle_problem *P, const double *v0, const double *v1,
                         const double *v2, double *pg0, double *pg1, double *pg2)
{
    const int n0 = P->n[0], n1 = P->n[1], n2 = P->n[2];
    for (int k = 0; k < n2; k++)
        for (int j = 0; j < n1; j++)
            for (int i = 0; i < n0; i++) {
                int64_t idx = i + (int64_t)n0 * (j + (int64_t)n1 * k);
                double xc = 0.5 * (P->edges[0][i] + P->edges[0][i + 1]);
                double yc = 0.5 * (P->edges[1][j] + P->edges[1][j + 1]);
                pg0[idx] = v0[idx];
                pg1[idx] = v1[idx];
                pg2[idx] = v2[idx];
                if (P->geom == OG_CYLINDRICAL) pg1[idx] = xc * v1[idx];
                if (P->geom == OG_SPHERICAL) {
                    pg1[idx] = xc * v1[idx];
                    pg2[idx] = xc * sin(yc) * v2[idx];
                }
            }
}
