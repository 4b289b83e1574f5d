"""Pins of the oracle's weighting factors (Sec. 3.4, App. C) against what the
paper and the mathematics fix, independently of the oracle's own formulas:

* quadrature of the defining integral W_i = int_zone S dV (Eq. weight) with
  the B-spline shapes b0 / b1 (Eqs. b0, b1) and the measure of each geometry
  (Eq. shape_curv: R dR, r^2 dr, sin(theta) dtheta);
* sum of the weights equal to one (Eq. shape_norm);
* the zero-curvature limit nu -> infinity gives the Cartesian weights;
* Cartesian CIC/TSC reproduce a linear field exactly;
* the printed (ungarbled) W_i of Eq. CIC_spherical_theta.
"""
import numpy as np
import pytest
from scipy.integrate import quad

import oracle as O

KINDS = list(range(8))
TSC_KINDS = (O.W1_CART_TSC, O.W1_CYL_R_TSC, O.W1_SPH_R_TSC, O.W1_SPH_TH_TSC)
MEASURE = {
    O.W1_CART_CIC: lambda r: 1.0, O.W1_CART_TSC: lambda r: 1.0,
    O.W1_CYL_R_CIC: lambda r: r, O.W1_CYL_R_TSC: lambda r: r,
    O.W1_SPH_R_CIC: lambda r: r * r, O.W1_SPH_R_TSC: lambda r: r * r,
    O.W1_SPH_TH_CIC: np.sin, O.W1_SPH_TH_TSC: np.sin,
}


def quad_weights(kind, x, lo, hi):
    """Brute-force Eq. weight: shape of the host zone's width centred on x,
    integrated with the geometry's measure over (-inf, lo], [lo, hi], [hi, inf)."""
    h = hi - lo
    tsc = kind in TSC_KINDS
    half = h if tsc else 0.5 * h
    b = (lambda u: max(0.0, 1.0 - abs(u) / h)) if tsc else (lambda u: 1.0)
    f = lambda s: b(s - x) * MEASURE[kind](s)  # noqa: E731
    a0, a1 = x - half, x + half
    vals = []
    for s0, s1 in ((a0, lo), (lo, hi), (hi, a1)):
        s0, s1 = max(s0, a0), min(s1, a1)
        if s1 <= s0:
            vals.append(0.0)
            continue
        pts = [x] if s0 < x < s1 else None
        vals.append(quad(f, s0, s1, epsabs=0.0, epsrel=1e-13, limit=200, points=pts)[0])
    vals = np.array(vals)
    return vals / vals.sum()


ZONES = {
    # uniform-ish radial zones, a small log-grid zone near the inner edge,
    # theta zones off and near the midplane
    "radial": [(0.7, 0.8), (0.4, 0.4055), (2.48, 2.5)],
    "theta": [(1.2, 1.25), (1.5, 1.5047), (np.pi / 2 - 0.3, np.pi / 2 - 0.3 + 0.6 / 128)],
}


@pytest.mark.parametrize("kind", KINDS)
def test_weights_match_quadrature_of_defining_integral(kind):
    rng = np.random.default_rng(100 + kind)
    zones = ZONES["theta"] if kind >= O.W1_SPH_TH_CIC else ZONES["radial"]
    for lo, hi in zones:
        xs = np.concatenate([rng.uniform(lo, hi, 12), [lo, 0.5 * (lo + hi)]])
        for x in xs:
            w = O.weights_1d(kind, x, lo, hi)
            assert np.allclose(w, quad_weights(kind, x, lo, hi), rtol=0, atol=1e-12), (kind, x)


@pytest.mark.parametrize("kind", KINDS)
def test_weights_sum_to_one_and_nonnegative(kind):
    rng = np.random.default_rng(7 + kind)
    for lo, hi in ([(0.4, 0.41), (1.0, 1.3), (0.05, 0.06)] if kind < 6
                   else [(0.3, 0.31), (1.5, 1.6), (2.9, 2.95)]):
        for x in rng.uniform(lo, hi, 200):
            w = O.weights_1d(kind, x, lo, hi)
            assert abs(w.sum() - 1.0) < 4e-16 * 4
            assert (w >= -1e-15).all()


@pytest.mark.parametrize("cyl,cart", [(O.W1_CYL_R_CIC, O.W1_CART_CIC),
                                      (O.W1_CYL_R_TSC, O.W1_CART_TSC),
                                      (O.W1_SPH_R_CIC, O.W1_CART_CIC),
                                      (O.W1_SPH_R_TSC, O.W1_CART_TSC)])
def test_zero_curvature_limit_gives_cartesian(cyl, cart):
    # nu = R_i / dR -> infinity (Sec. 3.4.1): far from the axis the curvilinear
    # weights tend to the Cartesian ones, with an O(1/nu) difference
    for x in np.linspace(1e6 + 0.01, 1e6 + 0.99, 9):
        w = O.weights_1d(cyl, x, 1e6, 1e6 + 1.0)
        wc = O.weights_1d(cart, x, 1e6, 1e6 + 1.0)
        assert np.abs(w - wc).max() < 3e-6


@pytest.mark.parametrize("kind", [O.W1_CART_CIC, O.W1_CART_TSC])
def test_cartesian_weights_reproduce_linear_field(kind):
    # b0 and b1 shapes are symmetric: sum_i W_i x_i = x_p on a uniform grid
    lo, hi = 2.0, 2.25
    centres = np.array([lo - 0.125, lo + 0.125, hi + 0.125])
    for x in np.linspace(lo, hi, 17)[:-1]:
        w = O.weights_1d(kind, x, lo, hi)
        assert abs((w * centres).sum() - x) < 1e-14


def test_theta_cic_host_weight_matches_printed_formula():
    # Eq. CIC_spherical_theta, W_i (not garbled): with x_{i-1/2}=lo, x_{i+1/2}=hi
    lo, hi = 1.1, 1.2
    tc = 0.5 * (lo + hi)
    for d in np.linspace(-0.049, 0.049, 11):
        if d == 0:
            continue
        D = np.cos(lo + d) - np.cos(hi + d)
        if d > 0:
            wi = (np.cos(lo + d) - np.cos(hi)) / D
        else:
            wi = (np.cos(lo) - np.cos(hi + d)) / D
        w = O.weights_1d(O.W1_SPH_TH_CIC, tc + d, lo, hi)
        assert abs(w[1] - wi) < 1e-14


def test_theta_tsc_flat_measure_limit():
    # derived theta-TSC: across a tiny zone at the equator sin(theta) is nearly
    # constant and the weights tend to the Cartesian TSC ones
    lo = np.pi / 2 - 5e-5
    hi = np.pi / 2 + 5e-5
    for x in np.linspace(lo, hi, 9)[:-1]:
        w = O.weights_1d(O.W1_SPH_TH_TSC, x, lo, hi)
        wc = O.weights_1d(O.W1_CART_TSC, x, lo, hi)
        assert np.abs(w - wc).max() < 1e-8


def test_radial_weights_at_zone_centre_printed_values():
    # delta = 0 in Eqs. CIC/TSC_cylindrical: W_i = 1 (CIC), W_i = 3/4 and
    # W_{i+-1} = (3 nu +- 2)/(3 nu) / 8 (TSC)
    nu = 7.5
    w = O.weights_1d(O.W1_CYL_R_CIC, nu, nu - 0.5, nu + 0.5)
    assert np.allclose(w, [0.0, 1.0, 0.0], atol=1e-15)
    w = O.weights_1d(O.W1_CYL_R_TSC, nu, nu - 0.5, nu + 0.5)
    assert np.allclose(w, [(3 * nu - 2) / (3 * nu) / 8, 0.75, (3 * nu + 2) / (3 * nu) / 8],
                       atol=1e-15)


def test_locate_half_open_zones():
    e = np.array([0.0, 0.25, 0.5, 0.75, 1.0])
    assert O.locate(e, 0.0) == 0
    assert O.locate(e, 0.25) == 1
    assert O.locate(e, np.nextafter(0.25, 0)) == 0
    assert O.locate(e, np.nextafter(1.0, 0)) == 3


# --------------------------------------------------------------------------
# Traditional volume weighting (Eq. CIC_vol): linear interpolation in the
# volume coordinate V between the centres of the two zones around the grain.
# The pins below use only what that statement fixes: V is R^2, r^3 or
# -cos(theta), so interpolating V itself must return V(x) exactly, the two
# weights sum to one and lie in [0, 1], the weight a zone receives is
# continuous as the grain crosses zone edges (the nodes are the zone
# centres), and the printed cylindrical case at a point.

VOL_V = {
    O.W1_CYL_R_VOL: lambda x: x * x,
    O.W1_SPH_R_VOL: lambda x: x ** 3,
    O.W1_SPH_TH_VOL: lambda x: -np.cos(x),
}


def _vol_grids():
    log = np.geomspace(0.4, 2.5, 25)
    return {
        O.W1_CYL_R_VOL: [np.linspace(0.7, 1.5, 9), log, np.linspace(0.0, 1.0, 11)],
        O.W1_SPH_R_VOL: [np.linspace(0.7, 1.5, 9), log, np.linspace(0.0, 1.0, 11)],
        O.W1_SPH_TH_VOL: [np.linspace(np.pi / 2 - 0.3, np.pi / 2 + 0.3, 17),
                          np.linspace(0.0, np.pi, 13),
                          np.pi / 2 + np.array([-0.4, -0.25, -0.05, 0.02, 0.2, 0.45])],
    }


def _centres(e):
    c = 0.5 * (e[1:] + e[:-1])
    return np.concatenate([[c[0] - (e[1] - e[0])], c, [c[-1] + (e[-1] - e[-2])]])


def test_volume_weights_printed_cylindrical_case():
    """Eq. CIC_vol at R_i = 1, R_{i+1} = 1.1, R_p = 1.05 (zone centres of a
    uniform grid of width 0.1): W_i = (1.21 - 1.1025) / (1.21 - 1) by hand."""
    edges = np.array([0.95, 1.05, 1.15, 1.25])
    w = O.weights_vol(O.W1_CYL_R_VOL, 1.05, edges, 1)
    assert abs(w[0] - 0.1075 / 0.21) < 1e-14 and abs(w[1] - 0.1025 / 0.21) < 1e-14
    assert w[2] == 0.0


@pytest.mark.parametrize("kind", [O.W1_CYL_R_VOL, O.W1_SPH_R_VOL, O.W1_SPH_TH_VOL])
def test_volume_weights_interpolate_the_volume_coordinate_exactly(kind):
    rng = np.random.default_rng(7 + kind)
    V = VOL_V[kind]
    for e in _vol_grids()[kind]:
        n = len(e) - 1
        c = _centres(e)
        for _ in range(200):
            i = int(rng.integers(0, n))
            x = rng.uniform(e[i], e[i + 1])
            w = O.weights_vol(kind, x, e, i)
            assert abs(w.sum() - 1.0) < 1e-14
            assert np.all(w >= -1e-15) and np.all(w <= 1.0 + 1e-15)
            assert w[0] == 0.0 or w[2] == 0.0    # two nodes only
            # V interpolated exactly where no node lies across the axis
            # (cylindrical) or a pole (polar angle); r^3 is the shell volume
            # on both sides of the origin
            if kind == O.W1_SPH_R_VOL:
                inside = True
            elif kind == O.W1_CYL_R_VOL:
                inside = c[i] >= 0.0
            else:
                inside = c[i] >= 0.0 and c[i + 2] <= np.pi
            if inside:
                got = w[0] * V(c[i]) + w[1] * V(c[i + 1]) + w[2] * V(c[i + 2])
                scale = abs(V(c[i + 2]) - V(c[i]))
                assert abs(got - V(x)) <= 1e-12 * scale, (kind, e[0], x)


@pytest.mark.parametrize("kind", [O.W1_CYL_R_VOL, O.W1_SPH_R_VOL, O.W1_SPH_TH_VOL])
def test_volume_weights_continuous_across_zone_edges(kind):
    for e in _vol_grids()[kind]:
        n = len(e) - 1
        for k in range(1, n):
            h = 1e-9 * (e[k + 1] - e[k - 1])
            below = O.weights_vol(kind, e[k] - h, e, k - 1)   # zones k-2, k-1, k
            above = O.weights_vol(kind, e[k] + h, e, k)       # zones k-1, k, k+1
            assert abs(below[1] - above[0]) < 1e-7 and abs(below[2] - above[1]) < 1e-7
            assert below[0] == 0.0 and above[2] == 0.0


def test_volume_weights_at_axis_and_pole_stay_in_unit_interval():
    """Next to the axis (R grid from 0) and the poles (theta from 0 to pi)
    the ghost centre lies across them; the shell volume keeps the weights in
    [0, 1] and equal to the ratio of the shell volumes between the nodes."""
    e = np.linspace(0.0, 1.0, 11)          # centre 0.05, ghost centre -0.05
    for x in (0.0, 0.01, 0.049):
        w = O.weights_vol(O.W1_CYL_R_VOL, x, e, 0)
        # shell from x to 0.05 over the shell from -0.05 to 0.05, |dV| = 2|R| dR
        assert abs(w[0] - (0.05 ** 2 - x * x) / (2 * 0.05 ** 2)) < 1e-14
    et = np.linspace(0.0, np.pi, 13)       # centre pi/24, ghost centre -pi/24
    h = np.pi / 24
    for x in (0.0, 0.05, h * 0.999):
        w = O.weights_vol(O.W1_SPH_TH_VOL, x, et, 0)
        assert abs(w[0] - (np.cos(x) - np.cos(h)) / (2 * (1 - np.cos(h)))) < 1e-13
        w = O.weights_vol(O.W1_SPH_TH_VOL, np.pi - x, et, 11)
        assert abs(w[2] - (np.cos(x) - np.cos(h)) / (2 * (1 - np.cos(h)))) < 1e-13


def test_volume_weights_tend_to_cic_far_from_the_axis():
    """Zero curvature: R^2 and r^3 are nearly linear over a zone far from the
    origin, so the weights approach the Cartesian CIC ones."""
    e = 1e6 + np.linspace(0.0, 1.0, 5)
    for kind in (O.W1_CYL_R_VOL, O.W1_SPH_R_VOL):
        for x in (1e6 + 0.3, 1e6 + 0.6):
            i = O.locate(e, x)
            w = O.weights_vol(kind, x, e, i)
            cic = O.weights_1d(O.W1_CART_CIC, x, e[i], e[i + 1])
            assert np.allclose(w, cic, atol=1e-5)


# --------------------------------------------------------------------------
# Mass deposit (Eq. deposition with q_p = m_p): dust mass per zone.

def _mass_problem(geom, weight, bc=(O.OB_PERIODIC,) * 3, n=(8, 6, 5)):
    if geom == O.OG_CARTESIAN:
        edges = [np.linspace(0.0, 1.0, n[0] + 1), np.linspace(0.0, 1.0, n[1] + 1),
                 np.linspace(0.0, 1.0, n[2] + 1)]
    elif geom == O.OG_CYLINDRICAL:
        edges = [np.geomspace(0.4, 2.0, n[0] + 1), np.linspace(0.0, 2 * np.pi, n[1] + 1),
                 np.linspace(-0.2, 0.2, n[2] + 1)]
    else:
        edges = [np.geomspace(0.5, 2.0, n[0] + 1), np.linspace(0.3, np.pi - 0.3, n[1] + 1),
                 np.linspace(0.0, 2 * np.pi, n[2] + 1)]
    return O.Problem(geom=geom, edges=edges, bc=bc, weight=weight,
                     species_mass=(0.25, 1.5), species_tau_mode=(O.OT_CONST, O.OT_CONST),
                     species_tau=(1.0, 1.0))


@pytest.mark.parametrize("geom", [O.OG_CARTESIAN, O.OG_CYLINDRICAL, O.OG_SPHERICAL])
@pytest.mark.parametrize("weight", [O.OW_CIC, O.OW_TSC, O.OW_VOLUME])
def test_mass_deposit_conserves_mass_with_outflow_folding(geom, weight):
    bc = (O.OB_OUTFLOW, O.OB_OUTFLOW if geom == O.OG_SPHERICAL else O.OB_PERIODIC, O.OB_PERIODIC)
    prob = _mass_problem(geom, weight, bc)
    rng = np.random.default_rng(21)
    n = 400
    q = [rng.uniform(e[0], e[-1], n) for e in prob.edges]
    q[0][:20] = prob.edges[0][0] + 1e-9          # grains at the outflow edges
    q[0][20:40] = prob.edges[0][-1] - 1e-9
    sp = (np.arange(n) % 2).astype(np.uint8)
    active = np.ones(n, np.uint8)
    active[::7] = 0
    m = O.deposit_mass(prob, q, active, sp)
    expect = np.where(sp == 0, 0.25, 1.5)[active.astype(bool)].sum()
    assert abs(m.sum() - expect) < 1e-12 * expect
    assert np.all(m >= -1e-15)


@pytest.mark.parametrize("weight", [O.OW_CIC, O.OW_TSC])
def test_mass_deposit_of_a_uniform_lattice_is_uniform(weight):
    """One grain per zone at the same offset in a periodic Cartesian box: by
    translation invariance and the partition of unity every zone receives
    exactly one grain mass, whatever the offset."""
    prob = _mass_problem(O.OG_CARTESIAN, weight)
    e = prob.edges
    n = prob.n
    for off in (0.0, 0.17, 0.5, 0.83):
        i, j, k = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
        q = [(idx.ravel() + off) / n[d] for d, idx in enumerate((i, j, k))]
        m = O.deposit_mass(prob, q, species=np.zeros(len(q[0]), np.uint8))
        assert np.allclose(m, 0.25, rtol=0, atol=1e-14), off


def test_mass_deposit_at_zone_centres_stays_in_the_zone():
    """CIC at a zone centre (delta = 0): the whole mass goes to that zone, in
    every geometry (Eq. CIC_cylindrical and its spherical analogue give
    W_i = 1 at delta = 0; the polar-angle CIC too)."""
    for geom in (O.OG_CARTESIAN, O.OG_CYLINDRICAL, O.OG_SPHERICAL):
        prob = _mass_problem(geom, O.OW_CIC)
        c = [0.5 * (e[1:] + e[:-1]) for e in prob.edges]
        q = [np.array([c[0][3]]), np.array([c[1][2]]), np.array([c[2][1]])]
        m = O.deposit_mass(prob, q, species=np.ones(1, np.uint8))
        idx = 3 + prob.n[0] * (2 + prob.n[1] * 1)
        assert abs(m[idx] - 1.5) < 1e-13 and abs(m.sum() - 1.5) < 1e-13


def _rigid_disk_density_error(weight, ratio, NR=800):
    """Sec. 4.7 particle assignment: uniform dust density on R in [0, 6]
    (NR zones) from Np = ratio NR grains at R(xi) = sqrt(xi (Re^2 - Rb^2) +
    Rb^2), xi equally spaced in (0, 1) (Eq. Rxi_constant); L1 error of
    rho_d (Eq. rigid_err) over the active zones 1 <= R <= 5, relative to the
    exact density."""
    Re = 6.0
    e = [np.linspace(0.0, Re, NR + 1), np.array([0.0, 2 * np.pi]), np.array([-0.5, 0.5])]
    npart = ratio * NR
    eps = 0.2
    m = eps * 0.5 * Re * Re * 2 * np.pi / npart    # total dust mass eps * volume
    prob = O.Problem(geom=O.OG_CYLINDRICAL, edges=e, bc=(O.OB_OUTFLOW, 0, 0), weight=weight,
                     species_mass=(m,))
    xi = (np.arange(npart) + 0.5) / npart
    R = np.sqrt(xi * Re * Re)
    mass = O.deposit_mass(prob, [R, np.zeros(npart), np.zeros(npart)])
    dV = 0.5 * np.diff(e[0] ** 2) * 2 * np.pi
    rho = mass / dV
    c = 0.5 * (e[0][1:] + e[0][:-1])
    act = (c >= 1.0) & (c <= 5.0)
    return np.sum(np.abs(rho[act] - eps) * dV[act]) / np.sum(dV[act]) / eps


def test_rigid_disk_deposit_noise_ordering():
    """Sec. 4.7: the 2-zone schemes (volume weighting, CIC) give the larger
    density errors and TSC smaller ones that fall faster with the number of
    grains.  Here, at Np/NR = 4: volume and CIC 5.0e-3, TSC 5.3e-4; from
    Np/NR = 4 to 16 the error falls 17 times with CIC and 73 times with
    TSC."""
    err = {w: [_rigid_disk_density_error(w, r) for r in (4, 16)]
           for w in (O.OW_VOLUME, O.OW_CIC, O.OW_TSC)}
    assert err[O.OW_VOLUME][0] > 5 * err[O.OW_TSC][0]
    assert err[O.OW_CIC][0] > 5 * err[O.OW_TSC][0]
    assert err[O.OW_TSC][0] / err[O.OW_TSC][1] > 40
    assert err[O.OW_CIC][0] / err[O.OW_CIC][1] < 25
