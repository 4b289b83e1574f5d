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
