"""The seeded workload generators follow the recipes of the benchmark
configurations: grids, grain counts, species, dust-to-gas ratios and the
distributions the disks draw from.  CPU only."""
import numpy as np
import pytest

from paper_1908_10793_gb300 import inputs as I


def _zone_volumes(w):
    e = w.edges
    if w.geom == I.CYLINDRICAL:
        a = 0.5 * np.diff(e[0] ** 2)
    elif w.geom == I.SPHERICAL:
        a = np.diff(e[0] ** 3) / 3.0
    else:
        a = np.diff(e[0])
    b = -np.diff(np.cos(e[1])) if w.geom == I.SPHERICAL else np.diff(e[1])
    c = np.diff(e[2])
    return (c[:, None, None] * b[None, :, None] * a[None, None, :]).ravel()


def _dust_to_gas(w):
    m = np.asarray(w.species_mass)
    dust = m[w.species].sum() if w.species is not None else m[0] * w.ngrains
    return dust / (w.rho * _zone_volumes(w)).sum()


def test_box2d_is_the_small_cartesian_configuration():
    w = I.box2d("full")
    assert w.geom == I.CARTESIAN and w.n == [64, 64, 1] and w.ngrains == 16384
    assert w.weight == I.TSC and w.feedback == 1 and w.steps == 100
    assert w.dt == 0.01 and w.species_tau == [0.1] and w.species_tau_mode == [I.TAU_CONST]
    assert np.all(w.rho == 1.0)
    assert np.all(w.vgas[0] == 0.3) and np.all(w.vgas[1] == -0.2)
    # grain velocities Gaussian with sigma 1, positions uniform in the box
    for d in range(2):
        assert abs(w.v[d].std() - 1.0) < 0.03 and abs(w.v[d].mean()) < 0.03
        assert w.q[d].min() >= 0.0 and w.q[d].max() < 1.0


def test_sbox3d_is_the_shearing_box_configuration():
    w = I.sbox3d("full")
    assert w.geom == I.SHEARING_BOX and w.n == [128, 128, 128]
    assert w.ngrains == 16_777_216 and w.fargo == 1
    assert w.species_tau_mode == [I.TAU_STOKES] and w.species_tau == [0.1]
    assert w.weight == I.TSC and w.steps == 200 and w.feedback == 1
    assert _dust_to_gas(w) == pytest.approx(0.02, rel=1e-12)
    # eight grains in every zone
    cells = [np.clip(np.searchsorted(w.edges[d], w.q[d], side="right") - 1, 0, 127)
             for d in range(3)]
    counts = np.bincount(cells[0] + 128 * (cells[1] + 128 * cells[2]), minlength=128 ** 3)
    assert counts.min() == 8 and counts.max() == 8
    # residual gas velocity: Gaussian perturbations of amplitude 1e-3
    for d in range(3):
        assert abs(w.vgas[d].std() - 1e-3) < 2e-5


def test_cylindrical_disk_recipe():
    w = I.cyldisk("small")
    e = w.edges
    assert w.geom == I.CYLINDRICAL and e[0][0] == pytest.approx(0.4) and e[0][-1] == pytest.approx(2.5)
    ratio = e[0][1:] / e[0][:-1]
    assert np.allclose(ratio, ratio[0])                      # log-spaced in R
    assert sorted(w.species_tau) == [0.01, 0.1, 1.0, 10.0]
    assert np.bincount(w.species, minlength=4).tolist() == [w.ngrains // 4] * 4
    assert _dust_to_gas(w) == pytest.approx(0.01, rel=1e-12)
    # Sigma ~ 1/R: the grains are uniform in R, the gas density is 1/R
    hist, _ = np.histogram(w.q[0], bins=8, range=(0.4, 2.5))
    assert hist.min() > 0.9 * hist.mean() and hist.max() < 1.1 * hist.mean()
    Rc = np.tile(0.5 * (e[0][1:] + e[0][:-1]), w.n[1] * w.n[2])
    assert np.allclose(w.rho * Rc, 1.0)
    # Keplerian gas with 1e-3 noise
    assert np.allclose(w.vgas[1], Rc ** -0.5, rtol=6e-3)


def test_spherical_disk_recipe():
    w = I.sphdisk("small")
    e = w.edges
    assert w.geom == I.SPHERICAL and e[0][0] == pytest.approx(0.5) and e[0][-1] == pytest.approx(3.0)
    assert e[1][0] == pytest.approx(0.5 * np.pi - 0.3) and e[1][-1] == pytest.approx(0.5 * np.pi + 0.3)
    ratio = e[0][1:] / e[0][:-1]
    assert np.allclose(ratio, ratio[0])                      # log-spaced in r
    st = w.param
    assert st.min() >= 1e-4 and st.max() <= 10.0
    hist, _ = np.histogram(np.log10(st), bins=5, range=(-4.0, 1.0))
    assert hist.min() > 0.9 * hist.mean()                    # log-uniform
    assert (st < 1e-3).any()                                 # the stiff range is present
    assert _dust_to_gas(w) == pytest.approx(0.01, rel=1e-12)
    # hydrostatic density rho ~ r^-1.5 exp(-cot^2(theta) / (2 h^2)), h = 0.05
    rc = np.tile(0.5 * (e[0][1:] + e[0][:-1]), w.n[1] * w.n[2])
    thc = np.tile(np.repeat(0.5 * (e[1][1:] + e[1][:-1]), w.n[0]), w.n[2])
    expect = rc ** -1.5 * np.exp(-(1.0 / np.tan(thc)) ** 2 / (2 * 0.05 ** 2))
    assert np.allclose(w.rho, expect, rtol=1e-12)


def test_streaming_instability_batch_recipe():
    b = I.si2d_batch("full")
    assert len(b) == 64
    sides = sorted({w.n[0] for w in b})
    assert sides == [32, 64, 128, 256, 512]
    assert all(w.n[1] == 1 and w.n[2] == w.n[0] for w in b)
    ppc = {w.ngrains // w.ncell for w in b}
    assert min(ppc) == 1 and max(ppc) == 16
    assert {w.species_tau[0] for w in b} == {0.01, 0.1, 1.0}
    assert {round(_dust_to_gas(w), 12) for w in b} == {0.01, 0.02, 0.1}
    for w in b:
        # seeded Gaussian gas perturbations of amplitude 1e-3 about the
        # equilibrium flow
        for d in (0, 2):
            assert abs((w.vgas[d] - w.vgas[d].mean()).std() - 1e-3) < 3e-4


def test_generators_are_seeded():
    a, b = I.sbox3d("small"), I.sbox3d("small")
    for d in range(3):
        assert np.array_equal(a.q[d], b.q[d]) and np.array_equal(a.vgas[d], b.vgas[d])
    c = I.sbox3d("small", seed=I.BASE_SEED + 99)
    assert not np.array_equal(a.q[0], c.q[0])
