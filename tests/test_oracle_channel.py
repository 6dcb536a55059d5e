"""Pins of the differentiation-form channel oracle (oracle/channel_oracle.c).

* Its tangent-linear pass against central differences of its own value part
  (a dropped or wrong derivative term anywhere in the step fails this).
* With x periodic and no plate, its lattice step against the main oracle
  (which the other test_oracle_* files pin): bitwise-close without
  obstacles, FP32-q-close with a fixed sphere.
* The rest state, continuity of the mass flux through an empty channel at
  steady state, and the sign of the drag and of its inlet derivative.
"""
import numpy as np
import pytest

import oracle

NO_PLATE = ((1, 1, 1), (0, 0, 0))  # empty node box


def small(**kw):
    base = dict(nx=24, ny=10, nz=12, tau0=0.6, cs=0.15, gx=2e-6, u_peak=0.04, plate_lo=(14, 2, 2),
                plate_hi=(15, 7, 9), steps=80, avg_from=41, X=np.array([[7.3, 4.6, 5.8], [19.1, 7.7, 3.2]]),
                R=np.array([2.6, 1.7]))
    base.update(kw)
    return base


@pytest.mark.parametrize("k", [0, 1, 2])
def test_tangent_linear_matches_central_differences(k):
    kw = small()
    names = ("u_peak", "gx", "cs")
    d = np.zeros(3)
    d[k] = 1.0
    tl = oracle.channel(**kw, dtheta=d)["dJ"]
    h = 1e-4 * kw[names[k]]
    jp = oracle.channel(**dict(kw, **{names[k]: kw[names[k]] + h}))["J"]
    jm = oracle.channel(**dict(kw, **{names[k]: kw[names[k]] - h}))["J"]
    fd = (jp - jm) / (2 * h)
    assert abs(tl - fd) <= 1e-6 * abs(tl), (tl, fd)


def test_tangent_is_linear_in_the_direction():
    kw = small(steps=40, avg_from=21)
    parts = [oracle.channel(**kw, dtheta=np.eye(3)[k])["dJ"] for k in range(3)]
    mix = oracle.channel(**kw, dtheta=(0.5, -2.0, 3.0))["dJ"]
    assert abs(mix - (0.5 * parts[0] - 2.0 * parts[1] + 3.0 * parts[2])) <= 1e-12 * max(abs(p) for p in parts)


def _main(shape, steps, tau0, cs, gx, X=None, R=None):
    o = oracle.Oracle(*shape, tau0=tau0, cs=cs, g=(gx, 0.0, 0.0))
    if X is not None:
        o.set_particles(X, V=np.zeros_like(X), R=R, fixed=np.ones(len(R), dtype=np.uint8))
    o.step(steps)
    return o.populations()


def test_periodic_channel_is_the_main_oracle_step():
    shape = (16, 8, 10)
    c = oracle.channel(*shape, tau0=0.7, cs=0.17, gx=3e-5, u_peak=0.0, plate_lo=NO_PLATE[0],
                       plate_hi=NO_PLATE[1], steps=30, avg_from=1, periodic_x=True, populations=True)
    m = _main(shape, 30, 0.7, 0.17, 3e-5)
    assert np.abs(c["f"] - m).max() <= 1e-14


def test_periodic_channel_with_a_fixed_sphere_is_the_main_oracle_step():
    # half-integer centre, R^2 = 8.41: every |x - X|^2 is 0.75 mod 2, so the
    # FP32 inside test of the main oracle and the FP64 test here agree
    shape = (20, 10, 12)
    X, R = np.array([[9.5, 4.5, 5.5]]), np.array([2.9])
    c = oracle.channel(*shape, tau0=0.7, cs=0.17, gx=3e-5, u_peak=0.0, plate_lo=NO_PLATE[0],
                       plate_hi=NO_PLATE[1], steps=30, avg_from=1, X=X, R=R, periodic_x=True, populations=True)
    m = _main(shape, 30, 0.7, 0.17, 3e-5, X=X, R=R)
    fluid = c["type"] == 0
    rel = np.abs(c["f"] - m)[:, fluid] / np.abs(m[:, fluid])
    assert rel.max() <= 1e-6  # the main oracle's link fractions are FP32


def test_rest_state_and_zero_drag():
    r = oracle.channel(20, 8, 10, tau0=0.7, cs=0.15, gx=0.0, u_peak=0.0, plate_lo=(10, 2, 2), plate_hi=(11, 5, 7),
                       steps=30, avg_from=11, populations=True)
    c, w, _ = oracle.tables()
    fluid = (r["type"] != 1) & (r["type"] != 4)
    assert np.abs(r["f"][:, fluid] - w[:, None]).max() <= 1e-14
    assert abs(r["J"]) <= 1e-13


def test_mass_flux_is_the_same_through_every_plane_at_steady_state():
    nx, ny, nz = 16, 6, 10
    r = oracle.channel(nx, ny, nz, tau0=0.8, cs=0.0, gx=0.0, u_peak=0.02, plate_lo=NO_PLATE[0],
                       plate_hi=NO_PLATE[1], steps=3000, avg_from=1, populations=True)
    c, _, _ = oracle.tables()
    f = r["f"]
    jx = np.tensordot(c[:, 0], f, axes=(0, 0))  # [nz, ny, nx]
    flux = jx.sum(axis=(0, 1))[1:-1]
    zh = (np.arange(nz) + 0.5) / nz
    inlet = ny * np.sum(0.02 * 4 * zh * (1 - zh))
    assert np.abs(flux - flux.mean()).max() <= 2e-3 * abs(flux.mean())
    assert abs(flux.mean() - inlet) <= 0.05 * inlet


def test_drag_and_its_inlet_derivative_are_positive():
    a = oracle.channel(**small(u_peak=0.02), dtheta=(1.0, 0.0, 0.0))
    b = oracle.channel(**small(u_peak=0.04))
    assert 0.0 < a["J"] < b["J"]
    assert a["dJ"] > 0.0
