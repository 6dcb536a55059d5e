"""Pins of the oracle's DEM (Sect. 2.1, Eq. 1, velocity Verlet), no fluid.

The linear spring-dashpot contact is a damped harmonic oscillator in the
normal relative coordinate: contact time t_c = pi / sqrt(k/m - (gamma/2m)^2)
and normal restitution exp(-gamma t_c / (2 m)) = e, with m the reduced mass.
"""
import numpy as np
import pytest

import oracle


def _collide(e, kn=10.0, R=(4.0, 4.0), v=0.02, steps=60, sub=32, fixed=None, wall=False):
    o = oracle.Oracle(64, 32, 40, tau0=0.8, rho_s=2.5, kn=kn, restitution=e, dem_substeps=sub, fluid=False)
    if wall:
        X = [[20.0, 16.0, R[0] - 0.5 + 0.05]]
        V = [[0.0, 0.0, -v]]
        o.set_particles(X, V=V, R=[R[0]])
    else:
        X = [[20.0, 16.0, 20.0], [20.0 + R[0] + R[1] + 0.05, 16.0, 20.0]]
        V = [[v, 0.0, 0.0], [-v, 0.0, 0.0]]
        o.set_particles(X, V=V, R=list(R), fixed=fixed)
    traj = []
    for _ in range(steps):
        o.step(1)
        traj.append(o.particles())
    return o, traj


def _mass(R, rho_s=2.5):
    return rho_s * 4.0 / 3.0 * np.pi * R ** 3


@pytest.mark.parametrize("R", [(4.0, 4.0), (3.0, 5.0)])
def test_restitution_and_contact_time(R):
    e, kn, v = 0.8, 10.0, 0.02
    o, traj = _collide(e, kn=kn, R=R, v=v)
    X, V, _ = traj[-1]
    rel_after = V[1, 0] - V[0, 0]
    assert abs(rel_after / (2 * v) - e) < 1e-3
    ma, mb = _mass(R[0]), _mass(R[1])
    # momentum conservation
    assert abs(ma * V[0, 0] + mb * V[1, 0] - (ma * v - mb * v)) < 1e-12
    meff = ma * mb / (ma + mb)
    le = np.log(e)
    gamma = -2 * le * np.sqrt(meff * kn) / np.sqrt(np.pi ** 2 + le ** 2)
    tc = np.pi / np.sqrt(kn / meff - (gamma / (2 * meff)) ** 2)
    # contact lasts tc: measure from overlap of the trajectory
    overl = [R[0] + R[1] - np.linalg.norm(x[1] - x[0]) > 0 for x, _, _ in traj]
    n_in = sum(overl)
    assert abs(n_in - tc) <= 1.5


def test_elastic_energy_conserved():
    _, traj = _collide(1.0, v=0.02)
    X, V, _ = traj[-1]
    assert abs((V[1, 0] - V[0, 0]) / 0.04 - 1.0) < 1e-3


def test_wall_restitution():
    v = 0.02
    _, traj = _collide(0.8, v=v, wall=True)
    X, V, _ = traj[-1]
    assert abs(V[0, 2] / v - 0.8) < 2e-3


def test_fixed_sphere_is_infinite_mass():
    v = 0.02
    _, traj = _collide(0.8, v=v, fixed=[0, 1])
    X, V, _ = traj[-1]
    # sphere 1 is prescribed at -v: sphere 0 sees a wall moving at -v
    assert V[1, 0] == -v
    assert abs((V[1, 0] - V[0, 0]) / (2 * v) - 0.8) < 2e-3


def test_external_load_constant_acceleration():
    """A constant external force and torque on a free sphere (no contacts,
    no fluid) give v = v0 + F t / m and Om = T t / I exactly (Verlet is exact
    for constant acceleration)."""
    R, m = 3.0, _mass(3.0)
    I = 0.4 * m * R * R
    o = oracle.Oracle(40, 40, 40, tau0=0.8, fluid=False, dem_substeps=8)
    o.set_particles([[20.0, 20.0, 20.0]], V=[[0.01, 0.0, 0.0]], R=[R])
    F, T = np.array([[1e-3, -2e-3, 5e-4]]), np.array([[0.0, 3e-3, -1e-3]])
    o.set_load(F, T)
    o.step(10)
    X, V, Om = o.particles()
    assert np.allclose(V[0], [0.01, 0, 0] + F[0] * 10 / m, rtol=1e-12, atol=1e-18)
    assert np.allclose(Om[0], T[0] * 10 / I, rtol=1e-12, atol=1e-18)
    assert np.allclose(X[0], [20.0, 20.0, 20.0] + np.array([0.01, 0, 0]) * 10 + 0.5 * F[0] * 100 / m, rtol=1e-12)
