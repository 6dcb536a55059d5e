"""Per-step host I/O of the sphere state: lbm_set_particle_load from host
arrays takes the values at the call, and lbm_particle_state returns what
lbm_forces and lbm_particles return, with one synchronisation.

The library stages host values in pinned memory before it returns (the copy
to the device then runs in stream order, without a stream synchronisation),
so a caller that overwrites its arrays right after the call, and keeps
setting loads step after step (both staging slots in turn, each reused only
after its previous copy), moves the spheres exactly as one that leaves them
alone, and as the oracle with the same loads.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SHAPE = (32, 32, 32)
KW = dict(tau0=0.8, cs=0.1, g=(0.0, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8)


def lbm():
    from paper_1703_05158_gb300 import lbm as mod

    mod.load()
    return mod


def loads(k):
    """The load of step k: a force along x and z and a torque about y."""
    F = np.array([[2e-3 * np.sin(0.3 * k), 0.0, 1e-3], [-1e-3, 1e-3 * np.cos(0.2 * k), 0.0]])
    T = np.array([[0.0, 1e-3, 0.0], [0.0, 0.0, -2e-3 * np.sin(0.1 * k)]])
    return F, T


def test_host_loads_are_taken_at_the_call():
    L = lbm()
    X = np.array([[10.3, 12.1, 14.7], [21.6, 18.2, 15.4]])
    R = np.array([3.0, 2.5])
    runs = []
    for overwrite in (False, True):
        lat = L.Lattice(*SHAPE, max_particles=2, max_radius=3.0, **KW)
        lat.set_particles(X, R=R)
        for k in range(12):
            F, T = loads(k)
            L.lbm_set_particle_load(lat.h, F, T)
            if overwrite:  # the caller reuses its arrays at once
                F[:] = 1e3
                T[:] = -1e3
            lat.step(1)
        runs.append(lat.particles())
        lat.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)
    orc = oracle.Oracle(*SHAPE, **KW)
    orc.set_particles(X, R=R)
    for k in range(12):
        orc.set_load(*loads(k))
        orc.step(1)
    Xo, Vo, Wo = orc.particles()
    Xg, Vg, Wg = runs[1]
    assert np.abs(Xg - Xo).max() <= 1e-6
    assert np.abs(Vg - Vo).max() <= 1e-4 * np.abs(Vo).max()
    assert np.abs(Wg - Wo).max() <= 1e-4 * np.abs(Wo).max()


def test_particle_state_is_forces_and_particles_in_one_call():
    L = lbm()
    lat = L.Lattice(*SHAPE, max_particles=2, max_radius=3.0, **KW)
    lat.set_particles(np.array([[10.3, 12.1, 14.7], [21.6, 18.2, 15.4]]), R=np.array([3.0, 2.5]))
    L.lbm_set_particle_load(lat.h, *loads(0))
    lat.step(5)
    F, T = lat.forces()
    X, V, W = lat.particles()
    out = [np.empty((2, 3)) for _ in range(5)]
    L.lbm_particle_state(lat.h, *out)
    for a, b in zip(out, (F, T, X, V, W)):
        assert np.array_equal(a, b)
    Fo = np.empty((2, 3))
    L.lbm_particle_state(lat.h, F=Fo)  # any output may be left out
    assert np.array_equal(Fo, F)
    lat.close()
