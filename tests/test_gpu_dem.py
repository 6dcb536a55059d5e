"""DEM precision on the GPU: centres and velocities are FP64, updated once
per lattice step from an in-step displacement and velocity change that the
16 sub-steps advance in FP32 (the reading of "FP64 DEM position
integration"; the sub-steps would cost ~64x in FP64 on this GPU).

Bound for one collision.  During a contact a sphere's FP32 velocity
increments add up to the impulse, |dv| <= 2|V| (a head-on bounce), over
t_c / h sub-steps (t_c the contact time of Eq. 1's spring-dashpot, h the
sub-step); each sub-step rounds the contact force and the increment, a few
(at most 4) operations of relative error 2^-24 each, so one collision leaves
a velocity error of at most eps_c = 4 (t_c / h) 2^-24 2 V_max.  The centre
error then grows at most linearly: eps_c T.  The in-step displacement itself
is a sum of 1/h FP32 increments of at most V_max h, rounded at most 2^-24
V_max each, so the committed centres gain at most (1/h) 2^-24 V_max per step.

Repeated collisions are not bounded this way: where a contact begins
relative to the sub-steps changes its outcome, so the velocity error one
collision leaves (~1e-8 here) moves the onset of the next, and each further
collision amplifies the difference (by ~400 in a head-on pair re-colliding
across a periodic edge); no test asserts a bound there.

The spheres are heavy (density ratio 1e6, k_n scaled with the mass so that
t_c is the production one), so that the hydrodynamic loads, which differ at
the FP32 level too, move them by far less than the contact arithmetic.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

RHO_S = 1e6
KN = 1e3 * RHO_S / 2.5  # the production k_n / m
ULP, VMAX, SUB = 2.0 ** -24, 0.02, 16


def _pairs(nx, e):
    """Sixteen pairs of spheres of radius 3, each pair on its own line along
    the periodic x axis of an nx x 48 x 48 box (walls in z, fluid at rest, no
    body force, no lid), approaching head on at +-0.02 (contact normal along
    x, so no glancing collisions)."""
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    shape = (nx, 48, 48)
    X, V = [], []
    for iy in range(4):
        for iz in range(4):
            y, z = 6.0 + 12.0 * iy, 6.0 + 12.0 * iz
            x0 = 3.5 + 0.25 * iy + 0.1 * iz
            X += [[x0, y, z], [x0 + 10.0, y, z]]
            V += [[VMAX, 0.0, 0.0], [-VMAX, 0.0, 0.0]]
    X, V = np.array(X), np.array(V)
    R = np.full(len(X), 3.0)
    kw = dict(tau0=0.6, cs=0.0, rho_s=RHO_S, kn=KN, restitution=e, dem_substeps=SUB)
    lat = lbm.Lattice(*shape, max_particles=len(R), max_radius=3.0, **kw)
    orc = oracle.Oracle(*shape, **kw)
    for o in (lat, orc):
        o.set_particles(X, V=V, R=R)
    meff = RHO_S * 4.0 / 3.0 * np.pi * 27.0 / 2
    t_c = np.sqrt(meff / KN) * np.sqrt(np.pi ** 2 + np.log(e) ** 2)  # contact time (steps)
    return lat, orc, (shape, kw, X, V, R), t_c


def _run(objs, steps, orc):
    """Step every object; count each sphere's collisions (contact onsets) on
    the oracle."""
    n = len(orc.particles()[0])
    in_contact = np.zeros(n, dtype=bool)
    hits = np.zeros(n, dtype=int)
    for _ in range(steps):
        for o in objs:
            o.step(1)
        now = np.abs(orc.contact_forces()).sum(1) > 0
        hits += now & ~in_contact
        in_contact = now
    return hits


def test_dem_drift_over_1000_steps_with_one_collision_per_sphere():
    """A 96-long box: each pair meets once (at step ~100) and not again within
    1000 steps; centres and velocities against the FP64 oracle within the
    one-collision bound."""
    lat, orc, _, t_c = _pairs(96, 0.8)
    T = 1000
    hits = _run([lat, orc], T, orc)
    Xg, Vg, _ = lat.particles()
    Xo, Vo, _ = orc.particles()
    dX, dV = float(np.abs(Xg - Xo).max()), float(np.abs(Vg - Vo).max())
    eps_c = 4 * (t_c * SUB) * ULP * 2 * VMAX
    n = int(hits.max())
    x_bound = n * eps_c * T + T * SUB * ULP * VMAX
    print("collisions per sphere %d, contact time %.2f steps: |dX| %.2e (bound %.2e), |dV| %.2e (bound %.2e)" % (
        n, t_c, dX, x_bound, dV, n * eps_c))
    assert hits.min() == 1 and n == 1
    assert dV <= n * eps_c
    assert dX <= x_bound
    lat.close()
