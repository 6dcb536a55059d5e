"""DEM precision on the GPU: centres and velocities are FP64, updated once
per lattice step from an in-step displacement and velocity change that the
16 sub-steps advance in FP32 (the reading of "FP64 DEM position
integration"; the sub-steps would cost ~64x in FP64 on this GPU).

Bound.  A sub-step adds its FP32 velocity increment with a relative rounding
error of at most 2^-24; during a contact the increments add up to the
impulse, |dv| <= 2|V| (a head-on bounce), over t_c / h sub-steps (t_c the
contact time of Eq. 1's spring-dashpot, h the sub-step), so one collision
leaves a velocity error of at most eps_c = (t_c / h) 2^-24 2 V_max.  With
n collisions in the run, |dV| <= n eps_c, and the centre error grows at most
linearly from each: n eps_c T.  The in-step displacement itself is a sum of
1/h FP32 increments of at most V_max h, rounded at most 2^-24 V_max each,
so the committed centres gain at most (1/h) 2^-24 V_max per step:
|dX| <= n eps_c T + T (1/h) 2^-24 V_max.  The hydrodynamic loads differ at
the FP32 level too; the spheres here are made heavy (density ratio 1e6,
k_n scaled with the mass so that t_c is the production one) so that those
loads move them by far less than the contact arithmetic.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_dem_drift_over_1000_steps_of_repeated_collisions():
    """Six spheres of radius 3 in a row along the periodic x axis of a
    48 x 24 x 24 box (walls in z, fluid at rest, no body force, no lid),
    neighbours 2 nodes apart moving at +-0.02 so that every pair collides
    again and again (restitution 0.95); 1000 steps against the FP64 oracle."""
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    shape = (48, 24, 24)
    n = 6
    X = np.array([[4.0 + 8.0 * k + 0.13 * (k % 3), 12.0 + 0.05 * k, 12.0 - 0.04 * k] for k in range(n)])
    V = np.array([[0.02 if k % 2 == 0 else -0.02, 0.0005 * k, -0.0003 * k] for k in range(n)])
    R = np.full(n, 3.0)
    rho_s, e = 1e6, 0.95
    kn = 1e3 * rho_s / 2.5  # the production k_n / m
    kw = dict(tau0=0.6, cs=0.0, rho_s=rho_s, kn=kn, restitution=e, dem_substeps=16)
    lat = lbm.Lattice(*shape, max_particles=n, max_radius=3.0, **kw)
    orc = oracle.Oracle(*shape, **kw)
    for o in (lat, orc):
        o.set_particles(X, V=V, R=R)
    m = rho_s * 4.0 / 3.0 * np.pi * 27.0
    meff = m / 2
    le = np.log(e)
    t_c = np.sqrt(meff / kn) * np.sqrt(np.pi ** 2 + le ** 2)  # contact time of the damped spring (steps)
    ulp, vmax, T, sub = 2.0 ** -24, 0.02, 1000, 16
    eps_c = (t_c * sub) * ulp * 2 * vmax
    x_bound = lambda nc: nc * eps_c * T + T * sub * ulp * vmax
    in_contact = np.zeros(n, dtype=bool)
    collisions = 0
    for s in range(1, T + 1):
        lat.step(1)
        orc.step(1)
        now = np.abs(orc.contact_forces()).sum(1) > 0
        collisions += int((now & ~in_contact).sum())
        in_contact = now
    Xg, Vg, _ = lat.particles()
    Xo, Vo, _ = orc.particles()
    dX, dV = float(np.abs(Xg - Xo).max()), float(np.abs(Vg - Vo).max())
    print("%d sphere collisions, contact time %.2f steps: |dX| %.2e (bound %.2e), |dV| %.2e (bound %.2e)" % (
        collisions, t_c, dX, x_bound(collisions), dV, collisions * eps_c))
    assert collisions >= 10
    assert dV <= collisions * eps_c
    assert dX <= x_bound(collisions)
    lat.close()
