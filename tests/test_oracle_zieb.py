"""Pins of the ZIEB face of the oracle (Sect. 2.6, Eqs. 8, 9): the plane
z = 0 exchanges fluid with a virtual cylinder of volume V_0 and
cross-section A_p whose piston moves at v_p.

* A piston at rest over a fluid at rest leaves everything exactly at rest.
* After every step the face holds exactly the cylinder density rho^{n+1}
  (Eq. 9 fixes the missing mass, the equilibrium keeps it) and its mean
  normal velocity is the v_f the next update of Eq. 8 uses.
* Quasi-static compression and expansion: fluid mass is conserved between
  cylinder and lattice (the face plane, shared by both, counted half), the
  lattice ends at the cylinder density, and that density is the closed form
  M / (V_lattice - A_p / 2 + V_0 - A_p H_p).
* A uniform flow along the face under a lid moving with it, piston at rest,
  is a fixed point: the face's five unknown populations carry the node's own
  tangential state, so its redistribution returns f^eq(1, u0).  A reading
  that filled them from the cylinder at rest (w rho) would take the
  tangential momentum of populations 7, 9, 15, 17 out of the face's velocity
  and break the fixed point.  (Own post- against pre-collision values, and
  rho^{n+1} against rho* in the velocity, coincide in this state.)
"""
import numpy as np
import pytest

import oracle

NX, NY, NZ = 8, 8, 24
A = NX * NY
V0 = 40.0 * A


def cylinder(vp, tau0=1.0):
    return oracle.Oracle(NX, NY, NZ, tau0=tau0, cs=0.0, zieb=dict(area=A, volume=V0, vp=vp))


def test_piston_at_rest_keeps_the_rest_state():
    o = cylinder(0.0)
    o.step(50)
    _, w, _ = oracle.tables()
    assert np.abs(o.populations() - w[:, None, None, None]).max() <= 1e-15
    rho, H, vf = o.zieb_state()
    assert abs(rho - 1.0) <= 1e-15 and H == 0.0 and abs(vf) <= 1e-15


def test_face_holds_the_cylinder_density_and_its_inflow():
    o = cylinder(0.02, tau0=0.8)
    for _ in range(30):
        o.step(1)
        rho, H, vf = o.zieb_state()
        r, u = o.fields()
        assert np.abs(r[0] - rho).max() <= 1e-14
        assert abs(u[2, 0].mean() - vf) <= 1e-15
    assert rho > 1.0 and abs(H - 0.6) <= 1e-12


def _half_face_mass(o):
    f = o.populations()
    return f[:, 1:].sum() + 0.5 * f[:, 0].sum()


@pytest.mark.parametrize("vp", [0.0025, -0.0025])
def test_slow_stroke_conserves_mass_and_reaches_the_closed_form_density(vp):
    o = cylinder(vp)
    M0 = _half_face_mass(o) + V0
    o.step(4000)  # stroke of 10 nodes
    o.zieb_set_piston(0.0)
    o.step(3000)  # at rest again
    rho, H, _ = o.zieb_state()
    assert abs(H - 4000 * vp) <= 1e-9
    M = _half_face_mass(o) + rho * (V0 - A * H)
    assert abs(M - M0) <= 1e-4 * M0
    r, _ = o.fields()
    assert np.abs(r - rho).max() <= 1e-4  # uniform at the cylinder density
    closed = M0 / (NX * NY * NZ - 0.5 * A + V0 - A * H)
    assert abs(rho - closed) <= 1e-4 * closed
    assert (rho > 1.0) == (vp > 0)


def test_uniform_tangential_flow_under_a_comoving_lid_is_a_fixed_point():
    u0 = np.array([0.04, -0.02, 0.0])
    o = oracle.Oracle(NX, NY, NZ, tau0=0.6, cs=0.15, u_hi=tuple(u0), zieb=dict(area=A, volume=V0, vp=0.0))
    f = np.broadcast_to(oracle.feq(1.0, u0)[:, None, None, None], (19, NZ, NY, NX)).copy()
    o.set_populations(f)
    o.step(30)
    assert np.abs(o.populations() - f).max() <= 1e-14
    rho, H, vf = o.zieb_state()
    assert rho == 1.0 and H == 0.0 and abs(vf) <= 1e-14
