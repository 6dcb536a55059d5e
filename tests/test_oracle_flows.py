"""Closed-form steady flows between the z walls (Sect. 2.2 with halfway walls).

* Couette: lid at z = nz - 1/2 moving at U, bottom wall at rest: the profile
  u(z) = U (z + 1/2) / nz is exact for BGK with halfway bounce-back.
* Poiseuille: body force g along x: u(z) = g/(2 nu) [(nz/2)^2 - (z - zc)^2],
  zc = (nz - 1)/2, nu = (tau - 1/2)/3.  With BGK and halfway walls the wall
  slip vanishes at (tau - 1/2)^2 = 3/16, where the profile is exact.
* Smagorinsky in uniform shear: the eddy viscosity must equal (C dx)^2 |S|
  with |S| = sqrt(2 S:S) = du/dz, i.e. tau_t = 3 C^2 du/dz (lattice units).
  This pins the reading of Eq. (18) independently of its printed form.
"""
import numpy as np

import oracle


def test_couette_linear_profile():
    nz, U = 16, 0.04
    o = oracle.Oracle(1, 1, nz, tau0=0.8, cs=0.0, u_hi=(U, 0.0, 0.0))
    o.step(20000)
    _, u = o.fields()
    z = np.arange(nz)
    assert np.allclose(u[0, :, 0, 0], U * (z + 0.5) / nz, rtol=0, atol=2e-13)
    assert np.abs(u[1:]).max() < 1e-13


def test_poiseuille_exact_at_magic_tau():
    nz, g = 16, 1e-5
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    o = oracle.Oracle(1, 1, nz, tau0=tau, cs=0.0, g=(g, 0.0, 0.0))
    o.step(9000)
    _, u = o.fields()
    z = np.arange(nz)
    zc = (nz - 1) / 2.0
    exact = g / (2 * nu) * ((nz / 2.0) ** 2 - (z - zc) ** 2)
    assert np.abs(u[0, :, 0, 0] - exact).max() / exact.max() < 1e-9


def test_poiseuille_curvature_other_tau():
    """At any tau the interior second difference is -g/nu exactly."""
    nz, g, tau = 20, 2e-6, 0.65
    nu = (tau - 0.5) / 3.0
    o = oracle.Oracle(1, 1, nz, tau0=tau, cs=0.0, g=(g, 0.0, 0.0))
    o.step(30000)
    _, u = o.fields()
    ux = u[0, :, 0, 0]
    d2 = ux[2:] - 2 * ux[1:-1] + ux[:-2]
    assert np.allclose(d2, -g / nu, rtol=1e-8)


def test_smagorinsky_eddy_viscosity_in_uniform_shear():
    nz, U, C, tau0 = 16, 0.05, 0.3, 0.6
    o = oracle.Oracle(1, 1, nz, tau0=tau0, cs=C, u_hi=(U, 0.0, 0.0))
    o.step(8000)
    _, u = o.fields()
    ux = u[0, :, 0, 0]
    shear = np.diff(ux)[3:-3]
    assert np.allclose(shear, shear.mean(), rtol=1e-4)  # linear up to O(u^2) terms
    tau_t = o.tau_eff()[4:-4, 0, 0] - tau0
    expected = 3.0 * C * C * shear.mean()
    assert np.allclose(tau_t, expected, rtol=2e-4)
    # the alternative reading with Pi = sqrt(2 Pi:Pi) would be off by ~sqrt(2)
    assert abs(tau_t.mean() / expected - 1.0) < 0.1
