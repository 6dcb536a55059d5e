"""Invariants of the oracle's time step that hold exactly (to rounding).

* a uniform rest state stays within one rounding unit of f = w (the FP64 sum
  of the 19 weights is not exactly 1) and stops changing: no drift;
* mass is conserved with halfway walls (tangentially moving lid included);
* the Smagorinsky path with C = 0 is bit-identical to plain BGK;
* a uniform flow with walls and a sphere translating at the flow velocity is
  a fixed point for every branch of Eq. (19), and the momentum-exchange force
  and torque on the sphere vanish (symmetry of the cut-link set);
* with a body force the post-collision momentum of a uniform node grows by
  exactly rho g per step (the Guo source carries the whole force);
* with the covered / uncovered momentum correction, the total momentum of
  fluid and free spheres in a fully periodic box is constant (and it is not
  without the correction).
"""
import numpy as np

import oracle
from paper_1703_05158_gb300 import inputs


def _perturbed(o, amp, seed):
    c, w, _ = oracle.tables()
    eps = inputs.perturbation((19,) + o.shape, amp, seed)
    return w[:, None, None, None] * (1.0 + eps)


def test_rest_state_is_fixed_point():
    o = oracle.Oracle(10, 9, 8, tau0=0.7, cs=0.17)
    f0 = o.populations().copy()
    o.step(3000)
    f1 = o.populations().copy()
    assert np.abs(f1 - f0).max() <= 1e-16
    o.step(1)
    assert np.array_equal(o.populations(), f1)


def test_mass_conserved_with_walls_and_lid():
    o = oracle.Oracle(12, 10, 9, tau0=0.56, cs=0.17, g=(2e-5, -1e-5, 0.0), u_hi=(0.05, 0.02, 0.0))
    o.set_populations(_perturbed(o, 0.02, 11))
    m0 = o.populations().sum()
    o.step(200)
    assert abs(o.populations().sum() - m0) / m0 < 1e-13


def test_smagorinsky_zero_is_bgk_bitwise():
    kw = dict(tau0=0.62, g=(1e-5, 0, 0), u_hi=(0.03, 0, 0))
    a = oracle.Oracle(11, 9, 10, cs=0.0, les=True, **kw)
    b = oracle.Oracle(11, 9, 10, cs=0.0, les=False, **kw)
    f = _perturbed(a, 0.05, 3)
    for o in (a, b):
        o.set_particles([[5.3, 4.1, 4.7]], V=[[0.01, 0.0, -0.005]], R=[2.6])
        o.set_populations(f)
        o.step(30)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.forces()[0], b.forces()[0])


def test_uniform_flow_past_comoving_sphere_is_fixed_point():
    V = np.array([0.02, -0.011, 0.0])
    o = oracle.Oracle(24, 22, 20, tau0=0.6, cs=0.17, u_lo=V, u_hi=V)
    o.set_particles([[11.3, 10.7, 9.9]], V=[V], R=[4.3], fixed=[1])
    feq = oracle.feq(1.0, V)
    f = np.broadcast_to(feq[:, None, None, None], (19,) + o.shape).copy()
    o.set_populations(f)
    node, d, q, pid = o.links()
    assert (q < 0.5).any() and (q >= 0.5).any()
    o.step(25)
    owner = o.owner()
    fl = o.populations()[:, owner < 0]
    assert np.abs(fl - feq[:, None]).max() < 2e-15
    F, T = o.forces()
    assert np.abs(F).max() < 1e-13 and np.abs(T).max() < 1e-12
    assert o.steps == 25


def test_body_force_momentum_per_step():
    g = np.array([3e-5, -2e-5, 1e-5])
    o = oracle.Oracle(6, 6, 8, tau0=0.8, cs=0.1, g=g)
    o.step(1)
    rho, u = o.fields()
    # interior planes saw uniform neighbours: sum f c = rho g exactly, and the
    # reported velocity adds the half-force shift, u = 1.5 g
    for z in range(2, 6):
        assert np.allclose(u[:, z], (1.5 * g)[:, None, None], rtol=1e-9, atol=0)
        assert np.allclose(rho[z], 1.0, atol=1e-15)


def _total_momentum(o, R, rho_s):
    """Fluid momentum sum_i c_i f_i over fluid nodes plus sum_p m_p V_p."""
    c, _, _ = oracle.tables()
    f = o.populations()
    fluid = o.owner() < 0
    P = np.tensordot(c.T.astype(np.float64), f, axes=(1, 0))[:, fluid].sum(axis=1)
    _, V, _ = o.particles()
    m = rho_s * 4.0 / 3.0 * np.pi * np.asarray(R) ** 3
    return P + (m[:, None] * V).sum(axis=0)


def test_momentum_correction_conserves_total_momentum():
    """Fully periodic box (no walls, no body force) with free spheres that
    cover and uncover nodes every few steps: with the covered / uncovered
    momentum correction the total momentum of fluid and spheres is constant
    to rounding; without it the dropped and refilled nodes change it."""
    shape = (24, 20, 18)
    X = np.array([[6.3, 5.2, 5.9], [16.8, 13.1, 11.4], [7.7, 14.6, 13.2]])
    V = np.array([[0.06, 0.02, -0.01], [-0.03, 0.05, 0.02], [0.01, -0.04, 0.05]])
    R = np.array([3.1, 2.6, 2.2])
    drift = {}
    for corr in (True, False):
        o = oracle.Oracle(*shape, tau0=0.7, cs=0.17, rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=8,
                          periodic_z=True, momentum_correction=corr)
        o.set_particles(X, V=V, R=R)
        P0 = _total_momentum(o, R, 2.5)
        worst, refills = 0.0, 0
        for _ in range(40):
            o.step(1)
            refills += o.refilled
            worst = max(worst, float(np.abs(_total_momentum(o, R, 2.5) - P0).max()))
        assert refills > 20  # nodes were uncovered (and covered) along the way
        drift[corr] = worst / float(np.abs(P0).max())
    assert drift[True] <= 1e-12, drift
    assert drift[False] >= 1e-6, drift
