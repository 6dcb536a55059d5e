"""Pins of the tangential contact law of the DEM oracle (Eqs. 2, 3: linear
tangential spring and dashpot, Coulomb cap), dry (no lattice).

* A sphere launched without spin along a wall it rests on under a load
  m g: while it slides the Coulomb force -mu m g decelerates it exactly
  (v = v0 - mu g t) and spins it up at the arm R - delta/2 of the contact
  point; it then rolls without slipping at the velocity those two laws fix,
  v0 * 2.5 r^2 / (1 + 2.5 r^2) with r = (R - delta/2) / R (5/7 v0 for a
  point contact).
* A tangential load F at the centre of a resting sphere: below the Coulomb
  limit it rolls with acceleration F / (m + I / l^2) (static friction), above
  it slides with (F - mu m g) / m.
* An oblique collision of two spinning spheres conserves the total linear
  momentum and the total angular momentum (orbital plus spin) to rounding,
  which fixes the contact point at the middle of the overlap and the sign of
  every tangential term; the contact dissipates energy.
* Friction off (mu = 0) leaves the frictionless oracle bit for bit.
* The tangential force lies in the contact's tangent plane even while the
  normal turns under a loaded displacement (a sphere sliding, then rolling,
  over a fixed sphere): with an elastic normal law the contact force along
  n is exactly k_n delta at every step.
"""
import numpy as np
import pytest

import oracle

R, RHO_S, KN = 4.0, 2.5, 1e3
M = RHO_S * 4.0 / 3.0 * np.pi * R ** 3
I = 0.4 * M * R ** 2


def resting(mu, g=1e-2, kt=0.5 * KN, et=0.5, **kw):
    """A sphere at rest on the wall z = -1/2 at the overlap m g / k_n."""
    pen = M * g / KN
    o = oracle.Oracle(32, 32, 16, tau0=0.6, rho_s=RHO_S, kn=KN, restitution=0.8, dem_substeps=16, fluid=False,
                      kt=kt, mu=mu, restitution_t=et)
    return o, pen, np.array([[10.0, 10.0, R - 0.5 - pen]])


@pytest.mark.parametrize("et", [0.5, 1.0])
def test_sliding_sphere_decelerates_at_mu_g_then_rolls(et):
    """Slip stops at t = 28.6; at t = 27 the slip velocity (1e-3) is so small
    that without the reset of delta_t to the Coulomb value after each sliding
    sub-step (and with no tangential damping, et = 1) the contact would
    stick-slip instead of sliding."""
    mu, g, v0 = 0.02, 1e-2, 0.02
    o, pen, X = resting(mu, g, et=et)
    o.set_particles(X, V=np.array([[v0, 0.0, 0.0]]), R=np.array([R]))
    o.set_load(F=np.array([[0.0, 0.0, -M * g]]))
    lever = R - 0.5 * pen
    # the first half kick uses the contact force of the initial state, where
    # delta_t = 0: with et = 1 that has no tangential part (mu g h / 2 of
    # velocity is missing); from there on the Coulomb force acts exactly
    o.step(5)
    _, Va, Wa = o.particles()
    h = 1.0 / 16
    assert abs(Va[0, 0] - (v0 - mu * g * 5) - (0.5 * mu * g * h if et == 1.0 else 0.0)) <= 1e-12
    for t in (10, 20, 27):
        o.step(t - o.steps)
        _, V, W = o.particles()
        assert abs((V[0, 0] - Va[0, 0]) + mu * g * (t - 5)) <= 1e-12
        assert abs((W[0, 1] - Wa[0, 1]) - lever * mu * M * g * (t - 5) / I) <= 1e-12
        assert np.abs(V[0, 1:]).max() <= 1e-12 and abs(W[0, 0]) + abs(W[0, 2]) <= 1e-12
    if et == 1.0:
        return  # without tangential damping the stuck contact rings on the tangential spring
    o.step(200 - o.steps)
    _, V, W = o.particles()
    r2 = (lever / R) ** 2
    v_roll = v0 * 2.5 * r2 / (1.0 + 2.5 * r2)
    assert abs(V[0, 0] - v_roll) <= 1e-5 * v_roll
    assert abs(V[0, 0] - lever * W[0, 1]) <= 1e-5 * v_roll  # the contact point is at rest


@pytest.mark.parametrize("regime", ["rolls", "slides"])
def test_tangential_load_rolls_below_the_coulomb_limit_and_slides_above(regime):
    mu, g = 0.05, 1e-2
    o, pen, X = resting(mu, g)
    lever = R - 0.5 * pen
    # rolling needs a static friction of F I / (I + m l^2) <= mu m g
    limit = mu * M * g * (I + M * lever ** 2) / I
    F = 0.5 * limit if regime == "rolls" else 2.0 * limit
    o.set_particles(X, R=np.array([R]))
    o.set_load(F=np.array([[F, 0.0, -M * g]]))
    o.step(40)
    _, V0, _ = o.particles()
    o.step(40)
    _, V1, W1 = o.particles()
    acc = (V1[0, 0] - V0[0, 0]) / 40.0
    want = F / (M + I / lever ** 2) if regime == "rolls" else (F - mu * M * g) / M
    assert abs(acc - want) <= 2e-3 * want, (acc, want)
    if regime == "rolls":
        assert abs(V1[0, 0] - lever * W1[0, 1]) <= 1e-3 * V1[0, 0]


def _momenta(o, R):
    X, V, W = o.particles()
    m = RHO_S * 4.0 / 3.0 * np.pi * R ** 3
    P = (m[:, None] * V).sum(axis=0)
    L = (m[:, None] * np.cross(X, V)).sum(axis=0) + ((0.4 * m * R ** 2)[:, None] * W).sum(axis=0)
    E = 0.5 * (m * (V ** 2).sum(axis=1)).sum() + 0.5 * ((0.4 * m * R ** 2) * (W ** 2).sum(axis=1)).sum()
    return P, L, E


def test_oblique_collision_conserves_momentum_and_angular_momentum():
    Rs = np.array([4.0, 3.0])
    X = np.array([[20.0, 20.0, 20.0], [27.2, 22.1, 20.9]])
    V = np.array([[0.03, 0.01, 0.0], [-0.02, 0.0, 0.005]])
    W = np.array([[0.0, 0.0, 0.004], [0.002, -0.003, 0.0]])
    o = oracle.Oracle(48, 48, 48, tau0=0.6, rho_s=RHO_S, kn=KN, restitution=0.7, dem_substeps=16, fluid=False,
                      periodic_z=True, kt=0.4 * KN, mu=0.3, restitution_t=0.6)
    o.set_particles(X, V=V, Om=W, R=Rs)
    P0, L0, E0 = _momenta(o, Rs)
    touched = False
    for _ in range(120):
        o.step(1)
        touched |= bool(np.abs(o.contact_torques()).max() > 0.0)
        P, L, _ = _momenta(o, Rs)
        assert np.abs(P - P0).max() <= 1e-13 * np.abs(P0).max()
        assert np.abs(L - L0).max() <= 1e-12 * np.abs(L0).max()
    assert touched  # friction acted
    _, _, E = _momenta(o, Rs)
    assert E < E0


def test_no_friction_is_the_frictionless_oracle():
    X = np.array([[10.0, 12.0, 3.3], [17.0, 12.5, 3.6]])
    V = np.array([[0.02, 0.0, -0.01], [-0.02, 0.0, 0.0]])
    W = np.array([[0.0, 0.01, 0.0], [0.0, 0.0, 0.0]])
    runs = []
    for kw in (dict(), dict(kt=500.0, mu=0.0, restitution_t=0.5)):
        o = oracle.Oracle(32, 32, 16, tau0=0.6, rho_s=RHO_S, kn=KN, restitution=0.8, dem_substeps=16, fluid=False,
                          **kw)
        o.set_particles(X, V=V, Om=W, R=np.array([4.0, 3.0]))
        o.step(60)
        runs.append(o.particles())
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_a_contact_that_opens_forgets_its_tangential_displacement():
    """A spinning sphere bouncing on the wall under a load m g: restarting a
    fresh oracle from the state between two bounces (which has delta_t = 0)
    gives bit for bit the same second bounce, so the first bounce left no
    tangential displacement behind (as the contact unloads, the Coulomb cap
    falls to 0 and takes delta_t with it; the reset on opening makes sure)."""
    g = 1e-2
    kw = dict(tau0=0.6, rho_s=RHO_S, kn=KN, restitution=0.8, dem_substeps=16, fluid=False, kt=0.5 * KN, mu=0.3,
              restitution_t=0.5)
    a = oracle.Oracle(32, 32, 24, **kw)
    a.set_particles(np.array([[10.0, 10.0, R]]), V=np.array([[0.02, 0.0, 0.0]]), Om=np.array([[0.0, 0.0, 0.003]]),
                    R=np.array([R]))
    load = np.array([[0.0, 0.0, -M * g]])
    a.set_load(F=load)
    seen = False
    for _ in range(200):
        a.step(1)
        touching = bool(np.abs(a.contact_forces()).max() > 0.0)
        seen |= touching
        if seen and not touching:
            break
    assert seen and not touching
    X, V, W = a.particles()
    b = oracle.Oracle(32, 32, 24, **kw)
    b.set_particles(X, V=V, Om=W, R=np.array([R]))
    b.set_load(F=load)
    second = False
    for _ in range(60):  # the second bounce
        for o in (a, b):
            o.step(1)
        second |= bool(np.abs(b.contact_torques()).max() > 0.0)
    assert second
    for u, v in zip(a.particles(), b.particles()):
        assert np.array_equal(u, v)


def test_tangential_force_stays_in_the_tangent_plane_while_the_normal_turns():
    """A sphere pressed onto the top of a fixed sphere by a constant load
    m g along -z and launched sideways slides, rolls and is carried round
    the fixed sphere, so the contact normal turns by tens of degrees while
    the stored displacement delta_t carries a load of up to mu f_n.  With
    e = 1 the normal law is k_n delta alone, so at every step in contact the
    force along n = (X_a - X_b) / |X_a - X_b| must be k_n delta, which holds
    only if delta_t is turned into the tangent plane as n moves (a
    displacement kept as a fixed vector would tilt the spring force out of
    that plane by about |f_t| times the angle turned)."""
    Ra, Rb, kt, g = 3.0, 4.0, 500.0, 1e-2
    m = RHO_S * 4.0 / 3.0 * np.pi * Ra ** 3
    o = oracle.Oracle(32, 32, 40, tau0=1.0, rho_s=RHO_S, kn=KN, restitution=1.0, dem_substeps=16, fluid=False,
                      kt=kt, mu=0.3, restitution_t=0.6)
    X = np.array([[16.0, 16.0, 20.0 + Ra + Rb - m * g / KN], [16.0, 16.0, 20.0]])
    o.set_particles(X, V=np.array([[0.02, 0.0, 0.0], [0.0, 0.0, 0.0]]), R=np.array([Ra, Rb]),
                    fixed=np.array([0, 1], dtype=np.uint8))
    o.set_load(F=np.array([[0.0, 0.0, -m * g], [0.0, 0.0, 0.0]]))
    tilt, ft_ratio, touching = [], 0.0, 0
    for _ in range(400):
        o.step(1)
        Xs = o.particles()[0]
        d = Xs[0] - Xs[1]
        delta = Ra + Rb - np.linalg.norm(d)
        if delta <= 0.0 or Xs[0, 2] - Ra <= -0.5:
            continue  # contact open (or the wall touched)
        n = d / np.linalg.norm(d)
        F = o.contact_forces()[0]
        fn = F @ n
        assert abs(fn - KN * delta) <= 1e-10 * np.linalg.norm(F), (fn, KN * delta)
        touching += 1
        tilt.append(np.degrees(np.arccos(n[2])))
        ft_ratio = max(ft_ratio, np.linalg.norm(F - fn * n) / fn)
    assert touching >= 50 and max(tilt) - min(tilt) > 30.0 and ft_ratio > 0.1
