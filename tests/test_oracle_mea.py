"""The Galilean-invariant momentum exchange of the oracle (option
mea="galilean"; Wen, Zhang & Fang 2014, not in the paper).  It differs from
Eqs. 25, 26 only by -(f^c_j - f_k) u_b per link, so a sphere whose surface
is at rest gets bit for bit the paper's load, while a moving one gets a
different load.

The extra term is pinned through the fluid's mass balance: the bounce-back
of a moving surface creates the mass f_k - f^c_j on each cut link, and
nothing else in a step changes the fluid mass of a fully periodic box
(collision and streaming conserve it) unless a node changes owner.  For a
sphere in pure translation every link has u_b = V, so on a step without
owner changes the Galilean force minus the paper's is V times the fluid
mass gained, a total read from the populations alone.

The rotational part and the torque are pinned on the first step of a sphere
spinning in place in a fully periodic box at rest: every post-collision
population is then exactly w (the rest state collides into itself), the
populations after the step's streaming come from the oracle's stream alone,
and the test forms -sum (w_j - f_k(x, t+1)) u_b and -sum (w_j - f_k) (l x u_b)
itself from the oracle's link list (node, direction, q), with
u_b = Omega x l and l = x + q c_j - X at the image nearest to the centre:
they equal the Galilean force and torque minus the paper's to rounding.
"""
import numpy as np

import oracle

KW = dict(tau0=0.7, cs=0.17, g=(3e-5, 0.0, 0.0), u_hi=(0.03, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8,
          dem_substeps=16)
X = np.array([[9.3, 10.6, 8.2], [20.7, 9.1, 9.4]])
R = np.array([3.2, 2.7])


def run(mea, V, Om, fixed):
    o = oracle.Oracle(28, 20, 18, mea=mea, **KW)
    o.set_particles(X, V=V, Om=Om, R=R, fixed=fixed)
    o.step(20)
    return o.forces(), o.populations()


def test_resting_surfaces_get_the_papers_load():
    z = np.zeros((2, 3))
    fixed = np.ones(2, dtype=np.uint8)
    (Fa, Ta), fa = run("paper", z, z, fixed)
    (Fb, Tb), fb = run("galilean", z, z, fixed)
    assert np.array_equal(Fa, Fb) and np.array_equal(Ta, Tb) and np.array_equal(fa, fb)
    assert np.abs(Fa).max() > 0.0


def test_moving_surfaces_get_a_different_load():
    V = np.array([[0.02, -0.01, 0.0], [-0.01, 0.0, 0.01]])
    Om = np.array([[0.0, 0.0, 0.004], [0.003, 0.0, 0.0]])
    fixed = np.ones(2, dtype=np.uint8)  # prescribed motion: same trajectories, loads compared
    (Fa, Ta), fa = run("paper", V, Om, fixed)
    (Fb, Tb), fb = run("galilean", V, Om, fixed)
    assert np.array_equal(fa, fb)  # the populations do not depend on how the load is summed
    d = np.abs(Fb - Fa).max() / np.abs(Fa).max()
    assert 1e-8 < d < 0.2, d


def _sheared_equilibrium(shape):
    """Populations of a smooth flow (second-order equilibrium written out
    here), so that the fluid moves against the sphere in every direction."""
    nx, ny, nz = shape
    c, w, _ = oracle.tables()
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = np.stack([0.01 * np.sin(2 * np.pi * yy / ny), 0.008 * np.cos(2 * np.pi * zz / nz),
                  0.006 * np.sin(2 * np.pi * xx / nx)])
    rho = 1.0 + 0.002 * np.cos(2 * np.pi * (xx / nx + zz / nz))
    cu = np.einsum("ia,azyx->izyx", c.astype(np.float64), u)
    return w[:, None, None, None] * rho * (1.0 + 3.0 * cu + 4.5 * cu ** 2 - 1.5 * (u * u).sum(0))


def test_extra_force_of_a_translating_sphere_is_its_velocity_times_the_created_mass():
    shape = (24, 22, 20)
    f0 = _sheared_equilibrium(shape)
    strong = 0  # steps where the extra term stands far above the rounding
    for V in (np.array([0.004, -0.0025, 0.0015]), np.array([0.02, 0.01, -0.015])):
        runs = []
        for mea in ("paper", "galilean"):
            o = oracle.Oracle(*shape, tau0=0.7, cs=0.17, g=(1e-5, 0.0, 0.0), periodic_z=True, mea=mea)
            o.set_populations(f0)
            o.set_particles(np.array([[11.3, 10.7, 9.6]]), V=V[None], R=np.array([3.3]),
                            fixed=np.ones(1, dtype=np.uint8))  # prescribed translation, no spin
            runs.append(o)
        a, b = runs
        for _ in range(30):
            own0 = a.owner()
            M0 = a.populations()[:, own0 < 0].sum()
            a.step(1)
            b.step(1)
            own1 = a.owner()
            if not np.array_equal(own0, own1):
                continue  # covered or refilled nodes move mass too
            M1 = a.populations()[:, own1 < 0].sum()
            dF = b.forces()[0][0] - a.forces()[0][0]
            # rounding of the two mass sums: ~N eps M per sum, times |V|
            tol = 64 * np.finfo(np.float64).eps * M0 * np.abs(V).max()
            assert np.abs(dF - V * (M1 - M0)).max() <= tol, (dF, V * (M1 - M0))
            strong += bool(np.abs(dF).max() > 1e3 * tol)
    assert strong >= 3


def test_extra_load_of_a_spinning_sphere_from_the_streamed_populations():
    c, w, opp = oracle.tables()
    nx, ny, nz = 24, 22, 20
    Xs = np.array([[11.3, 10.6, 9.8]])
    Om = np.array([[0.004, -0.007, 0.011]])
    out = {}
    for mea in ("paper", "galilean"):
        o = oracle.Oracle(nx, ny, nz, tau0=1.0, cs=0.0, periodic_z=True, mea=mea, rho_s=2.5)
        o.set_particles(Xs, V=np.zeros((1, 3)), Om=Om, R=np.array([4.1]), fixed=np.ones(1, dtype=np.uint8))
        o.step(1)
        out[mea] = (*o.forces(), o.populations().reshape(19, -1), o.links())
    Fp, Tp, f1, (node, d, q, _) = out["paper"]
    Fg, Tg = out["galilean"][:2]
    assert len(node) > 100
    dF, dT = np.zeros(3), np.zeros(3)
    for n, j, qj in zip(node, d, q):
        xi = np.array([n % nx, (n // nx) % ny, n // (nx * ny)], dtype=float)
        for a, L in enumerate((nx, ny, nz)):  # image nearest to the centre
            xi[a] -= L * np.round((xi[a] - Xs[0, a]) / L)
        l = xi + float(qj) * c[j] - Xs[0]
        ub = np.cross(Om[0], l)
        e = w[j] - f1[opp[j], n]  # f^c_j(x) - f_k(x, t+1)
        dF -= e * ub
        dT -= e * np.cross(l, ub)
    assert np.abs(dT).max() > 1e-4 and np.abs(dF).max() > 1e-4
    assert np.abs((Fg - Fp)[0] - dF).max() <= 1e-12
    assert np.abs((Tg - Tp)[0] - dT).max() <= 1e-12
