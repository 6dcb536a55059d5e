"""The Galilean-invariant momentum exchange of the oracle (option
mea="galilean"; Wen, Zhang & Fang 2014, not in the paper).  It differs from
Eqs. 25, 26 only by -(f^c_j - f_k) u_b per link, so a sphere whose surface
is at rest gets bit for bit the paper's load, while a moving one gets a
different load.  Beyond this reduction the option is parity unpinned: no
closed form or invariant of this suite fixes the extra term.
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
