"""The differentiation form with its spheres free (the coupled oracle's
channel option, oracle/lbm_oracle.c), and how far the fixed-sphere gradient
that the library's adjoint computes is from the derivative of the
free-sphere objective.

Pins of the channel option:
* with the spheres held fixed it is the channel oracle (channel_oracle.c,
  written separately, pinned in test_oracle_channel.py): per-step plate drag
  and J agree to 1e-8 relative; the two differ only in FP32 (coupled) and
  FP64 (channel) link fractions and in summation order, so a wrong inlet or
  outlet equilibrium, a plate link counted with the wrong sign or step, or a
  collided boundary plane fails;
* free spheres of very large density (1e9) give the fixed-sphere objective:
  the momentum exchange moves them by ~1e-9 lattice units;
* the plate contact (Eq. 1 against the plate's halfway surface, the node
  box grown by 1/2): a sphere meeting a face head-on, or an edge along the
  diagonal, leaves along the contact normal with the normal restitution
  (DEM only, no fluid), which a wrong surface offset, normal or sign fails.

The report: central differences of the free-sphere J (Sect. 2.3, Eqs. 19,
21, 25, 26 and the DEM of Sect. 2.1 moving the spheres) against the
fixed-sphere tangent-linear gradient on a 48 x 20 x 24 channel with four
spheres, printed.  The central differences at relative steps 1e-4 and 1e-2
agree with each other far more closely than with the fixed-sphere gradient:
the gap is the sphere-motion part of the derivative, which the fixed-sphere
adjoint leaves out (switch events only add noise on top of it).  The
full-size numbers come from tests/golden/make_free_sphere_report.py and are
printed by the GPU adjoint test.
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

MEDIUM = dict(nx=48, ny=20, nz=24, tau0=0.6, cs=0.15, gx=2e-6, u_peak=0.04, plate_lo=(30, 5, 6),
              plate_hi=(31, 14, 17), steps=160, avg_from=81)


def medium_spheres():
    return inputs.channel_spheres(seed=inputs.SEED_BASE + 30, n=4, radius=2.5, box=(48, 20, 24), x_range=(6.0, 24.0))


def test_channel_option_with_fixed_spheres_is_the_channel_oracle():
    X, R = medium_spheres()
    ref = oracle.channel(**MEDIUM, X=X, R=R)
    fx = oracle.free_channel(**MEDIUM, X=X, R=R, free=False)
    scale = np.abs(ref["drag"]).max()
    assert np.abs(fx["drag"] - ref["drag"]).max() <= 1e-8 * scale
    assert abs(fx["J"] - ref["J"]) <= 1e-8 * abs(ref["J"])
    assert np.array_equal(fx["X"], X)


@pytest.mark.parametrize("case", ["face_x", "face_z", "edge"])
def test_plate_contact_restitution_along_the_contact_normal(case):
    R, v, e = 4.0, 0.02, 0.8
    r2 = np.sqrt(0.5)
    X0, V0 = {"face_x": ([19.5 - R - 0.05, 10.0, 20.0], [v, 0.0, 0.0]),
              "face_z": ([21.5, 10.0, 14.5 - R - 0.05], [0.0, 0.0, v]),
              "edge": ([19.5 - (R + 0.05) * r2, 10.0, 14.5 - (R + 0.05) * r2], [v * r2, 0.0, v * r2])}[case]
    o = oracle.Oracle(48, 24, 40, tau0=0.8, rho_s=2.5, kn=10.0, restitution=e, dem_substeps=32, fluid=False,
                      channel=dict(u_peak=0.0, plate_lo=(20, 5, 15), plate_hi=(23, 14, 24)))
    o.set_particles(np.array([X0]), V=np.array([V0]), R=[R])
    o.step(60)
    V = o.particles()[1][0]
    assert np.abs(V - (-e) * np.array(V0)).max() <= 1e-3 * v


def test_very_heavy_free_spheres_give_the_fixed_objective():
    X, R = medium_spheres()
    fx = oracle.free_channel(**MEDIUM, X=X, R=R, free=False)
    heavy = oracle.free_channel(**MEDIUM, X=X, R=R, free=True, rho_s=1e9)
    assert np.abs(heavy["X"] - X).max() < 1e-6
    assert abs(heavy["J"] - fx["J"]) <= 1e-8 * abs(fx["J"])
    light = oracle.free_channel(**MEDIUM, X=X, R=R, free=True)
    assert np.abs(light["X"] - X).max() > 1.0  # the flow carries spheres of density 2.5 downstream
    assert abs(light["J"] - fx["J"]) > 1e-3 * abs(fx["J"])


def test_report_fixed_sphere_gradient_against_free_sphere_differences():
    X, R = medium_spheres()
    names = ("u_peak", "gx", "cs")
    for k, name in enumerate(names):
        tl = oracle.channel(**MEDIUM, X=X, R=R, dtheta=np.eye(3)[k])["dJ"]
        fd = []
        for rel in (1e-4, 1e-2):
            h = rel * MEDIUM[name]
            jp = oracle.free_channel(**dict(MEDIUM, **{name: MEDIUM[name] + h}), X=X, R=R)["J"]
            jm = oracle.free_channel(**dict(MEDIUM, **{name: MEDIUM[name] - h}), X=X, R=R)["J"]
            fd.append((jp - jm) / (2 * h))
        gap = (fd[0] - tl) / abs(tl)
        print("%s: fixed-sphere gradient %.9g  free-sphere central differences %.9g (h 1e-4), %.9g (h 1e-2);"
              " relative discrepancy %.3g" % (name, tl, fd[0], fd[1], gap))
        # the discrepancy is the sphere-motion part of the derivative, not noise of the differences
        assert abs(fd[0] - fd[1]) < 0.25 * abs(fd[0] - tl)
