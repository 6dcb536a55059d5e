"""Precision form: populations stored as deviations f - w in BF16 or FP16
(arithmetic FP32), against the FP64 oracle on the same seeded inputs.

Relative velocity error is ||u - u_64|| / ||u_64|| (L2 over nodes fluid on
both sides) after 200 steps.  FP16 storage (11-bit significand) meets 1e-3
(measured ~5e-4).  BF16 storage (8-bit significand) rounds each deviation to
~0.4%, and in these low-viscosity (tau0 = 0.51) flows the rounding noise
is weakly damped: measured ~4e-3, bounded here at 1e-2.  Spheres move with
the slightly different loads, so a node near a surface may change owner.
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu

VEL_TOL = {"bf16": 1e-2, "fp16": 1e-3}


def _pair(shape, parts, precision, **kw):
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    lat = lbm.Lattice(*shape, precision=precision, max_particles=max(len(parts["R"]), 1), max_radius=6.0, **kw)
    orc = oracle.Oracle(*shape, **kw)
    for o in (lat, orc):
        o.set_particles(parts["X"], V=parts["V"], R=parts["R"])
    return lat, orc


def _vel_error(lat, orc):
    _, ug = lat.fields()
    _, uo = orc.fields()
    fluid = (orc.owner() < 0) & (lat.owner() < 0)
    a, b = ug[:, fluid].astype(np.float64), uo[:, fluid]
    return float(np.linalg.norm(a - b) / np.linalg.norm(b)), float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_channel_with_polydisperse_spheres(precision):
    """Body-force channel between walls with spheres of radius 3-6 (the
    precision workload's sphere mix) on a 64^3 sub-box, 200 steps."""
    shape = (64, 64, 64)
    parts = inputs.polydisperse(shape, 24, (3.0, 6.0), seed=inputs.SEED_BASE + 3)
    kw = dict(tau0=0.51, cs=0.17, g=(5e-6, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = _pair(shape, parts, precision, **kw)
    lat.step(200)
    orc.step(200)
    l2, mx = _vel_error(lat, orc)
    print("%s: relative velocity error L2 %.2e, max %.2e" % (precision, l2, mx))
    assert l2 <= VEL_TOL[precision]


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_sheared_box_with_spheres(precision):
    """Sliding lid, Smagorinsky, moving spheres (the production physics) on
    a 64 x 48 x 40 box, 200 steps."""
    shape = (64, 48, 40)
    parts = inputs.slurry_box(box=shape, n=12, radius=4.0, seed=inputs.SEED_BASE + 4)
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = _pair(shape, parts, precision, **kw)
    lat.step(200)
    orc.step(200)
    l2, mx = _vel_error(lat, orc)
    print("%s: relative velocity error L2 %.2e, max %.2e" % (precision, l2, mx))
    assert l2 <= VEL_TOL[precision]
    Fg, _ = lat.forces()
    Fo, _ = orc.forces()
    # forces follow the velocity field; report their error
    print("%s: max relative force error %.2e" % (precision, float(
        (np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)).max())))


@pytest.mark.parametrize("variant", ["4000_spheres", "phi_matched_friction"])
def test_full_precision_workload_against_the_fp32_path(variant):
    """The precision workload at full size: a 512 x 256 x 256 channel with
    walls in z, body force 5e-6, Cs 0.17, tau0 0.51 and 4000 spheres with
    radii uniform in [3, 6] (solid fraction 0.051), or the count that gives
    the solid fraction 0.10 it names (7911) with tangential friction; 100
    steps in FP16 and BF16 storage against the FP32 path on the same inputs
    (relative L2 velocity difference over nodes fluid in both)."""
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    shape = (512, 256, 256)
    kw = dict(tau0=0.51, cs=0.17, g=(5e-6, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    if variant == "4000_spheres":
        n = 4000
        parts = inputs.polydisperse(shape, n, (3.0, 6.0), seed=inputs.SEED_BASE + 3)
    else:
        n = inputs.phi_matched_count(shape, 0.10, (3.0, 6.0))
        parts = inputs.polydisperse(shape, n, (3.0, 6.0), seed=inputs.SEED_BASE + 7)
        kw.update(kt=500.0, mu=0.3, restitution_t=0.6)
    u, own = {}, {}
    for prec in ("fp32", "fp16", "bf16"):
        lat = lbm.Lattice(*shape, precision=prec, max_particles=n, max_radius=6.0, **kw)
        lat.set_particles(parts["X"], V=parts["V"], R=parts["R"])
        lat.step(100)
        u[prec] = lat.fields()[1]
        own[prec] = lat.owner()
        lat.close()
    err = {}
    for prec in ("fp16", "bf16"):
        fluid = (own[prec] < 0) & (own["fp32"] < 0)
        a, b = u[prec][:, fluid].astype(np.float64), u["fp32"][:, fluid].astype(np.float64)
        err[prec] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print("%s vs fp32 at 512x256x256, %s: relative velocity difference %.2e" % (prec, variant, err[prec]))
    assert err["fp16"] <= VEL_TOL["fp16"]
    assert err["bf16"] <= VEL_TOL["bf16"]
