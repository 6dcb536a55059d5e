"""Precision form: populations stored as deviations f - w in BF16 or FP16
(arithmetic FP32), against the FP64 oracle on the same seeded inputs.

Relative velocity error is ||u - u_64|| / ||u_64|| (L2 over nodes fluid on
both sides) after 200 steps; the bound is 1e-3 for both 16-bit
forms.  FP16 storage (11-bit significand) meets it (measured ~5e-4).  BF16
storage (8-bit significand) rounds each deviation to ~0.4%, and in these
low-viscosity (tau0 = 0.51) flows the rounding noise is weakly damped: it
measures ~4e-3 and does not meet 1e-3, so its cases are strict expected
failures (a pass would flag that the bound or the storage changed).
Spheres move with the slightly different loads, so a node near a surface
may change owner.

At full size (512 x 256 x 256) the oracle is too slow, so the 16-bit paths
are compared with the FP32 path instead.  By the triangle inequality
||u_16 - u_32|| <= ||u_16 - u_64|| + ||u_32 - u_64||, so a 16-bit path that
meets 1e-3 against FP64 differs from the FP32 path by at most 1e-3 plus the
FP32 path's own error against FP64, which test_fp32_velocity_error_against_
fp64 bounds by FP32_VEL_TOL = 1e-4 (measured ~8e-5) on the same physics.
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu

VEL_TOL = {"bf16": 1e-3, "fp16": 1e-3}
FP32_VEL_TOL = 1e-4
BF16_MISSES = pytest.mark.xfail(strict=True, reason="BF16 storage measures ~4e-3 (5e-3 against FP32 at full "
                                                    "size), above the 1e-3 bound")
PRECISIONS = [pytest.param("bf16", marks=BF16_MISSES), "fp16"]


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


@pytest.mark.parametrize("precision", PRECISIONS)
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


@pytest.mark.parametrize("precision", PRECISIONS)
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


def test_fp32_velocity_error_against_fp64():
    """The FP32 path's own relative velocity error against the FP64 oracle
    on the sheared box of the production physics (64 x 48 x 40, 12 spheres,
    tau0 = 0.51, 200 steps): the FP32 term of the full-size bound below."""
    shape = (64, 48, 40)
    parts = inputs.slurry_box(box=shape, n=12, radius=4.0, seed=inputs.SEED_BASE + 4)
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = _pair(shape, parts, "fp32", **kw)
    lat.step(200)
    orc.step(200)
    l2, mx = _vel_error(lat, orc)
    print("fp32: relative velocity error L2 %.2e, max %.2e" % (l2, mx))
    assert l2 <= FP32_VEL_TOL


_FULL = {}


def _full_size_fields(variant, prec):
    """Velocity and owners of the precision workload at full size after 100
    steps (cached per variant and storage)."""
    from paper_1703_05158_gb300 import lbm

    key = (variant, prec)
    if key not in _FULL:
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
        lat = lbm.Lattice(*shape, precision=prec, max_particles=n, max_radius=6.0, **kw)
        lat.set_particles(parts["X"], V=parts["V"], R=parts["R"])
        lat.step(100)
        _FULL[key] = (lat.fields()[1], lat.owner())
        lat.close()
    return _FULL[key]


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("variant", ["4000_spheres", "phi_matched_friction"])
def test_full_precision_workload_against_the_fp32_path(variant, precision):
    """The precision workload at full size: a 512 x 256 x 256 channel with
    walls in z, body force 5e-6, Cs 0.17, tau0 0.51 and 4000 spheres with
    radii uniform in [3, 6] (solid fraction 0.051), or the count that gives
    the solid fraction 0.10 it names (7911) with tangential friction; 100
    steps in 16-bit storage against the FP32 path on the same inputs
    (relative L2 velocity difference over nodes fluid in both), bounded by
    VEL_TOL + FP32_VEL_TOL (module docstring)."""
    u32, own32 = _full_size_fields(variant, "fp32")
    u16, own16 = _full_size_fields(variant, precision)
    fluid = (own16 < 0) & (own32 < 0)
    a, b = u16[:, fluid].astype(np.float64), u32[:, fluid].astype(np.float64)
    err = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    print("%s vs fp32 at 512x256x256, %s: relative velocity difference %.2e" % (precision, variant, err))
    assert err <= VEL_TOL[precision] + FP32_VEL_TOL
