"""Tangential contact law (Eqs. 2, 3) on the GPU against the FP64 oracle,
whose dry pins (tests/test_oracle_friction.py) fix its behaviour.

The GPU keeps each contact's tangential displacement in FP32 and advances
the sub-steps in FP32 (as for the normal law), so loads agree with the
oracle to the FP32 level; the tolerances are the plain method's
(populations 1e-5, hydrodynamic forces 1e-4, identical owners) plus the
motion bounds a relative load error of 1e-4 implies, for the spins too
(spin error <= eps |T| / I t with T the total torque).
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
FORCE_TOL = 1e-4
KW = dict(tau0=0.6, cs=0.17, g=(2e-6, 0.0, 0.0), u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8,
          dem_substeps=16, kt=500.0, mu=0.3, restitution_t=0.6)


def lbm():
    from paper_1703_05158_gb300 import lbm as mod

    mod.load()
    return mod


def colliding(shape):
    """Spinning spheres with head-on and grazing pairs and two resting on
    the walls (the upper one under the moving lid)."""
    parts = inputs.polydisperse(shape, 12, (2.5, 4.5), seed=inputs.SEED_BASE + 70, vmax=0.02)
    extra_X = np.array([[20.0, 40.0, 30.0], [29.1, 41.5, 30.4], [44.0, 25.0, 3.45], [10.0, 10.0, shape[2] - 4.45],
                        [52.0, 12.0, 20.0], [52.0, 20.2, 21.0]])
    extra_V = np.array([[0.03, 0.0, 0.0], [-0.03, 0.0, 0.0], [0.02, 0.0, -0.01], [0.0, 0.0, 0.01],
                        [0.0, 0.02, 0.0], [0.0, -0.02, 0.0]])
    extra_W = np.array([[0.0, 0.0, 0.01], [0.0, 0.01, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0],
                        [0.005, 0.0, 0.0], [0.0, 0.0, -0.005]])
    extra_R = np.array([4.0, 4.2, 4.0, 4.0, 3.5, 3.8])
    keep = np.ones(len(parts["R"]), dtype=bool)
    for x, r in zip(extra_X, extra_R):
        d = parts["X"] - x
        d[:, :2] -= np.array(shape[:2]) * np.round(d[:, :2] / np.array(shape[:2]))
        keep &= np.linalg.norm(d, axis=1) > parts["R"] + r + 1.0
    n = int(keep.sum())
    return dict(X=np.vstack([parts["X"][keep], extra_X]), V=np.vstack([parts["V"][keep], extra_V]),
                Om=np.vstack([inputs.uniform_vectors(n, -3e-3, 3e-3, inputs.SEED_BASE + 71), extra_W]),
                R=np.concatenate([parts["R"][keep], extra_R]))


def place(o, p):
    o.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])


def test_friction_matches_the_oracle():
    shape = (64, 50, 40)
    p = colliding(shape)
    n = len(p["R"])
    lat = lbm().Lattice(*shape, max_particles=n, max_radius=5.0, **KW)
    orc = oracle.Oracle(*shape, **KW)
    for o in (lat, orc):
        place(o, p)
    torqued = False
    done = 0
    for k in (1, 9, 40, 50):
        lat.step(k)
        orc.step(k)
        done += k
        torqued |= bool(np.abs(orc.contact_torques()).max() > 0.0)
        assert np.array_equal(lat.owner(), orc.owner()), done
        fo, fg = orc.populations(), lat.populations()
        fluid = orc.owner() < 0
        assert float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max()) <= POP_TOL, done
        Fg, _ = lat.forces()
        Fo, To = orc.forces()
        ef = np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)
        assert ef.max() <= FORCE_TOL, (done, ef.max())
    assert torqued  # friction acted on some contact
    m = 2.5 * 4.0 / 3.0 * np.pi * p["R"] ** 3
    I = 0.4 * m * p["R"] ** 2
    Fo, To = orc.forces()
    a = np.linalg.norm(Fo + orc.contact_forces(), axis=1) / m
    al = np.linalg.norm(To + orc.contact_torques(), axis=1) / I
    (Xg, Vg, Wg), (Xo, Vo, Wo) = lat.particles(), orc.particles()
    assert np.abs(Xg - Xo).max() < FORCE_TOL * a.max() * done ** 2 / 2 + 1e-12
    assert np.abs(Vg - Vo).max() < FORCE_TOL * a.max() * done + 1e-14
    assert np.abs(Wg - Wo).max() < FORCE_TOL * al.max() * done + 1e-14


def test_sphere_sliding_on_the_wall_matches_the_oracle():
    """A sphere pressed on the lower wall by an external load, launched
    along it without spin: Coulomb sliding, then rolling, in a fluid."""
    shape = (48, 32, 24)
    R = 4.0
    m = 2.5 * 4.0 / 3.0 * np.pi * R ** 3
    g = 1e-2
    pen = m * g / 1e3
    kw = dict(KW, mu=0.05, u_hi=(0.0, 0.0, 0.0), g=(0.0, 0.0, 0.0))
    lat = lbm().Lattice(*shape, max_particles=1, max_radius=4.0, **kw)
    orc = oracle.Oracle(*shape, **kw)
    X = np.array([[20.0, 16.0, R - 0.5 - pen]])
    for o in (lat, orc):
        o.set_particles(X, V=np.array([[0.02, 0.0, 0.0]]), R=np.array([R]))
        o.set_load(F=np.array([[0.0, 0.0, -m * g]]))
    for k in (10, 30, 60):
        lat.step(k)
        orc.step(k)
    (_, Vg, Wg), (_, Vo, Wo) = lat.particles(), orc.particles()
    assert Wo[0, 1] > 0.0  # the contact spun it up
    assert abs(Vg[0, 0] - Vo[0, 0]) <= 1e-4 * abs(Vo[0, 0])
    assert abs(Wg[0, 1] - Wo[0, 1]) <= 1e-4 * abs(Wo[0, 1])


def test_batch_members_with_friction_are_bitwise_the_lattices_alone():
    L = lbm()
    shape = (64, 50, 40)
    p = colliding(shape)
    n = len(p["R"])
    cfgs = [dict(nx=shape[0], ny=shape[1], nz=shape[2], max_particles=n, max_radius=5.0, **KW),
            dict(nx=shape[0], ny=shape[1], nz=shape[2], max_particles=n, max_radius=5.0,
                 **dict(KW, kt=0.0, mu=0.0))]
    batch = L.Batch(cfgs)
    alone = [L.Lattice(**c) for c in cfgs]
    for o in list(batch.members) + alone:
        place(o, p)
    for k in (1, 2, 27):
        batch.step(k)
        for a in alone:
            a.step(k)
        batch.sync()
        for mbr, a in zip(batch.members, alone):
            assert np.array_equal(mbr.populations(), a.populations())
            for u, v in zip(mbr.particles(), a.particles()):
                assert np.array_equal(u, v)
    # the friction member really differs from the frictionless one
    assert not np.array_equal(batch.members[0].particles()[2], batch.members[1].particles()[2])
    batch.close()


def test_friction_parameters_are_checked():
    L = lbm()
    for bad in (dict(kt=-1.0), dict(mu=-0.1), dict(restitution_t=0.0), dict(restitution_t=1.5)):
        with pytest.raises(Exception):
            L.Lattice(32, 32, 16, tau0=0.6, max_particles=1, max_radius=4.0, **bad)


def test_full_size_dense_slurry_with_friction_sampled():
    """256^3 at the solid fraction 0.13 the production box names (8136
    spheres of radius 4) with friction, the launch configuration of
    bench.py --workload dense, two steps: geometry identical everywhere,
    forces of every sphere, populations at 200k sampled nodes, motion."""
    p = inputs.phi_matched_slurry()
    n = len(p["R"])
    assert abs(inputs.solid_fraction((256, 256, 256), p["R"]) - 0.13) < 1e-3
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16,
              kt=500.0, mu=0.3, restitution_t=0.6)
    lat = lbm().Lattice(256, 256, 256, max_particles=n, max_radius=4.0, **kw)
    orc = oracle.Oracle(256, 256, 256, **kw)
    for o in (lat, orc):
        place(o, p)
    lat.step(2)
    orc.step(2)
    assert np.array_equal(lat.owner(), orc.owner())
    Fg, _ = lat.forces()
    Fo, _ = orc.forces()
    # relative to max(|F_p|, median |F|): in a box this dense a few spheres
    # feel loads that cancel to 1e-3 of the typical one, below the FP32
    # level of their ~300 link terms (absolute errors stay ~1e-7 everywhere)
    no = np.linalg.norm(Fo, axis=1)
    assert (np.linalg.norm(Fg - Fo, axis=1) / np.maximum(no, np.median(no))).max() <= FORCE_TOL
    fo = orc.populations().reshape(19, -1)
    fg = lat.populations().reshape(19, -1)
    fluid = (orc.owner() < 0).reshape(-1)
    idx = np.flatnonzero(fluid)
    idx = idx[inputs.rng(5).choice(len(idx), 200000, replace=False)]
    assert (np.abs(fg[:, idx] - fo[:, idx]) / np.abs(fo[:, idx])).max() <= POP_TOL
    m = 2.5 * 4.0 / 3.0 * np.pi * p["R"] ** 3
    a = np.linalg.norm(Fo + orc.contact_forces(), axis=1) / m
    (Xg, Vg, _), (Xo, Vo, _) = lat.particles(), orc.particles()
    assert np.abs(Xg - Xo).max() < FORCE_TOL * a.max() * 2.0 + 1e-12
    assert np.abs(Vg - Vo).max() < FORCE_TOL * a.max() * 2.0 + 1e-14


@pytest.mark.parametrize("friction", [True, False])
def test_grid_and_cluster_dem_forms_agree(friction):
    """The DEM sub-steps on a cooperative grid (global exchange buffer,
    bounded grid barriers) and in one thread-block cluster (distributed
    shared memory) run the same per-sphere arithmetic: same results, and
    the grid form against the oracle."""
    shape = (64, 50, 40)
    p = colliding(shape)
    n = len(p["R"])
    kw = KW if friction else dict(KW, kt=0.0, mu=0.0)
    L = lbm()
    lats = [L.Lattice(*shape, max_particles=n, max_radius=5.0, dem_mode=m, **kw) for m in ("cluster", "grid")]
    orc = oracle.Oracle(*shape, **kw)
    for o in lats + [orc]:
        place(o, p)
    for k in (1, 9, 40):
        for o in lats + [orc]:
            o.step(k)
        a, b = lats
        for u, v in zip(a.particles(), b.particles()):
            assert np.allclose(u, v, rtol=1e-6, atol=1e-9)
        fo, fg = orc.populations(), b.populations()
        fluid = orc.owner() < 0
        assert np.array_equal(b.owner(), orc.owner())
        assert float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max()) <= POP_TOL
    print("grid vs cluster bitwise:", all(np.array_equal(u, v) for u, v in zip(lats[0].particles(), lats[1].particles())))
