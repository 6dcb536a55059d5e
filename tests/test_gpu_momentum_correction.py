"""Optional covered / uncovered-node momentum correction (Aidun, Lu & Ding
1998; the paper itself uses none) on the GPU, against the FP64 oracle that
the CPU suite pins by exact conservation of total momentum.

A node covered by a moving sphere hands its momentum sum_i c_i f_i to the
sphere; a node it uncovers takes an equilibrium whose momentum rho u_s the
sphere pays.  Both join the momentum-exchange load of the same step.  The
tolerances are the plain method's: populations 1e-5, forces 1e-4 relative,
identical node ownership, and the motion bounds those loads imply.
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
FORCE_TOL = 1e-4
KW = dict(tau0=0.6, cs=0.17, g=(3e-6, 0.0, 0.0), u_hi=(0.04, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8,
          dem_substeps=16)


def lbm():
    from paper_1703_05158_gb300 import lbm as mod

    mod.load()
    return mod


def suspension(shape=(48, 40, 36), n=10, seed=inputs.SEED_BASE + 60):
    """Fast, spinning spheres: nodes are covered and uncovered every step."""
    p = inputs.polydisperse(shape, n, (2.5, 4.5), seed=seed, vmax=0.05)
    p["Om"] = inputs.uniform_vectors(n, -5e-3, 5e-3, seed + 1)
    return p


def place(o, p):
    o.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])


def test_correction_matches_the_oracle():
    shape = (48, 40, 36)
    p = suspension(shape)
    lat = lbm().Lattice(*shape, max_particles=len(p["R"]), max_radius=5.0, momentum_correction=True, **KW)
    orc = oracle.Oracle(*shape, momentum_correction=True, **KW)
    plain = oracle.Oracle(*shape, **KW)
    for o in (lat, orc, plain):
        place(o, p)
    done, moved = 0, 0.0
    for n in (1, 1, 8, 40, 50):
        lat.step(n)
        orc.step(n)
        done += n
        if done <= 2:  # the spheres first move in the DEM of step 1: step 2 covers nodes
            plain.step(1)
            Fp, _ = plain.forces()
            Fo, _ = orc.forces()
            moved = max(moved, float(np.abs(Fo - Fp).max() / np.abs(Fo).max()))
        assert np.array_equal(lat.owner(), orc.owner()), done
        fo, fg = orc.populations(), lat.populations()
        fluid = orc.owner() < 0
        assert float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max()) <= POP_TOL, done
        Fg, Tg = lat.forces()
        Fo, To = orc.forces()
        ef = np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)
        dt = np.linalg.norm(Tg - To, axis=1)
        assert ef.max() <= FORCE_TOL, (done, ef.max())
        assert np.all((dt <= 1e-3 * np.linalg.norm(To, axis=1)) | (dt < 1e-7)), (done, dt, To)
    # the correction is a large part of the step-2 load (else this test
    # would not see it)
    assert moved > 100 * FORCE_TOL, moved
    F, _ = orc.forces()
    a = np.linalg.norm(F, axis=1) / (2.5 * 4.0 / 3.0 * np.pi * p["R"] ** 3)
    Xg, Vg, _ = lat.particles()
    Xo, Vo, _ = orc.particles()
    assert np.abs(Xg - Xo).max() < FORCE_TOL * a.max() * done ** 2 / 2 + 1e-12
    assert np.abs(Vg - Vo).max() < FORCE_TOL * a.max() * done + 1e-14


def test_correction_of_fixed_spheres_is_exactly_zero():
    """Fixed spheres cover and uncover nothing: the correction adds exact
    zeros, so the run is bitwise the uncorrected one."""
    shape = (40, 36, 32)
    p = suspension(shape, n=6, seed=inputs.SEED_BASE + 62)
    L = lbm()
    lats = [L.Lattice(*shape, max_particles=6, max_radius=5.0, momentum_correction=c, **KW) for c in (False, True)]
    for lat in lats:
        lat.set_particles(p["X"], V=np.zeros_like(p["X"]), R=p["R"], fixed=np.ones(6, dtype=np.uint8))
        lat.step(25)
    a, b = lats
    assert np.array_equal(a.populations(), b.populations())
    for u, v in zip(a.forces(), b.forces()):
        assert np.array_equal(u, v)


def test_batch_member_with_correction_is_bitwise_the_lattice_alone():
    L = lbm()
    shapes = [(48, 40, 36), (40, 44, 32)]
    parts = [suspension(s, n=8, seed=inputs.SEED_BASE + 64 + k) for k, s in enumerate(shapes)]
    cfgs = [dict(nx=s[0], ny=s[1], nz=s[2], max_particles=8, max_radius=5.0, momentum_correction=True, **KW)
            for s in shapes]
    batch = L.Batch(cfgs)
    alone = [L.Lattice(**c) for c in cfgs]
    for m, a, p in zip(batch.members, alone, parts):
        place(m, p)
        place(a, p)
    for n in (1, 2, 17):
        batch.step(n)
        for a in alone:
            a.step(n)
        batch.sync()
        for m, a in zip(batch.members, alone):
            assert np.array_equal(m.populations(), a.populations())
            for u, v in zip(m.forces(), a.forces()):
                assert np.array_equal(u, v)
            for u, v in zip(m.particles(), a.particles()):
                assert np.array_equal(u, v)
    batch.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_correction_with_16_bit_storage(precision):
    """16-bit deviation storage rounds each population to about 4e-3 of its
    deviation; the covered-node momentum sums those values, so the loads
    follow the FP32 path within the storage's own velocity error."""
    shape = (48, 40, 36)
    p = suspension(shape)
    L = lbm()
    ref = L.Lattice(*shape, max_particles=len(p["R"]), max_radius=5.0, momentum_correction=True, **KW)
    low = L.Lattice(*shape, max_particles=len(p["R"]), max_radius=5.0, momentum_correction=True,
                    precision=precision, **KW)
    for lat in (ref, low):
        place(lat, p)
        lat.step(20)
    Fr, _ = ref.forces()
    Fl, _ = low.forces()
    assert np.abs(Fl - Fr).max() <= 2e-2 * np.abs(Fr).max()


@pytest.mark.parametrize("corr", [False, True])
def test_galilean_invariant_exchange_matches_the_oracle(corr):
    """The Galilean-invariant momentum exchange (Wen, Zhang & Fang 2014),
    alone and with the covered / uncovered correction, against the oracle.
    The oracle's extra term is pinned in test_oracle_mea.py: its force on a
    translating sphere (the fluid mass the moving bounce-back creates) and
    its force and torque on a sphere spinning in place (formed from the
    streamed populations and the link list)."""
    shape = (48, 40, 36)
    p = suspension(shape, seed=inputs.SEED_BASE + 66)
    lat = lbm().Lattice(*shape, max_particles=len(p["R"]), max_radius=5.0, momentum_correction=corr,
                        mea="galilean", **KW)
    orc = oracle.Oracle(*shape, momentum_correction=corr, mea="galilean", **KW)
    for o in (lat, orc):
        place(o, p)
    done = 0
    for n in (1, 9, 40, 50):
        lat.step(n)
        orc.step(n)
        done += n
        assert np.array_equal(lat.owner(), orc.owner()), done
        fo, fg = orc.populations(), lat.populations()
        fluid = orc.owner() < 0
        assert float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max()) <= POP_TOL, done
        Fg, Tg = lat.forces()
        Fo, To = orc.forces()
        ef = np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)
        dt = np.linalg.norm(Tg - To, axis=1)
        assert ef.max() <= FORCE_TOL, (done, ef.max())
        assert np.all((dt <= 1e-3 * np.linalg.norm(To, axis=1)) | (dt < 1e-7)), (done, dt, To)
