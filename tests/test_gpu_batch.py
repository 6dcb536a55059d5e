"""Batched form: members of a batch, stepped together by graph replays of
the batched kernels, against the same simulations stepped alone (bitwise:
the batched kernels run the same per-node and per-sphere code) and one
member against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu


def lbm():
    from paper_1703_05158_gb300 import lbm as mod

    mod.load()
    return mod


def small_sweep():
    """Four uneven boxes, one without spheres, different tau0 / Cs / g."""
    cases = [
        ((48, 40, 36), 6, (3.0, 4.0), dict(tau0=0.55, cs=0.15, g=(4e-6, 0.0, 0.0))),
        ((64, 48, 40), 0, None, dict(tau0=0.7, cs=0.1, g=(1e-5, 0.0, 0.0), u_hi=(0.03, 0.0, 0.0))),
        ((40, 56, 44), 10, (2.0, 5.0), dict(tau0=0.6, cs=0.2, g=(2e-6, 0.0, 0.0))),
        ((56, 48, 48), 3, (4.0, 5.0), dict(tau0=0.51, cs=0.17, g=(6e-6, 0.0, 0.0), u_hi=(0.05, 0.0, 0.0))),
    ]
    out = []
    for k, (box, n, rr, kw) in enumerate(cases):
        parts = inputs.polydisperse(box, n, rr, seed=inputs.SEED_BASE + 40 + k, vmax=0.02) if n else None
        kw = dict(kw, rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16, max_particles=max(n, 1), max_radius=5.0)
        out.append((box, kw, parts))
    return out


def configs(sweep):
    return [dict(nx=b[0], ny=b[1], nz=b[2], **kw) for b, kw, _ in sweep]


def place(lat, parts):
    if parts is not None:
        lat.set_particles(parts["X"], V=parts["V"], R=parts["R"])


def test_batch_is_bitwise_the_members_stepped_alone():
    L = lbm()
    sweep = small_sweep()
    batch = L.Batch(configs(sweep))
    alone = [L.Lattice(*box, **kw) for box, kw, _ in sweep]
    for m, a, (_, _, parts) in zip(batch.members, alone, sweep):
        place(m, parts)
        place(a, parts)
    tpb, grid, ms = batch.tune()
    assert tpb in (128, 256, 512) and grid >= 1 and ms >= 0.0
    for n in (1, 2, 27):  # both graph parities, odd counts
        batch.step(n)
        for a in alone:
            a.step(n)
        batch.sync()
        for m, a in zip(batch.members, alone):
            assert np.array_equal(m.owner(), a.owner())
            assert np.array_equal(m.populations(), a.populations())
            if m.np:
                Fm, Tm = m.forces()
                Fa, Ta = a.forces()
                assert np.array_equal(Fm, Fa) and np.array_equal(Tm, Ta)
                for u, v in zip(m.particles(), a.particles()):
                    assert np.array_equal(u, v)
    for m, a in zip(batch.members, alone):
        assert m.info()["links"] == a.info()["links"]
    batch.close()


def test_batch_member_matches_oracle():
    L = lbm()
    sweep = small_sweep()
    batch = L.Batch(configs(sweep))
    box, kw, parts = sweep[0]
    okw = {k: v for k, v in kw.items() if k not in ("max_particles", "max_radius")}
    orc = oracle.Oracle(*box, **okw)
    for m, (_, _, p) in zip(batch.members, sweep):
        place(m, p)
    orc.set_particles(parts["X"], V=parts["V"], R=parts["R"])
    batch.step(60)
    orc.step(60)
    m = batch.members[0]
    assert np.array_equal(m.owner(), orc.owner())
    fo, fg = orc.populations(), m.populations()
    fluid = orc.owner() < 0
    assert float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max()) <= 1e-5
    Fg, _ = m.forces()
    Fo, _ = orc.forces()
    assert float((np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)).max()) <= 1e-4
    batch.close()


def test_batch_rules():
    L = lbm()
    sweep = small_sweep()[:2]
    batch = L.Batch(configs(sweep))
    for m, (_, _, p) in zip(batch.members, sweep):
        place(m, p)
    with pytest.raises(L.LbmError):
        L.lbm_step(batch.members[0].h, 1)  # members step only with their batch
    with pytest.raises(L.LbmError):
        L.lbm_destroy(batch.members[0].h)
    batch.step(1)
    place(batch.members[0], sweep[0][2])  # resets member 0 to step 0: parities differ
    with pytest.raises(L.LbmError):
        batch.step(1)
    batch.members[1].set_particles(np.zeros((0, 3)), R=np.zeros(0))  # member 1 back to step 0 as well
    batch.step(2)
    batch.sync()
    assert batch.members[0].info()["steps"] == 2
    batch.close()


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_batch_is_bitwise_the_members_alone_in_16_bit_storage(precision):
    L = lbm()
    sweep = small_sweep()[:3]
    cfgs = [dict(c, precision=precision) for c in configs(sweep)]
    batch = L.Batch(cfgs)
    alone = [L.Lattice(*box, precision=precision, **kw) for box, kw, _ in sweep]
    for m, a, (_, _, parts) in zip(batch.members, alone, sweep):
        place(m, parts)
        place(a, parts)
    batch.step(5)
    for a in alone:
        a.step(5)
    batch.sync()
    for m, a in zip(batch.members, alone):
        assert np.array_equal(m.populations(), a.populations())
    batch.close()


def test_full_sweep_batch_members_match_standalone_runs():
    """The 64-instance sweep (70 M nodes, ~22,700 spheres): 6 batched steps;
    the smallest and the largest member and one without spheres, if any,
    against the same simulations stepped alone, bitwise."""
    L = lbm()
    inst = inputs.batch_instances(count=64)
    cfgs = [dict(nx=i["box"][0], ny=i["box"][1], nz=i["box"][2], **i["params"]) for i in inst]
    batch = L.Batch(cfgs)
    for m, i in zip(batch.members, inst):
        if len(i["parts"]["R"]):
            place(m, i["parts"])
    batch.step(6)
    batch.sync()
    sizes = [int(np.prod(i["box"])) for i in inst]
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    pick |= {k for k, i in enumerate(inst) if len(i["parts"]["R"]) == 0}
    for k in sorted(pick)[:3]:
        a = L.Lattice(*inst[k]["box"], **inst[k]["params"])
        if len(inst[k]["parts"]["R"]):
            place(a, inst[k]["parts"])
        a.step(6)
        m = batch.members[k]
        assert np.array_equal(m.populations(), a.populations())
        if m.np:
            assert np.array_equal(m.forces()[0], a.forces()[0])
        a.close()
    batch.close()


@pytest.mark.parametrize("box,precision", [((520, 14, 10), "fp32"), ((301, 14, 12), "bf16")])
def test_rows_of_several_blocks_bitwise(box, precision):
    """Rows longer than one block of the single-instance collide (256-node
    row segments, the last one ragged; odd nx takes the one-node kernel in
    16-bit storage) against the batched kernels, which walk the nodes in
    flat chunks, bitwise, with spheres across the segment joints and the
    periodic seam, and a moving lid."""
    L = lbm()
    nx, ny, nz = box
    far = 511.3 if nx > 512 else nx - 6.0  # a third joint, else a sphere near the row's end
    X = np.array([[255.6, ny / 2, nz / 2], [1.2, ny / 2 - 0.3, nz / 2 + 0.4], [far, ny / 2 + 0.2, nz / 2 - 0.3]])
    V = np.tile([[0.02, -0.005, 0.003]], (len(X), 1))
    R = np.full(len(X), 3.0)
    kw = dict(tau0=0.6, cs=0.15, g=(3e-6, 0.0, 0.0), u_hi=(0.03, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8,
              dem_substeps=16, max_particles=len(X), max_radius=3.0, precision=precision)
    batch = L.Batch([dict(nx=nx, ny=ny, nz=nz, **kw)])
    alone = L.Lattice(nx, ny, nz, **kw)
    for lat in (batch.members[0], alone):
        lat.set_particles(X, V=V, R=R)
    for n in (1, 2, 7):
        batch.step(n)
        alone.step(n)
        batch.sync()
        m = batch.members[0]
        assert np.array_equal(m.owner(), alone.owner())
        assert np.array_equal(m.populations(), alone.populations())
        assert np.array_equal(m.forces()[0], alone.forces()[0])
    alone.close()
    batch.close()


def test_small_box_beside_a_large_sphere_member_bitwise():
    """A 20 x 20 box with spheres up to radius 4 (its own link tile 2 (4 + 2)
    + 1 = 13 nodes wide, 15 with the wrap margin) batched with a member of
    radius-8 spheres (tile 21 nodes, wider than the small box): every link
    CTA scans its own sphere's tile, so the small member is accepted and
    both step bitwise as alone."""
    L = lbm()
    kw = dict(tau0=0.7, cs=0.12, g=(2e-6, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    cases = [((20, 20, 16), 4.0, np.array([[5.2, 6.1, 7.3], [14.6, 13.8, 8.4]]), np.array([3.5, 4.0])),
             ((64, 64, 32), 8.0, np.array([[20.3, 30.2, 15.6], [45.1, 33.7, 16.2]]), np.array([7.0, 8.0]))]
    cfgs = [dict(nx=b[0], ny=b[1], nz=b[2], max_particles=2, max_radius=r, **kw) for b, r, _, _ in cases]
    batch = L.Batch(cfgs)
    alone = [L.Lattice(*b, max_particles=2, max_radius=r, **kw) for b, r, _, _ in cases]
    V = np.array([[0.01, -0.004, 0.002], [-0.006, 0.003, -0.001]])
    for m, a, (_, _, X, R) in zip(batch.members, alone, cases):
        m.set_particles(X, V=V, R=R)
        a.set_particles(X, V=V, R=R)
    for n in (1, 2, 9):
        batch.step(n)
        for a in alone:
            a.step(n)
        batch.sync()
        for m, a in zip(batch.members, alone):
            assert np.array_equal(m.owner(), a.owner())
            assert np.array_equal(m.populations(), a.populations())
            assert np.array_equal(m.forces()[0], a.forces()[0])
    for a in alone:
        a.close()
    batch.close()
