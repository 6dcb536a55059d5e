"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Tolerances: FP32 storage, per-population max relative error <= 1e-5 after
100 steps and per-sphere force within 1e-4 relative; node ownership must be
identical (both sides take the geometric decisions with the same FP32
operations).  Sphere centres and velocities are integrated in FP64 on both
sides from hydrodynamic loads that differ at the FP32 level; a relative load
error eps over t steps moves a sphere by at most eps a t^2 / 2 (a = |F|/m),
so centres must agree within 1e-5 a_max t^2 / 2 and velocities within
1e-5 a_max t.  Box sizes are deliberately not multiples of the 32-wide warp
or the block width, so every case has ragged rows.
"""
import numpy as np
import pytest

import oracle
from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu

POP_TOL = 1e-5
FORCE_TOL = 1e-4


def lbm():
    from paper_1703_05158_gb300 import lbm as mod

    mod.load()
    return mod


def make_pair(shape, parts=None, populations=None, precision="fp32", max_radius=4.0, **kw):
    nx, ny, nz = shape
    n = 0 if parts is None else len(parts["R"])
    lat = lbm().Lattice(nx, ny, nz, max_particles=max(n, 1), max_radius=max_radius, precision=precision, **kw)
    orc = oracle.Oracle(nx, ny, nz, **kw)
    if parts is not None:
        for o in (lat, orc):
            o.set_particles(parts["X"], V=parts["V"], Om=parts.get("Om"), R=parts["R"], fixed=parts.get("fixed"))
    if populations is not None:
        orc.set_populations(populations)
        lat.set_populations(orc.populations())
    return lat, orc


def perturbed(shape, amp, seed):
    c, w, _ = oracle.tables()
    eps = inputs.perturbation((19,) + tuple(reversed(shape)), amp, seed)
    return w[:, None, None, None] * (1.0 + eps)


def pop_error(lat, orc):
    fo = orc.populations()
    fg = lat.populations()
    fluid = orc.owner() < 0
    return float((np.abs(fg - fo)[:, fluid] / np.abs(fo[:, fluid])).max())


def force_error(lat, orc):
    Fg, Tg = lat.forces()
    Fo, To = orc.forces()
    ef = np.linalg.norm(Fg - Fo, axis=1) / np.linalg.norm(Fo, axis=1)
    et = np.linalg.norm(Tg - To, axis=1) / np.maximum(np.linalg.norm(To, axis=1), 1e-300)
    return float(ef.max()), float(et.max()), Fo, To


def motion_tolerance(orc, steps, rho_s=2.5):
    """Position and velocity bounds implied by the force tolerance: a relative
    load error eps = FORCE_TOL held over t steps moves a sphere by at most
    eps a t^2 / 2 and changes its velocity by at most eps a t (a = |F| / m)."""
    F, _ = orc.forces()
    _, _, _ = orc.particles()
    R = np.asarray(orc._keep[3])
    a = np.linalg.norm(F, axis=1) / (rho_s * 4.0 / 3.0 * np.pi * R ** 3)
    amax = float(a.max())
    return FORCE_TOL * amax * steps ** 2 / 2 + 1e-12, FORCE_TOL * amax * steps + 1e-14


def test_rest_state_is_exact():
    lat, _ = make_pair((37, 29, 23), tau0=0.7, cs=0.17)
    lat.step(50)
    c, w, _ = oracle.tables()
    f = lat.populations()
    assert np.array_equal(f, np.broadcast_to(w[:, None, None, None], f.shape))


def test_fluid_only_parity_walls_lid_force_smagorinsky():
    shape = (37, 29, 23)
    kw = dict(tau0=0.56, cs=0.17, g=(1e-5, 2e-6, 0.0), u_lo=(0.0, -0.01, 0.0), u_hi=(0.05, 0.01, 0.0))
    lat, orc = make_pair(shape, populations=perturbed(shape, 0.05, 101), **kw)
    lat.step(100)
    orc.step(100)
    assert pop_error(lat, orc) <= POP_TOL
    rg, ug = lat.fields()
    ro, uo = orc.fields()
    assert np.abs(rg - ro).max() < 1e-6
    assert np.abs(ug - uo).max() < 1e-7


def test_single_sphere_plain_method_200_steps():
    """One sphere of radius 4 at the centre of a 32^3 box moving at 0.01.
    Torque: within 1e-2 relative or 1e-7 absolute.  A sphere translating
    through the box centre feels a torque far below |F| R (it vanishes by
    symmetry but for the lattice), so a relative bound compares two numbers
    near the FP32 rounding level of the ~1000 link terms' moment sums; the
    absolute floor sits a few times above that level (2^-24 |F| R)."""
    p = inputs.sphere_in_box(32)
    kw = dict(tau0=0.8, cs=0.1, g=(1e-6, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = make_pair((32, 32, 32), parts=p, **kw)
    for n in (100, 100):
        lat.step(n)
        orc.step(n)
        assert np.array_equal(lat.owner(), orc.owner())
        assert pop_error(lat, orc) <= POP_TOL
        ef, et, Fo, _ = force_error(lat, orc)
        assert ef <= FORCE_TOL, (ef, Fo)
        assert et <= 1e-2 or np.abs(lat.forces()[1] - orc.forces()[1]).max() < 1e-7
    Xg, Vg, Wg = lat.particles()
    Xo, Vo, Wo = orc.particles()
    xt, vt = motion_tolerance(orc, 200)
    assert np.abs(Xg - Xo).max() < xt
    assert np.abs(Vg - Vo).max() < vt
    assert lat.info()["refilled"] >= 0


def test_many_spheres_moving_lid_contacts_periodic_edges():
    shape = (64, 50, 40)
    parts = inputs.polydisperse(shape, 20, (2.5, 4.5), seed=inputs.SEED_BASE + 11, vmax=0.02)
    # a head-on pair that collides within the run, one across the periodic x
    # edge, one close to the lower wall
    extra_X = np.array([[20.0, 40.0, 30.0], [29.3, 40.0, 30.0], [0.7, 10.0, 12.0], [44.0, 25.0, 4.2]])
    extra_V = np.array([[0.03, 0.0, 0.0], [-0.03, 0.0, 0.0], [-0.02, 0.01, 0.0], [0.0, 0.0, -0.02]])
    extra_R = np.array([4.0, 4.2, 3.0, 3.5])
    keep = np.ones(len(parts["R"]), dtype=bool)
    for x, r in zip(extra_X, extra_R):
        d = parts["X"] - x
        d[:, :2] -= np.array(shape[:2]) * np.round(d[:, :2] / np.array(shape[:2]))
        keep &= np.linalg.norm(d, axis=1) > parts["R"] + r + 1.0
    p = dict(X=np.vstack([parts["X"][keep], extra_X]), V=np.vstack([parts["V"][keep], extra_V]),
             Om=np.vstack([inputs.uniform_vectors(keep.sum(), -2e-3, 2e-3, 5), np.zeros((4, 3))]),
             R=np.concatenate([parts["R"][keep], extra_R]))
    kw = dict(tau0=0.6, cs=0.17, g=(2e-6, 0.0, 0.0), u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3,
              restitution=0.8, dem_substeps=16)
    lat, orc = make_pair(shape, parts=p, max_radius=5.0, **kw)
    touched = False
    for _ in range(10):
        lat.step(10)
        orc.step(10)
        touched |= bool(np.abs(orc.contact_forces()[-4:-2]).max() > 0.0)
    assert touched  # the head-on pair was in contact during the run
    assert np.array_equal(lat.owner(), orc.owner())
    assert pop_error(lat, orc) <= POP_TOL
    ef, et, Fo, To = force_error(lat, orc)
    assert ef <= FORCE_TOL, (ef, Fo)
    Xg, Vg, _ = lat.particles()
    Xo, Vo, _ = orc.particles()
    xt, vt = motion_tolerance(orc, 100)
    assert np.abs(Xg - Xo).max() < xt
    assert np.abs(Vg - Vo).max() < vt
    info = lat.info()
    node, _, _, _ = orc.links()
    assert info["links"] == len(node)
    assert info["fluid_nodes"] == int((orc.owner() < 0).sum())


def test_headline_physics_forces_until_the_first_switch_event():
    """The production physics (tau0 = 0.51, Cs = 0.17, lid 0.05, spheres of
    radius 4 at the 256^3 workload's density: 31 in a 64^3 sub-box).  After
    100 steps: populations within 1e-5, every sphere's force within 1e-4,
    identical owners.  Then step by step to 200: the force bound holds for as
    long as both sides have classified every node alike.  Both sides take
    the inside test in the same FP32 operations, but on centres that differ
    by the integrated effect of FP32-level load differences (~1e-6 here); a
    node that the surface crosses within that distance of a step boundary is
    covered or uncovered one step apart on the two sides (a switch event of
    the method), and the refill then differs locally by O(1e-2) of that
    sphere's load.  The oracle started from FP32-level perturbed populations
    (6e-8 relative) stays within 5e-6 of itself in force over 200 steps, so
    the departure is the switch event, not a growth of rounding noise."""
    shape = (64, 64, 64)
    p = inputs.slurry_box(box=shape, n=31, radius=4.0, seed=inputs.SEED_BASE + 8)
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = make_pair(shape, parts=p, **kw)
    # control: the oracle from rest populations perturbed at the FP32 level
    ctl = oracle.Oracle(*shape, **kw)
    ctl.set_particles(p["X"], V=p["V"], Om=p["Om"], R=p["R"])
    ctl.set_populations(perturbed(shape, 6e-8, 12345))
    lat.step(100)
    orc.step(100)
    ctl.step(100)
    assert np.array_equal(lat.owner(), orc.owner())
    pe = pop_error(lat, orc)
    ef, _, Fo, _ = force_error(lat, orc)
    print("tau0 = 0.51, 100 steps: populations %.2e, forces %.2e" % (pe, ef))
    assert pe <= POP_TOL
    assert ef <= FORCE_TOL, (ef, Fo)
    first_flip = None
    for s in range(101, 201):
        lat.step(1)
        orc.step(1)
        if first_flip is None and not np.array_equal(lat.owner(), orc.owner()):
            Xg, _, _ = lat.particles()
            Xo, _, _ = orc.particles()
            first_flip = s
            print("first switch event on one side only at step %d (centres differ by %.1e)" % (s, np.abs(Xg - Xo).max()))
        if first_flip is None:
            ef, _, Fo, _ = force_error(lat, orc)
            assert ef <= FORCE_TOL, (s, ef, Fo)
    print("forces within %.0e up to step %s" % (FORCE_TOL, first_flip - 1 if first_flip else 200))
    ctl.step(100)
    Fc, _ = ctl.forces()
    Fo, _ = orc.forces()
    self_div = float((np.linalg.norm(Fc - Fo, axis=1) / np.linalg.norm(Fo, axis=1)).max())
    print("control: oracle against its FP32-level perturbed copy after 200 steps: forces %.2e" % self_div)
    assert self_div <= 0.1 * FORCE_TOL


def test_mostly_far_nodes_overlapped_schedule():
    """A large box with a few spheres: most nodes are collided by the second
    stream while the link / DEM / geometry work runs; 100 steps must still
    match the oracle node for node.  (The centres differ from the oracle's
    by rounding, ~1e-6 after 100 steps, so over much longer runs a node
    right at a sphere surface can eventually fall on different sides.)"""
    shape = (96, 80, 72)
    p = inputs.polydisperse(shape, 5, (3.0, 4.5), seed=inputs.SEED_BASE + 21, vmax=0.03)
    kw = dict(tau0=0.55, cs=0.17, g=(3e-6, 0.0, 0.0), u_hi=(0.04, 0.0, 0.0), rho_s=2.5, kn=1e3,
              restitution=0.8, dem_substeps=16)
    lat, orc = make_pair(shape, parts=p, max_radius=5.0, **kw)
    for n in (1, 2, 47, 50):
        lat.step(n)
        orc.step(n)
        assert np.array_equal(lat.owner(), orc.owner())
        assert pop_error(lat, orc) <= POP_TOL
        ef, _, Fo, _ = force_error(lat, orc)
        assert ef <= FORCE_TOL, (ef, Fo)


@pytest.mark.parametrize("case", ["few_spheres_large_box", "dense_slurry"])
def test_overlapped_and_serial_schedules_are_bitwise_equal(case):
    """The far-node collisions on the second stream touch no location the
    link / refill / near-node work touches, so the overlapped schedule gives
    bitwise the serial schedule's populations, forces and motion."""
    if case == "few_spheres_large_box":
        shape = (96, 80, 72)
        p = inputs.polydisperse(shape, 5, (3.0, 4.5), seed=inputs.SEED_BASE + 21, vmax=0.03)
    else:
        shape = (64, 64, 48)
        p = inputs.slurry_box(box=shape, n=30, radius=4.0, seed=inputs.SEED_BASE + 22)
    kw = dict(tau0=0.55, cs=0.17, g=(3e-6, 0.0, 0.0), u_hi=(0.04, 0.0, 0.0), rho_s=2.5, kn=1e3,
              restitution=0.8, dem_substeps=16)
    L = lbm()
    lats = []
    for sched in ("overlap", "serial"):
        lat = L.Lattice(*shape, max_particles=len(p["R"]), max_radius=5.0, schedule=sched, **kw)
        lat.set_particles(p["X"], V=p["V"], R=p["R"])
        lats.append(lat)
    for n in (1, 2, 3, 60, 94):
        for lat in lats:
            lat.step(n)
        a, b = lats
        assert np.array_equal(a.owner(), b.owner())
        assert np.array_equal(a.populations(), b.populations())
        assert np.array_equal(a.forces()[0], b.forces()[0])
        for u, v in zip(a.particles(), b.particles()):
            assert np.array_equal(u, v)


def test_no_particles_and_capacity_errors():
    L = lbm()
    lat = L.Lattice(40, 40, 12, tau0=0.7, max_particles=2, max_radius=4.0)
    with pytest.raises(L.LbmError) as e:
        lat.set_particles(np.full((3, 3), 10.0), R=[3.0, 3.0, 3.0])
    assert e.value.code == L.LBM_ERR_CAPACITY
    with pytest.raises(L.LbmError) as e:
        lat.set_particles([[41.0, 10.0, 6.0]], R=[3.0])
    assert e.value.code == L.LBM_ERR_ARG
    lat.set_particles(np.zeros((0, 3)), R=np.zeros(0))
    lat.step(3)
    lat.sync()
    assert lat.info()["steps"] == 3


def test_exact_overlap_ties_match_the_oracle():
    """Mirror-image equal spheres: the nodes of the plane between them tie
    exactly (the same FP32 key from either centre) and go to the smaller
    index in the library as in the oracle, in either order, before and after
    a step."""
    R = 2.75
    for first, second in (((8.0, 8.5, 8.25), (12.0, 8.5, 8.25)), ((12.0, 8.5, 8.25), (8.0, 8.5, 8.25))):
        parts = dict(X=np.array([first, second]), V=np.zeros((2, 3)), R=np.array([R, R]),
                     fixed=np.array([1, 1], dtype=np.uint8))
        lat, orc = make_pair((22, 17, 16), parts=parts, tau0=0.8)
        assert np.array_equal(lat.owner(), orc.owner())
        assert ((orc.owner() == 0) & (np.arange(22)[None, None, :] == 10)).any()
        lat.step(1)
        orc.step(1)
        assert np.array_equal(lat.owner(), orc.owner())
        lat.close()


def test_largest_lattice_and_the_index_limit():
    """Populations are addressed with 32-bit element offsets: a box whose
    19 slot arrays (with the two wall planes and padding) reach 2^31
    elements is refused with LBM_ERR_UNSUPPORTED; the largest cube below the
    limit (480^3, 110.6 M nodes, 8.4 GB of FP32 populations) steps, and a
    rest state stays exactly at rest (its deviations are exactly zero)."""
    L = lbm()
    with pytest.raises(L.LbmError) as e:
        L.Lattice(512, 512, 512, tau0=0.7)
    assert e.value.code == L.LBM_ERR_UNSUPPORTED
    lat = L.Lattice(480, 480, 480, tau0=0.7, cs=0.17)
    lat.step(3)
    lat.sync()
    rho, u = lat.fields()
    assert np.all(rho == 1.0) and np.all(u == 0.0)
    lat.close()


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_odd_nx_takes_the_single_node_16_bit_kernel(precision):
    """nx odd: the 16-bit storage runs one node per thread (the pair kernel
    needs even rows); same tolerance as FP32 storage against the oracle on
    the rounding of one store, checked on velocities after 60 steps."""
    shape = (37, 29, 23)
    kw = dict(tau0=0.6, cs=0.17, g=(1e-5, 0.0, 0.0), u_hi=(0.04, 0.0, 0.0))
    lat = lbm().Lattice(*shape, precision=precision, **kw)
    orc = oracle.Oracle(*shape, **kw)
    lat.step(60)
    orc.step(60)
    ug = lat.fields()[1].astype(np.float64)
    uo = orc.fields()[1]
    err = float(np.linalg.norm(ug - uo) / np.linalg.norm(uo))
    print("%s, nx = 37: relative velocity error %.2e" % (precision, err))
    assert err <= (1e-3 if precision == "fp16" else 1e-2)


def test_mass_conservation_gpu():
    shape = (96, 64, 48)
    kw = dict(tau0=0.6, cs=0.17, u_hi=(0.05, 0.0, 0.0))
    lat, orc = make_pair(shape, populations=perturbed(shape, 0.02, 7), **kw)
    m0 = lat.populations().sum()
    lat.step(500)
    assert abs(lat.populations().sum() - m0) / m0 < 1e-7


@pytest.mark.slow
def test_full_size_slurry_box_sampled():
    """256^3 with 2000 spheres of radius 4, the benchmark's launch
    configuration, two steps: geometry identical everywhere, forces of every
    sphere, populations at 200k sampled nodes."""
    p = inputs.slurry_box()
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16)
    lat, orc = make_pair((256, 256, 256), parts=p, **kw)
    lat.step(2)
    orc.step(2)
    assert np.array_equal(lat.owner(), orc.owner())
    ef, _, Fo, _ = force_error(lat, orc)
    assert ef <= FORCE_TOL, ef
    fo = orc.populations().reshape(19, -1)
    fg = lat.populations().reshape(19, -1)
    fluid = (orc.owner() < 0).reshape(-1)
    idx = np.flatnonzero(fluid)
    idx = idx[inputs.rng(3).choice(len(idx), 200000, replace=False)]
    assert (np.abs(fg[:, idx] - fo[:, idx]) / np.abs(fo[:, idx])).max() <= POP_TOL


def test_full_size_slurry_with_every_option_sampled():
    """The benchmark box (256^3, 2000 spheres of radius 4) with every option
    of the extra bench lines at once: momentum correction, the
    Galilean-invariant exchange, tangential friction and a ZIEB face; three
    steps (spheres move, so nodes are covered and uncovered) against the
    oracle: geometry everywhere, every sphere's load, 200k sampled
    populations, the cylinder density."""
    p = inputs.slurry_box()
    A = 256.0 * 256.0
    zieb = dict(area=A, volume=40.0 * A, vp=0.005)
    kw = dict(tau0=0.51, cs=0.17, u_hi=(0.05, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16,
              kt=500.0, mu=0.3, restitution_t=0.6, momentum_correction=True, mea="galilean", zieb=zieb)
    lat = lbm().Lattice(256, 256, 256, max_particles=len(p["R"]), max_radius=4.0, **kw)
    orc = oracle.Oracle(256, 256, 256, **kw)
    for o in (lat, orc):
        o.set_particles(p["X"], V=p["V"], R=p["R"])
    lat.step(3)
    orc.step(3)
    assert np.array_equal(lat.owner(), orc.owner())
    ef, _, Fo, _ = force_error(lat, orc)
    assert ef <= FORCE_TOL, ef
    fo = orc.populations().reshape(19, -1)
    fg = lat.populations().reshape(19, -1)
    fluid = (orc.owner() < 0).reshape(-1)
    idx = np.flatnonzero(fluid)
    idx = idx[inputs.rng(7).choice(len(idx), 200000, replace=False)]
    assert (np.abs(fg[:, idx] - fo[:, idx]) / np.abs(fo[:, idx])).max() <= POP_TOL
    assert abs(lat.zieb_state()[0] - orc.zieb_state()[0]) <= 1e-6
