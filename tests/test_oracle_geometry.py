"""Pins of the oracle's geometry, link fractions and refill (Sect. 2.3).

Sphere centres are dyadic and the radius has few bits, so every FP32
distance below is exact and the oracle's FP32 decisions must equal exact
integer arithmetic.  Link fractions are compared with the root of the
quadratic in FP64.  The refill is checked node by node on a sphere shifted
by a prescribed motion.
"""
import itertools

import numpy as np
import pytest

import oracle

C = oracle.tables()[0]


def exact_inside(shape, X, R):
    """Brute force, exact rational test |x - X|^2 < R^2 (dyadic X, R), x,y periodic."""
    nz, ny, nx = shape
    den = 64
    Xi = [int(round(v * den)) for v in X]
    Ri = int(round(R * den))
    inside = np.zeros(shape, dtype=bool)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        d2 = 0
        for v, n, c, per in ((x, nx, Xi[0], True), (y, ny, Xi[1], True), (z, nz, Xi[2], False)):
            d = v * den - c
            if per:
                d = min((d + k * n * den for k in (-1, 0, 1)), key=abs)
            d2 += d * d
        inside[z, y, x] = d2 < Ri * Ri
    return inside


def test_node_count_of_centred_spheres():
    # integer points strictly inside a sphere centred on a node: sum of r3(n), n < R^2
    for R, count in ((3.0, 93), (4.0, 251)):
        brute = sum(1 for i, j, k in itertools.product(range(-5, 6), repeat=3) if i * i + j * j + k * k < R * R)
        assert brute == count
        o = oracle.Oracle(32, 32, 32, tau0=0.8)
        o.set_particles([[16.0, 16.0, 16.0]], R=[R])
        assert (o.owner() == 0).sum() == count


def test_solid_set_exact_off_lattice_and_across_periodic_edge():
    for X in ((15.25, 16.5, 9.75), (0.375, 19.625, 9.125)):
        R = 3.5
        o = oracle.Oracle(20, 21, 19, tau0=0.8)
        o.set_particles([X], R=[R])
        assert np.array_equal(o.owner() == 0, exact_inside(o.shape, X, R))


def test_cut_links_and_fractions_brute_force():
    X, R = np.array([10.25, 9.5, 8.75]), 3.75
    o = oracle.Oracle(20, 19, 18, tau0=0.8)
    o.set_particles([X], R=[R])
    solid = o.owner() == 0
    nz, ny, nx = o.shape
    want = []
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        if solid[z, y, x]:
            continue
        for j in range(1, 19):
            zz = z + C[j, 2]
            if 0 <= zz < nz and solid[zz, (y + C[j, 1]) % ny, (x + C[j, 0]) % nx]:
                want.append((x + nx * (y + ny * z), j))
    node, d, q, pid = o.links()
    assert sorted(want) == sorted(zip(node.tolist(), d.tolist()))
    assert (pid == 0).all()
    # q: smallest root of |x + t c - X| = R, from the quadratic in FP64
    for n, j, qq in zip(node, d, q):
        x = np.array([n % nx, (n // nx) % ny, n // (nx * ny)], dtype=float)
        c = C[j].astype(float)
        e = x - X
        a, b, c0 = c @ c, c @ e, e @ e - R * R
        t = (-b - np.sqrt(b * b - a * c0)) / a
        assert 0.0 <= t < 1.0
        assert abs(qq - t) < 2e-6
        # the boundary point is on the sphere
        assert abs(np.linalg.norm(x + qq * c - X) - R) < 1e-5
    assert (q < 0.5).any() and (q >= 0.5).any()


def test_overlap_tie_break():
    Xa, Xb, Ra, Rb = (8.25, 8.5, 8.0), (13.5, 8.5, 8.0), 3.5, 2.75
    o = oracle.Oracle(22, 17, 16, tau0=0.8)
    o.set_particles([Xa, Xb], R=[Ra, Rb])
    owner = o.owner()
    ina, inb = exact_inside(o.shape, Xa, Ra), exact_inside(o.shape, Xb, Rb)
    assert (owner[ina & ~inb] == 0).all() and (owner[inb & ~ina] == 1).all()
    both = np.argwhere(ina & inb)
    assert len(both) > 0
    for z, y, x in both:
        ka = np.linalg.norm(np.array([x, y, z]) - Xa) - Ra
        kb = np.linalg.norm(np.array([x, y, z]) - Xb) - Rb
        assert owner[z, y, x] == (0 if ka <= kb else 1)
    assert np.array_equal(owner >= 0, ina | inb)


def test_exact_ties_go_to_the_smaller_index():
    """Two equal spheres whose centres are mirror images across the node
    plane x = 10: every node of that plane inside both is at the same FP32
    distance from either centre, an exact tie of the keys |x - X| - R, and
    belongs to the sphere of smaller index whichever order they are given in."""
    R = 2.75
    for first, second in (((8.0, 8.5, 8.25), (12.0, 8.5, 8.25)), ((12.0, 8.5, 8.25), (8.0, 8.5, 8.25))):
        o = oracle.Oracle(22, 17, 16, tau0=0.8)
        o.set_particles([first, second], R=[R, R])
        owner = o.owner()
        both = exact_inside(o.shape, first, R) & exact_inside(o.shape, second, R)
        tied = np.argwhere(both)
        assert len(tied) > 0 and (tied[:, 2] == 10).all()
        assert (owner[both] == 0).all()


@pytest.mark.parametrize("Om", [(0.0, 0.0, 0.0), (0.01, -0.02, 0.015)])
def test_refill_of_uncovered_nodes(Om):
    """Shift a sphere by a prescribed motion; every node uncovered gets the
    equilibrium at the mean density of its neighbours fluid before and after,
    and at the surface velocity of the sphere, u_s = V + Om x (x - X) with X
    the new centre (Sect. 2.3, solid equilibrium)."""
    X0, R, V, Om = np.array([10.25, 9.5, 9.75]), 3.5, np.array([0.75, 0.0, 0.0]), np.array(Om)
    o = oracle.Oracle(22, 20, 20, tau0=0.7, cs=0.1, g=(1e-4, 0, 0))
    o.set_particles([X0], V=[V], Om=[Om], R=[R], fixed=[1])
    o.step(1)
    X1 = o.particles()[0][0]
    assert np.array_equal(X1, X0 + V)
    f_before = o.populations().copy()
    before = o.owner() == 0
    o.refill_only()
    after = o.owner() == 0
    assert np.array_equal(after, exact_inside(o.shape, X1, R))
    uncovered = before & ~after
    assert uncovered.sum() == o.refilled > 0
    f = o.populations()
    nz, ny, nx = o.shape
    for z, y, x in np.argwhere(uncovered):
        rhos = []
        for i in range(1, 19):
            zz = z + C[i, 2]
            if not 0 <= zz < nz:
                continue
            yy, xx = (y + C[i, 1]) % ny, (x + C[i, 0]) % nx
            if not before[zz, yy, xx] and not after[zz, yy, xx]:
                rhos.append(f_before[:, zz, yy, xx].sum())
        expect = oracle.feq(np.mean(rhos), V + np.cross(Om, np.array([x, y, z]) - X1))
        assert np.allclose(f[:, z, y, x], expect, rtol=0, atol=1e-15)
    # nodes not uncovered are untouched
    keep = ~uncovered & ~after
    assert np.array_equal(f[:, keep], f_before[:, keep])


def test_bounce_back_reads_the_fictitious_node():
    """Sect. 2.3: for q < 1/2 the reflected population is the one that left
    the fictitious node x_f' = x_f - (1 - 2q) c_j, reaching x_f after exactly
    one time step.  On a field whose post-collision populations are linear in
    space, f_j^c = w_j rho(z) with rho linear in z (rest fluid, tau = 1: the
    collision maps it to itself), the bounce-back value must therefore equal
    w_j rho(z_f').  For q >= 1/2 (and for q < 1/2 with x_f - c_j solid) both
    interpolated values sit at x_f and the result is w_j rho(z_f)."""
    c, w, opp = oracle.tables()
    nx, ny, nz, a = 20, 19, 22, 4e-3
    o = oracle.Oracle(nx, ny, nz, tau0=1.0, cs=0.0)
    o.set_particles([[9.75, 9.5, 10.25]], R=[4.25], fixed=[1])
    z = np.arange(nz, dtype=float)
    rho = 1.0 + a * (z - 10.0)
    f = w[:, None, None, None] * rho[None, :, None, None] * np.ones((19, nz, ny, nx))
    o.set_populations(f)
    node, d, q, pid = o.links()
    solid = o.owner() >= 0
    o.step(1)
    fn = o.populations().reshape(19, -1)
    n_lt = 0
    for n, j, qq in zip(node, d, q.astype(float)):
        x, y, zz = n % nx, (n // nx) % ny, n // (nx * ny)
        k = opp[j]
        zb = zz - c[j, 2]
        behind_fluid = 0 <= zb < nz and not solid[zb, (y - c[j, 1]) % ny, (x - c[j, 0]) % nx]
        if qq < 0.5 and behind_fluid:
            zf = zz - (1.0 - 2.0 * qq) * c[j, 2]
            n_lt += 1
        else:
            zf = zz
        assert abs(fn[k, n] - w[j] * (1.0 + a * (zf - 10.0))) < 1e-15
    assert n_lt > 50
