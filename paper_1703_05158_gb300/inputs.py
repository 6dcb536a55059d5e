"""Seeded synthetic inputs for the tests and the benchmark.

This module draws random numbers and places spheres; it holds none of the
method's arithmetic and imports neither the CUDA binding nor the oracle, so
both sides can be fed from it.

Workloads (all synthetic; the paper measures on no public dataset):
  * ``sphere_in_box``: one sphere of radius 4 at the centre of a 32^3 box
    moving at (0.01, 0, 0) (the plain-method workload).
  * ``slurry_box``: 256^3 box, 2000 monodisperse spheres of radius 4 placed by
    random sequential addition, velocities uniform in [-0.01, 0.01]^3 (the
    production workload).
  * ``polydisperse``: radii uniform in [r_min, r_max], as in the paper's
    polydispersity sweep (Sect. 3, d_max/d_min).
  * ``batch_instances``: a parameter sweep of independent boxes (edges from
    {48, 64, 96, 128, 160}, radii in [2, 6], solid fraction in [0.05, 0.25],
    Cs in [0.1, 0.2], tau0 in [0.51, 0.8], body force in [1e-6, 1e-5]) like
    the paper's sweep over particle size, packing fraction and
    polydispersity, all drawn from one master seed.
"""
import numpy as np

SEED_BASE = 20170315


def rng(seed):
    return np.random.default_rng(seed)


def rsa_spheres(box, n, radius, seed, gap=1.0, wall_gap=1.0, periodic_z=False, max_tries=10 ** 7, partial=False):
    """Random sequential addition of ``n`` non-overlapping spheres.

    ``box`` = (nx, ny, nz); x and y are periodic, the z walls sit at -1/2 and
    nz - 1/2.  ``radius`` is a scalar or a (r_min, r_max) pair (uniform).
    Proposals are uniform in the box; a proposal is rejected when its surface
    is closer than ``gap`` to an accepted sphere (minimum image) or closer
    than ``wall_gap`` to a z wall.  Radii are drawn once, largest first.
    Returns (X [n,3], R [n]).  With ``partial``, running out of proposals
    returns the spheres placed so far (the largest radii) instead of raising.
    """
    nx, ny, nz = box
    g = rng(seed)
    if np.isscalar(radius):
        R = np.full(n, float(radius))
    else:
        R = np.sort(g.uniform(radius[0], radius[1], size=n))[::-1].copy()
    rmax = float(R.max()) if n else 0.0
    cell = 2.0 * rmax + gap
    dims = np.maximum(1, (np.array([nx, ny, nz]) // cell).astype(int))
    csize = np.array([nx, ny, nz], dtype=float) / dims
    grid = {}
    X = np.zeros((n, 3))
    L = np.array([nx, ny, nz], dtype=float)
    per = np.array([True, True, bool(periodic_z)])
    tries = 0
    for a in range(n):
        r = R[a]
        while True:
            tries += 1
            if tries > max_tries:
                if partial:
                    return X[:a].copy(), R[:a].copy()
                raise RuntimeError("random sequential addition failed after %d proposals" % max_tries)
            lo_z, hi_z = (0.0, nz) if periodic_z else (r - 0.5 + wall_gap, nz - 0.5 - r - wall_gap)
            if hi_z < lo_z:
                raise ValueError("sphere of radius %g does not fit between the walls" % r)
            p = np.array([g.uniform(0, nx), g.uniform(0, ny), g.uniform(lo_z, hi_z)])
            c = (p // csize).astype(int)
            ok = True
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        key = ((c[0] + dx) % dims[0], (c[1] + dy) % dims[1], (c[2] + dz) % dims[2])
                        for b in grid.get(key, ()):
                            d = p - X[b]
                            d = np.where(per, d - L * np.round(d / L), d)
                            if np.dot(d, d) < (r + R[b] + gap) ** 2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                X[a] = p
                grid.setdefault(tuple(c % dims), []).append(a)
                break
    return X, R


def uniform_vectors(n, lo, hi, seed):
    return rng(seed).uniform(lo, hi, size=(n, 3))


def perturbation(shape, amplitude, seed):
    """Uniform noise in [-amplitude, amplitude] of the given shape."""
    return rng(seed).uniform(-amplitude, amplitude, size=shape)


def sphere_in_box(n=32):
    """One sphere, radius 4, at the box centre, velocity (0.01, 0, 0)."""
    X = np.array([[n / 2.0, n / 2.0, n / 2.0]])
    V = np.array([[0.01, 0.0, 0.0]])
    return dict(X=X, V=V, Om=np.zeros((1, 3)), R=np.array([4.0]))


def slurry_box(box=(256, 256, 256), n=2000, radius=4.0, seed=SEED_BASE + 2, vmax=0.01):
    """Monodisperse slurry: RSA placement and uniform velocities."""
    X, R = rsa_spheres(box, n, radius, seed)
    V = uniform_vectors(n, -vmax, vmax, seed + 1)
    return dict(X=X, V=V, Om=np.zeros((n, 3)), R=R)


def phi_matched_count(box, phi, radius):
    """Sphere count that gives solid fraction phi in the box: round(phi V / v),
    v the mean sphere volume (radius a scalar or a uniform (r_min, r_max))."""
    if np.isscalar(radius):
        r3 = float(radius) ** 3
    else:
        a, b = radius
        r3 = (b ** 4 - a ** 4) / (4.0 * (b - a))
    return int(round(phi * box[0] * box[1] * box[2] / (4.0 / 3.0 * np.pi * r3)))


def phi_matched_slurry(box=(256, 256, 256), phi=0.13, radius=4.0, seed=SEED_BASE + 6, vmax=0.01):
    """The production slurry box at the solid fraction it names (0.13: 8136
    spheres of radius 4 instead of 2000), RSA placement, uniform velocities."""
    n = phi_matched_count(box, phi, radius)
    X, R = rsa_spheres(box, n, radius, seed)
    V = uniform_vectors(n, -vmax, vmax, seed + 1)
    return dict(X=X, V=V, Om=np.zeros((n, 3)), R=R)


def polydisperse(box, n, r_range, seed, vmax=0.01):
    X, R = rsa_spheres(box, n, r_range, seed)
    V = uniform_vectors(n, -vmax, vmax, seed + 1)
    return dict(X=X, V=V, Om=np.zeros((n, 3)), R=R)


def solid_fraction(box, R):
    return float(np.sum(4.0 / 3.0 * np.pi * np.asarray(R) ** 3) / (box[0] * box[1] * box[2]))


def splitmix64(x):
    """One step of SplitMix64 (Steele, Lea and Flood 2014): (next state, output)."""
    m = (1 << 64) - 1
    x = (x + 0x9E3779B97F4A7C15) & m
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return x, z ^ (z >> 31)


def batch_instances(master_seed=SEED_BASE + 4, count=64, edges=(48, 64, 96, 128, 160), r_range=(2.0, 6.0),
                    phi_range=(0.05, 0.25), cs_range=(0.1, 0.2), tau_range=(0.51, 0.8), g_range=(1e-6, 1e-5),
                    max_spheres=500, vmax=0.01):
    """Independent instances of a parameter sweep, one seed each from a
    SplitMix64 stream on ``master_seed``.  Per instance: box edges drawn
    from ``edges``, a target solid fraction phi, sphere count
    min(max_spheres, round(phi V / v_mean)) with v_mean the mean sphere
    volume of radii uniform in ``r_range``, RSA placement (gap 1; a dense
    box keeps the spheres that fit), velocities uniform in [-vmax, vmax]^3,
    Cs, tau0 and a body force along x.  Returns a list of dicts with
    ``box``, ``params`` (Lattice keywords except the box), ``parts`` and the
    target and realised solid fractions."""
    r0, r1 = r_range
    v_mean = 4.0 / 3.0 * np.pi * (r1 ** 4 - r0 ** 4) / (4.0 * (r1 - r0))  # E[4/3 pi r^3]
    state = int(master_seed)
    out = []
    for _ in range(count):
        state, seed = splitmix64(state)
        g = rng(seed)
        box = tuple(int(v) for v in g.choice(edges, size=3))
        phi = float(g.uniform(*phi_range))
        cs = float(g.uniform(*cs_range))
        tau0 = float(g.uniform(*tau_range))
        gx = float(g.uniform(*g_range))
        V = box[0] * box[1] * box[2]
        n = int(min(max_spheres, round(phi * V / v_mean)))
        sub = int(g.integers(1 << 62))
        X, R = rsa_spheres(box, n, r_range, sub, max_tries=50 * n + 20000, partial=True)
        vel = uniform_vectors(len(R), -vmax, vmax, sub + 1)
        params = dict(tau0=tau0, cs=cs, g=(gx, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16,
                      max_particles=max(n, 1), max_radius=r1)
        out.append(dict(box=box, params=params, parts=dict(X=X, V=vel, Om=np.zeros((len(R), 3)), R=R),
                        phi_target=phi, phi=solid_fraction(box, R) if len(R) else 0.0))
    return out


def channel_spheres(seed=SEED_BASE + 5, n=200, radius=3.0, box=(128, 64, 64), x_range=(4.0, 74.0), gap=1.0,
                    max_tries=10 ** 6):
    """Random sequential addition of n spheres of one radius upstream in a
    channel: centres with x in [x_range[0] + R, x_range[1] - R] (x is not
    periodic), y periodic, at least ``gap`` from each other's surfaces and
    from the z walls (at -1/2 and nz - 1/2).  Returns (X [n, 3], R [n])."""
    nx, ny, nz = box
    g = rng(seed)
    X = np.zeros((n, 3))
    R = np.full(n, float(radius))
    lo = np.array([x_range[0] + radius, 0.0, radius - 0.5 + gap])
    hi = np.array([x_range[1] - radius, float(ny), nz - 0.5 - radius - gap])
    tries = 0
    for a in range(n):
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("channel sphere placement failed")
            p = g.uniform(lo, hi)
            d = X[:a] - p
            d[:, 1] -= ny * np.round(d[:, 1] / ny)
            if a == 0 or np.min(np.einsum("ij,ij->i", d, d)) >= (2 * radius + gap) ** 2:
                X[a] = p
                break
    return X, R
