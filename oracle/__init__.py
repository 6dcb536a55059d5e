"""FP64 CPU oracle of the coupled LBM-DEM hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  It shares no code with the CUDA library; the
arithmetic lives in ``lbm_oracle.c`` and this module only marshals arguments.

Parity pins (tests/test_oracle_*.py): D3Q19 moment identities, exact mass and
momentum balance, rest-state invariance, Couette and Poiseuille closed forms,
the Smagorinsky reduction to BGK and its strain-rate relation, the lattice
point count of a sphere, brute-force link fractions, bounce-back exactness on
uniform flow, refill on a shifted sphere, drag on a periodic sphere array
against Hasimoto/Sangani-Acrivos, and the DEM restitution and contact time;
for the options: exact total-momentum conservation with the covered /
uncovered momentum correction, the Coulomb sliding / rolling closed forms,
exact linear and angular momentum of frictional collisions and a tangential
force confined to the tangent plane as the contact normal turns, the ZIEB
face's rest state, face density and mass balance of a piston stroke, and
for the Galilean-invariant exchange its reduction to Eqs. 25, 26 at rest and
its extra force on a translating sphere (the velocity times the fluid mass
the moving bounce-back creates).  The coupled free-sphere trajectory itself
has no closed form: its transient is unpinned beyond those invariants; its
steady state is pinned by Galilean invariance (a free sphere's terminal
velocity under a constant force against the drag on the same sphere held
fixed in the co-moving frame, tests/test_oracle_galilean.py).  The
Galilean-invariant extra term is pinned in force (a translating sphere:
the fluid mass the moving bounce-back creates) and in force and torque (a
sphere spinning in place: the term formed from the streamed populations).
"""
import ctypes
import os

import numpy as np

from . import build as _build

NQ = 19


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau0", ctypes.c_double), ("cs", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("u_lo", ctypes.c_double * 3), ("u_hi", ctypes.c_double * 3),
        ("rho_s", ctypes.c_double), ("kn", ctypes.c_double), ("restitution", ctypes.c_double),
        ("dem_substeps", ctypes.c_int), ("les", ctypes.c_int), ("fluid", ctypes.c_int),
        ("periodic_z", ctypes.c_int), ("momentum_correction", ctypes.c_int),
        ("kt", ctypes.c_double), ("mu", ctypes.c_double), ("restitution_t", ctypes.c_double),
        ("zieb", ctypes.c_int), ("zieb_area", ctypes.c_double), ("zieb_volume", ctypes.c_double),
        ("zieb_vp", ctypes.c_double), ("mea", ctypes.c_int),
        ("channel", ctypes.c_int), ("u_peak", ctypes.c_double),
        ("plate_lo", ctypes.c_int * 3), ("plate_hi", ctypes.c_int * 3),
    ]


class ChanParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("tau0", ctypes.c_double), ("cs", ctypes.c_double), ("gx", ctypes.c_double), ("u_peak", ctypes.c_double),
        ("plate_lo", ctypes.c_int * 3), ("plate_hi", ctypes.c_int * 3),
        ("steps", ctypes.c_int), ("avg_from", ctypes.c_int), ("periodic_x", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(_build.build()))
    return _lib


class Planted:
    """Context in which new Oracle objects (and the channel oracle) run a
    modified oracle: the text of lbm_oracle.c, and optionally of
    channel_oracle.c, with a mistake planted, compiled into ``path`` (a test
    checks that its pins catch the mistake).  The library is restored on
    exit."""

    def __init__(self, oracle_source, path, channel_source=None):
        self.lib = _bind(ctypes.CDLL(_build.build_variant(oracle_source, path, channel_source)))

    def __enter__(self):
        global _lib
        self.saved, _lib = _load(), self.lib
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def source(name="lbm_oracle.c"):
    """The text of one of the oracle's C files (for planting a mistake in a
    copy)."""
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), name)) as fh:
        return fh.read()


def _bind(lib):
    """Declare the oracle's entry points on a loaded library."""
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.orc_create.restype = vp
    lib.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
    lib.orc_destroy.argtypes = [vp]
    lib.orc_set_particles.argtypes = [vp, ctypes.c_int, dp, dp, dp, dp, ctypes.c_void_p]
    lib.orc_set_populations.argtypes = [vp, dp]
    lib.orc_get_populations.argtypes = [vp, dp]
    lib.orc_step.argtypes = [vp, ctypes.c_int]
    lib.orc_forces.argtypes = [vp, dp, dp]
    lib.orc_contact_forces.argtypes = [vp, dp]
    lib.orc_contact_torques.argtypes = [vp, dp]
    lib.orc_contact_overflow.restype = ctypes.c_int
    lib.orc_contact_overflow.argtypes = [vp]
    lib.orc_zieb_state.argtypes = [vp, dp]
    lib.orc_zieb_set_piston.argtypes = [vp, ctypes.c_double]
    lib.orc_particles.argtypes = [vp, dp, dp, dp]
    lib.orc_fields.argtypes = [vp, dp, dp]
    lib.orc_tau_eff.argtypes = [vp, dp]
    lib.orc_owner.argtypes = [vp, ip]
    lib.orc_links.restype = ctypes.c_long
    lib.orc_links.argtypes = [vp, ctypes.c_long, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p]
    lib.orc_refilled.restype = ctypes.c_long
    lib.orc_refilled.argtypes = [vp]
    lib.orc_step_count.restype = ctypes.c_long
    lib.orc_step_count.argtypes = [vp]
    lib.orc_tables.argtypes = [ip, ip, ip, dp, ip]
    lib.orc_feq.argtypes = [ctypes.c_double, dp, dp]
    lib.orc_refill_only.argtypes = [vp]
    lib.orc_set_load.argtypes = [vp, ctypes.c_void_p, ctypes.c_void_p]
    lib.orc_plate_drag.restype = ctypes.c_double
    lib.orc_plate_drag.argtypes = [vp]
    lib.orc_channel_violation.restype = ctypes.c_int
    lib.orc_channel_violation.argtypes = [vp]
    lib.chan_run.restype = ctypes.c_int
    lib.chan_run.argtypes = [ctypes.POINTER(ChanParams), ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p, ctypes.c_void_p]
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One oracle simulation: x, y periodic, walls at z = -1/2 and nz - 1/2.

    Arrays use node index x + nx*(y + ny*z); populations are [19, nz, ny, nx].
    """

    def __init__(self, nx, ny, nz, tau0, cs=0.0, g=(0.0, 0.0, 0.0), u_lo=(0.0, 0.0, 0.0),
                 u_hi=(0.0, 0.0, 0.0), rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16,
                 les=True, fluid=True, periodic_z=False, momentum_correction=False, kt=0.0, mu=0.0,
                 restitution_t=1.0, zieb=None, mea="paper", channel=None, threads=None):
        if threads is not None:
            os.environ["OMP_NUM_THREADS"] = str(threads)
        lib = _load()
        p = OrcParams()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.tau0, p.cs = tau0, cs
        p.g[:] = list(g)
        p.u_lo[:] = list(u_lo)
        p.u_hi[:] = list(u_hi)
        p.rho_s, p.kn, p.restitution = rho_s, kn, restitution
        p.dem_substeps, p.les, p.fluid = dem_substeps, int(bool(les)), int(bool(fluid))
        p.periodic_z = int(bool(periodic_z))
        p.momentum_correction = int(bool(momentum_correction))
        p.kt, p.mu, p.restitution_t = kt, mu, restitution_t
        p.mea = {"paper": 0, "galilean": 1}[mea]
        if zieb is not None:  # dict(area=A_p, volume=V_0, vp=v_p)
            p.zieb, p.zieb_area, p.zieb_volume, p.zieb_vp = 1, zieb["area"], zieb["volume"], zieb.get("vp", 0.0)
        if channel is not None:  # dict(u_peak=..., plate_lo=(x, y, z), plate_hi=(x, y, z)): x open
            p.channel, p.u_peak = 1, channel["u_peak"]
            p.plate_lo[:] = list(channel.get("plate_lo", (1, 0, 0)))
            p.plate_hi[:] = list(channel.get("plate_hi", (0, -1, -1)))
        self._h = lib.orc_create(ctypes.byref(p))
        if not self._h:
            raise MemoryError("oracle allocation failed")
        self.lib, self.shape = lib, (nz, ny, nx)
        self.N = nx * ny * nz if fluid else 0
        self.np = 0

    def close(self):
        if self._h:
            self.lib.orc_destroy(self._h)
            self._h = None

    __del__ = close

    def set_particles(self, X, V=None, Om=None, R=None, fixed=None):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
        n = X.shape[0]
        V = np.zeros((n, 3)) if V is None else np.ascontiguousarray(V, dtype=np.float64).reshape(n, 3)
        Om = np.zeros((n, 3)) if Om is None else np.ascontiguousarray(Om, dtype=np.float64).reshape(n, 3)
        R = np.ascontiguousarray(R, dtype=np.float64).reshape(n)
        fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8).reshape(n)
        self._keep = (X, V, Om, R, fx)
        rc = self.lib.orc_set_particles(self._h, n, _dp(X), _dp(V), _dp(Om), _dp(R),
                                        None if fx is None else fx.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle allocation failed")
        self.np = n

    def set_load(self, F=None, T=None):
        """External force and torque per sphere, [n, 3] each (None = zero)."""
        F = None if F is None else np.ascontiguousarray(F, dtype=np.float64).reshape(self.np, 3)
        T = None if T is None else np.ascontiguousarray(T, dtype=np.float64).reshape(self.np, 3)
        self._load = (F, T)
        self.lib.orc_set_load(self._h, None if F is None else F.ctypes.data, None if T is None else T.ctypes.data)

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(NQ * self.N)
        self.lib.orc_set_populations(self._h, _dp(f))

    def populations(self):
        f = np.empty(NQ * self.N)
        self.lib.orc_get_populations(self._h, _dp(f))
        return f.reshape((NQ,) + self.shape)

    def step(self, n=1):
        self.lib.orc_step(self._h, int(n))
        if self.lib.orc_contact_overflow(self._h):
            raise RuntimeError("a sphere had more open contacts than the oracle keeps (64)")

    def forces(self):
        F, T = np.empty((self.np, 3)), np.empty((self.np, 3))
        if self.np:
            self.lib.orc_forces(self._h, _dp(F), _dp(T))
        return F, T

    def contact_forces(self):
        F = np.empty((self.np, 3))
        if self.np:
            self.lib.orc_contact_forces(self._h, _dp(F))
        return F

    def zieb_state(self):
        """(cylinder density rho^n, piston displacement H_p^n, mean inflow v_f^n)."""
        out = np.empty(3)
        self.lib.orc_zieb_state(self._h, _dp(out))
        return out

    def zieb_set_piston(self, vp):
        self.lib.orc_zieb_set_piston(self._h, float(vp))

    def contact_torques(self):
        T = np.empty((self.np, 3))
        if self.np:
            self.lib.orc_contact_torques(self._h, _dp(T))
        return T

    def particles(self):
        X, V, Om = np.empty((self.np, 3)), np.empty((self.np, 3)), np.empty((self.np, 3))
        if self.np:
            self.lib.orc_particles(self._h, _dp(X), _dp(V), _dp(Om))
        return X, V, Om

    def fields(self):
        rho, u = np.empty(self.N), np.empty(3 * self.N)
        self.lib.orc_fields(self._h, _dp(rho), _dp(u))
        return rho.reshape(self.shape), u.reshape((3,) + self.shape)

    def tau_eff(self):
        t = np.empty(self.N)
        self.lib.orc_tau_eff(self._h, _dp(t))
        return t.reshape(self.shape)

    def owner(self):
        o = np.empty(self.N, dtype=np.int32)
        self.lib.orc_owner(self._h, o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return o.reshape(self.shape)

    def links(self):
        n = self.lib.orc_links(self._h, 0, None, None, None, None)
        node = np.empty(n, dtype=np.int64)
        d = np.empty(n, dtype=np.int32)
        q = np.empty(n, dtype=np.float32)
        pid = np.empty(n, dtype=np.int32)
        self.lib.orc_links(self._h, n, node.ctypes.data, d.ctypes.data, q.ctypes.data, pid.ctypes.data)
        return node, d, q, pid

    def plate_drag(self):
        """Channel option: the plate drag (x) of the last step's collided populations."""
        return float(self.lib.orc_plate_drag(self._h))

    def channel_violation(self):
        """Channel option: whether a sphere ever covered a node of the planes x <= 1 or x >= nx - 2."""
        return bool(self.lib.orc_channel_violation(self._h))

    def refill_only(self):
        """Run only geometry and refill of the next step (test hook)."""
        self.lib.orc_refill_only(self._h)

    @property
    def refilled(self):
        return int(self.lib.orc_refilled(self._h))

    @property
    def steps(self):
        return int(self.lib.orc_step_count(self._h))


def tables():
    """(c [19,3] int, w [19], opp [19]) as the oracle uses them."""
    lib = _load()
    cx, cy, cz, opp = (np.empty(NQ, dtype=np.int32) for _ in range(4))
    w = np.empty(NQ)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_tables(cx.ctypes.data_as(ip), cy.ctypes.data_as(ip), cz.ctypes.data_as(ip), _dp(w),
                   opp.ctypes.data_as(ip))
    return np.stack([cx, cy, cz], axis=1), w, opp


def feq(rho, u):
    """The oracle's second-order equilibrium (Eq. 9) for one (rho, u)."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(3)
    out = np.empty(NQ)
    lib.orc_feq(float(rho), _dp(u), _dp(out))
    return out


def channel(nx, ny, nz, tau0, cs, gx, u_peak, plate_lo, plate_hi, steps, avg_from, X=None, R=None,
            dtheta=(0.0, 0.0, 0.0), periodic_x=False, populations=False):
    """The differentiation-form channel (channel_oracle.c): returns a dict with
    the mean plate drag ``J``, its derivative ``dJ`` along ``dtheta`` (a
    direction in (u_peak, gx, cs)), the per-step drag ``drag``, the node
    classes ``type`` [nz, ny, nx] (0 fluid, 1 sphere, 2 inlet, 3 outlet,
    4 plate) and, if asked, the final populations ``f`` [19, nz, ny, nx]."""
    lib = _load()
    p = ChanParams()
    p.nx, p.ny, p.nz = nx, ny, nz
    p.tau0, p.cs, p.gx, p.u_peak = tau0, cs, gx, u_peak
    p.plate_lo[:] = list(plate_lo)
    p.plate_hi[:] = list(plate_hi)
    p.steps, p.avg_from, p.periodic_x = steps, avg_from, int(bool(periodic_x))
    X = np.ascontiguousarray(np.zeros((0, 3)) if X is None else X, dtype=np.float64).reshape(-1, 3)
    R = np.ascontiguousarray(np.zeros(0) if R is None else R, dtype=np.float64).reshape(-1)
    dt = np.ascontiguousarray(dtheta, dtype=np.float64)
    J, dJ = ctypes.c_double(), ctypes.c_double()
    drag = np.zeros(max(steps, 1))
    N = nx * ny * nz
    f = np.zeros(NQ * N) if populations else None
    typ = np.zeros(N, dtype=np.uint8)
    rc = lib.chan_run(ctypes.byref(p), len(R), X.ctypes.data, R.ctypes.data, dt.ctypes.data, ctypes.byref(J),
                      ctypes.byref(dJ), drag.ctypes.data, None if f is None else f.ctypes.data, typ.ctypes.data)
    if rc != 0:
        raise ValueError("channel oracle rejected its input")
    out = dict(J=J.value, dJ=dJ.value, drag=drag[:steps], type=typ.reshape(nz, ny, nx))
    if f is not None:
        out["f"] = f.reshape(NQ, nz, ny, nx)
    return out


def free_channel(nx, ny, nz, tau0, cs, gx, u_peak, plate_lo, plate_hi, steps, avg_from, X, R, free=True,
                 rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16):
    """The differentiation-form channel run by the coupled oracle (lbm_oracle.c,
    channel option), with the spheres free (moved by the momentum exchange
    and the contacts of the coupled step, starting at rest) or held fixed.
    Returns dict(J, drag [steps], X [n, 3] final centres).

    The step order of the coupled oracle collides first, so its step k
    (k = 0 .. steps) collides f^k into G^k and its plate links give D^k;
    J is the mean of D^s over s in [avg_from, steps], as in channel()."""
    o = Oracle(nx, ny, nz, tau0, cs=cs, g=(gx, 0.0, 0.0), rho_s=rho_s, kn=kn, restitution=restitution,
               dem_substeps=dem_substeps, channel=dict(u_peak=u_peak, plate_lo=plate_lo, plate_hi=plate_hi))
    try:
        X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
        n = X.shape[0]
        o.set_particles(X, R=R, fixed=None if free else np.ones(n, dtype=np.uint8))
        drag = np.zeros(steps + 1)
        for k in range(steps + 1):
            o.step(1)
            drag[k] = o.plate_drag()
        if o.channel_violation():
            raise RuntimeError("a sphere reached the planes next to the inlet or the outlet")
        Xf = o.particles()[0]
    finally:
        o.close()
    return dict(J=float(drag[avg_from:steps + 1].mean()), drag=drag[1:], X=Xf)
