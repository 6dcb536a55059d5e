"""ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every entry point of the header has a function of the same name here; the
``Lattice`` class wraps a handle for convenience.  Arrays may be numpy arrays
(host) or CUDA torch tensors (device: their data pointers are passed with
``LBM_DEVICE``).  PyTorch is only used for device memory and the current
stream; nothing here computes any part of the method, and there is no
fallback: if the library cannot be loaded, importing this module fails.
"""
import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_CUDA = -2
LBM_ERR_NOMEM = -3
LBM_ERR_CAPACITY = -4
LBM_ERR_DIVERGED = -5
LBM_ERR_UNSUPPORTED = -6
LBM_ERR_TIMEOUT = -7
LBM_ERR_GEOMETRY = -8

LBM_FP32 = 0
LBM_BF16_DEV = 1
LBM_FP16_DEV = 2
LBM_HOST = 0
LBM_DEVICE = 1

PRECISIONS = {"fp32": LBM_FP32, "bf16": LBM_BF16_DEV, "fp16": LBM_FP16_DEV}

EXPORTS = ("lbm_create", "lbm_destroy", "lbm_set_particles", "lbm_set_particle_load", "lbm_set_populations",
           "lbm_step", "lbm_forces", "lbm_particles", "lbm_particle_state", "lbm_fields", "lbm_populations", "lbm_geometry", "lbm_info",
           "lbm_sync", "lbm_error_string", "lbm_profile", "lbm_profile_read", "lbm_fields_noalloc",
           "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_handle", "lbm_batch_tune", "lbm_batch_step",
           "lbm_batch_sync", "lbm_channel_create", "lbm_channel_destroy", "lbm_channel_set_theta",
           "lbm_channel_forward", "lbm_channel_backward", "lbm_channel_drag", "lbm_channel_populations",
           "lbm_channel_geometry", "lbm_zieb_state", "lbm_zieb_set_piston", "lbm_selftest_wait")


SCHEDULES = {"serial": 0, "overlap": 1}
MEAS = {"paper": 0, "galilean": 1}
DEM_MODES = {"auto": 0, "cluster": 1, "grid": 2}


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("periodic_z", ctypes.c_int32),
        ("tau0", ctypes.c_double), ("cs_smag", ctypes.c_double),
        ("body_accel", ctypes.c_double * 3),
        ("wall_vel_lo", ctypes.c_double * 3), ("wall_vel_hi", ctypes.c_double * 3),
        ("rho_particle", ctypes.c_double), ("kn", ctypes.c_double), ("restitution", ctypes.c_double),
        ("dem_substeps", ctypes.c_int32), ("precision", ctypes.c_int32), ("max_particles", ctypes.c_int32),
        ("max_radius", ctypes.c_double),
        ("cuda_stream", ctypes.c_void_p), ("device", ctypes.c_int32), ("schedule", ctypes.c_int32),
        ("momentum_correction", ctypes.c_int32),
        ("kt", ctypes.c_double), ("mu", ctypes.c_double), ("restitution_t", ctypes.c_double),
        ("zieb", ctypes.c_int32), ("zieb_area", ctypes.c_double), ("zieb_volume", ctypes.c_double),
        ("zieb_piston_velocity", ctypes.c_double), ("mea", ctypes.c_int32), ("dem_mode", ctypes.c_int32),
    ]


class lbm_channel_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("tau0", ctypes.c_double), ("cs_smag", ctypes.c_double), ("body_accel_x", ctypes.c_double),
        ("inlet_peak", ctypes.c_double),
        ("plate_lo", ctypes.c_int32 * 3), ("plate_hi", ctypes.c_int32 * 3),
        ("steps", ctypes.c_int32), ("avg_from", ctypes.c_int32), ("checkpoint_every", ctypes.c_int32),
        ("device", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
    ]


class lbm_info_t(ctypes.Structure):
    _fields_ = [
        ("nodes", ctypes.c_int64), ("fluid_nodes", ctypes.c_int64), ("links", ctypes.c_int64),
        ("refilled", ctypes.c_int64), ("steps", ctypes.c_int64), ("particles", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("device_bytes", ctypes.c_int64),
    ]


_lib = None


def library_path():
    return _build.LIB


def load(build=True):
    """Load (building first if needed) the CUDA library; raises if it is missing."""
    global _lib
    if _lib is None:
        path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing; run __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        vp, ip, dp, fp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p
        lib.lbm_create.argtypes = [ctypes.POINTER(lbm_params), ctypes.POINTER(vp)]
        lib.lbm_destroy.argtypes = [vp]
        lib.lbm_set_particles.argtypes = [vp, ip, dp, dp, dp, dp, vp]
        lib.lbm_set_particle_load.argtypes = [vp, dp, dp, ip]
        lib.lbm_set_populations.argtypes = [vp, dp, ip]
        lib.lbm_step.argtypes = [vp, ip]
        lib.lbm_forces.argtypes = [vp, dp, dp, ip]
        lib.lbm_particles.argtypes = [vp, dp, dp, dp, ip]
        lib.lbm_particle_state.argtypes = [vp, dp, dp, dp, dp, dp, ip]
        lib.lbm_fields.argtypes = [vp, fp, fp, ip]
        lib.lbm_populations.argtypes = [vp, dp, ip]
        lib.lbm_geometry.argtypes = [vp, vp, ip]
        lib.lbm_info.argtypes = [vp, ctypes.POINTER(lbm_info_t)]
        lib.lbm_sync.argtypes = [vp]
        lib.lbm_profile.argtypes = [vp, ip]
        lib.lbm_profile_read.argtypes = [vp, ctypes.c_void_p, ctypes.c_void_p]
        lib.lbm_fields_noalloc.argtypes = [vp, fp, fp]
        lib.lbm_batch_create.argtypes = [ctypes.POINTER(lbm_params), ip, ctypes.POINTER(vp)]
        lib.lbm_batch_destroy.argtypes = [vp]
        lib.lbm_batch_handle.argtypes = [vp, ip, ctypes.POINTER(vp)]
        lib.lbm_batch_tune.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_float)]
        lib.lbm_batch_step.argtypes = [vp, ip]
        lib.lbm_batch_sync.argtypes = [vp]
        lib.lbm_channel_create.argtypes = [ctypes.POINTER(lbm_channel_params), ip, dp, dp, ctypes.POINTER(vp)]
        lib.lbm_channel_destroy.argtypes = [vp]
        lib.lbm_channel_set_theta.argtypes = [vp, dp]
        lib.lbm_channel_forward.argtypes = [vp, dp]
        lib.lbm_channel_backward.argtypes = [vp, dp]
        lib.lbm_channel_drag.argtypes = [vp, dp]
        lib.lbm_channel_populations.argtypes = [vp, dp]
        lib.lbm_channel_geometry.argtypes = [vp, vp]
        lib.lbm_selftest_wait.argtypes = [vp]
        lib.lbm_zieb_state.argtypes = [vp, dp]
        lib.lbm_zieb_set_piston.argtypes = [vp, ctypes.c_double]
        lib.lbm_error_string.argtypes = [ctypes.c_int]
        lib.lbm_error_string.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "lbm_error_string":
                getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


class LbmError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s: %s (%d)" % (what, lbm_error_string(code), code))
        self.code = code


def _check(code, what):
    if code != LBM_OK:
        raise LbmError(code, what)
    return code


def _ptr(a):
    """(pointer, where) of a numpy array or a CUDA tensor; (None, HOST) for None."""
    if a is None:
        return None, LBM_HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr()), (LBM_DEVICE if a.is_cuda else LBM_HOST)
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data), LBM_HOST


# ---- the ABI, one function per entry point -------------------------------

def lbm_error_string(code):
    return load().lbm_error_string(int(code)).decode()


def lbm_create(params):
    h = ctypes.c_void_p()
    _check(load().lbm_create(ctypes.byref(params), ctypes.byref(h)), "lbm_create")
    return h


def lbm_destroy(h):
    return _check(load().lbm_destroy(h), "lbm_destroy")


def lbm_set_particles(h, pos, vel, omega, radius, fixed=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    n = pos.shape[0]
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3)
    omega = np.ascontiguousarray(omega, dtype=np.float64).reshape(n, 3)
    radius = np.ascontiguousarray(radius, dtype=np.float64).reshape(n)
    fx = None if fixed is None else np.ascontiguousarray(fixed, dtype=np.uint8).reshape(n)
    return _check(load().lbm_set_particles(h, n, pos.ctypes.data, vel.ctypes.data, omega.ctypes.data,
                                           radius.ctypes.data, None if fx is None else fx.ctypes.data),
                  "lbm_set_particles")


def lbm_set_particle_load(h, force=None, torque=None):
    pf, w1 = _ptr(force)
    pt, w2 = _ptr(torque)
    where = LBM_DEVICE if LBM_DEVICE in (w1, w2) else LBM_HOST
    return _check(load().lbm_set_particle_load(h, pf, pt, where), "lbm_set_particle_load")


def lbm_set_populations(h, f):
    p, where = _ptr(f)
    return _check(load().lbm_set_populations(h, p, where), "lbm_set_populations")


def lbm_step(h, nsteps=1):
    return _check(load().lbm_step(h, int(nsteps)), "lbm_step")


def lbm_forces(h, F, T):
    pF, where = _ptr(F)
    pT, _ = _ptr(T)
    return _check(load().lbm_forces(h, pF, pT, where), "lbm_forces")


def lbm_particles(h, pos, vel=None, omega=None):
    p1, where = _ptr(pos)
    p2, _ = _ptr(vel)
    p3, _ = _ptr(omega)
    return _check(load().lbm_particles(h, p1, p2, p3, where), "lbm_particles")


def lbm_particle_state(h, F=None, T=None, pos=None, vel=None, omega=None):
    arrays = (F, T, pos, vel, omega)
    ptrs = [_ptr(a) for a in arrays]
    where = next((w for a, (_, w) in zip(arrays, ptrs) if a is not None), LBM_HOST)
    return _check(load().lbm_particle_state(h, *[p for p, _ in ptrs], where), "lbm_particle_state")


def lbm_fields(h, rho, u):
    p1, w1 = _ptr(rho)
    p2, w2 = _ptr(u)
    where = w1 if rho is not None else w2
    return _check(load().lbm_fields(h, p1, p2, where), "lbm_fields")


LBM_NOALLOC_MAX_NODES = 1 << 20


def lbm_fields_noalloc(h, rho, u):
    """lbm_fields into host buffers without any device allocation (staging
    through the library's fixed array; lattices up to LBM_NOALLOC_MAX_NODES)."""
    p1, _ = _ptr(rho)
    p2, _ = _ptr(u)
    return _check(load().lbm_fields_noalloc(h, p1, p2), "lbm_fields_noalloc")


def lbm_populations(h, f):
    p, where = _ptr(f)
    return _check(load().lbm_populations(h, p, where), "lbm_populations")


def lbm_geometry(h, owner):
    p, where = _ptr(owner)
    return _check(load().lbm_geometry(h, p, where), "lbm_geometry")


def lbm_info(h):
    info = lbm_info_t()
    _check(load().lbm_info(h, ctypes.byref(info)), "lbm_info")
    return {name: getattr(info, name) for name, _ in lbm_info_t._fields_}


def lbm_sync(h):
    return _check(load().lbm_sync(h), "lbm_sync")


def lbm_selftest_wait(h):
    return _check(load().lbm_selftest_wait(h), "lbm_selftest_wait")


def lbm_zieb_state(h):
    out = np.empty(3)
    _check(load().lbm_zieb_state(h, out.ctypes.data), "lbm_zieb_state")
    return out


def lbm_zieb_set_piston(h, vp):
    return _check(load().lbm_zieb_set_piston(h, float(vp)), "lbm_zieb_set_piston")


PHASES = ("geometry", "collide", "links", "dem", "collide_far", "wait_far")


def lbm_profile(h, enable):
    return _check(load().lbm_profile(h, int(bool(enable))), "lbm_profile")


def lbm_profile_read(h):
    """({phase: total ms}, steps) since profiling was enabled."""
    ms = (ctypes.c_double * len(PHASES))()
    steps = ctypes.c_int64()
    _check(load().lbm_profile_read(h, ctypes.byref(ms), ctypes.byref(steps)), "lbm_profile_read")
    return dict(zip(PHASES, list(ms))), steps.value


def lbm_batch_create(params_list):
    arr = (lbm_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(load().lbm_batch_create(arr, len(params_list), ctypes.byref(b)), "lbm_batch_create")
    return b


def lbm_batch_destroy(b):
    return _check(load().lbm_batch_destroy(b), "lbm_batch_destroy")


def lbm_batch_handle(b, i):
    h = ctypes.c_void_p()
    _check(load().lbm_batch_handle(b, int(i), ctypes.byref(h)), "lbm_batch_handle")
    return h


def lbm_batch_tune(b):
    """(threads per block, blocks, ms per collide launch) picked by the autotuner."""
    t, g, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().lbm_batch_tune(b, ctypes.byref(t), ctypes.byref(g), ctypes.byref(ms)), "lbm_batch_tune")
    return t.value, g.value, ms.value


def lbm_batch_step(b, nsteps=1):
    return _check(load().lbm_batch_step(b, int(nsteps)), "lbm_batch_step")


def lbm_batch_sync(b):
    return _check(load().lbm_batch_sync(b), "lbm_batch_sync")


def make_params(nx, ny, nz, tau0, cs=0.0, g=(0.0, 0.0, 0.0), u_lo=(0.0, 0.0, 0.0), u_hi=(0.0, 0.0, 0.0),
                rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16, precision="fp32", max_particles=0,
                max_radius=4.0, stream=None, device=0, schedule="serial", momentum_correction=False, kt=0.0,
                mu=0.0, restitution_t=1.0, zieb=None, mea="paper", dem_mode="auto"):
    """lbm_params from keyword arguments (the Lattice constructor's); zieb:
    None or dict(area=A_p, volume=V_0, vp=v_p) for a ZIEB face on z = 0; mea:
    "paper" or "galilean" (momentum exchange); dem_mode: "auto", "cluster" or
    "grid" (how the DEM sub-steps run)."""
    p = lbm_params()
    p.nx, p.ny, p.nz, p.periodic_z = nx, ny, nz, 0
    p.tau0, p.cs_smag = tau0, cs
    p.body_accel[:] = list(g)
    p.wall_vel_lo[:] = list(u_lo)
    p.wall_vel_hi[:] = list(u_hi)
    p.rho_particle, p.kn, p.restitution = rho_s, kn, restitution
    p.dem_substeps = dem_substeps
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.max_particles, p.max_radius = max_particles, max_radius
    p.cuda_stream = stream
    p.device = device
    p.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    p.momentum_correction = int(bool(momentum_correction))
    p.kt, p.mu, p.restitution_t = kt, mu, restitution_t
    p.mea = MEAS[mea] if isinstance(mea, str) else int(mea)
    p.dem_mode = DEM_MODES[dem_mode] if isinstance(dem_mode, str) else int(dem_mode)
    if zieb is not None:
        p.zieb, p.zieb_area, p.zieb_volume = 1, zieb["area"], zieb["volume"]
        p.zieb_piston_velocity = zieb.get("vp", 0.0)
    return p


# ---- convenience wrappers ----------------------------------------------------

class Lattice:
    """One simulation handle; x, y periodic, walls at z = -1/2 and nz - 1/2.

    Host outputs are numpy arrays shaped like the oracle's: populations
    [19, nz, ny, nx], fields rho [nz, ny, nx] and u [3, nz, ny, nx].
    """

    def __init__(self, nx, ny, nz, tau0, cs=0.0, g=(0.0, 0.0, 0.0), u_lo=(0.0, 0.0, 0.0), u_hi=(0.0, 0.0, 0.0),
                 rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16, precision="fp32", max_particles=0,
                 max_radius=4.0, stream=None, device=0, schedule="serial", momentum_correction=False, kt=0.0,
                 mu=0.0, restitution_t=1.0, zieb=None, mea="paper", dem_mode="auto"):
        p = make_params(nx, ny, nz, tau0, cs, g, u_lo, u_hi, rho_s, kn, restitution, dem_substeps, precision,
                        max_particles, max_radius, stream, device, schedule, momentum_correction, kt, mu,
                        restitution_t, zieb, mea, dem_mode)
        self.params = p
        self.h = lbm_create(p)
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.np = 0
        self._owned = True

    @classmethod
    def member(cls, handle, params):
        """Wrap a batch member's handle (the batch owns it)."""
        self = cls.__new__(cls)
        self.params = params
        self.h = handle
        self.shape = (params.nz, params.ny, params.nx)
        self.N = params.nx * params.ny * params.nz
        self.np = 0
        self._owned = False
        return self

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, X, V=None, Om=None, R=None, fixed=None):
        X = np.asarray(X, dtype=np.float64).reshape(-1, 3)
        n = X.shape[0]
        V = np.zeros((n, 3)) if V is None else V
        Om = np.zeros((n, 3)) if Om is None else Om
        lbm_set_particles(self.h, X, V, Om, R, fixed)
        self.np = n

    def zieb_state(self):
        """(cylinder density, piston displacement, mean inflow velocity)."""
        return lbm_zieb_state(self.h)

    def zieb_set_piston(self, vp):
        lbm_zieb_set_piston(self.h, vp)

    def set_load(self, F=None, T=None):
        F = None if F is None else np.ascontiguousarray(F, dtype=np.float64).reshape(self.np, 3)
        T = None if T is None else np.ascontiguousarray(T, dtype=np.float64).reshape(self.np, 3)
        lbm_set_particle_load(self.h, F, T)

    def set_populations(self, f):
        if hasattr(f, "data_ptr"):
            lbm_set_populations(self.h, f)
        else:
            lbm_set_populations(self.h, np.ascontiguousarray(f, dtype=np.float64).reshape(19, -1))

    def step(self, n=1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def forces(self):
        F, T = np.zeros((self.np, 3)), np.zeros((self.np, 3))
        lbm_forces(self.h, F, T)
        return F, T

    def particles(self):
        X, V, Om = np.zeros((self.np, 3)), np.zeros((self.np, 3)), np.zeros((self.np, 3))
        lbm_particles(self.h, X, V, Om)
        return X, V, Om

    def fields(self):
        rho, u = np.empty(self.N, dtype=np.float32), np.empty(3 * self.N, dtype=np.float32)
        lbm_fields(self.h, rho, u)
        return rho.reshape(self.shape), u.reshape((3,) + self.shape)

    def populations(self):
        f = np.empty(19 * self.N)
        lbm_populations(self.h, f)
        return f.reshape((19,) + self.shape)

    def owner(self):
        o = np.empty(self.N, dtype=np.int32)
        lbm_geometry(self.h, o)
        return o.reshape(self.shape)

    def info(self):
        return lbm_info(self.h)

    def profile(self, enable=True):
        lbm_profile(self.h, enable)

    def profile_read(self):
        return lbm_profile_read(self.h)


class Batch:
    """Independent simulations stepped together (one graph replay per step).

    ``configs`` is a list of keyword dicts for the Lattice constructor (each
    with nx, ny, nz, tau0, ...); ``members`` are Lattice views of the members
    (set particles, read forces / fields through them; step the batch)."""

    def __init__(self, configs, stream=None, device=0):
        plist = []
        for c in configs:
            c = dict(c)
            c.setdefault("stream", stream)
            c.setdefault("device", device)
            plist.append(make_params(**c))
        self.params = plist
        self.b = lbm_batch_create(plist)
        self.members = [Lattice.member(lbm_batch_handle(self.b, i), p) for i, p in enumerate(plist)]

    def __len__(self):
        return len(self.members)

    def __getitem__(self, i):
        return self.members[i]

    def tune(self):
        return lbm_batch_tune(self.b)

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    def sync(self):
        lbm_batch_sync(self.b)

    def close(self):
        if getattr(self, "b", None):
            for m in self.members:
                m.h = None
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_channel_create(params, X, R):
    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 3)
    R = np.ascontiguousarray(R, dtype=np.float64).reshape(-1)
    c = ctypes.c_void_p()
    _check(load().lbm_channel_create(ctypes.byref(params), len(R), X.ctypes.data, R.ctypes.data, ctypes.byref(c)),
           "lbm_channel_create")
    return c


def lbm_channel_destroy(c):
    return _check(load().lbm_channel_destroy(c), "lbm_channel_destroy")


def lbm_channel_set_theta(c, theta):
    t = np.ascontiguousarray(theta, dtype=np.float64).reshape(3)
    return _check(load().lbm_channel_set_theta(c, t.ctypes.data), "lbm_channel_set_theta")


def lbm_channel_forward(c):
    J = ctypes.c_double()
    _check(load().lbm_channel_forward(c, ctypes.byref(J)), "lbm_channel_forward")
    return J.value


def lbm_channel_backward(c):
    g = np.zeros(3)
    _check(load().lbm_channel_backward(c, g.ctypes.data), "lbm_channel_backward")
    return g


def lbm_channel_drag(c, steps):
    d = np.zeros(steps)
    _check(load().lbm_channel_drag(c, d.ctypes.data), "lbm_channel_drag")
    return d


def lbm_channel_populations(c, n):
    f = np.zeros(19 * n)
    _check(load().lbm_channel_populations(c, f.ctypes.data), "lbm_channel_populations")
    return f


def lbm_channel_geometry(c, n):
    t = np.zeros(n, dtype=np.uint8)
    _check(load().lbm_channel_geometry(c, t.ctypes.data), "lbm_channel_geometry")
    return t


class Channel:
    """The differentiation form (lbm_channel_*): inlet / outlet channel with a
    fixed plate and fixed spheres; ``forward()`` -> mean plate drag J,
    ``backward()`` -> dJ/d(inlet_peak, body_accel_x, cs_smag)."""

    def __init__(self, nx, ny, nz, tau0, cs, gx, u_peak, plate_lo, plate_hi, steps, avg_from, checkpoint_every=50,
                 X=None, R=None, device=0, stream=None):
        p = lbm_channel_params()
        p.nx, p.ny, p.nz = nx, ny, nz
        p.tau0, p.cs_smag, p.body_accel_x, p.inlet_peak = tau0, cs, gx, u_peak
        p.plate_lo[:] = list(plate_lo)
        p.plate_hi[:] = list(plate_hi)
        p.steps, p.avg_from, p.checkpoint_every = steps, avg_from, checkpoint_every
        p.device, p.cuda_stream = device, stream
        self.c = lbm_channel_create(p, np.zeros((0, 3)) if X is None else X, np.zeros(0) if R is None else R)
        self.params = p
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.theta = (u_peak, gx, cs)

    def set_theta(self, theta):
        lbm_channel_set_theta(self.c, theta)
        self.theta = tuple(float(v) for v in np.asarray(theta, dtype=np.float64).reshape(3))

    def forward(self):
        return lbm_channel_forward(self.c)

    def backward(self):
        return lbm_channel_backward(self.c)

    def drag(self):
        return lbm_channel_drag(self.c, self.params.steps)

    def populations(self):
        return lbm_channel_populations(self.c, self.N).reshape((19,) + self.shape)

    def geometry(self):
        return lbm_channel_geometry(self.c, self.N).reshape(self.shape)

    def close(self):
        if getattr(self, "c", None):
            lbm_channel_destroy(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
