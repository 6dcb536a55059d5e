"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point include/lbm.h declares, the binding names them
all, lbm_create rejects invalid parameters before touching the device, and
the link kernel's tile index arithmetic is exact and the per-sphere link and
refill capacities hold the worst case for every radius the ABI takes."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1703_05158_gb300 import build as libbuild
from paper_1703_05158_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(lbm_\w+)\s*\(", text, re.M)))


def test_header_declares_abi():
    names = declared()
    assert "lbm_create" in names and "lbm_step" in names and len(names) >= 13


def test_library_exports_every_declared_symbol():
    path = libbuild.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s+(lbm_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    lib = lbm.load()
    for n in declared():
        assert hasattr(lib, n)
    assert sorted(lbm.EXPORTS) == declared()
    for n in declared():
        assert callable(getattr(lbm, n))


def test_error_strings():
    for code in range(-8, 1):
        s = lbm.lbm_error_string(code)
        assert s and s != "unknown error"
    assert lbm.lbm_error_string(-99) == "unknown error"


@pytest.mark.parametrize("field,value", [("tau0", 0.5), ("nx", 0), ("restitution", 0.0), ("dem_substeps", 0),
                                         ("precision", 7), ("max_radius", 20.0), ("schedule", 9),
                                         ("momentum_correction", 2), ("kt", -1.0), ("mu", -0.5),
                                         ("restitution_t", 0.0), ("restitution_t", 1.5), ("zieb", 2),
                                         ("mea", 5), ("dem_mode", 7), ("tau0", float("inf")),
                                         ("cs_smag", float("nan")), ("kn", float("inf")),
                                         ("rho_particle", float("inf")), ("kt", float("inf")),
                                         ("max_radius", float("nan")), ("max_radius", 0.0), ("nx", 14)])
def test_create_rejects_invalid_parameters(field, value):
    p = lbm.make_params(32, 32, 32, 0.8, max_particles=4, max_radius=4.0, dem_substeps=4)
    setattr(p, field, value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_ARG


def test_create_rejects_moving_wall_normal_and_periodic_z():
    p = lbm.lbm_params()
    p.nx = p.ny = p.nz = 32
    p.tau0, p.rho_particle, p.kn, p.restitution, p.dem_substeps = 0.8, 2.5, 1e3, 0.8, 4
    p.wall_vel_hi[2] = 0.01
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_ARG
    p.wall_vel_hi[2] = 0.0
    p.periodic_z = 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


def test_create_rejects_non_finite_vectors_and_lattices_beyond_32_bit_offsets():
    for field in ("body_accel", "wall_vel_lo", "wall_vel_hi"):
        p = lbm.make_params(32, 32, 32, 0.8)
        getattr(p, field)[0] = float("nan")
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(p)
        assert e.value.code == lbm.LBM_ERR_ARG
    # 19 slots of 1024^2 * 2050 nodes exceed the kernels' 32-bit element offsets
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_params(1024, 1024, 2048, 0.8))
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


def test_zieb_face_needs_a_cylinder_and_the_serial_schedule():
    for zieb in (dict(area=0.0, volume=100.0), dict(area=10.0, volume=-1.0),
                 dict(area=10.0, volume=100.0, vp=float("nan"))):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(lbm.make_params(16, 16, 8, 0.8, zieb=zieb))
        assert e.value.code == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_params(16, 16, 8, 0.8, schedule="overlap", zieb=dict(area=10.0, volume=100.0)))
    assert e.value.code == lbm.LBM_ERR_UNSUPPORTED


def test_binding_structs_match_the_header_layout(tmp_path):
    """Compile a C program against include/lbm.h that prints the offset of
    every field of the ABI structs, and compare with the ctypes layout."""
    structs = {"lbm_params": lbm.lbm_params, "lbm_channel_params": lbm.lbm_channel_params,
               "lbm_info_t": lbm.lbm_info_t}
    lines = ['#include <stdio.h>', '#include "lbm.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_link_tile_decode_by_multiply_high_is_exact_for_every_allowed_radius():
    """The link kernel splits a tile index t < B^3 into (x, y, z) with
    __umulhi(t, 2^32 / B + 1) in place of t / B (B = 2 e + 1, e = ceil(R) + 2
    for the CTA's sphere of radius R, at most that of max_radius); check the
    quotients for every t and every extent a radius the ABI accepts gives
    (R <= 16), and that the kernel still uses this form.  The 16-bit list of
    a sphere's own tile nodes needs B^3 <= 2^16."""
    src = open(os.path.join(ROOT, "paper_1703_05158_gb300", "csrc", "lbm_links.cuh")).read()
    assert src.count("Tile tl(e, 0xFFFFFFFFu / B + 1u, 0xFFFFFFFFu / (B * B) + 1u)") == 1
    for R in range(1, 17):
        B = 2 * (R + 2) + 1
        B2 = B * B
        assert B2 * B <= 1 << 16
        mB, mB2 = 0xFFFFFFFF // B + 1, 0xFFFFFFFF // B2 + 1
        t = np.arange(B2 * B, dtype=np.uint64)
        z = (t * np.uint64(mB2)) >> np.uint64(32)
        assert np.array_equal(z, t // np.uint64(B2))
        r = t - z * np.uint64(B2)
        assert np.array_equal((r * np.uint64(mB)) >> np.uint64(32), r // np.uint64(B))


def _channel_params(**kw):
    p = lbm.lbm_channel_params()
    p.nx, p.ny, p.nz = 48, 20, 24
    p.tau0, p.cs_smag, p.body_accel_x, p.inlet_peak = 0.6, 0.15, 1e-6, 0.04
    p.plate_lo[:] = [20, 4, 6]
    p.plate_hi[:] = [23, 15, 17]
    p.steps, p.avg_from, p.checkpoint_every = 40, 21, 10
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [("nx", 7), ("nz", 1), ("tau0", 0.5), ("tau0", float("inf")),
                                         ("cs_smag", -0.1), ("cs_smag", float("inf")),
                                         ("inlet_peak", float("nan")), ("body_accel_x", float("inf")),
                                         ("steps", 0), ("avg_from", 0), ("avg_from", 41),
                                         ("checkpoint_every", 0)])
def test_channel_create_rejects_invalid_parameters(field, value):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_channel_create(_channel_params(**{field: value}), np.zeros((0, 3)), np.zeros(0))
    assert e.value.code == lbm.LBM_ERR_ARG


def test_channel_create_keeps_obstacles_clear_of_the_inlet_and_outlet():
    """The plate and every sphere stay off the inlet / outlet planes and their
    neighbours (x - R > 1, x + R < nx - 2; plate 2 <= x <= nx - 3)."""
    cases = [(_channel_params(), np.array([[4.0, 10.0, 12.0]]), np.array([3.0])),  # x - R = 1
             (_channel_params(), np.array([[43.5, 10.0, 12.0]]), np.array([3.0])),  # x + R = nx - 1.5
             (_channel_params(), np.array([[20.0, float("nan"), 12.0]]), np.array([3.0])),
             (_channel_params(), np.array([[20.0, 10.0, 12.0]]), np.array([0.0]))]
    p = _channel_params()
    p.plate_lo[0] = 1
    cases.append((p, np.zeros((0, 3)), np.zeros(0)))
    p = _channel_params()
    p.plate_hi[0] = 46
    cases.append((p, np.zeros((0, 3)), np.zeros(0)))
    for prm, X, R in cases:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_channel_create(prm, X, R)
        assert e.value.code == lbm.LBM_ERR_ARG


def _d3q19_moving():
    c = [v for v in np.ndindex(3, 3, 3) if 0 < sum(abs(k - 1) for k in v) <= 2]
    return np.array(c) - 1


def _ball_nodes(R, X):
    e = int(np.ceil(R)) + 2
    b = np.floor(X).astype(int)
    g = np.stack(np.meshgrid(*[np.arange(b[k] - e, b[k] + e + 1) for k in range(3)], indexing="ij"), -1)
    return g.reshape(-1, 3)


def test_per_sphere_capacities_hold_sampled_worst_cases_up_to_radius_16():
    """The link kernel keeps a sphere's cut links in shared memory (capacity
    ceil(80 r^2) + 64) and the refill kernel its uncovered nodes (a fixed
    list); brute-force counts at sampled sub-node centre offsets (and the
    symmetric ones) stay below both, with the sphere moving just under the
    0.25 nodes a step allows along every axis, face diagonal and body
    diagonal (the likeliest worst cases for uncovered nodes) and along one
    random direction, for radii up to the ABI's 16.  The offsets are
    sampled, so this bounds the counts seen, not every position."""
    src_links = open(os.path.join(ROOT, "paper_1703_05158_gb300", "csrc", "lbm_links.cu")).read()
    a, b = re.search(r"std::ceil\(([\d.]+) \* r \* r\) \+ (\d+)", src_links).groups()
    src_geo = open(os.path.join(ROOT, "paper_1703_05158_gb300", "csrc", "lbm_geometry.cu")).read()
    refill_cap = int(re.search(r"constexpr int kRefillCap = (\d+);", src_geo).group(1))
    c = _d3q19_moving()
    assert len(c) == 18
    dirs = [np.array(v, dtype=float) - 1 for v in np.ndindex(3, 3, 3) if v != (1, 1, 1)]  # 26 directions
    rng = np.random.default_rng(11)
    for R in (2.5, 4.0, 8.0, 16.0):
        cap = int(np.ceil(float(a) * R * R)) + int(b)
        offsets = [np.zeros(3), np.full(3, 0.5)] + [rng.uniform(0.0, 1.0, 3) for _ in range(12)]
        most_links, most_uncovered = 0, 0
        for off in offsets:
            X = 40.0 + off
            g = _ball_nodes(R, X)
            inside = ((g - X) ** 2).sum(1) < R * R
            fluid = g[~inside]
            most_links = max(most_links, sum(int((((fluid + cj) - X) ** 2).sum(1).__lt__(R * R).sum()) for cj in c))
            for v in list(dirs) + [rng.normal(size=3)]:
                d = 0.2499 * v / np.linalg.norm(v)
                most_uncovered = max(most_uncovered, int((inside & (((g - X - d) ** 2).sum(1) >= R * R)).sum()))
        assert most_links < cap, (R, most_links, cap)
        assert most_uncovered < refill_cap, (R, most_uncovered)


def test_a_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without the compiled library the binding raises, whether asked to load
    it as built or through an entry point that builds first: there is no CPU
    fallback behind it."""
    from paper_1703_05158_gb300 import build as bld

    absent = str(tmp_path / "absent.so")
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(bld, "LIB", absent)
    with pytest.raises(RuntimeError, match="missing"):
        lbm.load(build=False)
    monkeypatch.setattr(bld, "build", lambda *a, **k: absent)
    with pytest.raises(RuntimeError, match="missing"):
        lbm.lbm_error_string(0)
