"""Host-side checks of the C ABI that need no GPU: the library builds, loads
and exports every entry point include/lbm.h declares, the binding names them
all, and lbm_create rejects invalid parameters before touching the device."""
import os
import re
import subprocess

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
                                         ("precision", 7), ("max_radius", 20.0)])
def test_create_rejects_invalid_parameters(field, value):
    p = lbm.lbm_params()
    p.nx = p.ny = p.nz = 32
    p.tau0, p.rho_particle, p.kn, p.restitution = 0.8, 2.5, 1e3, 0.8
    p.dem_substeps, p.max_particles, p.max_radius = 4, 4, 4.0
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
