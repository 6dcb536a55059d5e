"""lbm_fields_noalloc: the host read-out of density and velocity for callers
that must not allocate device memory (a framework allocator already holds
the device's memory, or a step loop that may not allocate).  It stages
through a fixed array built into the library instead of a temporary
allocation; its results must be those of lbm_fields, call after call, on
the state the array was left in by the previous call.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1703_05158_gb300 import inputs

pytestmark = pytest.mark.gpu


def _lattice():
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    p = inputs.polydisperse((48, 40, 36), 6, (2.5, 4.0), seed=inputs.SEED_BASE + 31, vmax=0.02)
    lat = lbm.Lattice(48, 40, 36, tau0=0.6, cs=0.17, g=(2e-6, 0.0, 0.0), u_hi=(0.04, 0.0, 0.0),
                      max_particles=len(p["R"]), max_radius=4.0)
    lat.set_particles(p["X"], V=p["V"], R=p["R"])
    return lbm, lat


def test_noalloc_fields_match_lbm_fields_on_consecutive_calls():
    lbm, lat = _lattice()
    for steps in (7, 4):
        lat.step(steps)
        rho_ref, u_ref = lat.fields()
        rho = np.full(lat.N, np.nan, dtype=np.float32)
        u = np.full(3 * lat.N, np.nan, dtype=np.float32)
        lbm.lbm_fields_noalloc(lat.h, rho, u)
        assert np.array_equal(rho.reshape(lat.shape), rho_ref)
        assert np.array_equal(u.reshape((3,) + lat.shape), u_ref)
    # one output only
    rho = np.zeros(lat.N, dtype=np.float32)
    lbm.lbm_fields_noalloc(lat.h, rho, None)
    assert np.array_equal(rho.reshape(lat.shape), lat.fields()[0])
    lat.close()


def test_noalloc_fields_take_no_device_memory():
    """After the first call on the device (which has the driver commit the
    built-in array), a call leaves the device's free memory unchanged."""
    import torch

    lbm, lat = _lattice()
    lat.step(3)
    rho = np.zeros(lat.N, dtype=np.float32)
    u = np.zeros(3 * lat.N, dtype=np.float32)
    lbm.lbm_fields_noalloc(lat.h, rho, u)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    lbm.lbm_fields_noalloc(lat.h, rho, u)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    lat.close()


def test_noalloc_rejects_lattices_beyond_its_array():
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    lat = lbm.Lattice(128, 128, 65, tau0=0.7)
    assert lat.N > lbm.LBM_NOALLOC_MAX_NODES
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_fields_noalloc(lat.h, np.zeros(lat.N, dtype=np.float32), None)
    assert e.value.code == lbm.LBM_ERR_CAPACITY
    lat.close()
