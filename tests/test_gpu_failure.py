"""Failure detection without a GPU fault: the only device-side wait of the
library (the grid barrier of the cooperative DEM) is bounded; a wait whose
partner never arrives gives up, the kernel returns, the host reads
LBM_ERR_TIMEOUT, and the device context stays usable."""
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def test_a_wait_that_runs_out_reports_a_timeout_and_the_context_survives():
    from paper_1703_05158_gb300 import lbm

    lbm.load()
    lat = lbm.Lattice(16, 16, 8, tau0=0.7)
    t0 = time.time()
    with pytest.raises(lbm.LbmError) as err:
        lbm.lbm_selftest_wait(lat.h)
    assert err.value.code == lbm.LBM_ERR_TIMEOUT
    assert time.time() - t0 < 60.0
    with pytest.raises(lbm.LbmError):  # the status is sticky on that handle
        lat.step(1)
    lat.close()
    fresh = lbm.Lattice(16, 16, 8, tau0=0.7)  # other handles run on
    fresh.step(20)
    _, w, _ = oracle.tables()
    assert np.array_equal(fresh.populations(), np.broadcast_to(w[:, None, None, None], (19, 8, 16, 16)))
