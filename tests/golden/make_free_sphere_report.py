"""Write tests/golden/channel_config5_free.json: the differentiation-form
workload (the configuration of make_channel_golden.py) with its 200 spheres
free instead of fixed, run by the coupled FP64 oracle (lbm_oracle.c, channel
option): the mean plate drag J, and central differences of J with respect to
(inlet peak, body force, Cs) at relative steps 1e-4, 1e-3 and 1e-2.

The library's adjoint differentiates the fixed-sphere J (node switch events
of moving spheres have no derivative); these values measure how far that
gradient is from the derivative of the free-sphere J, and whether the
free-sphere J is smooth enough at these steps for central differences to
settle.  Spheres start at rest with density 2.5, normal contact k_n = 1e3,
restitution 0.8 (the slurry workload's DEM), 16 DEM sub-steps.

Calls only oracle/ and the seeded input generator (no CUDA).  Takes about
half an hour on an 8-core host: python tests/golden/make_free_sphere_report.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1703_05158_gb300 import inputs  # noqa: E402

sys.path.insert(0, HERE)
from make_channel_golden import CONFIG  # noqa: E402

STEPS_REL = (1e-4, 1e-3, 1e-2)


def main():
    X, R = inputs.channel_spheres()
    names = ("u_peak", "gx", "cs")
    t0 = time.time()
    fixed = oracle.free_channel(**CONFIG, X=X, R=R, free=False)
    base = oracle.free_channel(**CONFIG, X=X, R=R, free=True)
    disp = np.linalg.norm(base["X"] - X, axis=1)
    print("J fixed %.12g  J free %.12g  displacement max %.3g mean %.3g  (%.0f s)" % (
        fixed["J"], base["J"], disp.max(), disp.mean(), time.time() - t0), flush=True)
    fd = {}
    for name in names:
        fd[name] = []
        for rel in STEPS_REL:
            h = rel * CONFIG[name]
            jp = oracle.free_channel(**dict(CONFIG, **{name: CONFIG[name] + h}), X=X, R=R)["J"]
            jm = oracle.free_channel(**dict(CONFIG, **{name: CONFIG[name] - h}), X=X, R=R)["J"]
            fd[name].append((jp - jm) / (2 * h))
            print(name, rel, fd[name][-1], "(%.0f s)" % (time.time() - t0), flush=True)
    out = dict(source="oracle/lbm_oracle.c (channel option) via oracle.free_channel, "
                      "inputs.channel_spheres(seed=20170320)",
               config=dict(CONFIG, plate_lo=list(CONFIG["plate_lo"]), plate_hi=list(CONFIG["plate_hi"]),
                           spheres=len(R), radius=3.0, rho_s=2.5, kn=1e3, restitution=0.8, dem_substeps=16),
               J_fixed=fixed["J"], J_free=base["J"], displacement_max=float(disp.max()),
               displacement_mean=float(disp.mean()), fd_relative_steps=list(STEPS_REL),
               grad_free_central_difference={k: v for k, v in fd.items()})
    with open(os.path.join(HERE, "channel_config5_free.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
