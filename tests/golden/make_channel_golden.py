"""Write tests/golden/channel_config5.json: the FP64 oracle's mean plate drag
and its gradient for the differentiation-form workload (a 128 x 64 x 64
channel, velocity inlet with peak 0.04, pressure outlet, 4 x 40 x 40 plate
at x = 80..83, y, z = 12..51, 200 spheres of radius 3 upstream held fixed,
Cs = 0.15, tau0 = 0.6, body force 1e-6, 500 steps, drag averaged over
steps 301..500).  The gradient with respect to (inlet peak, body force, Cs)
comes from the oracle's tangent-linear pass and, for comparison, from
central differences of the oracle with h = 1e-4 relative.

Calls only oracle/ and the seeded input generator (no CUDA).  Takes a few
minutes on a multi-core host: python tests/golden/make_channel_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1703_05158_gb300 import inputs  # noqa: E402

CONFIG = dict(nx=128, ny=64, nz=64, tau0=0.6, cs=0.15, gx=1e-6, u_peak=0.04, plate_lo=(80, 12, 12),
              plate_hi=(83, 51, 51), steps=500, avg_from=301)


def main():
    X, R = inputs.channel_spheres()
    names = ("u_peak", "gx", "cs")
    base = oracle.channel(**CONFIG, X=X, R=R)
    tl, fd = [], []
    for k, name in enumerate(names):
        tl.append(oracle.channel(**CONFIG, X=X, R=R, dtheta=np.eye(3)[k])["dJ"])
        h = 1e-4 * CONFIG[name]
        jp = oracle.channel(**dict(CONFIG, **{name: CONFIG[name] + h}), X=X, R=R)["J"]
        jm = oracle.channel(**dict(CONFIG, **{name: CONFIG[name] - h}), X=X, R=R)["J"]
        fd.append((jp - jm) / (2 * h))
        print(name, tl[-1], fd[-1], flush=True)
    out = dict(source="oracle/channel_oracle.c via oracle.channel, inputs.channel_spheres(seed=20170320)",
               config=dict(CONFIG, plate_lo=list(CONFIG["plate_lo"]), plate_hi=list(CONFIG["plate_hi"]),
                           spheres=len(R), radius=3.0),
               J=base["J"], grad_tangent_linear=tl, grad_central_difference=fd, fd_relative_step=1e-4)
    with open(os.path.join(HERE, "channel_config5.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
