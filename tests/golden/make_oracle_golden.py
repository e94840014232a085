"""Writes the oracle's reference results for the full benchmark batches.

Calls only ``oracle/`` (and the input data of ``sfb_workloads``): for the
precision workload (all 2,049 points of its Smolyak grid) and the batched
workload (its batch of the first 2,000 points) it solves every point's
interface problem densely from the multiscale flux bases of its local
realizations (Section 5.4 Steps 3-6), recovers the fields and forms the
collocation mean and centred variance of every field (Eq. 2.1, reading A12).
It stores those moments in full, and the mortar solutions of a sample of
points with the points' coordinates, as ``oracle_<workload>.npz`` beside
this script.

  python tests/golden/make_oracle_golden.py [precision] [batched]
"""

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import sfb_workloads as W  # noqa: E402
from oracle import coupled  # noqa: E402

FIELDS = ("darcy_p", "darcy_flux", "stokes_u", "stokes_p")
N_SAMPLE = 128   # points whose mortar solution is stored


def golden(name):
    w = W.ALL[name]()
    p = coupled.Problem(w)
    y, wt = p.grid()
    nb = w.get("n_batch") or len(y)
    y, wt = y[:nb], wt[:nb]
    t0 = time.time()
    lams, mom = coupled.solve_all(p, y, wt)
    sel = np.unique(np.linspace(0, nb - 1, N_SAMPLE).astype(np.int64))
    out = {"n_pts": np.int64(nb), "sample_index": sel, "sample_y": y[sel], "sample_lambda": lams[sel],
           "y_checksum": np.array([y.sum(), (y * y).sum(), wt.sum()])}
    for f in FIELDS:
        out[f + "_mean"], out[f + "_var"] = mom[f]
    path = os.path.join(HERE, "oracle_%s.npz" % name)
    np.savez_compressed(path, **out)
    print("%s: %d points, %.1f s -> %s" % (name, nb, time.time() - t0, path))


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["precision", "batched"]):
        golden(name)
