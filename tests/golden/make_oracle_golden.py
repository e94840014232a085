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

  python tests/golden/make_oracle_golden.py [precision] [batched] [large]
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


N_LARGE = 1000       # strided sub-batch of the Large workload's 341,505 points
N_FIELD_SAMPLE = 20000   # moment entries stored per field (strided)
LARGE_ITEMS = ((0, 0), (5, 40), (15, 80), (10, 17))


def golden_large():
    """The Large workload (4x4 Darcy subdomains of 128x128 cells, quadratic
    mortars, level-3 Smolyak grid over 64 dimensions, 128x128 Stokes) is too
    big for the oracle's whole grid; it stores the oracle's result on a
    strided sub-batch of N_LARGE points: the moments of that sub-batch at
    N_FIELD_SAMPLE strided entries per field (and the full fields' 2-norms),
    the mortar solutions of 32 of its points, the Stokes basis and the flux
    bases of a few items."""
    w = W.large()
    p = coupled.Problem(w)
    t0 = time.time()
    y, wt = p.grid()
    sel = np.unique(np.linspace(0, len(y) - 1, N_LARGE).astype(np.int64))
    ys, ws = y[sel], wt[sel]
    lams, mom = coupled.solve_all(p, ys, ws)
    out = {"n_pts_total": np.int64(len(y)), "sel": sel, "ys": ys, "ws": ws}
    li = np.unique(np.linspace(0, len(sel) - 1, 32).astype(np.int64))
    out["lam_index"] = li
    out["lam"] = lams[li]
    for f in FIELDS:
        m, v = mom[f]
        stride = max(1, len(m) // N_FIELD_SAMPLE)
        out[f + "_stride"] = np.int64(stride)
        out[f + "_mean"] = m[::stride]
        out[f + "_var"] = v[::stride]
        out[f + "_norms"] = np.array([np.linalg.norm(m), np.linalg.norm(v)])
    phs, gs, _, _ = p.stokes_basis()
    out["stokes_phi"], out["stokes_g"] = phs, gs
    for i, k in LARGE_ITEMS:
        loc = p.local_grids[p.region_of[i]]
        phi, g, _, _ = p.darcy_basis(i, loc[k])
        out["item_%d_%d_phi" % (i, k)] = phi
        out["item_%d_%d_g" % (i, k)] = g
        out["item_%d_%d_y" % (i, k)] = loc[k]
    path = os.path.join(HERE, "oracle_large.npz")
    np.savez_compressed(path, **out)
    print("large: %d of %d points, %.1f s -> %s" % (len(sel), len(y), time.time() - t0, path))


if __name__ == "__main__":
    for name in (sys.argv[1:] or ["precision", "batched", "large"]):
        golden_large() if name == "large" else golden(name)
