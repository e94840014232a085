"""GPU parity on the Large workload at its full problem size: 4x4 Darcy
subdomains of 128x128 cells (1,296 basis items of 81 local realizations
each), quadratic mortars with 8 elements per edge (672 mortar DOFs), a
128x128 Taylor-Hood Stokes subdomain (about 148,000 unknowns, factored by the
band LU), the level-3 Smolyak grid over 64 dimensions (341,505 points), and
GMRES(30) for the interface problem, as the benchmark runs it.

The oracle cannot solve all 341,505 points; ``tests/golden/oracle_large.npz``
(written by ``make_oracle_golden.py``, which calls only the oracle) holds its
result on a strided sub-batch of 1,000 of them: the moments of that
sub-batch at strided entries of every field and the full fields' norms, the
mortar solutions of 32 of its points, the Stokes basis and the flux bases of
four items. The GPU solves the same sub-batch after building every basis
item: FP64 form (FP64 GMRES to rtol 1e-12) within 1e-10, mixed form (GMRES
with FP32 Arnoldi products and FP64 restarts, to rtol 1e-12 as the benchmark
runs it: the grid's weights amplify per-point errors in the moments) within
1e-8."""

import functools
import os

import numpy as np
import pytest

import sfb_workloads as W
from gpu_common import TOL, assert_close

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_large.npz")
FIELDS = ("darcy_p", "darcy_flux", "stokes_u", "stokes_p")
RTOL = {0: 1e-12, 1: 1e-12}


@functools.lru_cache(maxsize=None)
def _golden():
    return dict(np.load(GOLDEN))


@pytest.fixture(scope="module")
def gpu():
    import torch
    import paper_1802_06263_gb300 as sfb
    assert torch.cuda.is_available()
    g = _golden()
    s = sfb.Solver(W.large())
    assert s.n_pts == int(g["n_pts_total"]) == 341505 and s.n_lambda == 672
    ys, ws = g["ys"], g["ws"]
    s.allocate(sfb.FP64, max_pts=len(ys))
    out = {"solver": s}
    for prec in (sfb.FP64, sfb.MIXED):
        st = s.build_basis(prec)
        items = {}
        for i in range(s.n_darcy):
            for key in g:
                if key.startswith("item_%d_" % i) and key.endswith("_y"):
                    loc = s.local_points(i)
                    k = int(np.argmin(np.abs(loc - g[key][None, :]).sum(axis=1)))
                    assert np.abs(loc[k] - g[key]).max() < 1e-12
                    items[key[:-2]] = s.get_basis(i, k)
        s.moments_reset()
        kr = sfb.GMRES if prec == sfb.FP64 else sfb.GMRES_MIXED
        lam, it, rc = s.solve_host(ys, ws, rtol=RTOL[prec], max_it=3000, krylov=kr)
        out[prec] = {"stats": st, "rc": rc, "lam": lam, "it": it, "items": items,
                     "mom": {f: s.moments(f) for f in FIELDS}, "stokes": s.get_basis(-1, 0)}
    return out


def test_the_grid_holds_the_golden_points(gpu):
    g = _golden()
    y, _ = gpu["solver"].points()
    keys = {tuple(np.round(r, 9)) for r in y}
    assert all(tuple(np.round(r, 9)) in keys for r in g["ys"])


@pytest.mark.parametrize("prec", [0, 1])
def test_basis_and_stokes_against_the_oracle(gpu, prec):
    g = _golden()
    st = gpu[prec]["stats"]
    assert st["n_items"] == 1296 and st["n_not_converged"] == 0
    phs, gs, _ = gpu[prec]["stokes"]
    assert_close(phs, g["stokes_phi"], 1e-10, "Stokes phi")
    assert_close(gs, g["stokes_g"], 1e-10, "Stokes g")
    assert len(gpu[prec]["items"]) == 4
    for key, (phi, gg, _) in gpu[prec]["items"].items():
        assert_close(phi, g[key + "_phi"], TOL[prec], (key, "phi"))
        assert_close(gg, g[key + "_g"], TOL[prec], (key, "g"))


@pytest.mark.parametrize("prec", [0, 1])
def test_sub_batch_against_the_oracle(gpu, prec):
    """GMRES on the 1,000-point sub-batch: every point converged, the sampled
    mortar solutions and the sampled moment entries within the form's
    tolerance, and the full moment fields' norms as well."""
    g = _golden()
    r = gpu[prec]
    assert r["rc"] == 0 and np.all(r["it"] > 0)
    for j, l in enumerate(g["lam_index"]):
        assert_close(r["lam"][l], g["lam"][j], TOL[prec], ("lambda", int(l)))
    for f in FIELDS:
        m, v = r["mom"][f]
        st = int(g[f + "_stride"])
        assert_close(m[::st], g[f + "_mean"], TOL[prec], (f, "mean"))
        assert_close(v[::st], g[f + "_var"], TOL[prec], (f, "variance"))
        nm, nv = g[f + "_norms"]
        assert abs(np.linalg.norm(m) - nm) <= TOL[prec] * nm, f
        assert abs(np.linalg.norm(v) - nv) <= TOL[prec] * nv, f


def test_mixed_matches_fp64_on_the_sub_batch(gpu):
    for f in FIELDS:
        for j in (0, 1):
            assert_close(gpu[1]["mom"][f][j], gpu[0]["mom"][f][j], 1e-8, (f, j))
