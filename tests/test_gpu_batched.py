"""GPU parity on the uneven batched workload at its full size: 4x3 Darcy
subdomains with grids drawn from {24,48,64,96}^2, mortar elements per edge
from {3,4,6,8}, N_term from 2..5 (9..243 local realizations, 558 basis items
of mixed shapes in one launch), and a batch of the first 2,000 points of the
Smolyak level-2 grid over 37 dimensions, solved as the benchmark solves it
(mixed CG to rtol 1e-10 after the mixed build, FP64 CG to rtol 1e-12 after the
FP64 build). The whole batch against the oracle's result for the same points
(``tests/golden/oracle_batched.npz``, written by a script that calls only the
oracle): moments entry by entry and the mortar solution at 128 sampled
points. Sampled items of every grid shape against the oracle; the two forms
against each other."""

import functools
import os

import numpy as np
import pytest

import sfb_workloads as W
from gpu_common import TOL, assert_close

pytestmark = pytest.mark.gpu

RTOL = 1e-10
RTOL_FP64 = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_batched.npz")
FIELDS = ("darcy_p", "darcy_flux", "stokes_u", "stokes_p")


@functools.lru_cache(maxsize=None)
def _oracle():
    from oracle import coupled
    w = W.batched()
    p = coupled.Problem(w)
    y, wt = p.grid()
    return w, p, y, wt


def _items(w):
    """One item per distinct grid shape (first, middle or last local point)."""
    seen, out = set(), []
    for i, g in enumerate(w["darcy_grid"]):
        if tuple(g) not in seen:
            seen.add(tuple(g))
            out.append(i)
    return out


@pytest.fixture(scope="module")
def gpu():
    import torch
    import paper_1802_06263_gb300 as sfb
    assert torch.cuda.is_available()
    w, p, _, _ = _oracle()
    s = sfb.Solver(w)
    y, wt = s.points()
    nb = w["n_batch"]
    y, wt = y[:nb], wt[:nb]
    s.allocate(sfb.FP64, max_pts=nb)
    yd = torch.tensor(y, device="cuda")
    wd = torch.tensor(wt, device="cuda")
    out = {"solver": s, "y": y, "w": wt}
    subs = _items(w)
    for prec in (sfb.FP64, sfb.MIXED):
        st = s.build_basis(prec)
        items = {}
        for j, i in enumerate(subs):
            n_loc = len(s.local_points(i))
            k = (0, n_loc // 2, n_loc - 1)[j % 3]
            items[(i, k)] = s.get_basis(i, k, with_x=True)
        lam = torch.empty((nb, s.n_lambda), dtype=torch.float64, device="cuda")
        it = torch.empty(nb, dtype=torch.int32, device="cuda")
        s.moments_reset()
        if prec == sfb.FP64:
            s.solve(yd, wd, RTOL_FP64, 2000, lam, it, krylov=sfb.CG)
        else:
            s.solve(yd, wd, RTOL, 2000, lam, it, krylov=sfb.CG_MIXED)
        torch.cuda.synchronize()
        out[prec] = {"stats": st, "items": items, "lam": lam.cpu().numpy(), "it": it.cpu().numpy(),
                     "mom": {f: s.moments(f) for f in FIELDS}}
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8)])
def test_sampled_items_of_every_shape(gpu, prec, tol):
    w, p, y, _ = _oracle()
    st = gpu[prec]["stats"]
    assert st["n_items"] == 558 and st["n_not_converged"] == 0
    for (i, k), (phi, g, X) in gpu[prec]["items"].items():
        loc = p.local_realizations(i, y)[0]
        phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[k])
        assert phi.shape == phi_o.shape
        assert_close(phi, phi_o, tol, ("phi", i, k, w["darcy_grid"][i]))
        assert_close(X, X_o, tol, ("X", i, k, w["darcy_grid"][i]))


@pytest.mark.parametrize("prec", [0, 1])
def test_full_batch_against_the_oracle(gpu, prec):
    g = np.load(GOLDEN)
    y = gpu["y"]
    assert int(g["n_pts"]) == len(y)
    assert np.allclose(g["y_checksum"], [y.sum(), (y * y).sum(), gpu["w"].sum()], rtol=1e-12, atol=1e-9)
    tol = TOL[prec]
    for f in FIELDS:
        m, v = gpu[prec]["mom"][f]
        assert_close(m, g[f + "_mean"], tol, (f, "mean"))
        assert_close(v, g[f + "_var"], tol, (f, "variance"))
    key = {tuple(np.round(r, 9)): i for i, r in enumerate(y)}
    lam = gpu[prec]["lam"]
    for j, r in enumerate(g["sample_y"]):
        assert_close(lam[key[tuple(np.round(r, 9))]], g["sample_lambda"][j], tol, ("lambda", j))
    assert np.all(gpu[prec]["it"] > 0)


def test_mixed_matches_fp64(gpu):
    for f in FIELDS:
        for j in (0, 1):
            assert_close(gpu[1]["mom"][f][j], gpu[0]["mom"][f][j], 1e-8, (f, j))
    for l in range(len(gpu["y"])):
        assert_close(gpu[1]["lam"][l], gpu[0]["lam"][l], 1e-8, ("lambda", l))
