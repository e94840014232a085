"""GPU parity at the full size of the precision workload (4x2 Darcy
subdomains of 64x64 cells, 81 local realizations each, Smolyak level 2 over
32 dimensions, 2,049 points), in the configuration the benchmark times: an
FP64-sized workspace holding both forms, every point in one batch on device
buffers, CG to rtol 1e-10 (FP64 CG after the FP64 build, mixed CG after the
mixed build).

The oracle cannot redo the whole batch in a test's time, so the checks are
(a) sampled outputs it computes one by one: basis items, the mortar solution
at sampled points, and the moments of a sampled sub-batch; (b) properties
that hold at any size: the two forms agree, moments of split batches add up,
variances are non-negative."""

import functools

import numpy as np
import pytest

import sfb_workloads as W
from gpu_common import rel

pytestmark = pytest.mark.gpu

RTOL = 1e-10
FIELDS = ("darcy_p", "darcy_flux", "stokes_u", "stokes_p")
ITEMS = [(0, 0), (0, 40), (3, 80), (4, 13), (5, 67), (7, 80)]
POINTS = [0, 1, 2, 33, 500, 1024, 2047, 2048]


@functools.lru_cache(maxsize=None)
def _oracle():
    from oracle import coupled
    p = coupled.Problem(W.precision())
    y, wt = p.grid()
    return p, y, wt


@pytest.fixture(scope="module")
def gpu():
    import torch
    import paper_1802_06263_gb300 as sfb
    assert torch.cuda.is_available()
    s = sfb.Solver(W.precision())
    s.allocate(sfb.FP64)
    y, wt = s.points()
    yd = torch.tensor(y, device="cuda")
    wd = torch.tensor(wt, device="cuda")
    out = {"solver": s, "y": y, "w": wt}
    for prec in (sfb.FP64, sfb.MIXED):
        st = s.build_basis(prec)
        items = {(i, k): s.get_basis(i, k, with_x=True) for i, k in ITEMS}
        lam = torch.empty((len(y), s.n_lambda), dtype=torch.float64, device="cuda")
        it = torch.empty(len(y), dtype=torch.int32, device="cuda")
        s.moments_reset()
        # as the benchmark runs them: FP64 CG after the FP64 build, the
        # mixed CG after the mixed build
        s.solve(yd, wd, RTOL, 2000, lam, it, krylov=sfb.CG if prec == sfb.FP64 else sfb.CG_MIXED)
        torch.cuda.synchronize()
        out[prec] = {"stats": st, "items": items, "lam": lam.cpu().numpy(), "it": it.cpu().numpy(),
                     "mom": {f: s.moments(f) for f in FIELDS}}
    return out


def test_points_match_the_oracle_grid(gpu):
    p, y, wt = _oracle()
    assert gpu["y"].shape == y.shape == (2049, 32)
    ref = {tuple(np.round(r, 10)): v for r, v in zip(y, wt)}
    for r, v in zip(gpu["y"], gpu["w"]):
        assert abs(ref[tuple(np.round(r, 10))] - v) < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8)])
def test_sampled_basis_items(gpu, prec, tol):
    p, y, wt = _oracle()
    st = gpu[prec]["stats"]
    assert st["n_items"] == 648 and st["n_not_converged"] == 0
    for (i, k), (phi, g, X) in gpu[prec]["items"].items():
        loc = p.local_realizations(i, y)[0]
        phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[k])
        assert rel(phi, phi_o) < tol, (i, k)
        assert rel(X, X_o) < tol, (i, k)
        if np.linalg.norm(g_o) > 0:
            assert rel(g, g_o) < tol, (i, k)
        else:
            assert np.abs(g).max() < 1e-12


def test_mixed_form_reports_refinement(gpu):
    st = gpu[1]["stats"]
    # the unrefined FP32 solve is far from 1e-8; refinement closes the gap
    assert 1e-6 < st["max_first_correction"] < 1e-2
    assert 1 <= st["max_refine_steps"] <= 8
    assert st["max_error_estimate"] <= 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_sampled_points_within_the_cg_bound(gpu, prec):
    """CG stops at ||g - S lam|| <= rtol ||g||, so the error of lam is at most
    cond(S) * rtol; a basis error eps_b in S adds at most cond(S) * eps_b."""
    p, _, _ = _oracle()
    y = gpu["y"]
    lam = gpu[prec]["lam"]
    it = gpu[prec]["it"]
    assert np.all(it > 0)
    eps_b = 1e-12 if prec == 0 else 1e-9
    for l in POINTS:
        lam_o, S, g, _ = p.interface_dense(y[l])
        kappa = np.linalg.cond(S)
        err = rel(lam[l], lam_o)
        assert err <= kappa * (RTOL + eps_b), (l, err, kappa)
        assert np.linalg.norm(g - S @ lam[l]) <= (1.5 * RTOL + kappa * eps_b) * np.linalg.norm(g)


@pytest.mark.parametrize("prec", [0, 1])
def test_moments_properties_full_batch(gpu, prec):
    for f in FIELDS:
        m, v = gpu[prec]["mom"][f]
        assert np.all(np.isfinite(m)) and np.all(np.isfinite(v))
        assert v.min() >= -1e-12 * max(1.0, np.abs(m).max() ** 2), f


def test_mixed_matches_fp64_moments_full_batch(gpu):
    """Both forms solve the same discrete problem; the mixed form stays within
    1e-8 of the FP64 form in mean and variance of every field."""
    for f in FIELDS:
        m0, v0 = gpu[0]["mom"][f]
        m1, v1 = gpu[1]["mom"][f]
        assert rel(m1, m0) < 1e-8, f
        assert rel(v1, v0) < 1e-8, f
    assert rel(gpu[1]["lam"], gpu[0]["lam"]) < 1e-8


def test_split_batches_full_size(gpu):
    """Moments accumulated over three uneven sub-batches equal the moments of
    the single batch."""
    s = gpu["solver"]
    y, wt = gpu["y"], gpu["w"]
    s.build_basis(0)
    s.moments_reset()
    for a, b in ((0, 700), (700, 701), (701, 2049)):
        s.solve_host(y[a:b], wt[a:b], rtol=RTOL, max_it=2000)
    for f in FIELDS:
        m, v = s.moments(f)
        m0, v0 = gpu[0]["mom"][f]
        assert rel(m, m0) < 1e-10, f
        assert rel(v, v0) < 1e-9, f


@pytest.mark.parametrize("factor", [0, 0.01])
def test_sampled_batch_moments_against_the_oracle(gpu, factor):
    """Moments of a 40-point sub-batch against the oracle's direct per-point
    accumulation; factor 0.01 sends every group through the coefficient-moment
    path, factor 0 every group through the per-point path."""
    from oracle import coupled
    p, y, wt = _oracle()
    sel = np.unique(np.linspace(0, len(y) - 1, 40).astype(int))
    lams_o, mom_o = coupled.solve_all(p, y[sel], wt[sel])
    s = gpu["solver"]
    s.build_basis(1)
    s.set_option("moments_group_factor", factor)
    try:
        s.moments_reset()
        lam, it, rc = s.solve_host(y[sel], wt[sel], rtol=1e-13, max_it=2000)
        assert rel(lam, lams_o) < 1e-8
        for f in FIELDS:
            m, v = s.moments(f)
            assert rel(m, mom_o[f][0]) < 1e-8, f
            assert rel(v, mom_o[f][1]) < 1e-8, f
    finally:
        s.set_option("moments_group_factor", 1)


def test_empty_batch_is_a_no_op(gpu):
    s = gpu["solver"]
    y, wt = gpu["y"], gpu["w"]
    s.build_basis(0)
    s.moments_reset()
    s.solve_host(y[:10], wt[:10], rtol=RTOL, max_it=2000)
    before = {f: s.moments(f) for f in FIELDS}
    lam, it, rc = s.solve_host(y[:0], wt[:0], rtol=RTOL, max_it=2000)
    assert rc == 0 and lam.shape == (0, s.n_lambda)
    for f in FIELDS:
        m, v = s.moments(f)
        assert np.array_equal(m, before[f][0]) and np.array_equal(v, before[f][1])
