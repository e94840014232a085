"""Launch shapes, autotuner and graph replay of the basis build (GPU).

The basis items fall into two size classes, grids more than 64 cells wide and
the rest, and each class is one launch of the basis kernel. This workload has
one subdomain in each class (72x6 and 13x9 cells). The CUDA-core launch shapes
of a class must build the same basis bit for bit up to 1e-12; the tensor-core
shape (narrow class only: 3xTF32 products on tcgen05, refined with the same
FP64 residuals) the same basis within the mixed form's tolerance, and the
oracle's. The autotuner must time every shape of each class and keep the
fastest. A replayed CUDA graph must give the same bits as plain launches."""

import numpy as np
import pytest

import sfb_workloads as W
from gpu_common import TOL, assert_close, make_workload, oracle_case, rel

pytestmark = pytest.mark.gpu


def _workload():
    w = W.small_test(nx=12, ny=10, px=2, py=1, n_sd=3, n_dd=2, n_term=2, degree=1, stokes=(7, 5), sigma2=2.0)
    w["darcy_grid"] = [(72, 6), (13, 9)]
    return w


def _solver():
    import torch
    import paper_1802_06263_gb300 as sfb
    assert torch.cuda.is_available()
    s = sfb.Solver(_workload())
    s.allocate(sfb.FP64)
    return s


def _items(s):
    return {(i, k): s.get_basis(i, k, with_x=True)
            for i in range(s.n_darcy) for k in range(len(s.local_points(i)))}


@pytest.mark.parametrize("prec", [0, 1])
def test_every_launch_shape_builds_the_same_basis(prec):
    import paper_1802_06263_gb300 as sfb
    s = _solver()
    s.set_option("basis_graph", 0)
    n_shapes = 3 if prec == sfb.MIXED else 2
    ref = None
    for v in range(n_shapes):
        s.set_option("basis_shape", v)
        st = s.build_basis(prec)
        tc = v == 2   # the tensor-core shape exists for the narrow class only
        # a class without shape v (FP64 narrow grids have one shape) keeps shape 0
        expect = [v if sfb.basis_launch_shape(prec, wide, v) else 0 for wide in (1, 0)]
        assert st["launch_shape"] == expect and st["graph"] == 0
        assert st["n_not_converged"] == 0
        items = _items(s)
        if ref is None:
            ref = items
            continue
        for key, (phi, g, X) in items.items():
            phi0, g0, X0 = ref[key]
            if tc and key[0] == 1:
                assert_close(phi, phi0, TOL[prec], (v, key))
                assert_close(X, X0, TOL[prec], (v, key))
                continue
            assert rel(phi, phi0) < 1e-12 and rel(X, X0) < 1e-12, (v, key)
            assert np.abs(g - g0).max() <= 1e-12 * max(1.0, np.abs(g0).max()), (v, key)
    # the basis is the method's: one item of each class against the oracle
    from oracle import coupled
    p = coupled.Problem(_workload())
    y, _ = p.grid()
    for i in (0, 1):
        loc = p.local_realizations(i, y)[0]
        phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[1])
        phi, g, X = ref[(i, 1)]
        assert rel(phi, phi_o) < TOL[prec] and rel(X, X_o) < TOL[prec], i
        if prec == sfb.MIXED:   # the tensor-core shape's item of the narrow class
            if i == 1:
                phi, g, X = items[(i, 1)]
                assert_close(phi, phi_o, TOL[prec], "tcgen05 phi")
                assert_close(X, X_o, TOL[prec], "tcgen05 X")


@pytest.mark.parametrize("key", ["tiny", "ragged", "medium", "anisotropic", "kl_regions", "paper_l2"])
def test_tensor_core_shape_against_the_oracle(key):
    """The tensor-core basis kernel, forced for every narrow item, against the
    oracle: every item's Phi, g and X, then the mortar solutions and the
    moments of the whole collocation grid, within the mixed form's 1e-8. The
    unrefined form of the same kernel (SFB_FP32_NOREFINE) is as far from the
    oracle as an FP32 solve (below 1e-3) and no closer than 1e-9."""
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case(key)
    s = sfb.Solver(make_workload(key))
    s.allocate(sfb.MIXED)
    s.set_option("basis_shape", 2)
    st = s.build_basis(sfb.MIXED)
    assert st["launch_shape"][1] == 2 and st["n_not_converged"] == 0
    tol = TOL[1]
    for i in range(len(p.subs)):
        loc = p.local_realizations(i, y)[0]
        for k in range(len(loc)):
            phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[k])
            phi, g, X = s.get_basis(i, k, with_x=True)
            assert_close(phi, phi_o, tol, ("phi", i, k))
            assert_close(X, X_o, tol, ("X", i, k))
            assert_close(g, g_o, tol, ("g", i, k))
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.CG_MIXED)
    assert rc == 0
    for l in range(len(y)):
        assert_close(lam[l], lams[l], tol, ("lambda", l))
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], tol, (f, "mean"))
        assert_close(v, mom[f][1], tol, (f, "variance"))
    st = s.build_basis(sfb.FP32_NOREFINE, check=False)
    worst = 0.0
    for i in range(len(p.subs)):
        loc = p.local_realizations(i, y)[0]
        phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[0])
        _, _, X = s.get_basis(i, 0, with_x=True)
        worst = max(worst, rel(X, X_o))
    assert 1e-9 < worst < 1e-3, worst


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_plain_launches(prec):
    s = _solver()
    s.set_option("basis_autotune", 0)
    s.set_option("basis_graph", 0)
    st = s.build_basis(prec)
    assert st["graph"] == 0
    plain = _items(s)
    s.set_option("basis_graph", 1)
    for rep in range(3):   # capture and replay; then a new refinement option forces a new capture
        if rep == 2:
            s.set_option("refine_max", 7)
        st = s.build_basis(prec)
        assert st["graph"] == 1 and st["n_not_converged"] == 0
        for key, (phi, g, X) in _items(s).items():
            phi0, g0, X0 = plain[key]
            assert np.array_equal(phi, phi0) and np.array_equal(g, g0) and np.array_equal(X, X0), (rep, key)
    n0 = s.launch_count()
    s.build_basis(prec)
    assert s.launch_count() - n0 == 3   # one launch per size class and the flux epilogue


def test_autotuner_times_every_shape_and_keeps_the_fastest():
    import paper_1802_06263_gb300 as sfb
    s = _solver()
    s.set_option("basis_autotune", 1)
    st = s.build_basis(sfb.MIXED)
    assert st["n_not_converged"] == 0
    for q, n in ((0, 2), (1, 3)):   # wide grids: two shapes; narrow: three, the tensor-core one last
        ms = st["tune_ms"][q][:n]
        assert all(m > 0 for m in ms), st["tune_ms"]
        assert all(m == 0 for m in st["tune_ms"][q][n:]), st["tune_ms"]
        assert st["launch_shape"][q] == int(np.argmin(ms)), st
    # tuned once per precision: the next build keeps the choice and times nothing
    n0 = s.launch_count()
    st2 = s.build_basis(sfb.MIXED)
    assert st2["launch_shape"] == st["launch_shape"] and s.launch_count() - n0 == 3
    # FP64: two shapes for the wide grids (G_b in shared or in global memory),
    # both timed; one for the narrow grids, not timed
    st64 = s.build_basis(sfb.FP64)
    assert all(m > 0 for m in st64["tune_ms"][0][:2]), st64["tune_ms"]
    assert st64["launch_shape"][0] == int(np.argmin(st64["tune_ms"][0][:2]))
    assert st64["launch_shape"][1] == 0 and all(m == 0 for m in st64["tune_ms"][1])
