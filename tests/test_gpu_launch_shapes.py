"""Launch shapes, autotuner and graph replay of the basis build (GPU).

The basis items fall into two size classes, grids more than 64 cells wide and
the rest, and each class is one launch of the basis kernel. This workload has
one subdomain in each class (72x6 and 13x9 cells). The CUDA-core launch shapes
of a class must build the same basis bit for bit up to 1e-12; the tensor-core
shape (narrow class only: 3xTF32 products on tcgen05, refined with the same
FP64 residuals) and the split shapes (factor launches, then one CTA per chunk
of at most 24 right-hand sides, each chunk refined to its own stopping test)
the same basis within the mixed form's tolerance, and the oracle's. The autotuner must time every shape of each class and keep the
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
    n_shapes = 4 if prec == sfb.MIXED else 2
    ref = None
    for v in range(n_shapes):
        s.set_option("basis_shape", v)
        st = s.build_basis(prec)
        # not bit for bit: the tensor-core shape (narrow class, v = 2) and the
        # split shapes (wide class v = 2, narrow class v = 3)
        loose = {0: prec == sfb.MIXED and v == 2, 1: prec == sfb.MIXED and v in (2, 3)}
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
            if loose[key[0]]:
                assert_close(phi, phi0, TOL[prec], (v, key))
                assert_close(X, X0, TOL[prec], (v, key))
                continue
            assert rel(phi, phi0) < 1e-12 and rel(X, X0) < 1e-12, (v, key)
            assert np.abs(g - g0).max() <= 1e-12 * max(1.0, np.abs(g0).max()), (v, key)
    # a split shape's pipeline groups run the same chunks: the same bits, and
    # two launches (factor, chunks) per group
    if prec == sfb.MIXED:
        s.set_option("basis_shape", 3)
        s.build_basis(prec)
        base = _items(s)
        n1 = s.launch_count()
        s.build_basis(prec)
        per_build = s.launch_count() - n1
        for groups in (2, 4):
            s.set_option("basis_pipe_groups", groups)
            n0 = s.launch_count()
            st = s.build_basis(prec)
            assert st["n_not_converged"] == 0 and st["launch_shape"] == [0, 3]
            assert s.launch_count() - n0 == per_build + 2 * (groups - 1)
            for key, (phi, g, X) in _items(s).items():
                assert np.array_equal(X, base[key][2]) and np.array_equal(phi, base[key][0]), (groups, key)
        s.set_option("basis_pipe_groups", 1)
    # the persistent launch (both classes' items as tasks of one launch)
    if prec == sfb.MIXED:
        s.set_option("basis_shape", 0)
        s.set_option("basis_persistent", 1)
        n0 = s.launch_count()
        st = s.build_basis(prec)
        assert st["persistent"] == 1 and st["n_not_converged"] == 0
        assert s.launch_count() - n0 == 2   # the persistent launch and the flux epilogue
        for key, (phi, g, X) in _items(s).items():
            phi0, g0, X0 = ref[key]
            assert_close(phi, phi0, TOL[prec], ("persistent", key))
            assert_close(X, X0, TOL[prec], ("persistent", key))
        s.set_option("basis_persistent", -1)
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
@pytest.mark.parametrize("shape", [2, 3, "persistent"])
def test_mixed_shape_against_the_oracle(key, shape):
    """The tensor-core basis kernel (shape 2), the split shape (3: factor
    launches, then column chunks) or the persistent launch (every item's factor
    and column chunks as tasks of one launch), forced for every item, against
    the oracle: every item's Phi, g and X, then the mortar solutions and the
    moments of the whole collocation grid, within the mixed form's 1e-8. The
    unrefined form of the same kernels (SFB_FP32_NOREFINE) is as far from the
    oracle as an FP32 solve (below 1e-3) and no closer than 1e-9."""
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case(key)
    s = sfb.Solver(make_workload(key))
    s.allocate(sfb.MIXED)
    if shape == "persistent":
        s.set_option("basis_shape", 0)
        s.set_option("basis_persistent", 1)
    else:
        s.set_option("basis_shape", shape)
    st = s.build_basis(sfb.MIXED)
    assert st["n_not_converged"] == 0
    assert st["persistent"] == 1 if shape == "persistent" else st["launch_shape"][1] == shape
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
    # wide grids: three shapes, the split one last; narrow: four, the
    # tensor-core one, then the split one
    for q, n in ((0, 3), (1, 4)):
        ms = st["tune_ms"][q][:n]
        assert all(m > 0 for m in ms), st["tune_ms"]
        assert all(m == 0 for m in st["tune_ms"][q][n:]), st["tune_ms"]
        assert st["launch_shape"][q] == int(np.argmin(ms)), st
    # tuned once per precision: the next build keeps the choice and times nothing
    n0 = s.launch_count()
    st2 = s.build_basis(sfb.MIXED)
    # one launch per size class and the flux epilogue; a split shape runs its
    # class as a pipeline of up to two item groups, two launches each
    per_class = []
    for q, sub in ((0, 0), (1, 1)):   # subdomain 0 is the wide grid, 1 the narrow one
        split = sfb.basis_launch_shape(sfb.MIXED, q == 0, st["launch_shape"][q])[4]
        per_class.append(2 * min(2, len(s.local_points(sub))) if split else 1)
    # (the autotuner also timed the persistent launch against these; when it won,
    # the build is one launch)
    assert st2["launch_shape"] == st["launch_shape"] and st2["persistent"] == st["persistent"]
    assert s.launch_count() - n0 == (2 if st["persistent"] else 1 + sum(per_class))
    # FP64: two shapes for the wide grids (G_b in shared or in global memory),
    # both timed; one for the narrow grids, not timed
    st64 = s.build_basis(sfb.FP64)
    assert all(m > 0 for m in st64["tune_ms"][0][:2]), st64["tune_ms"]
    assert st64["launch_shape"][0] == int(np.argmin(st64["tune_ms"][0][:2]))
    assert st64["launch_shape"][1] == 0 and all(m == 0 for m in st64["tune_ms"][1])
