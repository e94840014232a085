"""Launch shapes, autotuner and graph replay of the basis build (GPU).

The basis items fall into two size classes, grids more than 64 cells wide and
the rest, and each class is one launch of the basis kernel. This workload has
one subdomain in each class (72x6 and 13x9 cells). Every launch shape of a
class must build the same basis. The autotuner must time every shape of each
class and keep the fastest. A replayed CUDA graph must give the same bits as
plain launches."""

import numpy as np
import pytest

import sfb_workloads as W
from gpu_common import TOL, rel

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
    n_shapes = 2 if prec == sfb.MIXED else 1
    ref = None
    for v in range(n_shapes):
        s.set_option("basis_shape", v)
        st = s.build_basis(prec)
        assert st["launch_shape"] == [v, v] and st["graph"] == 0
        assert st["n_not_converged"] == 0
        items = _items(s)
        if ref is None:
            ref = items
            continue
        for key, (phi, g, X) in items.items():
            phi0, g0, X0 = ref[key]
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
    for q in (0, 1):
        ms = st["tune_ms"][q][:2]
        assert all(m > 0 for m in ms), st["tune_ms"]
        assert st["launch_shape"][q] == int(np.argmin(ms)), st
    # tuned once per precision: the next build keeps the choice and times nothing
    n0 = s.launch_count()
    st2 = s.build_basis(sfb.MIXED)
    assert st2["launch_shape"] == st["launch_shape"] and s.launch_count() - n0 == 3
    # FP64 has one shape per class: nothing to time
    st64 = s.build_basis(sfb.FP64)
    assert st64["launch_shape"] == [0, 0]
    assert all(m == 0 for r in st64["tune_ms"] for m in r)
