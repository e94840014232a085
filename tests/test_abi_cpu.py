"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point declared in include/sfb.h, and its set-up (KL eigenpairs,
collocation grids, mortar DOF maps, local realizations), computed by its own
host code, agrees with the oracle."""

import os
import re

import numpy as np
import pytest

import sfb_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import paper_1802_06263_gb300 as sfb
    if not os.path.exists(sfb.library_path()):
        sfb.build()
    return sfb


def test_library_exports_every_declared_symbol():
    sfb = _lib()
    lib = sfb.load()
    names = set()
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", hdr)).read()
            names |= set(re.findall(r"^\s*(?:sfb_status|void|const char\*)\s+(sfb_\w+)\s*\(", txt, re.M))
    assert len(names) >= 15
    for n in sorted(names):
        assert hasattr(lib, n), n


def _reordered_regions():
    """kl_regions with the region list in the other order: region 0 (whose
    stochastic dims come first) is the top row of subdomains."""
    w = W.kl_regions()
    w["kl"]["regions"] = [(0.0, 1.0, 0.25, 0.5), (0.0, 1.0, 0.0, 0.25)]
    w["kl"]["region_of"] = [1, 1, 0, 0]
    w["kl"]["n_term"] = [3, 2]
    w["kl"]["modes"] = [None, (2, 1)]
    return w


@pytest.mark.parametrize("name", ["tiny", "medium", "batched", "anisotropic", "kl_regions", "reordered_regions",
                                  "ragged", "ragged_tensor"])
def test_host_setup_matches_oracle(name):
    sfb = _lib()
    from oracle import coupled
    from gpu_common import make_workload
    if name == "reordered_regions":
        w = _reordered_regions()
    elif name.startswith("ragged"):
        w = make_workload(name)     # projections as local sets, quadratic mortars, sources
    else:
        w = W.ALL[name]()
    s = sfb.Solver(w)
    p = coupled.Problem(w)
    # eigenvalues region by region (each region's first subdomain carries them)
    first = [p.region_of.index(r) for r in range(len(p.n_term))]
    lam_o = np.concatenate([p.kl[i][0] for i in first])
    assert np.allclose(s.eigvals, lam_o, rtol=1e-13)
    # the tables the kernel evaluates: sqrt(lambda_j) and fx_j(x) fy_j(y) at
    # every cell centre, against the oracle's mode values (cells by y-rows)
    for i, sub in enumerate(p.subs):
        sl, fx, fy = s.kl_tables(i)
        lam, f = p.kl[i]
        assert np.allclose(sl ** 2, lam, rtol=1e-13)
        modes = np.einsum("jy,jx->jyx", fy, fx).reshape(len(lam), -1)
        assert np.allclose(modes, f, rtol=1e-12, atol=1e-13), i
    assert s.n_lambda == p.n_lambda
    y, wt = s.points()
    yo, wo = p.grid()
    assert y.shape == yo.shape
    ref = {tuple(np.round(r, 10)): v for r, v in zip(yo, wo)}
    for r, v in zip(y, wt):
        assert abs(ref[tuple(np.round(r, 10))] - v) < 1e-12
    for i in range(len(p.subs)):
        assert list(s.subdomain_dofs(i)) == p.subs[i].dofs
        assert np.allclose(s.local_points(i), p.local_realizations(i, yo)[0], atol=1e-15)
    assert list(s.subdomain_dofs(-1)) == p.stokes.dofs
    assert s.field_size("darcy_p") == sum(sub.n_cells for sub in p.subs)
    assert s.field_size("stokes_u") == 2 * p.stokes.n_nodes
    assert s.field_size("stokes_p") == p.stokes.n_p


def test_host_level_three_grid_matches_oracle():
    """The host's level-3 {1,3,3,3} grid over 40 dimensions (4 KL regions of
    10 terms): the oracle's points and weights, weights summing to one (each
    point's terms carry a compensation term)."""
    sfb = _lib()
    from oracle import collocation
    w = W.small_test(nx=6, ny=4, px=2, py=2, n_sd=2, n_dd=2, n_term=10, degree=1, stokes=(4, 4),
                     collocation={"kind": "smolyak", "lmax": 3, "rule": [1, 3, 3, 3]})
    s = sfb.Solver(w)
    y, wt = s.points()
    yo, wo = collocation.global_grid(w["collocation"], 40)
    assert y.shape == yo.shape == (82241, 40)
    # rounding of the terms themselves (coefficients up to 9,139 times products
    # of the 1-D weights) leaves about 2e-12; a plain running sum left 1.3e-9
    assert abs(wt.sum() - 1.0) < 1e-11
    ref = {tuple(np.round(r, 10)): v for r, v in zip(yo, wo)}
    assert max(abs(ref[tuple(np.round(r, 10))] - v) for r, v in zip(y, wt)) < 1e-11


def test_bad_arguments_are_rejected():
    sfb = _lib()
    w = W.tiny()
    w["mortar_degree"] = 3
    with pytest.raises(sfb.SfbError):
        sfb.Solver(w)
    w = W.tiny()
    w["darcy_grid"] = [(200, 8), (8, 8)]
    with pytest.raises(sfb.SfbError):
        sfb.Solver(w)


def test_workspace_size_grows_with_batch():
    sfb = _lib()
    s = sfb.Solver(W.medium())
    a = s.workspace_bytes(sfb.FP64, 10)
    b = s.workspace_bytes(sfb.FP64, 289)
    c = s.workspace_bytes(sfb.MIXED, 289)
    assert a < b and c < b


def test_basis_launch_shapes_and_options():
    """The launch-shape table the autotuner chooses from, and the options
    that steer it, are host logic: no kernel runs."""
    sfb = _lib()
    assert sfb.basis_launch_shape(sfb.MIXED, 0, 0) == (256, 4, 1, 0, 0)
    assert sfb.basis_launch_shape(sfb.MIXED, 0, 1) == (256, 3, 2, 0, 0)
    assert sfb.basis_launch_shape(sfb.MIXED, 0, 2) == (256, 3, 1, 1, 0)   # tensor-core form
    assert sfb.basis_launch_shape(sfb.MIXED, 0, 3) == (128, 7, 1, 0, 1)   # factor, then column chunks
    assert sfb.basis_launch_shape(sfb.MIXED, 1, 0) == (256, 1, 2, 0, 0)
    assert sfb.basis_launch_shape(sfb.MIXED, 1, 1) == (256, 2, 1, 0, 0)
    assert sfb.basis_launch_shape(sfb.MIXED, 1, 2) == (128, 2, 1, 0, 1)   # no tensor-core form beyond 64 cells
    assert sfb.basis_launch_shape(sfb.MIXED, 1, 3) is None
    assert sfb.basis_launch_shape(sfb.FP64, 0, 0) == (256, 2, 1, 0, 0)
    assert sfb.basis_launch_shape(sfb.FP64, 1, 0) == (512, 1, 1, 0, 0)
    assert sfb.basis_launch_shape(sfb.FP64, 1, 1) == (512, 1, 0, 0, 0)   # G_b from global memory
    assert sfb.basis_launch_shape(sfb.FP64, 0, 1) is None
    assert sfb.basis_launch_shape(sfb.MIXED, 0, 4) is None
    assert sfb.basis_launch_shape(sfb.MIXED, 0, -1) is None
    assert sfb.basis_launch_shape(5, 0, 0) is None
    s = sfb.Solver(W.tiny())
    for name, ok, bad in (("basis_autotune", (0, 1), (2, -1)), ("basis_graph", (0, 1), (0.5, 3)),
                          ("basis_shape", (0, 1, 2, 3), (4, 1.5, -1)), ("basis_persistent", (-1, 0, 1), (2, 0.5)),
                          ("basis_pipe_groups", (1, 2, 3, 4), (0, 5, 1.5))):
        for v in ok:
            s.set_option(name, v)
        for v in bad:
            with pytest.raises(sfb.SfbError):
                s.set_option(name, v)


def test_bad_kl_regions_and_rules_are_rejected():
    """Host-side checks of the region map, the mode sets and the anisotropic
    rule: each failure is an SfbError, not a crash."""
    sfb = _lib()
    bad = []
    w = W.kl_regions()
    w["kl"]["region_of"] = [0, 0, 0, 0]            # region 1 has no subdomain
    bad.append(w)
    w = W.kl_regions()
    w["kl"]["regions"] = [(0.0, 0.5, 0.0, 0.25), (0.0, 1.0, 0.25, 0.5)]   # subdomain 1 outside region 0
    bad.append(w)
    w = W.kl_regions()
    w["kl"]["region_of"] = [0, 0, 1, 2]            # no region 2
    bad.append(w)
    w = W.anisotropic()
    w["kl"]["modes"] = [(2, 2), (2, 2)]            # 4 modes for n_term 2
    bad.append(w)
    w = W.anisotropic()
    w["collocation"]["m"] = [2, 1, 3, 1, 2, 0]     # a 0-point rule
    bad.append(w)
    w = W.anisotropic()
    w["collocation"] = {"kind": "smolyak", "lmax": 1, "rule": [1, 3], "m": [2, 2, 2, 2, 2, 2]}
    bad.append(w)                                  # per-dimension sizes on a sparse grid
    for w in bad:
        with pytest.raises(sfb.SfbError):
            sfb.Solver(w)
    s = sfb.Solver(W.tiny())
    with pytest.raises(sfb.SfbError):
        s.kl_tables(5)


def test_calls_out_of_order_return_status_codes():
    """The C ABI's error conventions for calls made out of order or with bad
    arguments, all decided on the host before any device work: SFB_ERR_STATE
    (2) for a step before its prerequisite, SFB_ERR_WORKSPACE (4) without a
    workspace, SFB_ERR_ARG (1) for bad arguments. No exception crosses the
    ABI; each failure leaves a message."""
    import ctypes
    sfb = _lib()
    lib = sfb.load()
    s = sfb.Solver(W.tiny())
    h = s.h
    st = sfb.BasisStats()
    assert lib.sfb_build_stochastic_basis(h, sfb.MIXED, ctypes.byref(st)) == 4      # no workspace
    assert b"workspace" in lib.sfb_last_error(h)
    assert lib.sfb_build_stochastic_basis(h, 7, ctypes.byref(st)) == 1             # bad precision
    y, w = s.points()
    assert lib.sfb_interface_solve_batch(h, y.ctypes.data, w.ctypes.data, len(y), 0, 1e-10, 100,
                                         None, None) == 2                          # before any build
    assert lib.sfb_get_basis(h, 0, 0, None, None, None) == 2
    mean = np.zeros(s.field_size("darcy_p"))
    assert lib.sfb_moments(h, 0, mean.ctypes.data, mean.ctypes.data) == 2          # before any solve
    assert lib.sfb_set_option(h, b"no_such_option", 1.0) == 1
    assert lib.sfb_set_option(h, b"refine_tol", 2.0) == 1
    assert lib.sfb_set_option(h, b"cg_precond", 4.0) == 1
    n = ctypes.c_int64()
    assert lib.sfb_field_size(h, 9, ctypes.byref(n)) == 1
    nb = ctypes.c_size_t()
    assert lib.sfb_workspace_size(h, 5, 16, ctypes.byref(nb)) != 0                # bad precision
    assert lib.sfb_local_points(h, 7, None, None) == 1
    assert lib.sfb_build_basis_item_noalloc(h, 0, 99, 0, None, None, None) == 1    # no such item
