"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on the same inputs. FP64 form within 1e-10 relative, mixed form
(FP32 factor + FP64 refinement) within 1e-8 relative."""

import numpy as np
import pytest

from gpu_common import TOL, assert_close, make_workload, oracle_case, rel

pytestmark = pytest.mark.gpu

CASES = ["tiny", "ragged", "ragged_tensor", "medium", "anisotropic", "kl_regions", "paper_l2"]


def _solver(key, prec):
    import torch
    import paper_1802_06263_gb300 as sfb
    assert torch.cuda.is_available()
    s = sfb.Solver(make_workload(key))
    s.allocate(prec)
    st = s.build_basis(prec)
    return s, st


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", CASES)
def test_basis_parity(key, prec):
    p, y, wt, lams, mom = oracle_case(key)
    s, st = _solver(key, prec)
    tol = TOL[prec]
    worst = 0.0
    for i in range(len(p.subs)):
        loc = p.local_realizations(i, y)[0]
        for k in range(len(loc)):
            phi_o, g_o, X_o, _ = p.darcy_basis(i, loc[k])
            phi, g, X = s.get_basis(i, k, with_x=True)
            assert_close(phi, phi_o, tol, ("phi", i, k))
            assert_close(X, X_o, tol, ("X", i, k))
            assert_close(g, g_o, tol, ("g", i, k))
            worst = max(worst, rel(phi, phi_o), rel(X, X_o))
    phs, gs, _ = s.get_basis(-1, 0)
    phs_o, gs_o, _, _ = p.stokes_basis()
    assert_close(phs, phs_o, 1e-10, "Stokes phi")
    assert_close(gs, gs_o, 1e-10, "Stokes g")
    if prec == 1:
        assert st["max_first_correction"] > 0
    print(key, prec, "worst basis rel err", worst, st)


@pytest.mark.parametrize("krylov", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("key", CASES)
def test_interface_and_moments_parity(key, prec, krylov):
    """krylov 0: FP64 CG; 1: CG with FP32 products and FP64 residual
    replacement, which must reach the same FP64 residual tolerance; 2:
    restarted GMRES(30) in FP64, accepted on its FP64 true residual; 3: the
    same GMRES with FP32 Arnoldi products, restarted from FP64 residuals."""
    p, y, wt, lams, mom = oracle_case(key)
    s, _ = _solver(key, prec)
    rtol = 1e-14 if krylov == 0 else 1e-13
    lam, it, rc = s.solve_host(y, wt, rtol=rtol, max_it=5000, check=False, krylov=krylov)
    assert np.all(it != 0)
    tol = TOL[prec]
    for l in range(len(y)):
        assert_close(lam[l], lams[l], tol, ("lambda", l))
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], tol, (f, "mean"))
        assert_close(v, mom[f][1], tol, (f, "variance"))


def test_split_batches_accumulate_the_same_moments():
    """Moments over two half batches equal the moments over the full batch."""
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    h = len(y) // 2
    s.solve_host(y[:h], wt[:h], rtol=1e-14, max_it=5000)
    s.solve_host(y[h:], wt[h:], rtol=1e-14, max_it=5000)
    for f in ("darcy_p", "stokes_u"):
        m, v = s.moments(f)
        assert rel(m, mom[f][0]) < 1e-9
        assert rel(v, mom[f][1]) < 1e-8
    s.moments_reset()
    import paper_1802_06263_gb300 as sfb
    with pytest.raises(sfb.SfbError):
        s.moments("darcy_p")


def test_device_buffers_and_iteration_counts():
    import torch
    p, y, wt, lams, mom = oracle_case("tiny")
    s, _ = _solver("tiny", 0)
    yd = torch.tensor(y, device="cuda")
    wd = torch.tensor(wt, device="cuda")
    lam = torch.zeros((len(y), s.n_lambda), dtype=torch.float64, device="cuda")
    it = torch.zeros(len(y), dtype=torch.int32, device="cuda")
    s.solve(yd, wd, 1e-14, 100, lam, it)
    torch.cuda.synchronize()
    assert rel(lam.cpu().numpy(), lams) < 1e-10
    # CG on an N-dimensional SPD system converges in about N steps; rounding
    # at rtol = 1e-14 costs a few more
    assert it.cpu().numpy().max() <= 2 * s.n_lambda
    assert it.cpu().numpy().min() > 0


def test_not_converged_is_reported():
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    lam, it, rc = s.solve_host(y, wt, rtol=1e-14, max_it=2, check=False)
    assert rc == sfb.SFB_ERR_NOT_CONVERGED
    assert np.all(it == -2)


@pytest.mark.parametrize("krylov", [0, 1])
@pytest.mark.parametrize("precond", [0, 1, 2])
def test_cg_preconditioners_reach_the_same_solution(precond, krylov):
    """CG as the paper states it (no preconditioner), with the Jacobi and with
    the interface block-Jacobi preconditioner stop on the same
    unpreconditioned residual and give the same mortar solution and moments;
    each preconditioner in fewer iterations than the one before."""
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    s.set_option("cg_precond", precond)
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=krylov)
    assert rc == 0 and np.all(it > 0)
    assert rel(lam, lams) < 1e-9
    m, v = s.moments("darcy_flux")
    assert rel(m, mom["darcy_flux"][0]) < 1e-9
    assert rel(v, mom["darcy_flux"][1]) < 1e-8
    if precond < 2:
        s.set_option("cg_precond", precond + 1)
        _, it_next, _ = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=krylov)
        assert it_next.max() < it.max()


FIELD_NAMES = ("darcy_p", "darcy_flux", "stokes_u", "stokes_p")


@pytest.mark.parametrize("key,krylov,precond", [("medium", 0, 0), ("medium", 0, 1), ("medium", 0, 2),
                                                ("medium", 1, 0), ("medium", 1, 1), ("medium", 1, 2),
                                                ("ragged", 0, 1), ("ragged", 1, 1), ("tiny", 1, 2)])
def test_persistent_cg_matches_per_step_launches(key, krylov, precond):
    """The CG in one cooperative launch runs the same per-point and per-tile
    arithmetic in the same order as the loop of one launch per step: the
    mortar solutions, iteration counts and moments are bit-identical, with a
    handful of launches instead of two per iteration."""
    p, y, wt, lams, mom = oracle_case(key)
    s, _ = _solver(key, krylov)
    s.set_option("cg_precond", precond)
    res = {}
    for pers in (0, 1):
        s.set_option("cg_persistent", pers)
        s.moments_reset()
        n0 = s.launch_count()
        lam, it, rc = s.solve_host(y, wt, rtol=1e-12, max_it=5000, krylov=krylov)
        n_launch = s.launch_count() - n0
        res[pers] = (lam, it, rc, n_launch, s.solve_timings()["cg_iterations"],
                     {f: s.moments(f) for f in FIELD_NAMES})
    (l0, i0, r0, n0, c0, m0), (l1, i1, r1, n1, c1, m1) = res[0], res[1]
    assert r0 == 0 and r1 == 0 and np.all(i0 > 0)
    assert np.array_equal(l0, l1) and np.array_equal(i0, i1) and c0 == c1
    for f in FIELD_NAMES:
        assert np.array_equal(m0[f][0], m1[f][0]) and np.array_equal(m0[f][1], m1[f][1]), f
    assert rel(l1, lams) < 1e-9
    assert n0 > 2 * c0 and n1 < 30, (n0, n1, c0)


@pytest.mark.parametrize("factor", [1.0, 0.01])
def test_double_float_moments_match_fp64_contractions(factor):
    """After a mixed-form build the moments' contractions run in double-float
    (FP32 hi/lo pairs with error-free products and sums), about 1e-14 relative
    to the field values. The variances subtract the shift s, which scales that
    error by |v| / |v - s| (3e-12 measured on the face fluxes); both forms
    match the oracle. factor 0.01 sends every group through the quadratic
    forms."""
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 1)
    s.set_option("moments_group_factor", factor)
    res = {}
    for dfm in (0, 1):
        s.set_option("moments_double_float", dfm)
        s.moments_reset()
        s.solve_host(y, wt, rtol=1e-12, max_it=5000, krylov=1)
        res[dfm] = {f: s.moments(f) for f in FIELD_NAMES}
    for f in FIELD_NAMES:
        for j in (0, 1):
            assert rel(res[1][f][j], res[0][f][j]) < 1e-10, (f, j)
    assert rel(res[1]["darcy_flux"][0], mom["darcy_flux"][0]) < 1e-8
    assert rel(res[1]["darcy_p"][1], mom["darcy_p"][1]) < 1e-8


def test_persistent_cg_barrier_wait_runs_out_and_the_context_recovers():
    """Failure detection without a fault: with the test hook, CTA 0 of the
    one-launch CG skips its first grid barrier. The other CTAs' bounded waits
    run out after 1 s, set the abort word, and every CTA leaves; the solve
    reports SFB_ERR_TIMEOUT with the barrier named, and the next solve on the
    same context gives the same mortar solution as before."""
    import time
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    lam0, it0, rc0 = s.solve_host(y, wt, rtol=1e-12, max_it=5000, krylov=0)
    assert rc0 == 0
    s.set_option("cg_test_barrier_timeout", 1)
    s.moments_reset()
    t0 = time.time()
    _, _, rc = s.solve_host(y, wt, rtol=1e-12, max_it=5000, check=False, krylov=0)
    dt = time.time() - t0
    assert rc == sfb.SFB_ERR_TIMEOUT, rc
    assert "grid barrier" in s.lib.sfb_last_error(s.h).decode()
    assert 0.9 < dt < 60, dt
    s.moments_reset()
    lam1, it1, rc1 = s.solve_host(y, wt, rtol=1e-12, max_it=5000, krylov=0)
    assert rc1 == 0 and np.array_equal(lam1, lam0) and np.array_equal(it1, it0)


@pytest.mark.parametrize("m", [5, 30])
def test_gmres_restart_lengths_reach_the_same_solution(m):
    """GMRES(m) with a short restart (several cycles per point, each accepted
    or restarted on the FP64 true residual) and with the default 30 give the
    oracle's mortar solution; the short restart needs more Arnoldi steps. With
    no preconditioner GMRES is plain GMRES on S^l."""
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    its = {}
    for precond in (0, 2):
        s.set_option("cg_precond", precond)
        s.set_option("gmres_restart", m)
        s.moments_reset()
        lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.GMRES)
        assert rc == 0 and np.all(it > 0)
        for l in range(len(y)):
            assert_close(lam[l], lams[l], 1e-10, ("lambda", l))
        m_, v_ = s.moments("darcy_flux")
        assert_close(m_, mom["darcy_flux"][0], 1e-10, "mean")
        its[precond] = it.max()
    assert its[2] < its[0]   # the interface blocks help GMRES as they help CG
    if m == 5:
        assert its[0] > 5


def test_gmres_not_converged_is_reported():
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    s, _ = _solver("medium", 0)
    lam, it, rc = s.solve_host(y, wt, rtol=1e-14, max_it=3, check=False, krylov=sfb.GMRES)
    assert rc == sfb.SFB_ERR_NOT_CONVERGED
    assert np.all(it == -3)


@pytest.mark.parametrize("prec", [0, 1])
def test_method_s2_per_point_bases(prec):
    """Method S2 (Section 5.3): a multiscale flux basis built for every global
    point, with no reuse between points. The per-point local sets give each of
    the medium workload's 289 points its own items in every subdomain (289 x 4
    builds, the paper's N_S2 counts R + 2 subdomain solves per point and
    subdomain: R basis columns here, the particular column beside them, the
    recovery from the stored responses), and the same mortar solutions and
    moments as the oracle (and hence as Method S3)."""
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    w = make_workload("medium")
    w["collocation"] = dict(w["collocation"], local="per_point")
    s = sfb.Solver(w)
    assert s.n_pts == len(y) == 289
    for i in range(s.n_darcy):
        assert len(s.local_points(i)) == 289
    s.allocate(prec)
    st = s.build_basis(prec)
    assert st["n_items"] == 289 * 4
    assert st["n_flux_responses"] == 289 * sum(len(s.subdomain_dofs(i)) for i in range(4))
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=prec)
    assert rc == 0
    tol = TOL[prec]
    for l in range(len(y)):
        assert_close(lam[l], lams[l], tol, ("lambda", l))
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], tol, (f, "mean"))
        assert_close(v, mom[f][1], tol, (f, "variance"))


@pytest.mark.parametrize("case", ["tiny", "ragged", "paper_l2"])
def test_method_s1_against_the_oracle(case):
    """Method S1 (Section 5.2): FP64 block factors and the particular solution
    built once per local realization, then unpreconditioned FP64 CG whose
    Darcy products are one subdomain solve per (point, subdomain) and
    iteration. Against the oracle's own Method S1 (sparse LU solves inside
    CG): the mortar solutions within 1e-10; the CG iterations within three of
    each other (the two CGs round differently, and near rtol = 1e-13 that
    moves the last iterations: up to two were measured at 1e-12; the moments'
    flux entries at 1e-10 need the tighter rtol), so the solve counts
    of Section 5.2 (per Darcy subdomain the iterations plus the right-hand
    side and recovery solves of every point) within three per point; the
    moments agree with the oracle's Method S3 result, the same discrete
    solution."""
    import paper_1802_06263_gb300 as sfb
    from oracle import coupled
    p, y, wt, lams3, mom = oracle_case(case)
    lams1, its1, counts1 = coupled.method_s1(p, y, rtol=1e-13, max_it=5000)
    s = sfb.Solver(make_workload(case))
    s.allocate(sfb.FP64)
    st = s.build_basis(sfb.FACTOR_FP64)
    assert st["n_not_converged"] == 0 and st["n_flux_responses"] == 0
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.CG_DTN)
    assert rc == 0
    for l in range(len(y)):
        assert_close(lam[l], lams1[l], 1e-10, ("lambda", l))
        assert_close(lam[l], lams3[l], 1e-10, ("lambda vs S3", l))
    assert np.all(np.abs(it - its1) <= 3), (it, its1)
    n_gpu = int(np.sum(it)) + 2 * len(y)
    for sub in range(s.n_darcy):
        assert abs(n_gpu - int(counts1[sub])) <= 3 * len(y)
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], 1e-10, (f, "mean"))
        assert_close(v, mom[f][1], 1e-10, (f, "variance"))


@pytest.mark.parametrize("build", ["factor", "fp64"])
def test_method_s1_medium(build):
    """Method S1 on the medium workload (289 points, 4 subdomains of 32 x 32
    cells), from the factor-only build and from the full FP64 build (whose
    block factors it reuses): the mortar solutions and moments of the oracle
    within 1e-10, the CG iterations of Method S3's unpreconditioned FP64 CG
    on the same points within three (both apply the same operator, rounded
    differently), and the
    particular solutions' g equal to the full build's."""
    import paper_1802_06263_gb300 as sfb
    p, y, wt, lams, mom = oracle_case("medium")
    s = sfb.Solver(make_workload("medium"))
    s.allocate(sfb.FP64)
    s.set_option("cg_precond", 0)
    s.build_basis(sfb.FP64)
    g_full = [s.get_basis(i, 0)[1] for i in range(s.n_darcy)]
    _, it3, rc3 = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.CG)
    assert rc3 == 0
    if build == "factor":
        st = s.build_basis(sfb.FACTOR_FP64)
        assert st["n_items"] > 0 and st["n_not_converged"] == 0
        for i in range(s.n_darcy):
            phi, g, x = s.get_basis(i, 0, with_x=True)
            assert phi is None
            assert_close(g, g_full[i], 1e-12, ("g", i))
    s.moments_reset()
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.CG_DTN)
    assert rc == 0
    for l in range(len(y)):
        assert_close(lam[l], lams[l], 1e-10, ("lambda", l))
    assert np.all(np.abs(it - it3) <= 3)
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], 1e-10, (f, "mean"))
        assert_close(v, mom[f][1], 1e-10, (f, "variance"))


def test_method_s1_state_checks():
    """The factor-only build forms no flux basis: the basis-product solvers
    refuse it (SFB_ERR_STATE), and so does Method S1 after a mixed build,
    which stores FP32 factors."""
    import paper_1802_06263_gb300 as sfb
    s = sfb.Solver(make_workload("tiny"))
    y, wt = s.points()
    s.allocate(sfb.FP64)
    s.build_basis(sfb.FACTOR_FP64)
    for kr in (sfb.CG, sfb.CG_MIXED, sfb.GMRES, sfb.GMRES_MIXED):
        _, _, rc = s.solve_host(y, wt, krylov=kr, check=False)
        assert rc == 2
    s.build_basis(sfb.MIXED)
    _, _, rc = s.solve_host(y, wt, krylov=sfb.CG_DTN, check=False)
    assert rc == 2
    s.build_basis(sfb.FP64)
    lam, it, rc = s.solve_host(y, wt, rtol=1e-12, krylov=sfb.CG_DTN)
    assert rc == 0 and np.all(it > 0)


@pytest.mark.parametrize("case", ["tiny", "medium", "ragged", "kl_regions"])
@pytest.mark.parametrize("prec", [0, 1])
def test_balancing_preconditioner(case, prec):
    """The balancing Neumann-Neumann preconditioner (cg_precond = 3, FP64 CG)
    that Section 7 suggests: the oracle's mortar solutions and moments within
    the form's tolerance, the oracle's balanced-CG iteration counts within two
    on sampled points, and fewer iterations than the interface block-Jacobi
    preconditioner on every point. After a mixed build the operator and the
    pseudo-inverses come from the FP64 bases refined from FP32 factors."""
    import paper_1802_06263_gb300 as sfb
    from oracle import balancing
    p, y, wt, lams, mom = oracle_case(case)
    s = sfb.Solver(make_workload(case))
    s.allocate(sfb.FP64)
    s.build_basis(prec)
    s.set_option("cg_precond", 2)
    _, it2, rc2 = s.solve_host(y, wt, rtol=1e-13, max_it=5000, krylov=sfb.CG)
    assert rc2 == 0
    s.set_option("cg_precond", 3)
    s.moments_reset()
    # after a mixed build the bases are symmetric, and a floating item's null
    # space the constants, only to the refinement's stopping estimate of 1e-11
    # (an estimate: single items stop a little above it): the balanced CG then
    # stalls near 1e-11 on some points, and its tolerance is 1e-10
    lam, it, rc = s.solve_host(y, wt, rtol=1e-13 if prec == 0 else 1e-10, max_it=5000, krylov=sfb.CG)
    assert rc == 0 and np.all(it > 0)
    tol = TOL[prec]
    for l in range(len(y)):
        assert_close(lam[l], lams[l], tol, ("lambda", l))
    for f in ("darcy_p", "darcy_flux", "stokes_u", "stokes_p"):
        m, v = s.moments(f)
        assert_close(m, mom[f][0], tol, (f, "mean"))
        assert_close(v, mom[f][1], tol, (f, "variance"))
    assert np.all(it <= it2), (it, it2)
    if prec == 0:
        for l in sorted({0, len(y) // 2, len(y) - 1}):
            _, ito = balancing.solve_point(p, y[l], rtol=1e-13, max_it=500)
            assert abs(int(it[l]) - ito) <= 2, (l, it[l], ito)


def test_balancing_preconditioner_solver_checks():
    """cg_precond = 3 runs with SFB_CG: the mixed CG and GMRES refuse it
    (SFB_ERR_ARG); Method S1 ignores it (its CG is unpreconditioned)."""
    import paper_1802_06263_gb300 as sfb
    s = sfb.Solver(make_workload("tiny"))
    y, wt = s.points()
    s.allocate(sfb.FP64)
    s.build_basis(sfb.FP64)
    s.set_option("cg_precond", 3)
    for kr in (sfb.CG_MIXED, sfb.GMRES, sfb.GMRES_MIXED):
        _, _, rc = s.solve_host(y, wt, krylov=kr, check=False)
        assert rc == 1
    _, it, rc = s.solve_host(y, wt, rtol=1e-12, krylov=sfb.CG_DTN)
    assert rc == 0 and np.all(it > 0)
