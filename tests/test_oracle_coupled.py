"""Pins of the oracle's coupled problem and algorithms (Section 5): the
monolithic mortar system against the interface reduction, Methods S1, S2 and
S3 against each other, their solve counts against Eqs. 5.11-5.13 (with the
two extra solves per realization the paper counts), and the moments against
brute force over monolithic solves."""

import numpy as np
import pytest

import sfb_workloads as W
from oracle import coupled


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("wl", [
    W.tiny(),
    W.small_test(bottom_pressure=1.0, source=[0.5, -0.3, 0.2, 1.1]),
    W.small_test(nx=7, ny=9, px=3, py=1, n_sd=2, n_dd=3, degree=2, stokes=(9, 4)),
], ids=["tiny", "sources", "quadratic"])
def test_monolithic_equals_interface_reduction(wl):
    prob = coupled.Problem(wl)
    ys, _ = prob.grid()
    for y in ys[:3]:
        lam_d, S, g, bs = prob.interface_dense(y)
        lam_m, f_m = prob.monolithic(y)
        assert _rel(lam_d, lam_m) < 1e-10
        assert np.allclose(S, S.T, atol=1e-13 * np.abs(S).max())
        assert np.linalg.eigvalsh(S).min() > 0
        f_d = prob.recover(lam_d, bs)
        for k in f_d:
            assert _rel(f_d[k], f_m[k]) < 1e-10, k


def test_methods_agree_and_count_solves():
    wl = W.small_test(nx=6, ny=5, px=2, py=1, n_term=2, stokes=(6, 4),
                      collocation={"kind": "smolyak", "lmax": 1, "rule": "paper"})
    prob = coupled.Problem(wl)
    ys, ws = prob.grid()
    assert len(ys) == 2 * 4 + 1
    l1, it1, c1 = coupled.method_s1(prob, ys, rtol=1e-13)
    l2, it2, c2 = coupled.method_s2(prob, ys, rtol=1e-13)
    l3, it3, c3 = coupled.method_s3(prob, ys, rtol=1e-13)
    dense = np.array([prob.interface_dense(y)[0] for y in ys])
    for lam in (l1, l2, l3):
        assert _rel(lam, dense) < 1e-10
    assert np.all(it1 > 0) and np.all(it3 > 0)
    n_real = len(ys)
    for s, sub in enumerate(prob.subs):
        R = len(sub.dofs)
        loc, _ = prob.local_realizations(s, ys)
        assert c2[s] == (R + 2) * n_real                       # Eq. 5.12 + 2 extras
        assert c3[s] == R * len(loc) + 2 * n_real              # Eq. 5.13 + 2 extras
        assert c1[s] == it1.sum() + 2 * n_real                 # Eq. 5.11 + 2 extras
        assert c3[s] < c2[s]


def test_moments_brute_force_tiny():
    """Mean and variance over the 16 tensor points from one monolithic solve
    per point agree with the basis-driven pipeline."""
    prob = coupled.Problem(W.tiny())
    ys, ws = prob.grid()
    lams, mom = coupled.solve_all(prob, ys, ws)
    brute = {k: [] for k in mom}
    lam_m = []
    for y in ys:
        lam, f = prob.monolithic(y)
        lam_m.append(lam)
        for k in brute:
            brute[k].append(f[k])
    assert _rel(lams, lam_m) < 1e-10
    for k in mom:
        v = np.array(brute[k])
        mean = (ws[:, None] * v).sum(0)
        var = (ws[:, None] * (v - mean) ** 2).sum(0)
        assert _rel(mom[k][0], mean) < 1e-10, k
        assert _rel(mom[k][1], var) < 1e-8, k
    # the Stokes field is stochastic through the coupling (Section 6.2)
    assert mom["stokes_u"][1].max() > 0
    assert mom["darcy_p"][1].max() > 0


def test_moments_definition():
    rng = np.random.default_rng(5)
    v = rng.normal(size=(7, 4))
    w = rng.random(7)
    w /= w.sum()
    mean, var = coupled.moments(v, w)
    assert np.allclose(mean, sum(w[i] * v[i] for i in range(7)))
    assert np.allclose(var, sum(w[i] * v[i] ** 2 for i in range(7)) - mean ** 2)


def test_kl_region_spanning_subdomains_is_one_field():
    """A KL region that spans two subdomains (Section 2.1; Case 1 of Section
    6.1) carries one random field: on every cell its log-permeability equals
    that of a problem where the same rectangle is a single subdomain with
    the union's cells, for the same local coordinates. Evaluating the modes
    in each subdomain's own coordinates instead fails this."""
    wl = W.kl_regions()
    prob = coupled.Problem(wl)
    one = W.small_test(nx=16, ny=6, px=1, py=2, n_sd=2, n_dd=2, n_term=2, degree=1, stokes=(6, 5),
                       sigma2=1.0, eta=(0.2, 0.1))
    one["kl"]["n_term"] = [2, 3]
    one["kl"]["modes"] = [(2, 1), None]
    ref = coupled.Problem(one)
    rng = np.random.default_rng(7)
    for r, (left, right) in enumerate(((0, 1), (2, 3))):
        y = rng.normal(size=prob.n_term[r])
        whole = np.log(ref.permeability(r, y)).reshape(6, 16)
        assert np.allclose(np.log(prob.permeability(left, y)).reshape(6, 8), whole[:, :8], rtol=1e-13, atol=1e-13)
        assert np.allclose(np.log(prob.permeability(right, y)).reshape(6, 8), whole[:, 8:], rtol=1e-13, atol=1e-13)
    # subdomains of a region share its local realizations and dimensions
    ys, _ = prob.grid()
    assert ys.shape == (32, 5)
    for a, b in ((0, 1), (2, 3)):
        la, ka = prob.local_realizations(a, ys)
        lb, kb = prob.local_realizations(b, ys)
        assert np.array_equal(la, lb) and np.array_equal(ka, kb)


def test_methods_agree_on_shared_kl_regions():
    """Monolithic solve, dense interface reduction and Methods S1, S2, S3
    agree when KL regions span subdomains; S3's count of Eq. 5.13 uses the
    region's local realizations for each of its subdomains."""
    prob = coupled.Problem(W.kl_regions())
    ys, ws = prob.grid()
    sel = ys[::5]
    l1, it1, c1 = coupled.method_s1(prob, sel, rtol=1e-13)
    l2, _, c2 = coupled.method_s2(prob, sel, rtol=1e-13)
    l3, _, c3 = coupled.method_s3(prob, sel, rtol=1e-13)
    dense = np.array([prob.interface_dense(y)[0] for y in sel])
    mono = np.array([prob.monolithic(y)[0] for y in sel])
    assert _rel(dense, mono) < 1e-10
    for lam in (l1, l2, l3):
        assert _rel(lam, dense) < 1e-10
    for s, sub in enumerate(prob.subs):
        loc, _ = prob.local_realizations(s, sel)
        assert c3[s] == len(sub.dofs) * len(loc) + 2 * len(sel)


def _simpson_edge(u, h):
    """Integral along an edge of a continuous piecewise-quadratic function with
    nodal values ``u`` at the vertices and midpoints (2k+1 values, segments of
    length h): Simpson's rule, exact for quadratics."""
    u = np.asarray(u)
    return float(sum(h / 6.0 * (u[2 * k] + 4.0 * u[2 * k + 1] + u[2 * k + 2]) for k in range((len(u) - 1) // 2)))


@pytest.mark.parametrize("wl", [
    W.tiny(),
    W.small_test(nx=7, ny=9, px=3, py=1, n_sd=2, n_dd=3, degree=2, stokes=(9, 4)),
    W.small_test(nx=13, ny=9, px=3, py=2, n_sd=3, n_dd=2, n_term=2, degree=2, stokes=(7, 5)),
    W.kl_regions(),
], ids=["tiny", "quadratic", "ragged", "kl_regions"])
def test_global_mass_balance(wl):
    """Exact discrete conservation of the coupled scheme without sources: the
    Taylor-Hood pressure space holds the constants, so the Stokes boundary
    flux sums to zero; RT0 conserves mass cell by cell; and the mortar spaces
    hold a constant on every mortar element, so the interface fluxes cancel
    on each interface. Hence the Stokes inflow on the left equals the Stokes
    outflow on the right plus the Darcy outflow through the bottom, to solver
    precision, for every realization. A mortar projection that loses flux, a
    misplaced interface face or a wrong boundary face breaks it."""
    prob = coupled.Problem(wl)
    ys, _ = prob.grid()
    st = prob.stokes
    for y in ys[:3]:
        lam, f = prob.monolithic(y)
        u = f["stokes_u"]
        ux = u[:st.n_nodes].reshape(st.NY, st.NX)
        inflow = _simpson_edge(ux[:, 0], st.hy)
        out_right = _simpson_edge(ux[:, -1], st.hy)
        out_bottom, off = 0.0, 0
        for sub in prob.subs:
            n_ux = sub.ny * (sub.nx + 1)
            uy = f["darcy_flux"][off + n_ux: off + n_ux + (sub.ny + 1) * sub.nx].reshape(sub.ny + 1, sub.nx)
            if sub.rect[2] == wl["darcy_box"][2]:
                out_bottom += float(-uy[0, :].sum() * sub.hx)
            off += n_ux + (sub.ny + 1) * sub.nx
        assert inflow > 0.1 and out_bottom > 0.0 and out_right > 0.0
        assert abs(inflow - out_right - out_bottom) < 1e-11 * inflow, (inflow, out_right, out_bottom)
