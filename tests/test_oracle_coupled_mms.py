"""Oracle pin: a manufactured solution of the coupled Stokes-Darcy problem
with constant permeability (Section 2: Stokes Eqs. 2.2-2.4, Darcy Eqs.
2.5-2.7, interface conditions Eqs. 2.8-2.10), solved by the oracle's
monolithic mortar system (Eqs. 4.2-4.4) on refined grids and mortars.

The exact solution is written down here, independently of the oracle's
assembly. With t = y - 1/2 (the interface at t = 0, Stokes above, Darcy
below), nu_s = nu_d = K = alpha = 1:

  Stokes: u = (phi chi', -phi' chi) from the stream function phi(x) chi(t),
          phi = sin(pi x), chi = cos(pi t) + sin(pi t) / 2 + (pi / 4) t^2,
          p_s = cos(pi x) (1 - pi^2 + t), body force f = -Lap u + grad p_s;
  Darcy:  p_d = cos(pi x) (cosh(pi t) + sinh(pi t)) (harmonic: q_d = 0),
          u_d = -grad p_d.

It satisfies the interface conditions exactly (no interface data needed):
u_s.n_s + u_d.n_d = 0 (u_2 = -pi cos(pi x) on both sides at t = 0); the normal
stress p_s - 2 d_t u_2 = p_d (both cos(pi x) at t = 0); BJS
d_t u_1 + d_x u_2 = alpha u_1 (both (pi / 2) sin(pi x)). Outer data: Darcy
pressure p_d on the bottom, left and right, Stokes velocity u on the left, top
and right.

Grids: two Darcy subdomains of n x n cells under a Stokes grid of 2n x n
rectangles (each two Taylor-Hood triangles), mortar meshes refined with them
(H proportional to h: n / 2 linear or n / 4 quadratic elements per edge).
Checked: the observed orders of convergence of the Darcy pressure, the Darcy
normal velocities and the Stokes velocity (see the test's docstring).
"""

import numpy as np
import pytest

import sfb_workloads as W

PI = np.pi


def chi(t):
    return np.cos(PI * t) + 0.5 * np.sin(PI * t) + 0.25 * PI * t * t


def dchi(t):
    return -PI * np.sin(PI * t) + 0.5 * PI * np.cos(PI * t) + 0.5 * PI * t


def d2chi(t):
    return -PI * PI * np.cos(PI * t) - 0.5 * PI * PI * np.sin(PI * t) + 0.5 * PI


def d3chi(t):
    return PI ** 3 * np.sin(PI * t) - 0.5 * PI ** 3 * np.cos(PI * t)


def u_exact(x, y):
    t = y - 0.5
    return np.sin(PI * x) * dchi(t), -PI * np.cos(PI * x) * chi(t)


def p_stokes(x, y):
    return np.cos(PI * x) * (1.0 - PI * PI + (y - 0.5))


def force(x, y):
    """f = -Lap u + grad p_s."""
    t = y - 0.5
    s, c = np.sin(PI * x), np.cos(PI * x)
    lap1 = -PI * PI * s * dchi(t) + s * d3chi(t)                  # u_1 = s chi'
    # u_2 = -pi c chi: Lap u_2 = -pi (-pi^2 c chi + c chi'')
    lap2 = -PI * (-PI * PI * c * chi(t) + c * d2chi(t))
    gx = -PI * s * (1.0 - PI * PI + t)
    gy = c
    return -lap1 + gx, -lap2 + gy


def p_darcy(x, y):
    t = y - 0.5
    return np.cos(PI * x) * (np.cosh(PI * t) + np.sinh(PI * t))


def u_darcy(x, y):
    t = y - 0.5
    return (PI * np.sin(PI * x) * (np.cosh(PI * t) + np.sinh(PI * t)),
            -PI * np.cos(PI * x) * (np.sinh(PI * t) + np.cosh(PI * t)))


def test_exact_solution_satisfies_the_interface_conditions():
    """Independent check of the construction (finite differences, not the
    derivative formulas above): divergence-free Stokes velocity, harmonic
    Darcy pressure, and the three conditions on t = 0."""
    x = np.linspace(0.05, 0.95, 7)
    e = 1e-5
    y0 = np.full_like(x, 0.5)
    ux, uy = u_exact(x, y0)
    # mass: u_s.n_s + u_d.n_d = 0 with n_s = (0, -1), n_d = (0, 1)
    _, udy = u_darcy(x, y0)
    assert np.allclose(-uy + udy, 0.0, atol=1e-12)
    # normal stress: p_s - 2 d_y u_2 = p_d
    dy_u2 = (u_exact(x, y0 + e)[1] - u_exact(x, y0 - e)[1]) / (2 * e)
    assert np.allclose(p_stokes(x, y0) - 2.0 * dy_u2, p_darcy(x, y0), atol=1e-8)
    # BJS: d_y u_1 + d_x u_2 = alpha u_1
    dy_u1 = (u_exact(x, y0 + e)[0] - u_exact(x, y0 - e)[0]) / (2 * e)
    dx_u2 = (u_exact(x + e, y0)[1] - u_exact(x - e, y0)[1]) / (2 * e)
    assert np.allclose(dy_u1 + dx_u2, ux, atol=1e-8)
    assert np.abs(ux).max() > 0.5   # the interface slip is not trivially zero
    # interior: div u = 0, Lap p_d = 0, and -Lap u + grad p = f by differences
    xx, yy = np.meshgrid(np.linspace(0.1, 0.9, 5), np.linspace(0.6, 0.9, 4))
    xx, yy = xx.ravel(), yy.ravel()
    div = ((u_exact(xx + e, yy)[0] - u_exact(xx - e, yy)[0]) + (u_exact(xx, yy + e)[1] - u_exact(xx, yy - e)[1])) / (2 * e)
    assert np.abs(div).max() < 1e-7
    h = 1e-3
    for comp in (0, 1):
        lap = (u_exact(xx + h, yy)[comp] + u_exact(xx - h, yy)[comp] + u_exact(xx, yy + h)[comp]
               + u_exact(xx, yy - h)[comp] - 4.0 * u_exact(xx, yy)[comp]) / h ** 2
        gp = ((p_stokes(xx + e, yy) - p_stokes(xx - e, yy)) if comp == 0
              else (p_stokes(xx, yy + e) - p_stokes(xx, yy - e))) / (2 * e)
        assert np.allclose(-lap + gp, force(xx, yy)[comp], atol=1e-4)
    yd = yy - 0.5
    lapd = (p_darcy(xx + h, yd) + p_darcy(xx - h, yd) + p_darcy(xx, yd + h) + p_darcy(xx, yd - h)
            - 4.0 * p_darcy(xx, yd)) / h ** 2
    assert np.abs(lapd).max() < 1e-4


def test_triangle_rule_is_exact_to_degree_five():
    """The 7-point triangle rule of the Stokes load vector integrates
    x^a y^b, a + b <= 5, exactly on the reference triangle (closed form
    a! b! / (a + b + 2)!)."""
    from math import factorial
    from oracle.stokes import _TRI_R7, _TRI_R7_W
    for a in range(6):
        for b in range(6 - a):
            # reference triangle (0,0), (1,0), (0,1): x = L1, y = L2, area 1/2
            q = 0.5 * sum(w * L[1] ** a * L[2] ** b for L, w in zip(_TRI_R7, _TRI_R7_W))
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert abs(q - exact) < 1e-14, (a, b)


def _solve(n, deg):
    from oracle import coupled
    # mortar elements per edge: n / 2 linear or n / 4 quadratic ones, so that
    # the mortar DOFs of an edge stay below its n faces (the traces must
    # control the mortar space, else the interface system is singular)
    n_el = max(1, n // (2 * deg))
    w = W.small_test(nx=n, ny=n, px=2, py=1, n_sd=n_el, n_dd=n_el, n_term=1, degree=deg, stokes=(2 * n, n))
    p = coupled.Problem(w)
    for sub in p.subs:
        sub.sides["bottom"] = ("dirichlet", p_darcy)
        if sub.sides["left"][0] != "iface":
            sub.sides["left"] = ("dirichlet", p_darcy)
        if sub.sides["right"][0] != "iface":
            sub.sides["right"] = ("dirichlet", p_darcy)
    st = p.stokes
    st.force = force
    st.u_exact = u_exact
    st.dirichlet_sides = ("left", "top", "right")
    lam, f = p.monolithic(np.zeros(p.n_dim))   # y = 0: K = exp(E[Y]) = 1 everywhere
    # Darcy pressure at cell centres, normal velocity at face midpoints
    ep, ef, sp_, sf = [], [], [], []
    off_p = off_f = 0
    for sub in p.subs:
        xc, yc = sub.cell_centres()
        pe = p_darcy(xc, yc)
        ph = f["darcy_p"][off_p:off_p + sub.n_cells]
        ep.append(ph - pe)
        sp_.append(pe)
        off_p += sub.n_cells
        x0, x1, y0, y1 = sub.rect
        nfx = sub.ny * (sub.nx + 1)
        nfy = (sub.ny + 1) * sub.nx
        uxh = f["darcy_flux"][off_f:off_f + nfx]
        uyh = f["darcy_flux"][off_f + nfx:off_f + nfx + nfy]
        off_f += nfx + nfy
        xs, ys = np.meshgrid(x0 + np.arange(sub.nx + 1) * sub.hx, y0 + (np.arange(sub.ny) + 0.5) * sub.hy)
        uxe = u_darcy(xs.ravel(), ys.ravel())[0]
        xs, ys = np.meshgrid(x0 + (np.arange(sub.nx) + 0.5) * sub.hx, y0 + np.arange(sub.ny + 1) * sub.hy)
        uye = u_darcy(xs.ravel(), ys.ravel())[1]
        ef.append(np.concatenate([uxh - uxe, uyh - uye]))
        sf.append(np.concatenate([uxe, uye]))
    xs, ys = st.node_xy()
    ue = np.concatenate(u_exact(xs, ys))
    eu = f["stokes_u"] - ue
    rel = lambda e, s: np.linalg.norm(np.concatenate(e)) / np.linalg.norm(np.concatenate(s))
    return rel(ep, sp_), rel(ef, sf), np.linalg.norm(eu) / np.linalg.norm(ue)


@pytest.mark.slow
@pytest.mark.parametrize("deg", [1, 2])
def test_coupled_manufactured_solution_converges(deg):
    """Errors of the oracle's coupled solution against the exact one on
    n = 4, 8, 16 (Darcy cells per subdomain side; Stokes 2n x n; mortar
    elements per edge as in _solve). Observed: the RT0 pressure at the cell
    centres converges at second order (the cell-centred scheme's
    superconvergence on uniform grids; first order is all the L2 theory
    gives); the normal velocities at the face midpoints, interface faces
    included, at the mortar's order H^(m + 1/2) (1.5 for linear, about 1.75
    for quadratic mortars in this range); the Taylor-Hood velocity at the P2
    nodes at second order or better. A dropped term, a wrong sign or a
    transposed operand anywhere in the coupled assembly stops the
    convergence altogether."""
    errs = [_solve(n, deg) for n in (4, 8, 16)]
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    print("deg", deg, "errors", errs.tolist(), "orders", orders.tolist())
    assert np.all(orders[:, 0] >= 1.8), orders                         # Darcy pressure
    assert np.all(orders[:, 1] >= (1.4 if deg == 1 else 1.6)), orders   # Darcy normal velocity
    assert np.all(orders[:, 2] >= 1.9), orders                         # Stokes velocity
    assert errs[-1, 0] < 2e-3 and errs[-1, 1] < 1e-2 and errs[-1, 2] < 1e-4, errs[-1]
