"""Pins of the oracle's Darcy solver and mortar projections (Section 3.3,
Section 5.1 Eqs. 5.5-5.8, Section 5.3) against exact linear solutions, the
RT0 mixed system written out independently, and algebraic identities."""

import numpy as np
import pytest

from oracle.darcy import DarcySub
from oracle.mortar import Interface


def _sub_with_ifaces(rect, nx, ny, nu, n_el, deg, sides=("bottom", "right", "top", "left")):
    sub = DarcySub(0, rect, nx, ny, nu)
    x0, x1, y0, y1 = rect
    off = 0
    itfs = {}
    for s in sides:
        if s in ("bottom", "top"):
            itf = Interface("t", "x", x0, x1, n_el, deg, None, None, off)
        else:
            itf = Interface("t", "y", y0, y1, n_el, deg, None, None, off)
        off += itf.n_dof
        sub.sides[s] = ("iface", itf)
        itfs[s] = itf
    sub.finalize()
    return sub, itfs


def _nodal_coeffs(sub, itfs, fun, rect):
    """Mortar coefficients interpolating ``fun(x, y)`` at the mortar nodes."""
    x0, x1, y0, y1 = rect
    c = np.zeros(len(sub.dofs))
    for s, itf in itfs.items():
        h = (itf.s1 - itf.s0) / itf.n_el
        for e in range(itf.n_el):
            for a in range(itf.deg + 1):
                t = itf.s0 + (e + a / itf.deg) * h
                if s == "bottom":
                    xy = (t, y0)
                elif s == "top":
                    xy = (t, y1)
                elif s == "left":
                    xy = (x0, t)
                else:
                    xy = (x1, t)
                c[sub.local[itf.offset + e * (itf.deg + 1) + a]] = fun(*xy)
    return c


@pytest.mark.parametrize("deg", [1, 2])
def test_linear_pressure_reproduced_exactly(deg):
    """Constant K and linear p: the cell-centred scheme is exact at cell
    centres and the flux functional equals <-(K/nu) grad p . n, xi_l>; the
    mortar mesh (3 elements) does not match the 7x5 fine grid."""
    rect = (0.2, 0.7, 0.1, 0.4)
    K0, nu = 2.5, 1.3
    a, b, c = 0.7, -1.9, 3.1
    sub, itfs = _sub_with_ifaces(rect, 7, 5, nu, 3, deg)
    fun = lambda x, y: a + b * x + c * y
    coef = _nodal_coeffs(sub, itfs, fun, rect)
    K = np.full(sub.n_cells, K0)
    X, C = sub.solve(K, coef[:, None], with_particular=False)
    xc, yc = sub.cell_centres()
    assert np.allclose(X[:, 0], fun(xc, yc), atol=1e-13)
    flux = sub.interface_flux(K, X, C)[:, 0]
    grad = np.array([b, c])
    normals = {"bottom": (0, -1), "top": (0, 1), "left": (-1, 0), "right": (1, 0)}
    expect = np.zeros(len(sub.dofs))
    for s, itf in itfs.items():
        un = -(K0 / nu) * grad @ np.array(normals[s])
        ints = itf.integrate(itf.s0, itf.s1, lambda t: np.ones_like(t))
        for k, g in enumerate(itf.dofs()):
            expect[sub.local[g]] = un * ints[k]
    assert np.allclose(flux, expect, atol=1e-13)


def test_floating_subdomain_basis_annihilates_constants():
    rect = (0.0, 0.5, 0.0, 0.25)
    sub, itfs = _sub_with_ifaces(rect, 9, 6, 1.0, 2, 1)
    rng = np.random.default_rng(1)
    K = np.exp(rng.normal(0, 1.5, sub.n_cells))
    phi, g, X = sub.flux_basis(K)
    assert np.allclose(phi, phi.T, atol=1e-12 * np.abs(phi).max())
    assert np.allclose(phi @ np.ones(len(sub.dofs)), 0.0, atol=1e-11 * np.abs(phi).max())
    ev = np.linalg.eigvalsh(0.5 * (phi + phi.T))
    assert ev.min() > -1e-11 * ev.max()
    assert np.allclose(g, 0.0)


@pytest.mark.parametrize("n_el,deg", [(2, 1), (3, 2)])
def test_schur_complement_identity(n_el, deg):
    """Phi = P^T D_T P - B^T A^{-1} B (Section 5.1 reduction written densely).
    Phi is SPD when the mortar space is not richer than the face traces
    (2 linear elements on 5-6 faces); 3 quadratic elements (9 DOFs per side on
    5-6 faces) give a singular Phi."""
    rect = (0.0, 0.5, 0.0, 0.25)
    sub, itfs = _sub_with_ifaces(rect, 6, 5, 0.7, n_el, deg, sides=("right", "top", "left"))
    sub.sides["bottom"] = ("dirichlet", 0.0)
    rng = np.random.default_rng(7)
    K = np.exp(rng.normal(0, 2.0, sub.n_cells))
    phi, _, _ = sub.flux_basis(K)
    A, B, _ = sub.assemble(K)
    M = np.zeros_like(phi)
    for s in ("right", "top", "left"):
        p = sub.projection(s)
        M += p.T @ (sub.boundary_trans(K, s)[:, None] * p)
    ref = M - B.T @ np.linalg.solve(A.toarray(), B)
    assert np.allclose(phi, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    ev = np.linalg.eigvalsh(phi)
    if deg == 1:
        assert ev.min() > 1e-6 * ev.max()
    else:
        assert ev.min() < 1e-12 * ev.max()


def _rt0_trapezoid(nx, ny, rect, K, nu, q, side_vals):
    """Lowest-order RT mixed system on the rectangle grid with the trapezoidal
    rule for the velocity mass matrix, written out face by face: unknowns are
    the normal velocities of all faces (+x / +y orientation) and the cell
    pressures. ``side_vals[s]`` is a Dirichlet pressure or None (no flow)."""
    x0, x1, y0, y1 = rect
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    Kc = K.reshape(ny, nx)
    nfx, nfy = (nx + 1) * ny, nx * (ny + 1)
    nf, nc = nfx + nfy, nx * ny
    fx = lambda i, j: j * (nx + 1) + i          # x-face left of cell i
    fy = lambda i, j: nfx + j * nx + i          # y-face below cell (i, j)
    M = np.zeros((nf, nf)); Bd = np.zeros((nc, nf)); f = np.zeros(nf); g = np.zeros(nc)
    for j in range(ny):
        for i in range(nx):
            c = j * nx + i
            kinv = nu / Kc[j, i]
            # trapezoid: each face of the cell carries half the cell in its direction
            for e in (fx(i, j), fx(i + 1, j)):
                M[e, e] += kinv * hy * hx / 2.0
            for e in (fy(i, j), fy(i, j + 1)):
                M[e, e] += kinv * hx * hy / 2.0
            # b(v, w) = -(div v, w)
            Bd[c, fx(i + 1, j)] -= hy; Bd[c, fx(i, j)] += hy
            Bd[c, fy(i, j + 1)] -= hx; Bd[c, fy(i, j)] += hx
            g[c] = -q * hx * hy
    fixed = []
    for s, val in side_vals.items():
        if s == "left":
            faces, sign, length = [fx(0, j) for j in range(ny)], -1.0, hy
        elif s == "right":
            faces, sign, length = [fx(nx, j) for j in range(ny)], 1.0, hy
        elif s == "bottom":
            faces, sign, length = [fy(i, 0) for i in range(nx)], -1.0, hx
        else:
            faces, sign, length = [fy(i, ny) for i in range(nx)], 1.0, hx
        if val is None:
            fixed += faces
        else:
            for e in faces:
                f[e] -= val * sign * length    # -<g, v.n>
    free = np.setdiff1d(np.arange(nf), fixed)
    n = len(free)
    S = np.zeros((n + nc, n + nc))
    S[:n, :n] = M[np.ix_(free, free)]
    S[:n, n:] = Bd[:, free].T
    S[n:, :n] = Bd[:, free]
    rhs = np.concatenate([f[free], g])
    sol = np.linalg.solve(S, rhs)
    u = np.zeros(nf)
    u[free] = sol[:n]
    return sol[n:], u[:nfx].reshape(ny, nx + 1), u[nfx:].reshape(ny + 1, nx)


def test_ccfd_equals_rt0_with_trapezoid_rule():
    rect = (0.1, 0.6, 0.0, 0.3)
    nx, ny, nu, q = 5, 4, 1.7, 0.8
    rng = np.random.default_rng(3)
    K = np.exp(rng.normal(0, 1.0, nx * ny))
    vals = {"bottom": 1.5, "right": None, "top": -0.5, "left": 0.25}
    p_ref, ux_ref, uy_ref = _rt0_trapezoid(nx, ny, rect, K, nu, q, vals)
    sub = DarcySub(0, rect, nx, ny, nu, source=q)
    for s, v in vals.items():
        sub.sides[s] = ("noflow",) if v is None else ("dirichlet", v)
    sub.finalize()
    A, B, bbar = sub.assemble(K)
    p = np.linalg.solve(A.toarray(), bbar)
    assert np.allclose(p, p_ref, atol=1e-12)
    ux, uy = sub.fields(K, p, np.zeros(0))
    assert np.allclose(ux, ux_ref, atol=1e-12)
    assert np.allclose(uy, uy_ref, atol=1e-12)


def test_projection_is_face_average():
    """P[e, l] = face average of xi_l, also for faces cut by a breakpoint."""
    itf = Interface("t", "x", 0.0, 1.0, 3, 2, None, None, 0)
    faces = [(k / 8, (k + 1) / 8) for k in range(8)]
    P = itf.face_projection(faces)
    assert np.allclose(P.sum(1), 1.0)     # the basis sums to one on each element
    coef = np.zeros(itf.n_dof)
    h = 1.0 / 3.0
    for e in range(3):
        for a in range(3):
            t = (e + a / 2.0) * h
            coef[e * 3 + a] = t ** 2
    avg = np.array([(f1 ** 3 - f0 ** 3) / (3 * (f1 - f0)) for f0, f1 in faces])
    assert np.allclose(P @ coef, avg, atol=1e-14)


_NORMALS = {"bottom": (0, -1), "top": (0, 1), "left": (-1, 0), "right": (1, 0)}


@pytest.mark.parametrize("case", ["harmonic", "layered"])
def test_manufactured_solutions_converge_at_the_expected_orders(case):
    """Mesh refinement against exact solutions of div(K grad p) = 0 on the
    unit square, with quadratic mortars on all four sides (refined with the
    grid, 4 cells per mortar element):
    - "harmonic": K = 2, p = x^2 - y^2 + 0.3 x y, whose boundary trace the
      quadratic mortars hold exactly;
    - "layered": K = e^x, p = e^-x (K p_x is constant), K sampled at the
      cell centres.
    The cell-centre pressure converges at second order and the flux
    functionals <u.n, xi_l> at first order (the lowest-order RT flux), on
    grids of 8 to 64 cells per side. An inconsistent boundary
    transmissibility, projection or stencil stalls one of the rates."""
    nu = 1.0
    rect = (0.0, 1.0, 0.0, 1.0)
    if case == "harmonic":
        p = lambda x, y: x ** 2 - y ** 2 + 0.3 * x * y             # noqa: E731
        grad = lambda x, y: (2 * x + 0.3 * y, -2 * y + 0.3 * x)      # noqa: E731
        Kf = lambda x, y: np.full_like(x, 2.0)                       # noqa: E731
    else:
        p = lambda x, y: np.exp(-x) + 0 * y                          # noqa: E731
        grad = lambda x, y: (-np.exp(-x), 0 * y)                     # noqa: E731
        Kf = lambda x, y: np.exp(x) + 0 * y                          # noqa: E731
    e_p, e_f = [], []
    for n in (8, 16, 32, 64):
        sub, itfs = _sub_with_ifaces(rect, n, n, nu, n // 4, 2)
        coef = _nodal_coeffs(sub, itfs, p, rect)
        xc, yc = sub.cell_centres()
        K = Kf(xc, yc)
        X, C = sub.solve(K, coef[:, None], with_particular=False)
        e_p.append(np.abs(X[:, 0] - p(xc, yc)).max())
        flux = sub.interface_flux(K, X, C)[:, 0]
        expect = np.zeros(len(sub.dofs))
        for s, itf in itfs.items():
            nx_, ny_ = _NORMALS[s]

            def un(t, s=s, nx_=nx_, ny_=ny_):
                x, y = {"bottom": (t, 0.0 * t), "top": (t, 1.0 + 0.0 * t),
                        "left": (0.0 * t, t), "right": (1.0 + 0.0 * t, t)}[s]
                gx, gy = grad(x, y)
                return -(Kf(x, y) / nu) * (gx * nx_ + gy * ny_)
            if case == "harmonic":
                ints = itf.integrate(itf.s0, itf.s1, un)    # u.n is linear along each side
            else:
                # K p_x = -1 everywhere, so u.n is constant along each side
                c0 = float(un(np.array([0.5]))[0])
                ints = itf.integrate(itf.s0, itf.s1, lambda t, c0=c0: np.full_like(t, c0))
            for k, g in enumerate(itf.dofs()):
                expect[sub.local[g]] = ints[k]
        e_f.append(np.abs(flux - expect).max() / np.abs(expect).max())
    rate_p = [e_p[i] / e_p[i + 1] for i in range(3)]
    rate_f = [e_f[i] / e_f[i + 1] for i in range(3)]
    assert min(rate_p) > 3.3 and rate_p[-1] > 3.8, rate_p
    assert min(rate_f) > 1.9, rate_f
    assert e_p[-1] < 1e-4
