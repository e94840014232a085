"""Pins of the oracle's Taylor-Hood Stokes solver (Eqs. 2.2-2.4, BJS
Eq. 2.10, normal-stress data Eqs. 5.1-5.2): exact polynomial Stokes flows
that P2-P1 reproduces, and a slip flow that exercises the BJS term and the
mortar normal-stress load."""

import numpy as np
import pytest

from oracle.mortar import Interface
from oracle.stokes import StokesSub


def _nodal(st, fun):
    x, y = st.node_xy()
    return fun(x, y)


def _vertex_xy(st):
    x0, _, y0, _ = st.rect
    I, J = np.meshgrid(np.arange(st.sx + 1), np.arange(st.sy + 1))
    return x0 + I.ravel() * st.hx, y0 + J.ravel() * st.hy


@pytest.mark.parametrize("case", ["shear", "x2", "y2"])
def test_polynomial_stokes_flows_satisfy_interior_equations(case):
    """For divergence-free quadratic u with -2 nu div D(u) + grad p = 0 and
    linear p, the P2-P1 equations hold exactly at interior velocity DOFs and
    at every pressure DOF (a wrong sign, factor or transposed block fails)."""
    nu = 1.7
    st = StokesSub((0.1, 0.9, 0.3, 1.0), 5, 4, nu, 1.0, 0.0)
    if case == "shear":
        u = lambda x, y: (y ** 2, 0 * x)
        p = lambda x, y: 2 * nu * x
    elif case == "x2":
        u = lambda x, y: (x ** 2, -2 * x * y)
        p = lambda x, y: 2 * nu * x
    else:
        u = lambda x, y: (-2 * x * y, y ** 2)
        p = lambda x, y: 2 * nu * y
    A, B = st.assemble()
    ux, uy = _nodal(st, u)
    U = np.concatenate([ux, uy])
    P = p(*_vertex_xy(st))
    res_u = A @ U + B.T @ P
    res_p = B @ U
    assert np.abs(res_p).max() < 1e-12
    i, j = np.meshgrid(np.arange(st.NX), np.arange(st.NY))
    interior = ((i > 0) & (i < st.NX - 1) & (j > 0) & (j < st.NY - 1)).ravel()
    mask = np.concatenate([interior, interior])
    assert np.abs(res_u[mask]).max() < 1e-11
    assert np.abs(res_u[~mask]).max() > 1e-6    # boundary rows carry tractions


class _ThreeSideDirichlet(StokesSub):
    """Dirichlet data from an exact solution on left, top and right; BJS and
    normal stress remain on the bottom (the interface)."""

    def __init__(self, exact, *args, **kw):
        super().__init__(*args, **kw)
        self.exact = exact

    def dirichlet(self):
        nn = self.n_nodes
        mask = np.zeros(2 * nn, dtype=bool)
        val = np.zeros(2 * nn)
        x, y = self.node_xy()
        ux, uy = self.exact(x, y)
        i = np.tile(np.arange(self.NX), self.NY)
        j = np.repeat(np.arange(self.NY), self.NX)
        b = (i == 0) | (i == self.NX - 1) | (j == self.NY - 1)
        mask[:nn] = b; mask[nn:] = b
        val[:nn] = ux; val[nn:] = uy
        return mask, val


@pytest.mark.parametrize("deg", [1, 2])
def test_bjs_slip_flow_with_normal_stress_mortar(deg):
    """u = (a (1 + alpha (y - y0)), 0), p = p0 satisfies Stokes, BJS
    -2 nu (D(u) n).tau = nu alpha u.tau and -(T n).n = p0 on the bottom; the
    discrete solution with mortar data lambda = p0 reproduces it exactly."""
    nu, alpha, a, p0 = 0.8, 1.6, 0.9, 2.3
    rect = (0.0, 1.0, 0.5, 1.0)
    exact = lambda x, y: (a * (1.0 + alpha * (y - 0.5)), 0.0 * x)
    st = _ThreeSideDirichlet(exact, rect, 6, 5, nu, alpha, 0.0)
    itf = Interface("sd", "x", 0.0, 1.0, 4, deg, None, None, 0)
    st.ifaces.append(itf)
    st.finalize()
    N = st.neumann_matrix()
    c = np.full(len(st.dofs), p0)
    u, p = st.solve(-N @ c, dirichlet_on=True)
    ux, uy = _nodal(st, exact)
    assert np.allclose(u[:st.n_nodes, 0], ux, atol=1e-12)
    assert np.allclose(u[st.n_nodes:, 0], uy, atol=1e-12)
    assert np.allclose(p[:, 0], p0, atol=1e-11)


def test_stokes_flux_basis_symmetric_positive():
    st = StokesSub((0.0, 1.0, 0.5, 1.0), 6, 4, 1.0, 1.0, 1.0)
    for k in range(2):
        itf = Interface("sd", "x", 0.5 * k, 0.5 * (k + 1), 3, 1, None, None, 6 * k)
        st.ifaces.append(itf)
    st.finalize()
    phi, g, U, Pp = st.flux_basis()
    assert np.allclose(phi, phi.T, atol=1e-12 * np.abs(phi).max())
    ev = np.linalg.eigvalsh(phi)
    assert ev.min() > 1e-8 * ev.max()
    # the inflow drives a net downward normal velocity into the Darcy side
    assert np.abs(g).max() > 0
