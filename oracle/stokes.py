"""Stokes subdomain solver: Taylor-Hood P2-P1 triangles (Section 6) for
Eqs. 2.2-2.4 with the Beavers-Joseph-Saffman condition Eq. 2.10 and
normal-stress mortar data on the Stokes-Darcy interface (Eqs. 5.1-5.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Weak form (Section 3.2): ``a(u, v) = 2 nu (D u, D v) + <nu alpha / sqrt(K_l)
u.tau, v.tau>_{Gamma_sd}``, ``b(v, q) = -(div v, q)``, right-hand side
``-<lambda, v.n>_{Gamma_sd}`` for mortar data ``lambda``. The Stokes subdomain
sits above the Darcy region, so on the interface ``n = (0, -1)`` and
``tau = (1, 0)``.

Readings of the paper taken here: A6 boundary data (parabolic inflow on the left,
no slip on top, zero stress on the right); A7 ``K_l = 1`` in the BJS term, so
the Stokes basis is deterministic; A8 every rectangle is split along its
SW-NE diagonal.

Node lattice: P2 nodes are the ``(2 Sx + 1) x (2 Sy + 1)`` half-step lattice,
node ``n = j * (2 Sx + 1) + i``; velocity DOF ``c * n_nodes + n`` for
component ``c``; P1 pressures live on the vertices, ``J * (Sx + 1) + I``.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mortar import lagrange_1d

_GL_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GL_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])
# edge-midpoint rule on a triangle: exact for quadratics
_TRI_Q = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
# 7-point rule on a triangle, exact for degree 5 (Radon's rule, as tabulated
# by Strang and Fix): barycentric points and weights (relative to the area)
_R7_A1, _R7_B1 = 0.059715871789770, 0.470142064105115
_R7_A2, _R7_B2 = 0.797426985353087, 0.101286507323456
_TRI_R7 = np.array([[1 / 3, 1 / 3, 1 / 3],
                    [_R7_A1, _R7_B1, _R7_B1], [_R7_B1, _R7_A1, _R7_B1], [_R7_B1, _R7_B1, _R7_A1],
                    [_R7_A2, _R7_B2, _R7_B2], [_R7_B2, _R7_A2, _R7_B2], [_R7_B2, _R7_B2, _R7_A2]])
_TRI_R7_W = np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3)


def _p2_values(L):
    """The six P2 basis functions (vertices 0..2, then edges 01, 12, 20) at
    barycentric point ``L``."""
    v = np.empty(6)
    for i in range(3):
        v[i] = L[i] * (2.0 * L[i] - 1.0)
    for k, (i, j) in enumerate(((0, 1), (1, 2), (2, 0))):
        v[3 + k] = 4.0 * L[i] * L[j]
    return v


def _p2_grads(L, gl):
    """Gradients of the six P2 basis functions (vertices 0..2, then edges
    01, 12, 20) at barycentric point ``L``; ``gl[i]`` = grad lambda_i."""
    g = np.empty((6, 2))
    for i in range(3):
        g[i] = (4.0 * L[i] - 1.0) * gl[i]
    for k, (i, j) in enumerate(((0, 1), (1, 2), (2, 0))):
        g[3 + k] = 4.0 * (L[j] * gl[i] + L[i] * gl[j])
    return g


class StokesSub:
    def __init__(self, rect, sx, sy, nu, alpha, u_in, k_bjs=1.0):
        self.rect, self.sx, self.sy = rect, sx, sy
        self.nu, self.alpha, self.u_in, self.k_bjs = nu, alpha, u_in, k_bjs
        # optional data of Eqs. 2.2-2.4 beyond the test cases' (zero force,
        # parabolic inflow): a body force f_s(x, y) -> (f_x, f_y), and a velocity
        # u(x, y) -> (u_x, u_y) imposed on the sides listed in dirichlet_sides
        self.force = None
        self.u_exact = None
        self.dirichlet_sides = ("left", "top")
        x0, x1, y0, y1 = rect
        self.hx, self.hy = (x1 - x0) / sx, (y1 - y0) / sy
        self.NX, self.NY = 2 * sx + 1, 2 * sy + 1
        self.n_nodes = self.NX * self.NY
        self.n_p = (sx + 1) * (sy + 1)
        self.ifaces = []
        self.dofs = []

    def finalize(self):
        dofs = []
        for itf in self.ifaces:
            dofs += itf.dofs()
        self.dofs = sorted(dofs)
        self.local = {g: i for i, g in enumerate(self.dofs)}

    def node(self, i, j):
        return j * self.NX + i

    def node_xy(self):
        x0, _, y0, _ = self.rect
        i, j = np.meshgrid(np.arange(self.NX), np.arange(self.NY))
        return x0 + i.ravel() * 0.5 * self.hx, y0 + j.ravel() * 0.5 * self.hy

    def triangles(self):
        """Yield (P2 node ids [v0, v1, v2, m01, m12, m20], pressure ids, vertex xy)."""
        x0, _, y0, _ = self.rect
        for J in range(self.sy):
            for I in range(self.sx):
                i, j = 2 * I, 2 * J
                sw, se = self.node(i, j), self.node(i + 2, j)
                ne, nw = self.node(i + 2, j + 2), self.node(i, j + 2)
                psw, pse = J * (self.sx + 1) + I, J * (self.sx + 1) + I + 1
                pne, pnw = (J + 1) * (self.sx + 1) + I + 1, (J + 1) * (self.sx + 1) + I
                xsw = (x0 + I * self.hx, y0 + J * self.hy)
                xse = (xsw[0] + self.hx, xsw[1])
                xne = (xsw[0] + self.hx, xsw[1] + self.hy)
                xnw = (xsw[0], xsw[1] + self.hy)
                # lower-right triangle (SW, SE, NE)
                yield ([sw, se, ne, self.node(i + 1, j), self.node(i + 2, j + 1),
                        self.node(i + 1, j + 1)], [psw, pse, pne], [xsw, xse, xne])
                # upper-left triangle (SW, NE, NW)
                yield ([sw, ne, nw, self.node(i + 1, j + 1), self.node(i + 1, j + 2),
                        self.node(i, j + 1)], [psw, pne, pnw], [xsw, xne, xnw])

    def assemble(self):
        """Velocity block ``A`` (``2 nu_s (D u, D v)`` plus the BJS term of Eq.
        2.10 on Gamma_sd) and divergence block ``B`` of the Taylor-Hood
        discretisation of Eqs. 2.2-2.4 (Section 3.3)."""
        nn = self.n_nodes
        ar, ac, av, br, bc, bv = [], [], [], [], [], []
        nu = self.nu
        for nodes, pids, xy in self.triangles():
            (xa, ya), (xb, yb), (xc, yc) = xy
            det = (xb - xa) * (yc - ya) - (xc - xa) * (yb - ya)
            area = 0.5 * abs(det)
            gl = np.array([[yb - yc, xc - xb], [yc - ya, xa - xc], [ya - yb, xb - xa]]) / det
            Ae = np.zeros((12, 12))
            Be = np.zeros((3, 12))
            for L in _TRI_Q:
                w = area / 3.0
                g = _p2_grads(L, gl)
                gx, gy = g[:, 0], g[:, 1]
                Ae[:6, :6] += w * nu * (2.0 * np.outer(gx, gx) + np.outer(gy, gy))
                Ae[6:, 6:] += w * nu * (2.0 * np.outer(gy, gy) + np.outer(gx, gx))
                Ae[:6, 6:] += w * nu * np.outer(gy, gx)   # v comp 0, u comp 1
                Ae[6:, :6] += w * nu * np.outer(gx, gy)   # v comp 1, u comp 0
                # b(v, q) = -(div v, q), q = lambda_k
                for k in range(3):
                    Be[k, :6] += -w * L[k] * gx
                    Be[k, 6:] += -w * L[k] * gy
            dofs = np.array(nodes + [nn + n for n in nodes])
            ar.append(np.repeat(dofs, 12)); ac.append(np.tile(dofs, 12)); av.append(Ae.ravel())
            br.append(np.repeat(pids, 12)); bc.append(np.tile(dofs, 3)); bv.append(Be.ravel())
        # BJS on the bottom edge: nu alpha / sqrt(K) u_x v_x
        coef = self.nu * self.alpha / np.sqrt(self.k_bjs)
        for I in range(self.sx):
            ids = [self.node(2 * I, 0), self.node(2 * I + 1, 0), self.node(2 * I + 2, 0)]
            t = 0.5 + 0.5 * _GL_X
            phi = lagrange_1d(2, t)
            M = (phi * (_GL_W * 0.5 * self.hx)) @ phi.T * coef
            ar.append(np.repeat(ids, 3)); ac.append(np.tile(ids, 3)); av.append(M.ravel())
        A = sp.csr_matrix((np.concatenate(av), (np.concatenate(ar), np.concatenate(ac))),
                          shape=(2 * nn, 2 * nn))
        B = sp.csr_matrix((np.concatenate(bv), (np.concatenate(br), np.concatenate(bc))),
                          shape=(self.n_p, 2 * nn))
        return A, B

    def neumann_matrix(self):
        """``N[i, l] = <xi_l, phi_i . n>_{Gamma_sd}`` over velocity DOFs ``i`` and
        the local mortar DOFs ``l``; the right-hand side of Eq. 5.1 for data
        ``lambda = sum c_l xi_l`` is ``-N c`` and the flux functional of a
        velocity ``u`` is ``<u.n, xi_l> = (N^T u)_l``."""
        nn = self.n_nodes
        x0 = self.rect[0]
        N = np.zeros((2 * nn, len(self.dofs)))
        for I in range(self.sx):
            xa, xb = x0 + I * self.hx, x0 + (I + 1) * self.hx
            ids = [self.node(2 * I, 0), self.node(2 * I + 1, 0), self.node(2 * I + 2, 0)]
            for q, nid in enumerate(ids):
                wfn = (lambda s, q=q: lagrange_1d(2, (s - xa) / (xb - xa))[q])
                for itf in self.ifaces:
                    vals = itf.integrate(xa, xb, wfn)
                    for a, g in enumerate(itf.dofs()):
                        N[nn + nid, self.local[g]] += -vals[a]   # n = (0, -1)
        return N

    def load(self):
        """Load vector ``(f_s, v)`` of the body force over the velocity DOFs
        (Eq. 2.2), by the 7-point degree-5 rule on every triangle; zero
        without a force."""
        nn = self.n_nodes
        F = np.zeros(2 * nn)
        if self.force is None:
            return F
        for nodes, _, xy in self.triangles():
            (xa, ya), (xb, yb), (xc, yc) = xy
            area = 0.5 * abs((xb - xa) * (yc - ya) - (xc - xa) * (yb - ya))
            for L, w in zip(_TRI_R7, _TRI_R7_W):
                x = L[0] * xa + L[1] * xb + L[2] * xc
                y = L[0] * ya + L[1] * yb + L[2] * yc
                fx, fy = self.force(np.array([x]), np.array([y]))
                phi = _p2_values(L) * (w * area)
                F[nodes] += phi * float(fx[0])
                F[[nn + n for n in nodes]] += phi * float(fy[0])
        return F

    def dirichlet(self):
        """Dirichlet DOFs and values: inflow ``u = (u_in 4 s (1 - s), 0)`` on the
        left edge (``s`` the normalised height), no slip on the top edge (the
        outer data of Section 6.1, reading A6); or, with ``u_exact`` set, that
        velocity on the sides in ``dirichlet_sides``."""
        nn = self.n_nodes
        mask = np.zeros(2 * nn, dtype=bool)
        val = np.zeros(2 * nn)
        if self.u_exact is not None:
            xs, ys = self.node_xy()
            ux, uy = self.u_exact(xs, ys)
            sel = {"left": [self.node(0, j) for j in range(self.NY)],
                   "right": [self.node(self.NX - 1, j) for j in range(self.NY)],
                   "top": [self.node(i, self.NY - 1) for i in range(self.NX)]}
            for side in self.dirichlet_sides:
                for n in sel[side]:
                    mask[n] = mask[nn + n] = True
                    val[n], val[nn + n] = ux[n], uy[n]
            return mask, val
        for j in range(self.NY):
            n = self.node(0, j)
            s = j / (self.NY - 1)
            mask[n] = mask[nn + n] = True
            val[n] = self.u_in * 4.0 * s * (1.0 - s)
        for i in range(self.NX):
            n = self.node(i, self.NY - 1)
            mask[n] = mask[nn + n] = True
            val[n] = val[nn + n] = 0.0
        return mask, val

    def system(self):
        if not hasattr(self, "_sys"):
            A, B = self.assemble()
            mask, val = self.dirichlet()
            nu_ = 2 * self.n_nodes
            M = sp.bmat([[A, B.T], [B, None]], format="csc")
            free = np.concatenate([np.where(~mask)[0], nu_ + np.arange(self.n_p)])
            dirv = np.where(mask)[0]
            lu = spla.splu(M[free][:, free].tocsc())
            self._sys = (M, free, dirv, val, lu)
        return self._sys

    def solve(self, f_u, dirichlet_on):
        """Solve Eqs. 5.1-5.2 / 5.3-5.4 for velocity load ``f_u`` (columns over
        velocity DOFs); Dirichlet values are the inflow data when
        ``dirichlet_on`` else zero. Returns full ``u`` and ``p``."""
        M, free, dirv, val, lu = self.system()
        nu_ = 2 * self.n_nodes
        f_u = np.atleast_2d(f_u.T).T
        ncol = f_u.shape[1]
        full = np.zeros((nu_ + self.n_p, ncol))
        rhs = np.zeros((nu_ + self.n_p, ncol))
        rhs[:nu_] = f_u
        if dirichlet_on:
            full[dirv] = val[dirv][:, None]
            rhs = rhs - M[:, dirv] @ full[dirv]
        # the discrete solution of the saddle-point system: the pivoted LU
        # solve, then one step of iterative refinement with the assembled
        # matrix (a 128 x 128 Taylor-Hood system leaves the pressure about
        # 1e-9 off after the LU solve alone, at a residual of 1e-13)
        x = lu.solve(rhs[free])
        A_ff = M[free][:, free]
        x = x + lu.solve(rhs[free] - A_ff @ x)
        full[free] = x
        return full[:nu_], full[nu_:]

    def flux_basis(self):
        """Stokes multiscale basis (Section 5.3 Step 2; Eqs. 5.1-5.4): for each
        local mortar DOF ``j`` the velocity response to normal stress ``xi_j``;
        ``Phi_s[l, j] = -<u(xi_j).n, xi_l>``,
        ``g_s[l] = <u_bar.n, xi_l>`` for the inflow-driven particular solution;
        ``U`` (velocity x (R+1)) and ``Pp`` (pressure x (R+1)) responses."""
        N = self.neumann_matrix()
        R = len(self.dofs)
        U, Pp = self.solve(-N, dirichlet_on=False)
        ub, pb = self.solve(np.zeros(2 * self.n_nodes), dirichlet_on=True)
        phi = -(N.T @ U)
        g = (N.T @ ub)[:, 0]
        return phi, g, np.column_stack([U, ub]), np.column_stack([Pp, pb])
