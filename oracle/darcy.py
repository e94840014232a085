"""Darcy subdomain solver: lowest-order Raviart-Thomas on a uniform rectangle
grid with the trapezoidal rule for the velocity mass matrix, which reduces to
the cell-centred 5-point scheme with harmonic-mean transmissibilities
(Section 6: RT on quadrilaterals; Darcy law Eqs. 2.5-2.7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The subdomain problems are those of Section 5.1: Eqs. 5.5-5.6 (interface
pressure ``lambda`` as Dirichlet data, no source, zero outer data) and
Eqs. 5.7-5.8 (zero interface pressure, the source ``q_d`` and the outer
boundary data). The Dirichlet data reach the fine faces through the L2
projection onto the normal-trace space, i.e. face averages of the mortar
function (Section 5.2, step 1). The flux functional ``<u.n, xi_l>`` of a
face flux ``F_e`` (outward, integrated over the face) is ``sum_e F_e P[e, l]``.

Cell ``c = iy * nx + ix``; x-faces are ``(ny, nx+1)`` arrays, y-faces
``(ny+1, nx)`` arrays, both of normal velocity in the +x / +y direction.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

SIDES = ("bottom", "right", "top", "left")


_G3_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_G3_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


class DarcySub:
    """Geometry and boundary description of one Darcy subdomain.

    ``sides[s]`` is ``("iface", Interface)``, ``("noflow",)`` or
    ``("dirichlet", value)``; ``value`` is a constant or a function of the
    point ``(x, y)`` on the side (the outer pressure data of Eqs. 2.5-2.7,
    entering through its face averages). ``source`` is the constant ``q_d``
    or a function ``q_d(x, y)``, entering through its cell integrals. ``dofs``
    are the subdomain's mortar DOFs (sorted global indices); ``R_i`` of the
    paper is the restriction to them.
    """

    def __init__(self, sid, rect, nx, ny, nu, source=0.0):
        self.sid, self.rect, self.nx, self.ny, self.nu = sid, rect, nx, ny, nu
        x0, x1, y0, y1 = rect
        self.hx, self.hy = (x1 - x0) / nx, (y1 - y0) / ny
        self.source = source
        self.sides = {s: ("noflow",) for s in SIDES}
        self.dofs = []

    def finalize(self):
        dofs = []
        for s in SIDES:
            if self.sides[s][0] == "iface":
                dofs += self.sides[s][1].dofs()
        self.dofs = sorted(dofs)
        self.local = {g: i for i, g in enumerate(self.dofs)}

    @property
    def n_cells(self):
        return self.nx * self.ny

    def cell_centres(self):
        x0, _, y0, _ = self.rect
        ix, iy = np.meshgrid(np.arange(self.nx), np.arange(self.ny))
        return (x0 + (ix.ravel() + 0.5) * self.hx, y0 + (iy.ravel() + 0.5) * self.hy)

    def side_faces(self, side):
        """Cells adjacent to ``side`` and the fine faces as coordinate intervals
        along the side, in increasing coordinate."""
        x0, x1, y0, y1 = self.rect
        nx, ny = self.nx, self.ny
        if side == "bottom":
            cells = np.arange(nx)
            faces = [(x0 + i * self.hx, x0 + (i + 1) * self.hx) for i in range(nx)]
        elif side == "top":
            cells = (ny - 1) * nx + np.arange(nx)
            faces = [(x0 + i * self.hx, x0 + (i + 1) * self.hx) for i in range(nx)]
        elif side == "left":
            cells = np.arange(ny) * nx
            faces = [(y0 + j * self.hy, y0 + (j + 1) * self.hy) for j in range(ny)]
        else:
            cells = np.arange(ny) * nx + nx - 1
            faces = [(y0 + j * self.hy, y0 + (j + 1) * self.hy) for j in range(ny)]
        return cells, faces

    def source_integrals(self):
        """Cell integrals of the source ``q_d`` (3 x 3 Gauss-Legendre per cell
        for a function; ``q_d h_x h_y`` for a constant): the right-hand side of
        the mass balance Eq. 2.7 in cell-centred form."""
        if not callable(self.source):
            return np.full(self.n_cells, self.source * self.hx * self.hy)
        xc, yc = self.cell_centres()
        tot = np.zeros(self.n_cells)
        for a, wa in zip(_G3_X, _G3_W):
            for b, wb in zip(_G3_X, _G3_W):
                tot += wa * wb * self.source(xc + 0.5 * a * self.hx, yc + 0.5 * b * self.hy)
        return tot * 0.25 * self.hx * self.hy

    def dirichlet_values(self, side):
        """Face averages of a side's Dirichlet pressure (3-point Gauss-Legendre
        per face for a function, the constant itself otherwise)."""
        val = self.sides[side][1]
        cells, faces = self.side_faces(side)
        if not callable(val):
            return np.full(len(cells), float(val))
        x0, x1, y0, y1 = self.rect
        out = np.zeros(len(faces))
        for q, (a, b) in enumerate(faces):
            s = 0.5 * (a + b) + 0.5 * (b - a) * _G3_X
            if side == "bottom":
                v = val(s, np.full(3, y0))
            elif side == "top":
                v = val(s, np.full(3, y1))
            elif side == "left":
                v = val(np.full(3, x0), s)
            else:
                v = val(np.full(3, x1), s)
            out[q] = 0.5 * (_G3_W @ v)
        return out

    def boundary_trans(self, K, side):
        """Half-cell transmissibility ``2 K |e| / (nu h_perp)`` of the faces of a
        side (RT0 + trapezoid on the half cell next to the boundary; the
        lowest-order RT discretisation of Section 3.3 for Eqs. 2.5-2.7)."""
        cells, _ = self.side_faces(side)
        if side in ("bottom", "top"):
            return 2.0 * K[cells] * self.hx / (self.nu * self.hy)
        return 2.0 * K[cells] * self.hy / (self.nu * self.hx)

    def interior_trans(self, K):
        """Interior transmissibilities ``(|e|/h) 2 / (nu (1/K_a + 1/K_b))``
        (harmonic mean of the two cell permeabilities: RT0 with the trapezoidal
        rule on the two half cells, Section 3.3)."""
        Kc = K.reshape(self.ny, self.nx)
        tx = (self.hy / self.hx) * 2.0 / (self.nu * (1.0 / Kc[:, :-1] + 1.0 / Kc[:, 1:]))
        ty = (self.hx / self.hy) * 2.0 / (self.nu * (1.0 / Kc[:-1, :] + 1.0 / Kc[1:, :]))
        return tx, ty

    def projection(self, side):
        """``P`` of one interface side restricted to the subdomain's local
        mortar DOFs, ``(n_faces, len(dofs))``: the L2 projection of the mortar
        basis onto the normal traces (Section 5.2, step 1 of the S_H action)."""
        kind = self.sides[side]
        _, faces = self.side_faces(side)
        p = np.zeros((len(faces), len(self.dofs)))
        if kind[0] == "iface":
            itf = kind[1]
            pl = itf.face_projection(faces)
            for a, g in enumerate(itf.dofs()):
                p[:, self.local[g]] = pl[:, a]
        return p

    def assemble(self, K):
        """5-point matrix ``A`` (sparse), interface RHS block ``B = E^T D_T P``
        (``n_cells x R``) and the particular RHS ``b_bar`` (source plus outer
        Dirichlet data): Eqs. 5.5-5.6 and 5.7-5.8 in cell-centred form."""
        nx, ny, n = self.nx, self.ny, self.n_cells
        tx, ty = self.interior_trans(K)
        rows, cols, vals = [], [], []
        diag = np.zeros(n)
        idx = np.arange(n).reshape(ny, nx)
        a_, b_ = idx[:, :-1].ravel(), idx[:, 1:].ravel()
        t = tx.ravel()
        rows += [a_, b_]; cols += [b_, a_]; vals += [-t, -t]
        np.add.at(diag, a_, t); np.add.at(diag, b_, t)
        a_, b_ = idx[:-1, :].ravel(), idx[1:, :].ravel()
        t = ty.ravel()
        rows += [a_, b_]; cols += [b_, a_]; vals += [-t, -t]
        np.add.at(diag, a_, t); np.add.at(diag, b_, t)
        B = np.zeros((n, len(self.dofs)))
        bbar = self.source_integrals()
        for side in SIDES:
            kind = self.sides[side]
            if kind[0] == "noflow":
                continue
            cells, _ = self.side_faces(side)
            tb = self.boundary_trans(K, side)
            np.add.at(diag, cells, tb)
            if kind[0] == "iface":
                B[cells] += tb[:, None] * self.projection(side)
            else:
                bbar[cells] += tb * self.dirichlet_values(side)
        rows.append(np.arange(n)); cols.append(np.arange(n)); vals.append(diag)
        A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n))
        return A, B, bbar

    def interface_flux(self, K, X, C):
        """Flux functionals ``<u.n, xi_l>`` (rows ``l`` over local DOFs) of the
        solutions ``X`` (columns) with interface data ``C`` (local mortar
        coefficients, same columns): ``sum_e T_e (x_c - (P c)_e) P[e, l]``
        (Section 5.2, step 3 of the S_H action)."""
        out = np.zeros((len(self.dofs), X.shape[1]))
        for side in SIDES:
            if self.sides[side][0] != "iface":
                continue
            cells, _ = self.side_faces(side)
            tb = self.boundary_trans(K, side)
            p = self.projection(side)
            F = tb[:, None] * (X[cells] - p @ C)
            out += p.T @ F
        return out

    def solve(self, K, C, with_particular=True):
        """Dirichlet-to-Neumann action (Section 5.2 steps 1-3): pressures for
        interface data ``C`` (columns of local mortar coefficients) and
        optionally the particular problem Eqs. 5.7-5.8 as a last column."""
        A, B, bbar = self.assemble(K)
        rhs = B @ C
        if with_particular:
            rhs = np.column_stack([rhs, bbar])
            C = np.column_stack([C, np.zeros(len(self.dofs))])
        lu = spla.splu(A)
        X = lu.solve(rhs)
        return X, C

    def flux_basis(self, K):
        """Multiscale flux basis of Section 5.3: ``Phi[l, j] = s_H(xi_j, xi_l)
        = -<u*(xi_j).n, xi_l>``, one subdomain solve per mortar DOF, plus the
        particular contribution ``g[l] = <u_bar.n, xi_l>`` (Eq. 5.9 right-hand
        side) and the pressure responses ``X`` (``n_cells x (R+1)``)."""
        R = len(self.dofs)
        X, C = self.solve(K, np.eye(R), with_particular=True)
        flux = self.interface_flux(K, X, C)
        return -flux[:, :R], flux[:, R], X

    def fields(self, K, p, c_local):
        """Normal velocities on all faces for cell pressures ``p`` and
        interface data ``c_local``: ``ux (ny, nx+1)``, ``uy (ny+1, nx)``
        (the RT0 velocity of Eq. 2.5, recovered as in Section 5.1)."""
        nx, ny = self.nx, self.ny
        Pc = p.reshape(ny, nx)
        tx, ty = self.interior_trans(K)
        ux = np.zeros((ny, nx + 1))
        uy = np.zeros((ny + 1, nx))
        ux[:, 1:nx] = tx * (Pc[:, :-1] - Pc[:, 1:]) / self.hy
        uy[1:ny, :] = ty * (Pc[:-1, :] - Pc[1:, :]) / self.hx
        for side in SIDES:
            kind = self.sides[side]
            if kind[0] == "noflow":
                continue
            cells, _ = self.side_faces(side)
            tb = self.boundary_trans(K, side)
            if kind[0] == "iface":
                g = self.projection(side) @ c_local
            else:
                g = self.dirichlet_values(side)
            F = tb * (p[cells] - g)  # outward flux through each face
            if side == "left":
                ux[:, 0] = -F / self.hy
            elif side == "right":
                ux[:, nx] = F / self.hy
            elif side == "bottom":
                uy[0, :] = -F / self.hx
            else:
                uy[ny, :] = F / self.hx
        return ux, uy
