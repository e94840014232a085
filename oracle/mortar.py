"""Mortar spaces on the subdomain interfaces and the projections between them
and the subdomain traces (Section 3.3; the action of S_H in Section 5.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each interface carries a uniform coarse mesh of ``n_el`` elements with
discontinuous polynomials of degree 1 or 2 (the paper uses discontinuous
piecewise linears, Section 6; reading A5). The basis on an element is the
Lagrange basis at equally spaced local nodes. Global mortar DOFs are numbered
interface by interface (Stokes-Darcy edges left to right, then vertical
Darcy-Darcy edges row by row, then horizontal Darcy-Darcy edges row by row),
element by element along increasing coordinate, local node by local node.

Integrals of mortar functions against piecewise polynomials on the fine
subdomain traces are exact: every fine face is split at the mortar
breakpoints and each piece is integrated with 3-point Gauss-Legendre, exact
for degree 5.
"""

import numpy as np

_GL_X = np.array([-np.sqrt(0.6), 0.0, np.sqrt(0.6)])
_GL_W = np.array([5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0])


def lagrange_1d(deg, t):
    """Lagrange basis of degree 1 or 2 on [0, 1] at equally spaced nodes,
    evaluated at ``t``; returns ``(deg+1, len(t))``. The local shapes of the
    discontinuous mortar space of Section 3.3 (reading A5)."""
    t = np.asarray(t, dtype=np.float64)
    if deg == 1:
        return np.array([1.0 - t, t])
    if deg == 2:
        return np.array([2.0 * (t - 0.5) * (t - 1.0), 4.0 * t * (1.0 - t), 2.0 * t * (t - 0.5)])
    raise ValueError(deg)


class Interface:
    """One interface segment ``[s0, s1]`` of the coordinate ``axis`` ('x' for a
    horizontal edge, 'y' for a vertical one) with its mortar mesh."""

    def __init__(self, kind, axis, s0, s1, n_el, deg, side_a, side_b, offset):
        self.kind, self.axis = kind, axis
        self.s0, self.s1, self.n_el, self.deg = s0, s1, n_el, deg
        self.side_a, self.side_b = side_a, side_b  # (subdomain id or 'stokes', side)
        self.offset = offset
        self.n_dof = n_el * (deg + 1)
        self.breaks = s0 + (s1 - s0) * np.arange(n_el + 1) / n_el

    def dofs(self):
        return list(range(self.offset, self.offset + self.n_dof))

    def basis_at(self, s):
        """Values of all mortar basis functions xi_l of this interface (the
        basis of Section 5.3 Step 2) at points ``s`` inside ``[s0, s1]``:
        returns ``(n_dof, len(s))``."""
        s = np.asarray(s, dtype=np.float64)
        h = (self.s1 - self.s0) / self.n_el
        e = np.clip(np.floor((s - self.s0) / h).astype(int), 0, self.n_el - 1)
        t = (s - self.s0) / h - e
        loc = lagrange_1d(self.deg, t)
        out = np.zeros((self.n_dof, s.size))
        for a in range(self.deg + 1):
            out[e * (self.deg + 1) + a, np.arange(s.size)] = loc[a]
        return out

    def integrate(self, f0, f1, weight_fn):
        """Exact ``int_{f0}^{f1} xi_l(s) weight_fn(s) ds`` for every mortar DOF
        ``l`` (``weight_fn`` a polynomial of degree <= 3 on the piece), split at
        the mortar breakpoints. Returns ``(n_dof,)``."""
        lo, hi = max(f0, self.s0), min(f1, self.s1)
        out = np.zeros(self.n_dof)
        if hi <= lo:
            return out
        cuts = [lo] + [b for b in self.breaks if lo < b < hi] + [hi]
        for a, b in zip(cuts[:-1], cuts[1:]):
            mid = 0.5 * (a + b)
            half = 0.5 * (b - a)
            s = mid + half * _GL_X
            # evaluate on the element containing the piece (avoid the breakpoint)
            h = (self.s1 - self.s0) / self.n_el
            e = min(int((mid - self.s0) // h), self.n_el - 1)
            t = (s - self.s0) / h - e
            loc = lagrange_1d(self.deg, t)
            wv = weight_fn(s) * _GL_W * half
            for q in range(self.deg + 1):
                out[e * (self.deg + 1) + q] += np.sum(loc[q] * wv)
        return out

    def face_projection(self, faces):
        """L2 projection onto piecewise constants on the fine faces ``faces``
        (list of ``(f0, f1)``): ``P[e, l] = (1/|e|) int_e xi_l ds`` (the
        projection onto the Darcy normal traces, Section 5.2 step 1)."""
        p = np.zeros((len(faces), self.n_dof))
        for r, (f0, f1) in enumerate(faces):
            p[r] = self.integrate(f0, f1, lambda s: np.ones_like(s)) / (f1 - f0)
        return p
