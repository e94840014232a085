"""Balancing Neumann-Neumann preconditioner for the interface problem.

Test infrastructure: plain numpy FP64, called only by the tests and the
benchmark's CPU baseline; nothing in the CUDA path imports it.

Section 7 of the paper suggests a balancing preconditioner for the Darcy
region (Mandel's balancing domain decomposition, applied to mortar mixed
methods by Pencheva and Yotov) to cut the CG iterations of the interface
problem S lambda = g (Eqs. 5.9-5.10). This module writes that preconditioner
out from its definition for S = sum_u R_u^T Phi_u R_u over the units u (the
Darcy subdomains, then the Stokes subdomain):

* weights: every mortar DOF is shared by exactly two units; D_u is diagonal
  with the unit's share of the two local stiffnesses at the DOF,
  (D_u)_dd = (Phi_u)_dd / ((Phi_u)_dd + (Phi_v)_dd), so that
  sum_u R_u^T D_u R_u = I (a partition of unity). The Stokes and Darcy
  Dirichlet-to-Neumann maps differ in scale by orders of magnitude, and the
  multiplicity weights D_u = I / 2 make the balanced operator worse
  conditioned than S itself (73 against 44 CG iterations on the medium
  workload); the stiffness shares give 10;
* local Neumann step: N r = sum_u R_u^T D_u Phi_u^+ D_u R_u r, with the
  Moore-Penrose pseudo-inverse Phi_u^+ (Phi_u is singular for a floating
  Darcy subdomain, one with no outer Dirichlet side, whose flux basis
  annihilates the constant mortar pressure, and for a Stokes unit with more
  mortar DOFs than velocity nodes on its interface);
* coarse space: Z = [R_u^T D_u 1] over the floating units, the coarse
  operator S_0 = Z^T S Z and the projection Q = Z S_0^{-1} Z^T;
* the balanced preconditioner M^{-1} = Q + (I - Q S) N (I - S Q), applied
  in CG from the balanced start lambda_0 = Q g.
"""

import numpy as np


def units(prob, bases):
    """(dofs, Phi, floating) of every unit for one point: the Darcy
    subdomains with their flux bases ``bases`` (Phi, g per subdomain), then
    the Stokes subdomain with its deterministic basis. A Darcy subdomain
    floats when none of its sides carries outer Dirichlet data; the Stokes
    subdomain has its outflow side under natural data and never floats."""
    out = []
    for sub, (phi, _) in zip(prob.subs, bases):
        floating = all(v[0] != "dirichlet" for v in sub.sides.values())
        out.append((np.array(sub.dofs), phi, floating))
    phs = prob.stokes_basis()[0]
    out.append((np.array(prob.stokes.dofs), phs, False))
    return out


class Balancing:
    """The operators of the balancing preconditioner for one point."""

    def __init__(self, prob, bases):
        self.units = units(prob, bases)
        n = prob.n_lambda
        self.S, self.g = prob.assemble_interface(bases)
        count = np.zeros(n)
        stiff = np.zeros(n)
        for dofs, phi, _ in self.units:
            count[dofs] += 1.0
            stiff[dofs] += np.diag(phi)
        assert np.all(count == 2.0), "every mortar DOF is shared by two units"
        assert np.all(stiff > 0.0)
        self.D = [np.diag(phi) / stiff[dofs] for dofs, phi, _ in self.units]
        # the pseudo-inverse drops eigenvalues below 1e-10 of the largest: the
        # null directions of a floating subdomain, and of a Stokes unit with
        # more mortar DOFs than velocity nodes under them, come out of the
        # eigensolver as rounding noise
        self.pinv = [np.linalg.pinv(phi, rcond=1e-10, hermitian=True) for _, phi, _ in self.units]
        cols = []
        for (dofs, _, floating), D in zip(self.units, self.D):
            if floating:
                z = np.zeros(n)
                z[dofs] = D
                cols.append(z)
        self.Z = np.array(cols).T.reshape(n, len(cols))
        self.S0 = self.Z.T @ self.S @ self.Z

    def coarse(self, v):
        """Q v = Z S_0^{-1} Z^T v (zero without a coarse space)."""
        if self.Z.shape[1] == 0:
            return np.zeros_like(v)
        return self.Z @ np.linalg.solve(self.S0, self.Z.T @ v)

    def neumann(self, r):
        """N r = sum_u R_u^T D_u Phi_u^+ D_u R_u r."""
        w = np.zeros_like(r)
        for (dofs, _, _), D, pinv in zip(self.units, self.D, self.pinv):
            w[dofs] += D * (pinv @ (D * r[dofs]))
        return w

    def apply(self, r):
        """M^{-1} r = Q r + (I - Q S) N (I - S Q) r."""
        t = self.neumann(r - self.S @ self.coarse(r))
        return self.coarse(r) + t - self.coarse(self.S @ t)

    def start(self):
        """The balanced start lambda_0 = Q g."""
        return self.coarse(self.g)


def pcg(S, g, precond, lam0, rtol, max_it):
    """Preconditioned CG from ``lam0``; stops at ``||r|| <= rtol ||g||`` on
    the recursive residual, as the unpreconditioned CG of ``coupled.cg``.
    Returns ``(lambda, iterations)``, iterations negative if not converged."""
    lam = lam0.copy()
    r = g - S @ lam
    z = precond(r)
    p = z.copy()
    rz = r @ z
    gn = np.sqrt(g @ g)
    if gn == 0.0:
        return lam, 0
    for it in range(1, max_it + 1):
        q = S @ p
        alpha = rz / (p @ q)
        lam += alpha * p
        r -= alpha * q
        if np.sqrt(r @ r) <= rtol * gn:
            return lam, it
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return lam, -max_it


def solve_point(prob, y_global, rtol=1e-12, max_it=2000):
    """One point's interface problem by balancing-preconditioned CG with the
    stored-basis operator of Method S3. Returns ``(lambda, iterations)``."""
    bases = []
    for s in range(len(prob.subs)):
        phi, g, _, _ = prob.darcy_basis(s, prob.local_y(s, y_global))
        bases.append((phi, g))
    b = Balancing(prob, bases)
    return pcg(b.S, b.g, b.apply, b.start(), rtol, max_it)
