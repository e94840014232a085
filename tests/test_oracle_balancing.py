"""Pins of the oracle's balancing Neumann-Neumann preconditioner (the one
Section 7 suggests for the interface problem): the floating units are the
singular ones, the balanced preconditioner is symmetric positive definite,
the preconditioned operator's spectrum starts at exactly 1 (the coarse
directions) and stays at or above it (Mandel's bound for weights that form a
partition of unity), and balanced CG reaches the dense solution of
Eqs. 5.9-5.10 in fewer iterations than plain CG."""

import numpy as np
import pytest

from gpu_common import make_workload
from oracle import balancing, coupled


def _point_bases(p, l):
    y, _ = p.grid()
    bases = []
    for s in range(len(p.subs)):
        phi, g, _, _ = p.darcy_basis(s, p.local_y(s, y[l]))
        bases.append((phi, g))
    return bases


@pytest.mark.parametrize("case,n_float", [("tiny", 0), ("medium", 2), ("ragged", 3)])
def test_floating_units_are_the_singular_ones(case, n_float):
    """Floating Darcy subdomains have exactly the constant as null direction;
    the others, and the Stokes unit, are nonsingular, except the ragged
    case's Stokes unit: its 7 x 5 Taylor-Hood grid carries 27 quadratic
    mortar DOFs on 15 velocity nodes of its bottom side, so its flux basis
    has rank at most 15 (the pseudo-inverse takes care of it)."""
    p = coupled.Problem(make_workload(case))
    us = balancing.units(p, _point_bases(p, 1))
    assert sum(f for _, _, f in us) == n_float
    for u, (dofs, phi, floating) in enumerate(us):
        ev = np.linalg.eigvalsh(phi)
        scale = np.abs(ev).max()
        stokes = u == len(us) - 1
        if floating:
            # the constant mortar pressure drives no flux: one null direction
            assert np.abs(phi @ np.ones(len(dofs))).max() <= 1e-10 * scale
            assert abs(ev[0]) <= 1e-10 * scale and ev[1] > 1e-8 * scale
        elif stokes and case == "ragged":
            assert np.sum(ev > 1e-8 * scale) <= 15
        else:
            assert ev[0] > 1e-8 * scale


@pytest.mark.parametrize("case", ["tiny", "medium", "ragged"])
def test_preconditioned_spectrum(case):
    p = coupled.Problem(make_workload(case))
    b = balancing.Balancing(p, _point_bases(p, 2))
    n = p.n_lambda
    M = np.array([b.apply(e) for e in np.eye(n)]).T
    assert np.abs(M - M.T).max() <= 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T))[0] > 0.0
    ev = np.sort(np.linalg.eigvals(M @ b.S).real)
    # Mandel's lower bound needs every null direction of a local operator in
    # the coarse space; the ragged case's Stokes unit has null directions of
    # its own (more mortar DOFs than velocity nodes under them), which only
    # its Darcy neighbours' Neumann steps see
    assert ev[0] >= (0.99 if case == "ragged" else 1.0 - 1e-9)
    if b.Z.shape[1] > 0:
        if case != "ragged":
            assert abs(ev[0] - 1.0) <= 1e-9      # the coarse directions
        # the balanced start leaves no residual on the coarse space
        r0 = b.g - b.S @ b.start()
        assert np.abs(b.Z.T @ r0).max() <= 1e-12 * np.abs(b.g).max()
    assert ev[-1] / ev[0] < 0.25 * np.linalg.cond(b.S)


@pytest.mark.parametrize("case", ["medium", "ragged"])
def test_balanced_cg_reaches_the_dense_solution(case):
    p = coupled.Problem(make_workload(case))
    y, _ = p.grid()
    for l in (0, 3, len(y) - 1):
        lam, S, g, _ = p.interface_dense(y[l])
        lb, itb = balancing.solve_point(p, y[l], rtol=1e-13, max_it=500)
        _, itc = coupled.cg(lambda v: S @ v, g, 1e-13, 2000)
        assert itb > 0 and itb < itc
        assert np.linalg.norm(lb - lam) <= 1e-10 * np.linalg.norm(lam)
