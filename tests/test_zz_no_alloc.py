"""The allocation-free basis entry point against the workspace-based build.

sfb_build_basis_item_noalloc serves callers that cannot allocate device
memory (all of it already belongs to their own pool, or their hot path must
not call cudaMalloc). It keeps its working memory in a static device array
shared by every call, so this test calls it twice in a row on different
items (the second call must not see the first call's leftovers) and compares
each result with the same item from sfb_build_stochastic_basis, within the
parity tolerance of the precision used. This file sorts last so that a run
that stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import sfb_workloads as W

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-8}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_item_matches_workspace_build(prec):
    import torch
    import paper_1802_06263_gb300 as sfb

    w = W.small_test(nx=13, ny=9, px=3, py=2, n_sd=3, n_dd=2, n_term=2, degree=2, stokes=(7, 5),
                     bottom_pressure=0.5, source=[0.3, -0.2, 0.1, 0.7, -0.4, 0.2])
    s = sfb.Solver(w)
    s.allocate(prec)
    s.build_basis(prec)
    items = [(4, 3), (1, 0), (4, 3)]   # two different items in a row, then the first again
    for sub, k in items:
        R = len(s.subdomain_dofs(sub))
        nx, ny = w["darcy_grid"][sub]
        phi = np.zeros((R, R))
        g = np.zeros(R)
        x = torch.full((R + 1, nx * ny), float("nan"), dtype=torch.float64, device="cuda")
        s.build_item_noalloc(sub, k, prec, phi, g, x)
        torch.cuda.synchronize()
        phi_ref, g_ref, x_ref = s.get_basis(sub, k, with_x=True)
        assert _rel(phi, phi_ref) < TOL[prec], (sub, k)
        assert np.abs(g - g_ref).max() <= TOL[prec] * max(1.0, np.abs(g_ref).max()), (sub, k)
        assert _rel(x.cpu().numpy().T, x_ref) < TOL[prec], (sub, k)
