"""The allocation-free basis entry point against the workspace-based build
and against the oracle.

sfb_build_basis_item_noalloc serves callers that cannot allocate device
memory (all of it already belongs to their own pool, or their hot path must
not call cudaMalloc). It keeps its working memory in a static device array
shared by every call, so this test calls it several times in a row on
different items (a call must not see the previous call's leftovers) and
compares each result with the same item from sfb_build_stochastic_basis,
within the parity tolerance of the precision used, and with the oracle's
basis of the same local realization. An item larger than the static array
is refused before any copy or launch. This file sorts last so that a run
that stops at the first failure has already run every other test.
"""

import numpy as np
import pytest

import sfb_workloads as W

pytestmark = pytest.mark.gpu

# FP64 form, mixed form (refined), and the unrefined FP32 diagnostic form,
# whose error is the FP32 solve's (about cond(A) * 6e-8)
TOL = {0: 1e-10, 1: 1e-8, 2: 1e-3}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _workload():
    return W.small_test(nx=13, ny=9, px=3, py=2, n_sd=3, n_dd=2, n_term=2, degree=2, stokes=(7, 5),
                        bottom_pressure=0.5, source=[0.3, -0.2, 0.1, 0.7, -0.4, 0.2])


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_noalloc_item_matches_workspace_build(prec):
    import torch
    import paper_1802_06263_gb300 as sfb
    from oracle import coupled

    w = _workload()
    p = coupled.Problem(w)
    s = sfb.Solver(w)
    s.allocate(prec)
    s.build_basis(prec, check=prec != 2)
    items = [(4, 3), (1, 0), (4, 3)]   # two different items in a row, then the first again
    for sub, k in items:
        R = len(s.subdomain_dofs(sub))
        nx, ny = w["darcy_grid"][sub]
        phi = np.zeros((R, R))
        g = np.zeros(R)
        x = torch.full((R + 1, nx * ny), float("nan"), dtype=torch.float64, device="cuda")
        rc = s.build_item_noalloc(sub, k, prec, phi, g, x, check=prec != 2)
        assert rc in ((0,) if prec != 2 else (0, sfb.SFB_ERR_NOT_CONVERGED))
        torch.cuda.synchronize()
        xh = x.cpu().numpy().T
        phi_ref, g_ref, x_ref = s.get_basis(sub, k, with_x=True)
        assert _rel(phi, phi_ref) < TOL[prec], (sub, k)
        assert np.abs(g - g_ref).max() <= TOL[prec] * max(1.0, np.abs(g_ref).max()), (sub, k)
        assert _rel(xh, x_ref) < TOL[prec], (sub, k)
        # the same item from the oracle (local realization k of the subdomain)
        phi_o, g_o, x_o, _ = p.darcy_basis(sub, s.local_points(sub)[k])
        assert _rel(phi, phi_o) < TOL[prec], (sub, k)
        assert _rel(xh, x_o) < TOL[prec], (sub, k)
        assert np.abs(g - g_o).max() <= TOL[prec] * max(1.0, np.abs(g_o).max()), (sub, k)


def test_noalloc_refuses_an_item_beyond_its_static_array():
    """A 128 x 128 item in FP32 needs 8 MiB for its block inverses alone, more
    than the static array holds with the rest: SFB_ERR_UNSUPPORTED, and the
    output buffers stay untouched."""
    import torch
    import paper_1802_06263_gb300 as sfb

    w = W.small_test(nx=128, ny=128, px=1, py=1, n_sd=2, n_dd=2, n_term=1, degree=1, stokes=(4, 4),
                     collocation={"kind": "tensor", "m": 2, "local": "tensor"})
    s = sfb.Solver(w)
    R = len(s.subdomain_dofs(0))
    phi = np.full((R, R), 7.0)
    g = np.full(R, 7.0)
    x = torch.full((R + 1, 128 * 128), float("nan"), dtype=torch.float64, device="cuda")
    rc = s.build_item_noalloc(0, 0, sfb.MIXED, phi, g, x, check=False)
    assert rc == 8, rc   # SFB_ERR_UNSUPPORTED
    assert "bytes of scratch" in s.lib.sfb_last_error(s.h).decode()
    torch.cuda.synchronize()
    assert torch.isnan(x).all().item()
    assert np.all(phi == 7.0) and np.all(g == 7.0)
