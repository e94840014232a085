"""Pins of the oracle's collocation (Section 4) and index conversion
(Section 5.4 Step 4) against closed forms, exactness, point counts the paper
prints and the solve-count identities of Eqs. 5.12-5.13 with Tables 1-2."""

import math
import os

import numpy as np
import pytest

from oracle import collocation, kl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def test_gauss_hermite_closed_forms():
    x, w = collocation.gauss_hermite(2)
    assert np.allclose(np.sort(x), [-1.0, 1.0], atol=1e-15)
    assert np.allclose(w, [0.5, 0.5], atol=1e-15)
    x, w = collocation.gauss_hermite(3)
    order = np.argsort(x)
    assert np.allclose(x[order], [-math.sqrt(3.0), 0.0, math.sqrt(3.0)], atol=1e-14)
    assert np.allclose(w[order], [1 / 6, 2 / 3, 1 / 6], atol=1e-15)
    x, w = collocation.gauss_hermite(1)
    assert x[0] == 0.0 and w[0] == 1.0


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 10])
def test_gauss_hermite_exact_to_degree_2m_minus_1(m):
    """N(0,1) moments E[y^k] = (k-1)!! for even k, 0 for odd k (Section 4)."""
    x, w = collocation.gauss_hermite(m)
    for k in range(2 * m):
        exact = 0.0 if k % 2 else float(math.prod(range(k - 1, 0, -2)))
        scale = np.sum(w * np.abs(x) ** k)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13 * max(1.0, scale)
    # and not exact at degree 2m (the rule is Gaussian, not better)
    exact = float(math.prod(range(2 * m - 1, 0, -2)))
    assert abs(np.sum(w * x ** (2 * m)) - exact) > 1e-6


def test_tensor_grid_counts_and_weights():
    y, w = collocation.tensor_grid([2, 3, 2])
    assert y.shape == (12, 3)
    assert abs(w.sum() - 1.0) < 1e-15
    assert abs(np.sum(w * y[:, 1] ** 4) - 3.0) < 1e-13
    assert abs(np.sum(w * y[:, 0] ** 2 * y[:, 2] ** 2) - 1.0) < 1e-14


@pytest.mark.parametrize("n_dim,lmax,rule,count", [
    (50, 1, "paper", 101), (200, 1, "paper", 401), (100, 1, "paper", 201),
    (12, 2, [1, 3, 3], 289), (32, 2, [1, 3, 3], 2049), (3, 2, "paper", 37),
])
def test_smolyak_counts(n_dim, lmax, rule, count):
    """Level 1 gives 2N+1 points (Section 6: 101, 401, 201); level 2 with the
    {1,3,3} sequence 289 and 2,049; the paper's sequence gives 37 on 3 dims."""
    y, w = collocation.smolyak_grid(n_dim, lmax, rule)
    assert y.shape == (count, n_dim)
    assert abs(w.sum() - 1.0) < 1e-14 * np.abs(w).sum() * n_dim


def test_smolyak_exactness():
    """Level-2 {1,3,3} rule: exact for y_i^a y_j^b with a, b <= 5."""
    y, w = collocation.smolyak_grid(6, 2, [1, 3, 3])
    assert abs(np.sum(w * y[:, 0] ** 2) - 1.0) < 1e-13
    assert abs(np.sum(w * y[:, 2] ** 4) - 3.0) < 1e-13
    assert abs(np.sum(w * y[:, 1] ** 2 * y[:, 4] ** 2) - 1.0) < 1e-13
    assert abs(np.sum(w * y[:, 1] ** 4 * y[:, 3] ** 2) - 3.0) < 1e-12
    assert abs(np.sum(w * y[:, 1] * y[:, 3])) < 1e-14
    y, w = collocation.smolyak_grid(4, 2, "paper")
    assert abs(np.sum(w * y[:, 0] ** 6) - 15.0) < 1e-11     # 7-point rule at level 2
    assert abs(np.sum(w * y[:, 0] ** 2 * y[:, 3] ** 2) - 1.0) < 1e-12


def test_level_three_weights_sum_to_one():
    """The combination formula integrates constants exactly, so the weights
    of the level-3 {1,3,3,3} grid over 40 dimensions (82,241 points, the
    origin's weight a sum of about 1.2e4 terms of both signs) sum to one, and
    its moments of degree 2 and 4 are the Gaussian ones, to the rounding of
    the terms themselves (coefficients up to 9,139 times products of 1/6 and
    2/3: about 4e-13). A plain running sum per point misses the total by
    1.3e-9 here."""
    y, w = collocation.smolyak_grid(40, 3, [1, 3, 3, 3])
    assert len(w) == 82241
    assert abs(w.sum() - 1.0) < 1e-12
    assert abs(np.sum(w * y[:, 0] ** 2) - 1.0) < 1e-12
    assert abs(np.sum(w * y[:, 7] ** 2 * y[:, 31] ** 2) - 1.0) < 1e-12
    assert abs(np.sum(w * y[:, 5] ** 4) - 3.0) < 1e-12


def test_linear_kl_moments_exact_under_quadrature():
    """Y is linear in y, so E[Y] = mean and Var[Y] = sum lambda f^2 hold
    exactly for any rule of degree >= 2."""
    rect = (0.0, 0.5, 0.0, 0.25)
    xs, ys = np.array([0.1, 0.3]), np.array([0.05, 0.2])
    lam, f = kl.kl_region_fields(rect, 2.0, (0.2, 0.1), 4, xs, ys)
    for grid in (collocation.tensor_grid([2] * 4), collocation.smolyak_grid(4, 1, "paper"),
                 collocation.smolyak_grid(4, 2, [1, 3, 3])):
        y, w = grid
        Y = np.array([kl.log_permeability(lam, f, yy, 0.5) for yy in y])
        assert np.allclose(w @ Y, 0.5, atol=1e-14)
        assert np.allclose(w @ (Y - 0.5) ** 2, (lam[:, None] * f ** 2).sum(0), rtol=1e-13)


@pytest.mark.parametrize("n_terms,spec,local,n_proj", [
    ([3, 3, 3, 3], {"kind": "smolyak", "lmax": 2, "rule": [1, 3, 3], "local": "tensor"}, 27, 19),
    ([4] * 8, {"kind": "smolyak", "lmax": 2, "rule": [1, 3, 3], "local": "tensor"}, 81, 33),
    ([2, 2], {"kind": "tensor", "m": 2, "local": "tensor"}, 4, 4),
])
def test_local_realizations(n_terms, spec, local, n_proj):
    """The workloads' local tensor grids (27, 81, 4 local realizations per
    region) contain every projection of the global grid; a level-2 grid
    reaches only the points with at most two nonzero coordinates
    (1 + 2N + 4 C(N, 2) of them)."""
    y, w = collocation.global_grid(spec, sum(n_terms))
    for dims in collocation.region_dims(n_terms):
        grid = collocation.local_grid(spec, len(dims))
        loc, kmap = collocation.local_points(y, dims, grid)
        assert len(loc) == local
        assert np.allclose(loc[kmap], y[:, dims])
        proj, kp = collocation.local_points(y, dims)
        assert len(proj) == n_proj
        assert np.allclose(proj[kp], y[:, dims])


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        c, g, nt, nr, nreal, nloc, s2, s3, cite = line.split()
        rows.append((c, g, int(nt), int(nr), int(nreal), int(nloc), int(s2), int(s3), cite))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: r[0] + "-" + r[1])
def test_paper_counts(row):
    """Global and local point counts from the oracle's grids, and the printed
    S2/S3 solve counts: both Eq. 5.12 + 2 extra solves, S2 = (R+2) N_real,
    and Eq. 5.13 + 2 extras, S3 = R N_real(j) + 2 N_real, give the same
    integer mortar DOF count R for the busiest subdomain."""
    case, grid, nt, nr, nreal, nloc, s2, s3, _ = row
    if grid == "tensor":
        assert 2 ** nt == nreal and 2 ** nr == nloc
        y, _ = collocation.tensor_grid([2] * nt)
    else:
        y, _ = collocation.smolyak_grid(nt, 1, "paper")
    assert len(y) == nreal
    dims = list(range(nt - nr, nt)) if case == "case1" else list(range(nr))
    loc, _ = collocation.local_points(y, dims)
    assert len(loc) == nloc
    assert s2 % nreal == 0
    r_from_s2 = s2 // nreal - 2
    assert (s3 - 2 * nreal) % nloc == 0
    r_from_s3 = (s3 - 2 * nreal) // nloc
    assert r_from_s2 == r_from_s3


def test_anisotropic_tensor_rule():
    """Section 4.1's anisotropic tensor rule with m = (2, 1, 3, 4) points per
    dimension: Prod m points with weights summing to one, and in each
    dimension the moments of that dimension's own Gauss-Hermite rule, which
    are closed forms: the 1-point rule sits at the mean (E[y^2] = 0), the
    2-point rule at +-1 (E[y^4] = 1), the 3-point rule at {0, +-sqrt 3} with
    weights {2/3, 1/6, 1/6} (E[y^4] = 3, E[y^6] = 9), and the 4-point rule is
    exact to degree 7 (E[y^6] = 15). A reversed or shifted m fails these."""
    spec = {"kind": "tensor", "m": [2, 1, 3, 4]}
    y, w = collocation.global_grid(spec, 4)
    assert y.shape == (24, 4) and abs(w.sum() - 1.0) < 1e-15
    E = lambda f: float(np.dot(w, f))           # noqa: E731
    assert abs(E(y[:, 0] ** 2) - 1) < 1e-14 and abs(E(y[:, 0] ** 4) - 1) < 1e-14
    assert abs(E(y[:, 1] ** 2)) < 1e-15
    assert abs(E(y[:, 2] ** 4) - 3) < 1e-13 and abs(E(y[:, 2] ** 6) - 9) < 1e-12
    assert abs(E(y[:, 3] ** 6) - 15) < 1e-12
    assert abs(E(y[:, 0] ** 2 * y[:, 3] ** 2) - 1) < 1e-14
    iso = collocation.global_grid({"kind": "tensor", "m": 3}, 2)
    aniso = collocation.global_grid({"kind": "tensor", "m": [3, 3]}, 2)
    assert np.array_equal(iso[0], aniso[0]) and np.array_equal(iso[1], aniso[1])
    with pytest.raises(ValueError):
        collocation.global_grid(spec, 3)


def test_anisotropic_local_grids_are_the_projections():
    """On an anisotropic tensor grid each region's local tensor grid (its own
    rules) is exactly the set of distinct projections of the global points,
    and every global point maps onto it (Section 5.4 Step 4)."""
    spec = {"kind": "tensor", "m": [2, 1, 3, 1, 2, 2], "local": "tensor"}
    dims = collocation.region_dims([2, 4])
    y, _ = collocation.global_grid(spec, 6)
    for d, count in zip(dims, (2, 12)):
        grid = collocation.local_grid(spec, len(d), d)
        assert len(grid) == count
        loc, kmap = collocation.local_points(y, d, grid)
        assert np.allclose(loc[kmap], y[:, d], atol=1e-15)
        proj = {tuple(np.round(r, 12)) for r in y[:, d]}
        assert proj == {tuple(np.round(r, 12)) for r in grid}
