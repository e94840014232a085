"""Pins of the oracle's KL expansion (Section 2.1, Eqs. 2.11-2.13, Eq. 6.1)
against the Fredholm equation itself, orthonormality, the trace identity, an
independent Nystrom discretisation and the variance bound."""

import math

import numpy as np
import pytest

from oracle import kl


def _fredholm_apply(fun, x, length, eta, n_gl=64):
    """``int_{-a}^{a} exp(-|x - s|/eta) fun(s) ds`` by Gauss-Legendre split at
    the kink ``s = x`` (accurate to ~1e-14 for smooth ``fun``)."""
    a = 0.5 * length
    gx, gw = np.polynomial.legendre.leggauss(n_gl)
    out = 0.0
    for lo, hi in ((-a, x), (x, a)):
        if hi <= lo:
            continue
        # subdivide to resolve the exponential on short correlation lengths
        n_sub = max(1, int(math.ceil((hi - lo) / (0.25 * eta))))
        edges = np.linspace(lo, hi, n_sub + 1)
        for e0, e1 in zip(edges[:-1], edges[1:]):
            s = 0.5 * (e0 + e1) + 0.5 * (e1 - e0) * gx
            out += np.sum(gw * 0.5 * (e1 - e0) * np.exp(-np.abs(x - s) / eta) * fun(s))
    return out


@pytest.mark.parametrize("length,eta", [(0.5, 0.25), (0.25, 0.2), (0.5, 0.1), (1.0, 0.05)])
def test_roots_solve_transcendental_equations(length, eta):
    om, lam, par = kl.kl_1d(length, eta, 12)
    a, c = 0.5 * length, 1.0 / eta
    for w, p in zip(om, par):
        th = w * a
        # sign-regular forms: even c cos - w sin = 0, odd w cos + c sin = 0
        res = (c * math.cos(th) - w * math.sin(th)) if p == 0 else (w * math.cos(th) + c * math.sin(th))
        assert abs(res) < 1e-12 * max(1.0, w, c)
    assert np.all(np.diff(lam) < 0), "eigenvalues must decrease"
    assert list(par[:4]) == [0, 1, 0, 1]


@pytest.mark.parametrize("length,eta", [(0.5, 0.25), (0.25, 0.125), (0.5, 0.1)])
def test_eigenpairs_satisfy_fredholm_equation(length, eta):
    """Eq. 2.11 in 1-D: int C(x, s) f(s) ds = lambda f(x) at sample points."""
    om, lam, par = kl.kl_1d(length, eta, 6)
    xs = np.linspace(-0.5 * length, 0.5 * length, 7)
    for m in range(6):
        f = lambda s, m=m: kl.kl_1d_eval(s, length, om[m:m + 1], par[m:m + 1])[0]
        for x in xs:
            lhs = _fredholm_apply(f, x, length, eta)
            rhs = lam[m] * f(np.array([x]))[0]
            assert abs(lhs - rhs) < 1e-11 * max(1.0, abs(rhs))


def test_eigenfunctions_orthonormal():
    length, eta = 0.5, 0.1
    om, lam, par = kl.kl_1d(length, eta, 10)
    gx, gw = np.polynomial.legendre.leggauss(200)
    a = 0.5 * length
    f = kl.kl_1d_eval(a * gx, length, om, par)
    gram = (f * (gw * a)) @ f.T
    assert np.allclose(gram, np.eye(10), atol=1e-12)


def test_trace_identity():
    """sum_j lambda_j = int C(x, x) dx = L for unit variance. Beyond the first
    N modes there are two roots in every ``(k pi, (k+1) pi)`` (one even, one
    odd), so the missing mass is bracketed by sums of ``2c/(w^2 + c^2)`` with
    ``w`` at the bracket ends."""
    length, eta = 0.5, 0.2
    n = 4000
    om, lam, _ = kl.kl_1d(length, eta, n)
    a, c = 0.5 * length, 1.0 / eta
    ks = np.arange(n // 2, 400 * n, dtype=np.float64)
    upper = np.sum(2 * 2.0 * c / ((ks * math.pi / a) ** 2 + c ** 2))
    lower = np.sum(2 * 2.0 * c / (((ks + 1) * math.pi / a) ** 2 + c ** 2))
    rest = 4.0 * c * a * a / math.pi ** 2 / ks[-1]   # sum_{k > K} 1/k^2 ~ 1/K
    upper, lower = upper + rest * (1 + 1e-3), lower + rest * (1 - 1e-3)
    missing = length - lam.sum()
    assert lower * 0.999 < missing < upper * 1.001


def test_nystrom_cross_check():
    length, eta = 0.5, 0.125
    _, lam, _ = kl.kl_1d(length, eta, 6)
    ny = kl.nystrom_1d(length, eta, 4000, 6)
    assert np.allclose(ny, lam, rtol=2e-5)


def test_2d_modes_and_variance_bound():
    rect = (0.0, 0.5, 0.0, 0.25)
    sigma2, eta = 2.0, (0.2, 0.1)
    xs = np.array([0.01, 0.13, 0.25, 0.49])
    ys = np.array([0.02, 0.1, 0.2, 0.24])
    prev_var = np.zeros(xs.size)
    prev_sum = 0.0
    for n in (1, 2, 4, 9, 16):
        lam, f = kl.kl_region_fields(rect, sigma2, eta, n, xs, ys)
        assert np.all(np.diff(lam) <= 0)
        var = (lam[:, None] * f ** 2).sum(0)
        assert np.all(var <= sigma2 + 1e-12)
        assert np.all(var >= prev_var - 1e-15)
        assert lam.sum() <= sigma2 * 0.5 * 0.25 + 1e-14   # sum lambda <= sigma^2 |D|
        assert lam.sum() >= prev_sum
        prev_var, prev_sum = var, lam.sum()
    # the 2-D eigenvalues are products of the 1-D ones (separable Eq. 6.1)
    _, lx, _ = kl.kl_1d(0.5, 0.2, 3)
    _, ly, _ = kl.kl_1d(0.25, 0.1, 3)
    lam, _ = kl.kl_region_fields(rect, sigma2, eta, 3, xs, ys)
    prods = sorted((sigma2 * lx[a] * ly[b] for a in range(3) for b in range(3)), reverse=True)
    assert np.allclose(lam, prods[:3], rtol=1e-14)


def test_log_permeability_linear_in_y():
    lam = np.array([0.5, 0.25])
    f = np.array([[1.0, -2.0], [0.5, 3.0]])
    assert np.allclose(kl.log_permeability(lam, f, [0.0, 0.0], 0.3), 0.3)
    y = np.array([1.0, -2.0])
    expect = 0.3 + math.sqrt(0.5) * f[0] * 1.0 + math.sqrt(0.25) * f[1] * -2.0
    assert np.allclose(kl.log_permeability(lam, f, y, 0.3), expect)


def test_tensor_mode_sets_of_the_paper():
    """The paper's "N_term = n1 x n2" mode sets (Section 6.1). On a KL region
    the kept set is the full product of the n1 leading x-modes and the n2
    leading y-modes, so (i) the pointwise variance of the truncated field
    factorises into the two 1-D truncated variances and the eigenvalue sum
    into the two 1-D sums, and (ii) in "2 x 1" both modes share the leading
    y-mode: the ratio f_1 / f_0 does not depend on y. A selection by largest
    products, or n1 and n2 swapped, fails (i) or (ii) on this region."""
    rect, sigma2, eta = (0.0, 1.0, 0.0, 0.4), 1.0, (0.1, 0.1)   # Case 1, KL region 1
    lx, ly = 1.0, 0.4
    xs = np.linspace(0.03, 0.97, 7)
    ys = np.linspace(0.01, 0.39, 5)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    for n1, n2 in ((2, 1), (3, 3), (1, 4)):
        lam, f = kl.kl_region_fields(rect, sigma2, eta, n1 * n2, X.ravel(), Y.ravel(), modes=(n1, n2))
        omx, lamx, parx = kl.kl_1d(lx, eta[0], n1)
        omy, lamy, pary = kl.kl_1d(ly, eta[1], n2)
        assert abs(lam.sum() - sigma2 * lamx.sum() * lamy.sum()) < 1e-14
        assert np.all(np.diff(lam) <= 0)
        vx = (lamx[:, None] * kl.kl_1d_eval(xs - 0.5, lx, omx, parx) ** 2).sum(0)
        vy = (lamy[:, None] * kl.kl_1d_eval(ys - 0.2, ly, omy, pary) ** 2).sum(0)
        var = (lam[:, None] * f ** 2).sum(0).reshape(X.shape)
        assert np.allclose(var, sigma2 * vx[:, None] * vy[None, :], rtol=1e-13, atol=0)
    lam, f = kl.kl_region_fields(rect, sigma2, eta, 2, X.ravel(), Y.ravel(), modes=(2, 1))
    ratio = (f[1] / f[0]).reshape(X.shape)
    assert np.allclose(ratio, ratio[:, :1], rtol=1e-12, atol=1e-12)
    assert np.ptp(ratio[:, 0]) > 0.1            # and it does depend on x
    with pytest.raises(ValueError):
        kl.kl_2d_modes(lx, ly, sigma2, eta, 3, modes=(2, 2))
