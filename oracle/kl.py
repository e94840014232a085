"""Multi-region Karhunen-Loeve expansion (Section 2.1, Eqs. 2.11-2.13).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Each KL region carries the separable exponential covariance of Eq. 6.1,
``C(x, x') = sigma^2 exp(-|x1-x1'|/eta1 - |x2-x2'|/eta2)``. The Fredholm
problem Eq. 2.11 then separates into two 1-D problems whose solutions on a
segment ``[-a, a]`` are known in closed form up to the roots of two
transcendental equations (with ``c = 1/eta``):

* even modes ``cos(w x)``: ``c - w tan(w a) = 0``,
* odd modes  ``sin(w x)``: ``w + c tan(w a) = 0``,
* eigenvalue ``2 c / (w^2 + c^2)``.

The paper calls sigma_Y "the variance" but writes its square in Eq. 6.1; the
configured ``sigma2`` multiplies the kernel (reading A1).
"""

import math

import numpy as np


def _bisect(f, lo, hi, iters=200):
    flo = f(lo)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        fm = f(mid)
        if fm == 0.0 or hi - lo <= 4e-16 * max(1.0, abs(mid)):
            return mid
        if (fm < 0) == (flo < 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def kl_1d(length, eta, n_modes):
    """First ``n_modes`` eigenpairs of ``exp(-|x-x'|/eta)`` on a segment of the
    given length, centred at 0, in decreasing eigenvalue order: the 1-D
    factors of the Fredholm problem Eq. 2.11 for the separable covariance
    Eq. 6.1, from the textbook transcendental equations of the exponential
    kernel (even and odd modes).

    Returns ``(omega, lam, parity)`` with ``parity`` 0 for even (cosine) and 1
    for odd (sine) modes. Roots come from bisection on sign-regular forms of
    the transcendental equations: even roots ``theta = w a`` lie in
    ``(n pi, n pi + pi/2)``, odd roots in ``(n pi + pi/2, (n+1) pi)``, so the
    sorted roots alternate even, odd, even, ...
    """
    a = 0.5 * length
    c = 1.0 / eta
    ca = c * a
    omegas, parity = [], []
    n = 0
    while len(omegas) < n_modes:
        # even: theta sin(theta) - c a cos(theta) = 0 on (n pi, n pi + pi/2)
        lo, hi = n * math.pi, n * math.pi + 0.5 * math.pi
        th = _bisect(lambda t: t * math.sin(t) - ca * math.cos(t), lo, hi)
        omegas.append(th / a)
        parity.append(0)
        if len(omegas) == n_modes:
            break
        # odd: theta cos(theta) + c a sin(theta) = 0 on (n pi + pi/2, (n+1) pi)
        lo, hi = n * math.pi + 0.5 * math.pi, (n + 1) * math.pi
        th = _bisect(lambda t: t * math.cos(t) + ca * math.sin(t), lo, hi)
        omegas.append(th / a)
        parity.append(1)
        n += 1
    omega = np.array(omegas)
    lam = 2.0 * c / (omega ** 2 + c ** 2)
    return omega, lam, np.array(parity)


def kl_1d_eval(x, length, omega, parity):
    """Normalised 1-D eigenfunctions at points ``x`` (centred coordinates), the
    factors of the eigenfunctions in Eqs. 2.12-2.13.

    ``cos(w x) / sqrt(a + sin(2wa)/(2w))`` for even modes and
    ``sin(w x) / sqrt(a - sin(2wa)/(2w))`` for odd modes, which have unit
    L2 norm on ``[-a, a]``. Returns an array ``(len(omega), len(x))``.
    """
    a = 0.5 * length
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((len(omega), x.size))
    for m, (w, par) in enumerate(zip(omega, parity)):
        s = math.sin(2.0 * w * a) / (2.0 * w)
        if par == 0:
            out[m] = np.cos(w * x) / math.sqrt(a + s)
        else:
            out[m] = np.sin(w * x) / math.sqrt(a - s)
    return out


def kl_2d_modes(lx, ly, sigma2, eta, n_term, modes=None):
    """2-D modes of Eq. 6.1 on an ``lx x ly`` region.

    Separability gives eigenvalues ``sigma2 * lamx[a] * lamy[b]`` with
    eigenfunctions ``fx_a(x) fy_b(y)``. Without ``modes`` the ``n_term``
    largest products are kept (reading A2). With ``modes = (n1, n2)`` the
    kept set is every product of the n1 largest 1-D modes in x with the n2
    largest in y: the paper's ``N_term = n1 x n2`` form (Section 6.1, e.g.
    "2 x 1 = 2"), so ``n_term`` must be ``n1 * n2``. Either way the kept modes
    are ordered by decreasing eigenvalue with ties broken by ``(a + b, a)``.
    Returns a list of ``(lam, a, b)`` plus the 1-D data
    ``(omx, parx, omy, pary)``.
    """
    if modes is None:
        na = nb = n_term
    else:
        na, nb = modes
        if na * nb != n_term:
            raise ValueError("n1 x n2 mode set of %d modes, n_term %d" % (na * nb, n_term))
    omx, lamx, parx = kl_1d(lx, eta[0], na)
    omy, lamy, pary = kl_1d(ly, eta[1], nb)
    cand = []
    for a in range(na):
        for b in range(nb):
            cand.append((-(sigma2 * lamx[a] * lamy[b]), a + b, a, b))
    cand.sort()
    out = [(-c[0], c[2], c[3]) for c in cand[:n_term]]
    return out, (omx, parx, omy, pary)


def kl_region_fields(rect, sigma2, eta, n_term, xc, yc, modes=None):
    """Eigenvalues and eigenfunction values of one KL region at points.

    ``rect = (x0, x1, y0, y1)`` is the region; ``xc, yc`` are physical point
    coordinates (the region's own cell centres, reading A11). Returns
    ``lam[n_term]`` and ``f[n_term, npts]`` with ``f_j = fx_a fy_b`` evaluated in
    region-centred coordinates (Eq. 2.12 truncated as Eq. 2.13). ``modes``
    selects an ``n1 x n2`` tensor set as in ``kl_2d_modes``.
    """
    x0, x1, y0, y1 = rect
    lx, ly = x1 - x0, y1 - y0
    modes, (omx, parx, omy, pary) = kl_2d_modes(lx, ly, sigma2, eta, n_term, modes)
    fx = kl_1d_eval(np.asarray(xc) - 0.5 * (x0 + x1), lx, omx, parx)
    fy = kl_1d_eval(np.asarray(yc) - 0.5 * (y0 + y1), ly, omy, pary)
    lam = np.array([m[0] for m in modes])
    f = np.array([fx[a] * fy[b] for (_, a, b) in modes])
    return lam, f


def log_permeability(lam, f, y_local, mean_y=0.0):
    """Truncated local KL sum Eq. 2.13: ``Y = E[Y] + sum_j xi_j sqrt(lam_j) f_j``."""
    y_local = np.asarray(y_local, dtype=np.float64)
    return mean_y + (np.sqrt(lam) * y_local) @ f


def nystrom_1d(length, eta, n_grid, n_modes):
    """Independent cross-check of ``kl_1d``: eigenvalues of the midpoint-rule
    discretisation ``h * C(x_i, x_j)`` of the 1-D Fredholm operator."""
    h = length / n_grid
    x = (np.arange(n_grid) + 0.5) * h
    cmat = np.exp(-np.abs(x[:, None] - x[None, :]) / eta) * h
    ev = np.linalg.eigvalsh(cmat)[::-1]
    return ev[:n_modes]
