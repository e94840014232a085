"""Stochastic collocation points and weights (Section 4) and the global to
local index conversion of Method S3 (Section 5.4, Step 4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings of the paper taken here:

* A3: the random variables are N(0,1) (Section 2.1), so the 1-D rules are the
  probabilists' Gauss-Hermite rules (zeros of He_m) with weights normalised
  to sum to one, not the physicists' H_m printed in Section 4.
* A4: the Smolyak combination formula of Section 4.2 is implemented for any
  1-D rule sequence ``m(p)``; the workloads use ``m = {1, 3, 3, ...}`` and the
  paper's ``m(p) = 2^(p+1) - 1`` is available as ``rule="paper"``.
"""

import itertools
import math

import numpy as np

_Q = 1e12  # coordinate quantum used to identify equal abscissae


def gauss_hermite(m):
    """m-point probabilists' Gauss-Hermite rule by Golub-Welsch: the nodes are
    the eigenvalues of the Jacobi matrix of the monic He recurrence
    ``He_{k+1} = y He_k - k He_{k-1}`` (off-diagonal ``sqrt(k)``), the weights
    the squared first eigenvector components (total mass 1)."""
    if m == 1:
        return np.array([0.0]), np.array([1.0])
    off = np.sqrt(np.arange(1, m, dtype=np.float64))
    jac = np.diag(off, 1) + np.diag(off, -1)
    nodes, vecs = np.linalg.eigh(jac)
    weights = vecs[0, :] ** 2
    nodes = np.where(np.abs(nodes) < 1e-14, 0.0, nodes)
    return nodes, weights / weights.sum()


def _key(v):
    k = int(round(float(v) * _Q))
    return 0 if k == 0 else k


def tensor_grid(ms):
    """Anisotropic tensor grid of Section 4.1: abscissae
    ``T(m) = H(m(1)) x ... x H(m(N))``, weight = product of 1-D weights.
    Points are in lexicographic order, first dimension slowest."""
    rules = [gauss_hermite(m) for m in ms]
    pts, wts = [], []
    for idx in itertools.product(*[range(m) for m in ms]):
        pts.append([rules[d][0][i] for d, i in enumerate(idx)])
        wts.append(math.prod(rules[d][1][i] for d, i in enumerate(idx)))
    return np.array(pts, dtype=np.float64).reshape(len(pts), len(ms)), np.array(wts)


def _multi_indices(n_dim, total):
    """All sparse multi-indices (tuples of (dim, level>0)) with |p| == total."""
    if total == 0:
        yield ()
        return

    def rec(start, remaining):
        if remaining == 0:
            yield ()
            return
        for d in range(start, n_dim):
            for lev in range(1, remaining + 1):
                for rest in rec(d + 1, remaining - lev):
                    yield ((d, lev),) + rest

    yield from rec(0, total)


def rule_size(p, rule):
    """Points of the 1-D rule of sparse-grid level ``p``: the paper's
    Gauss-Hermite ``2^(p+1) - 1`` (Section 4.2) or a given sequence (reading
    A4)."""
    if rule == "paper":
        return 2 ** (p + 1) - 1
    return rule[p] if p < len(rule) else rule[-1]


def smolyak_grid(n_dim, lmax, rule):
    """Sparse grid of Section 4.2 by the combination formula

    ``sum_{lmin <= |p| <= lmax} (-1)^(lmax-|p|) C(N-1, lmax-|p|) I^TG_{m(p)}``,
    ``lmin = max(0, lmax - N + 1)``. The abscissae are the union of the tensor
    grids; equal abscissae are merged and their weights summed. A merged
    weight adds up terms of opposite signs whose running sums are far larger
    than the result (at level 3 over 64 dimensions, the origin collects about
    2e5 terms against a coefficient of C(63, 3) = 39,711), so each point's
    terms are summed exactly rounded (``math.fsum``); the weights then sum to
    one, as the combination formula integrates constants exactly. Returns
    ``(y[n_pts, N], w[n_pts])`` in lexicographic order of the coordinates.
    """
    lmin = max(0, lmax - n_dim + 1)
    acc = {}
    for q in range(lmin, lmax + 1):
        coef = (-1) ** (lmax - q) * math.comb(n_dim - 1, lmax - q)
        if coef == 0:
            continue
        for mi in _multi_indices(n_dim, q):
            dims = [d for d, _ in mi]
            rules = [gauss_hermite(rule_size(lev, rule)) for _, lev in mi]
            for idx in itertools.product(*[range(len(r[0])) for r in rules]):
                coords = {}
                w = float(coef)
                for d, r, i in zip(dims, rules, idx):
                    if _key(r[0][i]) != 0:
                        coords[d] = r[0][i]
                    w *= r[1][i]
                key = tuple(sorted((d, _key(v)) for d, v in coords.items()))
                if key in acc:
                    acc[key][1].append(w)
                else:
                    acc[key] = [coords, [w]]
    items = []
    for coords, terms in acc.values():
        w = math.fsum(terms)
        y = np.zeros(n_dim)
        for d, v in coords.items():
            y[d] = v
        items.append((tuple(_key(v) for v in y), y, w))
    items.sort(key=lambda t: t[0])
    y = np.array([t[1] for t in items]).reshape(len(items), n_dim)
    w = np.array([t[2] for t in items])
    return y, w


def tensor_sizes(spec, n_dim):
    """Points per global stochastic dimension of a tensor spec (Section 4.1):
    an isotropic ``m``, or the anisotropic multi-index ``m`` given as one count
    per dimension (``m(kappa(i, j)) = m(i, j)``, regions in order)."""
    m = spec["m"]
    if isinstance(m, (list, tuple)):
        if len(m) != n_dim:
            raise ValueError("anisotropic tensor rule of %d dims for %d stochastic dims" % (len(m), n_dim))
        return [int(v) for v in m]
    return [int(m)] * n_dim


def global_grid(spec, n_dim):
    """Global collocation grid for a workload's ``collocation`` spec: the
    tensor rule of Section 4.1 or the sparse grid of Section 4.2."""
    if spec["kind"] == "tensor":
        return tensor_grid(tensor_sizes(spec, n_dim))
    if spec["kind"] == "smolyak":
        return smolyak_grid(n_dim, spec["lmax"], spec["rule"])
    raise ValueError(spec["kind"])


def region_dims(n_terms):
    """Global stochastic index kappa(i, j) of Section 2.1: region i's j-th
    parameter sits at ``j + sum_{k<i} N_term(k)`` (0-based here)."""
    out, off = [], 0
    for n in n_terms:
        out.append(list(range(off, off + n)))
        off += n
    return out


def local_grid(spec, n_local, dims=None):
    """The set of local realizations of one region (Section 5.4, Steps 1-2).

    ``spec["local"] == "tensor"`` (the workloads' reading): the full tensor
    grid over the region's dims, in lexicographic order. On a tensor grid it
    uses the region's own 1-D rules (its entries of an anisotropic ``m``,
    picked by the region's global dims ``dims``); on a sparse grid, the largest
    1-D rule of the sequence (3^N for the rule {1, 3, 3}). Otherwise ``None``:
    the local set is the set of distinct projections of the global points, as
    in the paper's own experiments (Section 6.1: 51 local points of 101)."""
    if spec.get("local", "projections") != "tensor":
        return None
    if spec["kind"] == "tensor":
        m = spec["m"]
        if isinstance(m, (list, tuple)):
            return tensor_grid([int(m[d]) for d in dims])[0]
    else:
        m = max(rule_size(p, spec["rule"]) for p in range(spec["lmax"] + 1))
    return tensor_grid([m] * n_local)[0]


def local_points(y, dims, grid=None):
    """Local realizations of one region and the index map ``k(l)`` of
    Section 5.4 Step 4 from each global point to its local one.

    With ``grid`` (a local tensor grid) the projection of every global point
    is looked up in it; otherwise the local set is the distinct projections
    sorted lexicographically (first dim slowest)."""
    proj = y[:, dims]
    keys = [tuple(_key(v) for v in row) for row in proj]
    if grid is not None:
        pos = {tuple(_key(v) for v in row): i for i, row in enumerate(grid)}
        kmap = np.array([pos[k] for k in keys], dtype=np.int64)
        return np.asarray(grid), kmap
    uniq = sorted(set(keys))
    pos = {k: i for i, k in enumerate(uniq)}
    kmap = np.array([pos[k] for k in keys], dtype=np.int64)
    first = {}
    for l, k in enumerate(keys):
        first.setdefault(k, l)
    loc = np.array([proj[first[k]] for k in uniq]).reshape(len(uniq), len(dims))
    return loc, kmap
