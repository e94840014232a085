"""Synthetic Stokes-Darcy workloads shared by the oracle, the tests and the bench.

This module is pure input data: geometry, grid and mortar sizes, KL parameters,
collocation specification and the seeded draws of the uneven batched workload.
It holds none of the method's arithmetic, so both the CPU oracle (``oracle/``)
and the CUDA path (``paper_1802_06263_gb300``) can consume it without sharing
any computation.

Geometry convention (the paper's test cases, Section 6; where the paper is
silent, the reading stated with each item):

* The Darcy region ``darcy_box = (x0, x1, y0, y1)`` is tiled by a ``px x py``
  array of rectangular subdomains of equal size. Subdomain ``s = iy * px + ix``
  (bottom row first) has an ``nx x ny`` cell grid ``darcy_grid[s]`` and is its
  own KL region, unless ``kl["regions"]`` lists region rectangles and
  ``kl["region_of"]`` each subdomain's region (``n_term`` and ``modes`` are
  then per region).
* One Stokes subdomain covers ``stokes_box = (x0, x1, y1, y2)`` directly above
  the Darcy region, with an ``Sx x Sy`` rectangle grid (two triangles each).
* Interfaces: one Stokes-Darcy edge per top-row Darcy subdomain, one vertical
  Darcy-Darcy edge between horizontally adjacent subdomains, one horizontal
  Darcy-Darcy edge between vertically adjacent ones. ``mortar_sd[ix]``,
  ``mortar_dd_v[iy][ix]`` and ``mortar_dd_h[iy][ix]`` give the number of
  mortar elements on each.
* Boundary data: zero pressure (``bottom_pressure``) on the Darcy bottom,
  no flow on the Darcy left and right edges, parabolic inflow with peak
  ``u_in`` on the Stokes left edge, no slip on the Stokes top, zero stress on
  the Stokes right edge (Section 6.1).
"""

import random

PI_SEED = 20180216  # fixed seed of the uneven draws (arXiv 1802.06263)


def _uniform_edges(px, py, n_sd, n_dd):
    return (
        [n_sd] * px,
        [[n_dd] * (px - 1) for _ in range(py)],
        [[n_dd] * px for _ in range(py - 1)],
    )


def _base(name, px, py, grid, stokes_grid, n_sd, n_dd, n_term, sigma2, eta,
          collocation, degree=1):
    sd, dv, dh = _uniform_edges(px, py, n_sd, n_dd)
    return {
        "name": name,
        "darcy_box": (0.0, 1.0, 0.0, 0.5),
        "stokes_box": (0.0, 1.0, 0.5, 1.0),
        "px": px,
        "py": py,
        "darcy_grid": [tuple(grid)] * (px * py),
        "stokes_grid": tuple(stokes_grid),
        "mortar_degree": degree,
        "mortar_sd": sd,
        "mortar_dd_v": dv,
        "mortar_dd_h": dh,
        "kl": {
            "sigma2": sigma2,
            "eta": tuple(eta),
            "n_term": [n_term] * (px * py),
            "mean_Y": 0.0,
        },
        "collocation": dict(collocation),
        "nu_s": 1.0,
        "nu_d": 1.0,
        "alpha": 1.0,
        "u_in": 1.0,
        "bottom_pressure": 0.0,
        "source": [0.0] * (px * py),
        "n_batch": None,
    }


def tiny():
    """Two 8x8 Darcy subdomains side by side, 8x8 Stokes, 2 mortar elements
    per edge, N_term = 2 per region, tensor 2-point Gauss-Hermite (16 points)."""
    return _base("tiny", 2, 1, (8, 8), (8, 8), 2, 2, 2, 1.0, (0.25, 0.125),
                 {"kind": "tensor", "m": 2, "local": "tensor"})


def medium():
    """2x2 Darcy subdomains of 32x32 cells, N_term = 3 each (12 dims), 4
    linear mortar elements per edge, Smolyak level 2 with 1-D rules {1,3,3}."""
    return _base("medium", 2, 2, (32, 32), (32, 32), 4, 4, 3, 1.0, (0.2, 0.1),
                 {"kind": "smolyak", "lmax": 2, "rule": [1, 3, 3], "local": "tensor"})


def precision():
    """4x2 Darcy subdomains of 64x64 cells, N_term = 4 (81 local points),
    sigma^2 = 2, 8 linear mortar elements per edge, Smolyak level 2 over 32
    dims (2,049 points). Stokes 32x32."""
    return _base("precision", 4, 2, (64, 64), (32, 32), 8, 8, 4, 2.0, (0.2, 0.1),
                 {"kind": "smolyak", "lmax": 2, "rule": [1, 3, 3], "local": "tensor"})


def batched(seed=PI_SEED):
    """4x3 Darcy subdomains with nx, ny drawn from {24,48,64,96}, mortar
    elements per edge from {3,4,6,8} and N_term from 2..5 (9..243 local
    points), Smolyak level 2; the first 2,000 grid points form the batch."""
    rng = random.Random(seed)
    px, py = 4, 3
    w = _base("batched", px, py, (24, 24), (32, 32), 4, 4, 2, 1.0, (0.2, 0.1),
              {"kind": "smolyak", "lmax": 2, "rule": [1, 3, 3], "local": "tensor"})
    w["darcy_grid"] = [(rng.choice([24, 48, 64, 96]), rng.choice([24, 48, 64, 96]))
                       for _ in range(px * py)]
    w["mortar_sd"] = [rng.choice([3, 4, 6, 8]) for _ in range(px)]
    w["mortar_dd_v"] = [[rng.choice([3, 4, 6, 8]) for _ in range(px - 1)] for _ in range(py)]
    w["mortar_dd_h"] = [[rng.choice([3, 4, 6, 8]) for _ in range(px)] for _ in range(py - 1)]
    w["kl"]["n_term"] = [rng.choice([2, 3, 4, 5]) for _ in range(px * py)]
    w["n_batch"] = 2000
    w["seed"] = seed
    return w


def large():
    """4x4 Darcy subdomains of 128x128, N_term = 4, quadratic mortars with 8
    elements per edge, Smolyak level 3 over 64 dims, Stokes 128x128."""
    return _base("large", 4, 4, (128, 128), (128, 128), 8, 8, 4, 1.0, (0.2, 0.1),
                 {"kind": "smolyak", "lmax": 3, "rule": [1, 3, 3, 3], "local": "tensor"}, degree=2)


def small_test(nx=12, ny=10, px=2, py=2, n_sd=3, n_dd=2, n_term=2, degree=1,
               stokes=(6, 6), collocation=None, sigma2=1.0, eta=(0.2, 0.1),
               bottom_pressure=0.0, source=None, name="small_test"):
    """A parametrised small case for tests: ragged grid sizes and mortar
    counts that do not divide the cell counts."""
    col = collocation or {"kind": "tensor", "m": 2, "local": "tensor"}
    w = _base(name, px, py, (nx, ny), stokes, n_sd, n_dd, n_term, sigma2, eta,
              col, degree=degree)
    w["bottom_pressure"] = bottom_pressure
    if source is not None:
        w["source"] = list(source)
    return w


def anisotropic():
    """Two 10x6 Darcy subdomains whose KL regions keep the paper's n1 x n2
    mode sets (2 x 1 and 2 x 2, as written in Section 6.1), on an anisotropic
    tensor grid (Section 4.1) with 2, 1, 3, 1, 2, 2 points in the six
    stochastic dimensions (24 global points; 2 and 12 local ones). A 1-point
    rule fixes its dimension at the mean."""
    w = small_test(nx=10, ny=6, px=2, py=1, n_sd=2, n_dd=2, n_term=2, degree=1, stokes=(6, 5),
                   sigma2=1.5, eta=(0.3, 0.15),
                   collocation={"kind": "tensor", "m": [2, 1, 3, 1, 2, 2], "local": "tensor"},
                   name="anisotropic")
    w["kl"]["n_term"] = [2, 4]
    w["kl"]["modes"] = [(2, 1), (2, 2)]
    return w


def kl_regions():
    """2x2 Darcy subdomains of 8x6 cells whose KL regions are the two rows,
    (0,1)x(0,0.25) and (0,1)x(0.25,0.5), each spanning two subdomains, as in
    Case 1 of Section 6.1. The bottom region keeps the paper's 2 x 1 mode set,
    the top one its 3 largest modes. Tensor 2-point rule: 32 global points,
    4 and 8 local ones per region (shared by its two subdomains)."""
    w = small_test(nx=8, ny=6, px=2, py=2, n_sd=2, n_dd=2, n_term=2, degree=1, stokes=(6, 5),
                   sigma2=1.0, eta=(0.2, 0.1), name="kl_regions")
    w["kl"]["n_term"] = [2, 3]
    w["kl"]["modes"] = [(2, 1), None]
    w["kl"]["regions"] = [(0.0, 1.0, 0.0, 0.25), (0.0, 1.0, 0.25, 0.5)]
    w["kl"]["region_of"] = [0, 0, 1, 1]
    return w


ALL = {"tiny": tiny, "medium": medium, "precision": precision,
       "batched": batched, "large": large, "anisotropic": anisotropic, "kl_regions": kl_regions}
