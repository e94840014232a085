"""The coupled collocation-MMMFEM problem and the three algorithms of
Section 5, plus the statistical moments.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``Problem.monolithic``: the plain definition. For one collocation point the
  fully discrete mortar problem Eqs. 4.2-4.4 (all Darcy and Stokes unknowns
  and the mortar multiplier) is assembled as one sparse system and solved
  directly.
* ``Problem.interface_dense``: the interface problem Eqs. 5.9-5.10,
  ``S lambda = g`` with ``S = sum_i R_i^T Phi_i R_i`` built from the
  multiscale flux basis of every subdomain (Section 5.3) and solved densely.
* ``method_s1/s2/s3``: the boxed algorithms of Sections 5.2-5.4 with CG on
  the interface problem, counting subdomain solves (Eqs. 5.11-5.13).
* ``moments``: mean and variance of Eq. 2.1 as collocation-weighted sums,
  the variance in the centred two-pass form (reading A12).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import collocation, kl
from .darcy import DarcySub
from .mortar import Interface
from .stokes import StokesSub


class Problem:
    def __init__(self, w):
        self.w = w
        px, py = w["px"], w["py"]
        x0, x1, y0, y1 = w["darcy_box"]
        W, H = (x1 - x0) / px, (y1 - y0) / py
        deg = w["mortar_degree"]
        self.subs = []
        for iy in range(py):
            for ix in range(px):
                s = iy * px + ix
                nx, ny = w["darcy_grid"][s]
                rect = (x0 + ix * W, x0 + (ix + 1) * W, y0 + iy * H, y0 + (iy + 1) * H)
                self.subs.append(DarcySub(s, rect, nx, ny, w["nu_d"], w["source"][s]))
        sx0, sx1, sy0, sy1 = w["stokes_box"]
        sx, sy = w["stokes_grid"]
        self.stokes = StokesSub((sx0, sx1, sy0, sy1), sx, sy, w["nu_s"], w["alpha"], w["u_in"])
        self.ifaces = []
        off = 0
        for ix in range(px):
            s = (py - 1) * px + ix
            itf = Interface("sd", "x", x0 + ix * W, x0 + (ix + 1) * W, w["mortar_sd"][ix], deg,
                            (s, "top"), ("stokes", "bottom"), off)
            off += itf.n_dof
            self.ifaces.append(itf)
            self.subs[s].sides["top"] = ("iface", itf)
            self.stokes.ifaces.append(itf)
        for iy in range(py):
            for ix in range(px - 1):
                s = iy * px + ix
                itf = Interface("dd_v", "y", y0 + iy * H, y0 + (iy + 1) * H,
                                w["mortar_dd_v"][iy][ix], deg, (s, "right"), (s + 1, "left"), off)
                off += itf.n_dof
                self.ifaces.append(itf)
                self.subs[s].sides["right"] = ("iface", itf)
                self.subs[s + 1].sides["left"] = ("iface", itf)
        for iy in range(py - 1):
            for ix in range(px):
                s = iy * px + ix
                itf = Interface("dd_h", "x", x0 + ix * W, x0 + (ix + 1) * W,
                                w["mortar_dd_h"][iy][ix], deg, (s, "top"), (s + px, "bottom"), off)
                off += itf.n_dof
                self.ifaces.append(itf)
                self.subs[s].sides["top"] = ("iface", itf)
                self.subs[s + px].sides["bottom"] = ("iface", itf)
        for ix in range(px):
            self.subs[ix].sides["bottom"] = ("dirichlet", w["bottom_pressure"])
        self.n_lambda = off
        for sub in self.subs:
            sub.finalize()
        self.stokes.finalize()
        # KL regions (Section 2.1): statistically independent, each a union of
        # subdomains. By default one per Darcy subdomain; a workload may give
        # region rectangles ("regions") and each subdomain's region
        # ("region_of"), as in Case 1 of Section 6.1 (two regions of two
        # subdomains). n_term, modes and the stochastic dims are per region.
        klw = w["kl"]
        self.n_term = list(klw["n_term"])
        rects = klw.get("regions") or [sub.rect for sub in self.subs]
        self.region_of = list(klw.get("region_of") or range(len(self.subs)))
        self.dims = collocation.region_dims(self.n_term)
        self.n_dim = sum(self.n_term)
        self.kl = []
        for s, sub in enumerate(self.subs):
            r = self.region_of[s]
            xc, yc = sub.cell_centres()
            modes = (klw.get("modes") or [None] * len(self.n_term))[r]
            lam, f = kl.kl_region_fields(rects[r], klw["sigma2"], klw["eta"], self.n_term[r], xc, yc, modes)
            self.kl.append((lam, f))
        self.mean_y = klw["mean_Y"]
        spec = w["collocation"]
        self.local_grids = [collocation.local_grid(spec, n, d) for n, d in zip(self.n_term, self.dims)]
        self._stokes_basis = None
        self.n_solves = np.zeros(len(self.subs) + 1, dtype=np.int64)

    # ---- stochastic inputs -------------------------------------------------
    def grid(self):
        """Global collocation points and weights (Section 4)."""
        return collocation.global_grid(self.w["collocation"], self.n_dim)

    def local_realizations(self, s, ys):
        """Local realizations of subdomain ``s``'s KL region and the map from
        the global points ``ys`` to them (Section 5.4, Steps 1-2 and 4)."""
        r = self.region_of[s]
        return collocation.local_points(np.asarray(ys), self.dims[r], self.local_grids[r])

    def local_y(self, s, y_global):
        """Coordinates of a global point in subdomain ``s``'s KL region: its
        dims kappa(i, j) (Section 2.1; Section 5.4 Step 4)."""
        return np.asarray(y_global)[self.dims[self.region_of[s]]]

    def permeability(self, s, y_local):
        """Cell permeabilities ``K = exp(Y)`` with ``Y`` the truncated local KL
        sum of Eq. 2.13 at the cell centres (reading A11)."""
        lam, f = self.kl[s]
        return np.exp(kl.log_permeability(lam, f, y_local, self.mean_y))

    # ---- bases ---------------------------------------------------------------
    def darcy_basis(self, s, y_local):
        """(Phi_i, g_i, X_i, K) of Darcy subdomain ``s`` for one local
        realization: the multiscale flux basis of Section 5.3 Step 2 built per
        local realization as in Section 5.4 Step 2."""
        K = self.permeability(s, y_local)
        phi, g, X = self.subs[s].flux_basis(K)
        self.n_solves[s] += len(self.subs[s].dofs) + 1
        return phi, g, X, K

    def stokes_basis(self):
        """The Stokes subdomain's velocity-response basis (Section 5.3 Step 2),
        built once: Section 5.4 sets N_real = 1 for Stokes (reading A7)."""
        if self._stokes_basis is None:
            self._stokes_basis = self.stokes.flux_basis()
            self.n_solves[-1] += len(self.stokes.dofs) + 1
        return self._stokes_basis

    def assemble_interface(self, bases):
        """``S = sum_i R_i^T Phi_i R_i + R_s^T Phi_s R_s`` and
        ``g = sum_i R_i^T g_i + R_s^T g_s`` (Eqs. 5.9-5.10)."""
        S = np.zeros((self.n_lambda, self.n_lambda))
        g = np.zeros(self.n_lambda)
        for sub, (phi, gi) in zip(self.subs, bases):
            d = np.array(sub.dofs)
            S[np.ix_(d, d)] += phi
            g[d] += gi
        phs, gs, _, _ = self.stokes_basis()
        d = np.array(self.stokes.dofs)
        S[np.ix_(d, d)] += phs
        g[d] += gs
        return S, g

    def interface_dense(self, y_global):
        """Dense interface solve for one global point: ``S lambda = g`` of
        Eqs. 5.9-5.10 with ``S`` assembled from the flux bases and solved
        directly. Returns ``(lambda, S, g, per-subdomain (Phi, g, X, K))``."""
        bs = [self.darcy_basis(s, self.local_y(s, y_global)) for s in range(len(self.subs))]
        S, g = self.assemble_interface([(b[0], b[1]) for b in bs])
        lam = np.linalg.solve(S, g)
        return lam, S, g, bs

    # ---- recovery and fields ---------------------------------------------------
    def recover(self, lam, darcy_bases):
        """Fields of one point from the mortar solution: Darcy pressures
        ``X_i [R_i lambda; 1]`` and face velocities, Stokes velocity and
        pressure ``U_s [R_s lambda; 1]`` (``u = u*(lambda) + u_bar``, Section 5.1)."""
        out = {"darcy_p": [], "darcy_flux": [], "stokes_u": None, "stokes_p": None}
        for sub, (phi, gi, X, K) in zip(self.subs, darcy_bases):
            c = lam[np.array(sub.dofs)]
            p = X @ np.append(c, 1.0)
            ux, uy = sub.fields(K, p, c)
            out["darcy_p"].append(p)
            out["darcy_flux"].append(np.concatenate([ux.ravel(), uy.ravel()]))
        _, _, U, Pp = self.stokes_basis()
        cs = np.append(lam[np.array(self.stokes.dofs)], 1.0)
        out["stokes_u"] = U @ cs
        out["stokes_p"] = Pp @ cs
        out["darcy_p"] = np.concatenate(out["darcy_p"])
        out["darcy_flux"] = np.concatenate(out["darcy_flux"])
        return out

    # ---- the plain definition: one monolithic solve ----------------------------
    def monolithic(self, y_global):
        """Assemble and solve Eqs. 4.2-4.4 for one global point directly.

        Unknowns ``[p_1 .. p_Nd, u_s, p_s, lambda]``. Darcy rows
        ``A_i p_i - B_i lambda_i = b_bar_i``; Stokes rows
        ``A_s u + B_s^T p_s + N_s lambda_s = 0``, ``B_s u = 0`` with the Dirichlet
        data eliminated; mortar rows (weak flux continuity Eq. 4.4)
        ``sum_i R_i^T (B_i^T p_i - M_i lambda_i) + R_s^T N_s^T u = 0`` with
        ``M_i = P^T D_T P``. Returns ``(lambda, fields)``."""
        blocks = []
        nL = self.n_lambda
        offs = []
        off = 0
        for sub in self.subs:
            offs.append(off)
            off += sub.n_cells
        st = self.stokes
        nu_ = 2 * st.n_nodes
        off_u = off
        off_p = off_u + nu_
        off_l = off_p + st.n_p
        n = off_l + nL
        rows, cols, vals = [], [], []
        rhs = np.zeros(n)

        def add(mat, r0, c0, rmap=None, cmap=None):
            m = sp.coo_matrix(mat)
            r = m.row if rmap is None else np.asarray(rmap)[m.row]
            c = m.col if cmap is None else np.asarray(cmap)[m.col]
            rows.append(r + r0); cols.append(c + c0); vals.append(m.data)

        Ks = []
        for s, sub in enumerate(self.subs):
            K = self.permeability(s, self.local_y(s, y_global))
            Ks.append(K)
            A, B, bbar = sub.assemble(K)
            d = np.array(sub.dofs)
            add(A, offs[s], offs[s])
            add(-B, offs[s], off_l, cmap=d)
            rhs[offs[s]:offs[s] + sub.n_cells] = bbar
            # mortar rows: B_i^T p_i - M_i lambda_i
            M = np.zeros((len(d), len(d)))
            for side in ("bottom", "right", "top", "left"):
                if sub.sides[side][0] == "iface":
                    p = sub.projection(side)
                    M += p.T @ (sub.boundary_trans(K, side)[:, None] * p)
            add(B.T, off_l, offs[s], rmap=d)
            add(-M, off_l, off_l, rmap=d, cmap=d)
        A_s, B_s = st.assemble()
        N = st.neumann_matrix()
        ds = np.array(st.dofs)
        rhs[off_u:off_p] = st.load()
        mask, val = st.dirichlet()
        add(A_s, off_u, off_u)
        add(B_s.T, off_u, off_p)
        add(B_s, off_p, off_u)
        add(N, off_u, off_l, cmap=ds)
        add(N.T, off_l, off_u, rmap=ds)
        Mfull = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                              shape=(n, n))
        dir_idx = off_u + np.where(mask)[0]
        xdir = np.zeros(n)
        xdir[dir_idx] = val[mask]
        rhs = rhs - Mfull @ xdir
        keep = np.setdiff1d(np.arange(n), dir_idx)
        sol = np.zeros(n)
        sol[dir_idx] = val[mask]
        sol[keep] = spla.spsolve(Mfull[keep][:, keep].tocsc(), rhs[keep])
        lam = sol[off_l:]
        fields = {"darcy_p": sol[:off_u].copy(), "stokes_u": sol[off_u:off_p].copy(),
                  "stokes_p": sol[off_p:off_l].copy()}
        flux = []
        for s, sub in enumerate(self.subs):
            p = sol[offs[s]:offs[s] + sub.n_cells]
            ux, uy = sub.fields(Ks[s], p, lam[np.array(sub.dofs)])
            flux.append(np.concatenate([ux.ravel(), uy.ravel()]))
        fields["darcy_flux"] = np.concatenate(flux)
        return lam, fields


# ---- Krylov -----------------------------------------------------------------------
def cg(apply, g, rtol, max_it):
    """Plain conjugate gradients from zero (the interface operator is SPD,
    Section 5.1); stops at ``||r|| <= rtol ||g||``. Returns ``(x, iters)``."""
    x = np.zeros_like(g)
    r = g.copy()
    p = r.copy()
    rr = r @ r
    gn = np.sqrt(g @ g)
    if gn == 0.0:
        return x, 0
    for it in range(1, max_it + 1):
        q = apply(p)
        alpha = rr / (p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = r @ r
        if np.sqrt(rr_new) <= rtol * gn:
            return x, it
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, -max_it


# ---- the three algorithms -------------------------------------------------------------
def method_s1(prob, ys, rtol=1e-12, max_it=2000):
    """Method S1 (Section 5.2): every CG iteration applies S_H by one Dirichlet
    (Darcy) / Neumann (Stokes) subdomain solve per subdomain. Returns the
    per-point mortar solutions, CG iterations and per-subdomain solve counts."""
    counts = np.zeros(len(prob.subs) + 1, dtype=np.int64)
    lams, iters = [], []
    for y in ys:
        Ks = [prob.permeability(s, prob.local_y(s, y)) for s in range(len(prob.subs))]
        lus = []
        rhs_g = np.zeros(prob.n_lambda)
        for s, sub in enumerate(prob.subs):
            A, B, bbar = sub.assemble(Ks[s])
            lu = spla.splu(A)
            lus.append((lu, B))
            xb = lu.solve(bbar)                        # right-hand side solve
            fl = sub.interface_flux(Ks[s], xb[:, None], np.zeros((len(sub.dofs), 1)))
            rhs_g[np.array(sub.dofs)] += fl[:, 0]
            counts[s] += 1
        st = prob.stokes
        N = st.neumann_matrix()
        ub, _ = st.solve(np.zeros(2 * st.n_nodes), True)
        rhs_g[np.array(st.dofs)] += (N.T @ ub)[:, 0]
        counts[-1] += 1

        def apply(lmb):
            out = np.zeros(prob.n_lambda)
            for s, sub in enumerate(prob.subs):
                d = np.array(sub.dofs)
                lu, B = lus[s]
                c = lmb[d][:, None]
                x = lu.solve(B @ c)
                out[d] -= sub.interface_flux(Ks[s], x, c)[:, 0]
                counts[s] += 1
            u, _ = st.solve(-N @ lmb[np.array(st.dofs)], False)
            out[np.array(st.dofs)] -= (N.T @ u)[:, 0]
            counts[-1] += 1
            return out

        lam, it = cg(apply, rhs_g, rtol, max_it)
        for s in range(len(prob.subs)):
            counts[s] += 1                              # recovery solve
        counts[-1] += 1
        lams.append(lam)
        iters.append(it)
    return np.array(lams), np.array(iters), counts


def method_s2(prob, ys, rtol=1e-12, max_it=2000):
    """Method S2 (Section 5.3): a fresh multiscale flux basis (R_i solves)
    per global point, CG by linear combination of the basis, plus the RHS and
    recovery solves."""
    counts = np.zeros(len(prob.subs) + 1, dtype=np.int64)
    lams, iters = [], []
    for y in ys:
        bases = []
        for s, sub in enumerate(prob.subs):
            K = prob.permeability(s, prob.local_y(s, y))
            phi, g, _ = sub.flux_basis(K)
            bases.append((phi, g))
            counts[s] += len(sub.dofs) + 2
        S, g = prob.assemble_interface(bases)
        lam, it = cg(lambda v: S @ v, g, rtol, max_it)
        lams.append(lam)
        iters.append(it)
    counts[-1] = len(prob.stokes.dofs) + 2
    return np.array(lams), np.array(iters), counts


def method_s3(prob, ys, rtol=1e-12, max_it=2000):
    """Method S3 (Section 5.4): pre-computation loop over every subdomain's
    local realizations (Steps 1-2), then the global loop (Steps 3-6) that
    converts the global index to the local one and solves with the stored
    basis; 2 extra solves per global point (RHS and recovery)."""
    counts = np.zeros(len(prob.subs) + 1, dtype=np.int64)
    store, kmaps = [], []
    for s, sub in enumerate(prob.subs):
        loc, kmap = prob.local_realizations(s, ys)
        kmaps.append(kmap)
        entries = []
        for yl in loc:
            K = prob.permeability(s, yl)
            phi, g, _ = sub.flux_basis(K)
            entries.append((phi, g))
        store.append(entries)
        counts[s] += len(sub.dofs) * len(loc)
    lams, iters = [], []
    for l, y in enumerate(ys):
        bases = [store[s][kmaps[s][l]] for s in range(len(prob.subs))]
        S, g = prob.assemble_interface(bases)
        lam, it = cg(lambda v: S @ v, g, rtol, max_it)
        lams.append(lam)
        iters.append(it)
        for s in range(len(prob.subs)):
            counts[s] += 2
    counts[-1] = len(prob.stokes.dofs) + 2
    return np.array(lams), np.array(iters), counts


# ---- moments --------------------------------------------------------------------------------
def moments(values, weights):
    """Collocation mean ``sum_l w_l x_l`` and centred variance
    ``sum_l w_l (x_l - mean)^2`` (Eq. 2.1 and the variance below it, two-pass
    form, reading A12). ``values`` is ``(n_pts, n_entries)``."""
    v = np.asarray(values, dtype=np.float64)
    w = np.asarray(weights, dtype=np.float64)
    mean = w @ v
    var = w @ (v - mean) ** 2
    return mean, var


def solve_all(prob, ys, ws):
    """Reference result for a set of global points: per-point mortar solution
    and fields from the dense interface solve (Section 5.4 Steps 3-6), then
    the mean (Eq. 2.1) and variance of each field (reading A12)."""
    lams = []
    fields = {"darcy_p": [], "darcy_flux": [], "stokes_u": [], "stokes_p": []}
    cache = {}
    kmaps = [prob.local_realizations(s, ys)[1] for s in range(len(prob.subs))]
    for l, y in enumerate(ys):
        bases = []
        for s in range(len(prob.subs)):
            key = (s, kmaps[s][l])
            if key not in cache:
                cache[key] = prob.darcy_basis(s, prob.local_y(s, y))
            bases.append(cache[key])
        S, g = prob.assemble_interface([(b[0], b[1]) for b in bases])
        lam = np.linalg.solve(S, g)
        lams.append(lam)
        f = prob.recover(lam, bases)
        for k in fields:
            fields[k].append(f[k])
    mom = {k: moments(np.array(v), ws) for k, v in fields.items()}
    return np.array(lams), mom
