"""Python binding of the GB300 stochastic multiscale flux basis library.

Thin ctypes marshalling over the C ABI declared in ``include/sfb.h``; every
step of the method runs in the library's CUDA kernels. PyTorch is used only
for device memory (the workspace) and the CUDA stream. The binding fails
loudly if the compiled library is missing: there is no CPU fallback.

Method: Ambartsumyan, Khattatov, Wang, Yotov, "Stochastic multiscale flux
basis for Stokes-Darcy flows" (arXiv 1802.06263), Method S3 (Section 5.4).
"""

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH, build  # noqa: F401

SFB_OK = 0
SFB_ERR_NOT_CONVERGED = 6
SFB_ERR_TIMEOUT = 9
# basis builds: FACTOR_FP64 is Method S1's set-up (FP64 block factors and g, no flux basis)
FP64, MIXED, FP32_NOREFINE, FACTOR_FP64 = 0, 1, 2, 3
# interface solvers: CG_DTN is Method S1 (a subdomain solve per CG iteration)
CG, CG_MIXED, GMRES, GMRES_MIXED, CG_DTN = 0, 1, 2, 3, 4
FIELDS = {"darcy_p": 0, "darcy_flux": 1, "stokes_u": 2, "stokes_p": 3}
STATUS = {0: "OK", 1: "ARG", 2: "STATE", 3: "CUDA", 4: "WORKSPACE", 5: "NONFINITE",
          6: "NOT_CONVERGED", 7: "NOT_SPD", 8: "UNSUPPORTED", 9: "TIMEOUT"}

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    _fields_ = [("darcy_box", ctypes.c_double * 4), ("stokes_box", ctypes.c_double * 4),
                ("px", ctypes.c_int32), ("py", ctypes.c_int32),
                ("darcy_nx", _i32p), ("darcy_ny", _i32p),
                ("stokes_sx", ctypes.c_int32), ("stokes_sy", ctypes.c_int32),
                ("mortar_degree", ctypes.c_int32),
                ("mortar_sd", _i32p), ("mortar_dd_v", _i32p), ("mortar_dd_h", _i32p),
                ("nu_s", ctypes.c_double), ("nu_d", ctypes.c_double), ("alpha", ctypes.c_double),
                ("u_in", ctypes.c_double), ("bottom_pressure", ctypes.c_double),
                ("source", _f64p)]


class KLRegion(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("eta1", ctypes.c_double), ("eta2", ctypes.c_double),
                ("mean_y", ctypes.c_double), ("n_term", ctypes.c_int32),
                ("n_modes_x", ctypes.c_int32), ("n_modes_y", ctypes.c_int32)]


class Collocation(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("m", ctypes.c_int32), ("lmax", ctypes.c_int32),
                ("n_rule", ctypes.c_int32), ("rule", _i32p), ("local_tensor", ctypes.c_int32),
                ("m_dim", _i32p)]


class BasisStats(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int64), ("n_flux_responses", ctypes.c_int64),
                ("max_refine_steps", ctypes.c_int32), ("n_not_converged", ctypes.c_int32),
                ("max_rel_residual", ctypes.c_double), ("max_first_correction", ctypes.c_double),
                ("max_error_estimate", ctypes.c_double), ("ms", ctypes.c_double),
                ("phase_cycles", ctypes.c_double * 16), ("kernel_ms", ctypes.c_double),
                ("flops_fp32", ctypes.c_double), ("flops_fp64", ctypes.c_double),
                ("launch_shape", ctypes.c_int32 * 2), ("graph", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("tune_ms", (ctypes.c_double * 4) * 2), ("mean_refine_steps", ctypes.c_double)]


_SIGS = {
    "sfb_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "sfb_destroy": (None, [ctypes.c_void_p]),
    "sfb_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "sfb_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_sizes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), _i32p]),
    "sfb_subdomain_dofs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _i32p, ctypes.c_void_p]),
    "sfb_field_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "sfb_kl_setup": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KLRegion), ctypes.c_int32, ctypes.c_void_p]),
    "sfb_kl_tables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "sfb_kl_setup_regions": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(KLRegion), ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_collocation_setup": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Collocation),
                                             ctypes.POINTER(ctypes.c_int64)]),
    "sfb_collocation_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_local_points": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _i32p, ctypes.c_void_p]),
    "sfb_workspace_size": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "sfb_set_workspace": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "sfb_build_stochastic_basis": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(BasisStats)]),
    "sfb_get_basis": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_interface_solve_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                 ctypes.c_int32, ctypes.c_double, ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_void_p]),
    "sfb_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_moments_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "sfb_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_double]),
    "sfb_solve_timings": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _i32p]),
    "sfb_cg_phase_cycles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "sfb_launch_count": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "sfb_basis_launch_shape": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _i32p, _i32p, _i32p,
                                              _i32p, _i32p]),
    "sfb_build_basis_item_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}

_lib = None


def library_path():
    return _LIB_PATH


def load():
    """Load ``lib/libsfb.so`` (built by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError("libsfb.so is not built (%s); run __graft_entry__.build()" % _LIB_PATH)
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def basis_launch_shape(prec, wide, shape):
    """(threads per CTA, CTAs per SM, G buffers, tcgen05, split) of a
    basis-kernel launch shape (tcgen05 = 1: the tensor-core form; split = 1:
    factor launches, then launches over column chunks, which the other values
    describe), or None when the precision has no such shape for that size
    class."""
    lib = load()
    t, c, g, tc, sp = (ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32())
    rc = lib.sfb_basis_launch_shape(prec, int(bool(wide)), shape, ctypes.byref(t), ctypes.byref(c), ctypes.byref(g),
                                    ctypes.byref(tc), ctypes.byref(sp))
    if rc != SFB_OK:
        return None
    return t.value, c.value, g.value, tc.value, sp.value


class SfbError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def _ptr(a):
    """Address of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _i32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


class Solver:
    """One problem instance: marshals a workload description into the C ABI.

    ``workload`` is a dict as produced by ``sfb_workloads``. ``stream`` is a
    torch CUDA stream (default: the current stream).
    """

    def __init__(self, workload, stream=None):
        import torch

        self.lib = load()
        self.w = workload
        w = workload
        px, py = w["px"], w["py"]
        self._keep = []
        nx = _i32([g[0] for g in w["darcy_grid"]])
        ny = _i32([g[1] for g in w["darcy_grid"]])
        msd = _i32(w["mortar_sd"])
        mdv = _i32([v for row in w["mortar_dd_v"] for v in row]) if px > 1 else _i32([0])
        mdh = _i32([v for row in w["mortar_dd_h"] for v in row]) if py > 1 else _i32([0])
        src = np.ascontiguousarray(np.asarray(w["source"], dtype=np.float64))
        self._keep += [nx, ny, msd, mdv, mdh, src]
        P = Problem()
        P.darcy_box[:] = list(w["darcy_box"])
        P.stokes_box[:] = list(w["stokes_box"])
        P.px, P.py = px, py
        P.darcy_nx = nx.ctypes.data_as(_i32p)
        P.darcy_ny = ny.ctypes.data_as(_i32p)
        P.stokes_sx, P.stokes_sy = w["stokes_grid"]
        P.mortar_degree = w["mortar_degree"]
        P.mortar_sd = msd.ctypes.data_as(_i32p)
        P.mortar_dd_v = mdv.ctypes.data_as(_i32p)
        P.mortar_dd_h = mdh.ctypes.data_as(_i32p)
        P.nu_s, P.nu_d, P.alpha = w["nu_s"], w["nu_d"], w["alpha"]
        P.u_in, P.bottom_pressure = w["u_in"], w["bottom_pressure"]
        P.source = src.ctypes.data_as(_f64p)
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        sptr = ctypes.c_void_p(stream.cuda_stream) if stream is not None else ctypes.c_void_p()
        self._check(self.lib.sfb_create(ctypes.byref(P), sptr, ctypes.byref(h)), ctx=None)
        self.h = h
        n_l = ctypes.c_int64()
        n_d = ctypes.c_int32()
        self.lib.sfb_sizes(self.h, ctypes.byref(n_l), ctypes.byref(n_d))
        self.n_lambda, self.n_darcy = n_l.value, n_d.value
        kl = w["kl"]
        # KL regions: one per Darcy subdomain, or the workload's rectangles
        # ("regions") with each subdomain's region ("region_of")
        n_reg = len(kl["n_term"])
        regs = (KLRegion * n_reg)()
        for r in range(n_reg):
            regs[r].sigma2 = kl["sigma2"]
            regs[r].eta1, regs[r].eta2 = kl["eta"]
            regs[r].mean_y = kl["mean_Y"]
            regs[r].n_term = kl["n_term"][r]
            modes = (kl.get("modes") or [None] * n_reg)[r]
            if modes is not None:
                regs[r].n_modes_x, regs[r].n_modes_y = modes
        self.n_dim = int(sum(kl["n_term"]))
        self.eigvals = np.zeros(self.n_dim)
        if kl.get("regions"):
            rects = np.ascontiguousarray(np.asarray(kl["regions"], dtype=np.float64).reshape(n_reg, 4))
            region_of = _i32(kl["region_of"])
            self._keep += [rects, region_of]
            self._check(self.lib.sfb_kl_setup_regions(self.h, regs, n_reg, rects.ctypes.data, region_of.ctypes.data,
                                                      self.eigvals.ctypes.data))
        else:
            self._check(self.lib.sfb_kl_setup(self.h, regs, n_reg, self.eigvals.ctypes.data))
        col = w["collocation"]
        C = Collocation()
        C.kind = 0 if col["kind"] == "tensor" else 1
        m = col.get("m", 0)
        if isinstance(m, (list, tuple)):
            # anisotropic tensor rule: points per global stochastic dimension
            m_dim = _i32(m)
            self._keep.append(m_dim)
            C.m_dim = m_dim.ctypes.data_as(_i32p)
            m = 0
        C.m = m
        C.lmax = col.get("lmax", 0)
        rule = col.get("rule", [])
        if rule == "paper":
            rule = []
        rule_a = _i32(rule if rule else [0])
        self._keep.append(rule_a)
        C.n_rule = len(rule)
        C.rule = rule_a.ctypes.data_as(_i32p)
        # local realizations: "tensor" (the region's full local tensor grid),
        # "projections" (the distinct projections of the global grid: Method
        # S3) or "per_point" (one per global point, repeats kept: Method S2)
        C.local_tensor = {"projections": 0, "tensor": 1, "per_point": 2}[col.get("local", "projections")]
        npts = ctypes.c_int64()
        self._check(self.lib.sfb_collocation_setup(self.h, ctypes.byref(C), ctypes.byref(npts)))
        self.n_pts = npts.value
        self.ws = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self.lib.sfb_destroy(self.h)
                self.h = None
        except Exception:
            pass

    def _check(self, st, ctx=True):
        if st != SFB_OK:
            msg = self.lib.sfb_last_error(self.h).decode() if ctx else ""
            raise SfbError(st, msg)

    # ---- sizes and set-up data --------------------------------------------------------
    def subdomain_dofs(self, sub):
        n = ctypes.c_int32()
        self._check(self.lib.sfb_subdomain_dofs(self.h, sub, ctypes.byref(n), None))
        out = np.zeros(n.value, dtype=np.int64)
        self._check(self.lib.sfb_subdomain_dofs(self.h, sub, ctypes.byref(n), out.ctypes.data))
        return out

    def field_size(self, field):
        n = ctypes.c_int64()
        self._check(self.lib.sfb_field_size(self.h, FIELDS[field], ctypes.byref(n)))
        return n.value

    def points(self):
        y = np.zeros((self.n_pts, self.n_dim))
        w = np.zeros(self.n_pts)
        self._check(self.lib.sfb_collocation_points(self.h, y.ctypes.data, w.ctypes.data))
        return y, w

    def kl_tables(self, sub):
        """(sqrt(lambda) [n_term], fx [n_term x nx], fy [n_term x ny]) that the
        basis kernel evaluates for Darcy subdomain ``sub``."""
        self._check(self.lib.sfb_kl_tables(self.h, sub, None, None, None))   # validates sub
        kl = self.w["kl"]
        nt = kl["n_term"][(kl.get("region_of") or list(range(self.n_darcy)))[sub]]
        nx, ny = self.w["darcy_grid"][sub]
        sl, fx, fy = np.zeros(nt), np.zeros((nt, nx)), np.zeros((nt, ny))
        self._check(self.lib.sfb_kl_tables(self.h, sub, sl.ctypes.data, fx.ctypes.data, fy.ctypes.data))
        return sl, fx, fy

    def local_points(self, sub):
        """Local realizations [n_local x n_term] of Darcy subdomain ``sub``'s KL region."""
        kl = self.w["kl"]
        region = (kl.get("region_of") or list(range(self.n_darcy)))[sub]
        n = ctypes.c_int32()
        self._check(self.lib.sfb_local_points(self.h, sub, ctypes.byref(n), None))
        y = np.zeros((n.value, kl["n_term"][region]))
        self._check(self.lib.sfb_local_points(self.h, sub, ctypes.byref(n), y.ctypes.data))
        return y

    # ---- workspace and the hot path ------------------------------------------------------
    def workspace_bytes(self, prec, max_pts):
        b = ctypes.c_size_t()
        self._check(self.lib.sfb_workspace_size(self.h, prec, max_pts, ctypes.byref(b)))
        return b.value

    def allocate(self, prec=FP64, max_pts=None, device="cuda"):
        """Size and hand over the device workspace (a torch uint8 tensor)."""
        import torch

        max_pts = self.n_pts if max_pts is None else max_pts
        nbytes = self.workspace_bytes(prec, max_pts)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        self._check(self.lib.sfb_set_workspace(self.h, ctypes.c_void_p(aligned), nbytes))
        self.max_pts = max_pts
        return nbytes

    def build_basis(self, prec=FP64, check=True):
        st = BasisStats()
        rc = self.lib.sfb_build_stochastic_basis(self.h, prec, ctypes.byref(st))
        self.basis_prec = prec
        if check and rc != SFB_OK:
            self._check(rc)
        out = {k: getattr(st, k) for k, _ in BasisStats._fields_}
        out["phase_cycles"] = list(st.phase_cycles)
        out["launch_shape"] = list(st.launch_shape)
        out["tune_ms"] = [list(r) for r in st.tune_ms]
        out["status"] = rc
        return out

    def get_basis(self, sub, k, with_x=False):
        if sub < 0:
            R = len(self.subdomain_dofs(-1))
            phi, g = np.zeros((R, R)), np.zeros(R)
            self._check(self.lib.sfb_get_basis(self.h, -1, 0, phi.ctypes.data, g.ctypes.data, None))
            return phi, g, None
        R = len(self.subdomain_dofs(sub))
        nx, ny = self.w["darcy_grid"][sub]
        # after the factor-only build (Method S1) there is no phi, and x holds
        # the particular solution (its last column) only
        phi = None if getattr(self, "basis_prec", None) == FACTOR_FP64 else np.zeros((R, R))
        g = np.zeros(R)
        x = np.zeros((R + 1, nx * ny)) if with_x else None
        self._check(self.lib.sfb_get_basis(self.h, sub, k, phi.ctypes.data if phi is not None else None,
                                           g.ctypes.data, x.ctypes.data if with_x else None))
        return phi, g, (x.T.copy() if with_x else None)

    def build_item_noalloc(self, sub, k, prec, phi_out, g_out, x_out, check=True):
        """One basis item through the allocation-free entry point; the caller
        supplies the outputs (x_out a device tensor of (R+1) x n_cells).
        Raises ValueError, before any call into the library, for outputs of
        the wrong type, layout or size."""
        R = len(self.subdomain_dofs(sub))
        nx, ny = self.w["darcy_grid"][sub]

        def _check_out(a, n, name, device):
            if a is None:
                return
            if isinstance(a, np.ndarray):
                ok = a.dtype == np.float64 and a.flags["C_CONTIGUOUS"] and a.size == n and not device
            else:
                import torch
                ok = (a.dtype == torch.float64 and a.is_contiguous() and a.numel() == n
                      and (a.is_cuda or not device))
            if not ok:
                raise ValueError("%s must be a contiguous float64 %sarray of %d elements"
                                 % (name, "device " if device else "", n))

        if x_out is None or phi_out is None:
            raise ValueError("phi_out and x_out are required")
        _check_out(phi_out, R * R, "phi_out", False)
        _check_out(g_out, R, "g_out", False)
        _check_out(x_out, (R + 1) * nx * ny, "x_out", True)
        rc =self.lib.sfb_build_basis_item_noalloc(self.h, sub, k, prec, ctypes.c_void_p(_ptr(phi_out)),
                                                   ctypes.c_void_p(_ptr(g_out)), ctypes.c_void_p(_ptr(x_out)))
        if check:
            self._check(rc)
        return rc

    def solve(self, y, w, rtol=1e-10, max_it=1000, lam_out=None, iters_out=None, check=True, krylov=CG):
        """Interface CG for a batch of points (host numpy or device torch
        arrays); outputs go to the given buffers (host or device). ``krylov``
        is CG (FP64), CG_MIXED (FP32 products, FP64 residuals), GMRES (restarted
        GMRES(m) in FP64), GMRES_MIXED (FP32 Arnoldi products, FP64 restarts)
        or CG_DTN (Method S1: the Darcy products by a subdomain solve per
        iteration, after an FP64 or FACTOR_FP64 build)."""
        y = np.ascontiguousarray(y, dtype=np.float64) if isinstance(y, np.ndarray) else y
        w = np.ascontiguousarray(w, dtype=np.float64) if isinstance(w, np.ndarray) else w
        n = int(y.shape[0])
        rc = self.lib.sfb_interface_solve_batch(self.h, ctypes.c_void_p(_ptr(y)), ctypes.c_void_p(_ptr(w)), n, krylov,
                                                rtol, max_it, ctypes.c_void_p(_ptr(lam_out)),
                                                ctypes.c_void_p(_ptr(iters_out)))
        if check and rc not in (SFB_OK,):
            self._check(rc)
        return rc

    def solve_host(self, y, w, rtol=1e-10, max_it=1000, check=True, krylov=CG):
        lam = np.zeros((len(y), self.n_lambda))
        it = np.zeros(len(y), dtype=np.int32)
        rc = self.solve(y, w, rtol, max_it, lam, it, check=check, krylov=krylov)
        return lam, it, rc

    def moments(self, field):
        n = self.field_size(field)
        mean, var = np.zeros(n), np.zeros(n)
        self._check(self.lib.sfb_moments(self.h, FIELDS[field], mean.ctypes.data, var.ctypes.data))
        return mean, var

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.lib.sfb_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def solve_timings(self):
        ms = np.zeros(5)
        it = ctypes.c_int32()
        self._check(self.lib.sfb_solve_timings(self.h, ms.ctypes.data, ctypes.byref(it)))
        return {"index_ms": ms[0], "cg_ms": ms[1], "status_ms": ms[2], "darcy_moments_ms": ms[3],
                "stokes_moments_ms": ms[4], "cg_iterations": it.value}

    def cg_phase_cycles(self):
        """SM cycles per CTA of the last one-launch CG by step (tile products,
        barrier, updates, barrier, FP64 check products, rest of the checks)."""
        cyc = np.zeros(6)
        self._check(self.lib.sfb_cg_phase_cycles(self.h, cyc.ctypes.data))
        return dict(zip(("tiles", "tiles_barrier", "update", "update_barrier", "check_tiles", "check_rest"), cyc))

    def set_option(self, name, value):
        self._check(self.lib.sfb_set_option(self.h, name.encode(), float(value)))

    def moments_reset(self):
        self._check(self.lib.sfb_moments_reset(self.h))
