"""GB300-native wFQ / wFQFmu plasmonic linear-response solver.

Python front-end of the px C library (include/px.h).  The classes here only
marshal arguments; every step of the solve runs in the library's CUDA kernels.

    from paper_2510_12731_gb300 import Solver, structures
    w = structures.ag_sphere_791()
    with Solver(precision="fp64") as s:
        s.set_structure(w.model, w.xyz_ang, w.type_idx, w.types)
        out = s.solve(w.omega_ev, w.pol_dirs, w.alpha_ib)
    out["alpha"]        # (F, 3, P) complex polarisability, bohr^3
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

__all__ = ["Solver", "Server", "PxError", "options"]

PxError = L.PxError


def options(**kw) -> L.Options:
    """A px_options record: library defaults, overridden by keyword arguments.

    Keywords: precision ("fp64" | "fp32" | "bf16split" | "fp16split"), mode ("auto" |
    "matfree" | "materialised"), basis ("auto" | "fp64" | "ff32" | "fp32"), solver
    ("batched" | "shifted"), restart_m, max_iter, max_cycles, max_refine, gs_passes,
    gemm_tiles, cycle_graphs, sort_atoms, tol_rel, inner_tol, kcut_eps, mu_self_term,
    profile, hbm_budget_bytes, device_wait_limit_s, shift_krylov_max.
    """
    o = L.Options()
    L.lib().px_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "precision":
            v = L.PRECISIONS[v] if isinstance(v, str) else int(v)
        elif k == "mode":
            v = L.MODES[v] if isinstance(v, str) else int(v)
        elif k == "basis":
            v = L.BASES[v] if isinstance(v, str) else int(v)
        elif k == "solver":
            v = L.SOLVERS[v] if isinstance(v, str) else int(v)
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Solver:
    """One px handle: a loaded structure and its device-resident operators."""

    def __init__(self, **opts):
        self._lib = L.lib()
        self._h = C.c_void_p()
        self._opt = options(**opts)
        st = self._lib.px_create(C.byref(self._h), C.byref(self._opt))
        if st != L.PX_OK:
            raise PxError(st, self._lib.px_last_error(None).decode())
        self.model = None
        self.natoms = 0

    # ------------------------------------------------------------------ lifecycle
    def close(self):
        if self._h:
            self._lib.px_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, allow=()):
        if st != L.PX_OK and st not in allow:
            raise PxError(st, self._lib.px_last_error(self._h).decode())
        return st

    # ------------------------------------------------------------------ calls
    def set_options(self, **opts):
        self._opt = options(**opts)
        self._check(self._lib.px_set_options(self._h, C.byref(self._opt)))

    def set_structure(self, model, xyz_ang, type_idx, types):
        xyz = np.ascontiguousarray(xyz_ang, dtype=np.float64).reshape(-1, 3)
        tidx = np.ascontiguousarray(type_idx, dtype=np.int32).reshape(-1)
        tarr = (L.AtomType * len(types))(*[
            L.AtomType(**{k: float(t[k]) for k in (f for f, _ in L.AtomType._fields_)})
            for t in types])
        m = L.MODELS[model] if isinstance(model, str) else int(model)
        self._check(self._lib.px_set_structure(self._h, m, xyz.shape[0], L.dptr(xyz), L.iptr(tidx),
                                               tarr, len(types)))
        self.model = m
        self.natoms = xyz.shape[0]

    def set_mesh(self, pos_ang, normals, area_ang2, radius_ang, formulation="dpcm"):
        """Boundary-element surface (Sec. 2.3): barycentres (n, 3) Angstrom, outward unit
        normals (n, 3), areas (n,) Angstrom^2, enclosing radius R (Angstrom);
        formulation "dpcm" (Eq. 11) or "iefpcm" (Eq. 12)."""
        pos = np.ascontiguousarray(pos_ang, dtype=np.float64).reshape(-1, 3)
        nrm = np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, 3)
        area = np.ascontiguousarray(area_ang2, dtype=np.float64).reshape(-1)
        if nrm.shape != pos.shape or area.size != pos.shape[0]:
            raise ValueError("pos_ang, normals and area_ang2 describe different meshes")
        form = L.BEM_FORMULATIONS[formulation] if isinstance(formulation, str) else int(formulation)
        self._check(self._lib.px_set_mesh(self._h, pos.shape[0], L.dptr(pos), L.dptr(nrm),
                                          L.dptr(area), float(radius_ang), form))
        self.model = L.PX_WFQ   # one scalar unknown per tessera, no dipoles
        self.natoms = pos.shape[0]

    def alloc_outputs(self, n_freq, n_pol, want_q=True, want_mu=True, empty=np.zeros):
        """Host result arrays for solve(); ``empty`` may allocate pinned memory."""
        F, P, N = int(n_freq), int(n_pol), self.natoms
        out = {"alpha": empty((F, 3, P), dtype=np.complex128),
               "sigma_abs": empty((F,), dtype=np.float64),
               "sigma_abs_pol": empty((F, P), dtype=np.float64),
               "q": empty((F, P, N), dtype=np.complex128) if want_q else None,
               "mu": (empty((F, P, N, 3), dtype=np.complex128)
                      if (want_mu and self.model != L.PX_WFQ) else None),
               "rel_residual": empty((F, P), dtype=np.float64),
               "iters": empty((F, P), dtype=np.int32),
               "status": empty((F, P), dtype=np.int32)}
        return out

    def solve(self, omega_ev, pol_dirs, alpha_ib=None, e0=1.0, want_q=True, want_mu=True,
              stream=None, out=None):
        """Solve every (frequency, polarisation) column; returns a dict of numpy arrays.

        alpha (F, 3, P) complex, sigma_abs (F,) [P == 3], sigma_abs_pol (F, P),
        q (F, P, N) complex, mu (F, P, N, 3) complex [wFQFmu], rel_residual (F, P),
        iters (F, P), status (F, P), ok (bool: every column met tol_rel).
        ``out`` may hold preallocated arrays (see alloc_outputs).
        """
        w = np.ascontiguousarray(omega_ev, dtype=np.float64).reshape(-1)
        pol = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        F, P = w.size, pol.shape[0]
        aib = None
        if alpha_ib is not None:
            aib = np.ascontiguousarray(np.asarray(alpha_ib, dtype=np.complex128)).view(np.float64)
        o = out if out is not None else self.alloc_outputs(F, P, want_q, want_mu)
        cptr = lambda a: a.view(np.float64).ctypes.data_as(L._dp) if a is not None else None
        res = L.Result(cptr(o["alpha"]), L.dptr(o["sigma_abs"]), L.dptr(o["sigma_abs_pol"]),
                       cptr(o["q"]), cptr(o["mu"]), L.dptr(o["rel_residual"]),
                       L.iptr(o["iters"]), L.iptr(o["status"]))
        st = self._lib.px_solve(self._h, F, L.dptr(w), L.dptr(aib) if aib is not None else None, P,
                                L.dptr(pol), float(e0), C.byref(res),
                                C.c_void_p(stream) if stream else None)
        self._check(st, allow=(L.PX_ENOTCONV,))
        result = dict(o)
        result["ok"] = st == L.PX_OK
        if P != 3:
            result.pop("sigma_abs", None)
        return result

    def solve_bem(self, omega_ev, eps2, eps1, pol_dirs, e0=1.0, want_q=True, stream=None,
                  out=None):
        """Solve the loaded mesh for the permittivities eps2 (particle) and eps1 (medium),
        (F,) complex each (eps1 may be a scalar).  Returns the dict of solve(); q holds the
        tesserae's charges A_i sigma_i."""
        w = np.ascontiguousarray(omega_ev, dtype=np.float64).reshape(-1)
        pol = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        F, P = w.size, pol.shape[0]
        e2 = np.broadcast_to(np.asarray(eps2, dtype=np.complex128), (F,))
        e1 = np.broadcast_to(np.asarray(eps1, dtype=np.complex128), (F,))
        eps = np.ascontiguousarray(np.stack([e2.real, e2.imag, e1.real, e1.imag], axis=1))
        o = out if out is not None else self.alloc_outputs(F, P, want_q, False)
        cptr = lambda a: a.view(np.float64).ctypes.data_as(L._dp) if a is not None else None
        res = L.Result(cptr(o["alpha"]), L.dptr(o["sigma_abs"]), L.dptr(o["sigma_abs_pol"]),
                       cptr(o["q"]), None, L.dptr(o["rel_residual"]),
                       L.iptr(o["iters"]), L.iptr(o["status"]))
        st = self._lib.px_solve_bem(self._h, F, L.dptr(w), L.dptr(eps), P, L.dptr(pol), float(e0),
                                    C.byref(res), C.c_void_p(stream) if stream else None)
        self._check(st, allow=(L.PX_ENOTCONV,))
        result = dict(o)
        result["ok"] = st == L.PX_OK
        result.pop("mu", None)
        if P != 3:
            result.pop("sigma_abs", None)
        return result

    def solve_device(self, omega_ev, pol_dirs, alpha_ib=None, e0=1.0, d_alpha=None, d_q=None,
                     d_mu=None, d_relres=None, stream=None):
        """Solve with results written to caller-owned device buffers (e.g. torch tensors).

        Each d_* argument is an object with ``data_ptr()`` (a CUDA tensor of the right
        size, float64 / complex128) or None.  Returns True when every column met tol_rel.
        """
        w = np.ascontiguousarray(omega_ev, dtype=np.float64).reshape(-1)
        pol = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        aib = None
        if alpha_ib is not None:
            aib = np.ascontiguousarray(np.asarray(alpha_ib, dtype=np.complex128)).view(np.float64)
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        st = self._lib.px_solve_device(self._h, w.size, L.dptr(w),
                                       L.dptr(aib) if aib is not None else None, pol.shape[0],
                                       L.dptr(pol), float(e0), ptr(d_alpha), ptr(d_q), ptr(d_mu),
                                       ptr(d_relres), C.c_void_p(stream) if stream else None)
        self._check(st, allow=(L.PX_ENOTCONV,))
        return st == L.PX_OK

    def relres_device_noalloc(self, omega_ev, pol_dirs, d_q, d_relres, alpha_ib=None, d_mu=None,
                              e0=1.0, stream=None):
        """FP64 relative residuals of a device-resident solution (d_q, d_mu) into d_relres,
        without any device allocation (see px_relres_device_noalloc in include/px.h)."""
        w = np.ascontiguousarray(omega_ev, dtype=np.float64).reshape(-1)
        pol = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        aib = None
        if alpha_ib is not None:
            aib = np.ascontiguousarray(np.asarray(alpha_ib, dtype=np.complex128)).view(np.float64)
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._lib.px_relres_device_noalloc(
            self._h, w.size, L.dptr(w), L.dptr(aib) if aib is not None else None, pol.shape[0],
            L.dptr(pol), float(e0), ptr(d_q), ptr(d_mu), ptr(d_relres),
            C.c_void_p(stream) if stream else None))

    def fields(self, points_ang, d_q, d_mu=None, d_rho=None, d_phi=None, d_E=None, stream=None):
        """Induced density / potential / field maps of device-resident solved columns at
        probe points (see px_fields in include/px.h).  d_q: (C, N) complex128 CUDA tensor
        (C = F P, as px_solve_device writes it); d_mu: (C, N, 3) or None; outputs: (C, M)
        complex128 for d_rho / d_phi, (C, M, 3) for d_E, each optional."""
        pts = np.ascontiguousarray(points_ang, dtype=np.float64).reshape(-1, 3)
        C_ = int(d_q.numel() // max(self.natoms, 1))
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._lib.px_fields(self._h, pts.shape[0], L.dptr(pts), C_, ptr(d_q), ptr(d_mu),
                                        ptr(d_rho), ptr(d_phi), ptr(d_E),
                                        C.c_void_p(stream) if stream else None))

    def system_device(self, pol_dirs=None, e0=1.0, d_A0=None, d_b=None, stream=None):
        """The frequency-independent dense operator A0 (n_u x n_u, float64 CUDA tensor,
        row-major) and right-hand sides b (n_u x P) of the loaded structure (see
        px_system_device in include/px.h)."""
        pol = None if pol_dirs is None else np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        ld = d_A0.stride(0) if d_A0 is not None else 0
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        self._check(self._lib.px_system_device(
            self._h, 0 if pol is None else pol.shape[0], L.dptr(pol) if pol is not None else None,
            float(e0), ptr(d_A0), ld, ptr(d_b), C.c_void_p(stream) if stream else None))

    def stats(self) -> dict:
        s = L.Stats()
        self._check(self._lib.px_get_stats(self._h, C.byref(s)))
        return s.as_dict()


def _types_array(types):
    return (L.AtomType * len(types))(*[
        L.AtomType(**{k: float(t[k]) for k in (f for f, _ in L.AtomType._fields_)}) for t in types])


class Server:
    """Continuous-batching request loop (include/px_serve.h): slots with their own
    streams, admission by device footprint, device-resident operators reused for
    repeated structures."""

    def __init__(self, max_slots=4, hbm_budget_bytes=0, **opts):
        self._lib = L.lib()
        self._s = C.c_void_p()
        self._opt = options(**opts)
        st = self._lib.px_server_create(C.byref(self._s), C.byref(self._opt), int(max_slots),
                                        int(hbm_budget_bytes))
        if st != L.PX_OK:
            raise PxError(st, "px_server_create failed")
        self._meta = {}
        self._keep = {}

    def close(self):
        if self._s:
            self._lib.px_server_destroy(self._s)
            self._s = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, model, xyz_ang, type_idx, types, omega_ev, pol_dirs, alpha_ib=None, e0=1.0):
        """Queue a request; returns its id.  Inputs are copied by the library."""
        xyz = np.ascontiguousarray(xyz_ang, dtype=np.float64).reshape(-1, 3)
        tidx = np.ascontiguousarray(type_idx, dtype=np.int32).reshape(-1)
        w = np.ascontiguousarray(omega_ev, dtype=np.float64).reshape(-1)
        pol = np.ascontiguousarray(pol_dirs, dtype=np.float64).reshape(-1, 3)
        tarr = _types_array(types)
        aib = None
        if alpha_ib is not None:
            aib = np.ascontiguousarray(np.asarray(alpha_ib, dtype=np.complex128)).view(np.float64)
        m = L.MODELS[model] if isinstance(model, str) else int(model)
        req = L.Request(m, xyz.shape[0], L.dptr(xyz), L.iptr(tidx), tarr, len(types), w.size,
                        L.dptr(w), L.dptr(aib) if aib is not None else None, pol.shape[0],
                        L.dptr(pol), float(e0))
        rid = C.c_uint64()
        st = self._lib.px_submit(self._s, C.byref(req), C.byref(rid))
        if st != L.PX_OK:
            raise PxError(st, "px_submit failed")
        self._meta[rid.value] = (m, xyz.shape[0], w.size, pol.shape[0])
        return rid.value

    def _result(self, rid):
        m, N, F, P = self._meta[rid]
        out = {"alpha": np.zeros((F, 3, P), np.complex128), "sigma_abs": np.zeros(F),
               "sigma_abs_pol": np.zeros((F, P)), "q": np.zeros((F, P, N), np.complex128),
               "mu": np.zeros((F, P, N, 3), np.complex128) if m != L.PX_WFQ else None,
               "rel_residual": np.zeros((F, P)), "iters": np.zeros((F, P), np.int32),
               "status": np.zeros((F, P), np.int32)}
        cptr = lambda a: a.view(np.float64).ctypes.data_as(L._dp) if a is not None else None
        res = L.Result(cptr(out["alpha"]), L.dptr(out["sigma_abs"]), L.dptr(out["sigma_abs_pol"]),
                       cptr(out["q"]), cptr(out["mu"]), L.dptr(out["rel_residual"]),
                       L.iptr(out["iters"]), L.iptr(out["status"]))
        return out, res

    def wait(self, rid, timeout_s=600.0):
        """Block until request rid finishes; returns its result dict (raises on failure)."""
        out, res = self._result(rid)
        st = self._lib.px_wait(self._s, C.c_uint64(rid), C.byref(res), float(timeout_s))
        if st not in (L.PX_OK, L.PX_ENOTCONV):
            raise PxError(st, f"request {rid} failed")
        del self._meta[rid]
        out["ok"] = st == L.PX_OK
        return out

    def poll(self, rid):
        """Result dict if request rid finished, else None."""
        out, res = self._result(rid)
        done = C.c_int(0)
        st = self._lib.px_poll(self._s, C.c_uint64(rid), C.byref(res), C.byref(done))
        if not done.value:
            if st != L.PX_OK:
                raise PxError(st, f"poll of request {rid} failed")
            return None
        if st not in (L.PX_OK, L.PX_ENOTCONV):
            raise PxError(st, f"request {rid} failed")
        del self._meta[rid]
        out["ok"] = st == L.PX_OK
        return out

    def stats(self) -> dict:
        s = L.ServerStats()
        self._lib.px_server_get_stats(self._s, C.byref(s))
        return s.as_dict()
