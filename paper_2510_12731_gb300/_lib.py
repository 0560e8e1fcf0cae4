"""ctypes binding of the px C ABI (include/px.h): argument marshalling only.

Every computation happens in libpx.so on the GPU.  If the library has not been
built, importing this module raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpx.so")

PX_OK, PX_EINVAL, PX_ENOMEM, PX_ENOTCONV, PX_ETIMEOUT, PX_ECUDA, PX_EBUSY, PX_ENOTIMPL, PX_ENOTFOUND = range(9)
STATUS_NAMES = ["PX_OK", "PX_EINVAL", "PX_ENOMEM", "PX_ENOTCONV", "PX_ETIMEOUT", "PX_ECUDA",
                "PX_EBUSY", "PX_ENOTIMPL", "PX_ENOTFOUND"]
PX_WFQ, PX_WFQFMU, PX_WFQFMU_HETERO = 0, 1, 2
PX_FP64, PX_FP32, PX_BF16SPLIT, PX_FP16SPLIT = 0, 1, 2, 3
PX_MODE_AUTO, PX_MODE_MATFREE, PX_MODE_MATERIALISED = 0, 1, 2
PX_BASIS_AUTO, PX_BASIS_FP64, PX_BASIS_FF32, PX_BASIS_FP32 = 0, 1, 2, 3

MODELS = {"wfq": PX_WFQ, "wfqfmu": PX_WFQFMU, "wfqfmu_hetero": PX_WFQFMU_HETERO}
PRECISIONS = {"fp64": PX_FP64, "fp32": PX_FP32, "bf16split": PX_BF16SPLIT,
              "fp16split": PX_FP16SPLIT}
MODES = {"auto": PX_MODE_AUTO, "matfree": PX_MODE_MATFREE, "materialised": PX_MODE_MATERIALISED}
BASES = {"auto": PX_BASIS_AUTO, "fp64": PX_BASIS_FP64, "ff32": PX_BASIS_FF32, "fp32": PX_BASIS_FP32}
PX_SOLVER_BATCHED, PX_SOLVER_SHIFTED = 0, 1
SOLVERS = {"batched": PX_SOLVER_BATCHED, "shifted": PX_SOLVER_SHIFTED}
PX_BEM_DPCM, PX_BEM_IEFPCM = 0, 1
BEM_FORMULATIONS = {"dpcm": PX_BEM_DPCM, "iefpcm": PX_BEM_IEFPCM}


class AtomType(C.Structure):
    _fields_ = [("r0_ang", C.c_double), ("d", C.c_double), ("s", C.c_double),
                ("area_bohr2", C.c_double), ("Rq_bohr", C.c_double), ("Rmu_bohr", C.c_double),
                ("drude_n_au", C.c_double), ("tau_au", C.c_double)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("mode", C.c_int), ("restart_m", C.c_int),
                ("max_iter", C.c_int), ("max_cycles", C.c_int), ("max_refine", C.c_int),
                ("gs_passes", C.c_int), ("basis", C.c_int), ("gemm_tiles", C.c_int),
                ("cycle_graphs", C.c_int), ("sort_atoms", C.c_int),
                ("tol_rel", C.c_double), ("inner_tol", C.c_double), ("kcut_eps", C.c_double),
                ("mu_self_term", C.c_int), ("profile", C.c_int),
                ("hbm_budget_bytes", C.c_size_t), ("device_wait_limit_s", C.c_double),
                ("solver", C.c_int), ("shift_krylov_max", C.c_int)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class Result(C.Structure):
    _fields_ = [("alpha", _dp), ("sigma_abs", _dp), ("sigma_abs_pol", _dp), ("q", _dp),
                ("mu", _dp), ("rel_residual", _dp), ("iters", _ip), ("status", _ip)]


class Stats(C.Structure):
    _fields_ = [("setup_ms", C.c_double), ("solve_ms", C.c_double), ("matvec_ms", C.c_double),
                ("matvec_launches", C.c_longlong), ("matvec_flops", C.c_double),
                ("matvec_bytes", C.c_double), ("resid_ms", C.c_double),
                ("resid_launches", C.c_longlong), ("resid_flops", C.c_double),
                ("kernel_launches", C.c_longlong), ("setup_launches", C.c_longlong),
                ("cycles", C.c_int),
                ("total_iters", C.c_longlong), ("n_unknowns", C.c_longlong),
                ("used_mode", C.c_int), ("used_precision", C.c_int),
                ("gemm_tiles_used", C.c_int), ("graph_launches", C.c_longlong),
                ("graphs_built", C.c_longlong), ("solver_used", C.c_int),
                ("shift_steps", C.c_longlong), ("shift_matvec_launches", C.c_longlong),
                ("shift_matvec_ms", C.c_double), ("shift_matvec_bytes", C.c_double),
                ("shift_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("model", C.c_int), ("n_atoms", C.c_int), ("xyz_ang", _dp), ("type_idx", _ip),
                ("types", C.POINTER(AtomType)), ("n_types", C.c_int), ("n_freq", C.c_int),
                ("omega_ev", _dp), ("alpha_ib", _dp), ("n_pol", C.c_int), ("pol_dir", _dp),
                ("e0", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong),
                ("failed", C.c_longlong), ("running", C.c_longlong), ("queued", C.c_longlong),
                ("p50_latency_ms", C.c_double), ("p99_latency_ms", C.c_double),
                ("max_latency_ms", C.c_double), ("busy_points", C.c_double),
                ("wall_s", C.c_double), ("structure_reuses", C.c_longlong),
                ("peak_reserved_bytes", C.c_size_t), ("merged_requests", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# every function declared in include/px.h and include/px_serve.h, with its ctypes signature
SIGNATURES = {
    "px_abi_version": (C.c_int, []),
    "px_options_default": (C.c_int, [C.POINTER(Options)]),
    "px_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Options)]),
    "px_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "px_set_structure": (C.c_int, [C.c_void_p, C.c_int, C.c_int, _dp, _ip, C.POINTER(AtomType), C.c_int]),
    "px_solve": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, C.c_int, _dp, C.c_double,
                           C.POINTER(Result), C.c_void_p]),
    "px_solve_device": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, C.c_int, _dp, C.c_double,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "px_relres_device_noalloc": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, C.c_int, _dp,
                                           C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.c_void_p]),
    "px_fields": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_int, C.c_void_p, C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "px_system_device": (C.c_int, [C.c_void_p, C.c_int, _dp, C.c_double, C.c_void_p, C.c_size_t,
                                   C.c_void_p, C.c_void_p]),
    "px_set_mesh": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, _dp, C.c_double, C.c_int]),
    "px_solve_bem": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp, C.c_int, _dp, C.c_double,
                               C.POINTER(Result), C.c_void_p]),
    "px_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "px_destroy": (C.c_int, [C.c_void_p]),
    "px_last_error": (C.c_char_p, [C.c_void_p]),
    "px_server_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Options), C.c_int, C.c_size_t]),
    "px_submit": (C.c_int, [C.c_void_p, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "px_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result), C.POINTER(C.c_int)]),
    "px_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result), C.c_double]),
    "px_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    "px_server_destroy": (C.c_int, [C.c_void_p]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(
            f"libpx.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


class PxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def dptr(a: np.ndarray):
    return a.ctypes.data_as(_dp) if a is not None else None


def iptr(a: np.ndarray):
    return a.ctypes.data_as(_ip) if a is not None else None
