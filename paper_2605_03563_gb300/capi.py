"""ctypes binding of libpoisson.so (include/poisson.h): argument marshalling only.

Every computation runs in the CUDA library.  Loading fails loudly when the
library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpoisson.so")

PS_OK, PS_ERR_INVALID_ARG, PS_ERR_UNSUPPORTED, PS_ERR_OOM, PS_ERR_CUDA = 0, 1, 2, 3, 4
PS_NOT_CONVERGED, PS_DIVERGED, PS_ERR_TIMEOUT = 5, 6, 7
STATUS_NAMES = {0: "PS_OK", 1: "PS_ERR_INVALID_ARG", 2: "PS_ERR_UNSUPPORTED", 3: "PS_ERR_OOM",
                4: "PS_ERR_CUDA", 5: "PS_NOT_CONVERGED", 6: "PS_DIVERGED", 7: "PS_ERR_TIMEOUT"}
PS_GRID_CART_UNIFORM, PS_GRID_SPHERICAL = 0, 1
PS_BC_DIRICHLET_GIVEN, PS_BC_MULTIPOLE = 0, 1
PS_INNER_NONE, PS_INNER_NEUMANN, PS_INNER_MULTIPOLE = 0, 1, 2
PS_SOR, PS_CG, PS_MG, PS_BICGSTAB, PS_PCG = 0, 1, 2, 3, 4
PS_FP64, PS_MIXED_FP32, PS_MIXED_BF16 = 0, 1, 2
DT_F64, DT_F32, DT_BF16 = 0, 1, 2


class PsGrid(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3)]


class PsBC(C.Structure):
    _fields_ = [("outer", C.c_int32), ("inner", C.c_int32), ("origin", C.c_double * 3),
                ("G", C.c_double)]


class PsSolveOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("prec", C.c_int32), ("omega", C.c_double),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("max_iter", C.c_int32),
                ("inner_cycles", C.c_int32), ("stream", C.c_void_p), ("tile_min_n", C.c_int32),
                ("sor_schedule", C.c_int32), ("compact_order", C.c_int32), ("use_tuning", C.c_int32)]


class PsInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("rel_residual", C.c_double),
                ("rho_conv", C.c_double), ("t_mp_ms", C.c_double), ("t_iter_ms", C.c_double),
                ("inner_cycles", C.c_int64), ("coarse_iterations", C.c_int64),
                ("kernel_launches", C.c_int64), ("moments", C.c_double * 81)]


class PsKernelStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes_per_launch", C.c_double), ("ops_per_launch", C.c_double),
                ("fp64", C.c_int32), ("variant", C.c_int32)]


class PsTuning(C.Structure):
    _fields_ = [("nu1", C.c_int32), ("nu2", C.c_int32), ("inner_cycles", C.c_int32),
                ("tile_min_n", C.c_int32), ("sweep_tile", C.c_int32), ("restrict_tile", C.c_int32)]


# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "poisson_create": (C.c_int, [C.POINTER(PsGrid), C.POINTER(C.c_void_p), C.c_int,
                                 C.POINTER(PsBC), C.c_int, C.POINTER(C.c_void_p)]),
    "poisson_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                C.POINTER(PsSolveOpts), C.POINTER(PsInfo)]),
    "poisson_solve_batch": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                      C.POINTER(C.c_void_p), C.POINTER(C.c_double), C.c_int,
                                      C.POINTER(PsSolveOpts), C.POINTER(PsInfo)]),
    "poisson_solve_begin": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                      C.POINTER(PsSolveOpts)]),
    "poisson_solve_step": (C.c_int, [C.c_void_p, C.c_int]),
    "poisson_solve_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(PsInfo)]),
    "poisson_solve_end": (C.c_int, [C.c_void_p, C.POINTER(PsInfo)]),
    "poisson_destroy": (None, [C.c_void_p]),
    "poisson_last_error": (C.c_char_p, []),
    "poisson_workspace_bytes": (C.c_size_t, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_int]),
    "poisson_compact_operators": (C.c_int, [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "poisson_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(PsTuning)]),
    "poisson_get_tuning": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(PsTuning), C.POINTER(C.c_int)]),
    "poisson_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "poisson_profile_read": (C.c_int, [C.c_void_p, C.POINTER(PsKernelStat), C.c_int]),
    "ps_op_apply": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_op_residual": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "ps_op_residual_noalloc": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "ps_op_sweep": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                              C.c_double, C.c_void_p]),
    "ps_op_restrict": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_op_restrict_red": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_op_prolong": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_op_multipole_moments": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.c_void_p,
                                          C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_double),
                                          C.c_void_p]),
    "ps_op_multipole_boundary": (C.c_int, [C.POINTER(PsGrid), C.c_int, C.POINTER(C.c_double),
                                           C.POINTER(C.c_double), C.c_int, C.c_double,
                                           C.c_void_p, C.c_void_p]),
    "ps_op_spherical_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ps_op_scale_to_fp32": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "ps_op_add_scaled_fp32": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]),
    "ps_probe_fp64": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double),
                                C.c_void_p]),
    "ps_probe_bounded_wait": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "poisson_batch_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.POINTER(C.c_void_p)]),
    "poisson_batch_destroy": (None, [C.c_void_p]),
    "poisson_batch_add": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                    C.c_int, C.POINTER(C.c_int)]),
    "poisson_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "poisson_batch_poll": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "poisson_batch_remove": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(PsInfo)]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"CUDA library {LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PoissonError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().poisson_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str, allow=(PS_OK,)):
    if status not in allow:
        raise PoissonError(status, where)
    return status


def make_grid(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), kind=PS_GRID_CART_UNIFORM) -> PsGrid:
    nn = (n, n, n) if isinstance(n, int) else tuple(n)
    return PsGrid(kind, (C.c_int32 * 3)(*nn), (C.c_double * 3)(*lo), (C.c_double * 3)(*hi))
