"""ctypes declarations of the LGDM C ABI (include/lgdm.h).

Argument marshalling only.  Loading fails loudly when the compiled library is
absent: there is no CPU fallback for any call.
"""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblgdm.so")

L2, Q4, H8, L3, Q9 = 1, 2, 3, 4, 5
NEN = {L2: 2, Q4: 4, H8: 8, L3: 3, Q9: 9}
PREC_FP64, PREC_FP32_TANGENT = 0, 1
PRECOND_JACOBI, PRECOND_NODE_BLOCK, PRECOND_MULTIGRID = 0, 1, 2
FIELD_U, FIELD_KAPPA_HIST, FIELD_DAMAGE, FIELD_DELTA, FIELD_RESIDUAL, FIELD_RHS = range(6)
NPHASES = 6
PHASES = ("element", "gather", "precond", "krylov", "commit", "begin_step")
COUNTERS = ("kernel_launches", "assemblies", "krylov_iters", "newton_iters", "load_steps", "halvings",
            "secant_iters")
STATUS = {0: "ok", 1: "invalid argument", 2: "workspace too small", 3: "CUDA error",
          4: "Newton did not converge", 5: "non-finite value", 6: "device wait timed out",
          7: "call out of order"}

ABI_VERSION = 2
FAULT_NONE, FAULT_BARRIER_TIMEOUT, FAULT_NAN_STATE = 0, 1, 2

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


class Mesh(C.Structure):
    _fields_ = [("elem", C.c_int32), ("nnode", C.c_int32), ("nelem", C.c_int32),
                ("x", _dp), ("y", _dp), ("z", _dp), ("conn", _ip),
                ("e_scale", _dp), ("vol_scale", _dp)]


class Material(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("E", "nu", "k", "kappa0", "alpha", "beta", "R", "eta", "c", "h")] + \
               [("evm_variant", C.c_int32), ("h_stress", C.c_int32)]


class BCs(C.Structure):
    _fields_ = [("n_dir", C.c_int32), ("dir_dof", _ip), ("dir_scale", _dp)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("precond", C.c_int32), ("newton_tol", C.c_double),
                ("krylov_rtol", C.c_double), ("max_newton", C.c_int32), ("max_krylov", C.c_int32),
                ("max_halvings", C.c_int32), ("krylov_blocks", C.c_int32), ("gmres_m", C.c_int32),
                ("krylov_method", C.c_int32), ("wait_limit_s", C.c_double)]


class Sizes(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nen", C.c_int32), ("ngp", C.c_int32), ("nd", C.c_int32),
                ("nnode", C.c_int32), ("nelem", C.c_int32), ("ndof", C.c_int64), ("nnz", C.c_int64),
                ("npairs", C.c_int64), ("workspace_bytes", C.c_size_t), ("mg_levels", C.c_int32),
                ("mg_nnode", C.c_int32 * 10), ("mg_npairs", C.c_int64 * 10)]


class LgdmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_SIGS = {
    "lgdm_abi_version": (C.c_int32, []),
    "lgdm_status_string": (C.c_char_p, [C.c_int]),
    "lgdm_default_options": (C.c_int, [C.POINTER(Options)]),
    "lgdm_workspace_size": (C.c_int, [C.POINTER(Mesh), C.POINTER(Options), C.POINTER(C.c_size_t)]),
    "lgdm_create": (C.c_int, [C.POINTER(Mesh), C.POINTER(Material), C.POINTER(BCs), C.POINTER(Options),
                              C.c_void_p, C.c_size_t, C.c_void_p, C.POINTER(C.c_void_p)]),
    "lgdm_destroy": (None, [C.c_void_p]),
    "lgdm_last_error": (C.c_char_p, [C.c_void_p]),
    "lgdm_get_sizes": (C.c_int, [C.c_void_p, C.POINTER(Sizes)]),
    "lgdm_set_state": (C.c_int, [C.c_void_p, _dp, _dp]),
    "lgdm_reset_state": (C.c_int, [C.c_void_p]),
    "lgdm_get_field": (C.c_int, [C.c_void_p, C.c_int32, _dp, C.c_size_t]),
    "lgdm_begin_step": (C.c_int, [C.c_void_p, C.c_double]),
    "lgdm_assemble": (C.c_int, [C.c_void_p]),
    "lgdm_get_system": (C.c_int, [C.c_void_p, _ip, _ip, _dp, _dp]),
    "lgdm_solve": (C.c_int, [C.c_void_p, _ip, _dp]),
    "lgdm_update": (C.c_int, [C.c_void_p, _ip]),
    "lgdm_newton_step": (C.c_int, [C.c_void_p, _ip, _ip]),
    "lgdm_run_step": (C.c_int, [C.c_void_p, C.c_double, _ip]),
    "lgdm_commit": (C.c_int, [C.c_void_p]),
    "lgdm_last_solve": (C.c_int, [C.c_void_p, _ip, _ip, _dp, _dp]),
    "lgdm_get_reaction": (C.c_int, [C.c_void_p, _dp]),
    "lgdm_get_energy": (C.c_int, [C.c_void_p, _dp]),
    "lgdm_get_committed": (C.c_int, [C.c_void_p, _dp, _dp, _dp]),
    "lgdm_set_committed": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double]),
    "lgdm_get_dissipated_energy": (C.c_int, [C.c_void_p, _dp, _dp]),
    "lgdm_get_damaged_volume": (C.c_int, [C.c_void_p, C.c_double, _dp]),
    "lgdm_inject_fault": (C.c_int, [C.c_void_p, C.c_int32]),
    "lgdm_pattern_counts": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "lgdm_enable_timers": (C.c_int, [C.c_void_p, C.c_int32]),
    "lgdm_get_timers": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64)]),
    "lgdm_reset_timers": (C.c_int, [C.c_void_p]),
    "lgdm_get_counters": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_int32]),
    "lgdm_batch_workspace_size": (C.c_int, [C.c_int32, C.POINTER(C.c_size_t)]),
    "lgdm_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "lgdm_batch_destroy": (None, [C.c_void_p]),
    "lgdm_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "lgdm_batch_set_tuning": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "lgdm_batch_get_tuning": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "lgdm_batch_set_solve_tuning": (C.c_int, [C.c_void_p, C.c_int32]),
    "lgdm_batch_get_solve_tuning": (C.c_int, [C.c_void_p, _ip, _ip]),
    "lgdm_batch_get_launches": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "lgdm_batch_autotune": (C.c_int, [C.c_void_p, _ip, _ip, _dp]),
    "lgdm_batch_assemble": (C.c_int, [C.c_void_p, _ip]),
    "lgdm_batch_enable_timers": (C.c_int, [C.c_void_p, C.c_int32]),
    "lgdm_batch_get_timers": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), C.c_int32]),
    "lgdm_batch_newton_step": (C.c_int, [C.c_void_p, _ip, _ip, _ip]),
    "lgdm_batch_run_step": (C.c_int, [C.c_void_p, _dp, _ip, _ip]),
    "lgdm_solve_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_double, C.c_int32, C.c_void_p, _ip, _dp]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load liblgdm.so and declare every ABI function (raises if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"LGDM CUDA library not built ({path} missing); run "
                           "paper_2301_06503_gb300.build.build() or __graft_entry__.build()")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.lgdm_abi_version() != ABI_VERSION:
        raise RuntimeError("LGDM ABI version mismatch")
    _lib = lib
    return lib


def abi_names():
    return list(_SIGS)


def check(status: int, handle=None) -> None:
    if status != 0:
        msg = load().lgdm_last_error(handle)
        raise LgdmError(status, msg.decode() if msg else "")
