"""ctypes binding of librhmc.so (include/rhmc.h).  Argument marshalling only.

There is no fallback: if the shared library is missing or CUDA is not
available, loading raises.  Build it with ``paper_1808_01829_gb300._build.build()``
(``__graft_entry__.build()`` does so).
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librhmc.so")

RHMC_FP64 = 0
RHMC_MIXED_FP32 = 1
RHMC_DF64 = 2
RHMC_MAX_NRHS = 16
RHMC_MAX_SHIFTS = 64
# launch-setting keys (rhmc_tune_set / rhmc_ctx_tune_set) used from Python
RHMC_TUNE_UPDATE_TENSOR = 6
RHMC_TUNE_AXPY_SCALAR = 12
RHMC_TUNE_NO_DEFECT_CORRECTION = 13
RHMC_TUNE_BASIS_ITERS = 14
RHMC_TUNE_BASIS_GEMM = 15
RHMC_TUNE_BASIS_CHUNK = 16
RHMC_TUNE_NXN_FP64 = 18

STATUS = {
    0: "OK",
    1: "INVALID_ARG",
    2: "NOT_CONVERGED",
    3: "BREAKDOWN",
    4: "CUDA_ERROR",
    5: "DEVICE_TIMEOUT",
    6: "NO_GAUGE",
}


PROF_CATEGORIES = ["hop_fp32", "hop_fp64", "gram_fp32", "gram_fp64", "block_axpy", "update_fp32", "update_fp64",
                   "nxn", "force", "other", "hop_df", "nxn_shifts", "update_tc", "update_shifts_fp32",
                   "basis_tc"]


class RhmcError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Lattice(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int * 4), ("mass", ctypes.c_double), ("bc_t", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("dirac_calls", ctypes.c_int),
        ("reliable_updates", ctypes.c_int),
        ("refinements", ctypes.c_int),
        ("refine_iters", ctypes.c_int),
        ("true_rel_resid_max", ctypes.c_double),
        ("phase1_rel_resid_max", ctypes.c_double),
        ("per_shift_resid", ctypes.POINTER(ctypes.c_double)),
        ("phase1_ms", ctypes.c_double),
        ("refine_ms", ctypes.c_double),
    ]


class BatchItem(ctypes.Structure):
    _fields_ = [
        ("ctx", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("n_rhs", ctypes.c_int),
        ("n_shifts", ctypes.c_int),
        ("shifts", ctypes.POINTER(ctypes.c_double)),
        ("X", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("info", ctypes.POINTER(Info)),
        ("status", ctypes.c_int),
    ]


class Rational(ctypes.Structure):
    _fields_ = [("n_shifts", ctypes.c_int), ("alpha0", ctypes.c_double), ("alpha", ctypes.POINTER(ctypes.c_double)),
                ("beta", ctypes.POINTER(ctypes.c_double))]


class MdParams(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("tau", ctypes.c_double), ("n_steps", ctypes.c_int),
                ("n_gauge", ctypes.c_int), ("lam", ctypes.c_double), ("tol_md", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("precision_md", ctypes.c_int)]


class MdInfo(ctypes.Structure):
    _fields_ = [("force_evals", ctypes.c_int), ("gauge_force_evals", ctypes.c_int),
                ("solver_iters", ctypes.c_longlong), ("dirac_calls", ctypes.c_longlong),
                ("max_rel_resid", ctypes.c_double)]


class HmcInfo(ctypes.Structure):
    _fields_ = [("H_old", ctypes.c_double), ("H_new", ctypes.c_double), ("dH", ctypes.c_double),
                ("K", ctypes.c_double * 2), ("S_g", ctypes.c_double * 2), ("S_f", ctypes.c_double * 2),
                ("accepted", ctypes.c_int), ("md", MdInfo)]


_lock = threading.Lock()
_lib = None


def load():
    """Load librhmc.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} not built; run paper_1808_01829_gb300._build.build()")
        lib = ctypes.CDLL(LIB_PATH)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        PD = ctypes.POINTER(ctypes.c_double)
        lib.rhmc_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Lattice), I]
        lib.rhmc_destroy.argtypes = [P]
        lib.rhmc_set_gauge.argtypes = [P, P, P]
        lib.rhmc_workspace_bytes.argtypes = [P, I, I, I]
        lib.rhmc_workspace_bytes.restype = S
        lib.rhmc_apply_mdagm_mrhs.argtypes = [P, P, P, I, D, I, P]
        lib.rhmc_hop.argtypes = [P, P, P, I, I, I, P]
        lib.rhmc_apply_mdagm_mrhs_noalloc.argtypes = [P, P, P, I, D, P]
        lib.rhmc_apply_mdagm_mrhs_noalloc.restype = I
        lib.rhmc_block_multishift_cg.argtypes = [P, P, I, I, PD, P, D, I, I, P, ctypes.POINTER(Info), P]
        lib.rhmc_rational_solve.argtypes = [P, P, I, D, PD, PD, I, D, I, P, P, ctypes.POINTER(Info), P]
        lib.rhmc_rational_solve.restype = I
        lib.rhmc_rational_solve_bytes.argtypes = [P, I, I]
        lib.rhmc_rational_solve_bytes.restype = ctypes.c_size_t
        lib.rhmc_selftest_bounded_wait.argtypes = [I, D, P]
        lib.rhmc_selftest_bounded_wait.restype = I
        lib.rhmc_selftest_fp64_helpers.argtypes = [P, I, P, P]
        lib.rhmc_selftest_fp64_helpers.restype = I
        lib.rhmc_selftest_df_helpers.argtypes = [P, P, I, P, P]
        lib.rhmc_selftest_df_helpers.restype = I
        lib.rhmc_probe_alu_peaks.argtypes = [I, PD, PD, PD, P]
        lib.rhmc_probe_alu_peaks.restype = I
        lib.rhmc_ctx_tune_set.argtypes = [P, I, I]
        lib.rhmc_ctx_tune_set.restype = I
        lib.rhmc_ctx_tune_get.argtypes = [P, I]
        lib.rhmc_ctx_tune_get.restype = I
        lib.rhmc_block_multishift_cg_batch.argtypes = [ctypes.POINTER(BatchItem), I, D, I, I, P]
        lib.rhmc_block_multishift_cg_batch.restype = I
        lib.rhmc_multishift_cg_pervector.argtypes = [P, P, I, I, PD, P, D, I, P, ctypes.POINTER(Info), P]
        lib.rhmc_force.argtypes = [P, P, I, D, PD, PD, I, D, I, I, P, P, PD, P, ctypes.POINTER(Info), P]
        lib.rhmc_rational_apply.argtypes = [P, P, I, D, PD, I, P, P, P]
        lib.rhmc_force_lie.argtypes = [P, P, P, P, PD, P]
        lib.rhmc_force_lie.restype = I
        lib.rhmc_rational_apply.restype = I
        lib.rhmc_last_error.restype = ctypes.c_char_p
        lib.rhmc_kernel_launches.restype = ctypes.c_longlong
        lib.rhmc_tune_set.argtypes = [I, I]
        lib.rhmc_tune_set.restype = I
        lib.rhmc_tune_get.argtypes = [I]
        lib.rhmc_tune_get.restype = I
        lib.rhmc_profile_enable.argtypes = [I]
        lib.rhmc_profile_enable.restype = I
        lib.rhmc_profile_read.argtypes = [I, ctypes.POINTER(ctypes.c_longlong), PD, PD]
        lib.rhmc_profile_read.restype = I
        lib.rhmc_profile_read_flops.argtypes = [I, PD]
        lib.rhmc_profile_read_flops.restype = I
        lib.rhmc_gauge_action.argtypes = [P, P, D, PD, P]
        lib.rhmc_kinetic_energy.argtypes = [P, P, PD, P]
        lib.rhmc_momenta_from_normals.argtypes = [P, P, P, P]
        lib.rhmc_gauge_momentum.argtypes = [P, P, P, D, D, P]
        lib.rhmc_momentum_update.argtypes = [P, P, P, P, D, P]
        lib.rhmc_link_update.argtypes = [P, P, P, D, P]
        lib.rhmc_md_evolve.argtypes = [P, P, P, P, I, ctypes.POINTER(Rational), ctypes.POINTER(MdParams),
                                       ctypes.POINTER(MdInfo), P]
        lib.rhmc_hmc_trajectory.argtypes = [P, P, P, P, I, ctypes.POINTER(Rational), ctypes.POINTER(Rational),
                                            ctypes.POINTER(Rational), ctypes.POINTER(MdParams), D, D, P,
                                            ctypes.POINTER(HmcInfo), P]
        for name in ("rhmc_gauge_action", "rhmc_kinetic_energy", "rhmc_momenta_from_normals", "rhmc_gauge_momentum",
                     "rhmc_momentum_update", "rhmc_link_update", "rhmc_md_evolve", "rhmc_hmc_trajectory"):
            getattr(lib, name).restype = I
        for name in ("rhmc_create", "rhmc_destroy", "rhmc_set_gauge", "rhmc_apply_mdagm_mrhs", "rhmc_hop",
                     "rhmc_block_multishift_cg", "rhmc_multishift_cg_pervector", "rhmc_force"):
            getattr(lib, name).restype = I
        _lib = lib
        return lib


def check(rc: int, where: str, allow=()):
    if rc != 0 and rc not in allow:
        msg = load().rhmc_last_error().decode(errors="replace")
        raise RhmcError(rc, where, msg)
    return rc


def exported_symbols():
    """Names declared in include/rhmc.h that the library must export."""
    return [
        "rhmc_create", "rhmc_destroy", "rhmc_set_gauge", "rhmc_workspace_bytes", "rhmc_apply_mdagm_mrhs",
        "rhmc_hop", "rhmc_block_multishift_cg", "rhmc_multishift_cg_pervector", "rhmc_force", "rhmc_last_error", "rhmc_kernel_launches",
        "rhmc_profile_enable", "rhmc_profile_read", "rhmc_tune_set", "rhmc_tune_get",
        "rhmc_apply_mdagm_mrhs_noalloc", "rhmc_rational_apply", "rhmc_block_multishift_cg_batch", "rhmc_ctx_tune_set", "rhmc_ctx_tune_get",
        "rhmc_rational_solve", "rhmc_rational_solve_bytes", "rhmc_selftest_bounded_wait", "rhmc_force_lie",
        "rhmc_probe_alu_peaks", "rhmc_profile_read_flops", "rhmc_selftest_fp64_helpers", "rhmc_selftest_df_helpers",
        "rhmc_gauge_action", "rhmc_kinetic_energy", "rhmc_momenta_from_normals", "rhmc_gauge_momentum",
        "rhmc_momentum_update", "rhmc_link_update", "rhmc_md_evolve", "rhmc_hmc_trajectory",
    ]
