"""ctypes loader for libqm.so: the C ABI declared in include/qm.h.

There is no fallback: if the library is missing or cannot be loaded, importing the
binding raises, and every compute call needs CUDA device tensors.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqm.so")

c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)
c_int32_p = ctypes.POINTER(ctypes.c_int32)

# name -> (restype, argtypes); mirrors include/qm.h
SIGNATURES = {
    "qm_gspace_create": (ctypes.c_int, [c_double_p, ctypes.c_int, c_double_p, ctypes.c_double, c_int_p,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "qm_gspace_query": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p, c_int_p, c_int_p]),
    "qm_gspace_indices": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int32_p, c_int32_p, c_double_p]),
    "qm_gspace_sticks": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_int_p, c_int32_p, c_int_p, c_int32_p]),
    "qm_gspace_destroy": (None, [ctypes.c_void_p]),
    "qm_hpsi": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                               ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_void_p,
                               ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_int,
                               ctypes.c_int, ctypes.c_void_p]),
    "qm_launch_count": (ctypes.c_ulonglong, []),
    "qm_prof_enable": (ctypes.c_int, [ctypes.c_int]),
    "qm_prof_read": (ctypes.c_int, [ctypes.c_int, c_double_p, ctypes.POINTER(ctypes.c_longlong)]),
    "qm_prof_name": (ctypes.c_char_p, [ctypes.c_int]),
    "qm_last_error": (ctypes.c_char_p, []),
    "qm_version": (ctypes.c_char_p, []),
}

_lib = None


def load():
    """Load libqm.so once and attach the signatures; raises OSError if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is not built; run paper_2308_07277_gb300.build.build() (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DavidsonOpts(ctypes.Structure):
    """qm_davidson_opts of include/qm.h."""
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("nvecx", ctypes.c_int),
                ("prec", ctypes.c_int), ("precond", ctypes.c_int), ("mixed_switch", ctypes.c_double),
                ("nconv", ctypes.c_int), ("mixed_ortho", ctypes.c_int), ("history", c_double_p),
                ("mlp", ctypes.c_void_p), ("precond_stall", ctypes.c_double), ("plain_restart", ctypes.c_int),
                ("fp64_exact", ctypes.c_int)]


class DavidsonStats(ctypes.Structure):
    """qm_davidson_stats of include/qm.h."""
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("band_applies", ctypes.c_longlong),
                ("max_residual", ctypes.c_double), ("seconds", ctypes.c_double), ("iterations_mixed", ctypes.c_int),
                ("band_applies_mixed", ctypes.c_longlong), ("precond_fallback", ctypes.c_int),
                ("restarts", ctypes.c_int), ("restart_kept", ctypes.c_longlong)]


SIGNATURES["qm_davidson"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.POINTER(DavidsonOpts), c_double_p,
                                            ctypes.POINTER(DavidsonStats), ctypes.c_void_p])

SIGNATURES["qm_hpsi_noalloc"] = SIGNATURES["qm_hpsi"]
SIGNATURES["qm_hpsi_gamma"] = SIGNATURES["qm_hpsi"]
SIGNATURES["qm_hpsi_check"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_hpsi_prepare"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                ctypes.c_void_p])

SIGNATURES["qm_precond_apply"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_hamiltonian_diag"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p])

SIGNATURES["qm_eigh_lowest"] = (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p])
SIGNATURES["qm_zgemm"] = (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p])

_TDDFT_COMMON = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
_TDDFT_TAIL = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_int,
               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
SIGNATURES["qm_tddft_taylor"] = (ctypes.c_int, _TDDFT_COMMON + _TDDFT_TAIL)
SIGNATURES["qm_tddft_etrs"] = (ctypes.c_int, _TDDFT_COMMON + [ctypes.c_void_p] + _TDDFT_TAIL)
SIGNATURES["qm_gw_mel"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p])


class ScfOpts(ctypes.Structure):
    """qm_scf_opts of include/qm.h."""
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("alpha", ctypes.c_double),
                ("history", ctypes.c_int), ("dav_tol", ctypes.c_double), ("dav_max_iter", ctypes.c_int),
                ("prec", ctypes.c_int)]


class ScfStats(ctypes.Structure):
    """qm_scf_stats of include/qm.h."""
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("drho", ctypes.c_double),
                ("band_applies", ctypes.c_longlong), ("seconds", ctypes.c_double)]


SIGNATURES["qm_scf"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p,
                                       ctypes.POINTER(ScfOpts), c_double_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ScfStats), ctypes.c_void_p])

class HpsiJob(ctypes.Structure):
    """qm_hpsi_job of include/qm.h."""
    _fields_ = [("g", ctypes.c_void_p), ("ik", ctypes.c_int), ("nb", ctypes.c_int), ("psi", ctypes.c_void_p),
                ("ld_psi", ctypes.c_int), ("nproj", ctypes.c_int), ("vloc_r", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("ld_beta", ctypes.c_int), ("ld_out", ctypes.c_int),
                ("D", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class BatchShape(ctypes.Structure):
    """qm_batch_shape of include/qm.h."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("item_points", ctypes.c_int), ("group_mb", ctypes.c_int),
                ("fft_order", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    """qm_batch_info of include/qm.h."""
    _fields_ = [("ctas_per_sm", ctypes.c_int), ("item_points", ctypes.c_int), ("group_mb", ctypes.c_int),
                ("grid", ctypes.c_int),
                ("items", ctypes.c_int), ("cells", ctypes.c_int), ("candidates", ctypes.c_int),
                ("band_applies", ctypes.c_longlong), ("smem_bytes", ctypes.c_longlong),
                ("device_bytes", ctypes.c_longlong), ("tuned_ms", ctypes.c_double), ("fft_order", ctypes.c_int)]


SIGNATURES["qm_batch_create"] = (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(HpsiJob), ctypes.c_int,
                                                ctypes.POINTER(BatchShape), ctypes.c_void_p,
                                                ctypes.POINTER(ctypes.c_void_p)])
SIGNATURES["qm_batch_run"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_batch_check"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_batch_hold"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong])
SIGNATURES["qm_batch_query"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(BatchInfo)])
SIGNATURES["qm_batch_destroy"] = (None, [ctypes.c_void_p])


QM_MLP_NPARAM = 4481
SIGNATURES["qm_mlp_forward"] = (ctypes.c_int, [ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p])
SIGNATURES["qm_mlp_pairs"] = (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_mlp_loss_grad"] = (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                 c_double_p, ctypes.c_void_p, ctypes.c_void_p])
SIGNATURES["qm_mlp_train"] = (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_double, c_double_p, ctypes.c_void_p])


class DavidsonJob(ctypes.Structure):
    """qm_davidson_job of include/qm.h."""
    _fields_ = [("g", ctypes.c_void_p), ("ik", ctypes.c_int), ("nb", ctypes.c_int), ("psi_inout", ctypes.c_void_p),
                ("ld_psi", ctypes.c_int), ("nproj", ctypes.c_int), ("vloc_r", ctypes.c_void_p),
                ("beta", ctypes.c_void_p), ("ld_beta", ctypes.c_int), ("D", ctypes.c_void_p),
                ("eig_out", ctypes.c_void_p), ("stats", ctypes.POINTER(DavidsonStats)), ("history", ctypes.c_void_p),
                ("status", ctypes.c_int)]


SIGNATURES["qm_davidson_batched"] = (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(DavidsonJob),
                                                    ctypes.POINTER(DavidsonOpts), ctypes.c_int, ctypes.c_void_p])
