"""ctypes binding of libqedm2.so (the C-ABI declared in include/qed.h).

Argument marshalling only: every step of the |M|^2 evaluation runs in the
library's CUDA kernels.  Loading fails loudly when the library is missing;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqedm2.so")

QED_OK, QED_EINVAL, QED_ENOMEM, QED_ECUDA, QED_EUNSUPPORTED, QED_EDEVICE_TIMEOUT = range(6)
QED_FP64, QED_MIXED = 0, 1
QED_KERNEL_TABLE, QED_KERNEL_SPECIALISED = 0, 1


class QedError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class Process(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("mass", ctypes.c_double), ("charge", ctypes.c_double)]


class AbcProcess(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("mass_a", ctypes.c_double), ("mass_b", ctypes.c_double),
                ("mass_c", ctypes.c_double), ("coupling", ctypes.c_double)]


class TapeDesc(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in ("k", "n", "steps", "n_slots", "n_diag", "n_instr", "n_levels")] + \
               [(f, ctypes.c_longlong) for f in ("nodes", "compute_nodes", "flops")]


class SpinCfg(ctypes.Structure):
    _fields_ = [("summed", ctypes.c_int), ("hel", ctypes.c_byte * 10)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("n_photons", ctypes.c_int),
                ("n_diagrams", ctypes.c_longlong), ("n_states", ctypes.c_longlong),
                ("nodes_unreduced", ctypes.c_longlong), ("nodes_reduced", ctypes.c_longlong),
                ("compute_reduced", ctypes.c_longlong), ("v_nodes", ctypes.c_longlong),
                ("s1_nodes", ctypes.c_longlong), ("s2_nodes", ctypes.c_longlong),
                ("flops_per_point", ctypes.c_longlong),
                ("flops_executed_per_point", ctypes.c_longlong),
                ("flops_literal_s2_per_point", ctypes.c_longlong),
                ("team_threads", ctypes.c_int), ("smem_bytes_per_team", ctypes.c_int),
                ("precision", ctypes.c_int), ("reduction_steps", ctypes.c_int),
                ("kernel_form", ctypes.c_int), ("kernel_forms", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("grid_blocks", ctypes.c_int)]


class DagCounts(ctypes.Structure):
    _fields_ = [(f"{a}_{b}", ctypes.c_longlong)
                for a in ("unreduced", "reduced")
                for b in ("total", "data", "u", "v", "s1", "s2", "sum")]


class ScheduleDesc(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int) for f in (
        "k", "n", "h", "r", "ls", "rs", "summed", "n_left_leaves", "n_right_leaves",
        "stored_currents", "local_currents", "n_stored_phases", "n_set_phases", "n_sets",
        "n_instr", "n_phases")] + [("flops_algorithmic", ctypes.c_longlong),
                                   ("flops_executed", ctypes.c_longlong)]


_vp = ctypes.c_void_p
_ll = ctypes.c_longlong

# (name, restype, argtypes) of every function in include/qed.h
SIGNATURES = [
    ("qed_plan_create", ctypes.c_int, [ctypes.POINTER(Process), ctypes.POINTER(SpinCfg),
                                       ctypes.c_int, ctypes.POINTER(_vp)]),
    ("qed_plan_create_rewrite", ctypes.c_int, [ctypes.POINTER(Process), ctypes.POINTER(SpinCfg),
                                               ctypes.c_int, ctypes.POINTER(_vp)]),
    ("qed_abc_plan_create", ctypes.c_int, [ctypes.POINTER(AbcProcess), ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(_vp)]),
    ("qed_plan_info", ctypes.c_int, [_vp, ctypes.POINTER(PlanInfo)]),
    ("qed_plan_set_kernel_form", ctypes.c_int, [_vp, ctypes.c_int]),
    ("qed_plan_tune", ctypes.c_int, [_vp, _vp, _ll, _vp, _vp, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    ("qed_debug_inject_alloc_failure", ctypes.c_int, [ctypes.c_int]),
    ("qed_reduction_steps", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("qed_tape_export", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(TapeDesc), _vp,
                                       ctypes.POINTER(ctypes.c_int)]),
    ("qed_tape_plan_create", ctypes.c_int, [ctypes.POINTER(Process), ctypes.POINTER(SpinCfg), ctypes.c_int,
                                            ctypes.POINTER(_vp)]),
    ("qed_eval", ctypes.c_int, [_vp, _vp, _ll, _vp, _vp]),
    ("qed_eval_grad", ctypes.c_int, [_vp, _vp, _ll, _vp, _vp, _vp]),
    ("qed_grad_workspace_bytes", ctypes.c_int, [_vp, ctypes.POINTER(_ll)]),
    ("qed_eval_grad_ws", ctypes.c_int, [_vp, _vp, _ll, _vp, _vp, _vp, _ll, _vp]),
    ("qed_eval_host", ctypes.c_int, [_vp, _vp, _ll, _vp, _vp]),
    ("qed_plan_destroy", None, [_vp]),
    ("qed_dag_counts", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(DagCounts)]),
    ("qed_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("qed_measure_fma_peak", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp]),
    ("qed_batch_create", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_ll),
                                        ctypes.POINTER(_vp)]),
    ("qed_batch_eval", ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    ("qed_batch_tune", ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp,
                                      ctypes.POINTER(ctypes.c_double)]),
    ("qed_batch_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(_ll)]),
    ("qed_batch_set_kernel_form", ctypes.c_int, [_vp, ctypes.c_int]),
    ("qed_batch_kernel_form", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int)]),
    ("qed_batch_destroy", None, [_vp]),
    ("qed_batch_eval_static", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_ll),
                                             ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    ("qed_generate", ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_ulonglong,
                                    _ll, _ll, _vp, _vp, _vp]),
    ("qed_cross_section", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_ulonglong, _ll, _ll, _ll, _vp, _vp,
                                         _vp, _vp, _vp] + [ctypes.POINTER(ctypes.c_double)] * 4),
    ("qed_rewrite_schedule_export", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(ScheduleDesc), _vp, _vp, _vp]),
    ("qed_schedule_export", ctypes.c_int, [ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ScheduleDesc), _vp, _vp, _vp]),
]

_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2511_19456_b300.build` (no fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().qed_status_string(int(status)).decode()


def check(status: int, what: str) -> None:
    if status != QED_OK:
        raise QedError(status, what)
