"""Python front end of the C-ABI: plans, evaluation on device or host buffers.

PyTorch supplies device memory and streams; the arithmetic runs in the
library's kernels.  Momenta are float64 tensors of shape [N, k+3, 4] (slot 0
e- in, 1 gamma in, 2 e- out, 3.. gamma out; components E, px, py, pz).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import check

_PREC = {"fp64": _lib.QED_FP64, "mixed": _lib.QED_MIXED}


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A built CDAG for e- gamma -> e- + k gamma with its device tables.

    summed=True sums |M|^2 over all 2^(k+3) helicity/polarisation states;
    otherwise `hel` gives one state per slot (electrons +1/-1, photons 1/2).
    precision: "fp64" or "mixed".
    """

    def __init__(self, k: int, summed: bool = True, hel=None, precision: str = "fp64",
                 mass: float = 1.0, charge: float = 1.0, rewrite: bool = False):
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {sorted(_PREC)}")
        L = _lib.lib()
        proc = _lib.Process(int(k), float(mass), float(charge))
        spin = _lib.SpinCfg()
        spin.summed = 1 if summed else 0
        if not summed:
            if hel is None or len(hel) != k + 3:
                raise ValueError("a fixed state needs hel with k+3 entries")
            for i, v in enumerate(hel):
                spin.hel[i] = int(v)
        handle = ctypes.c_void_p()
        create = L.qed_plan_create_rewrite if rewrite else L.qed_plan_create
        check(create(ctypes.byref(proc), ctypes.byref(spin), _PREC[precision], ctypes.byref(handle)),
              "qed_plan_create")
        self.rewrite = bool(rewrite)
        self._h = handle
        self.k = int(k)
        self.summed = bool(summed)
        self.hel = None if summed else list(hel)
        self.precision = precision
        self.mass = float(mass)

    # -------------------------------------------------------------- info
    def info(self) -> dict:
        inf = _lib.PlanInfo()
        check(_lib.lib().qed_plan_info(self._h, ctypes.byref(inf)), "qed_plan_info")
        return {f: getattr(inf, f) for f, _ in _lib.PlanInfo._fields_}

    KERNEL_FORMS = {"table": _lib.QED_KERNEL_TABLE, "specialised": _lib.QED_KERNEL_SPECIALISED}

    @property
    def kernel_form(self) -> str:
        """The forward kernel in use: "table" (schedule read from device
        tables) or "specialised" (straight-line code generated at build time)."""
        f = self.info()["kernel_form"]
        return next(name for name, v in self.KERNEL_FORMS.items() if v == f)

    def kernel_forms(self) -> list:
        """The forms this plan has."""
        bits = self.info()["kernel_forms"]
        return [name for name, v in self.KERNEL_FORMS.items() if bits & (1 << v)]

    def set_kernel_form(self, form: str) -> None:
        check(_lib.lib().qed_plan_set_kernel_form(self._h, self.KERNEL_FORMS[form]), "qed_plan_set_kernel_form")

    def tune(self, momenta, out=None, stream=None) -> dict:
        """Times every kernel form and block size on these device buffers,
        keeps the fastest; returns {"form", "block", "ms"}.  Synchronous."""
        torch = _torch()
        self._check_momenta(momenta, device=True)
        n = momenta.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=momenta.device)
        f, b, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        check(_lib.lib().qed_plan_tune(self._h, ctypes.c_void_p(momenta.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream),
                                       ctypes.byref(f), ctypes.byref(b), ctypes.byref(ms)), "qed_plan_tune")
        name = next(nm for nm, v in self.KERNEL_FORMS.items() if v == f.value)
        return {"form": name, "block": b.value, "ms": ms.value}

    def _check_momenta(self, momenta, device: bool):
        torch = _torch()
        if momenta.dtype != torch.float64:
            raise TypeError("momenta must be float64")
        if momenta.dim() != 3 or momenta.shape[1] != self.k + 3 or momenta.shape[2] != 4:
            raise ValueError(f"momenta must have shape [N, {self.k + 3}, 4]")
        if not momenta.is_contiguous():
            raise ValueError("momenta must be contiguous")
        if device and not momenta.is_cuda:
            raise ValueError("momenta must be a CUDA tensor")
        if not device and momenta.is_cuda:
            raise ValueError("momenta must be a host tensor")

    # -------------------------------------------------------------- eval
    def eval(self, momenta, out=None, stream=None):
        """|M|^2 per point on the device (asynchronous on `stream`)."""
        torch = _torch()
        self._check_momenta(momenta, device=True)
        n = momenta.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=momenta.device)
        check(_lib.lib().qed_eval(self._h, ctypes.c_void_p(momenta.data_ptr()), n,
                                  ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "qed_eval")
        return out

    def eval_grad(self, momenta, out=None, grad=None, stream=None):
        """(|M|^2, d|M|^2/d k_j) with k_j the outgoing photons' 3-momenta."""
        torch = _torch()
        self._check_momenta(momenta, device=True)
        n = momenta.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=momenta.device)
        if grad is None:
            grad = torch.empty((n, self.k, 3), dtype=torch.float64, device=momenta.device)
        check(_lib.lib().qed_eval_grad(self._h, ctypes.c_void_p(momenta.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(grad.data_ptr()), _stream_handle(stream)),
              "qed_eval_grad")
        return out, grad

    def grad_workspace_bytes(self) -> int:
        """Device workspace that eval_grad(workspace=...) needs (0: none)."""
        v = ctypes.c_longlong()
        check(_lib.lib().qed_grad_workspace_bytes(self._h, ctypes.byref(v)), "qed_grad_workspace_bytes")
        return v.value

    def eval_grad_ws(self, momenta, workspace, out=None, grad=None, stream=None):
        """eval_grad with the adjoint's scratch in a caller-owned device
        buffer (a uint8 CUDA tensor of at least grad_workspace_bytes())."""
        torch = _torch()
        self._check_momenta(momenta, device=True)
        n = momenta.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=momenta.device)
        if grad is None:
            grad = torch.empty((n, self.k, 3), dtype=torch.float64, device=momenta.device)
        ws_ptr = workspace.data_ptr() if workspace is not None else 0
        ws_bytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        check(_lib.lib().qed_eval_grad_ws(self._h, ctypes.c_void_p(momenta.data_ptr()), n,
                                          ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                          ctypes.c_void_p(ws_ptr), ws_bytes, _stream_handle(stream)),
              "qed_eval_grad_ws")
        return out, grad

    def eval_host(self, momenta, out=None, stream=None):
        """End to end on host buffers: copy in, evaluate, copy back (synchronous)."""
        torch = _torch()
        self._check_momenta(momenta, device=False)
        n = momenta.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, pin_memory=momenta.is_pinned())
        check(_lib.lib().qed_eval_host(self._h, ctypes.c_void_p(momenta.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
              "qed_eval_host")
        return out

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().qed_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AbcPlan(Plan):
    """A plan for the ABC model (paper App. F): A B -> A + k B, k odd in
    1..7, through the node-reduced DAG (rewrite=False) or the rewritten DAG,
    with scalar currents.  Momenta as for QED (slot 0 A in, 1 B in, 2 A out,
    3.. B out).  mass_b enters only through the momenta."""

    def __init__(self, k: int, precision: str = "fp64", rewrite: bool = False, mass_a: float = 1.0,
                 mass_b: float = 0.0, mass_c: float = 1.0, coupling: float = 1.0):
        if precision not in _PREC:
            raise ValueError(f"precision must be one of {sorted(_PREC)}")
        proc = _lib.AbcProcess(int(k), float(mass_a), float(mass_b), float(mass_c), float(coupling))
        handle = ctypes.c_void_p()
        check(_lib.lib().qed_abc_plan_create(ctypes.byref(proc), _PREC[precision], 1 if rewrite else 0,
                                             ctypes.byref(handle)), "qed_abc_plan_create")
        self._h = handle
        self.rewrite = bool(rewrite)
        self.k = int(k)
        self.summed = False
        self.hel = None
        self.precision = precision
        self.mass = float(mass_a)
        self.mass_c = float(mass_c)
        self.coupling = float(coupling)


class TapePlan(Plan):
    """Node-by-node execution of the CDAG of e- gamma -> e- + k gamma (one
    fixed spin state, k <= 5, FP64) after `reduction_steps` single node
    reductions: the node-reduction sweep of the paper's Sec. III-D."""

    def __init__(self, k: int, hel, reduction_steps: int, mass: float = 1.0, charge: float = 1.0):
        if hel is None or len(hel) != k + 3:
            raise ValueError("a fixed state needs hel with k+3 entries")
        proc = _lib.Process(int(k), float(mass), float(charge))
        spin = _lib.SpinCfg()
        spin.summed = 0
        for i, v in enumerate(hel):
            spin.hel[i] = int(v)
        handle = ctypes.c_void_p()
        check(_lib.lib().qed_tape_plan_create(ctypes.byref(proc), ctypes.byref(spin), int(reduction_steps),
                                              ctypes.byref(handle)), "qed_tape_plan_create")
        self._h = handle
        self.rewrite = False
        self.k = int(k)
        self.summed = False
        self.hel = list(hel)
        self.precision = "fp64"
        self.mass = float(mass)


def inject_alloc_failure(after: int) -> None:
    """Test hook: after `after` more successful device allocations of the
    library the next one fails as out of memory (-1 switches it off)."""
    check(_lib.lib().qed_debug_inject_alloc_failure(int(after)), "qed_debug_inject_alloc_failure")


def reduction_steps(k: int) -> int:
    """Single node reductions from the per-diagram CDAG to its fixpoint."""
    out = ctypes.c_int()
    check(_lib.lib().qed_reduction_steps(int(k), ctypes.byref(out)), "qed_reduction_steps")
    return out.value


TAPE_DTYPE = np.dtype([("op", "u1"), ("side", "u1"), ("arg", "u1"), ("pad", "u1"), ("mask", "<u2"),
                       ("dst", "<u2"), ("src0", "<u2"), ("src1", "<u2"), ("pad2", "<u4")])


def tape_export(k: int, steps: int) -> dict:
    """The tape of the CDAG after `steps` node reductions (see TapePlan)."""
    L = _lib.lib()
    d = _lib.TapeDesc()
    check(L.qed_tape_export(int(k), int(steps), ctypes.byref(d), None, None), "qed_tape_export")
    instr = np.zeros(d.n_instr, dtype=TAPE_DTYPE)
    levels = np.zeros(d.n_levels + 1, dtype=np.int32)
    check(L.qed_tape_export(int(k), int(steps), ctypes.byref(d), instr.ctypes.data_as(ctypes.c_void_p),
                            levels.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "qed_tape_export")
    out = {f: getattr(d, f) for f, _ in _lib.TapeDesc._fields_}
    out.update(instr=instr, levels=levels)
    return out


def dag_counts(k: int) -> dict:
    """Node counts of the per-diagram CDAG and of its node-reduced form."""
    c = _lib.DagCounts()
    check(_lib.lib().qed_dag_counts(int(k), ctypes.byref(c)), "qed_dag_counts")
    return {f: getattr(c, f) for f, _ in _lib.DagCounts._fields_}


INSTR_DTYPE = np.dtype([("dst", "<i4"), ("src", "<i4"), ("side", "u1"), ("photon", "u1"),
                        ("rank", "u1"), ("level", "u1"), ("post", "<u2"), ("pad", "<u2")])
PHASE_DTYPE = np.dtype([("beg", "<i4", 2), ("cnt", "<i4", 2), ("level", "<i4", 2)])
SET_DTYPE = np.dtype([("mask", "<u4"), ("phase0", "<i4"), ("leaf_l", "<i4"), ("leaf_r", "<i4")])


SUM_INSTR_DTYPE = np.dtype([("dst", "<i4"), ("src", "<i4", 4), ("photon", "u1", 4), ("rank", "u1", 4),
                            ("nterms", "u1"), ("side", "u1"), ("level", "u1"), ("pad0", "u1"),
                            ("post", "<u2"), ("pad1", "<u2"), ("pad2", "<i4", 3)])


def schedule_export(k: int, summed: bool, rewrite: bool = False, group: int = 0) -> dict:
    """The linear schedule the kernels execute, as numpy structured arrays.
    rewrite: the distributively rewritten DAG; group: its photon sets per set
    phase (0: the default)."""
    L = _lib.lib()
    d = _lib.ScheduleDesc()
    if rewrite:
        def fn(*a):
            return L.qed_rewrite_schedule_export(a[0], a[1], int(group), *a[2:])
    else:
        fn = L.qed_schedule_export
    check(fn(int(k), int(summed), ctypes.byref(d), None, None, None), "qed_schedule_export")
    instr = np.zeros(d.n_instr, dtype=SUM_INSTR_DTYPE if rewrite else INSTR_DTYPE)
    phases = np.zeros(d.n_phases, dtype=PHASE_DTYPE)
    sets = np.zeros(d.n_sets, dtype=SET_DTYPE)
    check(fn(int(k), int(summed), ctypes.byref(d),
             instr.ctypes.data_as(ctypes.c_void_p),
             phases.ctypes.data_as(ctypes.c_void_p),
             sets.ctypes.data_as(ctypes.c_void_p)), "qed_schedule_export")
    out = {f: getattr(d, f) for f, _ in _lib.ScheduleDesc._fields_}
    out.update(instr=instr, phases=phases, sets=sets)
    if rewrite:
        out["group"] = int(np.sum(sets["phase0"] == sets["phase0"][0]))
    return out


def measure_fma_peak(precision: str = "fp64", stream=None) -> float:
    """FMA-pipe peak of the current device in TFLOP/s (FP64 or FP32)."""
    v = ctypes.c_double()
    check(_lib.lib().qed_measure_fma_peak(_PREC[precision], ctypes.byref(v), _stream_handle(stream)),
          "qed_measure_fma_peak")
    return v.value


class Batch:
    """Requests of different k evaluated in one persistent launch (CUDA graph).

    plans: Plan objects (spin-summed, k <= 5, one precision); n_points: the
    point count of each request.  The batch keeps references to the plans.
    """

    def __init__(self, plans, n_points):
        self.plans = list(plans)
        self.n_points = [int(n) for n in n_points]
        nreq = len(self.plans)
        ph = (ctypes.c_void_p * nreq)(*[p._h.value for p in self.plans])
        nn = (ctypes.c_longlong * nreq)(*self.n_points)
        h = ctypes.c_void_p()
        check(_lib.lib().qed_batch_create(ph, nreq, nn, ctypes.byref(h)), "qed_batch_create")
        self._h = h

    def _ptrs(self, momenta, outs):
        if len(momenta) != len(self.plans) or len(outs) != len(self.plans):
            raise ValueError("one momenta tensor and one output per request")
        for p, m, o, n in zip(self.plans, momenta, outs, self.n_points):
            p._check_momenta(m, device=True)
            if m.shape[0] != n or o.numel() != n:
                raise ValueError("request sizes differ from the batch's")
        nreq = len(self.plans)
        return ((ctypes.c_void_p * nreq)(*[m.data_ptr() for m in momenta]),
                (ctypes.c_void_p * nreq)(*[o.data_ptr() for o in outs]))

    def outputs(self, device="cuda"):
        torch = _torch()
        return [torch.empty(n, dtype=torch.float64, device=device) for n in self.n_points]

    def eval(self, momenta, outs=None, stream=None):
        outs = self.outputs() if outs is None else outs
        pm, po = self._ptrs(momenta, outs)
        check(_lib.lib().qed_batch_eval(self._h, pm, po, _stream_handle(stream)), "qed_batch_eval")
        return outs

    def tune(self, momenta, outs=None, stream=None) -> float:
        outs = self.outputs() if outs is None else outs
        pm, po = self._ptrs(momenta, outs)
        ms = ctypes.c_double()
        check(_lib.lib().qed_batch_tune(self._h, pm, po, _stream_handle(stream), ctypes.byref(ms)),
              "qed_batch_tune")
        return ms.value

    def info(self) -> dict:
        b, t, n, f = ctypes.c_int(), ctypes.c_double(), ctypes.c_longlong(), ctypes.c_int()
        check(_lib.lib().qed_batch_info(self._h, ctypes.byref(b), ctypes.byref(t), ctypes.byref(n)),
              "qed_batch_info")
        check(_lib.lib().qed_batch_kernel_form(self._h, ctypes.byref(f)), "qed_batch_kernel_form")
        form = next(name for name, v in Plan.KERNEL_FORMS.items() if v == f.value)
        return {"block": b.value, "work_target_flops": t.value, "n_items": n.value, "kernel_form": form}

    def set_kernel_form(self, form: str) -> None:
        """"table" or "specialised" (straight-line points for every k)."""
        check(_lib.lib().qed_batch_set_kernel_form(self._h, Plan.KERNEL_FORMS[form]), "qed_batch_set_kernel_form")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().qed_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(k: int, n_points: int, omega: float, seed: int, offset: int = 0, mass: float = 1.0,
             weights: bool = False, stream=None):
    """Phase-space points (and weights) generated on the device; the same
    recipe and random draws as phasespace.points()."""
    torch = _torch()
    mom = torch.empty((n_points, k + 3, 4), dtype=torch.float64, device="cuda")
    w = torch.empty(n_points, dtype=torch.float64, device="cuda") if weights else None
    check(_lib.lib().qed_generate(int(k), float(omega), float(mass), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                  int(offset), int(n_points), ctypes.c_void_p(mom.data_ptr()),
                                  ctypes.c_void_p(w.data_ptr() if w is not None else None),
                                  _stream_handle(stream)), "qed_generate")
    return (mom, w) if weights else mom


def cross_section(plan, omega: float, n_points: int, seed: int, offset: int = 0,
                  chunk: int = 1 << 20, stream=None) -> dict:
    """Monte Carlo total cross section of a spin-summed plan (e = m = 1 units
    unless the plan says otherwise): generated on the device, evaluated, and
    reduced on the device."""
    torch = _torch()
    chunk = int(min(chunk, n_points))
    k = plan.k
    mom = torch.empty((chunk, k + 3, 4), dtype=torch.float64, device="cuda")
    w = torch.empty(chunk, dtype=torch.float64, device="cuda")
    m2 = torch.empty(chunk, dtype=torch.float64, device="cuda")
    acc = torch.zeros(2, dtype=torch.float64, device="cuda")
    out = [ctypes.c_double() for _ in range(4)]
    check(_lib.lib().qed_cross_section(plan._h, float(omega), int(seed) & 0xFFFFFFFFFFFFFFFF, int(offset),
                                       int(n_points), chunk, ctypes.c_void_p(mom.data_ptr()),
                                       ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(m2.data_ptr()),
                                       ctypes.c_void_p(acc.data_ptr()), _stream_handle(stream),
                                       *[ctypes.byref(o) for o in out]), "qed_cross_section")
    return {"sigma": out[0].value, "sigma_err": out[1].value, "sum_wm2": out[2].value,
            "sum_wm2_sq": out[3].value, "n_points": int(n_points)}
