"""The C-ABI library loads on a host without a GPU, exports every function
declared in include/qed.h, and rejects invalid arguments before touching
CUDA."""
import ctypes
import os
import re

import pytest

from paper_2511_19456_b300 import _lib

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "qed.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\*?\s*(qed_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("qed_plan_create", "qed_eval", "qed_eval_grad", "qed_plan_destroy",
                 "qed_plan_info", "qed_status_string"):
        assert must in names


def test_library_exports_every_declared_symbol():
    L = _lib.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings():
    assert _lib.status_string(0) == "ok"
    assert _lib.status_string(1) == "invalid argument"
    assert _lib.status_string(99) == "unknown status"


def test_invalid_arguments_rejected_without_gpu():
    L = _lib.lib()
    out = ctypes.c_void_p()
    spin = _lib.SpinCfg()
    spin.summed = 1
    assert L.qed_plan_create(None, ctypes.byref(spin), 0, ctypes.byref(out)) == _lib.QED_EINVAL
    for k in (0, 8, -1):
        proc = _lib.Process(k, 1.0, 1.0)
        assert L.qed_plan_create(ctypes.byref(proc), ctypes.byref(spin), 0,
                                 ctypes.byref(out)) == _lib.QED_EINVAL
    proc = _lib.Process(2, -1.0, 1.0)
    assert L.qed_plan_create(ctypes.byref(proc), ctypes.byref(spin), 0, ctypes.byref(out)) == _lib.QED_EINVAL
    proc = _lib.Process(2, 1.0, 1.0)
    assert L.qed_plan_create(ctypes.byref(proc), ctypes.byref(spin), 7, ctypes.byref(out)) == _lib.QED_EINVAL
    bad = _lib.SpinCfg()
    bad.summed = 0
    for i, v in enumerate([1, 3, 1, 1, 1]):   # photon polarisation 3 is invalid
        bad.hel[i] = v
    assert L.qed_plan_create(ctypes.byref(proc), ctypes.byref(bad), 0, ctypes.byref(out)) == _lib.QED_EINVAL
    assert out.value is None
    assert L.qed_eval(None, None, 10, None, None) == _lib.QED_EINVAL
    assert L.qed_eval_grad(None, None, 10, None, None, None) == _lib.QED_EINVAL
    assert L.qed_eval_host(None, None, 10, None, None) == _lib.QED_EINVAL
    assert L.qed_plan_info(None, None) == _lib.QED_EINVAL
    assert L.qed_plan_set_kernel_form(None, 0) == _lib.QED_EINVAL
    assert L.qed_plan_tune(None, None, 10, None, None, None, None, None) == _lib.QED_EINVAL
    assert L.qed_dag_counts(0, None) == _lib.QED_EINVAL
    L.qed_plan_destroy(None)  # no-op


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no fallback"):
        _lib.lib()
