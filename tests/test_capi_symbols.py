"""The C-ABI library loads on a CPU-only host and exports every entry point
include/qsim.h declares (no compute calls: there may be no GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    return sorted(set(re.findall(r"QSIM_API\s+[\w\s\*]*?\b(qsim_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ["qsim_alloc", "qsim_apply_1q", "qsim_apply_ctrl", "qsim_apply_fused", "qsim_probs",
                 "qsim_norm", "qsim_swap_qubits", "qsim_run_circuit", "qsim_run_batch", "qsim_qubit_probs",
                 "qsim_get_state", "qsim_sample"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_quant_ph_0608239_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing
    # version string needs no device
    lib.qsim_version.restype = ctypes.c_char_p
    assert lib.qsim_version().startswith(b"qsim-gb300")


def test_binding_covers_the_header():
    from paper_quant_ph_0608239_gb300 import _capi
    assert sorted(_capi.EXPORTED) == declared()


def test_host_validation_without_device():
    # a NULL handle is rejected on the host before any CUDA call
    from paper_quant_ph_0608239_gb300 import _capi
    lib = _capi.load()
    U = (ctypes.c_double * 8)(1, 0, 0, 0, 0, 0, 1, 0)
    assert lib.qsim_apply_1q(None, 0, U) == _capi.QSIM_EINVAL
    assert b"null handle" in lib.qsim_last_error()
    h = _capi.c_handle()
    assert lib.qsim_alloc(0, 0, ctypes.byref(h)) == _capi.QSIM_EINVAL
    assert lib.qsim_alloc(35, 0, ctypes.byref(h)) == _capi.QSIM_EINVAL
    assert lib.qsim_alloc(10, 7, ctypes.byref(h)) == _capi.QSIM_EINVAL
    assert lib.qsim_free(None) == _capi.QSIM_OK
