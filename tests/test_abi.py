"""The C ABI library builds, loads and exports every symbol include/fwi.h declares (CPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fwi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fwi_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1504_08340_gb300 import build as b
    from paper_1504_08340_gb300.fwi import EXPORTS

    path = b.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert declared, "no declarations found"
    assert set(declared) == set(EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest

    from paper_1504_08340_gb300 import fwi

    with pytest.raises(ImportError):
        saved = fwi._lib
        fwi._lib = None
        try:
            fwi.load_library(str(tmp_path / "missing.so"))
        finally:
            fwi._lib = saved


def test_status_strings():
    from paper_1504_08340_gb300 import build as b

    lib = ctypes.CDLL(b.build())
    lib.fwi_status_string.restype = ctypes.c_char_p
    for code in range(8):
        assert lib.fwi_status_string(code)


def test_null_context_is_rejected_without_touching_the_gpu():
    """Every entry point that takes a context returns FWI_E_INVAL (1) for a null one,
    before any CUDA call, so the checks run here on the CPU."""
    import ctypes as C

    from paper_1504_08340_gb300 import build as b
    from paper_1504_08340_gb300 import fwi

    b.build()
    lib = fwi.load_library()
    inval = 1
    nul = None
    assert lib.fwi_create(nul, nul) == inval
    lib.fwi_destroy(nul)  # a no-op
    assert lib.fwi_last_error(nul) == b"null context"
    calls = {
        "fwi_get_dims": (nul, nul),
        "fwi_set_material": (nul, nul, nul, 0),
        "fwi_set_sources": (nul, 1, nul, nul, 0, nul),
        "fwi_set_receivers": (nul, 1, nul),
        "fwi_forward": (nul, 0, 1, nul, 0),
        "fwi_misfit": (nul, 0, 1, nul, 0, nul),
        "fwi_adjoint_gradient": (nul, 0, 1, nul, 0, nul, nul, nul),
        "fwi_get_mass_tilde": (nul, nul),
        "fwi_rhs": (nul, 0, nul, nul, 0),
        "fwi_set_timing": (nul, 1),
        "fwi_get_timing": (nul, 0, nul, nul),
        "fwi_reset_timing": (nul,),
        "fwi_step": (nul, nul, 0, nul, nul),
        "fwi_step_reset": (nul,),
        "fwi_get_material": (nul, nul, nul, 0),
        "fwi_set_checkpointing": (nul, 0),
        "fwi_regularization": (nul, 0, 0.0, nul, nul, nul, 0),
        "fwi_set_shot_batch": (nul, 2),
        "fwi_tune_shot_batch": (nul, 0, 1, 4, 3, 0.8, nul),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == inval, name
    # argument checks of the allocation-free misfit come before any device work too
    assert lib.fwi_trace_misfit_noalloc(nul, nul, 10, 4, 1e-3, nul, nul) == inval
    assert set(calls) | {"fwi_create", "fwi_destroy", "fwi_last_error", "fwi_status_string",
                         "fwi_trace_misfit_noalloc"} == set(fwi.EXPORTS)
