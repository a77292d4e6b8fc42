"""The C ABI library builds, loads and exports every symbol include/fwi.h declares (CPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fwi_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


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
    for code in range(9):
        assert lib.fwi_status_string(code).decode() != "unknown status", code


def test_bounds_checked_build_reports_itself():
    """The -DFWI_BOUNDS_CHECK variant builds, exports the same symbols and says so through
    fwi_bounds_checked; the normal build says it is not checked (host-only call)."""
    from paper_1504_08340_gb300 import build as b

    plain, checked = ctypes.CDLL(b.build()), ctypes.CDLL(b.build_checked())
    assert plain.fwi_bounds_checked() == 0 and checked.fwi_bounds_checked() == 1
    for name in _declared():
        assert hasattr(checked, name), name


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
        "fwi_get_state": (nul, nul, 0),
        "fwi_set_graphs": (nul, 1),
        "fwi_set_persistent": (nul, 1, ctypes.c_double(100.0), 0),
        "fwi_set_copy_wait": (nul, ctypes.c_double(100.0), 0),
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
        "fwi_tune_tiles": (nul, 0, 1, 3, nul),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == inval, name
    # argument checks of the allocation-free misfit come before any device work too
    assert lib.fwi_trace_misfit_noalloc(nul, nul, 10, 4, 1e-3, nul, nul) == inval
    assert set(calls) | {"fwi_create", "fwi_destroy", "fwi_last_error", "fwi_status_string", "fwi_bounds_checked",
                         "fwi_trace_misfit_noalloc"} == {e for e in fwi.EXPORTS if not e.startswith("fwi_nn_")}
    # the preconditioner kernels check pointers and sizes before any device work
    one = C.c_void_p(1)
    assert lib.fwi_nn_conv3d_forward(nul, one, nul, 1, 1, 2, 2, 2, 0, one, nul) == inval
    assert lib.fwi_nn_conv3d_forward(one, one, nul, 0, 1, 2, 2, 2, 0, one, nul) == inval
    assert lib.fwi_nn_conv3d_backward_data(one, one, 1, 1, 0, 2, 2, one, nul) == inval
    assert lib.fwi_nn_conv3d_backward_weight(one, one, 1, 1, 2, 2, 2, one, nul, nul, nul) == inval
    assert lib.fwi_nn_conv3d_backward_weight_work(0, 1, 2, 2, 2) == 0
    # one 2048-voxel slice x 16 output-channel columns x (27 x 8 + 1 rows, padded to 256)
    assert lib.fwi_nn_conv3d_backward_weight_work(3, 4, 2, 2, 2) == 1 * 16 * 256
    assert lib.fwi_nn_conv3d_backward_weight_work(3, 4, 20, 20, 24) == 5 * 16 * 256
    assert lib.fwi_nn_relu_backward(one, one, 0, one, nul) == inval
    assert lib.fwi_nn_mse(one, one, 10, one, nul, one, nul) == inval
    assert lib.fwi_nn_adam(one, nul, one, one, one, 10, 1e-3, 0.9, 0.999, 1e-8, 0, nul) == inval
    assert lib.fwi_nn_adam(one, nul, one, one, one, 10, 1e-3, 1.0, 0.999, 1e-8, 1, nul) == inval
    assert lib.fwi_nn_pool2_forward(nul, 1, 2, 2, 2, one, nul) == inval
    assert lib.fwi_nn_pool2_backward(one, 0, 2, 2, 2, 0, one, nul) == inval
    assert lib.fwi_nn_upsample2_forward(one, 1, 2, 0, 2, one, nul) == inval
    assert lib.fwi_nn_upsample2_backward(one, 1, 2, 2, 2, 1, nul, nul) == inval
    assert lib.fwi_nn_to_bf16(nul, 4, one, nul) == inval
    assert lib.fwi_nn_from_bf16(one, 4, nul, nul) == inval
