"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/vegas.h declares.  Host-only calls only: no GPU is needed."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "vegas.h")).read()
    return sorted(set(re.findall(r"VEGAS_API\s+[\w\s\*]*?\b(vegas_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vegas_create", "vegas_integrate", "vegas_destroy", "vegas_allocate", "vegas_fill",
                 "vegas_refine", "vegas_combine", "vegas_strerror"):
        assert must in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_2408_09229_gb300 import build_lib
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls():
    from paper_2408_09229_gb300 import build_lib
    lib = ctypes.CDLL(build_lib.build())
    lib.vegas_strerror.restype = ctypes.c_char_p
    assert lib.vegas_strerror(0) == b"ok"
    assert b"non-finite" in lib.vegas_strerror(-4)
    lib.vegas_allocate_scratch_bytes.restype = ctypes.c_size_t
    lib.vegas_allocate_scratch_bytes.argtypes = [ctypes.c_int64]
    assert lib.vegas_allocate_scratch_bytes(43046721) > 8 * (43046721 // 4096)
    assert lib.vegas_allocate_scratch_bytes(0) == 0
    # argument checks happen before any CUDA call
    lib.vegas_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.vegas_create(0, 50, 0, 0.5, 0.75, ctypes.byref(h)) == -1
    assert lib.vegas_create(4, 1, 0, 0.5, 0.75, ctypes.byref(h)) == -1
    assert lib.vegas_create(4, 50, 0, 0.5, 1.5, ctypes.byref(h)) == -1


def test_product_path_has_no_oracle_reference():
    pkg = os.path.join(ROOT, "paper_2408_09229_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "oracle_vegas" not in text, f


def test_flow_binding_refuses_wrong_buffers():
    """the flow entry points read raw FP32 device memory: the binding refuses host or FP64 tensors before the
    call instead of passing their bytes on"""
    torch = __import__("pytest").importorskip("torch")
    from paper_2408_09229_gb300 import vegas as V
    d, n = 4, 8
    p = torch.zeros(V.flow_param_count(d), dtype=torch.float64)
    x = torch.zeros((n, d), dtype=torch.float32)
    ld = torch.zeros(n, dtype=torch.float32)
    import pytest
    with pytest.raises(TypeError):
        V.flow_apply(d, V.FLOW_SAMPLE, p, x, x, ld)
    with pytest.raises(TypeError):
        V.flow_adam(x, x, x, x, 1)
