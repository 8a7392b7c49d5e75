"""CPU checks of the boundary: libes.so builds, loads and exports every entry
point declared in include/es.h; the Python binding has the same names."""
import os
import re

from paper_2003_08831_gb300 import _binding
from paper_2003_08831_gb300 import build as b

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "es.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(es_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib_path = b.build()
    assert os.path.exists(lib_path)
    lib = _binding.load(lib_path)
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
        assert hasattr(_binding, s), s
    assert set(syms) == set(_binding.EXPORTS)


def test_strerror_and_invalid_config_without_gpu():
    lib = _binding.load()
    assert _binding.strerror(0) == "ok"
    assert "root" in _binding.strerror(_binding.ES_ERR_NO_ROOT)
    # argument checks happen on the host before any CUDA call
    cfg = _binding.make_config(7, (2, 2, 2))
    import ctypes
    ctx = ctypes.c_void_p()
    assert lib.es_create(ctypes.byref(cfg), ctypes.byref(ctx)) == _binding.ES_ERR_INVALID
    cfg = _binding.make_config(3, (0, 2, 2))
    assert lib.es_create(ctypes.byref(cfg), ctypes.byref(ctx)) == _binding.ES_ERR_INVALID
    assert lib.es_create(None, ctypes.byref(ctx)) == _binding.ES_ERR_INVALID


def test_binding_constants_match_header():
    """Every integer constant the binding re-exports equals the header's #define, and
    the configuration enums (status, RK, precision, relaxation, boundary) are all there."""
    with open(os.path.join(ROOT, "include", "es.h")) as f:
        defs = dict(re.findall(r"#define\s+(ES_\w+)\s+(-?\d+)\s", f.read()))
    need = [k for k in defs if k.startswith(("ES_OK", "ES_ERR_", "ES_RK_", "ES_FP64", "ES_MIXED",
                                              "ES_RELAX_", "ES_BC_"))]
    assert {"ES_MIXED", "ES_MIXED_FF", "ES_FP64X"} <= set(need)
    for k in need:
        assert getattr(_binding, k) == int(defs[k]), k
