"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import glob
import os
import re

from paper_1907_12874_gb300 import bicgk, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(bicgk_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("bicgk_csr_create", "bicgk_solve", "bicgk_spmm", "bicgk_op_destroy", "bicgk_strerror"):
        assert f in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), name


def test_host_only_calls_work_without_gpu():
    lib = bicgk._load()
    assert bicgk.version().startswith("bicgk")
    assert bicgk.strerror(-2) == "malformed CSR matrix"
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    assert lib.bicgk_csr_create(ctypes.byref(h), 0, 0, None, None, None, 0, None) == -1
    assert lib.bicgk_solve(None, 1, None, None, 1e-8, 10, 1, 0, 0, None, None, None, None, None, None) == -1
    assert lib.bicgk_op_destroy(None) == 0


def test_binding_has_no_cpu_fallback():
    """The binding calls the library for every solve; it has no numpy/torch solver path."""
    src = open(os.path.join(ROOT, "paper_1907_12874_gb300", "bicgk.py")).read()
    assert "oracle" not in src and "np.linalg" not in src and "torch.linalg" not in src


def _header_enum(prefix):
    text = open(os.path.join(ROOT, "include", "bicgk.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]+)\s*=\s*(\d+)", text)}


def test_binding_constants_match_the_header():
    """The binding's option, flag, memory-space and form numbers are the header's."""
    opts = _header_enum("BICGK_OPT_")
    assert opts, "no options declared"
    for name, value in opts.items():
        assert getattr(bicgk, name[len("BICGK_"):]) == value, name
    assert bicgk.FLAG_NO_STOP_TEST == _header_enum("BICGK_FLAG_")["BICGK_FLAG_NO_STOP_TEST"]
    assert bicgk.FLAG_JACOBI == _header_enum("BICGK_FLAG_")["BICGK_FLAG_JACOBI"]
    for name, value in _header_enum("BICGK_BATCH_").items():
        assert getattr(bicgk, name[len("BICGK_"):]) == value, name
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "bicgk.h")).read(), flags=re.S)
    assert bicgk.E_TIMEOUT == int(re.search(r"BICGK_E_TIMEOUT\s*=\s*(-\d+)", text).group(1))
    forms = {k: v for k, v in _header_enum("BICGK_").items()
             if k.endswith(("_PLAIN", "_MERGED"))}
    assert len(forms) == 12
    for name, value in forms.items():
        assert bicgk.VARIANTS[name[len("BICGK_"):].lower()] == value, name
