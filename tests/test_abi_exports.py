"""The C-ABI library builds, loads without a GPU, and exports every function include/spgemm.h declares."""
import ctypes
import os
import re

from helpers import GOLDEN  # noqa: F401  (sets up sys.path through conftest)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "spgemm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:spgemm_status_t|void|const char\s*\*)\s*(spgemm_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("spgemm_plan", "spgemm_symbolic", "spgemm_numeric", "spgemm_summa_blocked", "spgemm_batch",
                 "spgemm_mat_csc", "spgemm_mat_csr", "spgemm_mat_to_dcsc", "spgemm_mat_export"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_1006_2183_gb300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
