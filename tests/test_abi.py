"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/kpsvd.h declares; status strings exist."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2311_15393_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kpsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w \t\*]*?\b([a-z_]\w*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


def test_header_declares_the_abi():
    names = declared_functions()
    for must in ["kp_create", "kp_setup", "tik_pcg", "choose_lambda", "kp_apply_A", "kp_apply_Minv", "kp_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libkpsvd.so does not export {name}"


def test_binding_lists_every_export():
    from paper_2311_15393_gb300 import kpsvd
    assert sorted(kpsvd.EXPORTS) == declared_functions()


def test_status_strings(lib):
    lib.kp_status_str.restype = ctypes.c_char_p
    for s in range(11):
        assert lib.kp_status_str(s)
    lib.kp_last_error.restype = ctypes.c_char_p
    assert lib.kp_last_error() is not None


def test_null_context_is_rejected_without_gpu(lib):
    # argument validation runs before any device call
    assert lib.tik_pcg(None, None, ctypes.c_double(0.1), ctypes.c_double(1e-6), 10, 0, None, 0, None) != 0
    assert lib.kp_setup(None, None, 8, 8, 4, 4, 0, 0, 0, 0, 0, 1) != 0
    assert lib.kp_create(None, 0, None) != 0
