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
    assert lib.kp_setup(None, None, 8, 8, 4, 4, 0, 0, 1, 0, 0, 0, 1) != 0
    assert lib.kp_create(None, 0, None) != 0


def test_batch_structs_match_the_header(tmp_path):
    """The binding's kp_problem / kp_batch_opts / kp_solve_info layouts equal
    the C compiler's (sizes and field offsets)."""
    import shutil
    import subprocess
    from paper_2311_15393_gb300 import kpsvd
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"kp_problem": (kpsvd.Problem, {"lambda_": "lambda"}), "kp_batch_opts": (kpsvd.BatchOpts, {}),
              "kp_solve_info": (kpsvd.SolveInfo, {})}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "kpsvd.h"', "int main(void) {"]
    for cname, (cls, ren) in fields.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{cname}.{f} %zu\\n", offsetof({cname}, {ren.get(f, f)}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                          check=True).stdout.split("\n") if l)
    for cname, (cls, _) in fields.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(out[f"{cname}.{f}"]) == getattr(cls, f).offset, f"{cname}.{f}"


def test_batch_rejects_bad_arguments_without_gpu(lib):
    assert lib.kp_solve_batch(0, None, 1, None, None) != 0
    assert lib.kp_solve_batch(0, None, -1, None, None) != 0


def test_learned_lambda_entry_points_reject_bad_arguments_without_gpu(lib):
    """Argument checks run before any device call."""
    h = ctypes.c_void_p()
    assert lib.kp_mlp_create(None, 0, None, 256, 3, 64) != 0
    assert lib.kp_mlp_create(ctypes.byref(h), 0, None, 0, 3, 64) != 0      # width
    assert lib.kp_mlp_create(ctypes.byref(h), 0, None, 256, 0, 64) != 0    # depth
    assert lib.kp_mlp_create(ctypes.byref(h), 0, None, 256, 3, 0) != 0     # max_batch
    lib.kp_mlp_param_count.restype = ctypes.c_longlong
    assert lib.kp_mlp_param_count(None) == -1
    assert lib.kp_mlp_set_params(None, None) != 0
    assert lib.kp_mlp_get_params(None, None) != 0
    assert lib.kp_mlp_forward(None, None, 1, None) != 0
    assert lib.kp_mlp_train_step(None, None, None, 1, ctypes.c_float(1e-3), None) != 0
    assert lib.kp_lambda_features(None, None, None) != 0
    lib.kp_mlp_destroy(None)  # NULL is allowed
