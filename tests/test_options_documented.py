"""Every option name kp_set_option accepts is documented in the C header (no
option exists only in code)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _accepted():
    src = open(os.path.join(ROOT, "paper_2311_15393_gb300", "csrc", "kp_api.cu")).read()
    body = src[src.index("kp_set_option("):]
    return re.findall(r'strcmp\(name, "([a-z0-9_]+)"\)', body)


def test_every_option_is_documented_in_the_header():
    names = _accepted()
    assert len(names) >= 20
    hdr = open(os.path.join(ROOT, "include", "kpsvd.h")).read()
    missing = [n for n in names if f'"{n}"' not in hdr]
    assert not missing, f"options without a header entry: {missing}"


def test_option_names_are_unique():
    names = _accepted()
    assert len(names) == len(set(names))
