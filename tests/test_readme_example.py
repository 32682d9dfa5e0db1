"""The README's Python example uses only names that exist: it compiles, and
every attribute it takes from the binding, the context, the input generator
and a generated problem is there (the calls themselves need a GPU)."""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def example():
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert len(blocks) == 1
    return blocks[0]


def _attrs(tree, base):
    return {n.attr for n in ast.walk(tree)
            if isinstance(n, ast.Attribute) and isinstance(n.value, ast.Name) and n.value.id == base}


def test_readme_example_names_exist(example):
    from paper_2311_15393_gb300 import build
    build.build()
    from paper_2311_15393_gb300 import kpsvd, synth
    tree = ast.parse(example)
    compile(tree, "README.md", "exec")
    for name in _attrs(tree, "kpsvd"):
        assert hasattr(kpsvd, name), name
    for name in _attrs(tree, "synth"):
        assert hasattr(synth, name), name
    for name in _attrs(tree, "ctx"):
        assert hasattr(kpsvd.KpContext, name), name
    P = synth.make_problem("deblur1024_mixed", n=64)
    for name in _attrs(tree, "P"):
        assert hasattr(P, name), name
    for name in _attrs(tree, "info"):
        assert name in kpsvd.Info.__dataclass_fields__, name
