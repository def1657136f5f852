"""The boundary between the product and the oracle, checked without a GPU.

* The library package never imports the oracle, and the oracle never imports the library (the
  two share only the seeded input generator, which holds no tensor-train arithmetic); no CUDA
  source includes anything from oracle/.
* The product path has no CPU fallback: a missing libtt.so raises, and host (CPU) tensors are
  rejected before any call reaches the library.
"""
import ast
import glob
import os
import re

import pytest

from paper_2602_20226_gb300 import _abi, inputs, qtt
import paper_2602_20226_gb300 as tt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _imported_modules(path):
    tree = ast.parse(open(path).read())
    out = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            out.add(node.module.split(".")[0])
    return out


def test_library_and_oracle_do_not_import_each_other():
    pkg = glob.glob(os.path.join(ROOT, "paper_2602_20226_gb300", "**", "*.py"), recursive=True)
    assert pkg
    for p in pkg:
        assert "oracle" not in _imported_modules(p), p
    orc = glob.glob(os.path.join(ROOT, "oracle", "*.py"))
    assert orc
    for p in orc:
        assert "paper_2602_20226_gb300" not in _imported_modules(p), p
    inc = re.compile(r'#\s*include\s*[<"]([^>"]+)[>"]')
    for p in glob.glob(os.path.join(ROOT, "paper_2602_20226_gb300", "csrc", "*")):
        for name in inc.findall(open(p).read()):
            assert "oracle" not in name, (p, name)


def test_input_generator_holds_no_tensor_train_arithmetic():
    """inputs.py (shared by both sides) imports nothing from either side."""
    mods = _imported_modules(os.path.join(ROOT, "paper_2602_20226_gb300", "inputs.py"))
    assert "oracle" not in mods
    assert not any(m.startswith("paper_2602_20226_gb300") for m in mods)


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        _abi.load(os.path.join(ROOT, "no_such_dir", "libtt.so"))


@pytest.fixture(scope="module")
def built_library():
    if not os.path.exists(_abi.LIB_PATH):
        from paper_2602_20226_gb300 import build

        build.build()


@pytest.mark.parametrize("op", ["apply", "hadamard", "round", "inner"])
def test_host_tensors_are_rejected(built_library, op):
    x = tt.TT.from_numpy(inputs.random_tt(1, 6, 2, 3), device="cpu")
    w = tt.MPO.from_numpy(qtt.second_difference_mpo(6), device="cpu")
    call = {"apply": lambda: tt.tt_apply_mpo(w, x), "hadamard": lambda: tt.tt_hadamard(x, x),
            "round": lambda: tt.tt_round(x, 1e-8), "inner": lambda: tt.tt_inner(x, x)}[op]
    with pytest.raises(ValueError, match="CUDA"):
        call()
