"""The oracle and the CUDA path share no code, and the product never reaches the oracle (no GPU).

* No source under the package (CUDA, C, Python) includes, imports or opens
  anything under oracle/, and no oracle source refers to the package.
* The package's Python modules import neither `oracle` nor a CPU fallback.
"""
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
REPO = os.path.dirname(HERE)
PKG = os.path.join(REPO, "paper_1805_00280_gb300")
ORACLE = os.path.join(REPO, "oracle")


def sources(root, exts):
    for d, _, files in os.walk(root):
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_never_touches_the_oracle():
    for p in sources(PKG, (".py", ".cu", ".cuh", ".h", ".c")):
        text = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), p
        assert "n2v_oracle" not in text, p
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*oracle", text), p


def test_oracle_never_touches_the_package():
    for p in sources(ORACLE, (".py", ".c", ".h")):
        text = open(p).read()
        assert not re.search(r"^\s*(import|from)\s+paper_1805_00280_gb300\b", text, re.M), p
        assert not re.search(r"[\"']paper_1805_00280_gb300[/\\]", text), p
        assert not re.search(r"#\s*include\s*[<\"][^>\"]*(n2v\.h|csrc)", text), p
        assert "libn2v" not in text, p


def test_only_allowed_callers_import_the_oracle():
    allowed = {os.path.join(REPO, "bench.py"), os.path.join(REPO, "__graft_entry__.py")}
    for p in sources(REPO, (".py",)):
        rel = os.path.relpath(p, REPO)
        if rel.startswith(("tests" + os.sep, "oracle" + os.sep, "_work" + os.sep, "baseline" + os.sep)):
            continue
        text = open(p).read()
        if re.search(r"^\s*(import|from)\s+oracle\b", text, re.M):
            assert p in allowed, rel
