"""The oracle and the CUDA path are independent, and the product path has no
fallback: a static check of the sources (CPU only).

* nothing in the package (Python or CUDA) imports, includes, loads or names
  a file of the oracle, and nothing in the oracle imports or includes the
  package;
* the only module the two share is the seeded input generator, and it holds
  none of the method's arithmetic (no Philox rounds of the sampler's noise,
  no Tweedie factor, no update);
* in bench.py the oracle is imported only by the CPU-baseline and reference
  legs;
* the binding refuses to run without the built library instead of computing
  anything itself.
"""
import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1506_01418_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(d, exts):
    out = []
    for base, _, names in os.walk(d):
        if "__pycache__" in base:
            continue
        out += [os.path.join(base, n) for n in names if n.endswith(exts)]
    return sorted(out)


def _imports(path):
    tree = ast.parse(open(path).read(), path)
    mods = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            mods |= {a.name.split(".")[0] for a in node.names}
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            mods.add(node.module.split(".")[0])
    return mods


def test_package_never_touches_the_oracle():
    for f in _files(PKG, (".py",)):
        assert "oracle" not in _imports(f), f
        src = open(f).read()
        assert "psgld_oracle" not in src and "liboracle" not in src, f
    for f in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        src = open(f).read()
        assert not re.search(r'#\s*include\s*[<"][^>"]*oracle', src), f
        assert "or_part_step" not in src and "or_drift" not in src, f


def test_oracle_never_touches_the_package():
    for f in _files(ORACLE, (".py",)):
        mods = _imports(f)
        assert "paper_1506_01418_gb300" not in mods and "torch" not in mods, (f, mods)
    for f in _files(ORACLE, (".c", ".h")):
        src = open(f).read()
        includes = re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', src)
        assert all(i in {"psgld_oracle.h", "stdint.h", "stddef.h", "stdlib.h", "string.h", "math.h",
                         "omp.h"} for i in includes), (f, includes)


def test_shared_input_generator_holds_no_method_arithmetic():
    src = open(os.path.join(PKG, "datagen.py")).read()
    assert _imports(os.path.join(PKG, "datagen.py")) <= {"__future__", "numpy", "torch", "math"}
    # (numpy's own Philox bit generator seeds the inputs; the method's
    # counter-based stream, with its round constants, lives on each side)
    for word in ("0xD2511F53", "0xCD9E8D57", "0x9E3779B9", "box_muller", "tweedie", "mirror",
                 "langevin", "sqrt(2", "beta_div"):
        assert word.lower() not in src.lower(), word


def test_bench_imports_the_oracle_only_in_its_cpu_legs():
    path = os.path.join(ROOT, "bench.py")
    tree = ast.parse(open(path).read(), path)
    allowed = {"oracle_setup", "cpu_baseline", "cpu_baseline_block", "batched_cpu_baseline",
               "run_reference"}
    users = set()
    for fn in ast.walk(tree):
        if isinstance(fn, ast.FunctionDef):
            for node in ast.walk(fn):
                if isinstance(node, ast.Import) and any(a.name == "oracle" for a in node.names):
                    users.add(fn.name)
    assert users and users <= allowed, users
    # no module-level import of the oracle
    top = [n for n in tree.body if isinstance(n, (ast.Import, ast.ImportFrom))]
    assert all("oracle" not in {a.name for a in n.names} for n in top if isinstance(n, ast.Import))


def test_binding_refuses_to_run_without_the_library(monkeypatch, tmp_path):
    from paper_1506_01418_gb300 import _build
    from paper_1506_01418_gb300 import psgld as P
    monkeypatch.setattr(P, "_lib", None)
    monkeypatch.setattr(_build, "LIB", str(tmp_path / "missing" / "libpsgld.so"))
    with pytest.raises(OSError):
        P.load(build_if_missing=False)
