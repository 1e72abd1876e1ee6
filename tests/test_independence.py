"""The oracle and the GPU library stay independent of each other.

The parity tests are only worth something if the two sides share no code:
the product package must never import the oracle (no CPU fallback can hide
behind it), the oracle must never import the product, and the seeded input
generators that both sides use import neither.  These checks read the
sources only, so they run without a GPU.
"""

import ast
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2608_03473_gb300")
ORACLE = os.path.join(ROOT, "oracle")
INPUTS = os.path.join(ROOT, "lexinputs")


def _py_files(d):
    return sorted(os.path.join(d, f) for f in os.listdir(d) if f.endswith(".py"))


def _c_files(d):
    return sorted(os.path.join(d, f) for f in os.listdir(d)
                  if f.endswith((".c", ".h", ".cu", ".cuh", ".cpp")))


def _imported_roots(path):
    tree = ast.parse(open(path).read(), filename=path)
    roots = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            roots.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            roots.add(node.module.split(".")[0])
    return roots


def _includes(path):
    return re.findall(r'^\s*#\s*include\s*[<"]([^">]+)[">]', open(path).read(), flags=re.M)


def test_product_never_imports_the_oracle():
    for f in _py_files(PKG):
        assert "oracle" not in _imported_roots(f), f


def test_oracle_never_imports_the_product():
    for f in _py_files(ORACLE):
        assert "paper_2608_03473_gb300" not in _imported_roots(f), f


def test_input_generators_import_neither_side():
    for f in _py_files(INPUTS):
        roots = _imported_roots(f)
        assert "oracle" not in roots and "paper_2608_03473_gb300" not in roots, f


def test_native_sources_share_no_header():
    product = {os.path.basename(f) for f in _c_files(os.path.join(PKG, "csrc"))}
    product |= {f for f in os.listdir(os.path.join(ROOT, "include"))}
    oracle_files = {os.path.basename(f) for f in _c_files(ORACLE)}
    for f in _c_files(ORACLE):
        for inc in _includes(f):
            assert os.path.basename(inc) not in product, (f, inc)
    for f in _c_files(os.path.join(PKG, "csrc")):
        for inc in _includes(f):
            assert os.path.basename(inc) not in oracle_files, (f, inc)
