"""The oracle and the GPU path share no code: neither package imports the other,
and neither's C/CUDA sources include the other's files."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1808_04580_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    out = []
    for d, dirs, files in os.walk(top):
        dirs[:] = [x for x in dirs if not x.startswith(("_build", "__pycache__"))]
        out += [os.path.join(d, f) for f in files if f.endswith(exts)]
    return out


def test_product_path_never_imports_the_oracle():
    for f in _files(PKG, (".py",)):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f


def test_oracle_never_imports_the_product_path():
    for f in _files(ORACLE, (".py",)):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+paper_1808_04580_gb300\b", text, re.M), f
        assert "libnfl" not in text, f          # nor loads the product's library


def test_sources_include_nothing_across():
    for f in _files(PKG, (".cu", ".cuh", ".h", ".cpp")):
        assert "oracle" not in "".join(re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read())), f
    for f in _files(ORACLE, (".c", ".h")):
        inc = re.findall(r'#include\s*[<"]([^>"]+)[>"]', open(f).read())
        assert not any("nfl" in i or "csrc" in i for i in inc), f
