"""The oracle and the CUDA path share no code: the package never imports the
oracle, the oracle never imports the package or includes the library's
sources, and the input generators hold no import of either.  CPU only."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(folder, exts):
    out = []
    for ext in exts:
        out += glob.glob(os.path.join(ROOT, folder, "**", "*" + ext), recursive=True)
    return out


def test_package_does_not_import_the_oracle():
    for path in _sources("paper_2305_04966_gb300", (".py", ".cu", ".cuh")):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), path
        assert "oracle.c" not in src and "liboracle" not in src, path


def test_oracle_does_not_use_the_package_or_its_sources():
    for path in _sources("oracle", (".py", ".c", ".h")):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+paper_2305_04966_gb300\b", src, flags=re.M), path
        assert not re.search(r'#\s*include\s*[<"](nacc|.*\.cuh)', src), path
        assert "libnacc" not in src, path


def test_input_generators_import_neither_side():
    for path in _sources("workloads", (".py",)):
        src = open(path).read()
        assert not re.search(r"^\s*(import|from)\s+(oracle|paper_2305_04966_gb300)\b", src, flags=re.M), path
