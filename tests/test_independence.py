"""The oracle and the CUDA path share no code: the product package (Python binding,
CUDA sources, headers) never mentions the oracle, the oracle never imports the product
package, and the shared input generators import neither."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _sources(folder, exts):
    for dirpath, _, files in os.walk(os.path.join(ROOT, folder)):
        if "__pycache__" in dirpath or "_lib" in os.path.relpath(dirpath, ROOT).split(os.sep):
            continue
        for f in files:
            if f.endswith(exts):
                path = os.path.join(dirpath, f)
                with open(path, encoding="utf-8") as fh:
                    yield os.path.relpath(path, ROOT), fh.read()


def test_product_path_does_not_use_the_oracle():
    py = re.compile(r"^\s*(from|import)\s+(\.\.)?oracle\b|importlib.*oracle|oracle/", re.M)
    inc = re.compile(r"^\s*#\s*include\s*[<\"][^>\"]*oracle", re.M)
    for path, text in _sources("paper_2410_06319_gb300", (".py",)):
        assert not py.search(text), path
    for path, text in list(_sources("paper_2410_06319_gb300", (".cu", ".cuh", ".h"))) + \
            list(_sources("include", (".h",))):
        assert not inc.search(text), path


def test_oracle_and_generators_do_not_import_the_product_path():
    pat = re.compile(r"^\s*(from|import)\s+paper_2410_06319_gb300\b", re.M)
    for folder in ("oracle", "lsq_synth"):
        for path, text in _sources(folder, (".py",)):
            assert not pat.search(text), path
    pat_oracle = re.compile(r"^\s*(from|import)\s+(\.\.)?oracle\b", re.M)
    for path, text in _sources("lsq_synth", (".py",)):
        assert not pat_oracle.search(text), path


def test_binding_fails_loudly_without_the_cuda_library(tmp_path):
    """Without liblsq.so the package does not import: there is no CPU fallback."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2410_06319_gb300"
    pkg.mkdir()
    for f in ("__init__.py", "_lib.py"):
        shutil.copy(os.path.join(ROOT, "paper_2410_06319_gb300", f), pkg / f)
    res = subprocess.run([sys.executable, "-c", "import paper_2410_06319_gb300"], cwd=str(tmp_path),
                         capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert res.returncode != 0
    assert "ImportError" in res.stderr and "no non-CUDA fallback" in res.stderr
