"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared symbol."""
import ctypes

import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_builder():
    path = os.path.join(ROOT, "paper_2410_06319_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("lsq_build", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def lsq():
    load_builder().build()
    import paper_2410_06319_gb300 as lsq
    return lsq


def test_every_declared_function_is_exported(lsq):
    names = lsq.declared_functions()
    for required in ("lsq_sketch", "lsq_qr_r", "lsq_lsqr", "lsq_lsir", "lsq_create", "lsq_destroy",
                     "lsq_omega"):
        assert required in names
    for name in names:
        assert hasattr(lsq.lib, name), name


def test_struct_layouts_match_header(lsq):
    assert lsq.lib.lsq_sizeof(0) == ctypes.sizeof(lsq.Opts)
    assert lsq.lib.lsq_sizeof(1) == ctypes.sizeof(lsq.Info)
    assert lsq.lib.lsq_sizeof(7) == 0


def test_status_strings(lsq):
    for code, name in lsq.STATUS.items():
        assert lsq.lib.lsq_status_string(code).decode() == name


def test_invalid_arguments_are_rejected_before_any_launch(lsq):
    # a NULL handle is rejected without touching CUDA
    args = [None, 1, 1, 100, 10, 40, 0, 1, 1, 0, 1e-6, 0, None, 1]
    assert lsq.lib.lsq_sketch(*args) == -1
    assert lsq.lib.lsq_omega(None, 4, 0, 4, 0, 0, 1) == -1


def test_struct_field_offsets_match_header(lsq, tmp_path):
    """Field by field: a C program compiled against include/lsq.h prints the offset of every
    field the binding declares, and each equals the ctypes offset (a reordering or a type
    change in either place fails here even where the sizes still agree)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "lsq.h"', 'int main(void) {']
    want = []
    for cname, cls in (("lsq_opts", lsq.Opts), ("lsq_info", lsq.Info)):
        for fname, _ in cls._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            want.append(getattr(cls, fname).offset)
    lines += ['  return 0;', '}']
    src = tmp_path / "offsets.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "offsets"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == want
