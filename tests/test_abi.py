"""The C ABI library builds for sm_103a, loads without a GPU, and exports every
entry point declared in include/romb.h (no compute calls here)."""
import ctypes
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build():
    spec = importlib.util.spec_from_file_location("_romb_build", os.path.join(ROOT, "paper_2604_09113_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()


def test_library_exports_header_symbols():
    lib_path = _build()
    lib = ctypes.CDLL(lib_path)
    header = open(os.path.join(ROOT, "include", "romb.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    names = sorted(set(re.findall(r"\b(romb_[a-z_0-9]+)\s*\(", header)))
    assert "romb_create" in names and "romb_bddc_solve" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_reports_status_strings():
    _build()
    import paper_2604_09113_gb300 as romb
    assert romb._lib.romb_strerror(-4).decode().startswith("threshold")
    # no GPU here: creating a context fails cleanly with a CUDA status
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        try:
            romb.romb_create(0)
        except romb.RombError as e:
            assert e.status == -2


def test_autograd_binding_imports():
    _build()
    torch = pytest.importorskip("torch")
    from paper_2604_09113_gb300.autograd import Compliance, compliance
    assert issubclass(Compliance, torch.autograd.Function) and callable(compliance)


def test_binding_structs_match_the_header(tmp_path):
    # the ctypes structures of the binding against the C compiler's layout of
    # romb_lattice and romb_train_spec (size and every field offset)
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    _build()
    import paper_2604_09113_gb300 as romb
    structs = {"romb_lattice": romb.RombLattice, "romb_train_spec": romb.RombTrainSpec}
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "romb.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, what, val = line.split()
            got[(cname, what)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
