"""The C-ABI library loads and exports every entry point that
include/*.h declares (CPU only: no compute call is made)."""

import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

from tests.conftest import ROOT


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            name = m.group(1)
            start = text.rfind("\n", 0, m.start()) + 1
            line = text[start:m.start()]
            if line.strip().startswith("#") or "typedef" in line:
                continue
            if re.search(r"\b(int|void|const char\s*\*|char\s*\*)\s*$", line.strip() + " ") or \
               re.match(r"^\s*(int|const char\s*\*|void)\s+$", line):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2010_03660_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("stencil7_create", "stencil7_destroy", "stencil7_apply", "bicgstab_solve",
              "bicgstab_solve_refined", "stencil7_residual", "s7_last_error"):
        assert n in names, n


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), "missing export %s" % name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(declared_functions()) <= exported


def test_binding_names_match_header():
    import paper_2010_03660_gb300 as s7
    assert set(s7.EXPORTS) == set(declared_functions())
    for name in s7.EXPORTS:
        assert callable(getattr(s7, name))


def test_version_and_error_text_without_gpu(libpath):
    import paper_2010_03660_gb300 as s7
    assert "sm_103a" in s7.s7_version()
    assert isinstance(s7.s7_last_error(), str)


def test_invalid_arguments_are_rejected_without_gpu(libpath):
    import paper_2010_03660_gb300 as s7
    lib = s7.lib()
    h = ctypes.c_void_p()
    # NULL coefficient struct and bad sizes fail before any CUDA call
    assert lib.stencil7_create(ctypes.byref(h), 4, 4, 4, None, None) == s7.EINVAL
    cs = s7.s7_coeffs()
    assert lib.stencil7_create(ctypes.byref(h), 0, 4, 4, ctypes.byref(cs), None) == s7.EINVAL
    assert "sizes" in s7.s7_last_error()
    assert lib.stencil7_apply(None, None, None, 1, None) == s7.EINVAL
    assert lib.bicgstab_solve(None, None, None, 1, 1e-6, 10, None, None, None, None) == s7.EINVAL


def test_product_path_has_no_oracle_dependency():
    # the package and its sources never import or name the oracle
    pkg = os.path.join(ROOT, "paper_2010_03660_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path


def test_binding_rejects_mismatched_vectors_without_gpu():
    """The entry points take one element type for all vectors of a call and
    no sizes: the binding refuses vectors of mixed types or of the wrong
    length before anything reaches the library."""
    import paper_2010_03660_gb300 as s7
    op = s7.Operator(0, 4, 3, 2, s7.S7_F32)
    b32 = np.zeros(24, np.float32)
    x64 = np.zeros(24)
    short = np.zeros(23, np.float32)
    calls = [lambda: s7.bicgstab_solve(op, b32, x64),
             lambda: s7.bicgstab_solve(op, b32, short),
             lambda: s7.stencil7_residual(op, b32, x64),
             lambda: s7.stencil7_residual_noalloc(op, b32, b32, x64),
             lambda: s7.stencil7_apply(op, short),
             lambda: s7.stencil7_apply(op, b32, x64),
             lambda: s7.bicgstab_solve_refined(op, b32, b32.copy()),
             lambda: s7.bicgstab_solve_batched([op], [b32], [x64]),
             lambda: s7.bicgstab_solve_batched([op, op], [b32], [b32]),
             lambda: s7.s7_server_submit(None, 4, 3, 2, {k: b32 for k in ("diag",) + s7.DIRS},
                                         b32, x64, 1e-6)]
    for call in calls:
        with pytest.raises(ValueError):
            call()
