"""The C-ABI library loads and exports every function include/dlbchem.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dlbchem.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(dlbchem_[a-z_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2011_07978_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("dlbchem_create", "dlbchem_integrate", "dlbchem_integrate_host", "dlbchem_destroy",
                 "dlbchem_last_error", "dlbchem_nspecies", "dlbchem_options_default"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (dlbchem_[a-z_]+)", out))
    assert set(declared_functions()) <= exported


def test_options_default_and_binding_layout(lib_path):
    from paper_2011_07978_gb300 import dlbchem
    o = dlbchem.options_default()
    assert o.rtol == 1e-6 and o.atol == 1e-10 and o.max_steps == 100000 and o.schedule == dlbchem.SCHED_PLAIN
    assert o.map_Ttol == 1e-4 and o.map_Ytol == 1e-4 and o.chunk == 1
    assert o.gate == 1e-4 and o.predictor == 0 and o.surrogate == 0 and o.precision == 0


def test_binding_struct_layout_matches_the_header(tmp_path):
    """sizeof and every field offset of dlbchem_options, from a C program
    compiled against include/dlbchem.h, equal the ctypes mirror's."""
    from paper_2011_07978_gb300 import dlbchem
    fields = [f for f, _ in dlbchem.dlbchem_options._fields_]
    src = tmp_path / "layout.c"
    body = "".join(f'  printf("%zu\\n", offsetof(dlbchem_options, {f}));\n' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "dlbchem.h"\nint main(void) {\n'
                   '  printf("%zu\\n", sizeof(dlbchem_options));\n' + body + '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)], text=True).split()]
    assert vals[0] == ctypes.sizeof(dlbchem.dlbchem_options)
    for f, off in zip(fields, vals[1:]):
        assert getattr(dlbchem.dlbchem_options, f).offset == off, f


def test_create_rejects_bad_arguments_without_gpu(lib_path):
    from paper_2011_07978_gb300 import dlbchem
    lib = dlbchem.load()
    h = ctypes.c_void_p()
    assert lib.dlbchem_create(b"/nonexistent/mech.bin", None, ctypes.byref(h)) == dlbchem.BAD_MECH
    assert h.value is None
    assert b"cannot read" in lib.dlbchem_last_error(None)
    o = dlbchem.options_default()
    o.rtol = -1.0
    assert lib.dlbchem_create(b"x", ctypes.byref(o), ctypes.byref(h)) == dlbchem.BAD_ARG
    assert lib.dlbchem_nspecies(None) == -1
    lib.dlbchem_destroy(None)


def test_no_cpu_fallback_without_a_gpu(lib_path):
    """Without a CUDA device a valid mechanism still fails to create a context
    (DLBCHEM_CUDA): the library has no CPU path to fall back on."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2011_07978_gb300 import dlbchem
    from synth import states
    lib = dlbchem.load()
    h = ctypes.c_void_p()
    rc = lib.dlbchem_create(states.mech_path(10, 20, 0).encode(), None, ctypes.byref(h))
    assert rc == dlbchem.CUDA and h.value is None
    with pytest.raises(dlbchem.DlbchemError):
        dlbchem.Context(states.mech_path(10, 20, 0))


def test_missing_library_fails_at_import(tmp_path):
    """If the .so is absent the binding raises instead of doing anything else."""
    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2011_07978_gb300 import dlbchem\n"
            "dlbchem.LIB_PATH = %r\n"
            "try:\n    dlbchem.load()\nexcept ImportError as e:\n    print('raised', e)\n") % (
        str(__import__('pathlib').Path(__file__).resolve().parents[1]), str(tmp_path / "absent.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised" in out.stdout and "no CPU fallback" in out.stdout, out.stdout + out.stderr
