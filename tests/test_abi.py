"""The C-ABI library loads and exports every function that include/*.h declares (no GPU calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2311_06926_gb300", "libstokes_hp.so")


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(stokes_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["stokes_setup", "stokes_apply_A", "stokes_apply_K", "stokes_apply_P",
                     "stokes_apply_hyperpower", "stokes_solve", "stokes_destroy"]:
        assert required in names


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(LIB)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.skipif(not os.path.exists(LIB), reason="library not built")
def test_setup_rejects_bad_arguments_without_touching_the_gpu():
    """Argument checks happen before any CUDA call."""
    from paper_2311_06926_gb300.binding import load_library, _Opts
    lib = load_library()
    h = ctypes.c_void_p()
    assert lib.stokes_setup(ctypes.byref(h), 0, 2, 1.0, None) == -1
    assert lib.stokes_setup(ctypes.byref(h), 4, 0, 1.0, None) == -1
    assert lib.stokes_setup(ctypes.byref(h), 4, 2, -1.0, None) == -1
    o = _Opts()
    lib.stokes_default_opts(ctypes.byref(o))
    assert o.c_pen == 14.0 and o.max_order == 3 and o.max_steps == 4
    o.precision = 3          # reduced precision with MINRES is refused
    assert lib.stokes_setup(ctypes.byref(h), 4, 2, 1.0, ctypes.byref(o)) == -1
    assert b"MINRES" in lib.stokes_last_error(None)
    assert lib.stokes_apply_K(None, None, None) == -1


def _c_layout(struct, fields):
    """sizeof and field offsets of a struct of include/stokes_hp.h, from a C program built with
    the host compiler (the header is plain C)."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    body = "\n".join(f'  printf("%zu\\n", offsetof({struct}, {f}));' for f in fields)
    src = (f'#include <stddef.h>\n#include <stdio.h>\n#include "stokes_hp.h"\n'
           f'int main(void) {{\n  printf("%zu\\n", sizeof({struct}));\n{body}\n  return 0;\n}}\n')
    with tempfile.TemporaryDirectory() as d:
        c_file, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(c_file, "w").write(src)
        subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        c_file, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    return [int(v) for v in out]


@pytest.mark.parametrize("struct,cls", [("stokes_opts", "_Opts"), ("stokes_tuning", "_Tuning"),
                                        ("stokes_kernel_stat", "KernelStat")])
def test_binding_structs_match_the_header(struct, cls):
    """The ctypes mirrors of the header's structs have the C sizes and field offsets."""
    import paper_2311_06926_gb300.binding as b
    py = getattr(b, cls)
    names = [f[0] for f in py._fields_]
    size, *offsets = _c_layout(struct, names)
    assert size == ctypes.sizeof(py)
    assert offsets == [getattr(py, n).offset for n in names]
