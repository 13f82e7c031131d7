"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2603_03150_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(?:pdhg_status|void|const char\s*\*)\s*\**\s*(pdhg_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_boundary():
    d = declared()
    for must in ["pdhg_create", "pdhg_solve", "pdhg_get", "pdhg_warmstart_point", "pdhg_destroy"]:
        assert must in d


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_declared_symbols(libpath):
    from paper_2603_03150_gb300 import pdhg
    L = pdhg.lib()
    for n in pdhg.declared_symbols():
        assert hasattr(L, n), n


def test_default_options_without_gpu(libpath):
    from paper_2603_03150_gb300 import pdhg
    o = pdhg.Options()
    pdhg.lib().pdhg_default_options(ctypes.byref(o))
    assert o.eval_freq == 64 and o.ruiz_iters == 10 and abs(o.eta_safety - 0.95) < 1e-15
    assert o.precision == 0 and o.use_graphs == 1


def test_header_is_plain_c(tmp_path):
    """include/pdhg.h compiles as C99 (no C++ in the boundary) and every
    declared entry point can be referenced from C."""
    gcc = "gcc"
    import shutil
    import subprocess
    if shutil.which(gcc) is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi_check.c"
    refs = "\n".join(f"  (pdhg_fn)&{n}," for n in declared())
    src.write_text('#include "pdhg.h"\n'
                   "typedef void (*pdhg_fn)(void);\n"
                   "pdhg_fn pdhg_abi_refs[] = {\n" + refs + "\n};\n"
                   "int main(void) { pdhg_options o; pdhg_default_options(&o); return (int)o.eval_freq == 0; }\n")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-c", str(src),
                        "-I", os.path.join(ROOT, "include"), "-o", str(tmp_path / "abi_check.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_options_struct_matches_the_header(tmp_path):
    """The ctypes mirror of pdhg_options has the C struct's size and every
    field at the C offset (a field added to one and not the other fails)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2603_03150_gb300 import pdhg
    names = [f[0] for f in pdhg.Options._fields_]
    lines = "\n".join(f'  printf("{n} %zu\\n", offsetof(pdhg_options, {n}));' for n in names)
    src = tmp_path / "opt_layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "pdhg.h"\n'
                   "int main(void) {\n" + lines +
                   '\n  printf("sizeof %zu\\n", sizeof(pdhg_options));\n  return 0;\n}\n')
    exe = tmp_path / "opt_layout"
    r = subprocess.run(["gcc", "-std=c99", str(src), "-I", os.path.join(ROOT, "include"),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for n in names:
        assert int(got[n]) == getattr(pdhg.Options, n).offset, n
    assert int(got["sizeof"]) == ctypes.sizeof(pdhg.Options)


def test_default_layout_options(libpath):
    from paper_2603_03150_gb300 import pdhg
    o = pdhg.Options()
    pdhg.lib().pdhg_default_options(ctypes.byref(o))
    assert o.spmv_layout == 0 and o.panel_width == 0 and o.method == 0
