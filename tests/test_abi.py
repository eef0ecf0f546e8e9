"""The C-ABI library builds, loads and exports every function the headers declare."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\**\s*\b(fmm_[A-Za-z0-9_]+)\s*\(", txt, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_header_symbols():
    import ctypes

    from paper_1712_07739_gb300 import build as b
    import paper_1712_07739_gb300 as gb

    b.build()
    names = _declared()
    assert len(names) >= 11, names
    lib = ctypes.CDLL(gb.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(gb.EXPORTS) <= set(names)


def test_missing_library_fails_loudly(tmp_path):
    import paper_1712_07739_gb300 as gb

    with pytest.raises(gb.GbfmmError):
        gb._lib_saved = gb._lib
        gb._lib = None
        try:
            gb.load_library(str(tmp_path / "nope.so"))
        finally:
            gb._lib = gb._lib_saved


def test_options_layout_matches_header(tmp_path):
    """The ctypes mirror of gbfmm_options has the header's size and field
    offsets (a C program compiled against include/gbfmm.h prints them)."""
    import ctypes
    import shutil
    import subprocess

    import paper_1712_07739_gb300 as gb

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = [f[0] for f in gb.Options._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gbfmm.h"', "int main(void) {",
             '  printf("%zu\\n", sizeof(gbfmm_options));']
    lines += [f'  printf("%zu\\n", offsetof(gbfmm_options, {n}));' for n in names]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert vals[0] == ctypes.sizeof(gb.Options)
    assert vals[1:] == [getattr(gb.Options, n).offset for n in names]
