"""C-ABI library: builds for sm_103a, loads without a GPU, and exports every symbol that
include/mto.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mto.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mto_status|const char\*)\s+(mto_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1811_09821_gb300 import _build
    return _build.build()


def test_header_declares_the_four_steps():
    syms = declared_symbols()
    for s in ("mto_build_elements", "mto_solve", "mto_sensitivity", "mto_indicator"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    L = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(L, s)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1811_09821_gb300 as mto
    assert sorted(mto.SYMBOLS) == declared_symbols()


def test_host_structs_match_header(tmp_path):
    """The ctypes mirrors of the option structs have the C compiler's size and field offsets."""
    import shutil
    import subprocess
    import paper_1811_09821_gb300 as mto
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "sizes.c"
    src.write_text("""#include <stdio.h>
#include <stddef.h>
#include "mto.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(mto_material), sizeof(mto_solve_opts), sizeof(mto_indicator_opts),
         offsetof(mto_solve_opts, max_iter), offsetof(mto_indicator_opts, alpha_qr), offsetof(mto_indicator_opts, d_max));
  return 0;
}
""")
    exe = tmp_path / "sizes"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [ctypes.sizeof(mto.Material), ctypes.sizeof(mto.SolveOpts), ctypes.sizeof(mto.IndicatorOpts),
            mto.SolveOpts.max_iter.offset, mto.IndicatorOpts.alpha_qr.offset, mto.IndicatorOpts.d_max.offset]
    assert got == want


def test_binding_fails_loudly_without_the_library(tmp_path):
    """No CPU fallback: loading a missing library raises instead of degrading."""
    import paper_1811_09821_gb300 as mto
    saved = mto._lib
    mto._lib = None
    try:
        with pytest.raises(OSError):
            mto.load_library(str(tmp_path / "libmto_missing.so"))
    finally:
        mto._lib = saved
