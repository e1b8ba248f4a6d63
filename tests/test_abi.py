"""The C ABI library builds, loads and exports every entry point that
include/mpcg.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpcg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(mpcg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_2309_08079_gb300 import build
    return build.build()


def test_header_declares_the_path():
    names = _declared()
    for n in ("mpcg_form_schur", "mpcg_form_precon", "mpcg_pcg_solve", "mpcg_recover_step",
              "mpcg_backward", "mpcg_pcg_solve_batched"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_export(lib_path):
    from paper_2309_08079_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()
    lib = _lib.load(lib_path)
    assert lib.mpcg_version().decode().count(".") == 2
    # return codes and status codes have distinct, non-empty messages
    msgs = {c: lib.mpcg_strerror(c).decode() for c in (0, -1, -2, -3, 1, 2, 3, 4, 5)}
    assert len(set(msgs.values())) == len(msgs)


def test_struct_layouts_match_header(lib_path, tmp_path):
    """Every ctypes struct of the binding has the size and field offsets a
    C compiler gives the header's struct."""
    import shutil
    import subprocess
    from paper_2309_08079_gb300 import _lib
    structs = {n: getattr(_lib, n) for n in ("mpcg_dims", "mpcg_lq", "mpcg_schur", "mpcg_opts",
                                             "mpcg_stats", "mpcg_grads", "mpcg_model", "mpcg_lq_out")}
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpcg.h"', "int main(void) {"]
    for n, st in structs.items():
        lines.append(f'printf("{n} size %zu\\n", sizeof({n}));')
        for f, _ in st._fields_:
            lines.append(f'printf("{n} {f} %zu\\n", offsetof({n}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for n, st in structs.items():
        assert got[(n, "size")] == ctypes.sizeof(st), n
        for f, _ in st._fields_:
            assert got[(n, f)] == getattr(st, f).offset, (n, f)


def test_workspace_bytes_is_host_only(lib_path):
    from paper_2309_08079_gb300 import _lib
    lib = _lib.load(lib_path)
    d = _lib.mpcg_dims(14, 7, 512, 0)
    n1 = lib.mpcg_workspace_bytes(d, 1)
    n256 = lib.mpcg_workspace_bytes(d, 256)
    assert n1 >= 2 * 512 * 14 * 4 and n256 > n1
    assert lib.mpcg_workspace_bytes(_lib.mpcg_dims(0, 7, 512, 0), 1) == 0


def test_argument_errors_are_reported_without_a_device(lib_path):
    """Null handles and bad dims are rejected before any CUDA call."""
    from paper_2309_08079_gb300 import _lib
    lib = _lib.load(lib_path)
    d = _lib.mpcg_dims(14, 7, 32, 0)
    assert lib.mpcg_form_schur(None, d, None, None, None) == _lib.MPCG_EINVAL
    assert lib.mpcg_pcg_solve(None, d, None, None, None, None, None) == _lib.MPCG_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    from paper_2309_08079_gb300 import _lib
    saved = _lib._lib
    try:
        _lib._lib = None
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            _lib.load(str(tmp_path / "libmpcg.so"))
    finally:
        _lib._lib = saved
