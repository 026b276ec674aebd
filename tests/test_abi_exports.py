"""CPU checks of the C ABI boundary: the library builds, loads and exports every
function declared in include/*.h (no compute call: no GPU here)."""
import ctypes
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
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*"
                             r"([A-Za-z_][A-Za-z0-9_]*)\s*\(", txt, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_core_entry_points():
    d = _declared()
    for n in ("spgemm_symbolic", "spgemm_numeric", "spgemm_workspace_size",
              "spgemm_transpose"):
        assert n in d


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as g
    g.build()
    from paper_2504_06408_gb300 import spgemm as api
    for path in (api.LIB_PATH, api.CHECKS_LIB_PATH):   # the library and its checked build
        lib = ctypes.CDLL(path)
        missing = [n for n in _declared() if not hasattr(lib, n)]
        assert not missing, (path, missing)
    # the Python binding covers every declared function
    assert set(_declared()) <= set(api.exported_symbols())


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2504_06408_gb300 import spgemm as api
    with pytest.raises(RuntimeError):
        api.load_library(str(tmp_path / "missing.so"))


def test_argument_errors_are_synchronous():
    """Argument checks run on the host: a NULL handle / bad id is refused before any
    CUDA call (these calls need no GPU)."""
    import __graft_entry__ as g
    g.build()
    from paper_2504_06408_gb300 import spgemm as api
    lib = api.load_library()
    n = ctypes.c_size_t()
    a = api.spg_csr(4, 5, 0, None, None, None)
    assert lib.spgemm_workspace_size(None, 0, ctypes.byref(a), ctypes.byref(a),
                                     ctypes.byref(n)) == 1
