"""The C-ABI library loads without a GPU and exports every entry point include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"SSTEP_API\s+[\w\s\*]+?\b(sstep_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sstep_setup", "sstep_solve", "sstep_solve_batched", "sstep_free",
                     "sstep_mpk", "sstep_block_gram", "sstep_fgs", "sstep_block_update"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2603_09790_gb300 import build, sstep
    build.build()
    lib = ctypes.CDLL(sstep.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # host-only entry points work without a device
    lib.sstep_status_string.restype = ctypes.c_char_p
    assert lib.sstep_status_string(0) == b"ok"


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2603_09790_gb300 import sstep
    monkeypatch.setattr(sstep, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(sstep, "_lib", None)
    with pytest.raises(RuntimeError, match="libsstep.so is missing"):
        sstep.load()


def test_default_opts_from_library():
    from paper_2603_09790_gb300 import build, sstep
    build.build()
    lib = sstep.load()
    o = sstep._Opts()
    lib.sstep_default_opts(ctypes.byref(o))
    assert (o.s, o.sweeps, o.max_outer, o.power_iters) == (4, 2, 10000, 50)
    assert o.rtol == 1e-8 and o.power_tol == 1e-3
