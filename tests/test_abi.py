"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol
(no compute calls: these run without a GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_1202_2355_gb300 import binding as B
from paper_1202_2355_gb300 import build as BUILD
from paper_1202_2355_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(m2m_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def so():
    return BUILD.build()


def test_every_declared_symbol_is_exported(so):
    lib = C.CDLL(so)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_last_error_without_context_is_callable(so):
    lib = C.CDLL(so)
    lib.m2m_last_error.restype = C.c_char_p
    lib.m2m_last_error.argtypes = [C.c_void_p]
    assert isinstance(lib.m2m_last_error(None), bytes)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(B, "_SO", str(tmp_path / "absent.so"))
    monkeypatch.setattr(B, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        B.lib()


def test_descriptor_marshalling_counts_observables():
    wl = W.make("c2", n=10, n_target=10)
    d = B.ObsDesc(wl.groups, wl.incl_deg)
    assert d.J == wl.J == 60 + 3 * 30
    assert d.o.n_groups == 2
    assert d.o.groups[1].n_kinds == 3 and list(d.o.groups[1].kinds[:3]) == [1, 13, 14]
    assert d.o.groups[0].edges[60] == pytest.approx(20.0)
    assert [B.kind_code(k) for k in ("mass", "v2", "gh0", "gh6")] == [0, 1, 10, 16]
