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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the size and field offsets of the C
    structures in include/m2m.h (compiled here with gcc), so every call marshals the
    layout the library reads."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [("m2m_potential", B.Potential, ["kind", "G", "q", "scf_n", "scf_lmax", "scf_r", "ups", "eps_ups"]),
             ("m2m_obs_group", B.ObsGroup, ["geometry", "edges", "n_kinds", "kinds", "Vp", "sp"]),
             ("m2m_observables", B.Observables, ["incl_deg", "n_groups", "groups", "Y", "sigY"]),
             ("m2m_prior_grid", B.PriorGrid, ["mode", "Emin", "smoothing", "lambda", "window_E", "window_x"]),
             ("m2m_options", B.Options, ["precision", "dt", "stream", "block", "deposit"]),
             ("m2m_sph_grid", B.SphGrid, ["n_r", "r_min", "r_max"])]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "m2m.h"', "int main(void) {"]
    for cname, _, fields in pairs:
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for cname, cls, fields in pairs:
        assert int(got[cname]) == C.sizeof(cls), cname
        for f in fields:
            pyname = "lam" if f == "lambda" and not hasattr(cls, "lambda") else f
            assert int(got[f"{cname}.{f}"]) == getattr(cls, pyname).offset, (cname, f)
