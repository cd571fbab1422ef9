"""The C ABI library builds, loads without a GPU, and exports exactly the entry points
include/bamg.h declares (and the binding declares them all)."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bamg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import paper_1004_1451_gb300.build as b

    return b.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("bamg_setup", "bamg_solve", "bamg_free"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (bamg_[a-z0-9_]+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_loads_and_covers_header(libpath):
    from paper_1004_1451_gb300 import _capi

    lib = _capi.load()
    assert set(_capi.SIGNATURES) == set(_declared())
    for n in _declared():
        assert hasattr(lib, n)


def test_default_opts_are_the_papers():
    import ctypes

    from paper_1004_1451_gb300 import _capi

    o = _capi.Opts()
    assert _capi.load().bamg_default_opts(ctypes.byref(o)) == 0
    assert o.omega == 0.7 and o.nu_pre == 2 and o.nu_post == 2 and o.caliber == 2 and o.k_ev == 6
    assert o.cr_theta == 0.85 and o.cr_nu == 8
    from oracle import bamg as ob

    d = ob.Opts()
    for k in ("omega", "nu_tv", "nu_ev", "nu_pre", "nu_post", "caliber", "z", "mmax", "k_ev", "coarse_max", "gmres_m",
              "tv_lo", "tv_hi", "ev_change_tol", "ridge", "weight_floor", "cr_theta", "cr_nu", "cr_omega"):
        assert getattr(o, k) == getattr(d, k), k


def test_struct_layouts_match_header(tmp_path):
    # the ctypes mirrors of the boundary's structs have the C compiler's size and field
    # offsets (a field added on one side only would shift every later field)
    import ctypes

    from paper_1004_1451_gb300 import _capi

    pairs = {"bamg_csr": _capi.Csr, "bamg_mat": _capi.Mat, "bamg_opts": _capi.Opts, "bamg_stats": _capi.Stats,
             "bamg_level_in": _capi.LevelIn}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bamg.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        parts = line.split()
        got[tuple(parts[:-1])] = int(parts[-1])
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)
