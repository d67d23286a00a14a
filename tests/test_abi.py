"""The C-ABI library builds for sm_103a, loads, and exports every function include/stmg.h
declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

from tests.helpers import build_and_load

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(stmg_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_function():
    lib = build_and_load()
    names = declared_functions()
    assert "stmg_apply" in names and "stmg_create" in names
    for name in names:
        assert hasattr(lib, name), name


def test_param_defaults_follow_the_paper():
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    p = stmg.default_params()
    assert (p.gamma1, p.gamma2) == (10.0, 10.0)
    assert (p.newton_rtol, p.newton_atol) == (1e-8, 1e-12)
    assert (p.ls_lambda0, p.ls_c, p.ls_tau, p.ls_alpha_min, p.ls_maxbt, p.ls_window) == (1.0, 1e-4, 0.5, 1e-3, 5, 5)
    assert (p.ew_eta0, p.ew_c, p.ew_theta, p.ew_min, p.ew_max) == (0.4, 0.5, 1.5, 1e-3, 0.8)
    assert (p.gmres_maxit, p.nu1, p.nu2) == (50, 1, 1)


def test_binding_rejects_missing_library(monkeypatch, tmp_path):
    from paper_2602_13841_gb300 import stmg
    monkeypatch.setattr(stmg, "_lib", None)
    monkeypatch.setattr(stmg, "LIBPATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError):
        stmg.load()


def test_footprint_follows_the_hierarchy_option():
    """stmg_footprint (host arithmetic, no allocation): with DG(k) kept on the coarse levels
    (keep_time_degree = 1) the levels below the finest carry k + 1 instead of k/2 + 1 time nodes,
    so the footprint grows; for k = 1 (nothing to coarsen in time) it is unchanged."""
    from paper_2602_13841_gb300 import stmg
    build_and_load()
    fp = lambda **kw: stmg.footprint(stmg.default_params(**dict(dict(dim=2, n_cells_1d=64, r=2), **kw)))
    assert fp(k=2, keep_time_degree=1) > fp(k=2, keep_time_degree=0)
    assert fp(k=1, keep_time_degree=1) == fp(k=1, keep_time_degree=0)
    assert fp(k=2, problem="CAV3D", dim=3, n_cells_1d=8) > 0


def _c_layout(tmp_path, ctype, fields):
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "stmg.h"', "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % ctype]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (ctype, f) for f in fields]
    lines += ["  return 0;", "}"]
    src = tmp_path / (ctype + ".c")
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / ctype
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]


@pytest.mark.parametrize("ctype,pyname", [("stmg_params", "Params"), ("stmg_stats", "Stats")])
def test_struct_layout_matches_the_header(tmp_path, ctype, pyname):
    """The ctypes mirrors of the ABI structs have the C structs' sizes and field offsets (compiled
    with the host C compiler from include/stmg.h)."""
    from paper_2602_13841_gb300 import stmg
    cls = getattr(stmg, pyname)
    fields = [f for f, _ in cls._fields_]
    out = _c_layout(tmp_path, ctype, fields)
    assert out[0] == ctypes.sizeof(cls)
    for f, off in zip(fields, out[1:]):
        assert getattr(cls, f).offset == off, f
