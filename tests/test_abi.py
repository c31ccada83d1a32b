"""The C-ABI library builds for sm_103a, loads, and exports every function
include/cswdg.h declares (no compute call: runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "cswdg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cswdg_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    from paper_2106_06280_gb300 import build
    build.build()
    from paper_2106_06280_gb300 import cswdg
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(cswdg.lib, n), n
    assert set(names) == set(cswdg.EXPORTED)


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing library is an import error."""
    import importlib.util
    src = os.path.join(ROOT, "paper_2106_06280_gb300", "cswdg.py")
    spec = importlib.util.spec_from_file_location("cswdg_copy", src)
    mod = importlib.util.module_from_spec(spec)
    monkeypatch.setattr(os.path, "exists", lambda p: False if p.endswith("libcswdg.so") else True)
    try:
        spec.loader.exec_module(mod)
    except ImportError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("binding loaded without its library")


def test_mesh_generator_counts():
    from paper_2106_06280_gb300 import workloads as W
    m = W.split_square_mesh(7, 5, 0.0, 1.0, 0.0, 2.0, seed=1, periodic=True)
    assert m.nc == 70 and m.nv == 48 and len(m.bface) == 2 * (7 + 5)
    assert (W.cell_areas(m) > 0).all()
    dm = W.double_mach(960, 240)
    assert dm.mesh.nc == 460800
