"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mcrt.h; host-side validation answers without a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_1810_00188_gb300 import build, mcrt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mcrt_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = C.CDLL(path)
    names = declared_entry_points()
    assert {"mcrt_create", "mcrt_set_kdist", "mcrt_set_fields", "mcrt_solve_qrad",
            "mcrt_destroy"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
    assert set(mcrt.EXPORTS) <= set(names)


def test_status_strings_and_null_handling():
    L = mcrt.load()
    assert mcrt.mcrt_status_string(0) == "ok"
    assert "range" in mcrt.mcrt_status_string(mcrt.MCRT_E_RANGE)
    assert L.mcrt_destroy(None) == mcrt.MCRT_OK
    out = C.c_void_p()
    assert L.mcrt_create(None, C.byref(out)) == mcrt.MCRT_E_ARG
    assert L.mcrt_set_kdist(None, None) == mcrt.MCRT_E_ARG
    assert L.mcrt_set_fields(None, None, None, 1, 0, None) == mcrt.MCRT_E_ARG
    assert L.mcrt_solve_qrad(None, None, None, None, 0, None) == mcrt.MCRT_E_ARG
    assert L.mcrt_get_stats(None, None) == mcrt.MCRT_E_ARG


def _grid(**kw):
    g = mcrt.mcrt_grid_desc()
    g.nx, g.ny, g.nz, g.lx, g.ly, g.lz = 4, 4, 4, 1.0, 1.0, 1.0
    g.eps_wall[0] = g.eps_wall[1] = 1.0
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ly=-1.0), dict(reflect=3), dict(device=-1),
                                 dict(nx=1 << 11, ny=1 << 11, nz=1 << 10)])
def test_create_rejects_bad_geometry(bad):
    out = C.c_void_p()
    rc = mcrt.load().mcrt_create(C.byref(_grid(**bad)), C.byref(out))
    assert rc in (mcrt.MCRT_E_ARG, mcrt.MCRT_E_CUDA)
    if "device" not in bad:
        assert rc == mcrt.MCRT_E_ARG
    assert not out.value


def test_create_bad_wall_emissivity():
    g = _grid()
    g.eps_wall[0] = 1.5
    out = C.c_void_p()
    assert mcrt.load().mcrt_create(C.byref(g), C.byref(out)) == mcrt.MCRT_E_ARG


def test_create_without_gpu_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    out = C.c_void_p()
    assert mcrt.load().mcrt_create(C.byref(_grid()), C.byref(out)) == mcrt.MCRT_E_CUDA
    with pytest.raises(mcrt.McrtError):
        mcrt.mcrt_create(_grid())


def test_probes_validate_arguments_before_touching_a_device():
    L = mcrt.load()
    r, m = C.c_double(), C.c_double()
    assert L.mcrt_probe_ex2(0, None, C.byref(m)) == mcrt.MCRT_E_ARG
    assert L.mcrt_probe_ex2(0, C.byref(r), None) == mcrt.MCRT_E_ARG
    for nbytes in (0, 1 << 11, (1 << 20) + 8, 3 << 20, 1 << 36):
        assert L.mcrt_probe_gather(0, nbytes, C.byref(r)) == mcrt.MCRT_E_ARG, nbytes
    assert L.mcrt_probe_gather(0, 1 << 20, None) == mcrt.MCRT_E_ARG


def test_probes_without_gpu_fail_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(mcrt.McrtError) as e:
        mcrt.mcrt_probe_ex2(0)
    assert e.value.status == mcrt.MCRT_E_CUDA
    with pytest.raises(mcrt.McrtError) as e:
        mcrt.mcrt_probe_gather(0, 1 << 20)
    assert e.value.status == mcrt.MCRT_E_CUDA
