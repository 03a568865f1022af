"""The C ABI boundary on the host: libstba.so builds, loads, exports every declared symbol, and rejects
invalid problems before touching the device."""
import os
import re

import numpy as np
import pytest

import scenes
from paper_2008_00446_gb300 import stba

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "stba.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(stba_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = stba.load()
    decl = declared_symbols()
    assert len(decl) >= 18
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(decl) == sorted(stba.EXPORTS)


def test_default_options_match_the_paper():
    # Sec. 5.1 / Algorithm 1: lambda0 = 1e-4; Sec. 4.3: correction when lambda >= 0.1
    o = stba.stba_default_options()
    assert o.lambda0 == 1e-4 and o.correction_lambda == 0.1 and o.correction == 1
    assert o.precision == stba.STBA_FP64 and o.refine_steps == 1
    assert o.huber_a == 0.0   # plain least squares unless the Huber loss is asked for


def header_struct_fields(name):
    """(type, field) of a `typedef struct {...} name;` of include/stba.h, in declaration order."""
    import os
    import re
    h = open(os.path.join(os.path.dirname(__file__), "..", "include", "stba.h")).read()
    end = h.index("} " + name + ";")
    body = h[h.rindex("typedef struct {", 0, end):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    out = []
    for t, names in re.findall(r"\b(int32_t|int64_t|double|float)\s+([\w\s,]+?)\s*;", body):
        out += [(t, nm.strip()) for nm in names.split(",")]
    return out


@pytest.mark.parametrize("cname, pyclass", [("stba_options", "StbaOptions"), ("stba_iter_info", "StbaIterInfo")])
def test_binding_structs_match_the_header(cname, pyclass):
    # the ctypes mirrors of the C structs: same fields, order and types (a missing field would let the
    # library write past the binding's struct)
    import ctypes
    ctype = {"int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "double": ctypes.c_double,
             "float": ctypes.c_float}
    want = [(f if f != "lambda" else "lambda_", ctype[t]) for t, f in header_struct_fields(cname)]
    got = list(getattr(stba, pyclass)._fields_)
    assert got == want


def test_status_strings():
    L = stba.load()
    for s in range(8):
        assert L.stba_status_string(s).decode() == stba.STATUS[s] or s == 4


def base():
    return scenes.make_tiny_scene(m=4, n=12, seed=1)


@pytest.mark.parametrize("mutate, status", [
    (lambda s: s.obs_cam.__setitem__(0, 99), 1),                       # camera index out of range
    (lambda s: s.obs_pt.__setitem__(0, -1), 1),                        # point index out of range
    (lambda s: s.obs_uv.__setitem__((1, 0), np.nan), 5),               # non-finite observation
    (lambda s: s.cameras.__setitem__((0, 6), np.inf), 5),              # non-finite camera
    (lambda s: s.clusters.__setitem__(1, 3), 1),                       # cluster ids 0..l-1 with a gap
])
def test_invalid_problems_are_rejected_on_the_host(mutate, status):
    s = base()
    s.clusters = np.zeros(s.m, np.int32)
    s.clusters[1] = 1
    mutate(s)
    with pytest.raises(stba.StbaError) as e:
        stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters)
    assert e.value.status == status


def test_point_with_one_observation_and_duplicates_are_rejected():
    s = base()
    # drop all but one observation of point 0
    keep = np.ones(s.q, bool)
    idx = np.flatnonzero(s.obs_pt == 0)
    keep[idx[1:]] = False
    with pytest.raises(stba.StbaError) as e:
        stba.stba_create(s.cameras, s.points, s.obs_cam[keep], s.obs_pt[keep], s.obs_uv[keep], s.clusters)
    assert e.value.status == 1 and "fewer than 2" in str(e.value)
    dup_c = np.concatenate([s.obs_cam, s.obs_cam[:1]])
    dup_p = np.concatenate([s.obs_pt, s.obs_pt[:1]])
    dup_uv = np.concatenate([s.obs_uv, s.obs_uv[:1]])
    with pytest.raises(stba.StbaError) as e:
        stba.stba_create(s.cameras, s.points, dup_c, dup_p, dup_uv, s.clusters)
    assert "twice" in str(e.value)


def test_invalid_options_are_rejected():
    s = base()
    with pytest.raises(stba.StbaError):
        stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lambda0=0.0)
    with pytest.raises(stba.StbaError):
        stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, precision=7)
    for bad_tile in (16, 48, -1):
        with pytest.raises(stba.StbaError):
            stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, precision=1,
                             factor_tile=bad_tile)
    with pytest.raises(stba.StbaError):   # the FP64 factor has one tile
        stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, factor_tile=64)
    # the tensor-core trailing update exists for the FP32 factor with tile 64 only
    for kw in (dict(factor_update=stba.STBA_FACTOR_UPDATE_TENSOR),
               dict(precision=1, factor_tile=32, factor_update=stba.STBA_FACTOR_UPDATE_TENSOR),
               dict(precision=1, factor_update=3), dict(precision=1, factor_update=-1),
               dict(factor_panel=stba.STBA_FACTOR_PANEL_SPLIT),
               dict(precision=1, factor_tile=32, factor_panel=stba.STBA_FACTOR_PANEL_SPLIT),
               dict(precision=1, factor_panel=4), dict(factor_panel=stba.STBA_FACTOR_PANEL_PERSISTENT),
               dict(precision=1, factor_tile=32, factor_panel=stba.STBA_FACTOR_PANEL_PERSISTENT),
               dict(solve_cluster=3), dict(solve_cluster=16), dict(solve_cluster=-2),
               # the FP64 factor of mixed precision: tile 32 on the CUDA cores, stacked panel
               dict(precision=1, factor_fp64=2), dict(precision=1, factor_fp64=-1),
               dict(precision=1, factor_fp64=1, factor_tile=64),
               dict(precision=1, factor_fp64=1, factor_update=stba.STBA_FACTOR_UPDATE_TENSOR),
               dict(precision=1, factor_fp64=1, factor_panel=stba.STBA_FACTOR_PANEL_SPLIT),
               dict(precision=1, factor_fp64=1, factor_panel=stba.STBA_FACTOR_PANEL_PERSISTENT)):
        with pytest.raises(stba.StbaError):
            stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, **kw)
    for bad in (-0.5, float("nan"), float("inf")):
        with pytest.raises(stba.StbaError):
            stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, huber_a=bad)


def test_noalloc_wrapper_rejects_wrong_shapes_before_any_launch():
    # the allocation-free cost sizes every device read from the shapes it is given, so the wrapper checks
    # them all (and dtype, contiguity, one CUDA device) before calling into the library
    torch = pytest.importorskip("torch")
    m, n, q = 4, 6, 10
    good = dict(cameras=torch.zeros((m, 9), dtype=torch.float64), points=torch.zeros((n, 3), dtype=torch.float64),
                obs_cam=torch.zeros(q, dtype=torch.int32), obs_pt=torch.zeros(q, dtype=torch.int32),
                obs_uv=torch.zeros((q, 2), dtype=torch.float64), F_out=torch.zeros(1, dtype=torch.float64))
    bad = [("cameras", torch.zeros(m * 9, dtype=torch.float64)), ("points", torch.zeros((n, 4), dtype=torch.float64)),
           ("obs_pt", torch.zeros(q - 1, dtype=torch.int32)), ("obs_uv", torch.zeros((q + 1, 2), dtype=torch.float64)),
           ("obs_uv", torch.zeros((q, 3), dtype=torch.float64)), ("F_out", torch.zeros(0, dtype=torch.float64)),
           ("cameras", torch.zeros((0, 9), dtype=torch.float64))]
    for name, t in bad:
        args = dict(good, **{name: t})
        with pytest.raises(ValueError):
            stba.stba_cost_noalloc(**args)
    with pytest.raises(TypeError):   # right shapes, wrong dtype
        stba.stba_cost_noalloc(**dict(good, obs_cam=torch.zeros(q, dtype=torch.int64)))
    with pytest.raises(TypeError):   # right shapes and dtypes, but host tensors
        stba.stba_cost_noalloc(**good)
