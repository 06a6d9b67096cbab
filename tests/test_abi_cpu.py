"""The C ABI library builds, loads and exports every entry point of include/*.h (CPU only).

No compute call is made here: only argument validation that returns before any CUDA work.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbm():
    from paper_2504_09041_gb300 import build as B
    B.build()
    from paper_2504_09041_gb300 import lbm as L
    return L


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"LBM_API\s+[\w\s\*]+?\b(lbm_\w+)\s*\(", text))
    return names


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for n in ("lbm_create", "lbm_destroy", "lbm_step", "lbm_fields", "lbm_nusselt",
              "lbm_set_wall_profile", "lbm_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lbm):
    L = ctypes.CDLL(lbm.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_has_the_same_names(lbm):
    for n in declared_symbols():
        assert callable(getattr(lbm, n)), n


def test_status_strings(lbm):
    assert lbm.lbm_status_string(lbm.LBM_OK) == "ok"
    assert lbm.lbm_status_string(lbm.LBM_EDIVERGED) == "simulation diverged"


@pytest.mark.parametrize("args,msg", [
    ((3, 8, 8, 1), "unknown lattice"),
    ((1 | 0x300, 8, 8, 1), "unknown precision"),
    ((1, 0, 8, 1), "empty"),
    ((1, 8, 8, 2), "nz = 1"),
    ((2, 2048, 2048, 1024), "2^31"),
])
def test_create_rejects_bad_boxes(lbm, args, msg):
    bc = lbm.Walls.cavity(2).to_c()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(*args, 1e4, 0.71, 0.1, bc)
    assert e.value.status == lbm.LBM_EINVAL
    assert msg in str(e.value)


def test_create_rejects_bad_parameters(lbm):
    bc = lbm.Walls.cavity(2).to_c()
    for Ra, Pr, Ma in ((0, 0.71, 0.1), (1e4, -1, 0.1), (1e4, 0.71, float("nan"))):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(1, 8, 8, 1, Ra, Pr, Ma, bc)
        assert e.value.status == lbm.LBM_EINVAL


def test_create_rejects_one_sided_periodic_and_bad_gravity(lbm):
    w = lbm.Walls.cavity(2)
    w.face = (lbm.LBM_PERIODIC, lbm.LBM_WALL_FIXED_T, 1, 1, 0, 0)
    with pytest.raises(lbm.LbmError, match="periodic on one face"):
        lbm.lbm_create(1, 8, 8, 1, 1e4, 0.71, 0.1, w.to_c())
    w = lbm.Walls.cavity(2)
    w.gravity_axis = 2
    with pytest.raises(lbm.LbmError, match="gravity axis"):
        lbm.lbm_create(1, 8, 8, 1, 1e4, 0.71, 0.1, w.to_c())


def test_allocator_needs_both_hooks(lbm):
    alloc = lbm.ALLOC_FN(lambda n, c: None)
    assert lbm.lib().lbm_set_allocator(alloc, lbm.FREE_FN(), None) == lbm.LBM_EINVAL
    assert lbm.lib().lbm_set_allocator(lbm.ALLOC_FN(), lbm.FREE_FN(), None) == lbm.LBM_OK


def test_binding_fails_loudly_without_the_library(lbm, monkeypatch):
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "liblbm.so"))
    with pytest.raises(ImportError):
        lbm.lib()


def test_batch_create_rejects_bad_requests(lbm):
    cav = lbm.Walls.cavity(2).to_c()
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create(lbm.LBM_D3Q27_D3Q15 | lbm.LBM_FP32, [8], [8], [1e4], [0.71], 0.1,
                             [lbm.Walls.cavity(3).to_c()])
    assert e.value.status == lbm.LBM_ENOTSUP
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create(lbm.LBM_D2Q9_D2Q9 | lbm.LBM_FP32, [8, 0], [8, 8], [1e4, 1e4],
                             [0.71, 0.71], 0.1, [cav, cav])
    assert e.value.status == lbm.LBM_EINVAL and "member 1" in str(e.value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create(lbm.LBM_D2Q9_D2Q9 | lbm.LBM_FP32, [8, 8], [8, 8], [1e4, -1.0],
                             [0.71, 0.71], 0.1, [cav, cav])
    assert e.value.status == lbm.LBM_EINVAL and "member 1" in str(e.value)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create(lbm.LBM_D2Q9_D2Q9 | lbm.LBM_FP32, [], [], [], [], 0.1, [])
    assert e.value.status == lbm.LBM_EINVAL
    with pytest.raises(ValueError):
        lbm.lbm_batch_create(lbm.LBM_D2Q9_D2Q9, [8], [8, 8], [1e4], [0.71], 0.1, [cav])


def test_batch_calls_reject_a_null_batch(lbm):
    L = lbm.lib()
    assert L.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    assert L.lbm_batch_sync(None, None) == lbm.LBM_EINVAL
    assert L.lbm_batch_destroy(None) == lbm.LBM_EINVAL
    assert L.lbm_batch_set_launch(None, 64, 2, 8, 32) == lbm.LBM_EINVAL
    assert L.lbm_batch_info(None, None) == lbm.LBM_EINVAL
    assert "NULL" in lbm.lbm_batch_last_error(None)


def test_bounded_wait_probe_validates_its_limit(lbm):
    t = ctypes.c_int(-1)
    for bad in (0.0, -1.0, 11.0, float("nan")):
        assert lbm.lib().lbm_probe_bounded_wait(bad, ctypes.byref(t)) == lbm.LBM_EINVAL
    assert lbm.lib().lbm_probe_bounded_wait(0.01, None) == lbm.LBM_EINVAL
    assert lbm.lbm_status_string(lbm.LBM_ETIMEOUT) == "a bounded device wait timed out"


@pytest.mark.parametrize("n,face,msg", [
    (1025, 0, "face 0 has 1050625 nodes, more than LBM_NUSSELT_STATIC_MAX_FACE_NODES"),
    (8, 2, "face 2 is not a fixed-temperature wall"),
])
def test_nusselt_static_reports_why_it_rejects_a_call(lbm, n, face, msg):
    """The allocation-free Nusselt entry validates its arguments before any CUDA call, and
    lbm_last_error(NULL) on the calling thread carries the library's own reason."""
    walls = lbm.Walls.cavity(3)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_nusselt_static(lbm.LBM_D3Q27_D3Q15 | lbm.LBM_FP64, 4, n, n, walls.face, walls.T_wall,
                               walls.T_ref, 16, face, 4.0, 1.0, 16)
    assert e.value.status == lbm.LBM_EINVAL
    assert msg in lbm.lbm_last_error(None)
    assert msg in str(e.value)
