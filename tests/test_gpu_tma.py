"""The TMA-staged 3D step (tma_rows = 1, 2, 4) against the plain 3D step.

Both kernels read the same stored values (through shared memory or straight from global memory)
and run the same node arithmetic, so the states must agree bit for bit: across ragged tiles in x
and y, x walls, periodic x, and every tile height.  The plain step itself is held to the oracle by
the parity tests.
"""
import numpy as np
import pytest

from tests import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402


def walls(kind):
    if kind == "cavity":
        return L.Walls.cavity(3)
    # periodic x, adiabatic y walls, fixed-T z walls (hot below), gravity along z
    face = (L.LBM_PERIODIC, L.LBM_PERIODIC, L.LBM_WALL_ADIABATIC, L.LBM_WALL_ADIABATIC,
            L.LBM_WALL_FIXED_T, L.LBM_WALL_FIXED_T)
    return L.Walls(face, (0, 0, 0, 0, 1.0, 0.0), 0.5, 0.5, 2)


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
@pytest.mark.parametrize("rows", [1, 2, 4])
@pytest.mark.parametrize("kind,shape", [("cavity", (13, 21, 64)), ("cavity", (9, 10, 72)),
                                        ("periodic_x", (7, 11, 136)), ("cavity", (3, 3, 8))])
def test_tma_step_equals_plain_step(precision, rows, kind, shape):
    nz, ny, nx = shape
    a = L.Lattice("d3q27", nx, ny, nz, Ra=1e5, walls=walls(kind), precision=precision)
    b = L.Lattice("d3q27", nx, ny, nz, Ra=1e5, walls=walls(kind), precision=precision)
    b.set_param("tma_rows", rows)
    f, g = a.get_populations()
    f = synth.perturbed(f, 71, 0.05); g = synth.perturbed(g, 72, 0.05)
    a.set_populations(f, g); b.set_populations(f, g)
    a.step(37); b.step(37)           # one graph replay of 32 steps and 5 plain launches
    a.sync(); b.sync()
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)


def test_tma_rows_is_validated():
    lat2 = L.Lattice("d2q9", 16, 16, Ra=1e4, precision="fp32")
    with pytest.raises(L.LbmError):
        lat2.set_param("tma_rows", 2)
    lat64 = L.Lattice("d3q27", 8, 8, 8, Ra=1e4, precision="fp64")
    with pytest.raises(L.LbmError):
        lat64.set_param("tma_rows", 2)
    odd = L.Lattice("d3q27", 30, 8, 8, Ra=1e4, precision="fp32")   # 120-byte rows
    with pytest.raises(L.LbmError) as e:
        odd.set_param("tma_rows", 2)
    assert e.value.status == L.LBM_ENOTSUP
    ok = L.Lattice("d3q27", 32, 8, 8, Ra=1e4, precision="fp32")
    for bad in (3, -1, 0.5):
        with pytest.raises(L.LbmError):
            ok.set_param("tma_rows", bad)
    ok.set_param("tma_rows", 4)
    ok.step(3)
    ok.sync()
    ok.set_param("tma_rows", 0)
    ok.step(3)
    ok.sync()


def test_bounded_device_wait_gives_up_and_the_context_survives():
    """An mbarrier wait that nothing completes runs out after its limit (10 ms here), records the
    timeout and returns: no trap, no hang.  The GPU then steps a TMA-staged box normally."""
    import time
    t0 = time.perf_counter()
    st, timed_out = L.lbm_probe_bounded_wait(0.01)
    assert st == L.LBM_ETIMEOUT and timed_out == 1
    assert time.perf_counter() - t0 < 5.0
    lat = L.Lattice("d3q27", 64, 16, 16, Ra=1e5, walls=L.Walls.cavity(3), precision="fp32")
    lat.set_param("tma_rows", 2)
    lat.step(10)
    lat.sync()
