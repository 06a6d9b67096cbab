"""The allocation-free Nusselt entry point against the handle-based one (GPU).

lbm_nusselt_static serves callers that may not allocate device memory (their memory belongs to
another allocator): it takes the energy populations and a result buffer the caller owns and keeps
its block partials in a fixed array inside the library.  Here its result must equal lbm_nusselt's
on the same state, within the 1e-11 used for every Nusselt comparison in these tests, on
consecutive calls that reuse the shared scratch array, for the three storage layouts and for a
face at the array's size limit.  The file is collected last so that a run stopping at the first
failure has already run every other test; it passes alone as well.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402

STATE_HEADER = 64          # bytes before the populations in an lbm_get_state checkpoint
ELEM = {"fp64": 8, "fp32": 4, "fp16s": 2}


def energy_planes(lat, precision):
    """The handle's energy populations, on the device, in the storage format of its precision:
    FP64 as lbm_get_populations writes them, FP32 / FP16S as stored (the g planes of the
    checkpoint, after the header and the flow planes)."""
    if precision == "fp64":
        return lat.get_populations(device=True)[1]
    n = lat.nx * lat.ny * lat.nz
    buf = lat.get_state()
    start = STATE_HEADER + lat.qf * n * ELEM[precision]
    g = buf[start:start + lat.qg * n * ELEM[precision]]
    assert g.size == lat.qg * n * ELEM[precision] and start + g.size == buf.size
    return torch.from_numpy(np.ascontiguousarray(g)).to("cuda")


def static_nusselt(lat, walls, g_dev, face, code, result):
    inf = lat.info()
    L.lbm_nusselt_static(code, lat.nx, lat.ny, lat.nz, walls.face, walls.T_wall, walls.T_ref,
                         g_dev.data_ptr(), face, inf.L, inf.dT, result.data_ptr(),
                         lat.stream.cuda_stream)
    lat.stream.synchronize()
    r = result.cpu().numpy()
    return r[0], r[1], r[3], int(r[2]), int(r[4])


def check_against_handle(lat, walls, g, face, code, result):
    want = lat.nusselt(face)
    got = static_nusselt(lat, walls, g, face, code, result)
    np.testing.assert_allclose(got[:3], want[:3], rtol=0, atol=1e-11)
    # the max / min location is unique unless another node ties within the tolerance; either
    # way the reported node must hold the extreme value
    prof = lat.nusselt_profile(face).cpu().numpy()
    for idx, ext in ((got[3], want[1]), (got[4], want[2])):
        assert abs(prof[idx] - ext) <= 1e-11
    for idx_g, idx_w, ext in ((got[3], want[3], want[1]), (got[4], want[4], want[2])):
        if np.sum(np.abs(prof - ext) <= 1e-11) == 1:
            assert idx_g == idx_w


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("dim,shape", [(2, (1, 64, 96)), (3, (16, 20, 24))])
def test_static_nusselt_matches_handle_nusselt_on_consecutive_calls(dim, shape, precision):
    nz, ny, nx = shape
    lattice = "d2q9" if dim == 2 else "d3q27"
    walls = L.Walls.cavity(dim)
    lat = L.Lattice(lattice, nx, ny, nz, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls, precision=precision)
    code = L.LATTICES[lattice] | L.PRECISIONS[precision]
    result = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    for steps in (150, 70):
        lat.step(steps)
        g = energy_planes(lat, precision)
        for face in (0, 1, 0):
            check_against_handle(lat, walls, g, face, code, result)
    lat.close()


def test_static_nusselt_on_a_face_at_the_scratch_limit():
    """A 2 x 1024 x 1024 box: its -x face has exactly LBM_NUSSELT_STATIC_MAX_FACE_NODES nodes,
    so every one of the array's 4096 block partials is used and the last block merges 16 per
    thread."""
    n = 1024
    assert n * n == L.NUSSELT_STATIC_MAX_FACE_NODES
    walls = L.Walls.cavity(3)
    lat = L.Lattice("d3q27", 2, n, n, Ra=1e5, Pr=0.71, Ma=0.1, walls=walls, precision="fp64")
    lat.step(6)
    g = energy_planes(lat, "fp64")
    result = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    code = L.LBM_D3Q27_D3Q15 | L.LBM_FP64
    for face in (0, 1):
        check_against_handle(lat, walls, g, face, code, result)
    lat.close()


def test_static_nusselt_rejects_a_face_beyond_its_scratch():
    walls = L.Walls.cavity(3)
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    n = 1025     # a 1025 x 1025 face: more nodes than LBM_NUSSELT_STATIC_MAX_FACE_NODES
    with pytest.raises(L.LbmError) as e:
        L.lbm_nusselt_static(L.LBM_D3Q27_D3Q15 | L.LBM_FP64, 4, n, n, walls.face, walls.T_wall,
                             walls.T_ref, buf.data_ptr(), 0, 4.0, 1.0, out.data_ptr())
    assert e.value.status == L.LBM_EINVAL
    # the reason comes from the library (lbm_last_error(NULL) on this thread)
    assert "more than LBM_NUSSELT_STATIC_MAX_FACE_NODES" in L.lbm_last_error(None)
