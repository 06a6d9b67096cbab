"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances:
  * FP64 storage: populations within 1e-14 after one step and 1e-12 after 100 steps (max-abs).
    Both sides compute in FP64 from identical inputs and differ only in rounding order
    (per-axis sweeps and fused multiply-adds on the GPU, the printed Step 1-5 formulas in the
    oracle): ~1e-16 per operation, a few hundred operations per step.
  * FP32 storage: fields within 1e-5 relative (max |diff| / max |reference| per field) after
    100 steps.
  * FP16S storage: populations are rounded to 11 significant bits of their deviation from the
    rest state each step; fields are compared at the tolerance derived in the test.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from tests import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402


def walls_pair(kind: str, dim: int, seed=0, perturb=0.0):
    """The same boundary description for both sides."""
    if kind == "cavity":
        return L.Walls.cavity(dim), O.cavity_bc(dim)
    if kind == "rb":
        return (L.Walls.rayleigh_benard(seed=seed, perturb=perturb),
                O.rayleigh_benard_bc(seed=seed, perturb=perturb))
    if kind == "mixed3d":
        # periodic x, adiabatic y walls, fixed-T z walls (hot below), gravity along z
        face = (O.PERIODIC, O.PERIODIC, O.WALL_ADIABATIC, O.WALL_ADIABATIC, O.WALL_FIXED_T,
                O.WALL_FIXED_T)
        T_wall = (0, 0, 0, 0, 1.0, 0.0)
        return (L.Walls(face, T_wall, 0.5, 0.5, 2, seed, perturb),
                O.BC(face, T_wall, 0.5, 0.5, 2, seed, perturb))
    if kind == "periodic":
        face = (O.PERIODIC,) * 6
        return L.Walls(face, (0,) * 6, 0.5, 0.5, 1 if dim == 2 else 2), O.BC(face, (0,) * 6, 0.5, 0.5,
                                                                             1 if dim == 2 else 2)
    raise ValueError(kind)


def make_pair(dim, nx, ny, nz=1, kind="cavity", precision="fp64", rates_seed=None, gbeta=None,
              Ra=1e4, Pr=0.71, Ma=0.1, seed=0, perturb=0.0):
    lat = "d2q9" if dim == 2 else "d3q27"
    wl, wo = walls_pair(kind, dim, seed, perturb)
    gpu = L.Lattice(lat, nx, ny, nz, Ra=Ra, Pr=Pr, Ma=Ma, walls=wl, precision=precision)
    if rates_seed is None:
        ora = O.Oracle(dim, nx, ny, nz, bc=wo, Ra=Ra, Pr=Pr, Ma=Ma)
    else:
        qf, qg = (9, 9) if dim == 2 else (27, 15)
        om_f, om_g = synth.rates(rates_seed, qf), synth.rates(rates_seed + 1, qg)
        ora = O.Oracle(dim, nx, ny, nz, bc=wo, om_f=om_f, om_g=om_g, gbeta=gbeta)
        gpu.set_omegas(om_f, om_g)
        gpu.set_param("gbeta", gbeta)
    return gpu, ora


def randomize(gpu, ora, seed, scale=0.3):
    f, g = ora.get_state()
    f = synth.perturbed(f, seed, scale)
    g = synth.perturbed(g, seed + 1, scale)
    ora.set_state(f, g)
    gpu.set_populations(f, g)


def pop_error(gpu, ora):
    fg, gg = gpu.get_populations()
    fo, go = ora.get_state()
    return max(np.abs(fg - fo).max(), np.abs(gg - go).max())


def field_errors(gpu, ora):
    fg = {k: v.cpu().numpy() for k, v in gpu.fields().items()}
    fo = ora.fields()
    out = {}
    for k in ("rho", "ux", "uy", "uz", "T"):
        ref = np.abs(fo[k]).max()
        if ref == 0.0:
            continue
        out[k] = np.abs(fg[k] - fo[k]).max() / ref
    return out


# ---------------------------------------------------------------------------------------------
# Initial state, parameters, host plumbing
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_initial_state_matches_oracle(dim):
    nx, ny, nz = (70, 33, 1) if dim == 2 else (19, 11, 7)
    gpu, ora = make_pair(dim, nx, ny, nz, kind="rb" if dim == 2 else "mixed3d", seed=77, perturb=1e-3)
    assert pop_error(gpu, ora) <= 1e-16


@pytest.mark.parametrize("dim,kind,shape", [(2, "cavity", (1, 64, 64)), (2, "rb", (1, 512, 1024)),
                                            (3, "cavity", (256, 256, 256))])
def test_parameter_mapping_matches_oracle(dim, kind, shape):
    nz, ny, nx = shape
    wl, wo = walls_pair(kind, dim)
    lat = "d2q9" if dim == 2 else "d3q27"
    h = L.lbm_create(L.LATTICES[lat] | L.LBM_FP32, nx, ny, nz, 1e6, 0.71, 0.1, wl.to_c())
    try:
        inf = L.lbm_info(h)
        ora = O.Oracle(dim, nx, ny, nz, bc=wo, Ra=1e6, Pr=0.71, Ma=0.1, init=False)
        assert inf.L == ora.L
        for k in ("nu", "alpha", "gbeta", "U"):
            assert getattr(inf, k) == pytest.approx(getattr(ora.tr, k), rel=1e-14)
        np.testing.assert_allclose(np.array(inf.om_f[:ora.qf]), ora.om_f, rtol=1e-14)
        np.testing.assert_allclose(np.array(inf.om_g[:ora.qg]), ora.om_g, rtol=1e-14)
        bpn = 2 * (ora.qf + ora.qg) * 4
        assert inf.bytes_per_node_update == bpn
    finally:
        L.lbm_destroy(h)


def test_out_of_memory_is_reported():
    def fail_alloc(n, ctx):
        return None

    hooks = (L.ALLOC_FN(fail_alloc), L.FREE_FN(lambda p, c: None))
    assert L.lib().lbm_set_allocator(hooks[0], hooks[1], None) == 0
    try:
        with pytest.raises(L.LbmError) as e:
            L.lbm_create(L.LBM_D2Q9_D2Q9, 16, 16, 1, 1e4, 0.71, 0.1, L.Walls.cavity(2).to_c())
        assert e.value.status == L.LBM_ENOMEM
    finally:
        L.use_cuda_allocator()


def test_rates_outside_range_are_rejected():
    gpu, _ = make_pair(2, 8, 8)
    with pytest.raises(L.LbmError) as e:
        gpu.set_omegas(np.full(9, 2.0))
    assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LbmError):
        gpu.set_param("no_such_key", 1.0)
    with pytest.raises(L.LbmError):
        gpu.nusselt(2)          # adiabatic face
    with pytest.raises(L.LbmError):
        L.lbm_step(gpu.h, -1)


# ---------------------------------------------------------------------------------------------
# FP64 parity of the fused step
# ---------------------------------------------------------------------------------------------

PARITY_2D = [("cavity", (1, 70, 150)), ("rb", (1, 37, 131)), ("periodic", (1, 9, 40))]
PARITY_3D = [("cavity", (13, 21, 37)), ("mixed3d", (9, 10, 70))]


@pytest.mark.parametrize("kind,shape", PARITY_2D)
def test_fp64_step_parity_2d(kind, shape):
    nz, ny, nx = shape
    gpu, ora = make_pair(2, nx, ny, kind=kind, rates_seed=11, gbeta=3e-3)
    randomize(gpu, ora, 5)
    gpu.step(1); ora.step(1)
    assert pop_error(gpu, ora) <= 1e-14
    gpu.step(99); ora.step(99)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12


@pytest.mark.parametrize("kind,shape", PARITY_3D)
def test_fp64_step_parity_3d(kind, shape):
    nz, ny, nx = shape
    gpu, ora = make_pair(3, nx, ny, nz, kind=kind, rates_seed=21, gbeta=3e-3)
    randomize(gpu, ora, 6)
    gpu.step(1); ora.step(1)
    assert pop_error(gpu, ora) <= 1e-14
    gpu.step(99); ora.step(99)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12


@pytest.mark.parametrize("dim,shape", [(2, (1, 1, 1)), (2, (1, 2, 2)), (2, (1, 3, 1)),
                                       (3, (2, 2, 2)), (3, (1, 3, 2)), (3, (3, 1, 1))])
def test_fp64_degenerate_boxes(dim, shape):
    """Boxes one or two nodes wide: every link of every node is a wall or wrap case."""
    nz, ny, nx = shape
    kind = "cavity" if min(shape[1:]) > 1 or dim == 3 else "periodic"
    gpu, ora = make_pair(dim, nx, ny, nz, kind=kind, rates_seed=31, gbeta=1e-2)
    randomize(gpu, ora, 7, scale=0.2)
    gpu.step(10); ora.step(10)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_fields_and_nusselt_match_oracle(dim):
    nx, ny, nz = (90, 41, 1) if dim == 2 else (23, 17, 11)
    gpu, ora = make_pair(dim, nx, ny, nz, kind="cavity", rates_seed=41, gbeta=2e-3)
    randomize(gpu, ora, 8, scale=0.1)
    gpu.step(20); ora.step(20)
    fg = {k: v.cpu().numpy() for k, v in gpu.fields().items()}
    fo = ora.fields()
    for k in ("rho", "ux", "uy", "uz", "T"):
        np.testing.assert_allclose(fg[k], fo[k], rtol=0, atol=1e-13, err_msg=k)
    for face in (0, 1):
        mg = gpu.nusselt(face)
        mo = ora.nusselt(face)
        assert mg[0] == pytest.approx(mo[0], abs=1e-11)
        assert mg[1] == pytest.approx(mo[1], abs=1e-11)
        assert mg[2] == pytest.approx(mo[2], abs=1e-11)
        assert mg[3:] == mo[3:]
        np.testing.assert_allclose(gpu.nusselt_profile(face).cpu().numpy(), ora.nusselt_profile(face),
                                   rtol=0, atol=1e-11)


def test_wall_profile_parity():
    """Per-node hot-wall temperature (1 + 0.05 * seeded sine modes) on the anti-bounce-back."""
    nx = ny = 48
    gpu, ora = make_pair(2, nx, ny, kind="cavity", Ra=1e5)
    prof = synth.sine_profile(3, ny)
    gpu.set_wall_profile(0, prof)
    ora.set_wall_profile(0, prof)
    gpu.step(200); ora.step(200)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12
    assert gpu.nusselt(1)[0] == pytest.approx(ora.nusselt(1)[0], abs=1e-11)
    gpu.set_wall_profile(0, None)


def test_checkpoint_round_trip_is_exact():
    gpu, _ = make_pair(3, 20, 12, 10, kind="cavity", precision="fp32")
    gpu.step(5)
    state = gpu.get_state()
    gpu.step(10)
    f1, g1 = gpu.get_populations()
    gpu.set_state(state)
    assert gpu.info().steps == 5
    gpu.step(10)
    f2, g2 = gpu.get_populations()
    assert np.array_equal(f1, f2) and np.array_equal(g1, g2)
    with pytest.raises(L.LbmError):
        gpu.set_state(state[:-1])


def test_divergence_is_reported_without_a_fault():
    """Host-side fault injection: a NaN population uploaded, one step, LBM_EDIVERGED on sync."""
    gpu, ora = make_pair(2, 16, 16)
    f, g = ora.get_state()
    f[3, 0, 5, 5] = np.nan
    gpu.set_populations(f, g)
    gpu.step(1)
    with pytest.raises(L.LbmError) as e:
        gpu.sync()
    assert e.value.status == L.LBM_EDIVERGED
    f[3, 0, 5, 5] = f[3, 0, 5, 4]
    gpu.set_populations(f, g)
    gpu.step(1)
    gpu.sync()


# ---------------------------------------------------------------------------------------------
# Reduced-precision storage
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("dim,shape", [(2, (1, 70, 150)), (3, (13, 21, 37))])
def test_fp32_fields_within_1e5(dim, shape):
    nz, ny, nx = shape
    gpu, ora = make_pair(dim, nx, ny, nz, kind="cavity", precision="fp32", rates_seed=51, gbeta=3e-3)
    randomize(gpu, ora, 9)
    # the FP64 oracle starts from the FP32-rounded state the GPU holds
    f, g = gpu.get_populations()
    ora.set_state(f, g)
    gpu.step(100); ora.step(100)
    gpu.sync()
    errs = field_errors(gpu, ora)
    assert max(errs.values()) <= 1e-5, errs


@pytest.mark.parametrize("dim,shape", [(2, (1, 64, 64)), (3, (16, 16, 16))])
def test_fp16s_fields_near_fp64(dim, shape):
    """FP16 storage of the deviation from rest: 100 steps of the cavity from its initial state.

    Each stored deviation d carries a rounding error of at most 2^-11 |d|; with |d| <= 0.1 w and
    about 10 roundings reaching a node's moments per step, the fields drift by O(1e-4) of their
    range in 100 steps.  Tolerance 2e-3 of each field's range.
    """
    nz, ny, nx = shape
    gpu, ora = make_pair(dim, nx, ny, nz, kind="cavity", precision="fp16s", Ra=1e5)
    gpu.step(100); ora.step(100)
    gpu.sync()
    fg = {k: v.cpu().numpy() for k, v in gpu.fields().items()}
    fo = ora.fields()
    for k in ("rho", "ux", "uy", "T"):
        scale = max(np.ptp(fo[k]), np.abs(fo[k]).max() if k != "rho" else 0.0)
        assert np.abs(fg[k] - fo[k]).max() <= 2e-3 * scale, k


# ---------------------------------------------------------------------------------------------
# Whole-method checks against the printed tables
# ---------------------------------------------------------------------------------------------

def test_cavity_64_nusselt_fp64_matches_oracle_and_table():
    """64^2 cavity, Ra 1e4, 20000 steps: GPU FP64 vs oracle (tight) and vs Table con2 (1 %)."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    gpu, ora = make_pair(2, 64, 64, kind="cavity", Ra=1e4)
    gpu.step(20000); ora.step(20000)
    gpu.sync()
    mg, mo = gpu.nusselt(0), ora.nusselt(0)
    assert mg[0] == pytest.approx(mo[0], rel=1e-9)
    assert mg[3:] == mo[3:]
    assert mg[0] == pytest.approx(gold["nu0_mean_2d_512"]["1e4"], rel=0.01)


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
def test_cavity_64_reduced_precision_nusselt_within_half_percent(precision):
    gpu, ora = make_pair(2, 64, 64, kind="cavity", precision=precision, Ra=1e4)
    gpu.step(20000); ora.step(20000)
    gpu.sync()
    assert gpu.nusselt(0)[0] == pytest.approx(ora.nusselt(0)[0], rel=5e-3)
