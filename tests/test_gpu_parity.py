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
              Ra=1e4, Pr=0.71, Ma=0.1, seed=0, perturb=0.0, rate_range=(0.6, 1.9), g_option=0):
    lat = "d2q9" if dim == 2 else "d3q27"
    wl, wo = walls_pair(kind, dim, seed, perturb)
    gpu = L.Lattice(lat, nx, ny, nz, Ra=Ra, Pr=Pr, Ma=Ma, walls=wl, precision=precision)
    gpu.set_param("g_attractors", g_option)
    if rates_seed is None:
        ora = O.Oracle(dim, nx, ny, nz, bc=wo, Ra=Ra, Pr=Pr, Ma=Ma, g_option=g_option)
    else:
        qf, qg = (9, 9) if dim == 2 else (27, 15)
        om_f = synth.rates(rates_seed, qf, *rate_range)
        om_g = synth.rates(rates_seed + 1, qg, *rate_range)
        ora = O.Oracle(dim, nx, ny, nz, bc=wo, om_f=om_f, om_g=om_g, gbeta=gbeta, g_option=g_option)
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
    # the oracle forms w T through its moment transforms (Steps 4-5), the GPU as w * T: one ulp
    assert pop_error(gpu, ora) <= 2e-16


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
    # 3D: a milder random state (5 %) and rates in [0.7, 1.7]; stronger perturbations with rates
    # near 2 on the fourth- to sixth-order moments drive the state to negative densities
    gpu, ora = make_pair(3, nx, ny, nz, kind=kind, rates_seed=21, gbeta=3e-3, rate_range=(0.7, 1.7))
    randomize(gpu, ora, 6, scale=0.05)
    gpu.step(1); ora.step(1)
    assert pop_error(gpu, ora) <= 1e-14
    gpu.step(99); ora.step(99)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12


@pytest.mark.parametrize("kind,shape", PARITY_3D)
@pytest.mark.parametrize("random_flow_rates", [False, True])
def test_fp64_step_parity_3d_unit_energy_rates(kind, shape, random_flow_rates):
    """With the energy rates of lbm_create (every rate 1 except the first-order ones) the 3D step
    takes the reduced energy collision (only T and the first-order moments enter).  Against the
    oracle, which runs App. C's full Steps 1-5: the same bars as the general step, with the
    default rates and with random flow rates and first-order energy rates."""
    nz, ny, nx = shape
    gpu, ora = make_pair(3, nx, ny, nz, kind=kind)
    om_f, om_g = ora.om_f.copy(), ora.om_g.copy()
    assert np.all(om_g[4:] == 1.0)
    if random_flow_rates:
        om_f = synth.rates(31, 27, 0.7, 1.7)
        om_g[1:4] = synth.rates(32, 3, 0.7, 1.7)
    ora = O.Oracle(3, nx, ny, nz, bc=walls_pair(kind, 3)[1], om_f=om_f, om_g=om_g, gbeta=3e-3)
    gpu.set_omegas(om_f, om_g)
    gpu.set_param("gbeta", 3e-3)
    randomize(gpu, ora, 16, scale=0.05)
    gpu.step(1); ora.step(1)
    assert pop_error(gpu, ora) <= 1e-14
    gpu.step(99); ora.step(99)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12


@pytest.mark.parametrize("dim,shape", [(2, (1, 37, 131)), (3, (13, 21, 37))])
def test_fp64_step_parity_option_b(dim, shape):
    """The renormalized option-B energy attractors (Eq. MvT2DoptionB, Sec. 5.3 D3Q15 list), with
    random second-order rates so that they differ from option A."""
    nz, ny, nx = shape
    kind = "rb" if dim == 2 else "cavity"
    rr = (0.6, 1.9) if dim == 2 else (0.7, 1.7)
    gpu, ora = make_pair(dim, nx, ny, nz, kind=kind, rates_seed=51, gbeta=3e-3, rate_range=rr,
                         g_option=1)
    assert gpu.info().g_attractors == 1
    randomize(gpu, ora, 8, scale=0.3 if dim == 2 else 0.05)
    gpu.step(1); ora.step(1)
    assert pop_error(gpu, ora) <= 1e-14
    gpu.step(99); ora.step(99)
    gpu.sync()
    assert pop_error(gpu, ora) <= 1e-12


def test_g_attractors_parameter_is_validated():
    gpu = L.Lattice("d2q9", 8, 8, Ra=1e4, precision="fp32")
    for bad in (-1, 2, 0.5):
        with pytest.raises(L.LbmError):
            gpu.set_param("g_attractors", bad)
    assert gpu.info().g_attractors == 0


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
@pytest.mark.parametrize("g_option", [0, 1])
def test_fp32_fields_within_1e5(dim, shape, g_option):
    nz, ny, nx = shape
    gpu, ora = make_pair(dim, nx, ny, nz, kind="cavity", precision="fp32", rates_seed=51, gbeta=3e-3,
                         rate_range=(0.6, 1.9) if dim == 2 else (0.7, 1.7), g_option=g_option)
    randomize(gpu, ora, 9, scale=0.3 if dim == 2 else 0.05)
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

    Each stored deviation d is rounded to 11 significant bits, |error| <= 2^-11 |d|, once per step.
    A field summing q populations drifts by at most q 2^-11 d_max per step if every rounding had
    the same sign; independent roundings add up as sqrt(N) over N steps.  The bound used here is
    3 q 2^-11 d_max sqrt(N), with d_max the largest deviation of the oracle's final state.
    """
    nz, ny, nx = shape
    steps = 100
    gpu, ora = make_pair(dim, nx, ny, nz, kind="cavity", precision="fp16s", Ra=1e5)
    gpu.step(steps); ora.step(steps)
    gpu.sync()
    fg = {k: v.cpu().numpy() for k, v in gpu.fields().items()}
    fo = ora.fields()
    f, g = ora.get_state()
    w_f = O.equilibrium_f(dim, 1.0)
    w_g = O.equilibrium_g(dim, 1.0) * 0.5
    dmax_f = np.abs(f - w_f.reshape(-1, 1, 1, 1)).max()
    dmax_g = np.abs(g - w_g.reshape(-1, 1, 1, 1)).max()
    qf, qg = ora.qf, ora.qg
    bound = lambda q, d: 3 * q * 2.0 ** -11 * d * math.sqrt(steps)
    errs = {k: np.abs(fg[k] - fo[k]).max() for k in ("rho", "ux", "uy", "uz", "T")}
    tol = {"rho": bound(qf, dmax_f), "ux": bound(qf, dmax_f), "uy": bound(qf, dmax_f),
           "uz": bound(qf, dmax_f), "T": bound(qg, dmax_g)}
    for k in errs:
        assert errs[k] <= tol[k], (k, errs, tol)


# ---------------------------------------------------------------------------------------------
# Full-size sampled parity
# ---------------------------------------------------------------------------------------------

def neighbourhood_box(f, g, node, walls_o, dims):
    """Populations of the (up to) 3^d box around `node` (device tensors in, numpy out) and the
    oracle boundary description that reproduces the node's streaming: real walls where the box
    touches them, wrapped neighbours on periodic axes.  Returns (f_box, g_box, local, BC)."""
    nz, ny, nx = f.shape[1:]
    ext = (nx, ny, nz)
    c = (node[2], node[1], node[0])
    idx, loc, face = [], [], list(walls_o.face)
    for ax in range(3):
        if ax >= dims:
            idx.append([0]); loc.append(0); continue
        n = ext[ax]
        if walls_o.face[2 * ax] == O.PERIODIC:
            idx.append([(c[ax] - 1) % n, c[ax], (c[ax] + 1) % n]); loc.append(1)
        elif c[ax] == 0:
            idx.append([0, 1]); loc.append(0)
        elif c[ax] == n - 1:
            idx.append([n - 2, n - 1]); loc.append(1)
        else:
            idx.append([c[ax] - 1, c[ax], c[ax] + 1]); loc.append(1)
            face[2 * ax] = face[2 * ax + 1] = O.PERIODIC

    def take(t):
        d = t.device
        t = t.index_select(1, torch.tensor(idx[2], device=d))
        t = t.index_select(2, torch.tensor(idx[1], device=d))
        return t.index_select(3, torch.tensor(idx[0], device=d)).cpu().numpy()

    bc = O.BC(tuple(face), walls_o.T_wall, walls_o.T_init, walls_o.T_ref, walls_o.gravity_axis)
    return take(f), take(g), (loc[2], loc[1], loc[0]), bc


def sampled_parity(dim, shape, kind, precision, warm_steps, nsamples, seed):
    """Largest |GPU - oracle| over sampled nodes after one step of a full-size box."""
    nz, ny, nx = shape
    lat = "d2q9" if dim == 2 else "d3q27"
    Ra = 1e6 if dim == 3 else 1e8
    wl, wo = walls_pair(kind, dim, seed=seed, perturb=1e-3)
    gpu = L.Lattice(lat, nx, ny, nz, Ra=Ra, Pr=0.71, Ma=0.1, walls=wl, precision=precision)
    ref = O.Oracle(dim, nx, ny, nz, bc=wo, Ra=Ra, Pr=0.71, Ma=0.1, init=False)
    gpu.step(warm_steps)
    f0, g0 = gpu.get_populations(device=True)
    gpu.step(1)
    f1, g1 = gpu.get_populations(device=True)
    gpu.sync()
    worst = 0.0
    for node in synth.sample_nodes(seed, shape, nsamples):
        fb, gb, loc, bc = neighbourhood_box(f0, g0, node, wo, dim)
        bz, by, bx = fb.shape[1:]
        o = O.Oracle(dim, bx, by, bz, bc=bc, om_f=ref.om_f, om_g=ref.om_g, gbeta=ref.gbeta,
                     init=False)
        o.set_state(fb, gb)
        o.step(1)
        fo, go = o.get_state()
        got_f = f1[(slice(None), *node)].cpu().numpy()
        got_g = g1[(slice(None), *node)].cpu().numpy()
        worst = max(worst, np.abs(got_f - fo[(slice(None), *loc)]).max(),
                    np.abs(got_g - go[(slice(None), *loc)]).max())
    del f0, g0, f1, g1
    gpu.close()
    torch.cuda.empty_cache()
    return worst


def test_full_size_sampled_parity_3d_fp32():
    """The bench workload (256^3 cavity, FP32, bench launch shape): 64 sampled nodes, including
    the 8 corners and 6 face centres, after one step from a developed state, against the FP64
    oracle applied to each node's neighbourhood.  FP32 arithmetic on deviations of size <= 0.05
    gives absolute errors of a few 1e-9; bound 1e-7."""
    assert sampled_parity(3, (256, 256, 256), "cavity", "fp32", 200, 64, 3) <= 1e-7


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-14), ("fp32", 1e-7)])
def test_full_size_sampled_parity_2d_rayleigh_benard(precision, tol):
    """The 1024 x 512 Rayleigh-Benard box (periodic x, walls y) after 500 steps."""
    assert sampled_parity(2, (1, 512, 1024), "rb", precision, 500, 64, 4) <= tol


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


def test_cavity_64_fp32_nusselt_within_half_percent():
    gpu, ora = make_pair(2, 64, 64, kind="cavity", precision="fp32", Ra=1e4)
    gpu.step(20000); ora.step(20000)
    gpu.sync()
    assert gpu.nusselt(0)[0] == pytest.approx(ora.nusselt(0)[0], rel=5e-3)


@pytest.mark.parametrize("stochastic,rel", [(1, 0.01), (0, 0.06)])
def test_cavity_64_fp16s_nusselt_stated_accuracy(stochastic, rel):
    """FP16 storage of the deviations.  With round-to-nearest, a population that changes by less
    than half an FP16 step per step stagnates, and the steady state of the rounded iteration
    differs from the exact one (slow diffusive modes): 6 % on <Nu_0>.  Stochastic rounding (the
    default) is unbiased, so those updates accumulate: 1 %."""
    gpu, ora = make_pair(2, 64, 64, kind="cavity", precision="fp16s", Ra=1e4)
    gpu.set_param("fp16_stochastic", stochastic)
    gpu.step(20000); ora.step(20000)
    gpu.sync()
    assert gpu.nusselt(0)[0] == pytest.approx(ora.nusselt(0)[0], rel=rel)


@pytest.mark.parametrize("stochastic", [1, 0])
def test_fp16s_rounding_under_a_small_uniform_force(stochastic):
    """A periodic box at rest under a uniform force F = g beta (T - T_o) = 1e-8: each collision adds
    exactly F to the momentum, so after N steps the mean momentum density is N F.  The per-step
    change of a population is below half an FP16 step of its stored deviation: round-to-nearest
    stagnates, stochastic rounding tracks N F."""
    face = (L.LBM_PERIODIC,) * 6
    lat = L.Lattice("d2q9", 64, 64, 1, Ra=1e4, walls=L.Walls(face, (0,) * 6, 1.5, 0.5, 1),
                    precision="fp16s")
    lat.set_param("fp16_stochastic", stochastic)
    F, N = 1e-8, 20000
    lat.set_param("gbeta", F)                 # T - T_o = 1
    lat.step(N)
    fl = {k: v.cpu().numpy() for k, v in lat.fields().items()}
    j = (fl["uy"] * fl["rho"]).mean() - 0.5 * F  # u carries half of the force of the step
    if stochastic:
        assert j == pytest.approx(N * F, rel=5e-3)
    else:
        assert j < 0.5 * N * F


def test_rayleigh_benard_1024x512_precision_forms():
    """The 1024 x 512 Rayleigh-Benard box at Ra 1e8 (periodic x, seeded +-1e-3 temperature
    perturbation) for 200k steps in FP64, FP32 and FP16S storage.  The flow is chaotic, so the
    three runs decorrelate; the comparison is statistical: the time-averaged wall Nusselt number
    over steps 100k-200k (sampled every 2000 steps, both walls) of FP32 and FP16S within 15 % of
    FP64 (FP64's own 20k-step window means span about +-12 %), and the r.m.s. velocity within 30 %.
    FP16S with round-to-nearest stays conductive (Nu ~ 40, u ~ 1e-4): the buoyancy increments are
    below half an FP16 step, which is why stochastic rounding is the default."""
    def run(prec, stochastic=1):
        lat = L.Lattice("d2q9", 1024, 512, 1, Ra=1e8, Pr=0.71, Ma=0.1,
                        walls=L.Walls.rayleigh_benard(seed=7, perturb=1e-3), precision=prec)
        lat.set_param("fp16_stochastic", stochastic)
        lat.step(100000)
        nu = []
        for _ in range(50):
            lat.step(2000)
            nu.append(0.5 * (lat.nusselt(2)[0] + lat.nusselt(3)[0]))
        fl = {k: v.cpu().numpy() for k, v in lat.fields().items()}
        lat.close()
        return float(np.mean(nu)), float(np.sqrt((fl["ux"] ** 2 + fl["uy"] ** 2).mean()))

    nu64, u64 = run("fp64")
    assert nu64 > 10.0 and u64 > 1e-3           # convection has developed
    for prec in ("fp32", "fp16s"):
        nu, u = run(prec)
        assert nu == pytest.approx(nu64, rel=0.15), prec
        assert u == pytest.approx(u64, rel=0.3), prec
    nu_rn, u_rn = run("fp16s", stochastic=0)
    assert nu_rn > 30.0 and u_rn < 1e-3


@pytest.mark.parametrize("Ra,steps", [(1e3, 100000), (1e4, 150000), (1e5, 350000), (1e6, 500000)])
def test_square_cavity_512_matches_tables_con(Ra, steps):
    """The 512^2 differentially heated cavity (D2Q9 flow + D2Q9 energy, FP32, Ma 0.1) at steady
    state against Tables con1-con4 (512^2, Pr 0.71): hot-wall <Nu_0> within 0.5 % and (Nu_0)_max
    within 0.5 % (at Ra 1e4 also its location y = 0.136 within two nodes); the peak horizontal
    velocity on the vertical centre line and the peak vertical velocity on the horizontal one
    within 1 % (2 % at Ra 1e6), their locations within three nodes.  (Nu_0)_min, near the top
    corner where the edge-link rule of reading R7 acts, within 6 %: at Ma 0.1 (U_o = 0.058, the
    tables use 0.01) it lies 5 % below the table at Ra 1e3 and within 1.3 % above it otherwise;
    the paper's own Mach number is checked in FP64 by the next test."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    lat = L.Lattice("d2q9", 512, 512, 1, Ra=Ra, Pr=0.71, Ma=0.1, walls=L.Walls.cavity(2),
                    precision="fp32")
    lat.step(steps)
    lat.sync()
    mean, nu_max, nu_min, j_max, j_min = lat.nusselt(0)
    inf = lat.info()
    fl = {k: v.cpu().numpy()[0] for k, v in lat.fields().items()}
    lat.close()
    key = {1e3: "1e3", 1e4: "1e4", 1e5: "1e5", 1e6: "1e6"}[Ra]
    assert mean == pytest.approx(gold["nu0_mean_2d_512"][key], rel=5e-3)
    # peak velocities on the centre lines (midway between the two middle node columns / rows),
    # in units of alpha / L, and their locations
    vel = gold["velocity_2d_512"][key]
    scale = inf.L / inf.alpha
    u_c = 0.5 * (fl["ux"][:, 255] + fl["ux"][:, 256]) * scale
    v_c = 0.5 * (fl["uy"][255, :] + fl["uy"][256, :]) * scale
    # at Ra 1e6 the tables' own reference solutions differ from the FPC-LBM column by 0.7 % (u)
    # and 1.7 % (v): the bar there is 2 %
    vrel = 2e-2 if Ra == 1e6 else 1e-2
    assert u_c.max() == pytest.approx(vel["u_max"], rel=vrel)
    assert v_c.max() == pytest.approx(vel["v_max"], rel=vrel)
    assert abs((u_c.argmax() + 0.5) / 512 - vel["y"]) <= 3.0 / 512
    assert abs((v_c.argmax() + 0.5) / 512 - vel["x"]) <= 3.0 / 512
    assert nu_max == pytest.approx(gold["nu0_max_2d_512"][key], rel=5e-3)
    if Ra == 1e4:
        ext = gold["nu0_extremes_2d_512_ra1e4"]
        assert abs((j_max + 0.5) / 512 - ext["y_max"]) <= 2.0 / 512
    assert nu_min == pytest.approx(gold["nu0_extremes_2d_512"][key]["min"], rel=0.06)


def test_square_cavity_512_fp64_at_the_papers_mach_matches_table_con2():
    """Table con2 at the paper's own settings: 512^2, Ra 1e4, Pr 0.71, U_o = 0.01 (Ma = 0.0173),
    FP64 storage, 866,025 steps (0.75 diffusion times L^2 / alpha).  Hot-wall <Nu_0>,
    (Nu_0)_max and (Nu_0)_min within 0.5 %; the minimum at the top node (y = 511.5 / 512 =
    0.9990, as printed), which the edge links of reading R7 decide: with anti-bounce-back on the
    top node's corner link instead, its Nu comes out about 10 % low.  The maximum's location is
    held to five nodes (runs put it about four nodes above the printed 0.136; the table's Ref. 1
    gives 0.149); the centre-line velocity peaks within 1 %, their locations within three
    nodes."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    lat = L.Lattice("d2q9", 512, 512, 1, Ra=1e4, Pr=0.71, Ma=0.01 * 3 ** 0.5,
                    walls=L.Walls.cavity(2), precision="fp64")
    lat.step(866025)
    lat.sync()
    mean, nu_max, nu_min, j_max, j_min = lat.nusselt(0)
    inf = lat.info()
    fl = {k: v.cpu().numpy()[0] for k, v in lat.fields().items()}
    lat.close()
    ext = gold["nu0_extremes_2d_512"]["1e4"]
    assert mean == pytest.approx(gold["nu0_mean_2d_512"]["1e4"], rel=5e-3)
    assert nu_max == pytest.approx(ext["max"], rel=5e-3)
    assert nu_min == pytest.approx(ext["min"], rel=5e-3)
    assert round((j_min + 0.5) / 512, 4) == ext["y_min"]
    assert abs((j_max + 0.5) / 512 - ext["y_max"]) <= 5.0 / 512
    vel = gold["velocity_2d_512"]["1e4"]
    scale = inf.L / inf.alpha
    u_c = 0.5 * (fl["ux"][:, 255] + fl["ux"][:, 256]) * scale
    v_c = 0.5 * (fl["uy"][255, :] + fl["uy"][256, :]) * scale
    assert u_c.max() == pytest.approx(vel["u_max"], rel=1e-2)
    assert v_c.max() == pytest.approx(vel["v_max"], rel=1e-2)
    assert abs((u_c.argmax() + 0.5) / 512 - vel["y"]) <= 3.0 / 512
    assert abs((v_c.argmax() + 0.5) / 512 - vel["x"]) <= 3.0 / 512


@pytest.mark.parametrize("Ra,steps,walls_rel", [(1e5, 200000, 2e-3), (1e6, 250000, 2e-3),
                                               (1e7, 300000, 5e-3)])
def test_cubic_cavity_128_matches_table_compare_nu3d(Ra, steps, walls_rel):
    """128^3 cubic cavity (D3Q27 flow + D3Q15 energy, FP32, Ma 0.1) at steady state against the
    hot-wall <Nu> of Table CompareNu3D (128^3, U_o = 0.01): within 1 %; hot and cold wall agree
    within 0.2 % (0.5 % at Ra 1e7, whose thinner boundary layers take longer to settle: after
    300k steps the hot wall is within 0.06 % of its 800k-step value).  This pins the D3Q27
    reading of the flow collision against the paper's own 3D results."""
    import json, os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    lat = L.Lattice("d3q27", 128, 128, 128, Ra=Ra, Pr=0.71, Ma=0.1, walls=L.Walls.cavity(3),
                    precision="fp32")
    lat.step(steps)
    lat.sync()
    hot, cold = lat.nusselt(0)[0], lat.nusselt(1)[0]
    lat.close()
    key = {1e5: "1e5", 1e6: "1e6", 1e7: "1e7"}[Ra]
    assert hot == pytest.approx(gold["nu_mean_3d"][key], rel=0.01)
    assert cold == pytest.approx(hot, rel=walls_rel)


@pytest.mark.parametrize("precision", ["fp32", "fp16s"])
@pytest.mark.parametrize("shape", [(9, 13, 70), (6, 8, 40)])
def test_rows_per_thread_give_identical_states(shape, precision):
    """The 3D FP32 / FP16S step lets each thread update 1, 2 or 4 rows of its column in turn
    ("rows3d"); every node runs the same arithmetic, so the populations are bitwise equal, also
    when the row count does not divide ny (13 rows)."""
    nz, ny, nx = shape
    lats = []
    for rows in (1, 2, 4):
        lt = L.Lattice("d3q27", nx, ny, nz, Ra=1e5, walls=L.Walls.cavity(3), precision=precision)
        lt.set_param("rows3d", rows)
        lats.append(lt)
    f, g = lats[0].get_populations()
    f = synth.perturbed(f, 81, 0.05)
    g = synth.perturbed(g, 82, 0.05)
    for lt in lats:
        lt.set_populations(f, g)
        lt.step(30)
        lt.sync()
    ref = lats[0].get_populations()
    for lt in lats[1:]:
        fo, go = lt.get_populations()
        assert np.array_equal(fo, ref[0]) and np.array_equal(go, ref[1])
    with pytest.raises(L.LbmError):
        lats[0].set_param("rows3d", 3)
    for lt in lats:
        lt.close()


@pytest.mark.parametrize("dim,shape", [(2, (1, 40, 70)), (3, (9, 12, 20))])
def test_graph_replay_equals_plain_launches(dim, shape):
    """lbm_step replays runs of graph_steps steps from a CUDA graph; the state must be bit-for-bit
    the one of plain launches, also after a parameter change invalidates the graph."""
    nz, ny, nx = shape
    lat = "d2q9" if dim == 2 else "d3q27"
    a = L.Lattice(lat, nx, ny, nz, Ra=1e5, walls=L.Walls.cavity(dim), precision="fp32")
    b = L.Lattice(lat, nx, ny, nz, Ra=1e5, walls=L.Walls.cavity(dim), precision="fp32")
    b.set_param("graph_steps", 0)
    assert a.info().graph_steps == 32 and b.info().graph_steps == 0
    for lt in (a, b):
        lt.step(77)
        lt.set_param("gbeta", 2.5e-3)
        lt.step(45)
        lt.sync()
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    assert a.info().steps == b.info().steps == 122


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16s"])
@pytest.mark.parametrize("dim,shape,tma", [(2, (1, 40, 70), 0), (3, (9, 14, 40), 0), (3, (9, 14, 40), 2)])
def test_64bit_offsets_match_32bit(dim, shape, tma, precision):
    """Boxes with q n >= 2^32 nodes x links (above 541^3 for D3Q27) run the 64-bit-offset
    instantiation of the step.  Forced on a small box (index64 = 1), through walls and the
    interior, it must give bitwise the populations of the 32-bit form (also on the TMA-staged
    path)."""
    if tma and precision == "fp64":
        pytest.skip("the TMA-staged step covers FP32 and FP16S")
    nz, ny, nx = shape
    lat = "d2q9" if dim == 2 else "d3q27"
    a = L.Lattice(lat, nx, ny, nz, Ra=1e5, walls=L.Walls.cavity(dim), precision=precision)
    b = L.Lattice(lat, nx, ny, nz, Ra=1e5, walls=L.Walls.cavity(dim), precision=precision)
    f, g = a.get_populations()
    f = synth.perturbed(f, 71, 0.05)
    g = synth.perturbed(g, 72, 0.05)
    for lt in (a, b):
        lt.set_populations(f, g)
        if tma:
            lt.set_param("tma_rows", tma)
    b.set_param("index64", 1)
    with pytest.raises(L.LbmError):
        b.set_param("index64", 2)
    for lt in (a, b):
        lt.step(40)
        lt.sync()
    fa, ga = a.get_populations()
    fb, gb = b.get_populations()
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    a.close()
    b.close()
