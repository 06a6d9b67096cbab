"""The adjoint step (lbm_adjoint_step) against finite differences.

  * Small cavity, FP64: every component of dJ/dT_w against central differences of the FP64 oracle,
    within 1e-6 relative.  The gradients here are ~4e-6 while J carries ~1e-14 of rounding noise
    from its 150 steps, so the differences use h = 1e-2: the noise over 2h is then 5e-13, and the
    truncation (third derivative times h^2 / 6) stays below 1e-8 of the gradient (central
    differences with h from 1e-2 to 1e-3 agree to that level).
  * The 256^2, Ra = 1e5, 2000-step workload, FP64 adjoint: directional derivatives against
    central differences of the FP64 GPU forward.  Two random directions use h = 1e-4.  Along a
    unit direction J moves by only ~1e-11 over 2h = 2e-4, so a few ulps of rounding in J
    (~6e-15) would already be 3e-4 of that difference; those directions use h = 1e-2, where the
    difference is 100 times larger and the truncation error stays below 1e-8 (as on the small
    cavity).  With FP64 forward states each directional derivative is within 1e-4 relative.  With FP32 forward states the adjoint
    linearises about the FP32 trajectory, whose rounding moves the smallest gradient components
    by a few 1e-4 of themselves; there the error of each directional derivative is bounded by
    1e-4 of its Cauchy-Schwarz scale |grad| |v| (the relative error of the gradient vector).
  * The FP32 adjoint arithmetic (adjoint_fp64 = 0) against the FP64 adjoint on that workload.
  * Double-float arithmetic (adjoint_arith = 2, pairs of FP32 numbers with a 48-bit significand)
    is held to every FP64 bar above, and to the FP64 adjoint's gradient within 1e-10 of its
    largest component on the 2000-step workload.
  * The torch.autograd.Function wrapper returns the same gradient.
  * The oracle adjoint: directional derivatives of the generic-form oracle by complex step, exact
    to rounding, against the GPU gradient (FP64 states) within 1e-8 relative, options A and B.
"""
import numpy as np
import pytest

from oracle import generic2d as GEN
from oracle import oracle as O
from tests import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402

HOT, COLD = 0, 1
# adjoint arithmetic held to the FP64 bars: 1 = FP64, 2 = double-float (FP32 pairs)
ARITH = [1, 2]


def oracle_J(nx, ny, Ra, prof, steps):
    o = O.Oracle(2, nx, ny, bc=O.cavity_bc(2), Ra=Ra, Pr=0.71, Ma=0.1)
    o.set_wall_profile(HOT, prof)
    o.step(steps)
    return o.nusselt(COLD)[0]


@pytest.mark.parametrize("arith", ARITH)
def test_adjoint_matches_oracle_finite_differences(arith):
    nx, ny, steps, Ra, h = 24, 20, 150, 1e5, 1e-2
    prof = synth.sine_profile(5, ny)
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
    lat.set_param("adjoint_arith", arith)
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)
    assert J == pytest.approx(oracle_J(nx, ny, Ra, prof, steps), abs=1e-11)
    fd = np.zeros(ny)
    for j in range(ny):
        e = np.zeros(ny); e[j] = h
        fd[j] = (oracle_J(nx, ny, Ra, prof + e, steps) - oracle_J(nx, ny, Ra, prof - e, steps)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("arith", ARITH)
def test_adjoint_option_b_matches_oracle_finite_differences(arith):
    """The option-B energy attractors (Eq. MvT2DoptionB) with second-order energy rates away from
    1, so that they differ from option A: adjoint against oracle central differences."""
    nx, ny, steps, Ra, h = 22, 18, 120, 1e5, 1e-2
    prof = synth.sine_profile(6, ny)
    o0 = O.Oracle(2, nx, ny, bc=O.cavity_bc(2), Ra=Ra, Pr=0.71, Ma=0.1)
    om_g = o0.om_g.copy()
    om_g[3:6] = (1.3, 0.8, 1.6)

    def J_of(p):
        o = O.Oracle(2, nx, ny, bc=O.cavity_bc(2), Ra=Ra, Pr=0.71, Ma=0.1, om_g=om_g, g_option=1)
        o.set_wall_profile(HOT, p)
        o.step(steps)
        return o.nusselt(COLD)[0]

    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
    lat.set_omegas(None, om_g)
    lat.set_param("g_attractors", 1)
    lat.set_param("adjoint_arith", arith)
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)
    assert J == pytest.approx(J_of(prof), abs=1e-11)
    fd = np.zeros(ny)
    for j in range(ny):
        e = np.zeros(ny); e[j] = h
        fd[j] = (J_of(prof + e) - J_of(prof - e)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("g_option", [0, 1])
def test_adjoint_matches_the_complex_step_oracle(g_option, arith):
    """grad . v from lbm_adjoint_step against Im(J(T_w + i h v)) / h of the generic-form oracle."""
    nx, ny, steps, Ra = 24, 20, 150, 1e5
    bc = O.cavity_bc(2)
    prof = synth.sine_profile(7, ny)
    ora = O.Oracle(2, nx, ny, bc=bc, Ra=Ra, Pr=0.71, Ma=0.1)
    om_g = ora.om_g.copy()
    if g_option:
        om_g[3:6] = (1.3, 0.8, 1.6)    # second-order energy rates away from 1: options differ
    f0, g0 = ora.get_state()

    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
    lat.set_omegas(None, om_g)
    lat.set_param("g_attractors", g_option)
    lat.set_param("adjoint_arith", arith)
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)

    rng = np.random.default_rng(17)
    dirs = [rng.uniform(-1, 1, ny), np.eye(ny)[3], np.eye(ny)[ny // 2]]
    h = 1e-20
    for v in dirs:
        gen = GEN.Generic2D(nx, ny, bc.face, bc.T_wall, bc.T_ref, ora.gbeta, bc.gravity_axis, ora.om_f,
                            om_g, g_option, dtype=np.complex128)
        gen.set_state(f0, g0)
        gen.set_wall_profile(HOT, prof + 1j * h * v)
        gen.step(steps)
        Jc = gen.nusselt_mean(COLD, ora.L, ora.dT)
        assert Jc.real == pytest.approx(J, abs=1e-11)
        assert grad @ v == pytest.approx(Jc.imag / h, rel=1e-8)


@pytest.mark.parametrize("steps,overlap", [(144, 1), (144, 0), (4, 1), (1, 1)])
def test_adjoint_segment_layouts_match_the_complex_step_oracle(steps, overlap):
    """The backward pass's bookkeeping for other segment layouts: 144 steps are 12 full segments
    of an even length (adjoint graphs that keep the buffer parity), with and without the
    recompute overlapped on the second stream; 4 steps are two segments of 2 (no recompute
    graph); 1 step has no segment to recompute.  Directional derivative against the generic-form
    oracle's complex step, 1e-8 relative."""
    nx, ny, Ra = 22, 18, 1e5
    bc = O.cavity_bc(2)
    prof = synth.sine_profile(9, ny)
    ora = O.Oracle(2, nx, ny, bc=bc, Ra=Ra, Pr=0.71, Ma=0.1)
    f0, g0 = ora.get_state()
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
    lat.set_param("adjoint_overlap", overlap)
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)
    lat.close()
    v = np.random.default_rng(23).uniform(-1, 1, ny)
    h = 1e-20
    gen = GEN.Generic2D(nx, ny, bc.face, bc.T_wall, bc.T_ref, ora.gbeta, bc.gravity_axis, ora.om_f,
                        ora.om_g, 0, dtype=np.complex128)
    gen.set_state(f0, g0)
    gen.set_wall_profile(HOT, prof + 1j * h * v)
    gen.step(steps)
    Jc = gen.nusselt_mean(COLD, ora.L, ora.dT)
    assert Jc.real == pytest.approx(J, abs=1e-11)
    assert grad @ v == pytest.approx(Jc.imag / h, rel=1e-8)


def test_adjoint_handles_uneven_segments_and_fp32():
    """47 steps (segments of 7, the last one shorter), FP32 states against FP64 states on the same
    problem (default adjoint arithmetic)."""
    nx, ny = 30, 26
    prof = synth.sine_profile(8, ny)
    grads = {}
    for prec in ("fp64", "fp32"):
        lat = L.Lattice("d2q9", nx, ny, Ra=1e5, walls=L.Walls.cavity(2), precision=prec)
        lat.set_wall_profile(HOT, prof)
        grads[prec] = lat.adjoint(47, COLD, HOT)[1]
    np.testing.assert_allclose(grads["fp32"], grads["fp64"], rtol=0,
                               atol=1e-5 * np.abs(grads["fp64"]).max())


def gpu_J(nx, ny, Ra, prof, steps, precision="fp64"):
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision=precision)
    lat.set_wall_profile(HOT, prof)
    lat.step(steps)
    J = lat.nusselt(COLD)[0]
    lat.close()
    return J


@pytest.fixture(scope="module")
def workload_fd():
    """Central differences of the FP64 forward of the 256^2 adjoint workload along two random
    directions (h = 1e-4) and two unit directions (h = 1e-2)."""
    nx = ny = 256
    steps, Ra = 2000, 1e5
    prof = synth.sine_profile(2024, ny)
    rng = np.random.default_rng(9)
    dirs = [(rng.uniform(-1, 1, ny), 1e-4), (rng.uniform(-1, 1, ny), 1e-4),
            (np.eye(ny)[37], 1e-2), (np.eye(ny)[200], 1e-2)]
    fds = [(gpu_J(nx, ny, Ra, prof + h * v, steps) - gpu_J(nx, ny, Ra, prof - h * v, steps)) / (2 * h)
           for v, h in dirs]
    return prof, [v for v, _ in dirs], fds


@pytest.mark.parametrize("arith", ARITH)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_256_2000_steps_matches_central_differences(precision, arith, workload_fd):
    """The adjoint workload: 256^2 cavity, Ra 1e5, 2000 steps, hot-wall profile 1 + 0.05 * seeded
    sine modes, J = mean cold-wall Nu; FP64 adjoint accumulation; FD of the FP64 forward."""
    nx = ny = 256
    steps, Ra = 2000, 1e5
    prof, dirs, fds = workload_fd
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision=precision)
    lat.set_param("adjoint_arith", arith)
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)
    gn = np.linalg.norm(grad)
    for v, fd in zip(dirs, fds):
        if precision == "fp64":
            assert grad @ v == pytest.approx(fd, rel=1e-4)
        else:
            assert abs(grad @ v - fd) <= 1e-4 * gn * np.linalg.norm(v)


@pytest.fixture(scope="module")
def workload_fd_full():
    """All 256 central differences dJ/dT_w(j) of the 256^2 adjoint workload, from the FP64 forward
    on the GPU, at h = 1e-2 and at the configured h = 1e-4 (one handle, its state reset before every
    run)."""
    nx = ny = 256
    steps, Ra = 2000, 1e5
    prof = synth.sine_profile(2024, ny)
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
    state0 = lat.get_state()

    def J(p):
        lat.set_state(state0)
        lat.set_wall_profile(HOT, p)
        lat.step(steps)
        return lat.nusselt(COLD)[0]

    J0 = J(prof)
    assert J(prof) == J0                     # the forward is deterministic
    fd = {}
    for h in (1e-2, 1e-4):
        d = np.zeros(ny)
        for j in range(ny):
            e = np.zeros(ny)
            e[j] = h
            d[j] = (J(prof + e) - J(prof - e)) / (2 * h)
        fd[h] = d
    lat.close()
    return prof, fd


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_256_whole_gradient_matches_central_differences(precision, workload_fd_full):
    """The whole design gradient of the adjoint workload (256^2, Ra 1e5, 2000 steps, default
    double-float VJPs with FP64 accumulation) against all 256 central differences of the FP64
    forward: ||g - g_FD|| / ||g_FD|| <= 1e-4, at h = 1e-2 and at h = 1e-4.
    Noise of the differences: J (~6.85) carries a few 1e-15 of rounding from 2000 steps, which over
    2h is 3e-11 per component at h = 1e-4 (components are ~4e-7, so 1e-4 of each) and 3e-13 at
    h = 1e-2; the truncation error of h = 1e-2 (h^2 / 6 times the third derivative) stays below 1e-8
    of the gradient, as on the small cavity.  Per component, every difference at h = 1e-2 larger
    than 1e-3 of the largest (all but the few near sign changes, far above the 3e-13 floor) is
    matched within 1e-4 of itself (FP64 states) or within 1e-4 of the largest (FP32 states, which
    the adjoint linearises about; their rounding moves small components by a few 1e-4 of
    themselves)."""
    prof, fd = workload_fd_full
    lat = L.Lattice("d2q9", 256, 256, Ra=1e5, walls=L.Walls.cavity(2), precision=precision)
    lat.set_wall_profile(HOT, prof)
    _, g = lat.adjoint(2000, COLD, HOT)
    lat.close()
    for h, d in fd.items():
        rel = np.linalg.norm(g - d) / np.linalg.norm(d)
        print(f"{precision} h={h:g}: ||g - fd|| / ||fd|| = {rel:.3e}")
        assert rel <= 1e-4, (h, rel)
    d = fd[1e-2]
    big = np.abs(d) > 1e-3 * np.abs(d).max()
    assert big.sum() >= 200
    err = np.abs(g - d)[big]
    worst = (err / np.abs(d[big])).max()
    print(f"{precision}: per-component worst |g - fd| / |fd| = {worst:.3e} over {big.sum()} components")
    if precision == "fp64":
        assert worst <= 1e-4
    else:
        assert err.max() <= 1e-4 * np.abs(d).max()


def test_torch_autograd_function_returns_the_adjoint_gradient():
    nx, ny, steps = 28, 24, 60
    lat = L.Lattice("d2q9", nx, ny, Ra=1e5, walls=L.Walls.cavity(2), precision="fp64")
    state0 = lat.get_state()
    fn = L.wall_nusselt_objective(lat, state0, steps, COLD, HOT)
    T_w = torch.tensor(synth.sine_profile(3, ny), dtype=torch.float64, requires_grad=True)
    J = fn(T_w)
    J.backward()
    lat.set_state(state0)
    lat.set_wall_profile(HOT, T_w.detach().numpy())
    J2, grad = lat.adjoint(steps, COLD, HOT)
    assert float(J.detach()) == pytest.approx(J2, abs=1e-13)
    np.testing.assert_allclose(T_w.grad.numpy(), grad, rtol=0, atol=1e-14)
    # one directional derivative by central differences of the same function
    v = torch.tensor(np.random.default_rng(1).uniform(-1, 1, ny))
    h = 1e-2
    fd = (float(fn(T_w.detach() + h * v)) - float(fn(T_w.detach() - h * v))) / (2 * h)
    assert float(T_w.grad @ v) == pytest.approx(fd, rel=1e-6)


def test_fp32_adjoint_arithmetic_stated_accuracy():
    """adjoint_fp64 = 0: the vector-Jacobian products in FP32 (FP64 gradient accumulation).  On the
    256^2, 2000-step workload its gradient stays within 1e-4 of the FP64 adjoint's (relative to the
    largest component; 7e-5 measured)."""
    nx = ny = 256
    prof = synth.sine_profile(2024, ny)
    grads = {}
    for flag in (1, 0):
        lat = L.Lattice("d2q9", nx, ny, Ra=1e5, walls=L.Walls.cavity(2), precision="fp32")
        lat.set_wall_profile(HOT, prof)
        lat.set_param("adjoint_fp64", flag)
        grads[flag] = lat.adjoint(2000, COLD, HOT)[1]
        lat.close()
    np.testing.assert_allclose(grads[0], grads[1], rtol=0, atol=1e-4 * np.abs(grads[1]).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_double_float_adjoint_equals_fp64_adjoint(precision):
    """adjoint_arith = 2 against the FP64 adjoint on the 256^2, 2000-step workload: the gradients
    agree within 1e-10 of the largest component (each VJP operation carries a relative error of a
    few 2^-48, and the adjoint is linear in mu, so the difference stays at that level)."""
    nx = ny = 256
    prof = synth.sine_profile(2024, ny)
    grads = {}
    for arith in (1, 2):
        lat = L.Lattice("d2q9", nx, ny, Ra=1e5, walls=L.Walls.cavity(2), precision=precision)
        lat.set_wall_profile(HOT, prof)
        lat.set_param("adjoint_arith", arith)
        grads[arith] = lat.adjoint(2000, COLD, HOT)[1]
        lat.close()
    scale = np.abs(grads[1]).max()
    err = np.abs(grads[2] - grads[1]).max()
    assert err <= 1e-10 * scale, err / scale


def test_adjoint_arith_rejects_unknown_values():
    lat = L.Lattice("d2q9", 16, 12, Ra=1e4, walls=L.Walls.cavity(2), precision="fp32")
    for bad in (3, 1.5, -1):
        with pytest.raises(L.LbmError):
            lat.set_param("adjoint_arith", bad)
    lat.set_param("adjoint_arith", 2)
    lat.close()
