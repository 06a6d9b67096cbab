"""The adjoint step (lbm_adjoint_step) against finite differences.

  * Small cavity, FP64: every component of dJ/dT_w against central differences of the FP64 oracle,
    within 1e-6 relative.  The gradients here are ~4e-6 while J carries ~1e-14 of rounding noise
    from its 150 steps, so the differences use h = 1e-2: the noise over 2h is then 5e-13, and the
    truncation (third derivative times h^2 / 6) stays below 1e-8 of the gradient (central
    differences with h from 1e-2 to 1e-3 agree to that level).
  * The 256^2, Ra = 1e5, 2000-step workload with an FP32 forward and FP64 adjoint: directional
    derivatives against central differences of the FP64 GPU forward (h = 1e-4), within 1e-4.
  * The FP32 adjoint arithmetic (adjoint_fp64 = 0) against the FP64 default on that workload.
  * The torch.autograd.Function wrapper returns the same gradient.
"""
import numpy as np
import pytest

from oracle import oracle as O
from tests import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2504_09041_gb300 import lbm as L  # noqa: E402

HOT, COLD = 0, 1


def oracle_J(nx, ny, Ra, prof, steps):
    o = O.Oracle(2, nx, ny, bc=O.cavity_bc(2), Ra=Ra, Pr=0.71, Ma=0.1)
    o.set_wall_profile(HOT, prof)
    o.step(steps)
    return o.nusselt(COLD)[0]


def test_adjoint_matches_oracle_finite_differences():
    nx, ny, steps, Ra, h = 24, 20, 150, 1e5, 1e-2
    prof = synth.sine_profile(5, ny)
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp64")
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


def test_adjoint_handles_uneven_segments_and_fp32():
    """47 steps (segments of 7, the last one shorter), FP32 states and FP64 adjoint, against the
    FP64 adjoint on the same problem."""
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


def test_adjoint_256_2000_steps_matches_central_differences():
    """The adjoint workload: 256^2 cavity, Ra 1e5, 2000 steps, hot-wall profile 1 + 0.05 * seeded
    sine modes, J = mean cold-wall Nu; FP32 forward, FP64 adjoint; FD of the FP64 forward."""
    nx = ny = 256
    steps, Ra, h = 2000, 1e5, 1e-4
    prof = synth.sine_profile(2024, ny)
    lat = L.Lattice("d2q9", nx, ny, Ra=Ra, walls=L.Walls.cavity(2), precision="fp32")
    lat.set_wall_profile(HOT, prof)
    J, grad = lat.adjoint(steps, COLD, HOT)
    rng = np.random.default_rng(9)
    dirs = [rng.uniform(-1, 1, ny), rng.uniform(-1, 1, ny), np.eye(ny)[37], np.eye(ny)[200]]
    for v in dirs:
        fd = (gpu_J(nx, ny, Ra, prof + h * v, steps) - gpu_J(nx, ny, Ra, prof - h * v, steps)) / (2 * h)
        assert grad @ v == pytest.approx(fd, rel=1e-4)


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
