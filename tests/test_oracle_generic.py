"""The generic-form 2D oracle (oracle/generic2d.py) against the printed-form C oracle, and its
complex-step derivative against finite differences (CPU only).

The two oracles are independent restatements: one takes the paper's printed Steps 1-5, the other
the moment definitions and a linear solve per node.  Agreement to rounding after many steps of
every wall and force configuration pins each against the other.  The complex-step derivative of
the generic oracle is the oracle of the adjoint.
"""
import numpy as np
import pytest

from oracle import generic2d as G
from oracle import oracle as O
from tests import synth


def make_pair(nx, ny, bc, Ra=1e5, rates_seed=None, g_option=0, gbeta=None, dtype=np.float64):
    if rates_seed is None:
        ora = O.Oracle(2, nx, ny, bc=bc, Ra=Ra, Pr=0.71, Ma=0.1, g_option=g_option)
    else:
        om_f = synth.rates(rates_seed, 9, 0.6, 1.9)
        om_g = synth.rates(rates_seed + 1, 9, 0.6, 1.9)
        ora = O.Oracle(2, nx, ny, bc=bc, om_f=om_f, om_g=om_g, gbeta=gbeta, g_option=g_option)
    gen = G.Generic2D(nx, ny, bc.face, bc.T_wall, bc.T_ref, ora.gbeta, bc.gravity_axis, ora.om_f,
                      ora.om_g, g_option, dtype=dtype)
    return ora, gen


def randomize(ora, gen, seed, scale):
    f, g = ora.get_state()
    f = synth.perturbed(f, seed, scale)
    g = synth.perturbed(g, seed + 1, scale)
    ora.set_state(f, g)
    gen.set_state(f, g)


def state_error(ora, gen):
    f, g = ora.get_state()
    return max(np.abs(f.reshape(gen.f.shape) - gen.f).max(), np.abs(g.reshape(gen.g.shape) - gen.g).max())


@pytest.mark.parametrize("g_option", [0, 1])
@pytest.mark.parametrize("kind", ["cavity", "rb", "periodic"])
def test_generic_oracle_equals_printed_oracle(kind, g_option):
    nx, ny = 23, 17
    if kind == "cavity":
        bc = O.cavity_bc(2)
    elif kind == "rb":
        bc = O.rayleigh_benard_bc(seed=3, perturb=1e-3)
    else:
        bc = O.BC((O.PERIODIC,) * 6, (0,) * 6, 0.5, 0.5, 1)
    ora, gen = make_pair(nx, ny, bc, rates_seed=90 + g_option, g_option=g_option, gbeta=3e-3)
    randomize(ora, gen, 11, 0.3)
    if kind == "cavity":
        prof = synth.sine_profile(4, ny)
        ora.set_wall_profile(0, prof)
        gen.set_wall_profile(0, prof)
    ora.step(1)
    gen.step(1)
    assert state_error(ora, gen) <= 1e-14
    ora.step(40)
    gen.step(40)
    assert state_error(ora, gen) <= 1e-12
    if kind != "periodic":
        face = 0 if kind == "cavity" else 2
        assert gen.nusselt_mean(face, ora.L, ora.dT) == pytest.approx(ora.nusselt(face)[0], abs=1e-12)


def test_complex_step_run_has_the_real_run_as_its_real_part():
    nx, ny = 16, 12
    bc = O.cavity_bc(2)
    _, real = make_pair(nx, ny, bc)
    ora, cplx = make_pair(nx, ny, bc, dtype=np.complex128)
    f, g = ora.get_state()
    real.set_state(f, g)
    cplx.set_state(f, g)
    prof = synth.sine_profile(5, ny)
    v = np.random.default_rng(1).uniform(-1, 1, ny)
    real.set_wall_profile(0, prof)
    cplx.set_wall_profile(0, prof + 1e-20j * v)
    real.step(30)
    cplx.step(30)
    assert np.abs(cplx.f.real - real.f).max() <= 1e-15
    assert np.abs(cplx.g.real - real.g).max() <= 1e-15


def test_complex_step_derivative_matches_finite_differences_of_the_c_oracle():
    """dJ/dT_w . v by complex step against central differences of the printed-form oracle
    (h = 1e-2, whose truncation and noise are below 1e-7 of the derivative here)."""
    nx, ny, steps = 16, 12, 60
    bc = O.cavity_bc(2)
    prof = synth.sine_profile(5, ny)
    v = np.random.default_rng(2).uniform(-1, 1, ny)

    def c_J(p):
        o = O.Oracle(2, nx, ny, bc=bc, Ra=1e5, Pr=0.71, Ma=0.1)
        o.set_wall_profile(0, p)
        o.step(steps)
        return o.nusselt(1)[0]

    ora, cplx = make_pair(nx, ny, bc, dtype=np.complex128)
    f, g = ora.get_state()
    cplx.set_state(f, g)
    h = 1e-20
    cplx.set_wall_profile(0, prof + 1j * h * v)
    cplx.step(steps)
    d_cs = cplx.nusselt_mean(1, ora.L, ora.dT).imag / h
    hd = 1e-2
    d_fd = (c_J(prof + hd * v) - c_J(prof - hd * v)) / (2 * hd)
    assert d_cs == pytest.approx(d_fd, rel=1e-6)
