"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Every check here is independent of the oracle's own formulas:
  * moments are recomputed from their definitions as sums over the printed velocity sets
    (Sec. 4.2 discrete moment definitions; Sec. 5.2; Sec. 5.4);
  * attractors are regenerated from the recurrence (Eqs. Mvcmattractor2D, Mvcmattractor3D,
    Mvcmattractor2D_g, Mvcmattractor3Dg) with the diffusion-tensor selection rules
    (Eqs. Dij2Dselection, diffusion-tensor-parameter-3D, option A for g);
  * the whole collision is checked black-box as a relaxation in moment space
    (Eqs. FPcollision, FPcollision_g, FPcoll3d, FPcoll3dg with the sources of Eqs. sourceCM2D /
    forcing:3D);
  * rest states reproduce the textbook D2Q9 / D3Q15 / D3Q27 weights;
  * shear and thermal waves decay at nu k^2 and alpha k^2 with the rates of App. A/B/C;
  * pure conduction between fixed-temperature walls is linear with Nu = 1;
  * the 64^2 Ra = 1e4 cavity lands within a few percent of the printed Table con2 values.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------------------------
# Independent helpers (definitions written out, no oracle code)
# ---------------------------------------------------------------------------------------------

def moments_by_definition(pops, E, M, u=(0.0, 0.0, 0.0)):
    """kappa_mnp = sum_a pops_a (e_ax - ux)^m (e_ay - uy)^n (e_az - uz)^p."""
    d = E - np.asarray(u)[None, :]
    out = np.zeros(len(M))
    for j, (m, n, p) in enumerate(M):
        out[j] = np.sum(pops * d[:, 0] ** m * d[:, 1] ** n * d[:, 2] ** p)
    return out


def recurrence_attractor(mnp, lower, D):
    """Eqs. Mvcmattractor2D / Mvcmattractor3D: Pi^Mv_mnp from lower moments and D'.

    lower: dict (m, n, p) -> value of the lower central moment used on the right-hand side.
    D: dict with keys 'xx', 'yy', 'zz', 'xy', 'xz', 'yz'.
    """
    m, n, p = mnp
    s = m + n + p
    get = lambda a, b, c: lower.get((a, b, c), 0.0) if min(a, b, c) >= 0 else 0.0
    return (m * (m - 1) / s * D["xx"] * get(m - 2, n, p)
            + n * (n - 1) / s * D["yy"] * get(m, n - 2, p)
            + p * (p - 1) / s * D["zz"] * get(m, n, p - 2)
            + 2 * m * n / s * D["xy"] * get(m - 1, n - 1, p)
            + 2 * n * p / s * D["yz"] * get(m, n - 1, p - 1)
            + 2 * m * p / s * D["xz"] * get(m - 1, n, p - 1))


def random_pops(rng, base, scale):
    return base * (1.0 + scale * rng.uniform(-1, 1, base.size))


# ---------------------------------------------------------------------------------------------
# Lattices and rest states
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("E,q", [(O.E_D2Q9, 9), (O.E_D3Q27, 27), (O.E_D3Q15, 15)])
def test_velocity_sets_unique_and_symmetric(E, q):
    assert E.shape == (q, 3)
    assert len({tuple(e) for e in E}) == q
    for e in E:
        assert any((E == -e).all(axis=1))


def test_rest_states_are_textbook_weights():
    w9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    w15 = np.array([2 / 9] + [1 / 9] * 6 + [1 / 72] * 8)
    w27 = np.array([8 / 27] + [2 / 27] * 6 + [1 / 54] * 12 + [1 / 216] * 8)
    np.testing.assert_allclose(O.equilibrium_f(2, 1.0), w9, atol=1e-15)
    np.testing.assert_allclose(O.equilibrium_g(2, 1.0), w9, atol=1e-15)
    np.testing.assert_allclose(O.equilibrium_g(3, 1.0), w15, atol=1e-15)
    np.testing.assert_allclose(O.equilibrium_f(3, 1.0), w27, atol=1e-15)
    # isotropy of the weights: sum w e_i e_j = delta_ij / 3
    for E, w in [(O.E_D2Q9, w9), (O.E_D3Q15, w15), (O.E_D3Q27, w27)]:
        np.testing.assert_allclose(np.einsum("a,ai,aj->ij", w, E, E)[:2, :2], np.eye(2) / 3,
                                   atol=1e-15)


def test_equilibrium_moments_are_the_attractors():
    rng = np.random.default_rng(1)
    u = rng.uniform(-0.1, 0.1, 3)
    f = O.equilibrium_f(2, 1.3, u[:2])
    k = moments_by_definition(f, O.E_D2Q9, O.M_D2Q9, (u[0], u[1], 0))
    cs2 = 1 / 3
    np.testing.assert_allclose(k, [1.3, 0, 0, cs2 * 1.3, cs2 * 1.3, 0, 0, 0, cs2 * cs2 * 1.3],
                               atol=1e-14)


# ---------------------------------------------------------------------------------------------
# Transforms: printed Steps 1, 2, 4, 5 against definitions and as exact inverses
# ---------------------------------------------------------------------------------------------

def test_d2q9_steps_against_definitions():
    rng = np.random.default_rng(2)
    for _ in range(20):
        f = rng.uniform(0.0, 1.0, 9)
        ux, uy = rng.uniform(-0.3, 0.3, 2)
        r = O.d2q9_step1(f)
        np.testing.assert_allclose(r, moments_by_definition(f, O.E_D2Q9, O.M_D2Q9), atol=1e-14)
        c = O.d2q9_step2(r, ux, uy)
        np.testing.assert_allclose(c, moments_by_definition(f, O.E_D2Q9, O.M_D2Q9, (ux, uy, 0)),
                                   atol=1e-14)
        np.testing.assert_allclose(O.d2q9_step4(c, ux, uy), r, atol=1e-14)
        np.testing.assert_allclose(O.d2q9_step5(r), f, atol=1e-14)


def test_d3q15_steps_against_definitions():
    rng = np.random.default_rng(3)
    P = np.array([[e[0] ** m * e[1] ** n * e[2] ** p for e in O.E_D3Q15] for m, n, p in O.M_D3Q15],
                 dtype=float)
    assert np.linalg.matrix_rank(P) == 15
    for _ in range(20):
        g = rng.uniform(0.0, 1.0, 15)
        u = rng.uniform(-0.3, 0.3, 3)
        r = O.d3q15_step1(g)
        np.testing.assert_allclose(r, P @ g, atol=1e-14)
        c = O.d3q15_step2(r, *u)
        # central moments by definition on the lattice (this includes the aliasing of
        # e_x^2 e_y with e_y e_z^2 on D3Q15 that Step 2 relies on)
        np.testing.assert_allclose(c, moments_by_definition(g, O.E_D3Q15, O.M_D3Q15, u),
                                   atol=1e-14)
        np.testing.assert_allclose(O.d3q15_step4(c, *u), r, atol=1e-14)
        np.testing.assert_allclose(O.d3q15_step5(r), np.linalg.solve(P, r), atol=1e-14)
        np.testing.assert_allclose(O.d3q15_step5(r), g, atol=1e-14)


def test_d3q27_transforms_against_definitions():
    rng = np.random.default_rng(4)
    P = np.array([[e[0] ** m * e[1] ** n * e[2] ** p for e in O.E_D3Q27] for m, n, p in O.M_D3Q27],
                 dtype=float)
    for _ in range(10):
        f = rng.uniform(0.0, 1.0, 27)
        u = rng.uniform(-0.3, 0.3, 3)
        r = O.d3q27_raw(f)
        np.testing.assert_allclose(r, P @ f, atol=1e-14)
        k = O.d3q27_central(f, *u)
        np.testing.assert_allclose(k, moments_by_definition(f, O.E_D3Q27, O.M_D3Q27, u), atol=1e-14)
        np.testing.assert_allclose(O.d3q27_raw_from_central(k, *u), r, atol=1e-13)
        np.testing.assert_allclose(O.d3q27_pop_from_raw(r), f, atol=1e-13)


# ---------------------------------------------------------------------------------------------
# Attractors against the recurrence
# ---------------------------------------------------------------------------------------------

def test_d3q27_printed_attractors_match_recurrence():
    """Sec. 5.2 discrete attractors of orders 4-6 equal the recurrence with D' = kt/rho.

    This pins reading R4 (kappa^Mv_122 uses kappa~_110 kappa~_012).
    """
    rng = np.random.default_rng(5)
    for _ in range(10):
        kt = rng.uniform(-0.5, 0.5, 27)
        rho = rng.uniform(0.8, 1.2)
        kt[0] = rho
        Mv = O.d3q27_attractors_high(kt, rho)
        post = {mnp: kt[j] for j, mnp in enumerate(O.M_D3Q27)}
        # first-order central moments of f are collision invariants (Eq. collisioninvariantf)
        lower = dict(post)
        lower[(1, 0, 0)] = lower[(0, 1, 0)] = lower[(0, 0, 1)] = 0.0
        D = {"xx": post[(2, 0, 0)] / rho, "yy": post[(0, 2, 0)] / rho, "zz": post[(0, 0, 2)] / rho,
             "xy": post[(1, 1, 0)] / rho, "xz": post[(1, 0, 1)] / rho, "yz": post[(0, 1, 1)] / rho}
        for j, mnp in enumerate(O.M_D3Q27):
            if sum(mnp) >= 4:
                assert Mv[j] == pytest.approx(recurrence_attractor(mnp, lower, D), abs=1e-14), mnp


# ---------------------------------------------------------------------------------------------
# Black-box collision checks in moment space
# ---------------------------------------------------------------------------------------------

def _forcing_sources(M, pre, F, rho):
    """Eq. forcing:2D / forcing:3D with the pre-collision moments; order-2 sources are zero."""
    idx = {mnp: j for j, mnp in enumerate(M)}
    s = np.zeros(len(M))
    for j, (m, n, p) in enumerate(M):
        order = m + n + p
        if order == 1:
            s[j] = m * F[0] + n * F[1] + p * F[2]
        elif order >= 3:
            for ax, c in enumerate((m, n, p)):
                if c > 0:
                    low = [m, n, p]; low[ax] -= 1
                    s[j] += c * F[ax] / rho * pre[idx[tuple(low)]]
    return s


def _check_relaxation(pre, post, Mv, om, sig, j):
    expect = pre[j] + om * (Mv - pre[j]) + (1 - om / 2) * sig
    assert post[j] == pytest.approx(expect, abs=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_d2q9_f_collision_is_fp_relaxation(seed):
    rng = np.random.default_rng(100 + seed)
    f = random_pops(rng, O.equilibrium_f(2, 1.0, rng.uniform(-0.1, 0.1, 2)), 0.3)
    F = np.array([*rng.uniform(-1e-3, 1e-3, 2), 0.0])
    om = rng.uniform(0.3, 1.9, 9)
    rho, ux, uy = O.macro_f(f, F)
    ft = O.collide_f(f, rho, (ux, uy), F, om)
    u = (ux, uy, 0.0)
    pre = moments_by_definition(f, O.E_D2Q9, O.M_D2Q9, u)
    post = moments_by_definition(ft, O.E_D2Q9, O.M_D2Q9, u)
    # invariants (Eq. collisioninvariantf) and the momentum source
    assert post[0] == pytest.approx(pre[0], abs=1e-14)
    np.testing.assert_allclose(ft @ O.E_D2Q9[:, :2] - f @ O.E_D2Q9[:, :2], F[:2], atol=1e-14)
    sig = _forcing_sources(O.M_D2Q9, pre, F, rho)
    cs2 = 1 / 3
    _check_relaxation(pre, post, rho, om[0], 0.0, 0)
    _check_relaxation(pre, post, 0.0, om[1], sig[1], 1)
    _check_relaxation(pre, post, 0.0, om[2], sig[2], 2)
    # kappa_2s, kappa_2d with omega_3, omega_4 (App. A Step 3)
    assert post[3] + post[4] == pytest.approx(pre[3] + pre[4] + om[3] * (2 * cs2 * rho - pre[3] - pre[4]),
                                              abs=1e-13)
    assert post[3] - post[4] == pytest.approx((pre[3] - pre[4]) * (1 - om[4]), abs=1e-13)
    _check_relaxation(pre, post, 0.0, om[5], 0.0, 5)
    post_d = {mnp: post[j] for j, mnp in enumerate(O.M_D2Q9)}
    lower = dict(post_d); lower[(1, 0, 0)] = lower[(0, 1, 0)] = 0.0
    D = {"xx": post_d[(2, 0, 0)] / rho, "yy": post_d[(0, 2, 0)] / rho, "zz": 0.0,
         "xy": post_d[(1, 1, 0)] / rho, "xz": 0.0, "yz": 0.0}
    for j in (6, 7, 8):
        Mv = recurrence_attractor(O.M_D2Q9[j], lower, D)
        _check_relaxation(pre, post, Mv, om[j], sig[j], j)


def _g_diffusion(option, post, M, T):
    """D-hat' used for the attractors of orders above 2: option A keeps c_s^2-hat (Eq.
    Dij2D_goptionA), option B renormalizes with the post-collision second moments (Eq. Dij2D_g
    and its 3D counterpart)."""
    c = 1 / 3
    if option == 0:
        return {"xx": c, "yy": c, "zz": c, "xy": 0.0, "xz": 0.0, "yz": 0.0}
    k = {mnp: post[j] for j, mnp in enumerate(M)}
    g = lambda mnp: k.get(mnp, 0.0) / T
    return {"xx": g((2, 0, 0)), "yy": g((0, 2, 0)), "zz": g((0, 0, 2)), "xy": g((1, 1, 0)),
            "xz": g((1, 0, 1)), "yz": g((0, 1, 1))}


@pytest.mark.parametrize("option", [0, 1])
@pytest.mark.parametrize("seed", range(6))
def test_d2q9_g_collision_is_fp_relaxation(seed, option):
    rng = np.random.default_rng(200 + seed)
    u = np.array([*rng.uniform(-0.1, 0.1, 2), 0.0])
    g = random_pops(rng, O.equilibrium_g(2, 0.7, u[:2]), 0.3)
    om = rng.uniform(0.3, 1.9, 9)
    gt = O.collide_g(g, u[:2], om, option)
    pre = moments_by_definition(g, O.E_D2Q9, O.M_D2Q9, u)
    post = moments_by_definition(gt, O.E_D2Q9, O.M_D2Q9, u)
    T = pre[0]
    assert post[0] == pytest.approx(T, abs=1e-14)        # Eq. collisioninvariantg
    c = 1 / 3
    _check_relaxation(pre, post, 0.0, om[1], 0.0, 1)
    _check_relaxation(pre, post, 0.0, om[2], 0.0, 2)
    assert post[3] + post[4] == pytest.approx(pre[3] + pre[4] + om[3] * (2 * c * T - pre[3] - pre[4]),
                                              abs=1e-13)
    assert post[3] - post[4] == pytest.approx((pre[3] - pre[4]) * (1 - om[4]), abs=1e-13)
    _check_relaxation(pre, post, 0.0, om[5], 0.0, 5)
    # orders 3-4 from the post-collision lower moments and the option's D-hat'
    lower = {mnp: post[j] for j, mnp in enumerate(O.M_D2Q9)}
    D = _g_diffusion(option, post, O.M_D2Q9, T)
    for j in (6, 7, 8):
        _check_relaxation(pre, post, recurrence_attractor(O.M_D2Q9[j], lower, D), om[j], 0.0, j)


@pytest.mark.parametrize("dim", [2, 3])
def test_g_options_coincide_when_second_moments_reach_equilibrium(dim):
    """With the second-order energy rates at 1 the post-collision second moments are exactly
    c_s^2-hat T (diagonal) and 0 (off-diagonal), so option B's D-hat' = eta~ / T equals option A's
    and the two collisions agree; with other second-order rates they differ."""
    rng = np.random.default_rng(500 + dim)
    q = 9 if dim == 2 else 15
    u = rng.uniform(-0.1, 0.1, 3)[:dim]
    g = random_pops(rng, O.equilibrium_g(dim, 0.7, u), 0.3)
    om = rng.uniform(0.3, 1.9, q)
    second = [3, 4, 5] if dim == 2 else [4, 5, 6, 7, 8, 9]
    om[second] = 1.0
    np.testing.assert_allclose(O.collide_g(g, u, om, 1), O.collide_g(g, u, om, 0), rtol=0,
                               atol=1e-15)
    om[second[0]] = 1.4
    assert np.abs(O.collide_g(g, u, om, 1) - O.collide_g(g, u, om, 0)).max() > 1e-6


@pytest.mark.parametrize("option", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_d3q15_g_collision_is_fp_relaxation(seed, option):
    """Pins reading R3 (eta^Mv_012 carries c_s^2-hat) and the option-B list."""
    rng = np.random.default_rng(300 + seed)
    u = rng.uniform(-0.1, 0.1, 3)
    g = random_pops(rng, O.equilibrium_g(3, 0.7, u), 0.3)
    om = rng.uniform(0.3, 1.9, 15)
    gt = O.collide_g(g, u, om, option)
    pre = moments_by_definition(g, O.E_D3Q15, O.M_D3Q15, u)
    post = moments_by_definition(gt, O.E_D3Q15, O.M_D3Q15, u)
    T = pre[0]
    assert post[0] == pytest.approx(T, abs=1e-14)
    c = 1 / 3
    lower = {mnp: post[j] for j, mnp in enumerate(O.M_D3Q15)}
    D = _g_diffusion(option, post, O.M_D3Q15, T)
    for j, mnp in enumerate(O.M_D3Q15):
        if j == 0:
            continue
        Mv = c * T if sum(mnp) == 2 and max(mnp) == 2 else (
            0.0 if sum(mnp) <= 2 else recurrence_attractor(mnp, lower, D))
        _check_relaxation(pre, post, Mv, om[j], 0.0, j)


@pytest.mark.parametrize("seed", range(3))
def test_d3q27_f_collision_is_fp_relaxation(seed):
    rng = np.random.default_rng(400 + seed)
    f = random_pops(rng, O.equilibrium_f(3, 1.0, rng.uniform(-0.1, 0.1, 3)), 0.3)
    F = rng.uniform(-1e-3, 1e-3, 3)
    om = rng.uniform(0.3, 1.9, 27)
    rho, ux, uy, uz = O.macro_f(f, F)
    u = (ux, uy, uz)
    ft = O.collide_f(f, rho, u, F, om)
    pre = moments_by_definition(f, O.E_D3Q27, O.M_D3Q27, u)
    post = moments_by_definition(ft, O.E_D3Q27, O.M_D3Q27, u)
    assert post[0] == pytest.approx(pre[0], abs=1e-14)
    np.testing.assert_allclose(ft @ O.E_D3Q27 - f @ O.E_D3Q27, F, atol=1e-14)
    sig = _forcing_sources(O.M_D3Q27, pre, F, rho)
    cs2 = 1 / 3
    idx = {mnp: j for j, mnp in enumerate(O.M_D3Q27)}
    # second-order diagonal: trace with om[7], deviators with om[8], om[9]
    tr = lambda k: k[idx[(2, 0, 0)]] + k[idx[(0, 2, 0)]] + k[idx[(0, 0, 2)]]
    assert tr(post) == pytest.approx(tr(pre) + om[7] * (3 * cs2 * rho - tr(pre)), abs=1e-13)
    d1 = lambda k: k[idx[(2, 0, 0)]] - k[idx[(0, 2, 0)]]
    d2 = lambda k: k[idx[(2, 0, 0)]] - k[idx[(0, 0, 2)]]
    assert d1(post) == pytest.approx(d1(pre) * (1 - om[8]), abs=1e-13)
    assert d2(post) == pytest.approx(d2(pre) * (1 - om[9]), abs=1e-13)
    post_d = {mnp: post[j] for j, mnp in enumerate(O.M_D3Q27)}
    lower = dict(post_d)
    lower[(1, 0, 0)] = lower[(0, 1, 0)] = lower[(0, 0, 1)] = 0.0
    D = {"xx": post_d[(2, 0, 0)] / rho, "yy": post_d[(0, 2, 0)] / rho, "zz": post_d[(0, 0, 2)] / rho,
         "xy": post_d[(1, 1, 0)] / rho, "xz": post_d[(1, 0, 1)] / rho, "yz": post_d[(0, 1, 1)] / rho}
    for j, mnp in enumerate(O.M_D3Q27):
        order = sum(mnp)
        if order == 0:
            _check_relaxation(pre, post, rho, om[j], 0.0, j)
        elif order == 1 or (order == 2 and max(mnp) == 1):
            _check_relaxation(pre, post, 0.0, om[j], sig[j], j)
        elif order >= 3:
            _check_relaxation(pre, post, recurrence_attractor(mnp, lower, D), om[j], sig[j], j)


# ---------------------------------------------------------------------------------------------
# Grid-level pins
# ---------------------------------------------------------------------------------------------

def _set_uniform(o: O.Oracle, rho, u, T):
    fe = O.equilibrium_f(o.dim, rho, u)
    ge = O.equilibrium_g(o.dim, T, u)
    f = np.broadcast_to(fe[:, None, None, None], (o.qf, *o.shape)).copy()
    g = np.broadcast_to(ge[:, None, None, None], (o.qg, *o.shape)).copy()
    o.set_state(f, g)
    return f, g


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_flow_is_a_fixed_point(dim):
    """Galilean check: a uniform moving equilibrium on a periodic box does not change."""
    rng = np.random.default_rng(7)
    of, og = rng.uniform(0.5, 1.9, 27 if dim == 3 else 9), rng.uniform(0.5, 1.9, 15 if dim == 3 else 9)
    o = O.Oracle(dim, 5, 4, 3, om_f=of, om_g=og, gbeta=0.0, init=False)
    f0, g0 = _set_uniform(o, 1.1, (0.05, -0.03, 0.02), 0.8)
    o.step(5)
    f1, g1 = o.get_state()
    np.testing.assert_allclose(f1, f0, atol=1e-14)
    np.testing.assert_allclose(g1, g0, atol=1e-14)


def _decay_rate(series, t1, t2):
    return math.log(series[t1] / series[t2]) / (t2 - t1)


@pytest.mark.parametrize("dim", [2, 3])
def test_shear_wave_decays_at_nu_k2(dim):
    """u_x = A sin(k y) decays as exp(-nu k^2 t), nu = c_s^2 (1/omega - 1/2) (App. A)."""
    N, A, omega = 32, 1e-3, 1.25
    nu = (1 / 3) * (1 / omega - 0.5)
    om_f, om_g = O.default_omegas(dim, omega, 1.0)
    o = O.Oracle(dim, 2, N, 2, om_f=om_f, om_g=om_g, gbeta=0.0, init=False)
    y = np.arange(N)
    f = np.zeros((o.qf, *o.shape)); g = np.zeros((o.qg, *o.shape))
    for j in range(N):
        f[:, :, j, :] = O.equilibrium_f(dim, 1.0, (A * math.sin(2 * math.pi * j / N), 0, 0))[:, None, None]
        g[:, :, j, :] = O.equilibrium_g(dim, 1.0, (0, 0, 0))[:, None, None]
    o.set_state(f, g)
    amp = {}
    for t in range(0, 301):
        if t in (60, 300):
            ux = o.fields()["ux"][0, :, 0]
            amp[t] = 2 / N * np.sum(ux * np.sin(2 * math.pi * y / N))
        o.step(1)
    k2 = (2 * math.pi / N) ** 2
    assert _decay_rate(amp, 60, 300) == pytest.approx(nu * k2, rel=0.01)


@pytest.mark.parametrize("dim", [2, 3])
def test_thermal_wave_decays_at_alpha_k2(dim):
    """T = 1 + A sin(k x) decays as exp(-alpha k^2 t), alpha = c_s^2-hat (1/omega - 1/2)."""
    N, A, omega = 32, 1e-2, 1.4
    alpha = (1 / 3) * (1 / omega - 0.5)
    om_f, om_g = O.default_omegas(dim, 1.0, omega)
    o = O.Oracle(dim, N, 2, 2, om_f=om_f, om_g=om_g, gbeta=0.0, init=False)
    x = np.arange(N)
    f = np.zeros((o.qf, *o.shape)); g = np.zeros((o.qg, *o.shape))
    for i in range(N):
        f[:, :, :, i] = O.equilibrium_f(dim, 1.0)[:, None, None]
        g[:, :, :, i] = O.equilibrium_g(dim, 1.0 + A * math.sin(2 * math.pi * i / N))[:, None, None]
    o.set_state(f, g)
    amp = {}
    for t in range(0, 301):
        if t in (60, 300):
            T = o.fields()["T"][0, 0, :]
            amp[t] = 2 / N * np.sum((T - 1.0) * np.sin(2 * math.pi * x / N))
        o.step(1)
    k2 = (2 * math.pi / N) ** 2
    assert _decay_rate(amp, 60, 300) == pytest.approx(alpha * k2, rel=0.01)


def test_nusselt_of_linear_profile_is_one():
    """A linear T between half-way walls gives Nu = 1 exactly (Sec. 6.1 three-point derivative)."""
    N, TH, TC = 12, 1.0, 0.0
    bc = O.BC(face=(O.WALL_FIXED_T, O.WALL_FIXED_T, O.PERIODIC, O.PERIODIC, 0, 0),
              T_wall=(TH, TC, 0, 0, 0, 0), T_init=0.5, T_ref=0.5)
    o = O.Oracle(2, N, 3, bc=bc, gbeta=0.0, init=False)
    f = np.zeros((9, *o.shape)); g = np.zeros((9, *o.shape))
    for i in range(N):
        f[:, :, :, i] = O.equilibrium_f(2, 1.0)[:, None, None]
        g[:, :, :, i] = O.equilibrium_g(2, TH + (TC - TH) * (i + 0.5) / N)[:, None, None]
    o.set_state(f, g)
    for face in (0, 1):
        mean, mx, mn, _, _ = o.nusselt(face)
        assert mean == pytest.approx(1.0, abs=1e-13)
        assert mx - mn < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_conduction_state_is_linear_with_unit_nusselt(dim):
    """Fixed-T walls on x, periodic elsewhere, no buoyancy: steady T is linear, Nu = 1."""
    N, TH, TC = 10, 1.0, 0.0
    face = (O.WALL_FIXED_T, O.WALL_FIXED_T, O.PERIODIC, O.PERIODIC, O.PERIODIC, O.PERIODIC)
    bc = O.BC(face=face, T_wall=(TH, TC, 0, 0, 0, 0), T_init=0.5, T_ref=0.5,
              gravity_axis=1 if dim == 2 else 2)
    om_f, om_g = O.default_omegas(dim, 1.3, 1.1)
    o = O.Oracle(dim, N, 2, 2, bc=bc, om_f=om_f, om_g=om_g, gbeta=0.0)
    o.step(3000 if dim == 2 else 2000)
    T = o.fields()["T"]
    x = (np.arange(N) + 0.5) / N
    expect = TH + (TC - TH) * x
    np.testing.assert_allclose(T.reshape(-1, N), np.broadcast_to(expect, (T.size // N, N)), atol=1e-9)
    for face_id in (0, 1):
        assert o.nusselt(face_id)[0] == pytest.approx(1.0, abs=1e-8)


def test_rayleigh_benard_onset_sign():
    """Heated from below: Ra = 1e3 < Ra_c stays conductive (Nu = 1); Ra = 2e4 convects (Nu > 1).

    A wrong buoyancy sign would leave both layers conductive.
    """
    res = {}
    for Ra in (1e3, 2e4):
        bc = O.rayleigh_benard_bc(seed=11, perturb=1e-2)
        o = O.Oracle(2, 32, 16, bc=bc, Ra=Ra, Pr=0.71, Ma=0.1)
        o.step(25000)
        res[Ra] = o.nusselt(2)[0]
    assert res[1e3] == pytest.approx(1.0, abs=2e-3)
    assert res[2e4] > 1.5


@pytest.mark.slow
def test_cavity_64_ra1e4_matches_table_con2():
    """64^2 cavity, Ra 1e4, Pr 0.71, Ma 0.1, 20000 steps vs the 512^2 values of Table con2."""
    gold = load_golden("paper_values.json")
    o = O.Oracle(2, 64, 64, bc=O.cavity_bc(2), Ra=1e4, Pr=0.71, Ma=0.1)
    o.step(20000)
    mean, mx, mn, jmax, jmin = o.nusselt(0)
    assert mean == pytest.approx(gold["nu0_mean_2d_512"]["1e4"], rel=0.01)
    ext = gold["nu0_extremes_2d_512_ra1e4"]
    assert mx == pytest.approx(ext["max"], rel=0.01)
    assert (jmax + 0.5) / 64 == pytest.approx(ext["y_max"], abs=1.5 / 64)
    # The minimum sits in the top corner at the last node centre, 63.5/64 = 0.992 here against
    # 511.5/512 = 0.999 in the table, where Nu_0(y) is steep: only a loose band is meaningful.
    assert mn == pytest.approx(ext["min"], rel=0.15)
    assert jmin == 63


def test_node_centre_location_convention():
    """The printed (Nu_0)min location 0.9990 at 512^2 is the last node centre (511 + 1/2)/512."""
    gold = load_golden("paper_values.json")["nu0_min_location_512"]
    assert round((gold["n"] - 1 + 0.5) / gold["n"], 4) == gold["y"]


def test_splitmix64_reference_outputs():
    vec = load_golden("splitmix64.json")
    for i, h in enumerate(vec["seed0"]):
        assert O.lib().orc_splitmix64(0, i) == int(h, 16)


def test_transport_mapping_matches_worked_numbers():
    """Ma = sqrt(3) U_o (Sec. 7), nu = U L sqrt(Pr/Ra), omega = 1/(nu/c_s^2 + 1/2) (App. A)."""
    tr = O.transport(1e4, 0.71, 0.1, 64)
    assert tr.U == pytest.approx(0.1 / math.sqrt(3))
    assert tr.nu == pytest.approx(0.0311351, rel=1e-5)
    assert tr.omega_nu == pytest.approx(1.685186, rel=1e-5)
    assert tr.alpha == pytest.approx(tr.nu / 0.71)
    assert tr.gbeta * 1.0 * 64 == pytest.approx(tr.U ** 2)
    # Ra recovered from the definition of Sec. 6.1
    assert tr.gbeta * 1.0 * 64 ** 3 / (tr.alpha * tr.nu) == pytest.approx(1e4)


# ---------------------------------------------------------------------------------------------
# Walls at edges and corners (reading R7)
# ---------------------------------------------------------------------------------------------

# Order in which the faces -x, +x, -y, +y, -z, +z decide a link that crosses several walls
# (reading R7: the crossed face that comes last in the order -z, -y, -x, +x, +y, +z).
R7_ORDER = ("-z", "-y", "-x", "+x", "+y", "+z")
FACE_NAMES = ("-x", "+x", "-y", "+y", "-z", "+z")


def pulled_T_by_hand(dim, g, kinds, T_wall, E, W, x, y, z):
    """T at node (x, y, z) after streaming, written out link by link: a link whose upwind node
    lies inside takes that node's population; one whose upwind node lies beyond walls takes the
    rule of the deciding face (R7_ORDER): bounce-back g_abar(x) at an adiabatic face,
    anti-bounce-back -g_abar(x) + 2 w_a T_w at a fixed-temperature face."""
    q, nz, ny, nx = g.shape
    ext = (nx, ny, nz)
    c = (x, y, z)
    T = 0.0
    for a in range(q):
        e = E[a]
        opp = [b for b in range(q) if all(E[b][d] == -e[d] for d in range(3))][0]
        src = [c[d] - e[d] for d in range(3)]
        crossed = []
        for d in range(dim):
            if src[d] < 0:
                crossed.append(2 * d)
            elif src[d] >= ext[d]:
                crossed.append(2 * d + 1)
        if not crossed:
            T += g[a, src[2], src[1], src[0]]
            continue
        face = max(crossed, key=lambda f: R7_ORDER.index(FACE_NAMES[f]))
        back = g[opp, z, y, x]
        T += -back + 2.0 * W[a] * T_wall[face] if kinds[face] == O.WALL_FIXED_T else back
    return T


@pytest.mark.parametrize("dim,shape", [(2, (1, 3, 3)), (3, (3, 3, 3)), (3, (3, 4, 2))])
def test_edge_and_corner_links_follow_reading_r7(dim, shape):
    """Every node of a box two to four nodes wide (so that every node is an edge or corner node
    of the cavity: hot -x, cold +x, adiabatic elsewhere): the oracle's streamed temperature equals
    the link-by-link sum of the walls' rules, with edge and corner links decided as reading R7
    states.  A random state makes every link's contribution distinct."""
    nz, ny, nx = shape
    bc = O.cavity_bc(dim, T_hot=1.0, T_cold=0.0)
    o = O.Oracle(dim, nx, ny, nz, bc=bc, Ra=1e4, Pr=0.71, Ma=0.1)
    rng = np.random.default_rng(40 + dim)
    f, g = o.get_state()
    g = g * rng.uniform(0.5, 1.5, g.shape)
    o.set_state(f, g)
    E = O.E_D2Q9 if dim == 2 else O.E_D3Q15
    W = O.equilibrium_g(dim, 1.0)
    T = o.fields()["T"]
    for z in range(o.nz):
        for y in range(ny):
            for x in range(nx):
                want = pulled_T_by_hand(dim, g, bc.face, bc.T_wall, E, W, x, y, z)
                assert T[z, y, x] == pytest.approx(want, abs=1e-14), (x, y, z)
