"""FP64 CPU oracle for the FPC-LBM of thermal convection (Schupbach & Premnath, arXiv 2504.09041).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It loads ``liboracle.so`` built from
``fpc_oracle.c`` (plain C, FP64, ``-ffp-contract=off``) and shares no code with the CUDA path.

Parity status: every per-node routine is pinned by ``tests/test_oracle_pins.py`` against
definitions (moment sums over the velocity sets), the attractor recurrence (Eqs. Mvcmattractor2D,
Mvcmattractor3D), collision invariants, textbook lattice weights and decay rates, and the printed
Nusselt numbers of Tables con2 and CompareNu3D.  The D3Q27 flow collision follows a reading of a
passage the paper defers to earlier work; its parity against the authors' code is unpinned beyond
the definitional checks and the 3D Nusselt table.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fpc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

PERIODIC, WALL_ADIABATIC, WALL_FIXED_T = 0, 1, 2

# Velocity sets in the paper's order (Eqs. ex/ey, Sec. 5.2, Sec. 5.4).
E_D2Q9 = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0],
                   [1, 1, 0], [-1, 1, 0], [-1, -1, 0], [1, -1, 0]])
E_D3Q27 = np.array([
    [0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, 1], [1, 0, -1],
    [-1, 0, -1], [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1], [1, 1, 1], [-1, 1, 1],
    [1, -1, 1], [-1, -1, 1], [1, 1, -1], [-1, 1, -1], [1, -1, -1], [-1, -1, -1]])
E_D3Q15 = np.array([
    [0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 1], [-1, 1, 1], [1, -1, 1], [-1, -1, 1], [1, 1, -1], [-1, 1, -1], [1, -1, -1],
    [-1, -1, -1]])

# Moment orders: D2Q9 (Sec. 4.2), D3Q27 (Sec. 5.2), D3Q15 (Sec. 5.4).
M_D2Q9 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (2, 0, 0), (0, 2, 0), (1, 1, 0), (2, 1, 0),
          (1, 2, 0), (2, 2, 0)]
M_D3Q27 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
           (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 2, 0), (1, 0, 2), (2, 1, 0), (0, 1, 2),
           (2, 0, 1), (0, 2, 1), (1, 1, 1), (2, 2, 0), (2, 0, 2), (0, 2, 2), (2, 1, 1),
           (1, 2, 1), (1, 1, 2), (1, 2, 2), (2, 1, 2), (2, 2, 1), (2, 2, 2)]
M_D3Q15 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1),
           (2, 0, 0), (0, 2, 0), (0, 0, 2), (1, 2, 0), (0, 1, 2), (2, 0, 1), (1, 1, 1),
           (2, 2, 0)]

CS2 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` from ``fpc_oracle.c`` with gcc (FP64, no contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, v, dp, ip = (ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int))
        L.orc_create.restype = v
        L.orc_create.argtypes = [i, i, i, i]
        L.orc_destroy.argtypes = [v]
        L.orc_set_bc.argtypes = [v, ip, dp, d, i, d]
        L.orc_set_omegas.argtypes = [v, dp, dp]
        L.orc_set_wall_profile.argtypes = [v, i, dp, ctypes.c_long]
        L.orc_set_state.argtypes = [v, dp, dp]
        L.orc_get_state.argtypes = [v, dp, dp]
        L.orc_step.argtypes = [v, ctypes.c_long]
        L.orc_update_box.argtypes = [v, i, i, i, i, i, i]
        L.orc_fields.argtypes = [v, dp, dp, dp, dp, dp]
        L.orc_nusselt.argtypes = [v, i, d, d, dp]
        L.orc_nusselt.restype = i
        L.orc_init_rest.argtypes = [v, d, ctypes.c_uint64, d]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_uniform01.restype = d
        L.orc_uniform01.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_threads.restype = i
        for name, nargs in [("orc_d2q9_step1", 2), ("orc_d2q9_step5", 2), ("orc_d3q15_step1", 2),
                            ("orc_d3q15_step5", 2), ("orc_d3q27_raw", 2),
                            ("orc_d3q27_pop_from_raw", 2)]:
            getattr(L, name).argtypes = [dp] * nargs
        L.orc_d2q9_step2.argtypes = [dp, d, d, dp]
        L.orc_d2q9_step4.argtypes = [dp, d, d, dp]
        L.orc_d3q15_step2.argtypes = [dp, d, d, d, dp]
        L.orc_d3q15_step4.argtypes = [dp, d, d, d, dp]
        L.orc_d3q27_central.argtypes = [dp, d, d, d, dp]
        L.orc_d3q27_raw_from_central.argtypes = [dp, d, d, d, dp]
        L.orc_d3q27_attractors_high.argtypes = [dp, d, dp]
        L.orc_d2q9_macro.argtypes = [dp, d, d, dp]
        L.orc_d3q27_macro.argtypes = [dp, d, d, d, dp]
        L.orc_d2q9_f_collide.argtypes = [dp, d, d, d, d, d, dp, dp]
        L.orc_d2q9_g_collide.argtypes = [dp, d, d, dp, i, dp]
        L.orc_d3q15_g_collide.argtypes = [dp, d, d, d, dp, i, dp]
        L.orc_set_g_option.argtypes = [v, i]
        L.orc_d3q27_f_collide.argtypes = [dp, d, d, d, d, d, d, d, dp, dp]
        L.orc_equilibrium_f.argtypes = [i, d, d, d, d, dp]
        L.orc_equilibrium_g.argtypes = [i, d, d, d, d, dp]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(x, n=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        assert a.size == n
    return a


# ----------------------------------------------------------------------------------------------
# Per-node routines (thin wrappers, one node at a time)
# ----------------------------------------------------------------------------------------------

def d2q9_step1(f):
    out = np.zeros(9); lib().orc_d2q9_step1(_p(_vec(f, 9)), _p(out)); return out


def d2q9_step2(r, ux, uy):
    out = np.zeros(9); lib().orc_d2q9_step2(_p(_vec(r, 9)), ux, uy, _p(out)); return out


def d2q9_step4(c, ux, uy):
    out = np.zeros(9); lib().orc_d2q9_step4(_p(_vec(c, 9)), ux, uy, _p(out)); return out


def d2q9_step5(r):
    out = np.zeros(9); lib().orc_d2q9_step5(_p(_vec(r, 9)), _p(out)); return out


def d3q15_step1(g):
    out = np.zeros(15); lib().orc_d3q15_step1(_p(_vec(g, 15)), _p(out)); return out


def d3q15_step2(r, ux, uy, uz):
    out = np.zeros(15); lib().orc_d3q15_step2(_p(_vec(r, 15)), ux, uy, uz, _p(out)); return out


def d3q15_step4(c, ux, uy, uz):
    out = np.zeros(15); lib().orc_d3q15_step4(_p(_vec(c, 15)), ux, uy, uz, _p(out)); return out


def d3q15_step5(r):
    out = np.zeros(15); lib().orc_d3q15_step5(_p(_vec(r, 15)), _p(out)); return out


def d3q27_raw(f):
    out = np.zeros(27); lib().orc_d3q27_raw(_p(_vec(f, 27)), _p(out)); return out


def d3q27_central(f, ux, uy, uz):
    out = np.zeros(27); lib().orc_d3q27_central(_p(_vec(f, 27)), ux, uy, uz, _p(out)); return out


def d3q27_raw_from_central(k, ux, uy, uz):
    out = np.zeros(27)
    lib().orc_d3q27_raw_from_central(_p(_vec(k, 27)), ux, uy, uz, _p(out))
    return out


def d3q27_pop_from_raw(r):
    out = np.zeros(27); lib().orc_d3q27_pop_from_raw(_p(_vec(r, 27)), _p(out)); return out


def d3q27_attractors_high(kt, rho):
    out = np.zeros(27); lib().orc_d3q27_attractors_high(_p(_vec(kt, 27)), rho, _p(out)); return out


def macro_f(f, F):
    """(rho, u) of flow populations with the half-force velocity (App. A Step 7)."""
    f = _vec(f)
    if f.size == 9:
        out = np.zeros(3); lib().orc_d2q9_macro(_p(f), F[0], F[1], _p(out))
    else:
        out = np.zeros(4); lib().orc_d3q27_macro(_p(f), F[0], F[1], F[2], _p(out))
    return out


def collide_f(f, rho, u, F, om):
    f = _vec(f)
    out = np.zeros(f.size)
    if f.size == 9:
        lib().orc_d2q9_f_collide(_p(f), rho, u[0], u[1], F[0], F[1], _p(_vec(om, 9)), _p(out))
    else:
        lib().orc_d3q27_f_collide(_p(f), rho, u[0], u[1], u[2], F[0], F[1], F[2],
                                  _p(_vec(om, 27)), _p(out))
    return out


def collide_g(g, u, om, option: int = 0):
    """Energy collision; option 0 = option-A attractors, 1 = option B (renormalized)."""
    g = _vec(g)
    out = np.zeros(g.size)
    if g.size == 9:
        lib().orc_d2q9_g_collide(_p(g), u[0], u[1], _p(_vec(om, 9)), option, _p(out))
    else:
        lib().orc_d3q15_g_collide(_p(g), u[0], u[1], u[2], _p(_vec(om, 15)), option, _p(out))
    return out


def equilibrium_f(dim, rho, u=(0.0, 0.0, 0.0)):
    out = np.zeros(9 if dim == 2 else 27)
    lib().orc_equilibrium_f(dim, rho, u[0], u[1], u[2] if len(u) > 2 else 0.0, _p(out))
    return out


def equilibrium_g(dim, T, u=(0.0, 0.0, 0.0)):
    out = np.zeros(9 if dim == 2 else 15)
    lib().orc_equilibrium_g(dim, T, u[0], u[1], u[2] if len(u) > 2 else 0.0, _p(out))
    return out


def uniform01(seed: int, i: int) -> float:
    return lib().orc_uniform01(seed, i)


# ----------------------------------------------------------------------------------------------
# Problem parameters (Sec. 6.1 and App. A/B/C relaxation-rate paragraphs)
# ----------------------------------------------------------------------------------------------

@dataclass
class Transport:
    U: float        # characteristic velocity U_o = Ma / sqrt(3)  (Ma = sqrt(3) U_o, Sec. 7)
    nu: float       # kinematic viscosity
    alpha: float    # thermal diffusivity
    gbeta: float    # g*beta with g*beta*dT*L = U_o^2 (F_o = U_o^2 / L_o, Sec. 6.1)
    omega_nu: float     # nu = c_s^2 (1/omega - 1/2)         (App. A)
    omega_alpha: float  # alpha = c_s^2-hat (1/omega - 1/2)  (App. B, App. C)


def transport(Ra: float, Pr: float, Ma: float, L: float, dT: float = 1.0) -> Transport:
    """Ra = g beta dT L^3 / (alpha nu), Pr = nu / alpha, with g beta dT L = U_o^2."""
    U = Ma / math.sqrt(3.0)
    nu = U * L * math.sqrt(Pr / Ra)
    alpha = nu / Pr
    gbeta = U * U / (L * dT)
    return Transport(U, nu, alpha, gbeta, 1.0 / (nu / CS2 + 0.5), 1.0 / (alpha / CS2 + 0.5))


def default_omegas(dim: int, omega_nu: float, omega_alpha: float, omega_bulk: float = 1.0):
    """Relaxation rates of the paper: viscosity/diffusivity rates from nu, alpha; all free ones 1.0.

    2D f: omega_3 (bulk) = omega_bulk, omega_4 = omega_5 = omega_nu (App. A).
    2D g: omega_1 = omega_2 = omega_alpha (App. B).  3D g: omega_1..3 = omega_alpha (App. C).
    3D f (order of Sec. 5.2): the three off-diagonal second-order moments and the two deviator
    slots (index 8, 9) take omega_nu; the trace slot (index 7) takes omega_bulk.
    """
    if dim == 2:
        om_f = np.ones(9); om_f[3] = omega_bulk; om_f[4] = om_f[5] = omega_nu
        om_g = np.ones(9); om_g[1] = om_g[2] = omega_alpha
    else:
        om_f = np.ones(27); om_f[4:7] = omega_nu; om_f[7] = omega_bulk; om_f[8] = om_f[9] = omega_nu
        om_g = np.ones(15); om_g[1:4] = omega_alpha
    return om_f, om_g


@dataclass
class BC:
    face: tuple = (PERIODIC,) * 6          # -x, +x, -y, +y, -z, +z
    T_wall: tuple = (0.0,) * 6
    T_init: float = 0.5
    T_ref: float = 0.5
    gravity_axis: int = 1
    seed: int = 0
    perturb: float = 0.0


def cavity_bc(dim: int, T_hot=1.0, T_cold=0.0) -> BC:
    """Differentially heated cavity: hot -x, cold +x, other faces adiabatic, no-slip everywhere."""
    face = [WALL_FIXED_T, WALL_FIXED_T] + [WALL_ADIABATIC] * 4
    T_wall = [T_hot, T_cold, 0, 0, 0, 0]
    return BC(tuple(face), tuple(T_wall), 0.5 * (T_hot + T_cold), 0.5 * (T_hot + T_cold),
              1 if dim == 2 else 2)


def rayleigh_benard_bc(T_hot=1.0, T_cold=0.0, seed=0, perturb=1e-3) -> BC:
    """Rayleigh-Benard in 2D: periodic x, hot bottom (-y), cold top (+y), gravity along y."""
    face = (PERIODIC, PERIODIC, WALL_FIXED_T, WALL_FIXED_T, PERIODIC, PERIODIC)
    return BC(face, (0, 0, T_hot, T_cold, 0, 0), 0.5 * (T_hot + T_cold), 0.5 * (T_hot + T_cold),
              1, seed, perturb)


def characteristic_length(dim, n, bc: BC) -> int:
    """L_o: node count along the axis of the first fixed-temperature face (nx if none)."""
    for f in range(2 * dim):
        if bc.face[f] == WALL_FIXED_T:
            return n[f // 2]
    return n[0]


def temperature_difference(bc: BC, dim: int) -> float:
    T = [bc.T_wall[f] for f in range(2 * dim) if bc.face[f] == WALL_FIXED_T]
    return (max(T) - min(T)) if len(T) >= 2 and max(T) > min(T) else 1.0


class Oracle:
    """A box of nx*ny*nz nodes (nz = 1 in 2D) advanced by the FP64 oracle.

    State arrays are the post-collision populations, shape (q, nz, ny, nx) in the paper's link
    order, x fastest.
    """

    def __init__(self, dim, nx, ny, nz=1, bc: BC | None = None, Ra=None, Pr=None, Ma=None,
                 om_f=None, om_g=None, gbeta=None, init=True, g_option: int = 0):
        self.dim = dim
        self.nx, self.ny, self.nz = nx, ny, (nz if dim == 3 else 1)
        self.qf, self.qg = (9, 9) if dim == 2 else (27, 15)
        self.bc = bc or BC()
        self.h = lib().orc_create(dim, nx, ny, self.nz)
        if not self.h:
            raise ValueError("bad dimensions")
        n = (self.nx, self.ny, self.nz)
        self.L = characteristic_length(dim, n, self.bc)
        self.dT = temperature_difference(self.bc, dim)
        self.tr = None
        if Ra is not None:
            self.tr = transport(Ra, Pr, Ma, self.L, self.dT)
            of, og = default_omegas(dim, self.tr.omega_nu, self.tr.omega_alpha)
            om_f = of if om_f is None else om_f
            om_g = og if om_g is None else om_g
            gbeta = self.tr.gbeta if gbeta is None else gbeta
        if om_f is None:
            om_f = np.ones(self.qf)
        if om_g is None:
            om_g = np.ones(self.qg)
        self.om_f, self.om_g = _vec(om_f, self.qf), _vec(om_g, self.qg)
        self.gbeta = 0.0 if gbeta is None else float(gbeta)
        lib().orc_set_omegas(self.h, _p(self.om_f), _p(self.om_g))
        self.g_option = int(g_option)
        lib().orc_set_g_option(self.h, self.g_option)
        faces = (ctypes.c_int * 6)(*self.bc.face)
        tw = _vec(self.bc.T_wall, 6)
        lib().orc_set_bc(self.h, faces, _p(tw), self.bc.T_ref, self.bc.gravity_axis, self.gbeta)
        if init:
            lib().orc_init_rest(self.h, self.bc.T_init, self.bc.seed, self.bc.perturb)

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def set_state(self, f, g):
        f = _vec(f).reshape(self.qf, *self.shape)
        g = _vec(g).reshape(self.qg, *self.shape)
        lib().orc_set_state(self.h, _p(np.ascontiguousarray(f)), _p(np.ascontiguousarray(g)))

    def get_state(self):
        f = np.zeros((self.qf, *self.shape)); g = np.zeros((self.qg, *self.shape))
        lib().orc_get_state(self.h, _p(f), _p(g))
        return f, g

    def set_wall_profile(self, face, Tw):
        Tw = _vec(Tw)
        if lib().orc_set_wall_profile(self.h, face, _p(Tw), Tw.size) != 0:
            raise ValueError("profile length does not match the face")

    def step(self, n=1):
        lib().orc_step(self.h, int(n))

    def update_box(self, x0, x1, y0, y1, z0=0, z1=1):
        lib().orc_update_box(self.h, x0, x1, y0, y1, z0, z1)

    def fields(self):
        out = [np.zeros(self.shape) for _ in range(5)]
        lib().orc_fields(self.h, *[_p(a) for a in out])
        return dict(zip(("rho", "ux", "uy", "uz", "T"), out))

    def nusselt_profile(self, face):
        ax = face // 2
        n = [self.nx, self.ny, self.nz]
        tang = [n[a] for a in range(3) if a != ax]
        nu = np.zeros(tang[0] * tang[1])
        if lib().orc_nusselt(self.h, face, float(self.L), float(self.dT), _p(nu)) != 0:
            raise ValueError("face is not a fixed-temperature wall")
        return nu

    def nusselt(self, face):
        """Mean, max, min of the local wall Nusselt number and the argmax/argmin node index."""
        nu = self.nusselt_profile(face)
        return float(nu.mean()), float(nu.max()), float(nu.min()), int(nu.argmax()), int(nu.argmin())


def threads() -> int:
    return lib().orc_threads()
