"""Generic-form FP64 restatement of the 2D method (D2Q9 flow + D2Q9 energy), in real or complex
arithmetic.  TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests may use it.

This is a second, independent oracle for the 2D path, written from the paper's definitions
rather than from its printed step-by-step formulas (which fpc_oracle.c follows):

  * central moments by their definition, kappa_mn = sum_a f_a (e_ax - u_x)^m (e_ay - u_y)^n
    (Sec. 4.2, moment order 00, 10, 01, 20, 02, 11, 21, 12, 22), and the populations back from
    the relaxed moments by solving that 9 x 9 system at every node (numpy.linalg.solve), which is
    what App. A/B Steps 4-5 compute in closed form;
  * the relaxation of App. A Step 3 (flow, with the forcing sources of Eq. forcing:2D and
    readings R5, R8, R9) and App. B Step 3 (energy, option A, Eq. MvT2D, or option B,
    Eq. MvT2DoptionB), on those moments;
  * the pull streaming of Eqs. LBMsteps-stream / LBMsteps-streamg with the half-way walls of
    Sec. 6.1 (bounce-back of f; bounce-back or anti-bounce-back of g, decided at edge links by the
    crossed face that comes last in the order -y, -x, +x, +y, reading R7), the Boussinesq force and
    velocity of App. A Step 7 (reading R10), and the
    wall Nusselt number of Sec. 6.1 (readings R13-R15).

Every node is processed at once with numpy arrays of shape (9, ny, nx).  With dtype complex128
and a wall-temperature profile T_w + i h v, Im(J) / h is the directional derivative dJ/dT_w . v
of any output J, exact to rounding for h far below the scale of the state (complex-step
differentiation, Squire and Trapp 1998): the tests use it as the oracle of the adjoint.
"""
from __future__ import annotations

import numpy as np

# Eqs. ex, ey: the D2Q9 links in the paper's order
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)    # rest-state attractor weights
MOMENTS = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]
CS2 = 1.0 / 3.0
PERIODIC, WALL_ADIABATIC, WALL_FIXED_T = 0, 1, 2
# faces -x, +x, -y, +y in the order that decides edge links (reading R7): -y, -x, +x, +y
FACE_RANK = {0: 1, 1: 2, 2: 0, 3: 3}


def central_matrix(ux, uy):
    """C[..., j, a] = (e_ax - ux)^m_j (e_ay - uy)^n_j for every node (last two axes 9 x 9)."""
    dx = E[:, 0][None, None, :] - ux[..., None]
    dy = E[:, 1][None, None, :] - uy[..., None]
    return np.stack([dx ** m * dy ** n for m, n in MOMENTS], axis=-2)


def central_moments(p, ux, uy):
    """kappa[j] (shape (9, ny, nx)) of the populations p (9, ny, nx) at velocity u."""
    C = central_matrix(ux, uy)
    return np.einsum("yxja,ayx->jyx", C, p), C


def populations(C, k):
    """Populations whose central moments (matrix C) are k: solve C p = k at every node."""
    rhs = np.moveaxis(k, 0, -1)[..., None]
    return np.moveaxis(np.linalg.solve(C, rhs)[..., 0], -1, 0)


def collide_f(f, rho, ux, uy, Fx, Fy, om):
    """App. A Step 3 on the definition moments; returns the post-collision populations."""
    k, C = central_moments(f, ux, uy)
    k00, k10, k01, k20, k02, k11, k21, k12, k22 = k
    # sources of Eq. forcing:2D with the pre-collision moments; order 2 zero (reading R5)
    s10, s01 = Fx, Fy
    s21 = 2.0 * (Fx / rho) * k11 + (Fy / rho) * k20
    s12 = (Fx / rho) * k02 + 2.0 * (Fy / rho) * k11          # reading R8
    s22 = 2.0 * ((Fx / rho) * k12 + (Fy / rho) * k21)

    def relax(kv, Mv, w, s=0.0):
        return kv + w * (Mv - kv) + (1.0 - w / 2.0) * s

    t00 = relax(k00, rho, om[0])
    t10 = relax(k10, 0.0, om[1], s10)
    t01 = relax(k01, 0.0, om[2], s01)
    t2s = relax(k20 + k02, 2.0 * CS2 * rho, om[3])
    t2d = relax(k20 - k02, 0.0, om[4])
    t11 = relax(k11, 0.0, om[5])
    t21 = relax(k21, 0.0, om[6], s21)
    t12 = relax(k12, 0.0, om[7], s12)
    t20 = 0.5 * (t2s + t2d)
    t02 = 0.5 * (t2s - t2d)
    # renormalized attractor of order 4 from the post-collision second moments (Eq. MvCM2D)
    t22 = relax(k22, (t20 * t02 + 2.0 * t11 * t11) / rho, om[8], s22)
    return populations(C, np.stack([t00, t10, t01, t20, t02, t11, t21, t12, t22]))


def collide_g(g, ux, uy, om, option=0):
    """App. B Step 3 on the definition moments (no sources); option 0 = A, 1 = B."""
    n, C = central_moments(g, ux, uy)
    n00, n10, n01, n20, n02, n11, n21, n12, n22 = n
    T = n00

    def relax(nv, Mv, w):
        return nv + w * (Mv - nv)

    t00 = relax(n00, T, om[0])
    t10 = relax(n10, 0.0, om[1])
    t01 = relax(n01, 0.0, om[2])
    t2s = relax(n20 + n02, 2.0 * CS2 * T, om[3])
    t2d = relax(n20 - n02, 0.0, om[4])
    t11 = relax(n11, 0.0, om[5])
    t20 = 0.5 * (t2s + t2d)
    t02 = 0.5 * (t2s - t2d)
    if option == 0:      # Eq. MvT2D
        M21, M12, M22 = 2.0 / 3.0 * CS2 * t01, 2.0 / 3.0 * CS2 * t10, 0.5 * CS2 * (t20 + t02)
    else:                # Eq. MvT2DoptionB
        M21 = 2.0 / (3.0 * T) * (t20 * t01 + 2.0 * t11 * t10)
        M12 = 2.0 / (3.0 * T) * (t02 * t10 + 2.0 * t11 * t01)
        M22 = (t20 * t02 + 2.0 * t11 * t11) / T
    t21, t12, t22 = relax(n21, M21, om[6]), relax(n12, M12, om[7]), relax(n22, M22, om[8])
    return populations(C, np.stack([t00, t10, t01, t20, t02, t11, t21, t12, t22]))


class Generic2D:
    """A 2D box (faces -x, +x, -y, +y) stepped with the generic-form method.  The state is the
    post-collision populations f, g of shape (9, ny, nx), x fastest, in the paper's link order."""

    def __init__(self, nx, ny, face, T_wall, T_ref, gbeta, gravity_axis, om_f, om_g, g_option=0,
                 dtype=np.float64):
        self.nx, self.ny = nx, ny
        self.face = list(face)[:4]
        self.T_wall = [float(t) for t in list(T_wall)[:4]]
        self.T_ref, self.gbeta, self.gaxis = float(T_ref), float(gbeta), int(gravity_axis)
        self.om_f, self.om_g = np.asarray(om_f, float), np.asarray(om_g, float)
        self.g_option = int(g_option)
        self.dtype = dtype
        self.profile = [None] * 4     # per-node wall temperature of a face (tangential index)
        self.f = self.g = None
        self._links()

    def _links(self):
        """Source index, wall mask and anti-bounce-back face of every link at every node."""
        ny, nx = self.ny, self.nx
        y, x = np.mgrid[0:ny, 0:nx]
        self.src = np.zeros((9, ny, nx), dtype=np.int64)
        self.out = np.zeros((9, ny, nx), dtype=bool)
        self.fixed = -np.ones((9, ny, nx), dtype=np.int64)
        for a in range(9):
            sx, sy = x - E[a, 0], y - E[a, 1]
            out = np.zeros((ny, nx), dtype=bool)
            fixed = -np.ones((ny, nx), dtype=np.int64)
            rank = -np.ones((ny, nx), dtype=np.int64)       # rank of the deciding face so far
            for ax, (c, ext) in enumerate(((sx, nx), (sy, ny))):
                for face, beyond in ((2 * ax, c < 0), (2 * ax + 1, c >= ext)):
                    if self.face[face] == PERIODIC:
                        c[beyond] = (c[beyond] + ext) % ext
                    else:
                        out |= beyond
                        # an edge link takes the rule of the crossed face that comes last in the
                        # order -y, -x, +x, +y (reading R7)
                        wins = beyond & (FACE_RANK[face] > rank)
                        rank[wins] = FACE_RANK[face]
                        fixed[wins] = face if self.face[face] == WALL_FIXED_T else -1
            self.src[a] = np.where(out, 0, sx + nx * sy)
            self.out[a] = out
            self.fixed[a] = fixed

    def set_wall_profile(self, face, Tw):
        self.profile[face] = np.asarray(Tw)

    def wall_T(self, face):
        """Wall temperature of `face` seen from every node, shape (ny, nx)."""
        ny, nx = self.ny, self.nx
        if self.profile[face] is None:
            return np.full((ny, nx), self.T_wall[face], dtype=self.dtype)
        p = self.profile[face]
        return np.broadcast_to(p[:, None] if face < 2 else p[None, :], (ny, nx)).astype(self.dtype)

    def set_state(self, f, g):
        self.f = np.array(f, dtype=self.dtype).reshape(9, self.ny, self.nx)
        self.g = np.array(g, dtype=self.dtype).reshape(9, self.ny, self.nx)

    def pull(self):
        """Populations after streaming, with the wall rules."""
        ff = self.f.reshape(9, -1)
        gg = self.g.reshape(9, -1)
        fo = np.empty_like(self.f)
        go = np.empty_like(self.g)
        tw = {fc: self.wall_T(fc) for fc in range(4) if self.face[fc] == WALL_FIXED_T}
        for a in range(9):
            o = OPP[a]
            inside_f = ff[a][self.src[a]]
            inside_g = gg[a][self.src[a]]
            fo[a] = np.where(self.out[a], self.f[o], inside_f)
            back = self.g[o]
            wall_g = back
            for fc, T_w in tw.items():
                wall_g = np.where(self.fixed[a] == fc, -back + 2.0 * W[a] * T_w, wall_g)
            go[a] = np.where(self.out[a], wall_g, inside_g)
        return fo, go

    def step(self, n=1):
        for _ in range(n):
            fo, go = self.pull()
            T = go.sum(axis=0)
            Fb = self.gbeta * (T - self.T_ref)
            zero = np.zeros_like(Fb)
            Fx, Fy = (Fb, zero) if self.gaxis == 0 else (zero, Fb)
            rho = fo.sum(axis=0)
            ux = ((fo * E[:, 0, None, None]).sum(axis=0) + 0.5 * Fx) / rho
            uy = ((fo * E[:, 1, None, None]).sum(axis=0) + 0.5 * Fy) / rho
            self.f = collide_f(fo, rho, ux, uy, Fx, Fy, self.om_f)
            self.g = collide_g(go, ux, uy, self.om_g, self.g_option)

    def nusselt_mean(self, face, L, dT):
        """Mean over the face of Nu = -sgn (L / dT)(-8/3 T_w + 3 T_1 - 1/3 T_2), sgn = +1 on a face at
        or above T_ref (Sec. 6.1, readings R14, R15)."""
        _, go = self.pull()
        T = go.sum(axis=0)
        ax, hi = face // 2, face & 1
        Tw = self.wall_T(face)
        if ax == 0:
            idx = [self.nx - 1, self.nx - 2] if hi else [0, 1]
            T1, T2, Twf = T[:, idx[0]], T[:, idx[1]], Tw[:, idx[0]]
        else:
            idx = [self.ny - 1, self.ny - 2] if hi else [0, 1]
            T1, T2, Twf = T[idx[0], :], T[idx[1], :], Tw[idx[0], :]
        sgn = 1.0 if self.T_wall[face] >= self.T_ref else -1.0
        return np.mean(-sgn * (L / dT) * (-8.0 / 3.0 * Twf + 3.0 * T1 - T2 / 3.0))
