"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name; they raise ``LbmError`` on a
non-zero status.  ``Lattice`` bundles a handle with torch-owned device memory and streams:
``use_torch_allocator()`` routes the library's device allocations through PyTorch's caching
allocator, and the handle's kernels are queued on the current torch stream.  There is no CPU
fallback: importing this module on a machine without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EDIVERGED, LBM_ETIMEOUT, LBM_ENOTSUP = 0, 1, 2, 3, 4, 5, 6
LBM_D2Q9_D2Q9, LBM_D3Q27_D3Q15 = 1, 2
LBM_FP64, LBM_FP32, LBM_FP16S = 0x000, 0x100, 0x200
LBM_PERIODIC, LBM_WALL_ADIABATIC, LBM_WALL_FIXED_T = 0, 1, 2

PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S}
LATTICES = {"d2q9": LBM_D2Q9_D2Q9, "d3q27": LBM_D3Q27_D3Q15}


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class lbm_bc(ctypes.Structure):
    _fields_ = [("face", ctypes.c_int * 6), ("T_wall", ctypes.c_double * 6),
                ("T_init", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("gravity_axis", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("perturb", ctypes.c_double)]


class lbm_info_t(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("precision", ctypes.c_int), ("nx", ctypes.c_int),
                ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("q_f", ctypes.c_int),
                ("q_g", ctypes.c_int), ("L", ctypes.c_double), ("dT", ctypes.c_double),
                ("U", ctypes.c_double), ("nu", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gbeta", ctypes.c_double), ("T_ref", ctypes.c_double),
                ("om_f", ctypes.c_double * 27), ("om_g", ctypes.c_double * 15),
                ("steps", ctypes.c_longlong), ("bytes_per_node_update", ctypes.c_double),
                ("state_bytes", ctypes.c_size_t), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("g_attractors", ctypes.c_int),
                ("fp16_stochastic", ctypes.c_int)]


class lbm_batch_info_t(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("total_nodes", ctypes.c_longlong),
                ("n_tiles", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("grid", ctypes.c_int),
                ("graph_steps", ctypes.c_int), ("steps", ctypes.c_longlong),
                ("bytes_per_node_update", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def lib() -> ctypes.CDLL:
    """Load liblbm.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        i, d, v, s = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        H = ctypes.c_void_p
        sig = {
            "lbm_set_allocator": [ALLOC_FN, FREE_FN, v],
            "lbm_create": [i, i, i, i, d, d, d, ctypes.POINTER(lbm_bc), ctypes.POINTER(H)],
            "lbm_destroy": [H],
            "lbm_set_stream": [H, v],
            "lbm_set_omegas": [H, dp, i, dp, i],
            "lbm_set_param": [H, ctypes.c_char_p, d],
            "lbm_info": [H, ctypes.POINTER(lbm_info_t)],
            "lbm_step": [H, ctypes.c_long],
            "lbm_sync": [H],
            "lbm_fields": [H, v, v, v, v, v, i],
            "lbm_nusselt": [H, i, dp, dp, dp, ip, ip],
            "lbm_nusselt_profile": [H, i, v, ctypes.c_long, i],
            "lbm_set_wall_profile": [H, i, dp, ctypes.c_long],
            "lbm_get_populations": [H, v, v, i],
            "lbm_set_populations": [H, v, v, i],
            "lbm_get_state": [H, v, s],
            "lbm_set_state": [H, v, s],
            "lbm_nusselt_static": [i, i, i, i, ip, dp, d, v, i, d, d, v, v],
            "lbm_adjoint_step": [H, ctypes.c_long, i, i, dp, dp, ctypes.c_long],
            "lbm_probe_bounded_wait": [d, ip],
            "lbm_batch_create": [i, i, ip, ip, dp, dp, d, ctypes.POINTER(lbm_bc), ctypes.POINTER(H)],
            "lbm_batch_destroy": [H],
            "lbm_batch_set_stream": [H, v],
            "lbm_batch_set_launch": [H, i, i, i, i],
            "lbm_batch_tune": [H, i, ip, ip, ip],
            "lbm_batch_step": [H, ctypes.c_long],
            "lbm_batch_sync": [H, ip],
            "lbm_batch_nusselt": [H, i, i, dp, dp, dp, ip, ip],
            "lbm_batch_get_populations": [H, i, dp, dp],
            "lbm_batch_set_populations": [H, i, dp, dp],
            "lbm_batch_info": [H, ctypes.POINTER(lbm_batch_info_t)],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.lbm_last_error.argtypes = [H]
        L.lbm_last_error.restype = ctypes.c_char_p
        L.lbm_batch_last_error.argtypes = [H]
        L.lbm_batch_last_error.restype = ctypes.c_char_p
        L.lbm_status_string.argtypes = [i]
        L.lbm_status_string.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, h=None):
    if status != LBM_OK:
        msg = lib().lbm_last_error(h).decode()
        raise LbmError(status, msg or lib().lbm_status_string(status).decode())


def _dptr(a):
    return None if a is None else ctypes.cast(a, ctypes.POINTER(ctypes.c_double))


# ---------------------------------------------------------------------------------------------
# Entry points under their C names
# ---------------------------------------------------------------------------------------------

def lbm_set_allocator(alloc=None, free=None, ctx=None):
    _check(lib().lbm_set_allocator(alloc or ALLOC_FN(), free or FREE_FN(), ctx))


def lbm_create(lattice: int, nx: int, ny: int, nz: int, Ra: float, Pr: float, Ma: float,
               bc: lbm_bc) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().lbm_create(lattice, nx, ny, nz, Ra, Pr, Ma, ctypes.byref(bc), ctypes.byref(h)))
    return h


def lbm_destroy(h):
    _check(lib().lbm_destroy(h))


def lbm_set_stream(h, stream: int):
    _check(lib().lbm_set_stream(h, ctypes.c_void_p(stream)), h)


def lbm_set_omegas(h, om_f=None, om_g=None):
    af = None if om_f is None else np.ascontiguousarray(om_f, dtype=np.float64)
    ag = None if om_g is None else np.ascontiguousarray(om_g, dtype=np.float64)
    _check(lib().lbm_set_omegas(h, _dptr(None if af is None else af.ctypes.data),
                                0 if af is None else af.size,
                                _dptr(None if ag is None else ag.ctypes.data),
                                0 if ag is None else ag.size), h)


def lbm_set_param(h, key: str, value: float):
    _check(lib().lbm_set_param(h, key.encode(), value), h)


def lbm_info(h) -> lbm_info_t:
    out = lbm_info_t()
    _check(lib().lbm_info(h, ctypes.byref(out)), h)
    return out


def lbm_step(h, n: int):
    _check(lib().lbm_step(h, n), h)


def lbm_sync(h):
    _check(lib().lbm_sync(h), h)


def lbm_fields(h, rho, ux, uy, uz, T, device_ptrs: int):
    _check(lib().lbm_fields(h, rho, ux, uy, uz, T, device_ptrs), h)


def lbm_nusselt(h, face: int):
    mean, mx, mn = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    jmx, jmn = ctypes.c_int(), ctypes.c_int()
    _check(lib().lbm_nusselt(h, face, ctypes.byref(mean), ctypes.byref(mx), ctypes.byref(mn),
                             ctypes.byref(jmx), ctypes.byref(jmn)), h)
    return mean.value, mx.value, mn.value, jmx.value, jmn.value


def lbm_nusselt_profile(h, face: int, ptr: int, n: int, device_ptrs: int):
    _check(lib().lbm_nusselt_profile(h, face, ptr, n, device_ptrs), h)


def lbm_set_wall_profile(h, face: int, T_w):
    if T_w is None:
        _check(lib().lbm_set_wall_profile(h, face, None, 0), h)
        return
    a = np.ascontiguousarray(T_w, dtype=np.float64)
    _check(lib().lbm_set_wall_profile(h, face, _dptr(a.ctypes.data), a.size), h)


def lbm_get_populations(h, f_ptr: int, g_ptr: int, device_ptrs: int):
    _check(lib().lbm_get_populations(h, f_ptr, g_ptr, device_ptrs), h)


def lbm_set_populations(h, f_ptr: int, g_ptr: int, device_ptrs: int):
    _check(lib().lbm_set_populations(h, f_ptr, g_ptr, device_ptrs), h)


def lbm_get_state(h, buf: np.ndarray):
    _check(lib().lbm_get_state(h, buf.ctypes.data, buf.nbytes), h)


def lbm_set_state(h, buf: np.ndarray):
    _check(lib().lbm_set_state(h, buf.ctypes.data, buf.nbytes), h)


def lbm_adjoint_step(h, n_steps: int, objective_face: int, design_face: int, n: int):
    """(J, dJ/dT_w) for J = mean Nu on objective_face after n_steps, T_w the design-face profile."""
    J = ctypes.c_double()
    grad = np.zeros(n)
    _check(lib().lbm_adjoint_step(h, n_steps, objective_face, design_face, ctypes.byref(J),
                                  _dptr(grad.ctypes.data), n), h)
    return J.value, grad


NUSSELT_STATIC_MAX_FACE_NODES = 1048576


def lbm_nusselt_static(lattice: int, nx: int, ny: int, nz: int, face_kind, T_wall, T_ref: float,
                       g_ptr: int, face: int, L: float, dT: float, result_ptr: int, stream: int = 0):
    """The allocation-free Nusselt reduction: populations and the 5-double result are device
    buffers the caller owns (see include/lbm.h)."""
    fk = (ctypes.c_int * 6)(*face_kind)
    tw = (ctypes.c_double * 6)(*T_wall)
    st = lib().lbm_nusselt_static(lattice, nx, ny, nz, fk, tw, T_ref, ctypes.c_void_p(g_ptr), face,
                                  L, dT, ctypes.c_void_p(result_ptr), ctypes.c_void_p(stream))
    if st != LBM_OK:
        raise LbmError(st, lib().lbm_last_error(None).decode() or lib().lbm_status_string(st).decode())


def _bcheck(status: int, b=None):
    if status != LBM_OK:
        msg = lib().lbm_batch_last_error(b).decode()
        raise LbmError(status, msg or lib().lbm_status_string(status).decode())


def lbm_batch_create(lattice: int, nx, ny, Ra, Pr, Ma: float, bcs) -> ctypes.c_void_p:
    n = len(nx)
    if not (len(ny) == len(Ra) == len(Pr) == len(bcs) == n):
        raise ValueError("nx, ny, Ra, Pr and bcs must have one entry per member")
    b = ctypes.c_void_p()
    _bcheck(lib().lbm_batch_create(lattice, n, (ctypes.c_int * n)(*nx), (ctypes.c_int * n)(*ny),
                                   (ctypes.c_double * n)(*Ra), (ctypes.c_double * n)(*Pr), Ma,
                                   (lbm_bc * n)(*bcs), ctypes.byref(b)))
    return b


def lbm_batch_destroy(b):
    _bcheck(lib().lbm_batch_destroy(b), b)


def lbm_batch_set_stream(b, stream: int):
    _bcheck(lib().lbm_batch_set_stream(b, ctypes.c_void_p(stream)), b)


def lbm_batch_set_launch(b, tile_x: int, tile_y: int, ctas_per_sm: int, graph_steps: int):
    _bcheck(lib().lbm_batch_set_launch(b, tile_x, tile_y, ctas_per_sm, graph_steps), b)


def lbm_batch_tune(b, trial_steps: int):
    """Autotune the launch shape; returns (tile_x, tile_y, ctas_per_sm)."""
    tx, ty, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().lbm_batch_tune(b, trial_steps, ctypes.byref(tx), ctypes.byref(ty),
                                 ctypes.byref(c)), b)
    return tx.value, ty.value, c.value


def lbm_batch_step(b, n: int):
    _bcheck(lib().lbm_batch_step(b, n), b)


def lbm_batch_sync(b, count: int):
    """Per-member divergence flags (numpy int32); raises nothing for diverged members."""
    flags = np.zeros(count, dtype=np.int32)
    st = lib().lbm_batch_sync(b, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if st not in (LBM_OK, LBM_EDIVERGED):
        _bcheck(st, b)
    return flags


def lbm_batch_nusselt(b, member: int, face: int):
    mean, mx, mn = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    jx, jn = ctypes.c_int(), ctypes.c_int()
    _bcheck(lib().lbm_batch_nusselt(b, member, face, ctypes.byref(mean), ctypes.byref(mx),
                                    ctypes.byref(mn), ctypes.byref(jx), ctypes.byref(jn)), b)
    return mean.value, mx.value, mn.value, jx.value, jn.value


def lbm_batch_get_populations(b, member: int, f: np.ndarray, g: np.ndarray):
    _bcheck(lib().lbm_batch_get_populations(b, member, _dptr(f.ctypes.data), _dptr(g.ctypes.data)), b)


def lbm_batch_set_populations(b, member: int, f: np.ndarray, g: np.ndarray):
    _bcheck(lib().lbm_batch_set_populations(b, member, _dptr(f.ctypes.data), _dptr(g.ctypes.data)), b)


def lbm_batch_info(b) -> lbm_batch_info_t:
    out = lbm_batch_info_t()
    _bcheck(lib().lbm_batch_info(b, ctypes.byref(out)), b)
    return out


def lbm_batch_last_error(b=None) -> str:
    return lib().lbm_batch_last_error(b).decode()


def lbm_probe_bounded_wait(seconds: float):
    """Self-test of the bounded device waits: returns (status, timed_out); LBM_ETIMEOUT with
    timed_out = 1 is the expected outcome (the wait runs out and the kernel returns)."""
    t = ctypes.c_int(-1)
    st = lib().lbm_probe_bounded_wait(float(seconds), ctypes.byref(t))
    if st not in (LBM_OK, LBM_ETIMEOUT):
        raise LbmError(st, lib().lbm_status_string(st).decode())
    return st, t.value


def lbm_last_error(h=None) -> str:
    return lib().lbm_last_error(h).decode()


def lbm_status_string(status: int) -> str:
    return lib().lbm_status_string(status).decode()


# ---------------------------------------------------------------------------------------------
# Torch plumbing: device memory and streams
# ---------------------------------------------------------------------------------------------

_torch_hooks = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _torch_hooks
    import torch

    def _alloc(nbytes, _ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None

    def _free(ptr, _ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    if _torch_hooks is None:
        _torch_hooks = (ALLOC_FN(_alloc), FREE_FN(_free))
    _check(lib().lbm_set_allocator(_torch_hooks[0], _torch_hooks[1], None))


def use_cuda_allocator():
    _check(lib().lbm_set_allocator(ALLOC_FN(), FREE_FN(), None))


@dataclass
class Walls:
    """Boundary description of a box (faces -x, +x, -y, +y, -z, +z)."""
    face: tuple = (LBM_PERIODIC,) * 6
    T_wall: tuple = (0.0,) * 6
    T_init: float = 0.5
    T_ref: float = 0.5
    gravity_axis: int = 1
    seed: int = 0
    perturb: float = 0.0

    def to_c(self) -> lbm_bc:
        return lbm_bc((ctypes.c_int * 6)(*self.face), (ctypes.c_double * 6)(*self.T_wall),
                      self.T_init, self.T_ref, self.gravity_axis, self.seed, self.perturb)

    @staticmethod
    def cavity(dim: int, T_hot: float = 1.0, T_cold: float = 0.0) -> "Walls":
        """Hot -x, cold +x, other walls adiabatic, no slip everywhere (Sec. 6.1, Sec. 6.2)."""
        face = (LBM_WALL_FIXED_T, LBM_WALL_FIXED_T) + (LBM_WALL_ADIABATIC,) * 4
        mid = 0.5 * (T_hot + T_cold)
        return Walls(face, (T_hot, T_cold, 0, 0, 0, 0), mid, mid, 1 if dim == 2 else 2)

    @staticmethod
    def rayleigh_benard(T_hot=1.0, T_cold=0.0, seed=0, perturb=1e-3) -> "Walls":
        """Periodic x, hot bottom (-y), cold top (+y), gravity along y."""
        face = (LBM_PERIODIC, LBM_PERIODIC, LBM_WALL_FIXED_T, LBM_WALL_FIXED_T,
                LBM_PERIODIC, LBM_PERIODIC)
        mid = 0.5 * (T_hot + T_cold)
        return Walls(face, (0, 0, T_hot, T_cold, 0, 0), mid, mid, 1, seed, perturb)


class Lattice:
    """A box advanced by liblbm.so with torch-managed device memory and stream."""

    def __init__(self, lattice: str, nx: int, ny: int, nz: int = 1, Ra: float = 1e4,
                 Pr: float = 0.71, Ma: float = 0.1, walls: Walls | None = None,
                 precision: str = "fp32", stream=None, torch_allocator: bool = True):
        import torch
        self.torch = torch
        if torch_allocator:
            use_torch_allocator()
        else:
            use_cuda_allocator()
        self.dim = 2 if lattice == "d2q9" else 3
        self.walls = walls or Walls.cavity(self.dim)
        code = LATTICES[lattice] | PRECISIONS[precision]
        self.h = lbm_create(code, nx, ny, nz if self.dim == 3 else 1, Ra, Pr, Ma, self.walls.to_c())
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lbm_set_stream(self.h, self.stream.cuda_stream)
        inf = self.info()
        self.nx, self.ny, self.nz = inf.nx, inf.ny, inf.nz
        self.qf, self.qg = inf.q_f, inf.q_g
        self.n = self.nx * self.ny * self.nz

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    def info(self) -> lbm_info_t:
        return lbm_info(self.h)

    def set_omegas(self, om_f=None, om_g=None):
        lbm_set_omegas(self.h, om_f, om_g)

    def set_param(self, key, value):
        lbm_set_param(self.h, key, value)

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def sync(self):
        lbm_sync(self.h)

    def fields(self) -> dict:
        """rho, ux, uy, uz, T as FP64 torch tensors on the device, shape (nz, ny, nx)."""
        t = self.torch
        out = {k: t.empty(self.shape, dtype=t.float64, device="cuda") for k in
               ("rho", "ux", "uy", "uz", "T")}
        lbm_fields(self.h, *[out[k].data_ptr() for k in ("rho", "ux", "uy", "uz", "T")], 1)
        return out

    def nusselt(self, face: int):
        return lbm_nusselt(self.h, face)

    def nusselt_profile(self, face: int):
        ax = face // 2
        n = {0: self.ny * self.nz, 1: self.nx * self.nz, 2: self.nx * self.ny}[ax]
        out = self.torch.empty(n, dtype=self.torch.float64, device="cuda")
        lbm_nusselt_profile(self.h, face, out.data_ptr(), n, 1)
        return out

    def set_wall_profile(self, face: int, T_w):
        lbm_set_wall_profile(self.h, face, T_w)

    def face_nodes(self, face: int) -> int:
        return {0: self.ny * self.nz, 1: self.nx * self.nz, 2: self.nx * self.ny}[face // 2]

    def adjoint(self, n_steps: int, objective_face: int, design_face: int):
        """J and dJ/dT_w (numpy) by the checkpointed adjoint; the state advances n_steps."""
        return lbm_adjoint_step(self.h, n_steps, objective_face, design_face,
                                self.face_nodes(design_face))

    def get_populations(self, device: bool = False):
        """Post-collision state as FP64 arrays (q, nz, ny, nx): numpy, or torch on the device."""
        t = self.torch
        if device:
            f = t.empty((self.qf, *self.shape), dtype=t.float64, device="cuda")
            g = t.empty((self.qg, *self.shape), dtype=t.float64, device="cuda")
            lbm_get_populations(self.h, f.data_ptr(), g.data_ptr(), 1)
            return f, g
        f = np.empty((self.qf, *self.shape)); g = np.empty((self.qg, *self.shape))
        lbm_get_populations(self.h, f.ctypes.data, g.ctypes.data, 0)
        return f, g

    def set_populations(self, f, g):
        t = self.torch
        if isinstance(f, t.Tensor) and f.is_cuda:
            f = f.to(t.float64).contiguous(); g = g.to(t.float64).contiguous()
            lbm_set_populations(self.h, f.data_ptr(), g.data_ptr(), 1)
            self.stream.synchronize()
            return
        f = np.ascontiguousarray(f, dtype=np.float64); g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.qf * self.n and g.size == self.qg * self.n
        lbm_set_populations(self.h, f.ctypes.data, g.ctypes.data, 0)

    def get_state(self) -> np.ndarray:
        buf = np.empty(self.info().state_bytes, dtype=np.uint8)
        lbm_get_state(self.h, buf)
        return buf

    def set_state(self, buf: np.ndarray):
        lbm_set_state(self.h, np.ascontiguousarray(buf, dtype=np.uint8))


class Batch:
    """Many 2D boxes advanced together by one kernel launch per step (lbm_batch_*)."""

    def __init__(self, sizes, Ra, Pr, Ma: float = 0.1, walls=None, precision: str = "fp32",
                 stream=None, torch_allocator: bool = True):
        import torch
        self.torch = torch
        if torch_allocator:
            use_torch_allocator()
        else:
            use_cuda_allocator()
        self.sizes = [(int(a), int(b)) for a, b in sizes]
        self.count = len(self.sizes)
        if walls is None:
            walls = [Walls.cavity(2)] * self.count
        elif isinstance(walls, Walls):
            walls = [walls] * self.count
        self.walls = list(walls)
        self.b = lbm_batch_create(LBM_D2Q9_D2Q9 | PRECISIONS[precision],
                                  [s[0] for s in self.sizes], [s[1] for s in self.sizes],
                                  list(Ra), list(Pr), Ma, [w.to_c() for w in self.walls])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        lbm_batch_set_stream(self.b, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> lbm_batch_info_t:
        return lbm_batch_info(self.b)

    def set_launch(self, tile_x: int, tile_y: int, ctas_per_sm: int, graph_steps: int = 32):
        lbm_batch_set_launch(self.b, tile_x, tile_y, ctas_per_sm, graph_steps)

    def tune(self, trial_steps: int = 20):
        return lbm_batch_tune(self.b, trial_steps)

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n)

    def sync(self):
        """Wait for the batch; returns the per-member divergence flags."""
        return lbm_batch_sync(self.b, self.count)

    def nusselt(self, member: int, face: int):
        return lbm_batch_nusselt(self.b, member, face)

    def get_populations(self, member: int):
        nx, ny = self.sizes[member]
        f = np.empty((9, 1, ny, nx)); g = np.empty((9, 1, ny, nx))
        lbm_batch_get_populations(self.b, member, f, g)
        return f, g

    def set_populations(self, member: int, f, g):
        nx, ny = self.sizes[member]
        f = np.ascontiguousarray(f, dtype=np.float64); g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == 9 * nx * ny and g.size == 9 * nx * ny
        lbm_batch_set_populations(self.b, member, f, g)


def wall_nusselt_objective(lattice: "Lattice", state0, n_steps: int, objective_face: int,
                           design_face: int):
    """A torch function T_w -> J: the mean Nusselt number on objective_face after n_steps steps
    from the checkpoint state0, as a differentiable function of the design-face temperatures.
    Its backward is the library's adjoint (lbm_adjoint_step)."""
    import torch

    class _WallNusselt(torch.autograd.Function):
        @staticmethod
        def forward(ctx, T_w):
            lattice.set_state(state0)
            lattice.set_wall_profile(design_face, T_w.detach().cpu().double().numpy())
            J, grad = lattice.adjoint(n_steps, objective_face, design_face)
            ctx.save_for_backward(torch.from_numpy(grad).to(T_w.device, T_w.dtype))
            return torch.tensor(J, dtype=T_w.dtype, device=T_w.device)

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ * grad

    return _WallNusselt.apply
