"""Thin ctypes binding of the C ABI declared in ``include/lbmtau1.h``.

The functions keep the C names and only marshal arguments; every step of the
LBMTau1 path runs in the sm_103a kernels of ``liblbmtau1.so``.  PyTorch is
used by ``Domain`` for the device workspace and the CUDA stream only.
Importing this module raises if the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

LBM_OK = 0
LBM_E_INVAL = -1
LBM_E_WORKSPACE = -2
LBM_E_CUDA = -3
LBM_E_UNSTABLE = -4
LBM_E_STATE = -5
LBM_FLUID, LBM_SOLID, LBM_FIXED = 0, 1, 2
LBM_STORAGE_F32 = 0
LBM_STORAGE_F16 = 1
LBM_STORAGE_BF16 = 2
STORAGE_NAMES = {"f32": LBM_STORAGE_F32, "f16": LBM_STORAGE_F16,
                 "bf16": LBM_STORAGE_BF16}
LBM_ROUND_DEFAULT = 0      # 16-bit: stochastic, FP32: nearest
LBM_ROUND_NEAREST = 1
LBM_ROUND_STOCHASTIC = 2
ROUNDING_NAMES = {"default": LBM_ROUND_DEFAULT,
                  "stochastic": LBM_ROUND_STOCHASTIC,
                  "nearest": LBM_ROUND_NEAREST}
# host dtype of the exact state transfers (bfloat16 as raw 16-bit words)
STATE_DTYPE = {LBM_STORAGE_F32: np.float32, LBM_STORAGE_F16: np.float16,
               LBM_STORAGE_BF16: np.uint16}

LIB_PATH = _build.LIB
if not os.path.exists(LIB_PATH):
    raise ImportError(
        "liblbmtau1.so is not built (run __graft_entry__.build()); the LBMTau1 "
        "path has no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)


class lbm_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("storage", ctypes.c_int32), ("rounding", ctypes.c_int32),
                ("sc_g", ctypes.c_double)]


_P = ctypes.POINTER(lbm_params)
_vp = ctypes.c_void_p
_lib.lbm_workspace_bytes.argtypes = [_P]
_lib.lbm_workspace_bytes.restype = ctypes.c_size_t
_lib.lbm_create.argtypes = [_P, _vp, ctypes.c_size_t, _vp,
                            ctypes.POINTER(_vp)]
_lib.lbm_create.restype = ctypes.c_int
_lib.lbm_set_geometry.argtypes = [_vp, _vp]
_lib.lbm_set_geometry.restype = ctypes.c_int
_lib.lbm_set_moments.argtypes = [_vp, _vp, _vp, _vp]
_lib.lbm_set_moments.restype = ctypes.c_int
_lib.lbm_step.argtypes = [_vp, ctypes.c_int64]
_lib.lbm_step.restype = ctypes.c_int
_lib.lbm_step_count.argtypes = [_vp, _vp]
_lib.lbm_step_count.restype = ctypes.c_int
_lib.lbm_set_step_count.argtypes = [_vp, ctypes.c_int64]
_lib.lbm_set_step_count.restype = ctypes.c_int
_lib.lbm_set_variant.argtypes = [_vp, ctypes.c_int32]
_lib.lbm_set_variant.restype = ctypes.c_int
_lib.lbm_variant.argtypes = [_vp]
_lib.lbm_variant.restype = ctypes.c_int32
_lib.lbm_set_copy_wait_ns.argtypes = [_vp, ctypes.c_int64]
_lib.lbm_set_copy_wait_ns.restype = ctypes.c_int
_lib.lbm_snapshot_bytes.argtypes = [_P]
_lib.lbm_snapshot_bytes.restype = ctypes.c_size_t
_lib.lbm_snapshot.argtypes = [_vp, _vp, ctypes.c_size_t]
_lib.lbm_snapshot.restype = ctypes.c_int
_lib.lbm_change_since.argtypes = [_vp, _vp, ctypes.c_int64,
                                  ctypes.POINTER(ctypes.c_double)]
_lib.lbm_change_since.restype = ctypes.c_int
_lib.lbm_moments.argtypes = [_vp, _vp, _vp, _vp]
_lib.lbm_moments.restype = ctypes.c_int
_lib.lbm_get_state.argtypes = [_vp, _vp, _vp, _vp]
_lib.lbm_get_state.restype = ctypes.c_int
_lib.lbm_set_state.argtypes = [_vp, _vp, _vp, _vp]
_lib.lbm_set_state.restype = ctypes.c_int
_lib.lbm_residual.argtypes = [_vp, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double)]
_lib.lbm_residual.restype = ctypes.c_int
_lib.lbm_step_noalloc.argtypes = [_vp] * 7 + [ctypes.c_int64] * 3 + \
    [ctypes.c_int32] * 2 + [ctypes.c_double] * 2 + [_vp, _vp, _vp]
_lib.lbm_step_noalloc.restype = ctypes.c_int
_lib.lbm_batch_workspace_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64]
_lib.lbm_batch_workspace_bytes.restype = ctypes.c_size_t
_lib.lbm_batch_create.argtypes = [ctypes.c_int32, ctypes.c_int64, _vp,
                                  ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]
_lib.lbm_batch_create.restype = ctypes.c_int
_lib.lbm_batch_add.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_int32)]
_lib.lbm_batch_add.restype = ctypes.c_int
_lib.lbm_batch_remove.argtypes = [_vp, ctypes.c_int32]
_lib.lbm_batch_remove.restype = ctypes.c_int
_lib.lbm_batch_members.argtypes = [_vp]
_lib.lbm_batch_members.restype = ctypes.c_int32
_lib.lbm_batch_step.argtypes = [_vp, ctypes.c_int64]
_lib.lbm_batch_step.restype = ctypes.c_int
_lib.lbm_variant_count.argtypes = []
_lib.lbm_variant_count.restype = ctypes.c_int32
_lib.lbm_tile_count.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32]
_lib.lbm_tile_count.restype = ctypes.c_int64
_lib.lbm_variant_tile.argtypes = [ctypes.c_int32, _vp, _vp, _vp]
_lib.lbm_variant_tile.restype = ctypes.c_int
_lib.lbm_variant_has_clean_code.argtypes = [ctypes.c_int32]
_lib.lbm_variant_has_clean_code.restype = ctypes.c_int32
_lib.lbm_batch_set_variant.argtypes = [_vp, ctypes.c_int32]
_lib.lbm_batch_set_variant.restype = ctypes.c_int
_lib.lbm_batch_variant.argtypes = [_vp]
_lib.lbm_batch_variant.restype = ctypes.c_int32
_lib.lbm_batch_autotune.argtypes = [_vp, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32), _vp]
_lib.lbm_batch_autotune.restype = ctypes.c_int
_lib.lbm_batch_residuals.argtypes = [_vp, _vp, _vp, _vp]
_lib.lbm_batch_residuals.restype = ctypes.c_int
_lib.lbm_batch_destroy.argtypes = [_vp]
_lib.lbm_batch_destroy.restype = None
_lib.lbm_batch_last_error.argtypes = [_vp]
_lib.lbm_batch_last_error.restype = ctypes.c_char_p
_lib.lbm_destroy.argtypes = [_vp]
_lib.lbm_destroy.restype = None
_lib.lbm_last_error.argtypes = [_vp]
_lib.lbm_last_error.restype = ctypes.c_char_p
_lib.lbm_status_string.argtypes = [ctypes.c_int]
_lib.lbm_status_string.restype = ctypes.c_char_p


class LbmError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (lbm_status_string(status), message))
        self.status = status


def lbm_status_string(status: int) -> str:
    return _lib.lbm_status_string(int(status)).decode()


def lbm_last_error(ctx) -> str:
    return _lib.lbm_last_error(ctx).decode()


def _check(status, ctx=None):
    if status != LBM_OK:
        raise LbmError(status, lbm_last_error(ctx) if ctx else "")
    return status


def make_params(nx, ny, periodic=(False, False), force=(0.0, 0.0),
                storage=LBM_STORAGE_F32,
                rounding=LBM_ROUND_DEFAULT, sc_g=0.0) -> lbm_params:
    if isinstance(rounding, str):
        rounding = ROUNDING_NAMES[rounding]
    return lbm_params(int(nx), int(ny), int(bool(periodic[0])),
                      int(bool(periodic[1])), float(force[0]), float(force[1]),
                      int(storage), int(rounding), float(sc_g))


def _ptr(a):
    """Address of a host buffer: a C-contiguous numpy array or CPU tensor."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous")
        return a.ctypes.data
    return int(a.data_ptr())


def lbm_workspace_bytes(params: lbm_params) -> int:
    return int(_lib.lbm_workspace_bytes(ctypes.byref(params)))


def lbm_create(params: lbm_params, dev_workspace: int, workspace_bytes: int,
               cuda_stream: int = 0):
    ctx = _vp()
    _check(_lib.lbm_create(ctypes.byref(params), _vp(dev_workspace),
                           workspace_bytes, _vp(cuda_stream),
                           ctypes.byref(ctx)))
    return ctx


def lbm_set_geometry(ctx, host_mask) -> None:
    if isinstance(host_mask, np.ndarray):
        host_mask = np.ascontiguousarray(host_mask, dtype=np.uint8)
    _check(_lib.lbm_set_geometry(ctx, _vp(_ptr(host_mask))), ctx)


def lbm_set_moments(ctx, rho, jx, jy) -> None:
    """Host density and momentum (float64, nx*ny each)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64)
            if isinstance(a, np.ndarray) else a for a in (rho, jx, jy)]
    _check(_lib.lbm_set_moments(ctx, *[_vp(_ptr(a)) for a in arrs]), ctx)


def lbm_step(ctx, nsteps: int) -> None:
    _check(_lib.lbm_step(ctx, int(nsteps)), ctx)


def lbm_step_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(_lib.lbm_step_count(ctx, ctypes.byref(n)), ctx)
    return int(n.value)


def lbm_set_step_count(ctx, steps: int) -> None:
    _check(_lib.lbm_set_step_count(ctx, int(steps)), ctx)


def lbm_set_variant(ctx, variant: int) -> None:
    """Tile variant of the context's step kernel; -1 = automatic."""
    _check(_lib.lbm_set_variant(ctx, int(variant)), ctx)


def lbm_variant(ctx) -> int:
    return int(_lib.lbm_variant(ctx))


def lbm_set_copy_wait_ns(ctx, ns: int) -> None:
    """Wait limit of the step kernel for a staged row copy (0 .. 1e9 ns)."""
    _check(_lib.lbm_set_copy_wait_ns(ctx, int(ns)), ctx)


def lbm_moments(ctx, rho, jx, jy) -> None:
    """Fills caller-owned host float64 buffers (numpy or pinned tensors)."""
    for a in (rho, jx, jy):
        if isinstance(a, np.ndarray) and a.dtype != np.float64:
            raise TypeError("moment buffers must be float64")
    _check(_lib.lbm_moments(ctx, *[_vp(_ptr(a)) for a in (rho, jx, jy)]), ctx)


def lbm_get_state(ctx, drho, jx, jy) -> None:
    """Fills host buffers with the stored rho - 1, jx, jy (storage format;
    the caller's arrays must have its element size)."""
    _check(_lib.lbm_get_state(ctx, *[_vp(_ptr(a)) for a in (drho, jx, jy)]), ctx)


def lbm_set_state(ctx, drho, jx, jy) -> None:
    """Loads rho - 1, jx, jy in the storage format exactly."""
    arrs = [np.ascontiguousarray(a) if isinstance(a, np.ndarray) else a
            for a in (drho, jx, jy)]
    _check(_lib.lbm_set_state(ctx, *[_vp(_ptr(a)) for a in arrs]), ctx)


def lbm_residual(ctx):
    """(residual, mass) of the last step; raises LbmError(LBM_E_UNSTABLE)."""
    r = ctypes.c_double(); m = ctypes.c_double()
    st = _lib.lbm_residual(ctx, ctypes.byref(r), ctypes.byref(m))
    _check(st, ctx)
    return r.value, m.value


def lbm_step_noalloc(drho_in, jx_in, jy_in, drho_out, jx_out, jy_out, mask,
                     nx, ny, pitch, periodic, force, dev_sums, dev_flags,
                     cuda_stream=0) -> None:
    """One reduced step between caller-owned device buffers (addresses as
    ints), with no allocation; see include/lbmtau1.h."""
    st = _lib.lbm_step_noalloc(
        *[_vp(int(p)) for p in (drho_in, jx_in, jy_in, drho_out, jx_out,
                                 jy_out, mask)],
        int(nx), int(ny), int(pitch), int(bool(periodic[0])),
        int(bool(periodic[1])), float(force[0]), float(force[1]),
        _vp(int(dev_sums)), _vp(int(dev_flags)), _vp(int(cuda_stream)))
    if st != LBM_OK:
        raise LbmError(st, "lbm_step_noalloc")


def lbm_destroy(ctx) -> None:
    _lib.lbm_destroy(ctx)


def _bcheck(status, b):
    if status != LBM_OK:
        raise LbmError(status, _lib.lbm_batch_last_error(b).decode())


def lbm_batch_workspace_bytes(capacity: int, max_tiles: int) -> int:
    return int(_lib.lbm_batch_workspace_bytes(int(capacity), int(max_tiles)))


def lbm_batch_create(capacity, max_tiles, dev_workspace, workspace_bytes,
                     cuda_stream=0):
    b = _vp()
    _check(_lib.lbm_batch_create(int(capacity), int(max_tiles),
                                 _vp(dev_workspace), workspace_bytes,
                                 _vp(cuda_stream), ctypes.byref(b)))
    return b


def lbm_batch_add(b, ctx) -> int:
    slot = ctypes.c_int32()
    _bcheck(_lib.lbm_batch_add(b, ctx, ctypes.byref(slot)), b)
    return slot.value


def lbm_batch_remove(b, slot) -> None:
    _bcheck(_lib.lbm_batch_remove(b, int(slot)), b)


def lbm_batch_members(b) -> int:
    return int(_lib.lbm_batch_members(b))


def lbm_batch_step(b, nsteps) -> None:
    _bcheck(_lib.lbm_batch_step(b, int(nsteps)), b)


def lbm_variant_count() -> int:
    return int(_lib.lbm_variant_count())


def lbm_variant_has_clean_code(variant: int) -> bool:
    r = int(_lib.lbm_variant_has_clean_code(int(variant)))
    if r < 0:
        raise LbmError(LBM_E_INVAL, "no tile variant %d" % variant)
    return r == 1


def lbm_variant_tile(variant: int):
    """(tile_x, tile_y, columns per lane) of a tile variant."""
    tx, ty = ctypes.c_int64(), ctypes.c_int64()
    cols = ctypes.c_int32()
    st = _lib.lbm_variant_tile(int(variant), ctypes.byref(tx), ctypes.byref(ty),
                               ctypes.byref(cols))
    if st != LBM_OK:
        raise LbmError(st, "invalid variant %d" % variant)
    return int(tx.value), int(ty.value), int(cols.value)


def lbm_tile_count(nx: int, ny: int, variant: int = -1) -> int:
    """Block tiles of an nx x ny domain (variant -1: the most over all)."""
    n = int(_lib.lbm_tile_count(int(nx), int(ny), int(variant)))
    if n < 0:
        raise LbmError(LBM_E_INVAL, "invalid tile count arguments")
    return n


def lbm_batch_set_variant(b, variant) -> None:
    _bcheck(_lib.lbm_batch_set_variant(b, int(variant)), b)


def lbm_batch_variant(b) -> int:
    return int(_lib.lbm_batch_variant(b))


def lbm_batch_autotune(b, steps_per_variant=10):
    """Returns (chosen variant, per-variant ms/step list)."""
    n = lbm_variant_count()
    ms = (ctypes.c_double * n)()
    chosen = ctypes.c_int32()
    _bcheck(_lib.lbm_batch_autotune(b, int(steps_per_variant),
                                    ctypes.byref(chosen), ms), b)
    return chosen.value, list(ms)


def lbm_batch_residuals(b, capacity):
    """(residual, mass, status) arrays indexed by slot."""
    res = np.zeros(capacity, np.float64)
    mass = np.zeros(capacity, np.float64)
    st = np.zeros(capacity, np.int32)
    _bcheck(_lib.lbm_batch_residuals(b, _vp(res.ctypes.data),
                                     _vp(mass.ctypes.data),
                                     _vp(st.ctypes.data)), b)
    return res, mass, st


def lbm_batch_destroy(b) -> None:
    _lib.lbm_batch_destroy(b)


class Batch:
    """A batch of Domains stepped together (one launch per step); the
    workspace comes from torch, the stream is shared with the members."""

    def __init__(self, capacity, max_tiles, device="cuda", stream=None):
        import torch
        self.capacity = int(capacity)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = lbm_batch_workspace_bytes(capacity, max_tiles)
        if nbytes == 0:
            raise LbmError(LBM_E_INVAL, "invalid batch size")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.handle = lbm_batch_create(capacity, max_tiles,
                                       self.workspace.data_ptr(), nbytes,
                                       self.stream.cuda_stream)
        self.members = {}

    def add(self, dom):
        slot = lbm_batch_add(self.handle, dom.ctx)
        self.members[slot] = dom
        return slot

    def remove(self, slot):
        lbm_batch_remove(self.handle, slot)
        self.members.pop(slot, None)

    def step(self, nsteps=1):
        lbm_batch_step(self.handle, nsteps)

    def set_variant(self, v):
        lbm_batch_set_variant(self.handle, v)

    def variant(self):
        return lbm_batch_variant(self.handle)

    def autotune(self, steps_per_variant=10):
        return lbm_batch_autotune(self.handle, steps_per_variant)

    def residuals(self):
        return lbm_batch_residuals(self.handle, self.capacity)

    def close(self):
        if self.handle:
            lbm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Domain:
    """One LBMTau1 domain on a GPU: a torch-allocated workspace, a stream and
    a context.  Methods map one-to-one to the C calls."""

    def __init__(self, nx, ny, periodic=(False, False), force=(0.0, 0.0),
                 device="cuda", stream=None, storage=LBM_STORAGE_F32,
                 rounding=LBM_ROUND_DEFAULT, sc_g=0.0):
        import torch
        self.nx, self.ny = int(nx), int(ny)
        if isinstance(storage, str):
            storage = STORAGE_NAMES[storage]
        self.storage = int(storage)
        self.params = make_params(nx, ny, periodic, force, self.storage,
                                  rounding, sc_g)
        nbytes = lbm_workspace_bytes(self.params)
        if nbytes == 0:
            raise LbmError(LBM_E_INVAL, "invalid domain parameters")
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = lbm_create(self.params, self.workspace.data_ptr(), nbytes,
                              self.stream.cuda_stream)

    @classmethod
    def from_problem(cls, prob, **kw):
        ny, nx = prob.mask.shape
        if "sc_g" in prob.meta and "sc_g" not in kw:
            kw["sc_g"] = prob.meta["sc_g"]
        d = cls(nx, ny, prob.periodic, prob.force, **kw)
        d.set_geometry(prob.mask)
        d.set_moments(prob.rho, prob.jx, prob.jy)
        return d

    def set_geometry(self, mask):
        lbm_set_geometry(self.ctx, mask)

    def set_moments(self, rho, jx, jy):
        lbm_set_moments(self.ctx, rho, jx, jy)

    def step(self, nsteps=1):
        lbm_step(self.ctx, nsteps)

    def set_variant(self, v):
        lbm_set_variant(self.ctx, v)

    def set_copy_wait_ns(self, ns):
        lbm_set_copy_wait_ns(self.ctx, ns)

    def snapshot(self):
        """A device copy of the current state (a torch buffer) to measure
        the change over a span of steps against (change_since)."""
        import torch
        n = _lib.lbm_snapshot_bytes(ctypes.byref(self.params))
        buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        _check(_lib.lbm_snapshot(self.ctx, _vp(buf.data_ptr()), n), self.ctx)
        return buf

    def change_since(self, snap, steps):
        """Mean relative velocity change per step since `snap` was taken,
        `steps` steps ago."""
        out = ctypes.c_double()
        _check(_lib.lbm_change_since(self.ctx, _vp(snap.data_ptr()),
                                     int(steps), ctypes.byref(out)), self.ctx)
        return out.value

    def step_count(self):
        return lbm_step_count(self.ctx)

    def set_step_count(self, steps):
        lbm_set_step_count(self.ctx, steps)

    def variant(self):
        return lbm_variant(self.ctx)

    def moments(self, out=None):
        if out is None:
            out = tuple(np.empty((self.ny, self.nx), np.float64) for _ in range(3))
        lbm_moments(self.ctx, *out)
        return out

    def get_state(self, out=None):
        if out is None:
            dt = STATE_DTYPE[self.storage]
            out = tuple(np.empty((self.ny, self.nx), dt) for _ in range(3))
        lbm_get_state(self.ctx, *out)
        return out

    def set_state(self, drho, jx, jy):
        lbm_set_state(self.ctx, drho, jx, jy)

    def residual(self):
        return lbm_residual(self.ctx)

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
