"""FP64 CPU oracle of the LBMTau1 D2Q9 step (arXiv:1912.09327).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The oracle is written from the paper alone (Section 2 equations,
Algorithm 1, the Appendix A listing for the cavity conventions) and shares no
code with the CUDA path; see ``lbm_oracle.c`` for the readings it takes.

State convention: ``R`` is the density, ``U``/``V`` the x/y momentum
(Eq. utau1 sums e_k f_k, so the stored "velocity" fields carry rho*u).
Node types in ``mask``: 0 fluid, 1 solid (no-slip, Eq. feqnoslip), 2 fixed
equilibrium (the moving lid of Section 3).  Arrays are ``[ny, nx]`` row-major.

Pinned by ``tests/test_oracle_pins.py`` (brute-force full-population BGK at
tau = 1, the closed-form discrete Poiseuille profile and its L^-2 error,
periodic conservation laws, the wall mass-exchange identity, the quiescent
fixed point, lattice symmetries).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over rows) into an in-tree .so."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                           "-std=c11", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    vp = ctypes.c_void_p
    lib.oracle_lattice.argtypes = [vp, vp, vp, vp]
    lib.oracle_step.argtypes = [i64, i64, i32, i32, f64, f64] + [vp] * 7
    lib.oracle_run.argtypes = [i64, i64, i32, i32, f64, f64] + [vp] * 4 + [i64]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_step_nodes.argtypes = ([i64, i64, i32, i32, f64, f64]
                                      + [vp] * 5 + [i64, vp])
    lib.oracle_residual.argtypes = [i64] + [vp] * 9
    lib.oracle_step_sc.argtypes = [i64, i64, i32, i32, f64, f64, f64] + [vp] * 7
    lib.oracle_run_sc.argtypes = ([i64, i64, i32, i32, f64, f64, f64]
                                  + [vp] * 4 + [i64])
    lib.oracle_run_sc.restype = ctypes.c_int
    lib.oracle_sc_force.argtypes = [i64, i64, i32, i32, f64] + [vp] * 4
    lib.oracle_set_threads.argtypes = [i32]
    lib.oracle_max_threads.restype = i32
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def lattice():
    """(ex, ey, inv, w) as the oracle holds them."""
    lib = _load()
    ex = np.zeros(9, np.int32); ey = np.zeros(9, np.int32)
    inv = np.zeros(9, np.int32); w = np.zeros(9, np.float64)
    lib.oracle_lattice(_p(ex), _p(ey), _p(inv), _p(w))
    return ex, ey, inv, w


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def run(mask, R, U, V, nsteps, periodic=(False, False), force=(0.0, 0.0)):
    """``nsteps`` LBMTau1 steps from (R, U, V); returns new (R, U, V)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    R, U, V = _f64(R).copy(), _f64(U).copy(), _f64(V).copy()
    rc = lib.oracle_run(nx, ny, int(periodic[0]), int(periodic[1]),
                        float(force[0]), float(force[1]), _p(mask),
                        _p(R), _p(U), _p(V), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle_run could not allocate its scratch grid")
    return R, U, V


def step(mask, R, U, V, periodic=(False, False), force=(0.0, 0.0)):
    """One step; returns new (R, U, V)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    R, U, V = _f64(R), _f64(U), _f64(V)
    out = [np.empty_like(R) for _ in range(3)]
    lib.oracle_step(nx, ny, int(periodic[0]), int(periodic[1]),
                    float(force[0]), float(force[1]), _p(mask), _p(R), _p(U),
                    _p(V), _p(out[0]), _p(out[1]), _p(out[2]))
    return tuple(out)


def step_nodes(mask, R, U, V, nodes, periodic=(False, False),
               force=(0.0, 0.0)):
    """New (R, U, V) of the flat node indices ``nodes`` after one step;
    returns an array of shape [len(nodes), 3]."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    nodes = np.ascontiguousarray(nodes, dtype=np.int64)
    R, U, V = _f64(R), _f64(U), _f64(V)
    out = np.empty((nodes.size, 3), np.float64)
    lib.oracle_step_nodes(nx, ny, int(periodic[0]), int(periodic[1]),
                          float(force[0]), float(force[1]), _p(mask), _p(R),
                          _p(U), _p(V), _p(nodes), nodes.size, _p(out))
    return out


def residual(mask, old, new):
    """(residual, mass) between two states ``old``/``new`` = (R, U, V)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    a = [_f64(x) for x in old]
    b = [_f64(x) for x in new]
    res = ctypes.c_double(); mass = ctypes.c_double()
    lib.oracle_residual(mask.size, _p(mask), *[_p(x) for x in a],
                        *[_p(x) for x in b], ctypes.byref(res),
                        ctypes.byref(mass))
    return res.value, mass.value


def step_sc(mask, R, U, V, g, periodic=(True, True), force=(0.0, 0.0)):
    """One Shan-Chen multiphase step with coupling ``g`` (Section 4,
    Eq. f_sc; see lbm_oracle.c for the readings); returns new (R, U, V)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    R, U, V = _f64(R), _f64(U), _f64(V)
    out = [np.empty_like(R) for _ in range(3)]
    lib.oracle_step_sc(nx, ny, int(periodic[0]), int(periodic[1]),
                       float(force[0]), float(force[1]), float(g), _p(mask),
                       _p(R), _p(U), _p(V), _p(out[0]), _p(out[1]),
                       _p(out[2]))
    return tuple(out)


def run_sc(mask, R, U, V, nsteps, g, periodic=(True, True),
           force=(0.0, 0.0)):
    """``nsteps`` multiphase steps from (R, U, V); returns new (R, U, V)."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    R, U, V = _f64(R).copy(), _f64(U).copy(), _f64(V).copy()
    rc = lib.oracle_run_sc(nx, ny, int(periodic[0]), int(periodic[1]),
                           float(force[0]), float(force[1]), float(g),
                           _p(mask), _p(R), _p(U), _p(V), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle_run_sc could not allocate its scratch grid")
    return R, U, V


def sc_force(mask, R, g, periodic=(True, True)):
    """The Shan-Chen force (FX, FY) of every non-solid node."""
    lib = _load()
    mask = np.ascontiguousarray(mask, dtype=np.uint8)
    ny, nx = mask.shape
    R = _f64(R)
    FX, FY = np.empty_like(R), np.empty_like(R)
    lib.oracle_sc_force(nx, ny, int(periodic[0]), int(periodic[1]), float(g),
                        _p(mask), _p(R), _p(FX), _p(FY))
    return FX, FY
