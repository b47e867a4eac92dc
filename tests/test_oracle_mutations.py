"""The pins are strong enough: each plausible mistake planted in a copy of the
oracle's C source (compiled to a temporary library, on the CPU) makes at least
one independent check fail.  The checks are the brute-force full-population
BGK code, the closed-form Poiseuille profile, periodic conservation and the
quiescent fixed point, as in test_oracle_pins.py."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1912_09327_gb300 import workloads as wl
from tests import fullpop_bgk

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "oracle", "lbm_oracle.c")

MUTATIONS = {
    "wall uses the neighbour's density":
        ("feq = omega[k] * R[i];", "feq = omega[k] * R[p >= 0 ? p : i];"),
    "force dropped from v": ("(V[p] + d->fy) / r", "V[p] / r"),
    "sign of the linear term": ("+ 3.0 * eu +", "- 3.0 * eu +"),
    "quadratic term dropped": ("+ 4.5 * eu * eu", ""),
    "momentum accumulated along k, not its inverse":
        ("u_new += ex[ik] * feq;", "u_new += ex[k] * feq;"),
    "fixed nodes updated": ("if (d->mask[i] != NODE_FLUID) {",
                            "if (d->mask[i] == NODE_SOLID) {"),
    "diagonal inverses swapped": ("{0, 3, 4, 1, 2, 7, 8, 5, 6}",
                                  "{0, 3, 4, 1, 2, 8, 7, 6, 5}"),
    "transposed neighbour offset": ("neighbour_index(d, x + ex[k], y + ey[k])",
                                    "neighbour_index(d, x + ey[k], y + ex[k])"),
}


def build_mutant(tmp_path, name, old, new):
    text = open(SRC).read()
    assert old in text, name
    path = tmp_path / "mutant.c"
    path.write_text(text.replace(old, new, 1))
    lib = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                           str(path), "-o", str(lib), "-lm"])
    so = ctypes.CDLL(str(lib))
    i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    so.oracle_run.argtypes = [i64, i64, i32, i32, f64, f64] + [vp] * 4 + [i64]
    so.oracle_run.restype = ctypes.c_int

    def run(mask, R, U, V, n, periodic, force):
        mask = np.ascontiguousarray(mask, np.uint8)
        R, U, V = (np.array(a, np.float64) for a in (R, U, V))
        ny, nx = mask.shape
        so.oracle_run(nx, ny, int(periodic[0]), int(periodic[1]), force[0],
                      force[1], mask.ctypes.data, R.ctypes.data, U.ctypes.data,
                      V.ctypes.data, n)
        return R, U, V
    return run


def checks_pass(run):
    """True when every independent check passes."""
    for nx, ny, per, seed in [(8, 7, (True, False), 1), (6, 6, (False, True), 2)]:
        p = wl.random_problem(nx, ny, seed, 0.2, 0.1, amp=0.05, periodic=per,
                              force=(2e-3, -1e-3))
        a = run(p.mask, *p.state(), 8, p.periodic, p.force)
        b = fullpop_bgk.run(p.mask, *p.state(), 8, p.periodic, p.force)
        if max(np.abs(x - y).max() for x, y in zip(a, b)) > 1e-13:
            return False
    # closed-form Poiseuille
    ny, fx = 12, 1e-5
    mask = np.zeros((ny, 3), np.uint8); mask[0] = mask[-1] = 1
    R, U, V = run(mask, np.ones((ny, 3)), np.zeros((ny, 3)), np.zeros((ny, 3)),
                  6000, (True, False), (fx, 0.0))
    y = np.arange(1, ny - 1); H = ny - 1
    if np.abs(U[1:-1, 0] - (3 * fx * y * (H - y) - fx)).max() > 1e-12:
        return False
    # periodic conservation
    p = wl.periodic_box(7, 5, seed=3, amp=0.05)
    R1, U1, V1 = run(p.mask, *p.state(), 5, (True, True), (1e-3, 0.0))
    if abs(R1.sum() - p.rho.sum()) > 1e-12 or \
            abs(U1.sum() - p.jx.sum() - 5 * 35 * 1e-3) > 1e-12:
        return False
    # quiescent fixed point
    mask = wl.random_mask((6, 7), 4, 0.3, 0.1)
    R2, U2, V2 = run(mask, np.full((6, 7), 1.2), np.zeros((6, 7)),
                     np.zeros((6, 7)), 4, (False, False), (0.0, 0.0))
    return np.abs(R2 - 1.2).max() < 1e-14 and np.abs(U2).max() < 1e-15


def test_unmutated_source_passes(tmp_path):
    run = build_mutant(tmp_path, "none", "#include <math.h>", "#include <math.h>")
    assert checks_pass(run)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    run = build_mutant(tmp_path, name, old, new)
    assert not checks_pass(run), name


# Mistakes planted in the multiphase (Shan-Chen) step; the check is the
# independent full-population code with the force from array shifts.
SC_MUTATIONS = {
    "coupling sign flipped": ("*fsx = -g * own * sx;", "*fsx = g * own * sx;"),
    "own potential dropped": ("*fsy = -g * own * sy;", "*fsy = -g * sy;"),
    "potential of a wall not zero":
        ("if (p < 0 || d->mask[p] == NODE_SOLID) return 0.0;",
         "if (p < 0) return 0.0;"),
    "force taken at the receiving node":
        ("sc_force(d, g, R, p % d->nx, p / d->nx, &fsx, &fsy);",
         "sc_force(d, g, R, x, y, &fsx, &fsy);"),
    "axis weights on the diagonals":
        ("sx += omega[i] * ps * ex[i];", "sx += omega[1] * ps * ex[i];"),
    "force dropped from the density division":
        ("(U[p] + d->fx + fsx) / r", "(U[p] + d->fx) / r + fsx"),
}


def build_sc_mutant(tmp_path, old, new):
    text = open(SRC).read()
    assert old in text, old
    path = tmp_path / "mutant_sc.c"
    path.write_text(text.replace(old, new, 1))
    lib = tmp_path / "mutant_sc.so"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                           str(path), "-o", str(lib), "-lm"])
    so = ctypes.CDLL(str(lib))
    i64, i32, f64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
    so.oracle_run_sc.argtypes = [i64, i64, i32, i32, f64, f64, f64] + [vp] * 4 + [i64]
    so.oracle_run_sc.restype = ctypes.c_int

    def run(mask, R, U, V, n, g, periodic, force):
        mask = np.ascontiguousarray(mask, np.uint8)
        R, U, V = (np.array(a, np.float64) for a in (R, U, V))
        ny, nx = mask.shape
        so.oracle_run_sc(nx, ny, int(periodic[0]), int(periodic[1]), force[0],
                         force[1], g, mask.ctypes.data, R.ctypes.data,
                         U.ctypes.data, V.ctypes.data, n)
        return R, U, V
    return run


def sc_checks_pass(run):
    rng = np.random.default_rng(11)
    for nx, ny, per, ps in [(7, 6, (True, True), 0.15), (6, 7, (False, True), 0.1)]:
        mask = (rng.random((ny, nx)) < ps).astype(np.uint8)
        R = rng.uniform(0.3, 2.0, (ny, nx))
        U = 0.02 * rng.standard_normal((ny, nx))
        V = 0.02 * rng.standard_normal((ny, nx))
        R[mask == 1], U[mask == 1], V[mask == 1] = 1.0, 0.0, 0.0
        a = run(mask, R, U, V, 6, -5.0, per, (1e-3, -1e-3))
        b = fullpop_bgk.run_sc(mask, R, U, V, 6, -5.0, per, (1e-3, -1e-3))
        if max(np.abs(x - y).max() for x, y in zip(a, b)) > 1e-13:
            return False
    return True


def test_unmutated_sc_source_passes(tmp_path):
    run = build_sc_mutant(tmp_path, "#include <math.h>", "#include <math.h>")
    assert sc_checks_pass(run)


@pytest.mark.parametrize("name", sorted(SC_MUTATIONS))
def test_sc_mutation_is_caught(tmp_path, name):
    old, new = SC_MUTATIONS[name]
    run = build_sc_mutant(tmp_path, old, new)
    assert not sc_checks_pass(run), name
