"""Pins of the oracle's Shan-Chen multiphase step (Section 4, Eq. f_sc) against
facts fixed by the mathematics and by the model, not against itself (CPU
only).

- with g = 0, or a uniform density on a periodic domain, the force vanishes
  and the step is the single-phase step bit for bit;
- agreement to roundoff with an independent full-population tau = 1 BGK code
  whose force comes from array shifts of the potential (tests/fullpop_bgk.py),
  with walls, body force and every periodicity;
- on a periodic domain the force sums to zero (pairs of opposite directions
  cancel for a symmetric G), so mass and total momentum are conserved;
- x-mirror symmetry;
- a flat liquid slab in its vapour settles at the coexistence densities that
  the mechanical-stability condition of the model's equation of state
  p = rho / 3 + g psi^2 / 6 predicts (Shan-Chen, psi = 1 - exp(-rho)):
  p(rho_g) = p(rho_l) = p0 and the integral of (p0 - p) psi' / psi^2 over
  [rho_g, rho_l] vanishes.
"""
import numpy as np
import pytest

import oracle
from tests import fullpop_bgk


def random_state(shape, seed, p_solid=0.0, lo=0.3, hi=2.0, amp=0.02):
    rng = np.random.default_rng(seed)
    mask = (rng.random(shape) < p_solid).astype(np.uint8)
    R = rng.uniform(lo, hi, shape)
    U = amp * rng.standard_normal(shape)
    V = amp * rng.standard_normal(shape)
    R[mask == 1], U[mask == 1], V[mask == 1] = 1.0, 0.0, 0.0
    return mask, R, U, V


def test_zero_coupling_and_uniform_density_reduce_to_single_phase():
    mask, R, U, V = random_state((9, 11), 1, p_solid=0.15)
    for per in [(True, True), (False, True), (False, False)]:
        a = oracle.step(mask, R, U, V, per, (1e-3, 2e-3))
        b = oracle.step_sc(mask, R, U, V, 0.0, per, (1e-3, 2e-3))
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    free = np.zeros((9, 11), np.uint8)
    Ru = np.full((9, 11), 1.3)
    a = oracle.step(free, Ru, U, V, (True, True))
    b = oracle.step_sc(free, Ru, U, V, -5.0, (True, True))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


CASES = [
    # (nx, ny, periodic, p_solid, force, seed)
    (8, 7, (True, True), 0.0, (0.0, 0.0), 3),
    (7, 6, (True, True), 0.15, (1e-3, -2e-3), 4),
    (6, 8, (False, True), 0.1, (2e-3, 0.0), 5),
    (7, 7, (False, False), 0.1, (0.0, 1e-3), 6),
]


@pytest.mark.parametrize("nx,ny,per,ps,force,seed", CASES)
def test_matches_full_population_sc(nx, ny, per, ps, force, seed):
    mask, R, U, V = random_state((ny, nx), seed, p_solid=ps)
    a = oracle.run_sc(mask, R, U, V, 15, -5.0, per, force)
    b = fullpop_bgk.run_sc(mask, R, U, V, 15, -5.0, per, force)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-13


def test_force_sums_to_zero_and_moments_are_conserved():
    mask, R, U, V = random_state((24, 32), 7, lo=0.2, hi=2.2)
    FX, FY = oracle.sc_force(mask, R, -5.5)
    scale = np.abs(FX).sum() + np.abs(FY).sum()
    assert abs(FX.sum()) < 1e-14 * scale and abs(FY.sum()) < 1e-14 * scale
    R1, U1, V1 = oracle.run_sc(mask, R, U, V, 50, -5.5)
    assert abs(R1.sum() - R.sum()) < 1e-12 * R.sum()
    assert abs(U1.sum() - U.sum()) < 1e-12 * R.sum()
    assert abs(V1.sum() - V.sum()) < 1e-12 * R.sum()


def test_mirror_symmetry():
    mask, R, U, V = random_state((10, 12), 8, p_solid=0.1)
    per = (False, True)
    a = oracle.run_sc(mask, R, U, V, 10, -5.0, per)
    b = oracle.run_sc(mask[:, ::-1], R[:, ::-1], -U[:, ::-1], V[:, ::-1], 10,
                      -5.0, per)
    assert np.abs(a[0] - b[0][:, ::-1]).max() < 1e-13
    assert np.abs(a[1] + b[1][:, ::-1]).max() < 1e-13
    assert np.abs(a[2] - b[2][:, ::-1]).max() < 1e-13


def coexistence(g):
    from scipy.integrate import quad
    from scipy.optimize import fsolve

    def psi(r):
        return 1.0 - np.exp(-r)

    def pressure(r):
        return r / 3.0 + g / 6.0 * psi(r) ** 2

    def eqs(v):
        rg, rl = v
        p0 = pressure(rg)
        area = quad(lambda r: (p0 - pressure(r)) * np.exp(-r) / psi(r) ** 2,
                    rg, rl)[0]
        return [pressure(rl) - p0, area]

    return fsolve(eqs, [0.1, 2.0])


@pytest.mark.parametrize("g", [-5.0, -6.0])
def test_flat_interface_coexistence(g):
    pytest.importorskip("scipy")
    rho_g, rho_l = coexistence(g)
    ny, nx = 128, 4
    y = np.arange(ny)
    R0 = np.where(np.abs(y - ny / 2) < ny / 4, rho_l, rho_g)[:, None] * np.ones((1, nx))
    mask = np.zeros((ny, nx), np.uint8)
    Z = np.zeros_like(R0)
    oracle.set_threads(oracle.max_threads())
    R, _, _ = oracle.run_sc(mask, R0, Z, Z, 20000, g)
    assert R[0, 0] == pytest.approx(rho_g, rel=0.02)
    assert R[ny // 2, 0] == pytest.approx(rho_l, rel=0.002)
