"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not against itself (CPU only).

- the lattice tables against the values printed in the paper (golden file);
- brute-force agreement with a full-population BGK code at tau = 1 that uses
  the wall rule of Eq. (feqnoslip), on tiny grids with obstacles, fixed nodes,
  forcing and every periodicity combination (Eq. LBMTau1 is exact, so the two
  must agree to roundoff);
- the closed-form discrete Poiseuille steady state, and the L^-2 scaling of the
  centre-line error claimed in Section 3;
- exact conservation of mass and the exact momentum gain N*f per step on a
  fully periodic domain;
- the mass-exchange identity at walls implied by Eq. (feqnoslip);
- the quiescent fixed point for any geometry;
- mirror and transpose symmetry of the D2Q9 update.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1912_09327_gb300 import workloads as wl
from tests import fullpop_bgk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_lattice_matches_paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "d2q9_lattice.txt"), dtype=np.int64)
    ex, ey, inv, w = oracle.lattice()
    assert (rows[:, 1] == ex).all() and (rows[:, 2] == ey).all()
    assert (rows[:, 3] == inv).all()
    assert np.allclose(w, rows[:, 4] / rows[:, 5], rtol=0, atol=1e-16)
    # lattice isotropy: moments of the weights up to second order
    assert abs(w.sum() - 1) < 1e-15
    assert abs((w * ex).sum()) < 1e-16 and abs((w * ey).sum()) < 1e-16
    assert abs((w * ex * ex).sum() - 1 / 3) < 1e-15
    assert abs((w * ex * ey).sum()) < 1e-16
    assert (ex[inv] == -ex).all() and (ey[inv] == -ey).all()


CASES = [
    # (nx, ny, periodic, force, p_solid, p_fixed, seed)
    (8, 8, (True, True), (2e-3, -1e-3), 0.2, 0.0, 1),
    (7, 5, (False, False), (1e-3, 3e-3), 0.15, 0.1, 2),
    (6, 9, (True, False), (0.0, 0.0), 0.25, 0.1, 3),
    (5, 7, (False, True), (-2e-3, 1e-3), 0.1, 0.05, 4),
]


@pytest.mark.parametrize("nx,ny,per,force,ps,pf,seed", CASES)
def test_matches_full_population_bgk(nx, ny, per, force, ps, pf, seed):
    p = wl.random_problem(nx, ny, seed, ps, pf, amp=0.05, periodic=per,
                          force=force)
    steps = 25
    a = oracle.run(p.mask, *p.state(), steps, p.periodic, p.force)
    b = fullpop_bgk.run(p.mask, *p.state(), steps, p.periodic, p.force)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-13


def test_standard_bounce_back_differs():
    """Negative control: half-way bounce-back is a different boundary rule, so
    the brute-force comparison above is sensitive to the wall rule."""
    p = wl.random_problem(8, 8, 5, 0.2, 0.0, amp=0.05)
    a = oracle.run(p.mask, *p.state(), 5, p.periodic, p.force)
    b = fullpop_bgk.run(p.mask, *p.state(), 5, p.periodic, p.force,
                        wall="bounce")
    assert np.abs(a[1] - b[1]).max() > 1e-4


def poiseuille_steady(ny, fx, nx=4, tol=1e-13, chunk=4000, max_steps=400000):
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = mask[-1] = 1
    R, U, V = np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    done = 0
    while done < max_steps:
        R2, U2, V2 = oracle.run(mask, R, U, V, chunk, (True, False), (fx, 0))
        done += chunk
        change = np.abs(U2 - U).max()
        R, U, V = R2, U2, V2
        if change < tol * np.abs(U).max():
            break
    return R, U, V


def test_closed_form_poiseuille():
    """Exact discrete steady state with walls on the solid node centres:
    rho = 1, V = 0, U(y) = 3 f y (H - y) - f for the fluid rows (H = ny - 1).
    The interior update reduces to U = 2/3 (U + f) + 1/6 (U_{y-1} + f) +
    1/6 (U_{y+1} + f), which this profile satisfies, with the wall rows
    receiving zero x momentum from the wall."""
    ny, fx = 32, 1e-5
    R, U, V = poiseuille_steady(ny, fx)
    H = ny - 1
    y = np.arange(1, ny - 1)
    exact = 3 * fx * y * (H - y) - fx
    assert np.abs(U[1:-1, :] - exact[:, None]).max() < 1e-11 * exact.max()
    # rho = 1 up to FP64 roundoff accumulated over ~10^4 steps of O(1) sums
    assert np.abs(R - 1).max() < 1e-10
    assert np.abs(V).max() < 1e-14


def test_error_scales_as_inverse_square_of_width():
    """Section 3: the relative centre-line error against the analytic
    parabola u = 3 f y (H - y) (nu = 1/6) scales as L^-2; with the closed form
    above it is exactly 4 / (3 H^2)."""
    fx = 1e-6
    Hs, errs = [], []
    for ny in (17, 33, 65):
        R, U, V = poiseuille_steady(ny, fx)
        H = ny - 1
        u_c = U[H // 2, 0] / R[H // 2, 0]
        u_analytic = 3 * fx * (H / 2) * (H / 2)
        errs.append(abs(u_c - u_analytic) / u_analytic)
        Hs.append(H)
        assert errs[-1] == pytest.approx(4 / (3 * H * H), rel=1e-8)
    slope = np.polyfit(np.log(Hs), np.log(errs), 1)[0]
    assert slope == pytest.approx(-2.0, abs=1e-6)


def test_periodic_conservation():
    """All-fluid periodic box: sum rho is conserved (sum_k f^eq_k = rho) and the
    total momentum grows by exactly N * f per step (sum_k e_k f^eq_k = rho u')."""
    p = wl.periodic_box(9, 7, seed=3, amp=0.05)
    force = (3e-4, -2e-4)
    R0, U0, V0 = p.state()
    R1, U1, V1 = oracle.run(p.mask, R0, U0, V0, 10, (True, True), force)
    N = p.mask.size
    assert abs(R1.sum() - R0.sum()) < 1e-12
    assert abs(U1.sum() - U0.sum() - 10 * N * force[0]) < 1e-12
    assert abs(V1.sum() - V0.sum() - 10 * N * force[1]) < 1e-12


def test_wall_mass_exchange_identity():
    """Eq. (feqnoslip) is not mass conserving: across every fluid-to-solid
    link (fluid x, direction k toward a solid node) the node sends f^eq_k of
    its own state into the wall and receives w_k rho(x) back.  So the change
    of total fluid mass in one step is the sum over links of
    w_k rho(x) - f^eq_k(rho(x), (j(x) + F) / rho(x))."""
    p = wl.random_problem(11, 9, 7, p_solid=0.25, p_fixed=0.0, amp=0.05,
                          periodic=(True, False), force=(1e-3, 2e-3))
    ex, ey, inv, w = oracle.lattice()
    R0, U0, V0 = p.state()
    R1, _, _ = oracle.step(p.mask, R0, U0, V0, p.periodic, p.force)
    fluid = p.mask == 0
    ny, nx = p.mask.shape
    expected = 0.0
    for y in range(ny):
        for x in range(nx):
            if not fluid[y, x]:
                continue
            ux = (U0[y, x] + p.force[0]) / R0[y, x]
            uy = (V0[y, x] + p.force[1]) / R0[y, x]
            for k in range(1, 9):
                xs, ys = (x + ex[k]) % nx, y + ey[k]
                if 0 <= ys < ny and p.mask[ys, xs] != 1:
                    continue
                eu = ex[k] * ux + ey[k] * uy
                feq = w[k] * R0[y, x] * (1 + 3 * eu + 4.5 * eu * eu
                                         - 1.5 * (ux * ux + uy * uy))
                expected += w[k] * R0[y, x] - feq
    got = R1[fluid].sum() - R0[fluid].sum()
    assert abs(expected) > 1e-4
    assert got == pytest.approx(expected, rel=1e-10, abs=1e-15)


def test_quiescent_fixed_point():
    """Uniform density at rest, no force: every pulled equilibrium is
    w_k rho, so nothing changes, whatever the geometry."""
    mask = wl.random_mask((10, 12), 9, 0.3, 0.1)
    R = np.full(mask.shape, 1.3)
    Z = np.zeros(mask.shape)
    for per in [(True, True), (False, False), (True, False)]:
        R1, U1, V1 = oracle.run(mask, R, Z, Z, 7, per, (0.0, 0.0))
        assert np.abs(R1 - 1.3).max() < 1e-15
        assert np.abs(U1).max() < 1e-16 and np.abs(V1).max() < 1e-16


def test_mirror_and_transpose_symmetry():
    p = wl.random_problem(9, 7, 11, 0.2, 0.05, amp=0.05, periodic=(True, False),
                          force=(1e-3, 5e-4))
    R0, U0, V0 = p.state()
    base = oracle.run(p.mask, R0, U0, V0, 6, p.periodic, p.force)
    # x mirror: x -> nx-1-x, U -> -U, fx -> -fx
    m = oracle.run(p.mask[:, ::-1], R0[:, ::-1], -U0[:, ::-1], V0[:, ::-1], 6,
                   p.periodic, (-p.force[0], p.force[1]))
    assert np.abs(m[0][:, ::-1] - base[0]).max() < 1e-14
    assert np.abs(-m[1][:, ::-1] - base[1]).max() < 1e-14
    assert np.abs(m[2][:, ::-1] - base[2]).max() < 1e-14
    # transpose: swap x and y, U and V, periodicity and force components
    t = oracle.run(p.mask.T, R0.T, V0.T, U0.T, 6, p.periodic[::-1],
                   p.force[::-1])
    assert np.abs(t[0].T - base[0]).max() < 1e-14
    assert np.abs(t[2].T - base[1]).max() < 1e-14
    assert np.abs(t[1].T - base[2]).max() < 1e-14


def test_step_nodes_matches_step():
    p = wl.random_problem(13, 6, 4, 0.2, 0.1, amp=0.05)
    R0, U0, V0 = p.state()
    full = oracle.step(p.mask, R0, U0, V0, p.periodic, p.force)
    nodes = np.array([0, 5, 12, 13, 40, 77])
    part = oracle.step_nodes(p.mask, R0, U0, V0, nodes, p.periodic, p.force)
    for j, i in enumerate(nodes):
        for f in range(3):
            assert part[j, f] == full[f].ravel()[i]


def test_residual_definition():
    """Residual is zero between equal states and equals the relative L2
    velocity change otherwise; mass sums fluid densities only."""
    mask = np.array([[0, 1], [0, 2]], np.uint8)
    R = np.array([[1.0, 5.0], [2.0, 7.0]])
    U = np.array([[0.1, 9.0], [0.4, 9.0]])
    V = np.zeros((2, 2))
    assert oracle.residual(mask, (R, U, V), (R, U, V)) == (0.0, 3.0)
    U2 = U.copy(); U2[0, 0] = 0.2
    res, mass = oracle.residual(mask, (R, U, V), (R, U2, V))
    # u_old = (0.1, 0.2), u_new = (0.2, 0.2) on the two fluid nodes
    assert res == pytest.approx(0.1 / np.sqrt(0.08), rel=1e-15)
    assert mass == 3.0
