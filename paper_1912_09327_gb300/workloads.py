"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds geometry and initial-state generators only: it contains none
of the LBMTau1 arithmetic, so both the CUDA path and the CPU oracle can take
their inputs from it.  Arrays are ``[ny, nx]`` row-major (``idx = y*nx + x``).

Node types (the ``F`` flag array of Section 2.1, widened to three values):
0 fluid, 1 solid no-slip wall (Eq. feqnoslip), 2 fixed-equilibrium node (the
moving lid of the cavity in Section 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, SOLID, FIXED = 0, 1, 2
NU = 1.0 / 6.0  # lattice viscosity at tau = 1, Eq. (viscosity) with c_s^2 = 1/3


@dataclass
class Problem:
    """A domain: node types, periodicity, body force and initial moments."""
    name: str
    mask: np.ndarray                     # uint8 [ny, nx]
    periodic: tuple = (False, False)
    force: tuple = (0.0, 0.0)
    rho: np.ndarray = None               # float64 [ny, nx] density
    jx: np.ndarray = None                # float64 [ny, nx] x momentum rho*u_x
    jy: np.ndarray = None                # float64 [ny, nx] y momentum rho*u_y
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.mask.shape

    def state(self):
        return self.rho.copy(), self.jx.copy(), self.jy.copy()


def _rest_state(shape):
    return np.ones(shape), np.zeros(shape), np.zeros(shape)


def channel(nx: int = 64, ny: int = 32, u_max: float = 0.01) -> Problem:
    """Poiseuille channel of Section 3: periodic in x, no-slip rows y = 0 and
    y = ny - 1, driven by a body force chosen so that the plane-Poiseuille
    centre-line speed is ``u_max``: f = 8 nu u_max / H^2, H = ny - 1 (walls on
    the solid node centres)."""
    mask = np.zeros((ny, nx), np.uint8)
    mask[0, :] = SOLID
    mask[-1, :] = SOLID
    H = ny - 1
    fx = 8.0 * NU * u_max / (H * H)
    r, u, v = _rest_state(mask.shape)
    return Problem("channel", mask, (True, False), (fx, 0.0), r, u, v,
                   {"u_max": u_max, "H": H})


def cavity(n: int = 1024, u_lid: float = 0.1, ny: int | None = None) -> Problem:
    """Lid-driven cavity of Section 3 / Appendix A: walls at x = 0, x = nx-1,
    y = 0 and the two top corners; the top row y = ny-1 (x = 1..nx-2) holds
    fixed nodes with density 1 and momentum (u_lid, 0)."""
    nx = n
    ny = n if ny is None else ny
    mask = np.zeros((ny, nx), np.uint8)
    mask[:, 0] = SOLID
    mask[:, -1] = SOLID
    mask[0, :] = SOLID
    mask[-1, 1:-1] = FIXED
    r, u, v = _rest_state(mask.shape)
    u[-1, 1:-1] = u_lid
    return Problem("cavity", mask, (False, False), (0.0, 0.0), r, u, v,
                   {"u_lid": u_lid, "Re": u_lid * (nx - 2) / NU})


def porous(n: int = 4096, seed: int = 0, r_min: int = 8, r_max: int = 24,
           solid_fraction: float = 0.30, fx: float = 1e-5,
           ny: int | None = None, max_tries: int = 2_000_000) -> Problem:
    """Periodic porous sample: non-overlapping discs with integer radii drawn
    uniformly from [r_min, r_max], placed by random sequential addition with
    periodic minimum-image distances, until the solid fraction reaches
    ``solid_fraction``.  A node is solid when its centre lies within a disc."""
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    mask = np.zeros((ny, nx), np.uint8)
    cx = np.empty(0); cy = np.empty(0); cr = np.empty(0)
    tries = 0
    solid = 0                      # discs never share nodes (gap of one node)
    target = solid_fraction * nx * ny
    while solid < target and tries < max_tries:
        tries += 1
        r = int(rng.integers(r_min, r_max + 1))
        x0 = rng.uniform(0, nx); y0 = rng.uniform(0, ny)
        if cx.size:
            dx = np.abs(cx - x0); dx = np.minimum(dx, nx - dx)
            dy = np.abs(cy - y0); dy = np.minimum(dy, ny - dy)
            if np.any(dx * dx + dy * dy <= (cr + r + 1.0) ** 2):
                continue
        cx = np.append(cx, x0); cy = np.append(cy, y0); cr = np.append(cr, r)
        xs = np.arange(math.floor(x0 - r), math.ceil(x0 + r) + 1)
        ys = np.arange(math.floor(y0 - r), math.ceil(y0 + r) + 1)
        X, Y = np.meshgrid(xs, ys)
        inside = (X - x0) ** 2 + (Y - y0) ** 2 <= r * r
        mask[Y[inside] % ny, X[inside] % nx] = SOLID
        solid += int(inside.sum())
    rr, u, v = _rest_state(mask.shape)
    return Problem("porous", mask, (True, True), (fx, 0.0), rr, u, v,
                   {"discs": int(cx.size), "solid_fraction": float(mask.mean()),
                    "mean_diameter": float(2 * cr.mean()) if cr.size else 0.0})


def periodic_box(nx: int, ny: int, seed: int = 0, amp: float = 1e-3) -> Problem:
    """Fully periodic, all-fluid box with a small random perturbation:
    delta rho ~ amp N(0,1), u ~ amp N(0,1)."""
    mask = np.zeros((ny, nx), np.uint8)
    r, u, v = random_state((ny, nx), seed, amp)
    return Problem("periodic", mask, (True, True), (0.0, 0.0), r, u, v)


def periodic_box_tiled(n: int, seed: int = 0, amp: float = 1e-3,
                       tile: int = 512) -> Problem:
    """The bandwidth-sweep domain: a fully periodic, all-fluid n x n box whose
    small random perturbation (as periodic_box) is drawn on one tile x tile
    block and repeated, so that large sweep sizes are generated in seconds
    (the field stays periodic when n is a multiple of the tile)."""
    t = min(tile, n)
    r0, u0, v0 = random_state((t, t), seed, amp)
    reps = (-(-n // t), -(-n // t))
    r, u, v = (np.tile(a, reps)[:n, :n] for a in (r0, u0, v0))
    mask = np.zeros((n, n), np.uint8)
    return Problem("periodic", mask, (True, True), (0.0, 0.0), r, u, v)


def random_state(shape, seed: int = 0, amp: float = 1e-3):
    """(rho, rho*u_x, rho*u_y) with rho = 1 + amp N(0,1), u = amp N(0,1)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp * rng.standard_normal(shape)
    ux = amp * rng.standard_normal(shape)
    uy = amp * rng.standard_normal(shape)
    return rho, rho * ux, rho * uy


def random_mask(shape, seed: int = 0, p_solid: float = 0.2,
                p_fixed: float = 0.0) -> np.ndarray:
    """Independent random node types: solid with p_solid, fixed with p_fixed."""
    rng = np.random.default_rng(seed)
    u = rng.random(shape)
    mask = np.zeros(shape, np.uint8)
    mask[u < p_solid] = SOLID
    mask[(u >= p_solid) & (u < p_solid + p_fixed)] = FIXED
    return mask


def random_problem(nx: int, ny: int, seed: int = 0, p_solid: float = 0.2,
                   p_fixed: float = 0.05, amp: float = 0.02,
                   periodic=(True, True), force=(1e-4, -5e-5)) -> Problem:
    """Random node types and a random state on the non-solid nodes (solid
    nodes hold no fluid state: rest, rho = 1): the general parity case."""
    mask = random_mask((ny, nx), seed, p_solid, p_fixed)
    r, u, v = random_state((ny, nx), seed + 1, amp)
    solid = mask == SOLID
    r[solid], u[solid], v[solid] = 1.0, 0.0, 0.0
    return Problem("random", mask, tuple(periodic), tuple(force), r, u, v)


def _log_uniform_side(rng, lo, hi):
    return int(round(float(np.exp(rng.uniform(np.log(lo), np.log(hi))))))


def mixed_domain(kind: str, nx: int, ny: int, seed: int = 0) -> Problem:
    """One domain of the batch and serving mixes: a channel (u_max 0.01), a
    lid-driven cavity (lid 0.1) or a periodic porous sample with disc radii
    scaled to the domain (8..24 nodes at 512 nodes across, at least 2..3)."""
    if kind == "channel":
        return channel(nx, max(ny, 5), 0.01)
    if kind == "cavity":
        return cavity(nx, 0.1, ny=max(ny, 4))
    side = min(nx, ny)
    r_min = max(2, int(round(8 * side / 512)))
    r_max = max(r_min + 1, int(round(24 * side / 512)))
    return porous(nx, seed=seed, r_min=r_min, r_max=r_max, ny=ny, fx=1e-5)


KINDS = ("channel", "cavity", "porous")


def batch_mix(count: int = 512, seed: int = 0, lo: int = 64, hi: int = 1024):
    """The batched workload: a seeded mix of channels, cavities and porous
    samples in equal thirds, side lengths log-uniform in [lo, hi] with nx and
    ny drawn independently."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = _log_uniform_side(rng, lo, hi)
        ny = _log_uniform_side(rng, lo, hi)
        out.append(mixed_domain(KINDS[i % 3], nx, ny, seed=seed * 100003 + i))
    return out


@dataclass
class Request:
    rid: int
    arrival: float        # seconds after the start of the run
    kind: str
    nx: int
    ny: int
    seed: int

    def problem(self) -> Problem:
        return mixed_domain(self.kind, self.nx, self.ny, self.seed)


def request_stream(count: int, rate: float = 200.0, seed: int = 0,
                   lo: int = 64, hi: int = 2048):
    """Poisson arrivals at `rate` requests per second (exponential gaps),
    kinds drawn uniformly from the three mixes, sides log-uniform in
    [lo, hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        kind = KINDS[int(rng.integers(0, 3))]
        nx = _log_uniform_side(rng, lo, hi)
        ny = _log_uniform_side(rng, lo, hi)
        out.append(Request(i, t, kind, nx, ny, seed * 100003 + i))
    return out


def drop(n: int = 1024, g: float = -5.0, radius: float | None = None,
         rho_l: float = 2.0, rho_g: float = 0.15, width: float = 2.0,
         ny: int | None = None) -> Problem:
    """The multiphase test of Section 4: a drop of liquid in a periodic box
    of its vapour, at rest, for the Shan-Chen step with coupling g.  The
    density is a smoothed disc (tanh profile of the given width) of radius
    n/4 by default; rho_l and rho_g are near the coexistence densities of
    g = -5, which the flow then settles to."""
    ny = n if ny is None else ny
    r = min(n, ny) / 4.0 if radius is None else radius
    y, x = np.mgrid[0:ny, 0:n]
    dist = np.hypot(x - (n - 1) / 2.0, y - (ny - 1) / 2.0)
    rho = rho_g + 0.5 * (rho_l - rho_g) * (1.0 - np.tanh((dist - r) / width))
    mask = np.zeros((ny, n), np.uint8)
    z = np.zeros((ny, n))
    return Problem("drop", mask, (True, True), (0.0, 0.0), rho, z, z.copy(),
                   {"sc_g": g, "radius": r})


def multiphase_random(nx: int, ny: int, seed: int = 0, g: float = -5.0,
                      lo: float = 0.85, hi: float = 1.15, amp: float = 0.01,
                      p_solid: float = 0.1, p_fixed: float = 0.03,
                      periodic=(True, True), force=(1e-4, -5e-5)) -> Problem:
    """Random node types and a random density in [lo, hi] with small random
    momentum: the general parity case of the multiphase step."""
    rng = np.random.default_rng(seed)
    mask = random_mask((ny, nx), seed, p_solid, p_fixed)
    rho = rng.uniform(lo, hi, (ny, nx))
    jx = amp * rng.standard_normal((ny, nx))
    jy = amp * rng.standard_normal((ny, nx))
    solid = mask == SOLID
    rho[solid], jx[solid], jy[solid] = 1.0, 0.0, 0.0
    return Problem("multiphase_random", mask, tuple(periodic), tuple(force),
                   rho, jx, jy, {"sc_g": g})
