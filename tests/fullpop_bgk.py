"""Brute-force full-population D2Q9 BGK code, used only to pin the oracle.

It keeps all nine populations per node and runs the textbook two-step form of
Eq. (lbm): BGK collision with a general relaxation time (called here with
tau = 1), then pull streaming.  The wall rule of Eq. (feqnoslip) replaces a
population arriving from a solid node by the zero-velocity equilibrium of the
receiving node; ``wall="bounce"`` gives the standard half-way bounce-back
(the reflected post-collision population of the receiving node) instead, as a
negative control.  Body force: velocity shift of the equilibrium (Section 2).
Pure-Python loops: tiny grids only.
"""
import numpy as np

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
WEIGHT = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4


def opposite(k):
    ex, ey = E[k]
    return E.index((-ex, -ey))


def equilibrium(rho, ux, uy):
    feq = np.empty(9)
    usq = ux * ux + uy * uy
    for k, (ex, ey) in enumerate(E):
        eu = ex * ux + ey * uy
        feq[k] = WEIGHT[k] * rho * (1 + 3 * eu + 4.5 * eu * eu - 1.5 * usq)
    return feq


def run(mask, R, U, V, nsteps, periodic=(False, False), force=(0.0, 0.0),
        tau=1.0, wall="paper"):
    ny, nx = mask.shape
    R = np.array(R, float); U = np.array(U, float); V = np.array(V, float)
    # populations consistent with the stored moments
    f = np.zeros((ny, nx, 9))
    for y in range(ny):
        for x in range(nx):
            f[y, x] = equilibrium(R[y, x], U[y, x] / R[y, x], V[y, x] / R[y, x])

    def source(x, y):
        if not 0 <= x < nx:
            if not periodic[0]:
                return None
            x %= nx
        if not 0 <= y < ny:
            if not periodic[1]:
                return None
            y %= ny
        return x, y

    for _ in range(nsteps):
        post = np.zeros_like(f)
        for y in range(ny):
            for x in range(nx):
                if mask[y, x] == 1:
                    continue
                rho = R[y, x]
                ux = (U[y, x] + force[0]) / rho
                uy = (V[y, x] + force[1]) / rho
                post[y, x] = f[y, x] - (f[y, x] - equilibrium(rho, ux, uy)) / tau
        newf = f.copy()
        for y in range(ny):
            for x in range(nx):
                if mask[y, x] != 0:
                    continue
                for k, (ex, ey) in enumerate(E):
                    s = source(x - ex, y - ey)
                    if s is not None and mask[s[1], s[0]] != 1:
                        newf[y, x, k] = post[s[1], s[0], k]
                    elif wall == "paper":
                        newf[y, x, k] = WEIGHT[k] * R[y, x]
                    else:
                        newf[y, x, k] = post[y, x, opposite(k)]
        f = newf
        for y in range(ny):
            for x in range(nx):
                if mask[y, x] != 0:
                    continue
                R[y, x] = f[y, x].sum()
                U[y, x] = sum(E[k][0] * f[y, x, k] for k in range(9))
                V[y, x] = sum(E[k][1] * f[y, x, k] for k in range(9))
    return R, U, V


def run_sc(mask, R, U, V, nsteps, g, periodic=(True, True), force=(0.0, 0.0)):
    """Full-population tau = 1 BGK with the Shan-Chen force of Section 4
    (Eq. f_sc with psi = 1 - exp(-rho), alpha_i = w_i, G(e_i) = -g e_i;
    psi = 0 at solid nodes and outside non-periodic edges), applied as a
    velocity shift of the equilibrium.  Densities come from the populations;
    the force of a node is computed from its neighbours' potentials with
    array shifts, not with the oracle's two-fold loop."""
    ny, nx = mask.shape
    R = np.array(R, float); U = np.array(U, float); V = np.array(V, float)
    f = np.zeros((ny, nx, 9))
    for y in range(ny):
        for x in range(nx):
            f[y, x] = equilibrium(R[y, x], U[y, x] / R[y, x], V[y, x] / R[y, x])
    solid = mask == 1

    def shifted(a, dx, dy):
        """a at (x + dx, y + dy), 0 where that point is outside a
        non-periodic edge."""
        out = np.roll(a, (-dy, -dx), axis=(0, 1))
        if not periodic[0]:
            if dx > 0:
                out[:, nx - dx:] = 0.0
            elif dx < 0:
                out[:, :-dx] = 0.0
        if not periodic[1]:
            if dy > 0:
                out[ny - dy:, :] = 0.0
            elif dy < 0:
                out[:-dy, :] = 0.0
        return out

    def source(x, y):
        if not 0 <= x < nx:
            if not periodic[0]:
                return None
            x %= nx
        if not 0 <= y < ny:
            if not periodic[1]:
                return None
            y %= ny
        return x, y

    for _ in range(nsteps):
        psi = np.where(solid, 0.0, 1.0 - np.exp(-R))
        sx = np.zeros_like(R); sy = np.zeros_like(R)
        for k, (ex, ey) in enumerate(E):
            nb = shifted(psi, ex, ey)
            sx += WEIGHT[k] * ex * nb
            sy += WEIGHT[k] * ey * nb
        FX = -g * psi * sx
        FY = -g * psi * sy
        post = np.zeros_like(f)
        for y in range(ny):
            for x in range(nx):
                if solid[y, x]:
                    continue
                rho = R[y, x]
                ux = (U[y, x] + force[0] + FX[y, x]) / rho
                uy = (V[y, x] + force[1] + FY[y, x]) / rho
                post[y, x] = equilibrium(rho, ux, uy)
        newf = f.copy()
        for y in range(ny):
            for x in range(nx):
                if mask[y, x] != 0:
                    continue
                for k, (ex, ey) in enumerate(E):
                    s = source(x - ex, y - ey)
                    if s is not None and mask[s[1], s[0]] != 1:
                        newf[y, x, k] = post[s[1], s[0], k]
                    else:
                        newf[y, x, k] = WEIGHT[k] * R[y, x]
        f = newf
        for y in range(ny):
            for x in range(nx):
                if mask[y, x] != 0:
                    continue
                R[y, x] = f[y, x].sum()
                U[y, x] = sum(E[k][0] * f[y, x, k] for k in range(9))
                V[y, x] = sum(E[k][1] * f[y, x, k] for k in range(9))
    return R, U, V
