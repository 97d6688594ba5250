"""Standard single-relaxation-time LBM, Eq. (1), that stores the distributions f.

TEST INFRASTRUCTURE ONLY (used by ``tests/`` to pin the oracle, and as the
oracle of the GPU stream-and-collide comparator at any tau).  It is written
independently of ``maclab_oracle.c``: numpy, its own velocity tables, and the
two-step stream-and-collide form of Eq. (1) instead of the macroscopic update.

The Methods section derives MacLAB from Eq. (1) by setting tau = 1: then
f_a(x + e_a dt, t + dt) = f_a^eq(x, t) (Eq. (9)), and the moments of Eq. (13)
give Eqs. (4)-(5).  So on a periodic grid started from f = f^eq(rho0, u0), this
program at tau = 1 must produce the same (rho, u) as MacLAB at every step.
"""
from __future__ import annotations

import numpy as np

# velocity sets in the order the paper lists them (lattice units c_a = e_a / e)
C_D2Q9 = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
                   [1, 1], [-1, 1], [-1, -1], [1, -1]])
W_D2Q9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
C_D3Q19 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1],
                    [0, 0, -1], [1, 1, 0], [-1, -1, 0], [-1, 1, 0], [1, -1, 0], [0, 1, 1],
                    [0, -1, -1], [0, -1, 1], [0, 1, -1], [1, 0, 1], [-1, 0, -1], [-1, 0, 1],
                    [1, 0, -1]])
W_D3Q19 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _tables(d):
    return (C_D2Q9, W_D2Q9) if d == 2 else (C_D3Q19, W_D3Q19)


def equilibrium(rho, u):
    """Eq. (2) for all directions at once: returns f^eq with shape [Q, *grid].

    rho: [*grid]; u: [d, *grid] in lattice units (u / e).
    """
    d = u.shape[0]
    c, w = _tables(d)
    # c_a . u for every direction: array axes of u are (component, *grid)
    cu = np.tensordot(c.astype(np.float64), u, axes=([1], [0]))
    uu = np.sum(u * u, axis=0)
    return w.reshape((-1,) + (1,) * d) * rho * (1.0 + 3.0 * cu + 4.5 * cu ** 2 - 1.5 * uu)


def moments(f, d):
    """Eq. (3): rho = sum f, u = (1/rho) sum c f (lattice units)."""
    c, _ = _tables(d)
    rho = np.sum(f, axis=0)
    mom = np.tensordot(c.T.astype(np.float64), f, axes=([1], [0]))
    return rho, mom / rho


def stream(f, d):
    """Move f_a one node along c_a with periodic wrap (array axes are [z,] y, x)."""
    c, _ = _tables(d)
    out = np.empty_like(f)
    for a in range(f.shape[0]):
        # grid array axes are reversed relative to (x, y, z)
        shifts = tuple(int(c[a][i]) for i in reversed(range(d)))
        out[a] = np.roll(f[a], shifts, axis=tuple(range(d)))
    return out


def run(rho0, u0, nsteps, tau=1.0, record=False):
    """Eq. (1) on a fully periodic grid from f = f^eq(rho0, u0).

    Returns (rho, u) after ``nsteps`` (and the per-step history if ``record``).
    """
    rho0 = np.asarray(rho0, dtype=np.float64)
    u0 = np.asarray(u0, dtype=np.float64)
    d = u0.shape[0]
    f = equilibrium(rho0, u0)
    hist = []
    for _ in range(nsteps):
        rho, u = moments(f, d)
        f = f + (equilibrium(rho, u) - f) / tau   # collide
        f = stream(f, d)                          # stream
        if record:
            hist.append(moments(f, d))
    rho, u = moments(f, d)
    return (rho, u, hist) if record else (rho, u)
