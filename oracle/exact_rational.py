"""Exact rational MacLAB on tiny grids (fractions.Fraction), for pinning the oracle.

TEST INFRASTRUCTURE ONLY.  Independent of ``maclab_oracle.c``: pure Python,
exact arithmetic, its own velocity lists, and each equilibrium term written out
as the paper states it.  Used on 4x4 (D2Q9) and 4x4x4 (D3Q19) grids for a few
steps, where it is cheap.

Per step, for every fluid node x (Eqs. (4)-(5) with the Eq. (2) equilibrium in
lattice units, the Test 2 force added after the division):
    rho'(x)  = sum_a w_a rho(y) (1 + 3 c_a.u(y) + 9/2 (c_a.u(y))^2 - 3/2 u(y).u(y)),
    u'_i(x)  = [sum_a c_ai (same term)] / rho'(x) + force_i,     y = x - c_a,
with periodic wrap on periodic axes; wall nodes keep their values.
"""
from __future__ import annotations

from fractions import Fraction as Fr
from itertools import product

D2Q9 = [((0, 0), Fr(4, 9)), ((1, 0), Fr(1, 9)), ((0, 1), Fr(1, 9)), ((-1, 0), Fr(1, 9)),
        ((0, -1), Fr(1, 9)), ((1, 1), Fr(1, 36)), ((-1, 1), Fr(1, 36)), ((-1, -1), Fr(1, 36)),
        ((1, -1), Fr(1, 36))]
D3Q19 = ([((0, 0, 0), Fr(1, 3))]
         + [(c, Fr(1, 18)) for c in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1),
                                     (0, 0, -1)]]
         + [(c, Fr(1, 36)) for c in [(1, 1, 0), (-1, -1, 0), (-1, 1, 0), (1, -1, 0), (0, 1, 1),
                                     (0, -1, -1), (0, -1, 1), (0, 1, -1), (1, 0, 1), (-1, 0, -1),
                                     (-1, 0, 1), (1, 0, -1)]])


def step(lattice_d, dims, periodic, rho, u, wall=None, force=None):
    """One exact step.  dims = (nx, ny[, nz]); rho: dict coord->Fraction;
    u: dict coord->tuple of Fractions; wall: set of wall coords."""
    vel = D2Q9 if lattice_d == 2 else D3Q19
    wall = wall or set()
    force = force or tuple(Fr(0) for _ in range(lattice_d))
    rho_n, u_n = {}, {}
    for x in product(*[range(n) for n in dims]):
        if x in wall:
            rho_n[x], u_n[x] = rho[x], u[x]
            continue
        r = Fr(0)
        m = [Fr(0)] * lattice_d
        for c, w in vel:
            y = []
            for i in range(lattice_d):
                yi = x[i] - c[i]
                if not 0 <= yi < dims[i]:
                    if not (periodic >> i) & 1:
                        raise ValueError("fluid node next to an open boundary")
                    yi %= dims[i]
                y.append(yi)
            y = tuple(y)
            uy = u[y]
            cu = sum(c[i] * uy[i] for i in range(lattice_d))
            uu = sum(uy[i] * uy[i] for i in range(lattice_d))
            f = w * rho[y] * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu)
            r += f
            for i in range(lattice_d):
                m[i] += c[i] * f
        rho_n[x] = r
        u_n[x] = tuple(m[i] / r + force[i] for i in range(lattice_d))
    return rho_n, u_n


def bgk_run(dims, rho, u, nsteps, tau):
    """Exact rational single-relaxation-time LBM (Eq. (1) with a BGK
    collision of relaxation time tau) on a fully periodic D2Q9 grid, started
    from f = f^eq(rho, u) (Eq. (2)).  Each step: moments (Eq. (3)), collide
    f <- f + (f^eq - f) / tau, then stream f_a(x + c_a) <- f_a(x).  Returns the
    moments (rho, u) after nsteps; tau is a Fraction."""
    def feq(r, v):
        uu = sum(vi * vi for vi in v)
        out = []
        for c, w in D2Q9:
            cu = c[0] * v[0] + c[1] * v[1]
            out.append(w * r * (1 + 3 * cu + Fr(9, 2) * cu * cu - Fr(3, 2) * uu))
        return out

    def mom(fx):
        r = sum(fx)
        m = [sum(c[i] * fa for (c, _), fa in zip(D2Q9, fx)) for i in range(2)]
        return r, (m[0] / r, m[1] / r)

    nodes = list(product(range(dims[0]), range(dims[1])))
    f = {x: feq(rho[x], u[x]) for x in nodes}
    for _ in range(nsteps):
        post = {}
        for x in nodes:
            r, v = mom(f[x])
            e = feq(r, v)
            post[x] = [fa + (ea - fa) / tau for fa, ea in zip(f[x], e)]
        f = {x: [None] * 9 for x in nodes}
        for x in nodes:
            for a, (c, _) in enumerate(D2Q9):
                y = ((x[0] + c[0]) % dims[0], (x[1] + c[1]) % dims[1])
                f[y][a] = post[x][a]
    rho_n, u_n = {}, {}
    for x in nodes:
        rho_n[x], u_n[x] = mom(f[x])
    return rho_n, u_n
