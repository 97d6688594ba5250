"""FP64 CPU oracle of the MacLAB step (Zhou, "Macroscopic Lattice Boltzmann Method").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this module.  The CUDA
library never does, and this module imports nothing from it.

The arithmetic lives in ``maclab_oracle.c`` (plain loops, FP64, no FMA
contraction); this file builds it with gcc, loads it with ctypes and adds the
host-side formulas the paper states outright:

* ``params``: particle speed e = 6 nu / dx (Eq. (6)) and dt = dx / e (the
  sentence after Eq. (6)), so dt = dx^2 / (6 nu).
* unit maps between physical (rho, u) and the lattice units the C code uses
  (ut = u / e; rho is kept as rho / rho0, which Eqs. (2), (4), (5) allow because
  they are homogeneous of degree one in rho).
* the Test 2 body force in lattice units (see ``force_lattice``).
* plain diagnostics (mass, kinetic energy, momentum, residual) as sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "maclab_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libmaclab_oracle.so")
_lock = threading.Lock()
_lib = None

D2Q9, D3Q19 = 0, 1
DIMS = {D2Q9: 2, D3Q19: 3}


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2, no FMA contraction, no fast-math).

    With OpenMP where gcc has it (the node loops then run on several host
    threads, with results bitwise independent of the thread count); without it
    if that build fails.
    """
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u32, vp, dp = ctypes.c_int64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p
            lib.oracle_step.argtypes = [ctypes.c_int, i64, i64, i64, u32, vp, dp, dp, dp, dp, dp]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_run.argtypes = [ctypes.c_int, i64, i64, i64, u32, vp, dp, dp, dp, i64]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_adjoint_step.argtypes = [ctypes.c_int, i64, i64, i64, u32, vp, dp, dp, dp,
                                                dp, dp, dp, dp, dp]
            lib.oracle_adjoint_step.restype = ctypes.c_int
            lib.oracle_adjoint_step_gather.argtypes = lib.oracle_adjoint_step.argtypes
            lib.oracle_adjoint_step_gather.restype = ctypes.c_int
            lib.oracle_nu_term.argtypes = [ctypes.c_int, i64, i64, i64, u32, vp, dp, dp, dp, dp, dp,
                                           ctypes.POINTER(ctypes.c_int)]
            lib.oracle_nu_term.restype = ctypes.c_double
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_lattice_table.argtypes = [ctypes.c_int, vp, vp]
            lib.oracle_lattice_table.restype = ctypes.c_int
            lib.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_feq.restype = ctypes.c_double
            _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's node loops (0: keep); returns the count in use.

    Results do not depend on it (each value is formed by one thread in the
    single-thread order).
    """
    return _load().oracle_set_threads(int(n))


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"oracle {what} failed with code {rc} "
                         "(-1 bad argument, -2 fluid node next to an open boundary, -3 no memory)")


def lattice_table(lattice: int):
    """Velocity set c_a (Q x 3 ints) and weights w_a as the oracle holds them."""
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    q = _load().oracle_lattice_table(lattice, _ptr(c), _ptr(w))
    _check(0 if q > 0 else q, "lattice_table")
    return c.reshape(19, 3)[:q].copy(), w[:q].copy()


def feq(lattice: int, a: int, rho: float, ut) -> float:
    """Eq. (2) in lattice units for one direction (exported for the tests)."""
    u3 = np.zeros(3)
    u3[: len(ut)] = ut
    return _load().oracle_feq(lattice, a, float(rho), _ptr(u3))


def _shape(lattice, rho):
    d = DIMS[lattice]
    if rho.ndim != d:
        raise ValueError(f"rho must have {d} dims, got {rho.shape}")
    if d == 2:
        ny, nx = rho.shape
        nz = 1
    else:
        nz, ny, nx = rho.shape
    return d, nx, ny, nz


def step(lattice, rho, u, periodic, wall=None, force=None, nsteps=1):
    """Advance (rho, ut) by ``nsteps`` MacLAB steps; returns new arrays.

    rho: [ny, nx] or [nz, ny, nx]; u: [d, ...] lattice-unit velocity; periodic:
    bitmask (bit0 x, bit1 y, bit2 z); wall: bool/uint8 array (nonzero = wall
    node, keeps its values); force: d lattice-unit increments (Test 2 term).
    """
    rho = _f64(rho).copy()
    d, nx, ny, nz = _shape(lattice, rho)
    u = _f64(u).copy()
    if u.shape != (d,) + rho.shape:
        raise ValueError(f"u must have shape {(d,) + rho.shape}, got {u.shape}")
    wall_b = None if wall is None else np.ascontiguousarray(wall, dtype=np.uint8)
    f = None if force is None else _f64(np.asarray(force, dtype=np.float64).reshape(d))
    rc = _load().oracle_run(lattice, nx, ny, nz, int(periodic), _ptr(wall_b), _ptr(rho),
                            _ptr(u), _ptr(f), int(nsteps))
    _check(rc, "run")
    return rho, u


def adjoint_step(lattice, rho, u, periodic, lam_rho_next, lam_u_next, wall=None, force=None,
                 gather=False):
    """Adjoint of one ``step``: returns (lam_rho, lam_u, grad_force).

    gather=False: the plain scatter, one thread.  gather=True: the same sums
    as a gather over sources, on the oracle's host threads (bitwise equal).
    """
    rho = _f64(rho)
    d, nx, ny, nz = _shape(lattice, rho)
    u = _f64(u)
    lr1, lu1 = _f64(lam_rho_next), _f64(lam_u_next)
    lr, lu = np.zeros_like(rho), np.zeros_like(u)
    gf = np.zeros(d)
    wall_b = None if wall is None else np.ascontiguousarray(wall, dtype=np.uint8)
    f = None if force is None else _f64(np.asarray(force, dtype=np.float64).reshape(d))
    lib = _load()
    fn = lib.oracle_adjoint_step_gather if gather else lib.oracle_adjoint_step
    rc = fn(lattice, nx, ny, nz, int(periodic), _ptr(wall_b), _ptr(rho), _ptr(u), _ptr(f),
            _ptr(lr1), _ptr(lu1), _ptr(lr), _ptr(lu), _ptr(gf))
    _check(rc, "adjoint_step")
    return lr, lu, gf


def nu_term(lattice, rho, u, periodic, lam_rho_next, lam_u_next, wall=None, force=None):
    """The viscosity term of one reverse step (see maclab_oracle.c): summed over
    a rollout's steps it gives e dL/de (Eq. (6): nu enters only through e)."""
    rho = _f64(rho)
    d, nx, ny, nz = _shape(lattice, rho)
    u = _f64(u)
    lr, lu = _f64(lam_rho_next), _f64(lam_u_next)
    wall_b = None if wall is None else np.ascontiguousarray(wall, dtype=np.uint8)
    f = None if force is None else _f64(np.asarray(force, dtype=np.float64).reshape(d))
    st = ctypes.c_int(0)
    v = _load().oracle_nu_term(lattice, nx, ny, nz, int(periodic), _ptr(wall_b), _ptr(rho), _ptr(u),
                               _ptr(f), _ptr(lr), _ptr(lu), ctypes.byref(st))
    _check(st.value, "nu_term")
    return v


def rollout_adjoint(lattice, rho0, u0, periodic, nsteps, lam_rho_T, lam_u_T, wall=None,
                    force=None, checkpoint_every=None, gather=False):
    """Reverse-mode gradient of an n-step rollout.

    Returns (lam_rho_0, lam_u_0, grad_force) for a loss whose adjoint on the
    final state is (lam_rho_T, lam_u_T).  lam_rho_T may instead be a function
    of the final state, (rho_T, u_T) -> (lam_rho_T, lam_u_T) (lam_u_T is then
    ignored), for a loss on the state the forward pass reaches.
    checkpoint_every=None stores every
    state; an integer K keeps only the states of steps 0, K, 2K, ... and
    recomputes each segment's states from its checkpoint when the reverse pass
    reaches it (the forward step is deterministic, so the states and the
    result are the same).  gather: see ``adjoint_step``.
    """
    gf = np.zeros(DIMS[lattice])
    k = nsteps if not checkpoint_every else max(1, int(checkpoint_every))
    checkpoints = {0: (_f64(rho0), _f64(u0))}
    state = checkpoints[0]
    for s in range(1, nsteps + 1):
        state = step(lattice, *state, periodic, wall=wall, force=force)
        if s % k == 0 and s < nsteps:
            checkpoints[s] = state
    if callable(lam_rho_T):
        lam_rho_T, lam_u_T = lam_rho_T(*state)
    lr, lu = _f64(lam_rho_T), _f64(lam_u_T)
    for start in sorted(checkpoints, reverse=True):
        stop = min(start + k, nsteps)
        seg = [checkpoints[start]]
        for _ in range(start, stop - 1):
            seg.append(step(lattice, *seg[-1], periodic, wall=wall, force=force))
        for s in range(stop - 1, start - 1, -1):
            lr, lu, g = adjoint_step(lattice, *seg[s - start], periodic, lr, lu, wall=wall,
                                     force=force, gather=gather)
            gf += g
    return lr, lu, gf


# ---------------------------------------------------------------- unit maps

def params(dx: float, nu: float):
    """(e, dt): Eq. (6) e = 6 nu / dx and dt = dx / e."""
    if dx <= 0 or nu <= 0:
        raise ValueError("dx and nu must be positive")
    e = 6.0 * nu / dx
    return e, dx / e


def lattice_reynolds(u_max: float, dx: float, nu: float) -> float:
    """R_le = U_m dx / nu, the stability indicator stated after Eq. (6)."""
    return u_max * dx / nu


def force_lattice(accel, dx: float, nu: float):
    """Lattice-unit velocity increment per step of a body acceleration.

    Test 2 adds a pressure-gradient term of size dx/(e rho) dp/dx = dt/rho dp/dx
    to the velocity of Eq. (5).  With accel = -(1/rho0) dp/dx (the sign for
    which the closed form Eq. (8) holds) the physical increment is accel * dt,
    i.e. accel * dt / e in lattice units.
    """
    e, dt = params(dx, nu)
    return np.asarray(accel, dtype=np.float64) * dt / e


def to_lattice(rho, u, dx, nu, rho0=1.0):
    e, _ = params(dx, nu)
    return _f64(rho) / rho0, _f64(u) / e


def to_physical(rho_l, u_l, dx, nu, rho0=1.0):
    e, _ = params(dx, nu)
    return _f64(rho_l) * rho0, _f64(u_l) * e


# ---------------------------------------------------------------- diagnostics

def diagnostics(rho, u, u_prev=None, fluid=None):
    """Plain FP64 sums over fluid nodes, in lattice units.

    Returns dict: mass = sum rho, kinetic = sum 1/2 rho |ut|^2, momentum[i] =
    sum rho ut_i, residual = ||ut - ut_prev||_2 / ||ut||_2 (if u_prev given).
    Conservation of the first three on periodic grids is the property stated
    with Eq. (15).
    """
    rho = _f64(rho)
    u = _f64(u)
    m = np.ones(rho.shape, dtype=bool) if fluid is None else np.asarray(fluid, dtype=bool)
    out = {
        "mass": float(np.sum(rho[m])),
        "kinetic": float(np.sum(0.5 * rho[m] * np.sum(u[:, m] ** 2, axis=0))),
        "momentum": [float(np.sum(rho[m] * u[i][m])) for i in range(u.shape[0])],
    }
    if u_prev is not None:
        du = u[:, m] - _f64(u_prev)[:, m]
        out["residual"] = float(np.sqrt(np.sum(du ** 2)) / np.sqrt(np.sum(u[:, m] ** 2)))
    return out
