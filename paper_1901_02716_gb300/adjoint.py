"""Differentiable MacLAB rollouts on the GPU (torch.autograd.Function).

The forward pass creates a solver for the given viscosity and wall values,
sets the initial physical fields and runs ``nsteps`` steps, keeping the raw
state every ``checkpoint_every`` steps (default ~sqrt(nsteps)).  The backward
pass walks the segments from the last to the first: it recomputes the states
of a segment from its checkpoint, then runs maclab_adjoint_step back through
them.  Memory: about 2 sqrt(nsteps) raw states.  All arithmetic is in the
library's kernels; this module only moves device buffers and calls the C ABI.

Gradients are returned for the initial density and velocity (physical, zero on
wall nodes), the wall velocities (one row per wall id) and the viscosity nu (at
a fixed number of steps: e = 6 nu / dx changes the lattice velocities and the
time step).  dL/dnu is summed step by step during the reverse pass
(maclab_adjoint_nu_term: the defect of each step under the e-scaling, dotted
with the adjoint it produced), which keeps FP32 rollouts accurate where the
end-point form (the difference of two nearly equal products, kept as
``grads_extra["nu_endpoint"]``) loses digits.  That term is a pass of its own
per reverse step, so it is formed only when the viscosity's gradient is
requested (nu.requires_grad).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import torch

from . import maclab as M


@dataclasses.dataclass
class RolloutSpec:
    lattice: int
    dims: tuple
    dx: float
    nsteps: int
    periodic: int = 0
    node_type: np.ndarray | None = None
    wall_rho: np.ndarray | None = None
    precision: int = M.F32
    body_force: tuple | None = None
    rho0: float = 1.0
    checkpoint_every: int = 0       # 0: about sqrt(nsteps)


def _raw(solver):
    buf = torch.empty(solver.state_bytes(), dtype=torch.uint8, device="cuda")
    solver.get_lattice_state(buf)
    return buf


class MacLABRollout(torch.autograd.Function):
    """(rho0, u0, wall_u, nu) -> (rho_T, u_T) after spec.nsteps MacLAB steps."""

    @staticmethod
    def forward(ctx, rho0, u0, wall_u, nu, spec: RolloutSpec):
        n_walls = 0 if wall_u is None else int(wall_u.shape[0])
        wu = None if n_walls == 0 else wall_u.detach().double().cpu().numpy()
        s = M.Solver(spec.lattice, spec.dims, spec.dx, float(nu), spec.precision, spec.periodic,
                     spec.node_type, spec.wall_rho, wu, spec.body_force, spec.rho0)
        s.set_state(rho0.detach().contiguous(), u0.detach().contiguous())
        n = int(spec.nsteps)
        seg = spec.checkpoint_every or max(1, int(round(math.sqrt(max(n, 1)))))
        ckpts = []
        done = 0
        while done < n:
            ckpts.append(_raw(s))
            k = min(seg, n - done)
            s.step(k)
            done += k
        state_T = _raw(s)
        if not ckpts:
            ckpts.append(state_T)
        rho_T = torch.empty_like(rho0)
        u_T = torch.empty_like(u0)
        s.get_state_into(rho_T, u_T)
        ctx.solver, ctx.ckpts, ctx.state_T, ctx.seg, ctx.n = s, ckpts, state_T, seg, n
        ctx.dx = float(spec.dx)
        ctx.n_walls = n_walls
        ctx.d = u0.shape[0]
        ctx.wall_dtype = None if wall_u is None else wall_u.dtype
        ctx.nu_dtype = nu.dtype if torch.is_tensor(nu) else torch.float64
        return rho_T, u_T

    @staticmethod
    def backward(ctx, g_rho, g_u):
        s = ctx.solver
        h = s.handle
        nb = s.adjoint_bytes()
        lam = torch.empty(nb, dtype=torch.uint8, device="cuda")
        lam2 = torch.empty_like(lam)
        dot_T = M.maclab_adjoint_seed(h, None if g_rho is None else g_rho.contiguous(),
                                      None if g_u is None else g_u.contiguous(), ctx.state_T, lam)
        gforce = torch.zeros(3, dtype=torch.float64, device="cuda")
        nu_acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        # the viscosity term costs a pass per reverse step: only when dL/dnu is asked for
        need_nu = bool(ctx.needs_input_grad[3])
        n, seg, ckpts = ctx.n, ctx.seg, ctx.ckpts
        bounds = [(i * seg, min((i + 1) * seg, n)) for i in range(len(ckpts))] if n else []
        for idx in range(len(bounds) - 1, -1, -1):
            a, b = bounds[idx]
            end_state = ckpts[idx + 1] if idx + 1 < len(ckpts) else ctx.state_T
            states = [ckpts[idx]]
            s.set_lattice_state(ckpts[idx])
            for _ in range(b - a - 1):
                s.step(1)
                states.append(_raw(s))
            states.append(end_state)
            for k in range(b - a - 1, -1, -1):
                if need_nu:
                    M.maclab_adjoint_nu_term(h, states[k], lam, nu_acc, states[k + 1])
                M.maclab_adjoint_step(h, states[k], states[k + 1], lam, lam2, gforce)
                lam, lam2 = lam2, lam
        ref = g_u if g_u is not None else g_rho
        grad_rho0 = torch.empty(ref.shape[1:] if g_u is not None else ref.shape, dtype=ref.dtype,
                                device="cuda")
        grad_u0 = torch.empty((ctx.d,) + tuple(grad_rho0.shape), dtype=ref.dtype, device="cuda")
        res = M.maclab_adjoint_finish(h, lam, ckpts[0], grad_rho0, grad_u0, dot_T,
                                      gforce.cpu().tolist(), ctx.n_walls)
        grad_wall = None
        if ctx.n_walls:
            grad_wall = torch.tensor([w[1:1 + ctx.d] for w in res["wall"]], dtype=ctx.wall_dtype,
                                     device="cuda")
        # e dL/de = sum of the step terms; dL/dnu = (de/dnu) dL/de, de/dnu = 6 / dx
        e = s.params["e"]
        res["nu_endpoint"] = res["nu"]
        grad_nu = None
        if need_nu:
            grad_nu_steps = (6.0 / ctx.dx) * float(nu_acc.item()) / e
            res["nu"] = grad_nu_steps
            grad_nu = torch.tensor(grad_nu_steps, dtype=ctx.nu_dtype)
        ctx.grads_extra = res
        return grad_rho0, grad_u0, grad_wall, grad_nu, None


def rollout(rho0, u0, wall_u, nu, spec: RolloutSpec):
    """Differentiable n-step MacLAB rollout; returns (rho_T, u_T) (physical)."""
    if not torch.is_tensor(nu):
        nu = torch.tensor(float(nu), dtype=torch.float64)
    return MacLABRollout.apply(rho0, u0, wall_u, nu, spec)
