"""Gradients of a wake and power objective through the hand-written adjoint.

The objective of a rotor run of N fixed-dt steps from a uniform stream U_inf:

    J(s, U_inf) = mean over the cells of the plane x-index `iplane` of
                  (U_inf - rho U / rho) after the last step  +  beta * P_N,

with s the per-actuator-point force scales and P_N the rotor power of the
last step. :class:`RotorObjective` is a ``torch.autograd.Function``: the
forward pass runs the CUDA steps and keeps the state every K steps; the
backward pass recomputes each segment from its checkpoint and runs the
reverse steps backwards through it (checkpointed recomputation). With room
on the device for K step tapes (``gks_step_record``), each segment is run
forward once with its tapes kept and reversed from them
(``gks_step_reverse``); otherwise the segment's states are recomputed and
each reverse step recomputes its own forward step (``gks_step_adjoint``).
The state and adjoint stay on the device; the objective's own seed
(dJ/dW after the last step) is formed with torch.
"""
from __future__ import annotations

import numpy as np
import torch



def uniform_state(grid, uinf, rho=1.0):
    Q = torch.zeros(grid.shape, dtype=torch.float64, device=grid.device)
    Q[0] = rho
    Q[1] = rho * uinf
    return Q


def plane_deficit(state, iplane, uinf):
    u = state[1, :, :, iplane] / state[0, :, :, iplane]
    return float((uinf - u).mean().item())


def plane_deficit_seed(state, iplane):
    """dJ/dW of the plane-mean deficit term."""
    lam = torch.zeros_like(state)
    rho = state[0, :, :, iplane]
    mx = state[1, :, :, iplane]
    n = rho.numel()
    lam[1, :, :, iplane] = -1.0 / (n * rho)
    lam[0, :, :, iplane] = mx / (n * rho * rho)
    return lam


def _tapes(grid, k, mode):
    """k tapes for recorded steps, or None (mode "off", or "auto" without room
    for them next to the scratch and a 4 GiB margin)."""
    if mode == "off":
        return None
    need = k * grid.adjoint_tape_bytes()
    if mode == "auto":
        free, _ = torch.cuda.mem_get_info(grid.device)
        free += torch.cuda.memory_reserved(grid.device) - torch.cuda.memory_allocated(grid.device)
        if need + (4 << 30) > free:
            return None
    return [grid.adjoint_tape() for _ in range(k)]


class RotorObjective(torch.autograd.Function):
    """J(scales, uinf) for a configured FP64 grid with one rotor and a fixed
    time step. Arguments after uinf are not differentiated: grid, nsteps,
    checkpoint interval K, plane index, power weight beta, tape mode."""

    @staticmethod
    def forward(ctx, scales, uinf, grid, nsteps, K, iplane, beta, tape):
        u = float(uinf.item())
        grid.set_force_scales(0, scales.detach().cpu().numpy())
        grid.set_inflow(1.0, u, 0.0, 0.0)
        grid.set_state_tensor(uniform_state(grid, u))
        grid.set_time(0.0)
        dt = grid.dt_fixed
        ckpts = {0: uniform_state(grid, u)}
        for n in range(nsteps):
            grid.step(1, sync=False)   # stream-ordered; device errors surface at the sync below
            if (n + 1) % K == 0 and n + 1 < nsteps:
                ckpts[n + 1] = grid.state_tensor()
        grid.sync()
        WN = grid.state_tensor()
        P = grid.forces(0)["power"]
        J = plane_deficit(WN, iplane, u) + beta * P
        ctx.grid, ctx.nsteps, ctx.K, ctx.iplane, ctx.beta, ctx.u, ctx.dt = grid, nsteps, K, iplane, beta, u, dt
        ctx.ckpts, ctx.WN, ctx.tape = ckpts, WN, tape
        ctx.nscales = scales.numel()
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        g, N, K, dt = ctx.grid, ctx.nsteps, ctx.K, ctx.dt
        tapes = _tapes(g, min(K, N), ctx.tape)
        work = g.adjoint_scratch() if tapes else g.adjoint_workspace()
        lam = plane_deficit_seed(ctx.WN, ctx.iplane)
        gs = np.zeros(ctx.nscales)
        gu = 0.0
        starts = sorted(ctx.ckpts)
        for si in range(len(starts) - 1, -1, -1):
            k0 = starts[si]
            k1 = starts[si + 1] if si + 1 < len(starts) else N
            g.set_state_tensor(ctx.ckpts[k0])
            g.set_time(k0 * dt)
            if tapes:
                # the segment forward once, each step keeping its tape
                for n in range(k0, k1):
                    g.step_record(tapes[n - k0])
                for n in range(k1 - 1, k0 - 1, -1):
                    seed = ctx.beta if n == N - 1 else 0.0
                    lam, gun = g.step_reverse(tapes[n - k0], work, lam, seed, gs)
                    gu += gun
                continue
            # recompute the segment's states from its checkpoint
            states = [ctx.ckpts[k0]]
            for _ in range(k0, k1 - 1):
                g.step(1)
                states.append(g.state_tensor())
            for n in range(k1 - 1, k0 - 1, -1):
                seed = ctx.beta if n == N - 1 else 0.0
                lam, gun = g.step_adjoint(work, n * dt, states[n - k0], lam, seed, gs)
                gu += gun
        # the initial state (rho, rho U_inf, 0, 0) and the explicit U_inf of J
        gu += float(lam[1].sum().item()) + 1.0
        gJ = float(gJ)
        return (torch.from_numpy(gs * gJ), torch.tensor(gu * gJ, dtype=torch.float64),
                None, None, None, None, None, None)


def rotor_objective(grid, scales, uinf, nsteps, K=20, iplane=None, beta=1.0, tape="auto"):
    """J as a differentiable function of (scales, uinf) (float64 CPU tensors
    with requires_grad); the grid must have one rotor and dt_fixed > 0. On an
    FP64 grid the gradient is that of the FP64 steps; on an FP32C grid that of
    the FP32C steps (FP32 reverse arithmetic). tape:
    "auto" (recorded steps when K tapes fit on the device), "on" (always; the
    allocation fails if they do not fit) or "off" (recompute every reverse
    step)."""
    if iplane is None:
        raise ValueError("iplane (x index of the sampling plane) is required")
    if scales.dtype != torch.float64 or uinf.dtype != torch.float64:
        raise TypeError("scales and uinf must be float64 tensors (FP64 adjoint)")
    if tape not in ("auto", "on", "off"):
        raise ValueError("tape must be 'auto', 'on' or 'off'")
    return RotorObjective.apply(scales, uinf, grid, int(nsteps), int(K), int(iplane), float(beta), tape)
