"""Gradients through a P3M run: a torch.autograd.Function over the C ABI's reverse-mode pieces.

The loss is the L2 distance of the final CIC density contrast from a target mesh; the input is
the initial displacement field psi (3, N) on a lattice q, from which the run starts with the
Zel'dovich state x = q + psi, p = m a_0^(1/2) psi (Einstein-de Sitter linear growth).  The
backward pass is the reverse sweep of the kick-drift-kick steps,

    lam_x <- dL/dx_n,  lam_p <- 0
    for k = n-1 .. 0:   lam_x += m (K2_k + K1_{k+1}) (dA/dx)^T|_{x_{k+1}} lam_p   (K1_n = 0)
                        lam_p += (D_k / m) lam_x
    lam_x += m K1_0 (dA/dx)^T|_{x_0} lam_p;   dL/dpsi = lam_x + m a_0^(1/2) lam_p,

with the states x_k recomputed from checkpoints kept every `every` steps (about sqrt(n)).
Every arithmetic step runs in the library's kernels (p3m_step, p3m_force_vjp,
p3m_density_loss, p3m_axpy); torch only holds the device arrays.
"""

from __future__ import annotations

import math

import torch


def _state(sim):
    n = sim.n
    dev = torch.device("cuda", torch.cuda.current_device())
    pos = torch.empty((3, n), dtype=torch.float64, device=dev)
    mom = torch.empty_like(pos)
    acc = torch.empty_like(pos)
    sim.get_particles(pos, mom, acc)
    return pos, mom, acc


class DensityLossRun(torch.autograd.Function):
    """loss = DensityLossRun.apply(psi, sim, q, a_list, target, every)."""

    @staticmethod
    def forward(ctx, psi, sim, q, a_list, target, every):
        m = getattr(sim, "mass", 1.0)
        a_list = [float(v) for v in a_list]
        n = len(a_list) - 1
        x0 = q.clone()
        sim.axpy(1.0, psi, x0)
        p0 = torch.zeros_like(psi)
        sim.axpy(m * math.sqrt(a_list[0]), psi, p0)
        sim.set_particles(x0, p0, mass=m, a=a_list[0])
        acc0 = torch.empty_like(psi)
        sim.forces(a_list[0], out=acc0)
        ckpt = {0: _state(sim)}
        for k in range(n):
            sim.step(a_list[k], a_list[k + 1] - a_list[k])
            if (k + 1) % every == 0 and k + 1 < n:
                ckpt[k + 1] = _state(sim)
        grad_x = torch.empty_like(psi)
        loss, _ = sim.density_loss(target, grad_x)
        ctx.sim, ctx.a_list, ctx.every, ctx.ckpt, ctx.m = sim, a_list, every, ckpt, m
        ctx.save_for_backward(grad_x)
        return psi.new_tensor(loss)

    @staticmethod
    def backward(ctx, gout):
        (grad_x,) = ctx.saved_tensors
        sim, a, every, ckpt, m = ctx.sim, ctx.a_list, ctx.every, ctx.ckpt, ctx.m
        n = len(a) - 1
        fac = [sim.step_factors(a[k], a[k + 1] - a[k]) for k in range(n)]  # (m K1, D/m, m K2)
        lam_x = torch.zeros_like(grad_x)
        sim.axpy(float(gout), grad_x, lam_x)
        lam_p = torch.zeros_like(grad_x)
        out = torch.empty_like(grad_x)
        for s in sorted(ckpt, reverse=True):
            e = min(s + every, n)
            pos, mom, acc = ckpt[s]
            sim.set_particles(pos, mom, acc, mass=m, a=a[s])
            states = {s: (pos, mom, acc)}
            for k in range(s, e):
                sim.step(a[k], a[k + 1] - a[k])
                states[k + 1] = _state(sim)
            for k in range(e - 1, s - 1, -1):
                p_, m_, a_ = states[k + 1]
                sim.set_particles(p_, m_, a_, mass=m, a=a[k + 1])
                sim.force_vjp(lam_p, out)
                kf = fac[k][2] + (fac[k + 1][0] if k + 1 < n else 0.0)
                sim.axpy(kf, out, lam_x)
                sim.axpy(fac[k][1], lam_x, lam_p)
        p_, m_, a_ = ckpt[0]
        sim.set_particles(p_, m_, a_, mass=m, a=a[0])
        sim.force_vjp(lam_p, out)
        sim.axpy(fac[0][0], out, lam_x)
        sim.axpy(m * math.sqrt(a[0]), lam_p, lam_x)
        return lam_x, None, None, None, None, None
