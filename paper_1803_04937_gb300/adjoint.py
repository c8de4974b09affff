"""Differentiable D3Q19 runs: a ``torch.autograd.Function`` whose backward pass
is the hand-written reverse-mode adjoint of the lattice Boltzmann step
(``lbm_adjoint_*`` in include/lbm.h), with sqrt(T) checkpointing.

Forward: f(0) = feq(rho, u0) (Eq. 14 or Eq. 22), T steps of Eq. 15 (A/B
pattern), output (rho(T), u(T)) of Eq. 16-17.  Every ceil(sqrt(T)) steps the
raw A/B grid is copied into a checkpoint.  Backward: lambda(T) from dL/du(T)
and dL/drho(T); then, segment by segment from the last, the states of the
segment are recomputed from its checkpoint into a ring of grids and the
adjoint steps run in reverse; finally dL/du0 through f(0) = feq(rho, u0) and
dL/dtau from the FP64 accumulators of dL/domega+-.  Memory: ~2 sqrt(T) grids.
Supports rho0 = 1 (the paper's choice) only.
"""
import ctypes
import math

import torch

from . import _lib
from ._lib import check
from .lbm import Simulation, _field_dtype, _ptr


def _dp(t):
    return ctypes.cast(ctypes.c_void_p(t.data_ptr()), ctypes.POINTER(ctypes.c_double))


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, tau, rho, spec, nsteps, every):
        sim = Simulation(**dict(spec, tau=float(tau)))
        u0c = u0.detach().contiguous()
        rhoc = rho.detach().to(u0c.dtype).contiguous() if rho is not None else None
        sim.init(rhoc, u0c)
        ckpts = []
        t = 0
        while t < nsteps:
            if t % every == 0:
                ckpts.append(sim.grids[t % 2].clone())
            k = min(every - t % every, nsteps - t)
            sim.step(k)
            t += k
        r, u = sim.moments(u0.dtype)
        ctx.sim = sim
        ctx.ckpts = ckpts
        ctx.nsteps = nsteps
        ctx.every = every
        ctx.tau_meta = (tau.device, tau.dtype) if torch.is_tensor(tau) else (torch.device("cpu"), torch.float64)
        ctx.save_for_backward(u0c, rhoc if rhoc is not None else torch.empty(0, device=u0.device))
        return r, u

    @staticmethod
    def backward(ctx, grad_rho, grad_u):
        sim = ctx.sim
        lib = sim._lib
        h = sim.handle
        u0, rho = ctx.saved_tensors
        nsteps, every = ctx.nsteps, ctx.every
        dev = u0.device
        lam_dtype = torch.float64 if sim.precision == _lib.F64 else torch.float32
        shape = (19,) + sim.shape
        if grad_u is None:
            grad_u = torch.zeros_like(u0)
        grad_u = grad_u.contiguous()
        dt = _field_dtype(grad_u)
        grad_rho = grad_rho.to(grad_u.dtype).contiguous() if grad_rho is not None else None
        lam = [torch.empty(shape, dtype=lam_dtype, device=dev) for _ in range(2)]
        gw = torch.zeros(2, dtype=torch.float64, device=dev)
        # each step's dL/domega terms are summed inside the next step's kernel (bitwise the same sums)
        check(lib.lbm_set_option(h, _lib.OPT_ADJ_DEFER_SUM, 1.0), h)
        check(lib.lbm_adjoint_seed(h, _ptr(grad_rho), _ptr(grad_u), dt, _ptr(lam[0])), h)
        cur = 0
        ring = [torch.empty(shape, dtype=sim.storage_dtype, device=dev) for _ in range(min(every, nsteps) + 1)]
        nseg = len(ctx.ckpts)
        for s in range(nseg - 1, -1, -1):
            t0 = s * every
            t1 = min(t0 + every, nsteps)
            ring[0].copy_(ctx.ckpts[s])
            for i in range(1, t1 - t0):  # states t0+1 .. t1-1
                sim._bind(ring[i - 1], ring[i])
                sim.step(1)
            for t in range(t1 - 1, t0 - 1, -1):
                check(lib.lbm_adjoint_step(h, _ptr(ring[t - t0]), _ptr(lam[cur]), _ptr(lam[1 - cur]), _dp(gw)), h)
                cur = 1 - cur
        grad_u0 = torch.empty_like(u0)
        check(lib.lbm_adjoint_init_velocity(h, _ptr(rho) if rho.numel() else None, _ptr(u0), _field_dtype(u0),
                                            _ptr(lam[cur]), _ptr(grad_u0)), h)
        check(lib.lbm_adjoint_flush(h), h)
        gwh = gw.cpu()
        dtau = ctypes.c_double()
        check(lib.lbm_adjoint_tau_gradient(h, _dp(gwh), ctypes.byref(dtau)), h)
        ctx.sim = None
        ctx.ckpts = None
        sim.close()
        grad_tau = torch.tensor(dtau.value, dtype=ctx.tau_meta[1], device=ctx.tau_meta[0])
        return grad_u0, grad_tau, None, None, None, None


def simulate(u0, tau, nsteps, nx, ny, nz, rho=None, equilibrium="improved", collision="srt", precision="f32",
             force=(0.0, 0.0, 0.0), walls=(False, False, False), trt_magic=3.0 / 16.0, checkpoint_every=None):
    """Differentiable run of nsteps D3Q19 steps from f = feq(rho, u0).

    u0: [3, nz, ny, nx] float64/float32 CUDA tensor; tau: 0-d tensor (may
    require grad) or float.  Returns (rho(T), u(T)) in u0's dtype.  Gradients
    flow to u0 and tau through the adjoint; checkpoint_every defaults to
    ceil(sqrt(nsteps))."""
    if not torch.is_tensor(tau):
        tau = torch.tensor(float(tau), dtype=torch.float64)
    every = checkpoint_every or max(1, math.ceil(math.sqrt(max(nsteps, 1))))
    spec = dict(nx=nx, ny=ny, nz=nz, equilibrium=equilibrium, collision=collision, precision=precision,
                force=tuple(force), walls=tuple(walls), trt_magic=trt_magic, pattern="ab", device=u0.device)
    return _Run.apply(u0, tau, rho, spec, int(nsteps), int(every))


def forward_only(u0, tau, nsteps, nx, ny, nz, rho=None, **kw):
    """The same forward run without autograd bookkeeping (for finite differences)."""
    sim = Simulation(nx, ny, nz, tau=float(tau), device=u0.device, pattern="ab", **kw)
    sim.init(rho, u0)
    sim.step(nsteps)
    out = sim.moments(u0.dtype)
    sim.close()
    return out
