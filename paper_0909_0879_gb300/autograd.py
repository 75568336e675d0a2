"""torch.autograd binding of the differentiable leapfrog.

``leapfrog(x0, v0, m, nsteps, dt, eps)`` runs nsteps kick-drift-kick steps
(paper Sec. 3.1) on the GPU through libnbody and returns (x(T), v(T)); the
backward pass calls the library's checkpointed adjoint, so gradients with
respect to x0, v0 and m come from the hand-written adjoint kernel, not from
torch's tracing.  Tensors are float32 on one CUDA device; torch provides
only the device memory and the stream.
"""
from __future__ import annotations

import torch

from . import _lib


class LeapfrogFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, v0, m, nsteps: int, dt: float, eps: float, G: float, ckpt_every: int):
        for t in (x0, v0, m):
            if t.dtype != torch.float32 or not t.is_cuda:
                raise TypeError("leapfrog needs float32 CUDA tensors")
        n = m.shape[0]
        stream = torch.cuda.current_stream(x0.device)
        x = x0.detach().contiguous().clone()
        v = v0.detach().contiguous().clone()
        mm = m.detach().contiguous()
        acc = torch.empty_like(x)
        ckpt = torch.empty(_lib.lf_ckpt_floats(n, nsteps, ckpt_every), dtype=torch.float32,
                           device=x.device)
        _lib.lf_forward(n, mm, x, v, acc, nsteps, dt, ckpt, eps=eps, G=G, ckpt_every=ckpt_every,
                        stream=stream)
        ctx.save_for_backward(mm, ckpt)
        ctx.cfg = (n, nsteps, dt, eps, G, ckpt_every)
        return x, v

    @staticmethod
    def backward(ctx, gx, gv):
        mm, ckpt = ctx.saved_tensors
        n, nsteps, dt, eps, G, ckpt_every = ctx.cfg
        dev = mm.device
        lx = (gx.detach().contiguous().clone() if gx is not None
              else torch.zeros((n, 3), dtype=torch.float32, device=dev))
        lv = (gv.detach().contiguous().clone() if gv is not None
              else torch.zeros((n, 3), dtype=torch.float32, device=dev))
        lm = torch.empty(n, dtype=torch.float32, device=dev)
        work = torch.empty(_lib.lf_work_floats(n, ckpt_every), dtype=torch.float32, device=dev)
        _lib.lf_backward(n, mm, ckpt, nsteps, dt, lx, lv, lm, work, eps=eps, G=G,
                         ckpt_every=ckpt_every, stream=torch.cuda.current_stream(dev))
        return lx, lv, lm, None, None, None, None, None


def leapfrog(x0, v0, m, nsteps: int, dt: float, eps: float, G: float = 1.0, ckpt_every: int = 8):
    """Differentiable KDK leapfrog; returns (x(T), v(T))."""
    return LeapfrogFunction.apply(x0, v0, m, int(nsteps), float(dt), float(eps), float(G),
                                  int(ckpt_every))
