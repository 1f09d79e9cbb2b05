"""``torch.autograd.Function`` over the triples map (t1, t2) -> (X1, X2).

Forward runs ``rtcc3_triples_forward_dev`` (Eqs. A21-A22 with t3 from Eq. 4);
backward runs ``rtcc3_triples_vjp_dev``, the hand-written reverse pass of the
same kernels.  The map is holomorphic; PyTorch's complex autograd works with
conjugate-Wirtinger gradients, so backward conjugates the incoming gradient,
applies the plain transpose u^T J and conjugates the result.  With
u = (lambda1, lambda2 / 2) the (unconjugated) VJP is the triples part of the
lambda residuals (Eqs. A23-A24).
"""
from __future__ import annotations

import torch


class TriplesResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, t1, t2, engine, slot: int = 0, time: float = 0.0):
        if not (t1.is_cuda and t2.is_cuda):
            raise RuntimeError("TriplesResidual runs on the GPU only")
        t1c = t1.detach().to(torch.complex128).contiguous()
        t2c = t2.detach().to(torch.complex128).contiguous()
        x1 = torch.empty_like(t1c)
        x2 = torch.empty_like(t2c)
        stream = torch.cuda.current_stream(t1.device).cuda_stream
        engine.triples_forward_dev(slot, time, t1c.data_ptr(), t2c.data_ptr(), x1.data_ptr(),
                                   x2.data_ptr(), stream)
        ctx.save_for_backward(t1c, t2c)
        ctx.engine, ctx.slot, ctx.time = engine, slot, time
        return x1, x2

    @staticmethod
    def backward(ctx, gx1, gx2):
        t1c, t2c = ctx.saved_tensors
        u1 = (torch.zeros_like(t1c) if gx1 is None else gx1.to(torch.complex128)).conj().resolve_conj().contiguous()
        u2 = (torch.zeros_like(t2c) if gx2 is None else gx2.to(torch.complex128)).conj().resolve_conj().contiguous()
        g1 = torch.empty_like(t1c)
        g2 = torch.empty_like(t2c)
        stream = torch.cuda.current_stream(t1c.device).cuda_stream
        ctx.engine.triples_vjp_dev(ctx.slot, ctx.time, t1c.data_ptr(), t2c.data_ptr(), u1.data_ptr(),
                                   u2.data_ptr(), g1.data_ptr(), g2.data_ptr(), stream)
        return g1.conj().resolve_conj(), g2.conj().resolve_conj(), None, None, None
