"""torch.autograd.Function over the library's adjoint (pic_adjoint_forward / _backward).

Marshalling only: the forward run, the checkpoints, the recomputation and every transposed pass run
in the CUDA library. ``WPerp.apply(h, nsteps, every, psi_e, psi_b, *fields0)`` sets the correction
coefficients (Sec. 2) and, when given, the initial fields of the run held by handle ``h``, advances
it ``nsteps`` steps and returns the final transverse field energy W_perp as a 0-d FP64 tensor;
``backward`` returns its gradients with respect to ``psi_e``, ``psi_b`` (5 coefficients each, FP64
CPU tensors) and the six initial field tensors (device tensors of the run's precision, shape
(nz, ny, nx)). The handle must hold the run's initial particle state when ``apply`` is called
(``pic_create`` with ``init_beam`` and ``track_ids = 1``, or an import without explicit ids).
"""
from __future__ import annotations

import torch

from . import binding as B


class WPerp(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, nsteps, every, psi_e, psi_b, *fields0):
        B.pic_set_correction_stencil(h, psi_e.detach().cpu().tolist(), psi_b.detach().cpu().tolist())
        if fields0:
            assert len(fields0) == 6
            names = ("ex", "ey", "ez", "bx", "by", "bz")
            st = B.make_state(B.PIC_DEVICE, fields={n: f.detach().contiguous() for n, f in zip(names, fields0)})
            st.np = -1  # keep the particles
            torch.cuda.synchronize()  # the tensors may come from work still queued on another stream
            B.pic_set_state(h, st)
        w = B.pic_adjoint_forward(h, nsteps, every)
        ctx.h = h
        ctx.nfields = len(fields0)
        ctx.like = fields0[0] if fields0 else None
        return torch.tensor(w, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gw):
        gf = None
        if ctx.nfields and any(ctx.needs_input_grad[5:]):
            gf = [torch.empty_like(ctx.like) for _ in range(6)]
        ge, gb = B.pic_adjoint_backward(ctx.h, float(gw), gf)
        ge = torch.tensor(ge, dtype=torch.float64)
        gb = torch.tensor(gb, dtype=torch.float64)
        grads = [None, None, None, ge, gb]
        if ctx.nfields:
            grads += gf if gf is not None else [None] * 6
        return tuple(grads)
