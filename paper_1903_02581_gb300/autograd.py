"""torch.autograd.Function over the adjoint of libhom (hom_backward).

``BunchingProbability.apply(h, w, delay, prop, nsteps, K)`` returns the
bunching probability of every simulation after ``nsteps`` Strang steps as a
tensor; its backward multiplies the incoming gradient by dP_b/d(h, w, delay)
computed by the adjoint split-step in the CUDA library.  The QPC height h,
width w and the delay (centre shift of the second packet) are per-simulation
tensors of shape [batch].  The forward sets the simulation parameters and
re-initialises the packets with the delay applied, so every call starts from
the packets of the propagator's workload.
"""

from __future__ import annotations

import copy

import torch

from . import binding as H


class BunchingProbability(torch.autograd.Function):
    @staticmethod
    def forward(ctx, h, w, delay, prop: "H.Propagator", nsteps: int, K: int):
        hb, wb, db = (t.detach().double().cpu().tolist() for t in (h, w, delay))
        for b, s in enumerate(prop.w["sims"]):
            H.hom_set_sim_params(prop.ctx, b, hb[b], wb[b], s["lam"])
            beta = copy.deepcopy(s["beta"])
            beta["x0"] = beta["x0"] + db[b]
            H.hom_init_packets(prop.ctx, b, H.make_packet(s["alpha"]), H.make_packet(beta), s["exch"])
        loss, grad = prop.backward(nsteps, K)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=torch.float64))
        return torch.as_tensor(loss, dtype=torch.float64, device=h.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        g = gout.detach().double().cpu()[:, None] * grad
        dev = gout.device
        return g[:, 0].to(dev), g[:, 1].to(dev), g[:, 2].to(dev), None, None, None
