"""torch.autograd bridge: membrane-potential traces as a differentiable
function of the synaptic weights and the neuron-type table.

Forward runs ``psst_integrate`` (recording V every ``rec_stride`` steps of
the network); backward runs the discrete adjoint ``psst_adjoint`` of the
network's method (RK4 or forward Euler) from the same starting state.  Both are CUDA kernels of the library.
"""
from __future__ import annotations

import torch


class PsstTrace(torch.autograd.Function):
    """V frames [F, N] of the next ``n_steps`` steps of ``net``.

    ``weight`` [S] and ``neuron_params`` [n_types, 9] are float32 CUDA
    tensors written into the network before integrating; gradients flow back
    to both.  The network's state advances by ``n_steps`` (as after
    psst_integrate).  If the network records checkpoints
    (``net.record_checkpoints``), backward differentiates the recorded span
    directly; otherwise it re-runs the adjoint's own checkpointing pass from
    the saved starting state."""

    @staticmethod
    def forward(ctx, weight, neuron_params, net, n_steps: int, ckpt_every: int = 1000):
        net.set_weights(weight)
        net.set_neuron_params(neuron_params)
        info = net.info()
        s0 = info["steps_done"]
        y0 = net.get_state().clone()
        stride = net.rec_stride
        frames = (s0 + n_steps) // stride - s0 // stride if stride > 0 else 0
        if frames > net._cap:
            raise ValueError("the record ring holds fewer frames than the span produces")
        net.integrate(n_steps)
        out = torch.empty((max(frames, 0), net.N), dtype=torch.float32, device=y0.device)
        if frames:
            rec = net.read_record(out=torch.empty((min(net.info()["rec_frames"], net._cap), net.N),
                                                  dtype=torch.float32, device=y0.device))
            out.copy_(rec[-frames:])
        ctx.net, ctx.y0, ctx.s0, ctx.n, ctx.ck = net, y0, s0, n_steps, ckpt_every
        ctx.pshape = neuron_params.shape
        return out

    @staticmethod
    def backward(ctx, grad_frames):
        net = ctx.net
        if net.recording_checkpoints:
            # the forward call recorded its checkpoints: differentiate its span directly
            gw, gp, _ = net.adjoint(ctx.n, grad_frames.contiguous(), 0)
            net.status()
            return gw, gp.reshape(ctx.pshape), None, None, None
        y_end = net.get_state().clone()
        s_end = net.info()["steps_done"]
        net.set_state(ctx.y0)
        net.set_step(ctx.s0)
        gw, gp, _ = net.adjoint(ctx.n, grad_frames.contiguous(), ctx.ck)
        net.status()
        net.set_state(y_end)
        net.set_step(s_end)
        return gw, gp.reshape(ctx.pshape), None, None, None


def trace(net, weight, neuron_params, n_steps: int, ckpt_every: int = 1000):
    return PsstTrace.apply(weight, neuron_params, net, n_steps, ckpt_every)
