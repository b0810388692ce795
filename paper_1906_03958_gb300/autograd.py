"""torch.autograd bridge: membrane-potential traces as a differentiable
function of the synaptic weights and the neuron-type table.

Forward runs ``psst_integrate`` (recording V every ``rec_stride`` steps of
the network); backward runs the discrete adjoint ``psst_adjoint`` of the
network's method (RK4, forward Euler or its tableau) from the same starting
state, with the weights and neuron table of that forward.  Both are CUDA
kernels of the library.
"""
from __future__ import annotations

import torch


class PsstTrace(torch.autograd.Function):
    """V frames [F, N] of the next ``n_steps`` steps of ``net``.

    ``weight`` [S] and ``neuron_params`` [n_types, 9] are float32 CUDA
    tensors written into the network before integrating; gradients flow back
    to both.  The network's state advances by ``n_steps`` (as after
    psst_integrate).

    Backward differentiates exactly the span its forward integrated, with
    the tables that forward used, however many other trace calls ran in
    between: when the network still holds checkpoints recorded by this
    forward (``net.record_checkpoints``; the recorded span starts at this
    forward's step and the tables were not written since), the adjoint uses
    them; otherwise it sets the saved starting state, step and tables, runs
    the adjoint's own checkpointing pass (every ``ckpt_every`` steps) and
    puts the network's state, step and tables back.

    The starting state of a window is a constant of this function: when
    several windows are chained (each starting where the previous ended),
    the gradient of a later window's output does not flow back through its
    starting state into the earlier windows' weights."""

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
        ctx.save_for_backward(weight, neuron_params)
        ctx.net, ctx.y0, ctx.s0, ctx.n, ctx.ck = net, y0, s0, n_steps, ckpt_every
        ctx.version = net.tables_version
        ctx.pshape = neuron_params.shape
        return out

    @staticmethod
    def backward(ctx, grad_frames):
        net = ctx.net
        weight, neuron_params = ctx.saved_tensors
        info = net.info()
        own = (net.recording_checkpoints and info["ck_start"] == ctx.s0 and info["ck_steps"] == ctx.n
               and net.tables_version == ctx.version)
        if own:
            # the network still holds this forward's checkpoints and tables
            gw, gp, _ = net.adjoint(ctx.n, grad_frames.contiguous(), 0)
            net.status()
            return gw, gp.reshape(ctx.pshape), None, None, None
        y_end = net.get_state().clone()
        s_end = info["steps_done"]
        w_now, p_now = net.tables_source()
        version = net.tables_version
        net.set_weights(weight)
        net.set_neuron_params(neuron_params)
        net.set_state(ctx.y0)
        net.set_step(ctx.s0)
        gw, gp, _ = net.adjoint(ctx.n, grad_frames.contiguous(), ctx.ck)
        net.status()
        net.set_weights(w_now)
        net.set_neuron_params(p_now)
        net.tables_version = version  # the tables hold what they held before this backward
        net.set_state(y_end)
        net.set_step(s_end)
        return gw, gp.reshape(ctx.pshape), None, None, None


def trace(net, weight, neuron_params, n_steps: int, ckpt_every: int = 1000):
    return PsstTrace.apply(weight, neuron_params, net, n_steps, ckpt_every)
