"""Writes tests/golden/adjoint_al120_20k.npz: FP64 oracle gradients of the
full-size differentiated workload, for the GPU adjoint's parity test.

Workload: one parameter set of the 120-neuron antennal-lobe network with a
dense 120 x 120 weight matrix plus the LN -> PN GABA_B block
(``netgen.differentiated(n_sets=1)``), from rest, 20,000 RK4 steps of
dt = 0.01 ms, V recorded every step.  The loss is the workload's mean-square
trace loss over the 90 projection neurons,
  L(theta) = sum_{n=1..T} sum_{p in PN} (V_p(t_n; theta) - V*_p(t_n))^2 / (T 90),
at the starting parameters theta0, with the target traces V* integrated at
the hidden parameters theta* (both by the oracle).

Stored (all from the oracle, FP64):
  loss          L(theta0)
  gw, gp, gy0   the oracle's discrete adjoint of L (checkpoints every 1,000
                steps), dL/dV = 2 (V - V*) / (T 90) on the PN columns
  fd            central differences of L on 10 coordinates (4 nonzero and 2
                zero weights, 4 maximal conductances) for the step ladder
                h = H0 max(1, |x|) x 4^j, j = 0..3 (H0 = 1e-6): fd[j, c].
                At the smallest steps the differences carry the rounding
                noise of the FP64 trajectory divided by h; at the largest,
                truncation error O(h^2).  The agreement of neighbouring
                rungs measures both.

Run from the repository root:  python tests/golden/make_adjoint_al120.py
(about 6 minutes on 8 cores).
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NSTEPS = 20_000
STRIDE = 1
CKPT = 1000
N_PN = 90
COORD_SEED = 5101
H0 = 1e-6
LADDER = (1.0, 4.0, 16.0, 64.0)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_al120_20k.npz")


def workload():
    """(hidden, start): the hidden parameters and the starting point."""
    from paper_1906_03958_gb300 import netgen as ng
    return ng.differentiated(n_sets=1)


def target_traces():
    """V* [T, N]: the oracle's trajectory at the hidden parameters."""
    import oracle
    hidden, _ = workload()
    _, rec = oracle.integrate(hidden, oracle.rest_state(hidden), NSTEPS, rec_stride=STRIDE)
    return rec[: NSTEPS // STRIDE]


def loss_of(rec, vstar) -> float:
    return float(np.sum((rec[:, :N_PN] - vstar[:, :N_PN]) ** 2) / (rec.shape[0] * N_PN))


def loss_gradient(rec, vstar) -> np.ndarray:
    """dL/dV [T, N] of the mean-square PN trace loss."""
    g = np.zeros_like(rec, dtype=np.float64)
    g[:, :N_PN] = 2.0 * (rec[:, :N_PN] - vstar[:, :N_PN]) / (rec.shape[0] * N_PN)
    return g


def coordinates(spec):
    rng = np.random.default_rng(COORD_SEED)
    w = np.asarray(spec.weight)
    ks = list(rng.choice(np.nonzero(w != 0)[0], 4, replace=False)) + \
        list(rng.choice(np.nonzero(w == 0)[0], 2, replace=False))
    # (neuron type, column): PN gNa, PN gK, LN gL, LN gKL
    ps = [(0, 1), (0, 2), (1, 3), (1, 7)]
    return [int(k) for k in ks], ps


def _loss(args):
    kind, idx, delta, vstar = args
    import oracle
    _, spec = workload()
    net = oracle.OracleNet(spec)
    if kind == "w":
        net.w[idx] += delta
    elif kind == "p":
        net.nparams.reshape(-1, 9)[idx] += delta
    _, rec = oracle.integrate(net, oracle.rest_state(net), NSTEPS, rec_stride=STRIDE)
    return loss_of(rec[: NSTEPS // STRIDE], vstar)


def main():
    import oracle
    oracle.build()
    _, spec = workload()
    vstar = target_traces()
    ks, ps = coordinates(spec)
    P = np.asarray(spec.neuron_params, np.float64).reshape(-1, 9)
    jobs, steps = [], []
    for kind, idx, x in [("w", k, float(spec.weight[k])) for k in ks] + [("p", p, float(P[p])) for p in ps]:
        h = H0 * max(1.0, abs(x))
        steps.append(h)
        for mult in LADDER:
            jobs += [(kind, idx, mult * h, vstar), (kind, idx, -mult * h, vstar)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_loss, jobs)
        y0 = oracle.rest_state(spec)
        _, rec = oracle.integrate(spec, y0, NSTEPS, rec_stride=STRIDE)
        rec = rec[: NSTEPS // STRIDE]
        gy, gw, gp = oracle.adjoint(spec, y0, NSTEPS, loss_gradient(rec, vstar), STRIDE, ckpt=CKPT)
    res = np.array(res).reshape(len(steps), len(LADDER), 2)  # coordinate, rung, (+, -)
    h = np.array(steps)[:, None] * np.array(LADDER)[None, :]
    fd = ((res[:, :, 0] - res[:, :, 1]) / (2 * h)).T  # [rung, coordinate]
    np.savez_compressed(
        OUT, loss=loss_of(rec, vstar), gw=gw, gp=gp.reshape(-1, 9), gy0=gy[: 4 * spec.n_neurons], fd=fd,
        fd_h=h.T, fd_w_index=np.array(ks), fd_p_index=np.array(ps), nsteps=NSTEPS, stride=STRIDE, ckpt=CKPT,
        n_pn=N_PN, coord_seed=COORD_SEED)
    for i in range(fd.shape[1]):
        adj = gw[ks[i]] if i < len(ks) else gp.reshape(-1, 9)[ps[i - len(ks)]]
        print(f"coord {i}: adjoint {adj: .9e}  fd " + " ".join(f"{x: .9e}" for x in fd[:, i]))
    print("loss", loss_of(rec, vstar), "wrote", OUT)


if __name__ == "__main__":
    main()
