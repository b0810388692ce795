"""Writes tests/golden/adjoint_al120_20k.npz: FP64 oracle gradients of the
full-size differentiated workload, for the GPU adjoint's parity test.

Workload: one parameter set of the 120-neuron antennal-lobe network with a
dense 120 x 120 weight matrix plus the LN -> PN GABA_B block
(``netgen.differentiated(n_sets=1)``, the starting parameters theta0), from
rest, 20,000 RK4 steps of dt = 0.01 ms, V recorded every step.  The
functional is L = sum_f sum_i g[f, i] V_i(frame f) with a seeded g
(standard normal on the 90 projection-neuron columns, zero on the local
neurons, scaled by 1 / (frames x 90), the shape of the mean-square trace
loss's gradient).

Stored (all from the oracle, FP64):
  gw, gp, gy0   the oracle's discrete adjoint (checkpoints every 1,000 steps)
  fd            central differences of L on 10 coordinates (4 nonzero and 2
                zero weights, 4 maximal conductances) for the step ladder
                h = H0 max(1, |x|) x 4^j, j = 0..3 (H0 = 1e-6): fd[j, c].
                At the smallest steps the differences carry the rounding
                noise of the FP64 trajectory (about 1e-13 in L over 20,000
                spiking steps, divided by h); at the largest, truncation
                error O(h^2).  The agreement of neighbouring rungs measures
                both.

Run from the repository root:  python tests/golden/make_adjoint_al120.py
(about 8 minutes on 8 cores).
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
G_SEED = 5100
COORD_SEED = 5101
H0 = 1e-6
LADDER = (1.0, 4.0, 16.0, 64.0)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_al120_20k.npz")


def workload():
    from paper_1906_03958_gb300 import netgen as ng
    _, start = ng.differentiated(n_sets=1)
    return start


def functional_weights(n_neurons: int, n_pn: int = 90) -> np.ndarray:
    g = np.zeros((NSTEPS // STRIDE, n_neurons))
    g[:, :n_pn] = np.random.default_rng(G_SEED).standard_normal((NSTEPS // STRIDE, n_pn))
    return g / (g.shape[0] * n_pn)


def coordinates(spec):
    rng = np.random.default_rng(COORD_SEED)
    w = np.asarray(spec.weight)
    ks = list(rng.choice(np.nonzero(w != 0)[0], 4, replace=False)) + \
        list(rng.choice(np.nonzero(w == 0)[0], 2, replace=False))
    # (neuron type, column): PN gNa, PN gK, LN gL, LN gKL
    ps = [(0, 1), (0, 2), (1, 3), (1, 7)]
    return [int(k) for k in ks], ps


def _loss(args):
    kind, idx, delta = args
    import oracle
    spec = workload()
    net = oracle.OracleNet(spec)
    if kind == "w":
        net.w[idx] += delta
    elif kind == "p":
        net.nparams.reshape(-1, 9)[idx] += delta
    y0 = oracle.rest_state(net)
    _, rec = oracle.integrate(net, y0, NSTEPS, rec_stride=STRIDE)
    g = functional_weights(spec.n_neurons)
    return float(np.sum(rec[: g.shape[0]] * g))


def main():
    import oracle
    oracle.build()
    spec = workload()
    ks, ps = coordinates(spec)
    P = np.asarray(spec.neuron_params, np.float64).reshape(-1, 9)
    jobs, steps = [], []
    for kind, idx, x in [("w", k, float(spec.weight[k])) for k in ks] + [("p", p, float(P[p])) for p in ps]:
        h = H0 * max(1.0, abs(x))
        steps.append(h)
        for mult in LADDER:
            jobs += [(kind, idx, mult * h), (kind, idx, -mult * h)]
    with mp.get_context("spawn").Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        res = pool.map(_loss, jobs)
        g = functional_weights(spec.n_neurons)
        gy, gw, gp = oracle.adjoint(spec, oracle.rest_state(spec), NSTEPS, g, STRIDE, ckpt=CKPT)
    res = np.array(res).reshape(len(steps), len(LADDER), 2)  # coordinate, rung, (+, -)
    h = np.array(steps)[:, None] * np.array(LADDER)[None, :]
    fd = ((res[:, :, 0] - res[:, :, 1]) / (2 * h)).T  # [rung, coordinate]
    np.savez_compressed(
        OUT, gw=gw, gp=gp.reshape(-1, 9), gy0=gy[: 4 * spec.n_neurons], fd=fd, fd_h=h.T,
        fd_w_index=np.array(ks), fd_p_index=np.array(ps), nsteps=NSTEPS, stride=STRIDE, ckpt=CKPT,
        g_seed=G_SEED, coord_seed=COORD_SEED)
    for i in range(fd.shape[1]):
        adj = gw[ks[i]] if i < len(ks) else gp.reshape(-1, 9)[ps[i - len(ks)]]
        print(f"coord {i}: adjoint {adj: .9e}  fd " + " ".join(f"{x: .9e}" for x in fd[:, i]))
    print("wrote", OUT)


if __name__ == "__main__":
    main()
