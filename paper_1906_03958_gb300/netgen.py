"""Seeded synthetic network generators.

This module only draws random numbers and assembles arrays: it holds none of
the integration arithmetic, so both the CUDA library and the FP64 oracle can
be fed from it.  Every array is produced in the exact dtype the C interface
takes (float32 parameters and weights, int32/int64 indices), so the oracle
widens the very same values to float64.

Networks follow the paper's vectorised layout (Sec. "Brain simulations as
computational graphs", the reorganised state X' = [V, m, h, n]): neurons are
indexed globally across the batch, and synapses are stored sparsely (Sec.
"Circumventing memory constraints", item 1) as CSR rows keyed by the
postsynaptic neuron, with the presynaptic index local to its network.

Model constants that the paper leaves to textbooks (the squid-axon HH set in
the modern -65 mV convention, kinetic synapses with a sigmoidal transmitter)
are per-type *parameter tables* here, i.e. inputs, not code.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Column order of the neuron-type table (one row per neuron type).
NEURON_PARAM_NAMES = ("C", "gNa", "gK", "gL", "ENa", "EK", "EL", "gKL", "EKL")
# Column order of the synapse-type table (one row per synapse type).
# kind 0: first-order gate r,  dr/dt = a T (1 - r) - b r,  G = r
# kind 1: second-order pair r,s (slow GABA_B), dr/dt = a T (1-r) - b r,
#         ds/dt = K3 r - K4 s,  G = s^4 / (s^4 + Kd)
SYN_PARAM_NAMES = ("kind", "a", "b", "K3", "K4", "Kd", "E", "Vp", "Kp")

HH = dict(C=1.0, gNa=120.0, gK=36.0, gL=0.3, ENa=50.0, EK=-77.0, EL=-54.387,
          gKL=0.0, EKL=-95.0)
# Antennal-lobe neuron types (project-defined; the paper cites the model only).
PN = dict(HH, gKL=0.05)
LN = dict(HH, gNa=60.0, gKL=0.02)

ACH = dict(kind=0, a=1.1, b=0.19, K3=0.0, K4=0.0, Kd=0.0, E=0.0, Vp=2.0, Kp=5.0)
GABA_A = dict(kind=0, a=5.0, b=0.18, K3=0.0, K4=0.0, Kd=0.0, E=-80.0, Vp=2.0, Kp=5.0)
GABA_B = dict(kind=1, a=0.09, b=0.0012, K3=0.18, K4=0.034, Kd=100.0, E=-95.0,
              Vp=2.0, Kp=5.0)

DT = 0.01  # ms


def neuron_table(*types: dict) -> np.ndarray:
    return np.array([[t[k] for k in NEURON_PARAM_NAMES] for t in types], np.float32)


def synapse_table(*types: dict) -> np.ndarray:
    return np.array([[t[k] for k in SYN_PARAM_NAMES] for t in types], np.float32)


@dataclass
class NetworkSpec:
    """A batch of independent networks in the layout the C interface takes."""

    net_neuron_off: np.ndarray          # int32 [n_nets+1]
    neuron_type: np.ndarray             # int32 [N]
    neuron_params: np.ndarray           # float32 [n_ntypes, 9]
    row_ptr: np.ndarray                 # int64 [N+1], CSR rows = postsynaptic neuron
    pre: np.ndarray                     # int32 [S], presynaptic index local to the net
    weight: np.ndarray                  # float32 [S], mS/cm^2
    syn_type: np.ndarray                # int32 [S]
    syn_params: np.ndarray              # float32 [n_stypes, 9]
    i_const: np.ndarray                 # float32 [N], uA/cm^2
    pulse_amp: np.ndarray               # float32 [N], uA/cm^2 while the pulse is on
    pulse_on: np.ndarray                # int64 [n_nets], first step of the pulse
    pulse_off: np.ndarray               # int64 [n_nets], first step after the pulse
    noise_seed: int = 0
    noise_thresh: int = 0               # event if (philox word0 >> 8) < noise_thresh
    noise_amp: float = 0.0              # uA/cm^2 added for one step per event
    dt: float = DT
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_nets(self) -> int:
        return len(self.net_neuron_off) - 1

    @property
    def n_neurons(self) -> int:
        return int(self.net_neuron_off[-1])

    @property
    def n_synapses(self) -> int:
        return int(self.row_ptr[-1])

    def net_sizes(self) -> np.ndarray:
        return np.diff(self.net_neuron_off)

    def net_synapses(self) -> np.ndarray:
        return self.row_ptr[self.net_neuron_off[1:]] - self.row_ptr[self.net_neuron_off[:-1]]

    def subset(self, nets) -> "NetworkSpec":
        """The networks with the given indices, as a batch of their own."""
        nets = np.asarray(nets, dtype=np.int64)
        parts = [_net_arrays(self, int(b)) for b in nets]
        return _concat(parts, self.neuron_params, self.syn_params,
                       self.pulse_on[nets], self.pulse_off[nets], self.noise_seed,
                       self.noise_thresh, self.noise_amp, self.dt, self.name + "[subset]")


def _net_arrays(spec: NetworkSpec, b: int) -> dict:
    n0, n1 = int(spec.net_neuron_off[b]), int(spec.net_neuron_off[b + 1])
    s0, s1 = int(spec.row_ptr[n0]), int(spec.row_ptr[n1])
    return dict(neuron_type=spec.neuron_type[n0:n1],
                row_ptr=spec.row_ptr[n0:n1 + 1] - s0,
                pre=spec.pre[s0:s1], weight=spec.weight[s0:s1],
                syn_type=spec.syn_type[s0:s1], i_const=spec.i_const[n0:n1],
                pulse_amp=spec.pulse_amp[n0:n1])


def _concat(parts, ntab, stab, pulse_on, pulse_off, noise_seed, noise_thresh,
            noise_amp, dt, name) -> NetworkSpec:
    sizes = np.array([len(p["neuron_type"]) for p in parts], np.int64)
    noff = np.zeros(len(parts) + 1, np.int64)
    noff[1:] = np.cumsum(sizes)
    row_parts, base = [np.zeros(1, np.int64)], 0
    for p in parts:
        row_parts.append(p["row_ptr"][1:] + base)
        base += int(p["row_ptr"][-1])
    cat = lambda k, dt_: (np.concatenate([p[k] for p in parts]).astype(dt_)
                          if parts else np.zeros(0, dt_))
    return NetworkSpec(
        net_neuron_off=noff.astype(np.int32),
        neuron_type=cat("neuron_type", np.int32),
        neuron_params=np.asarray(ntab, np.float32),
        row_ptr=np.concatenate(row_parts).astype(np.int64),
        pre=cat("pre", np.int32), weight=cat("weight", np.float32),
        syn_type=cat("syn_type", np.int32), syn_params=np.asarray(stab, np.float32),
        i_const=cat("i_const", np.float32), pulse_amp=cat("pulse_amp", np.float32),
        pulse_on=np.asarray(pulse_on, np.int64), pulse_off=np.asarray(pulse_off, np.int64),
        noise_seed=int(noise_seed), noise_thresh=int(noise_thresh),
        noise_amp=float(noise_amp), dt=float(dt), name=name)


def _rows_from_edges(n: int, post: np.ndarray, pre: np.ndarray, w: np.ndarray,
                     stype: np.ndarray) -> dict:
    """CSR by postsynaptic row; within a row ordered by (pre, type)."""
    order = np.lexsort((stype, pre, post))
    post, pre, w, stype = post[order], pre[order], w[order], stype[order]
    row_ptr = np.zeros(n + 1, np.int64)
    np.add.at(row_ptr, post + 1, 1)
    return dict(row_ptr=np.cumsum(row_ptr), pre=pre.astype(np.int32),
                weight=w.astype(np.float32), syn_type=stype.astype(np.int32))


def _random_pairs(rng, n_post_idx, n_pre_idx, p, allow_self=False):
    """Each ordered pair (post, pre) independently with probability p."""
    mask = rng.random((len(n_post_idx), len(n_pre_idx))) < p
    if not allow_self:
        same = n_post_idx[:, None] == n_pre_idx[None, :]
        mask &= ~same
    ii, jj = np.nonzero(mask)
    return n_post_idx[ii], n_pre_idx[jj]


def single_network(neuron_type, i_const, post, pre, w, stype, ntab, stab,
                   pulse_amp=None, pulse_on=0, pulse_off=0, noise_seed=0,
                   noise_thresh=0, noise_amp=0.0, dt=DT, name="custom") -> NetworkSpec:
    """Build a one-network batch from explicit edge lists (post, pre local)."""
    n = len(neuron_type)
    rows = _rows_from_edges(n, np.asarray(post, np.int64), np.asarray(pre, np.int64),
                            np.asarray(w, np.float64), np.asarray(stype, np.int64))
    part = dict(neuron_type=np.asarray(neuron_type, np.int32), **rows,
                i_const=np.asarray(i_const, np.float32),
                pulse_amp=(np.zeros(n, np.float32) if pulse_amp is None
                           else np.asarray(pulse_amp, np.float32)))
    return _concat([part], ntab, stab, [pulse_on], [pulse_off], noise_seed,
                   noise_thresh, noise_amp, dt, name)


def concat_specs(specs) -> NetworkSpec:
    """Batch several single- or multi-network specs that share type tables."""
    parts, on, off = [], [], []
    for s in specs:
        for b in range(s.n_nets):
            parts.append(_net_arrays(s, b))
        on.extend(s.pulse_on.tolist())
        off.extend(s.pulse_off.tolist())
    s0 = specs[0]
    return _concat(parts, s0.neuron_params, s0.syn_params, on, off, s0.noise_seed,
                   s0.noise_thresh, s0.noise_amp, s0.dt, "+".join(s.name for s in specs))


# --------------------------------------------------------------------------
# The five workloads (sizes and distributions as stated for each).
# --------------------------------------------------------------------------

def plain20(seed: int = 1001, weight_scale: float = 1.0) -> NetworkSpec:
    """20 HH neurons, ordered pairs i != j with p = 0.5, excitatory first-order
    synapses with w ~ U[0, 0.5] mS/cm^2 (times ``weight_scale``), constant
    inputs I ~ U[0, 10] uA/cm^2."""
    rng = np.random.default_rng(seed)
    n = 20
    idx = np.arange(n)
    post, pre = _random_pairs(rng, idx, idx, 0.5)
    w = rng.uniform(0.0, 0.5, len(post)) * weight_scale
    i_const = rng.uniform(0.0, 10.0, n)
    return single_network(np.zeros(n), i_const, post, pre, w, np.zeros(len(post)),
                          neuron_table(HH), synapse_table(ACH),
                          name=f"plain20(seed={seed},wscale={weight_scale})")


def independent(n_neurons: int, seed: int = 1006, n_nets: int = 1, rate_hz: float = 0.0,
                noise_amp: float = 10.0, pulse: bool = True) -> NetworkSpec:
    """n_neurons uncoupled HH neurons (no synapses), the independent ODE systems
    of the paper's Fig. 2b benchmark: I ~ U[0, 10] uA/cm^2, optionally a
    10 uA/cm^2 pulse to every neuron from 20 to 150 ms and Philox shot noise
    at ``rate_hz``, split into ``n_nets`` networks of about equal size."""
    rng = np.random.default_rng(seed)
    n = int(n_neurons)
    cuts = np.linspace(0, n, n_nets + 1).round().astype(np.int64)
    dt = DT
    thresh = int(round(rate_hz * 1e-3 * dt * (1 << 24))) if rate_hz > 0 else 0
    return NetworkSpec(
        net_neuron_off=cuts.astype(np.int32),
        neuron_type=np.zeros(n, np.int32),
        neuron_params=np.asarray(neuron_table(HH), np.float32),
        row_ptr=np.zeros(n + 1, np.int64),
        pre=np.zeros(0, np.int32), weight=np.zeros(0, np.float32), syn_type=np.zeros(0, np.int32),
        syn_params=np.asarray(synapse_table(ACH), np.float32),
        i_const=rng.uniform(0.0, 10.0, n).astype(np.float32),
        pulse_amp=np.full(n, 10.0 if pulse else 0.0, np.float32),
        pulse_on=np.full(n_nets, int(round(20.0 / dt)), np.int64),
        pulse_off=np.full(n_nets, int(round(150.0 / dt)), np.int64),
        noise_seed=seed, noise_thresh=thresh, noise_amp=float(noise_amp) if thresh else 0.0,
        dt=dt, name=f"independent(n={n},nets={n_nets},seed={seed})")


def antennal_lobe(seed: int = 1002, n_pn: int = 90, n_ln: int = 30, p: float = 0.5,
                  odor_on_ms: float = 100.0, odor_off_ms: float = 600.0,
                  odor_frac: float = 1.0 / 3.0, odor_amp: float = 100.0,
                  w_max=(0.3, 0.6, 0.3), dt: float = DT) -> NetworkSpec:
    """90 PN + 30 LN.  PN->{PN,LN} cholinergic, LN->{PN,LN} GABA_A, LN->PN
    GABA_B (drawn independently), each type pair with probability p and
    weights U[0, w_max] mS/cm^2.  Odor: a current pulse of
    odor_amp * U[0.5, 1] to a random third of the neurons between
    odor_on_ms and odor_off_ms; background I ~ U[0, 5] uA/cm^2."""
    rng = np.random.default_rng(seed)
    n = n_pn + n_ln
    pn, ln = np.arange(n_pn), np.arange(n_pn, n)
    ntype = np.r_[np.zeros(n_pn), np.ones(n_ln)]
    posts, pres, ws, ts = [], [], [], []
    for (post_set, pre_set, t, wm) in ((np.arange(n), pn, 0, w_max[0]),
                                       (np.arange(n), ln, 1, w_max[1]),
                                       (pn, ln, 2, w_max[2])):
        po, pr = _random_pairs(rng, post_set, pre_set, p)
        posts.append(po), pres.append(pr)
        ws.append(rng.uniform(0.0, wm, len(po))), ts.append(np.full(len(po), t))
    i_const = rng.uniform(0.0, 5.0, n)
    stim = rng.permutation(n)[: int(round(odor_frac * n))]
    amp = np.zeros(n)
    amp[stim] = odor_amp * rng.uniform(0.5, 1.0, len(stim))
    return single_network(ntype, i_const, np.concatenate(posts), np.concatenate(pres),
                          np.concatenate(ws), np.concatenate(ts),
                          neuron_table(PN, LN), synapse_table(ACH, GABA_A, GABA_B),
                          pulse_amp=amp, pulse_on=int(round(odor_on_ms / dt)),
                          pulse_off=int(round(odor_off_ms / dt)), dt=dt,
                          name=f"antennal_lobe(seed={seed})")


def sparse_large(seed: int = 1003, n_e: int = 8000, n_i: int = 2000, p: float = 0.02,
                 rate_hz: float = 20.0, noise_amp: float = 20.0, dt: float = DT) -> NetworkSpec:
    """8k excitatory + 2k inhibitory HH neurons, pairs with p = 0.02, weights
    lognormal(mu=-1, sigma=0.5) mS/cm^2; E synapses first order (E = 0),
    I synapses GABA_A (E = -80); shot noise of noise_amp for one step with
    probability rate*dt per neuron-step; I_const ~ U[0, 10]."""
    rng = np.random.default_rng(seed)
    n = n_e + n_i
    # draw per-row presynaptic sets with the same per-pair probability, row by
    # row, to keep memory at O(S) instead of O(n^2)
    counts = rng.binomial(n - 1, p, n)
    post = np.repeat(np.arange(n), counts)
    pre = np.empty(post.size, np.int64)
    pos = 0
    for i in range(n):
        c = counts[i]
        sel = rng.choice(n - 1, size=c, replace=False)
        sel[sel >= i] += 1
        pre[pos:pos + c] = sel
        pos += c
    w = rng.lognormal(-1.0, 0.5, post.size)
    stype = (pre >= n_e).astype(np.int64)
    i_const = rng.uniform(0.0, 10.0, n)
    thresh = int(round(rate_hz * 1e-3 * dt * (1 << 24)))
    return single_network(np.zeros(n), i_const, post, pre, w, stype,
                          neuron_table(HH), synapse_table(ACH, GABA_A),
                          noise_seed=seed, noise_thresh=thresh, noise_amp=noise_amp,
                          dt=dt, name=f"sparse_large(seed={seed},n={n})")


def _batched_one(b: int, base_seed: int, n_min: int, n_max: int, dt: float) -> tuple:
    rng = np.random.default_rng(base_seed + b)
    n = int(rng.integers(n_min, n_max + 1))
    p = rng.uniform(0.1, 0.5)
    n_e = int(round(0.8 * n))
    idx = np.arange(n)
    post, pre = _random_pairs(rng, idx, idx, p)
    w = rng.uniform(0.0, 0.5, post.size) * (10.0 / (n * p))
    stype = (pre >= n_e).astype(np.int64)
    i_const = rng.uniform(0.0, 10.0, n)
    amp = np.where(rng.random(n) < 1.0 / 3.0, rng.uniform(0.0, 10.0, n), 0.0)
    on = int(rng.integers(0, int(round(100.0 / dt))))
    off = on + int(rng.integers(int(round(20.0 / dt)), int(round(100.0 / dt))))
    rows = _rows_from_edges(n, post, pre, w, stype)
    part = dict(neuron_type=np.zeros(n, np.int32), **rows,
                i_const=i_const.astype(np.float32), pulse_amp=amp.astype(np.float32))
    return part, on, off


def batched(n_nets: int = 4096, base_seed: int = 4000, n_min: int = 20, n_max: int = 300,
            dt: float = DT) -> NetworkSpec:
    """``n_nets`` independent networks, net b drawn from seed base_seed + b:
    N ~ U{n_min..n_max}, 80/20 E/I, pair probability p ~ U[0.1, 0.5],
    w ~ U[0, 0.5] * 10 / (N p), I_const ~ U[0, 10], and a random pulse of
    U[0, 10] uA/cm^2 to about a third of the neurons, starting in the first
    100 ms and lasting 20-100 ms."""
    parts, on, off = [], [], []
    for b in range(n_nets):
        part, o1, o2 = _batched_one(b, base_seed, n_min, n_max, dt)
        parts.append(part), on.append(o1), off.append(o2)
    return _concat(parts, neuron_table(HH), synapse_table(ACH, GABA_A), on, off,
                   0, 0, 0.0, dt, f"batched(n_nets={n_nets},N={n_min}..{n_max})")


def perturbed_params(spec: NetworkSpec, seed: int, rel: float = 0.2) -> NetworkSpec:
    """Same topology, weights and conductances scaled by (1 + rel U[-1, 1])."""
    rng = np.random.default_rng(seed)
    out = NetworkSpec(**{k: getattr(spec, k) for k in spec.__dataclass_fields__})
    out.weight = (spec.weight * (1.0 + rel * rng.uniform(-1, 1, spec.weight.size))).astype(np.float32)
    tab = spec.neuron_params.copy()
    for col in (1, 2, 3, 7):  # gNa, gK, gL, gKL
        tab[:, col] *= (1.0 + rel * rng.uniform(-1, 1, tab.shape[0]))
    out.neuron_params = tab.astype(np.float32)
    out.name = spec.name + f"[perturbed seed={seed}]"
    return out


def differentiated(n_sets: int = 64, seed: int = 5000, n_pn: int = 90, n_ln: int = 30, p: float = 0.5,
                   w_max=(0.3, 0.6, 0.3), rel: float = 0.2, dt: float = DT):
    """Parameter sets of the antennal-lobe network with dense weight
    matrices, for gradients with respect to every entry.

    Every ordered pair (post i, pre j), self pairs included, carries a
    synapse of the presynaptic neuron's fast type (cholinergic from PNs,
    GABA_A from LNs) and every (PN post, LN pre) pair a GABA_B synapse; a
    pair outside the random p-mask has weight 0.  Set q has its own neuron
    types (2q: PN, 2q+1: LN).  Returns (hidden, start): the hidden parameters
    theta* (drawn from ``seed``) and the starting point
    theta0 = theta* (1 + rel U[-1, 1]) (``seed + 1``), as two batches with the
    same topology, odor pulse and inputs."""
    rng = np.random.default_rng(seed)
    n = n_pn + n_ln
    pn, ln = np.arange(n_pn), np.arange(n_pn, n)
    parts, on, off = [], [], []
    tabs = []
    for q in range(n_sets):
        post_all = np.repeat(np.arange(n), n)
        pre_all = np.tile(np.arange(n), n)
        fast_t = np.where(pre_all < n_pn, 0, 1)
        w_fast = np.where(rng.random(n * n) < p, rng.uniform(0, 1, n * n), 0.0)
        w_fast *= np.where(pre_all < n_pn, w_max[0], w_max[1])
        w_fast[post_all == pre_all] = 0.0
        bpost = np.repeat(pn, n_ln)
        bpre = np.tile(ln, n_pn)
        w_b = np.where(rng.random(bpost.size) < p, rng.uniform(0, w_max[2], bpost.size), 0.0)
        post = np.concatenate([post_all, bpost])
        pre = np.concatenate([pre_all, bpre])
        w = np.concatenate([w_fast, w_b])
        st = np.concatenate([fast_t, np.full(bpost.size, 2)])
        rows = _rows_from_edges(n, post, pre, w, st)
        ntype = np.r_[np.zeros(n_pn), np.ones(n_ln)] + 2 * q
        i_const = rng.uniform(0.0, 5.0, n)
        amp = np.zeros(n)
        stim = rng.permutation(n)[: n // 3]
        amp[stim] = 10.0 * rng.uniform(0.5, 1.0, stim.size)
        parts.append(dict(neuron_type=ntype.astype(np.int32), **rows, i_const=i_const.astype(np.float32),
                          pulse_amp=amp.astype(np.float32)))
        on.append(int(round(20.0 / dt)))
        off.append(int(round(150.0 / dt)))
        tabs.extend([PN, LN])
    hidden = _concat(parts, neuron_table(*tabs), synapse_table(ACH, GABA_A, GABA_B), on, off, 0, 0, 0.0, dt,
                     f"differentiated(n_sets={n_sets},seed={seed})")
    start = perturbed_params(hidden, seed + 1, rel)
    # a perturbed absent synapse stays absent
    start.weight = np.where(hidden.weight == 0, 0.0, start.weight).astype(np.float32)
    return hidden, start
