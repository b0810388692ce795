#!/usr/bin/env python
"""Throughput benchmark: RK4 integration of coupled HH networks on GB300.

Default workload (the batched form): 4,096 independent networks, sizes
U{20..300}, 80/20 E/I, pair probability U[0.1, 0.5], 200 ms at dt = 0.01 ms
(20,000 RK4 steps), V recorded every 0.1 ms.  One benchmark step integrates
the whole batch for ``--chunk`` RK4 steps (default 2,000 = 20 ms), so 10
steps cover the full 200 ms.  Metric: neuron-RK4-steps per second
(sum over networks of neurons x RK4 steps / time).

Also reported: the single-network forward (the 120-neuron antennal-lobe
network) on the same GPU, the roofline of the dominant kernel, the FP64
oracle on the host cores (bounded sample), an end-to-end number through
the C interface with host buffers, and uncoupled neurons (the independent
ODE systems of the paper's Fig. 2b) with a sweep over their number.

Under torchrun each rank integrates its own batch (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "neuron-RK4-steps/sec FP32 (batched vs single); adjoint grad time / forward time"
UNIT = "neuron-steps/s"

# Algorithmic FP32 operation counts (FMA = 2) per unit and RK4 stage of the
# formulation the kernels evaluate; kept in sync with the CUDA sources.
FLOP_NEURON_STAGE = 80       # HH rates, currents, 4-variable stage update
FLOP_COEF1_STAGE = 16        # per (presynaptic neuron, synapse type): T, r-map update
FLOP_COEF2_STAGE = 20        # extra per (neuron, type) when second-order gates exist
FLOP_SYN1_STAGE = 6          # per-synapse gates, first order: r = P + Q r0, w r (V - E) accumulate
FLOP_SYN2_STAGE = 14         # per-synapse gates, second order: + s map, s^4 / (s^4 + Kd)
FLOP_SYN_PAIR_STAGE = 4      # per-pair gates: A += w G, B += wE G (the gate is gathered)
FLOP_PAIR1_STAGE = 2         # per-pair gates: G = P + Q r0 of a first-order (neuron, type) pair
FLOP_PAIR2_STAGE = 10        # per-pair gates, second order: + s map, s^4 / (s^4 + Kd)
# (per-pair gates: gate maps are updated for the pairs that have synapses only)
FP32_LANES_PER_SM = 128

# Discrete adjoint (psst_adjoint), FP32 FLOP per RK4 step, counted from the
# kernel source: the forward recompute of the segment (synapse: A and B
# sums, 5 per stage; neuron: 80 per stage; every (neuron, type) pair:
# transmitter, r and s slopes and stage values, G, 23 per stage) plus the
# reverse sweep (neuron: stage adjoint, rate derivatives, Jacobian-transpose
# products, nine parameter gradients, ~165 per stage and 8 per step;
# synapse: column sum 4 per stage, weight gradient 4 per stage and 1 per
# step; pair: stage adjoint, transmitter derivative, gate products ~35 per
# stage and 4 per step).
ADJ_FLOP_SYN_STEP = 4 * 5 + 4 * 4 + 4 * 4 + 1          # 53
ADJ_FLOP_NEURON_STEP = 4 * 80 + 4 * 165 + 8             # 988
ADJ_FLOP_PAIR_STEP = 4 * 23 + 4 * 35 + 4                # 236

# Bytes per RK4 step of the large sparse network if its state streamed from
# HBM every step (synapse: gate r read + written 8 B, weight + index 8 B;
# neuron: V, m, h, n read + written 32 B).
STREAM_BYTES_SYN_STEP = 16
STREAM_BYTES_NEURON_STEP = 32


def device_sms() -> int:
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def fp32_peak_tflops(smax_mhz: float) -> float:
    """FP32 FMA-pipe peak of the current device: SMs x 128 lanes x 2 FLOP x
    the maximum SM clock."""
    return device_sms() * FP32_LANES_PER_SM * 2 * smax_mhz * 1e6 / 1e12


def workload_flops_per_step(spec, pair_gates: bool = True) -> float:
    """Algorithmic FLOP per RK4 step of the whole batch, counted for the
    formulation the kernels execute (one gate per (presynaptic neuron, type)
    pair when pair_gates, else one per synapse)."""
    kinds = spec.syn_params[:, 0]
    nt = spec.syn_params.shape[0]
    N = spec.n_neurons
    syn2 = kinds[spec.syn_type] != 0
    n_syn2 = int(syn2.sum())
    n_syn1 = spec.n_synapses - n_syn2
    # networks with second-order synapses pay the extra coefficient work
    net_of_syn = np.searchsorted(spec.row_ptr[spec.net_neuron_off], np.nonzero(syn2)[0], side="right") - 1
    has2 = np.zeros(spec.n_nets, bool)
    has2[np.unique(net_of_syn)] = True
    n_has2 = int(spec.net_sizes()[has2].sum())
    if pair_gates:
        # gate maps and gates of the (presynaptic neuron, type) pairs that have synapses
        net_of_syn = np.searchsorted(spec.row_ptr[spec.net_neuron_off], np.arange(spec.n_synapses),
                                     side="right") - 1
        pre_global = spec.net_neuron_off[net_of_syn].astype(np.int64) + spec.pre
        pairs = np.unique(pre_global * nt + spec.syn_type)
        sec_pairs = int(np.count_nonzero(kinds[pairs % nt]))
        per_stage = (FLOP_NEURON_STAGE * N + FLOP_SYN_PAIR_STAGE * spec.n_synapses
                     + (FLOP_COEF1_STAGE + FLOP_PAIR1_STAGE) * len(pairs)
                     + (FLOP_COEF2_STAGE + FLOP_PAIR2_STAGE) * sec_pairs)
    else:
        per_stage = (FLOP_NEURON_STAGE * N + FLOP_COEF1_STAGE * N * nt + FLOP_COEF2_STAGE * n_has2 * nt
                     + FLOP_SYN1_STAGE * n_syn1 + FLOP_SYN2_STAGE * n_syn2)
    return 4.0 * per_stage


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# Sources that decide each kernel's memory traffic: its own file, the
# shared device headers and the host planner (launch shapes, layouts).
KERNEL_SOURCES = {
    "net_kernel": ("psst_cta.cu", "psst_syn.cuh"),
    "grid_kernel": ("psst_grid.cu", "psst_syn.cuh"),
    "adj_kernel": ("psst_adjoint.cu",),
    "indep_kernel": ("psst_indep.cu",),
}
COMMON_SOURCES = ("psst_device.cuh", "psst_internal.h", "psst_api.cu")


def kernel_source_hash(kernel: str) -> str:
    """Hash of the code of the sources a kernel's traffic depends on (line
    comments and blank lines dropped, so that a comment edit does not
    invalidate a capture)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1906_03958_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES[kernel] + COMMON_SOURCES):
        for line in open(os.path.join(csrc, f), encoding="utf-8"):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def traffic_for(kernel: str, workload: str, steps: int | None = None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources; else None.  An entry captured on a
    launch of fewer steps than the timed one (``captured_steps``) is scaled
    to ``steps`` (its traffic grows in proportion with the steps)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        t = json.load(open(p))
    except Exception:
        return None
    e = t.get(f"{kernel}:{workload}")
    if not e or e.get("source_hash") != kernel_source_hash(kernel):
        return None
    b = e.get("bytes_per_launch")
    if b is not None and steps and e.get("captured_steps"):
        b = b * steps / e["captured_steps"]
    return b


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: PSST_CLOCKS_DIR, else the system temporary directory
        out = os.environ.get("PSST_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_gpu{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------- cpu baseline

def _oracle_job(args):
    spec, nsteps = args
    import oracle
    t = time.perf_counter()
    oracle.integrate(spec, oracle.rest_state(spec), nsteps)
    return time.perf_counter() - t


def cpu_sample(spec, n_nets: int, nsteps: int, seed: int = 0):
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(spec.n_nets, size=min(n_nets, spec.n_nets), replace=False))
    return [spec.subset([int(b)]) for b in idx]


def run_cpu_baseline(sample, nsteps: int, cores: int):
    """FP64 oracle over the sample networks, one process per core (spawn)."""
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    neuron_steps = sum(s.n_neurons for s in sample) * nsteps
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_job, [(s, nsteps) for s in sample], chunksize=1)
    wall = time.perf_counter() - t0
    return neuron_steps / wall, wall


# --------------------------------------------------------------- workloads

def make_workload(name: str, rank: int):
    from paper_1906_03958_gb300 import netgen as ng
    if name == "batched":
        return ng.batched(n_nets=4096, base_seed=4000 + 4096 * rank), \
            "batched: 4096 HH networks, N~U{20..300}, 80/20 E/I, p~U[0.1,0.5], 200 ms, dt 0.01 ms", 20000
    if name == "antennal_lobe":
        return ng.antennal_lobe(seed=1002 + rank), \
            "antennal lobe: 90 PN + 30 LN, ACh/GABA_A/GABA_B, 1000 ms, dt 0.01 ms", 100000
    if name == "plain20":
        return ng.plain20(seed=1001 + rank), "plain: 20 HH neurons, p=0.5, 100 ms, dt 0.01 ms", 10000
    if name == "sparse_large":
        return ng.sparse_large(seed=1003 + rank), \
            "large sparse: 8000 E + 2000 I HH neurons, p=0.02 (~2M synapses), Philox shot noise, 500 ms", 50000
    if name == "differentiated":
        return ng.differentiated(n_sets=64, seed=5000 + 64 * rank)[1], \
            "differentiated forward: 64 antennal-lobe parameter sets, dense 120x120 W + GABA_B, 200 ms", 20000
    raise SystemExit(f"unknown workload {name}")


def reduce_over_ranks(t_local: float, neurons_local: float, device):
    """Job-wide timing under weak scaling: the slowest rank's time and the
    neurons of all ranks (no collective touches the integration itself)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    n = torch.tensor([neurons_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=2000, help="RK4 steps per benchmark step")
    ap.add_argument("--workload", default="batched")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rec-stride", type=int, default=10)
    ap.add_argument("--single-steps", type=int, default=20000)
    ap.add_argument("--cpu-nets", type=int, default=64)
    ap.add_argument("--cpu-steps", type=int, default=300)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=20000)
    ap.add_argument("--sparse-steps", type=int, default=2000)
    ap.add_argument("--autotune", type=int, default=200, help="trial steps per shape (0 = off)")
    ap.add_argument("--graph", type=int, default=1, help="CUDA-graph replay of the launch sequence")
    ap.add_argument("--ckpt-every", type=int, default=1000)
    ap.add_argument("--indep-steps", type=int, default=2000,
                    help="steps of the independent-neuron leg (0 = off)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        return reference_arm(args, rank, world)

    spec, wl_desc, sim_steps = make_workload(args.workload, rank)
    cores = os.cpu_count() or 1
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        # the FP64 oracle on the host cores, before any CUDA work (spawned pool)
        sample = cpu_sample(spec, args.cpu_nets, args.cpu_steps)
        val, wall = run_cpu_baseline(sample, args.cpu_steps, min(cores, len(sample)))
        cpu = {"value": val, "unit": UNIT, "cores": min(cores, len(sample)), "kind": "oracle",
               "sample": f"{len(sample)} networks drawn from the workload, {args.cpu_steps} RK4 steps each, "
                         f"FP64, one process per core; {wall:.1f} s wall"}

    import torch
    from paper_1906_03958_gb300 import psst

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    psst.load()
    frames = args.chunk // args.rec_stride if args.rec_stride else 0
    net = psst.Network(spec, rec_stride=args.rec_stride, rec_capacity=max(frames, 1))
    if args.autotune > 0:
        net.autotune(args.autotune)       # per size class CTA size (setup, not timed)
    if args.graph:
        net.set_graph_mode(True)          # replay the class launches through a CUDA graph
    info = net.info()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        net.integrate(args.chunk)
    net.status()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    barrier()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed launches
    ev0.record(stream)
    for _ in range(args.steps):
        net.integrate(args.chunk)
        launches += net.info()["kernel_launches"]
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()
    net.status()
    ms = ev0.elapsed_time(ev1)
    t_local = ms / 1e3
    if world > 1:
        t_max, total_neurons = reduce_over_ranks(t_local, float(spec.n_neurons), "cuda")
    else:
        t_max, total_neurons = t_local, float(spec.n_neurons)
    value = total_neurons * args.chunk * args.steps / t_max

    # ---- end to end through the C interface with host buffers
    dim = net.dim
    h_state = torch.empty(dim, dtype=torch.float32).pin_memory()
    h_state.copy_(net.get_state().cpu())
    h_rec = torch.empty((max(frames, 1), spec.n_neurons), dtype=torch.float32).pin_memory()
    h_out = torch.empty(dim, dtype=torch.float32).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        net.set_state(h_state)                  # H2D: the step's initial state
        net.integrate(args.chunk)
        net.read_record(out=h_rec.numpy())      # D2H: V frames of the chunk
        net.get_state(out=h_out.numpy())        # D2H: final state
    barrier()
    e2e_t = time.perf_counter() - t0
    e2e_val = spec.n_neurons * args.chunk * args.e2e_steps / e2e_t
    h2d = dim * 4
    d2h = frames * spec.n_neurons * 4 + dim * 4
    net.status()
    net.close()

    # ---- single-network forward on the same GPU (context for "batched vs single")
    single = None
    if rank == 0:
        from paper_1906_03958_gb300 import netgen as ng
        al = ng.antennal_lobe()
        with psst.Network(al) as sn:
            if args.autotune > 0:
                sn.autotune(args.autotune)    # CTA size and gate-table copies (setup, not timed)
            sn.integrate(2000)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sn.integrate(args.single_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            sn.status()
            sms = e0.elapsed_time(e1)
            sn_info = sn.info()
        single = {"workload": "antennal lobe, 120 neurons, one network per launch",
                  "value": al.n_neurons * args.single_steps / (sms / 1e3), "unit": UNIT,
                  "us_per_rk4_step": sms * 1e3 / args.single_steps,
                  "block_threads": sn_info["block_threads"]}

    # ---- independent neurons (the paper's Fig. 2b systems): one thread per
    # neuron, no coupling; throughput, ALU fraction and a sweep over N
    indep = None
    if rank == 0 and args.indep_steps > 0:
        from paper_1906_03958_gb300 import netgen as ng
        peaks = measured_peaks()
        smax = peaks.get("sm_max_mhz", 2070.0)
        peak_tflops = fp32_peak_tflops(smax)

        def timed(spec, nsteps, reps):
            with psst.Network(spec) as inet:
                inet.integrate(min(nsteps, 200))
                torch.cuda.synchronize()
                ms = []
                for _ in range(reps):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    inet.integrate(nsteps)
                    b.record(stream)
                    torch.cuda.synchronize()
                    ms.append(a.elapsed_time(b))
                inet.status()
            return float(np.median(ms))

        n_big = 1 << 22
        big = ng.independent(n_big, rate_hz=20.0)
        ms_big = timed(big, args.indep_steps, 3)
        flop = 4.0 * FLOP_NEURON_STAGE * n_big * args.indep_steps
        sweep = []
        for n_sys in (1_000, 10_000, 100_000, 1_000_000, 4_000_000):
            ms_n = timed(ng.independent(n_sys), 200, 20)
            sweep.append({"n": n_sys, "ms_per_200_steps": ms_n, "neuron_steps_per_s": n_sys * 200 / (ms_n / 1e3)})
        indep = {"workload": f"{n_big} uncoupled HH neurons (I ~ U[0,10], pulse, Philox shot noise), "
                             "one thread per neuron, no barriers",
                 "value": n_big * args.indep_steps / (ms_big / 1e3), "unit": UNIT,
                 "us_per_rk4_step": ms_big * 1e3 / args.indep_steps,
                 "roofline": {"bound": "alu", "achieved": flop / (ms_big / 1e3) / 1e12, "peak": peak_tflops,
                              "unit": "TFLOP/s", "frac": flop / (ms_big / 1e3) / 1e12 / peak_tflops},
                 "fig2b_sweep": {"method": "median of 20 replicates of 200 RK4 steps (the paper's Fig. 2 timing)",
                                 "points": sweep}}

    # ---- the large sparse network (one network over the whole GPU)
    sparse = None
    if rank == 0 and args.sparse_steps > 0:
        from paper_1906_03958_gb300 import netgen as ng
        sp = ng.sparse_large()
        with psst.Network(sp) as sn:
            sn.integrate(200)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sn.integrate(args.sparse_steps)
            e1.record(stream)
            torch.cuda.synchronize()
            sn.status()
            sinfo = sn.info()
            sms = e0.elapsed_time(e1)
        peaks = measured_peaks()
        smax = peaks.get("sm_max_mhz", 2070.0)
        sec = sms / 1e3
        sflop = workload_flops_per_step(sp, sinfo["n_pair_gate_nets"] == 1) * args.sparse_steps
        sbytes = (STREAM_BYTES_SYN_STEP * sp.n_synapses + STREAM_BYTES_NEURON_STEP * sp.n_neurons) \
            * args.sparse_steps
        hbm = peaks.get("hbm_gbs")
        straffic = traffic_for("grid_kernel", "sparse_large", args.sparse_steps)
        sparse = {"workload": "10,000 HH neurons (8k E, 2k I), p=0.02, ~2M synapses, Philox shot noise, "
                              f"grid mode over {sinfo['grid_ctas']} CTAs",
                  "value": sp.n_neurons * args.sparse_steps / sec, "unit": UNIT,
                  "us_per_rk4_step": sms * 1e3 / args.sparse_steps,
                  "synapse_steps_per_s": sp.n_synapses * args.sparse_steps / sec,
                  "roofline": {"bound": "alu", "achieved": sflop / sec / 1e12, "peak": fp32_peak_tflops(smax),
                               "unit": "TFLOP/s", "frac": sflop / sec / 1e12 / fp32_peak_tflops(smax),
                               "traffic": straffic,
                               "kernel": "grid_kernel (one launch of the timed call)",
                               "peak_source": "FP32 FMA pipes: SMs x 128 lanes x 2 x sm_max_mhz"},
                  "roofline_if_streamed": {
                      "bound": "hbm", "achieved": sbytes / sec / 1e9, "peak": hbm, "unit": "GB/s",
                      "frac": sbytes / sec / 1e9 / hbm if hbm else None,
                      "note": f"{STREAM_BYTES_SYN_STEP} B per synapse and {STREAM_BYTES_NEURON_STEP} B per neuron "
                              "per step if the state streamed from HBM; the kernel keeps it in shared memory, "
                              "so this bound does not bind (traffic per launch is the measured DRAM bytes)"}}

    # ---- differentiated form: adjoint gradient time / forward time
    adjoint = None
    if rank == 0 and args.adjoint_steps > 0:
        from paper_1906_03958_gb300 import netgen as ng
        hidden, start = ng.differentiated(n_sets=64)
        T = args.adjoint_steps
        with psst.Network(start, rec_stride=1, rec_capacity=T) as dn:
            dn.record_checkpoints(args.ckpt_every, T)
            y0 = dn.get_state().clone()
            dn.integrate(50)                      # warm-up (records its checkpoints)
            dn.adjoint(50, torch.zeros((50, start.n_neurons), device="cuda"), 0)
            torch.cuda.synchronize()
            dn.set_state(y0)
            dn.set_step(0)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            dn.integrate(T)
            e1.record(stream)
            frames = dn.read_record(out=torch.empty((T, start.n_neurons), device="cuda"))
            # gradient of a mean-square trace loss over the projection neurons
            pn = torch.from_numpy(start.neuron_type % 2 == 0).cuda()
            dldv = torch.where(pn, 2.0 * frames / (T * int(pn.sum())), torch.zeros_like(frames))
            torch.cuda.synchronize()
            e1b = torch.cuda.Event(enable_timing=True)
            e1b.record(stream)
            dn.adjoint(T, dldv, 0)                # the forward recorded its checkpoints
            e2.record(stream)
            torch.cuda.synchronize()
            dn.status()
            fwd_ms, adj_ms = e0.elapsed_time(e1), e1b.elapsed_time(e2)
        peaks = measured_peaks()
        smax = peaks.get("sm_max_mhz", 2070.0)
        pairs = start.n_neurons * start.syn_params.shape[0]
        aflop = (ADJ_FLOP_SYN_STEP * start.n_synapses + ADJ_FLOP_NEURON_STEP * start.n_neurons
                 + ADJ_FLOP_PAIR_STEP * pairs) * T
        atraffic = traffic_for("adj_kernel", "differentiated", T)
        adjoint = {"workload": f"64 antennal-lobe parameter sets, dense 120x120 W + GABA_B, {T} steps, "
                               f"checkpoint every {args.ckpt_every} (recorded by the forward), segment recompute",
                   "forward_ms": fwd_ms, "adjoint_ms": adj_ms, "ratio": adj_ms / fwd_ms,
                   "roofline": {"bound": "alu", "achieved": aflop / (adj_ms / 1e3) / 1e12,
                                "peak": fp32_peak_tflops(smax), "unit": "TFLOP/s",
                                "frac": aflop / (adj_ms / 1e3) / 1e12 / fp32_peak_tflops(smax),
                                "traffic": atraffic,
                                "kernel": "adj_kernel (one launch: segment recompute and reverse sweep)",
                                "flop_per_step": {"synapse": ADJ_FLOP_SYN_STEP, "neuron": ADJ_FLOP_NEURON_STEP,
                                                  "neuron_type_pair": ADJ_FLOP_PAIR_STEP}}}

    # ---- roofline of the dominant kernel (the CTA-resident integrator)
    peaks = measured_peaks()
    smax = peaks.get("sm_max_mhz", 2070.0)
    n_sms = device_sms()
    peak_tflops = fp32_peak_tflops(smax)
    # one integrate call = the size-class launches back to back, together
    # covering every network once: its FLOP over its duration
    pair_gates = info["n_pair_gate_nets"] == spec.n_nets
    flops_call = workload_flops_per_step(spec, pair_gates) * args.chunk
    dur = t_local / args.steps
    roof = {"bound": "alu", "achieved": flops_call / dur / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": flops_call / dur / 1e12 / peak_tflops,
            "traffic": traffic_for("net_kernel", args.workload),
            "kernel": f"net_kernel: the {info['n_launch_classes']} size-class launches of one integrate call",
            "gates": "per (presynaptic neuron, type) pair" if pair_gates else "per synapse",
            "peak_source": f"FP32 FMA pipes: {n_sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                           f"{smax:.0f} MHz (sm_max_mhz of MEASURED_PEAKS.json)"}

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": wl_desc, "rk4_steps_per_bench_step": args.chunk,
                          "n_nets": spec.n_nets, "neurons": spec.n_neurons, "synapses": spec.n_synapses,
                          "rec_stride": args.rec_stride, "l2": "working set larger than L2 (state+synapses "
                          f"{(dim * 4 + spec.n_synapses * 8) / 1e6:.0f} MB)",
                          "block_threads": info["block_threads"], "item_chunks": info["item_chunks"],
                          "grid_ctas": info["grid_ctas"], "smem_bytes": info["smem_bytes"],
                          "single_cta_nets": info["n_single_cta_nets"], "cluster_nets": info["n_cluster_nets"],
                          "launch_classes": info["n_launch_classes"],
                          "autotune_trial_steps": args.autotune, "cuda_graph": bool(args.graph),
                          "parallelism": f"replicas x{world}"},
               "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
               "gpu_launches": launches, "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
               "single": single, "sparse_large": sparse, "adjoint_over_forward": adjoint,
               "independent": indep}
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def reference_arm(args, rank, world):
    """The FP64 oracle as the reference implementation, on the host cores."""
    if rank != 0:
        return
    spec, wl_desc, _ = make_workload(args.workload, 0)
    cores = os.cpu_count() or 1
    sample = cpu_sample(spec, args.cpu_nets, args.cpu_steps)
    nc = min(cores, len(sample))
    for _ in range(args.warmup):
        run_cpu_baseline(sample[:nc], 20, nc)
    times = []
    for _ in range(args.steps):
        _, wall = run_cpu_baseline(sample, args.cpu_steps, nc)
        times.append(wall)
    neuron_steps = sum(s.n_neurons for s in sample) * args.cpu_steps
    t = sum(times)
    value = neuron_steps * args.steps / t
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": wl_desc},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": nc, "kind": "oracle",
                            "sample": f"{len(sample)} networks of the workload x {args.cpu_steps} RK4 steps per "
                                      f"step, FP64, one process per core"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
