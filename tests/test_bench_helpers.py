"""bench.py's measurement helpers on CPU: the DRAM-traffic lookup behind
`roofline.traffic` (keyed by each kernel's own sources, scaled by steps
where the capture says so) and the algorithmic FLOP count behind
`roofline.achieved`, against a count made synapse by synapse."""
import json
import os
import shutil

import numpy as np

import bench
from paper_1906_03958_gb300 import netgen as ng


def _fake_root(tmp_path):
    csrc = os.path.join(bench.ROOT, "paper_1906_03958_gb300", "csrc")
    dst = tmp_path / "paper_1906_03958_gb300" / "csrc"
    shutil.copytree(csrc, dst)
    (tmp_path / "profiles").mkdir()
    return dst


def test_traffic_lookup_keys_scaling_and_staleness(tmp_path, monkeypatch):
    csrc = _fake_root(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h_net, h_adj = bench.kernel_source_hash("net_kernel"), bench.kernel_source_hash("adj_kernel")
    assert h_net != h_adj
    table = {
        "net_kernel:batched": {"bytes_per_launch": 1000, "source_hash": h_net},
        "adj_kernel:differentiated": {"bytes_per_launch": 800, "captured_steps": 200, "source_hash": h_adj},
    }
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(table))
    assert bench.traffic_for("net_kernel", "batched") == 1000
    assert bench.traffic_for("net_kernel", "batched", 5000) == 1000  # no captured_steps: unscaled
    assert bench.traffic_for("adj_kernel", "differentiated", 20000) == 800 * 100
    assert bench.traffic_for("grid_kernel", "sparse_large") is None  # no entry
    # a comment edit keeps the captures; a code edit of one kernel's source
    # drops that kernel's capture only
    p = csrc / "psst_adjoint.cu"
    p.write_text(p.read_text() + "\n// a trailing comment\n")
    assert bench.traffic_for("adj_kernel", "differentiated", 200) == 800
    p.write_text(p.read_text() + "\nstatic int extra_symbol_for_the_test;\n")
    assert bench.traffic_for("adj_kernel", "differentiated", 200) is None
    assert bench.traffic_for("net_kernel", "batched") == 1000
    # a shared header invalidates every kernel's capture
    q = csrc / "psst_device.cuh"
    q.write_text(q.read_text() + "\nstatic int another_symbol_for_the_test;\n")
    assert bench.traffic_for("net_kernel", "batched") is None


def _flops_by_synapse(spec, pair_gates):
    """Per-RK4-step FLOP of the kernels' formulation, counted by walking the
    synapses one by one (the same per-unit constants as bench.py)."""
    nt = spec.syn_params.shape[0]
    kinds = spec.syn_params[:, 0]
    total = 0.0
    for b in range(spec.n_nets):
        n0, n1 = spec.net_neuron_off[b], spec.net_neuron_off[b + 1]
        total += bench.FLOP_NEURON_STAGE * (n1 - n0)
        pairs = set()
        has2 = False
        for k in range(spec.row_ptr[n0], spec.row_ptr[n1]):
            t = int(spec.syn_type[k])
            pairs.add((int(spec.pre[k]), t))
            has2 |= kinds[t] != 0
            if pair_gates:
                total += bench.FLOP_SYN_PAIR_STAGE
            else:
                total += bench.FLOP_SYN2_STAGE if kinds[t] != 0 else bench.FLOP_SYN1_STAGE
        if pair_gates:
            for _, t in pairs:
                total += bench.FLOP_COEF1_STAGE + bench.FLOP_PAIR1_STAGE
                if kinds[t] != 0:
                    total += bench.FLOP_COEF2_STAGE + bench.FLOP_PAIR2_STAGE
        else:
            total += bench.FLOP_COEF1_STAGE * (n1 - n0) * nt
            if has2:
                total += bench.FLOP_COEF2_STAGE * (n1 - n0) * nt
    return 4.0 * total


def test_workload_flops_match_a_synapse_by_synapse_count():
    # a ragged batch of first-order networks, and the antennal lobe
    # (second-order GABA_B pairs)
    for spec in (ng.batched(5, n_max=60), ng.antennal_lobe()):
        for pair_gates in (True, False):
            want = _flops_by_synapse(spec, pair_gates)
            got = bench.workload_flops_per_step(spec, pair_gates)
            assert np.isclose(got, want, rtol=0, atol=0.5), (spec.name, pair_gates, got, want)
