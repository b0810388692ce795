"""Shared helpers of the test-suite (comparison metrics, state layout)."""
import numpy as np


def split_state(y, N, S):
    y = np.asarray(y)
    return dict(V=y[:N], m=y[N:2 * N], h=y[2 * N:3 * N], n=y[3 * N:4 * N],
                r=y[4 * N:4 * N + S], s=y[4 * N + S:4 * N + 2 * S])


def step_error(y32, y64, N, S, s_v=1.0, s_gate=1e-3):
    """max_i |y32_i - y64_i| / max(|y64_i|, floor), floor 1 mV for V and 1e-3
    for the gates (m, h, n, r, s)."""
    y32 = np.asarray(y32, np.float64)
    y64 = np.asarray(y64, np.float64)
    floor = np.full(y64.shape, s_gate)
    floor[:N] = s_v
    return float(np.max(np.abs(y32 - y64) / np.maximum(np.abs(y64), floor)))
