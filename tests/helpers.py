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


# Per-coordinate floor of gradient comparisons, as a fraction of the
# largest coordinate of the expected vector.
GRAD_FLOOR = 1e-2


def grad_error(got, want, floor_frac=GRAD_FLOOR):
    """Per-coordinate relative error of a gradient vector:
    max_i |got_i - want_i| / max(|want_i|, floor_frac * max_j |want_j|).

    A coordinate at or above floor_frac of the vector's largest is compared
    relative to itself; a smaller one against the absolute bound
    tol * floor_frac * max_j |want_j|.  The floor exists because the FP32
    adjoint's rounding error in a coordinate comes from the sums it is
    accumulated from (stage adjoints, column sums, per-segment partials),
    whose terms scale with the largest gradients, not with the coordinate:
    a coordinate 1e-5 of the largest cannot be resolved to 1e-3 of itself
    in FP32.  With tol = 1e-3 and the 1e-2 floor, such coordinates are held
    to 1e-5 of the largest gradient, 100 times tighter than normalising by
    the largest."""
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    scale = floor_frac * max(float(np.max(np.abs(want))) if want.size else 0.0, 1e-300)
    return float(np.max(np.abs(got - want) / np.maximum(np.abs(want), scale))) if want.size else 0.0


def fd_reference(fd):
    """Per coordinate, a central-difference value and its error bound from a
    step ladder.  fd: [rungs, coordinates], the step growing by a constant
    factor per rung.  Small steps carry the rounding noise of the FP64
    trajectory divided by h, large ones truncation error O(h^2), so the
    differences converge toward the derivative and then drift away; the
    neighbouring pair of rungs that agree best is taken, its midpoint as the
    value and its full gap as the bound."""
    fd = np.asarray(fd, np.float64)
    e = np.abs(np.diff(fd, axis=0))
    j = np.argmin(e, axis=0)
    c = np.arange(fd.shape[1])
    return 0.5 * (fd[j, c] + fd[j + 1, c]), e[j, c]
