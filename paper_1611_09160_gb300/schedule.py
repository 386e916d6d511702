"""Choice of the concurrent schedule (colouring) for a WMCD simulation.

The paper applies moves one after another and names "parallel execution of multiple
non-overlapping wavelet moves" as future work (Sec. VIII). This library runs the moves of
one scale band (a layer, an octave of P_lambda, Eq. 32) concurrently when they are far
enough apart: the box is cut into G^3 coarse cells coloured by (cx mod K, cy mod K,
cz mod K); queues of one colour run at the same time. A move whose support, interaction
partners or displacement could leave its cell's region (the cell widened by (K-1)/2
cells) is deferred to a serial phase, so the schedule is exact whatever G is; G only
sets how often that happens and how much runs in parallel.

This module picks (K, fine grid, G per layer, concurrent support cap) from the physics
parameters. The values are ordinary parameters of a run: a caller may set them by hand.
"""
from __future__ import annotations

import math

WCA_CUT = 1.122462048309373   # 2^(1/6)
MAX_LAYERS = 16


def layer_bounds(lambda_min: float, lambda_max: float):
    """Octave bands [lmin 2^l, lmin 2^(l+1)) of P_lambda, the last one ending at lambda_max."""
    n = 1
    while lambda_min * 2.0 ** n < lambda_max:
        n += 1
    if n > MAX_LAYERS:
        raise ValueError("lambda_max / lambda_min exceeds 2^16")
    lo = [lambda_min * 2.0 ** l for l in range(n)]
    hi = [lambda_min * 2.0 ** (l + 1) for l in range(n - 1)] + [lambda_max]
    return lo, hi


def interaction_reach(wca_sigma: float, wca_eps: float) -> float:
    return WCA_CUT * wca_sigma if wca_eps != 0.0 else 0.0


def choose(box_L: float, lambda_min: float, lambda_max: float, A0: float, wca_sigma: float, wca_eps: float,
           colour_K: int = 2, slack: float = 1.0, max_fine: int = 512, n_cap: int = 64,
           min_queues_per_axis: int = 2, cell_scale: float = 1.0, serial_only: bool = False,
           n_beads: int | None = None, level2: int = 0) -> dict:
    """Return the schedule fields: colour_K, grid_f, n_cap, grid_layer (list of 16), level2.

    cell_scale widens the fine cells beyond the interaction reach (fewer, fuller cells to walk
    in dilute systems); serial_only runs every layer in the serial phase. With n_beads given,
    a layer whose mean support at the lower edge of its band (the beads of a ball of that
    radius at the mean density) already exceeds n_cap is left serial: a concurrent move with
    more than n_cap beads is deferred, so colouring such a layer would only add phases whose
    moves nearly all run again in the serial phase."""
    if colour_K not in (2, 3, 4):
        raise ValueError("colour_K must be 2, 3 or 4")
    if cell_scale < 1.0:
        raise ValueError("fine cells may not be narrower than the interaction reach")
    reach = interaction_reach(wca_sigma, wca_eps)
    hf = max(reach, 1.0) * cell_scale
    grid_f = max(1, min(max_fine, int(math.floor(box_L / hf))))
    lo, hi = layer_bounds(lambda_min, lambda_max)
    density = None if n_beads is None else float(n_beads) / box_L ** 3
    grid_layer = [0] * MAX_LAYERS
    for l, lh in enumerate(hi):
        if density is not None and density * (4.0 / 3.0) * math.pi * lo[l] ** 3 > n_cap:
            continue
        # everything a move reads or writes lies within R of its centre, and the centre
        # within lambda of the picked bead: margin = lambda + R + slack for drift
        margin = 2.0 * lh + 0.25 * A0 * lh + reach + slack
        h_min = 2.0 * margin / (colour_K - 1)
        G = colour_K * int(math.floor(box_L / (colour_K * h_min)))
        if G >= min_queues_per_axis * colour_K and not serial_only:
            grid_layer[l] = G
    return {"colour_K": colour_K, "grid_f": grid_f, "n_cap": n_cap, "grid_layer": grid_layer,
            "level2": int(level2)}
