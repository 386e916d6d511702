"""Autotuner for the concurrent schedule and the launch shapes, by measurement on the GPU.

Two kinds of choice are tuned, and they are kept apart because they differ in what they
change:

* The schedule of a simulation: fine-cell size (``cell_scale`` times the interaction reach),
  colouring stride (``colour_K``), which layers run coloured (``min_queues_per_axis``,
  ``serial_only``). The schedule fixes the order of moves, so it is part of a simulation's
  definition: it is chosen per system *shape* (bead count, box, potential, precision) from a
  table, never from what else shares a batch, so a request gets the same schedule, and the
  same trajectory, alone or in any batch.
* Launch shapes (warps per block of the concurrent kernel, threads of the serial block):
  results do not depend on them, so they are tuned per batch.

Every candidate is timed on throw-away simulations of a synthetic system of the shape (the
same generator as the workloads), a few sweeps after warm-up, with CUDA events; the score is
bead-updates per second. With ``copies`` > 1 the candidate runs as a batch of that many
independent copies of the shape, which measures the schedule where it will run: among many
other simulations, whose own work already fills the GPU.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

from . import inputs as I
from . import schedule as S
from . import wmcd

SCHEDULE_CANDIDATES = (
    {"colour_K": 2},
    {"colour_K": 2, "cell_scale": 1.5},
    {"colour_K": 2, "cell_scale": 2.0},
    {"colour_K": 3},
    {"colour_K": 2, "min_queues_per_axis": 3},
    {"colour_K": 2, "serial_only": True},
)
# in a batch the other simulations fill the GPU, so only the schedules that differ in kind
# (all serial, coloured with two or three colours per axis) are worth timing there
BATCH_SCHEDULE_CANDIDATES = (
    {"colour_K": 2, "serial_only": True},
    {"colour_K": 2},
    {"colour_K": 3},
)
LAUNCH_CANDIDATES = ((2, 512), (2, 128), (2, 32), (1, 32), (4, 32), (1, 128))
DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")


def shape_key(n_beads: int, box_L: float, precision: int, planewave_mode: int) -> str:
    """Table key: bead count to the nearest power of two, box side on a half-octave grid."""
    nb = 1 << max(0, int(round(math.log2(max(1, n_beads)))))
    lb = round(2 * math.log2(box_L)) / 2
    return f"N{nb}_L{lb:.3f}_p{precision}_w{planewave_mode}"


def _time_batch(params: dict, system, warm: int, sweeps: int, copies: int) -> float:
    import torch
    ps = [dict(params, sim_id=int(params.get("sim_id", 0)) + 7919 * c) for c in range(copies)]
    b = wmcd.Batch(copies, sum(wmcd.batch_need(p) for p in ps))
    try:
        slots = [b.admit(p, system.pos, system.chain_len) for p in ps]
        b.step(warm)
        torch.cuda.synchronize()
        b0 = sum(b.sim(k).stats().bead_updates for k in slots)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(sweeps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        return (sum(b.sim(k).stats().bead_updates for k in slots) - b0) / (ms / 1e3)
    finally:
        b.close()


def _time_sim(params: dict, system, warm: int, sweeps: int) -> float:
    import torch
    sim = wmcd.Simulation(params, system.pos, system.chain_len)
    try:
        sim.sweep(warm)
        torch.cuda.synchronize()
        b0 = sim.stats().bead_updates
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sim.sweep(sweeps)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        return (sim.stats().bead_updates - b0) / (ms / 1e3)
    finally:
        sim.close()


class Tuner:
    """Per-shape schedule table (optionally kept in a JSON file) and launch-shape tuning."""

    def __init__(self, path: str | None = None, warm: int = 2, sweeps: int = 4, copies: int = 1,
                 seed_table: str | None = None):
        """path: table read at start and written after each new measurement; seed_table: a
        read-only table (e.g. the one measured on GB300 and shipped with the package) whose
        entries are used as they are."""
        self.path = path
        self.warm, self.sweeps, self.copies = warm, sweeps, int(copies)
        self.table = {}
        for src in (seed_table, path):
            if src and os.path.exists(src):
                with open(src) as f:
                    self.table.update(json.load(f))

    def save(self):
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def schedule(self, base: dict, system=None, chain_lengths=None, candidates=None) -> dict:
        """Parameters ``base`` with the tuned schedule of its shape (measured on first use, over
        ``candidates`` if given, e.g. a short list for systems too large to time many ways)."""
        key = shape_key(base["n_beads"], base["box_L"], base.get("precision", 0), base.get("planewave_mode", 0))
        if self.copies > 1:
            key += f"_x{self.copies}"
        if key not in self.table:
            self.table[key] = self._tune_schedule(base, system, chain_lengths, candidates)
            self.save()
        return self.apply(base, self.table[key]["choice"])

    @staticmethod
    def apply(base: dict, choice: dict) -> dict:
        p = dict(base)
        p.update(S.choose(p["box_L"], p["lambda_min"], p["lambda_max"], p["A0"], p["wca_sigma"], p["wca_eps"],
                          **dict({"n_beads": p["n_beads"]}, **choice)))
        return p

    def _tune_schedule(self, base: dict, system, chain_lengths, candidates=None) -> dict:
        if system is None:
            lens = chain_lengths if chain_lengths is not None else [base["n_beads"]]
            system = I.make_system(list(lens), 0, base["box_L"], seed=12345)
        scores = []
        if candidates is None:
            candidates = BATCH_SCHEDULE_CANDIDATES if self.copies > 1 else SCHEDULE_CANDIDATES
        for cand in candidates:
            try:
                p = self.apply(base, cand)
            except ValueError:
                continue
            if self.copies > 1:
                scores.append((_time_batch(p, system, self.warm, self.sweeps, self.copies), cand))
            else:
                scores.append((_time_sim(p, system, self.warm, self.sweeps), cand))
        best = max(scores, key=lambda t: t[0])
        return {"choice": best[1], "scores": [[s, c] for s, c in scores]}

    def launch_shape(self, batch, sweeps: int = 2):
        """Time each launch shape on ``batch`` (advancing its simulations: results do not
        depend on the shape) and keep the fastest. Returns (stage_warps, serial_threads)."""
        import torch
        best, best_ms = None, float("inf")
        for shape in LAUNCH_CANDIDATES:
            batch.set_block(*shape)
            batch.step(1)                      # records the graph for this shape
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            batch.step(sweeps)
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            if ms < best_ms:
                best, best_ms = shape, ms
        batch.set_block(*best)
        return best


SMEM_SERIAL_MAX_N = 2048   # largest simulation whose small-scale serial phase runs in shared memory


def ensemble_params(systems, precision: int, planewave_mode: int, seed: int, tuner: Tuner | None = None,
                    policy: str = "per_shape"):
    """Parameters of an ensemble of single-chain systems (the uneven-size batch workload).

    policy "per_shape": each simulation gets its shape's tuned schedule; "serial_small": every
    simulation small enough for the shared-memory serial phase runs all its layers serially,
    the others get their shape's tuned schedule. Either way the schedule depends only on the
    simulation's own shape and the policy, never on the other members of a batch."""
    out = []
    for k, s in enumerate(systems):
        p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, sim_id=k, precision=precision,
                                planewave_mode=planewave_mode)
        if policy == "serial_small" and s.n_beads <= SMEM_SERIAL_MAX_N:
            p = Tuner.apply(p, {"colour_K": 2, "serial_only": True})
        elif tuner is not None:
            p = tuner.schedule(p, chain_lengths=s.chain_len)
        out.append(p)
    return out


def batch_throughput(params, systems, warm: int = 1, sweeps: int = 3) -> float:
    """Bead-updates per second of one batch holding all the given simulations."""
    import torch
    b = wmcd.Batch(len(params), sum(wmcd.batch_need(p) for p in params) + (1 << 20))
    try:
        slots = [b.admit(p, s.pos, s.chain_len) for p, s in zip(params, systems)]
        b.step(warm)
        torch.cuda.synchronize()
        b0 = sum(b.sim(k).stats().bead_updates for k in slots)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.step(sweeps)
        e1.record()
        e1.synchronize()
        return (sum(b.sim(k).stats().bead_updates for k in slots) - b0) / (e0.elapsed_time(e1) / 1e3)
    finally:
        b.close()


def choose_policy(systems, precision: int, planewave_mode: int, tuner: Tuner, sample: int = 256, seed: int = 7):
    """Pick the ensemble schedule policy by measuring whole batches of a sample of the workload:
    per-shape schedules interact in a batch (a coloured simulation adds colour phases that every
    batched sweep waits for), which a per-shape measurement cannot see."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(systems), size=min(sample, len(systems)), replace=False)
    sub = [systems[i] for i in idx]
    scores = {}
    for policy in ("per_shape", "serial_small"):
        ps = ensemble_params(sub, precision, planewave_mode, seed=1, tuner=tuner, policy=policy)
        scores[policy] = batch_throughput(ps, sub)
    best = max(scores, key=scores.get)
    return best, scores


def sample_shapes(n_beads: np.ndarray, n: int) -> np.ndarray:
    """Representative bead counts (quantiles) to tune ahead of a run."""
    return np.unique(np.quantile(n_beads, np.linspace(0, 1, n)).astype(int))


def main(argv=None):
    """Measure the schedule table for the uneven-size ensemble shapes (single chains, lengths
    log-uniform in [lo, hi], volume fraction phi) in batch context and write it as JSON."""
    import argparse
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--out", required=True)
    ap.add_argument("--sims", type=int, default=1024)
    ap.add_argument("--lo", type=int, default=16)
    ap.add_argument("--hi", type=int, default=2048)
    ap.add_argument("--phi", type=float, default=1e-3)
    ap.add_argument("--copies", type=int, default=152)
    ap.add_argument("--precision", type=int, default=wmcd.MIXED)
    ap.add_argument("--planewave", type=int, default=wmcd.PLANEWAVE_PERIODIC)
    a = ap.parse_args(argv)
    wmcd.build()
    wmcd.load()
    tuner = Tuner(path=a.out, warm=1, sweeps=2, copies=a.copies)
    for seed in (1, 2):
        lens = I.loguniform_lengths(a.sims, a.lo, a.hi, seed)
        for n in sorted(set(int(x) for x in lens)):
            L = I.box_for_volume_fraction(n, a.phi)
            p = wmcd.default_params(n, L, seed=1, precision=a.precision, planewave_mode=a.planewave)
            tuner.schedule(p, chain_lengths=[n])
    print(json.dumps({k: v["choice"] for k, v in tuner.table.items()}, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
