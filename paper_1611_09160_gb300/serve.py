"""Serving loop: continuous batching of independent WMCD simulations on one GPU.

Requests (a simulation's parameters, initial configuration and the number of sweeps wanted)
arrive over time. The server keeps one batch (``wmcd.Batch``) resident on the device: a
request is admitted as soon as a slot and a large enough block of the batch's memory pool are
free, joins the batched sweeps already running (one CUDA graph launch per sweep for all
resident simulations), and leaves the batch when its sweeps are done, freeing its slot and
memory for the next. Admission of new requests runs on the batch's own stream while the
previous batched step is still on the GPU, so arrivals overlap with running work.

Each simulation's random stream, schedule and reduction order are its own, so a request's
result does not depend on what else shares the batch (tested against the same request run
alone). The loop reports throughput (bead-updates/s, simulated time per second) with the
per-sweep latency seen by resident simulations (p50 / p99) and the request latency from
arrival to completion.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import wmcd


@dataclass
class Request:
    rid: int
    params: dict
    pos: np.ndarray
    chain_len: np.ndarray
    n_sweeps: int
    arrival: float = 0.0          # seconds after the start of the run


@dataclass
class Result:
    rid: int
    positions: np.ndarray         # unwrapped, after n_sweeps sweeps
    bead_updates: int
    sim_time: float
    accepted: int
    arrival: float
    admitted: float
    finished: float


@dataclass
class ServeReport:
    results: dict = field(default_factory=dict)
    wall_s: float = 0.0
    gpu_ms: float = 0.0
    bead_updates: int = 0
    sim_time: float = 0.0
    sweep_ms: list = field(default_factory=list)     # one entry per batched sweep
    steps: int = 0
    max_resident: int = 0
    rejected_full: int = 0                           # admission attempts refused for lack of slot / memory

    def summary(self) -> dict:
        lat = np.array([r.finished - r.arrival for r in self.results.values()]) if self.results else np.zeros(1)
        sw = np.array(self.sweep_ms) if self.sweep_ms else np.zeros(1)
        return {
            "requests": len(self.results),
            "wall_s": self.wall_s,
            "gpu_ms": self.gpu_ms,
            "bead_updates_per_s": self.bead_updates / self.wall_s if self.wall_s > 0 else 0.0,
            "sim_time_per_s": self.sim_time / self.wall_s if self.wall_s > 0 else 0.0,
            "sweep_ms_p50": float(np.percentile(sw, 50)),
            "sweep_ms_p99": float(np.percentile(sw, 99)),
            "request_s_p50": float(np.percentile(lat, 50)),
            "request_s_p99": float(np.percentile(lat, 99)),
            "batched_sweeps": len(self.sweep_ms),
            "steps": self.steps,
            "max_resident": self.max_resident,
            "admission_waits": self.rejected_full,
        }


class CudaStepTimer:
    """Device time of each sweep of a batched step: a CUDA event on the step's stream before
    the first sweep and after every sweep."""

    def __init__(self):
        import torch
        self._torch = torch
        self.stream = torch.cuda.current_stream()

    def start(self):
        e = self._torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.events = [e]

    def mark(self):
        """End of one sweep."""
        e = self._torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.events.append(e)

    def wait_ms(self) -> list:
        """Milliseconds of each sweep marked since start()."""
        self.events[-1].synchronize()
        return [a.elapsed_time(b) for a, b in zip(self.events[:-1], self.events[1:])]


class Server:
    """Continuous-batching request loop over one batch.

    capacity: most simulations resident at once; pool_bytes: device memory reserved for their
    state; chunk: most sweeps per batched step (a step ends early when a resident request
    finishes, so no request runs past its sweep count). ``batch`` and ``timer`` default to a
    ``wmcd.Batch`` and CUDA-event timing; any objects with the same methods will do."""

    def __init__(self, capacity: int = 0, pool_bytes: int = 0, chunk: int = 16, stage_warps: int = 2,
                 serial_threads: int = 512, batch=None, timer=None):
        self.batch = batch if batch is not None else wmcd.Batch(capacity, pool_bytes)
        self.batch.set_block(stage_warps, serial_threads)
        self.timer = timer if timer is not None else CudaStepTimer()
        self.chunk = int(chunk)

    def close(self):
        self.batch.close()

    def run(self, requests, realtime: bool = True) -> ServeReport:
        """Serve ``requests`` (arrival times in seconds from now when ``realtime``; otherwise
        every request is available at once). Returns the report with each request's result."""
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        resident = {}             # slot -> [request, sweeps left, admitted time]
        rep = ServeReport()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731

        def admit_arrived():
            """Admit arrived requests in arrival order; False if the first one did not fit."""
            while pending and (not realtime or pending[0].arrival <= now()):
                r = pending[0]
                slot = self.batch.admit(r.params, r.pos, r.chain_len)
                if slot is None:
                    rep.rejected_full += 1
                    return False
                pending.popleft()
                resident[slot] = [r, int(r.n_sweeps), now()]
                rep.max_resident = max(rep.max_resident, len(resident))
            return True

        def retire_done():
            for slot in [k for k, v in resident.items() if v[1] <= 0]:
                r, _, t_adm = resident.pop(slot)
                sim = self.batch.sim(slot)
                pos = sim.positions(unwrapped=True)
                st = sim.stats()
                self.batch.retire(slot)
                res = Result(r.rid, pos, int(st.bead_updates), float(st.sim_time), int(st.accepted_total),
                             r.arrival, t_adm, now())
                rep.results[r.rid] = res
                rep.bead_updates += res.bead_updates
                rep.sim_time += res.sim_time

        while pending or resident:
            fits = admit_arrived()
            if not resident:
                if not fits:
                    raise RuntimeError(f"request {pending[0].rid} does not fit in an empty batch")
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival - now(), 0.01)))
                continue
            k = min(self.chunk, min(v[1] for v in resident.values()))
            in_step = list(resident)
            # one graph launch per sweep, with a CUDA event after each, so that the latency of
            # every batched sweep is measured on its own
            self.timer.start()
            for _ in range(k):
                self.batch.step(1)
                self.timer.mark()
            # requests arriving while the step runs are admitted now, on the batch's own stream
            admit_arrived()
            per_sweep = self.timer.wait_ms()
            rep.gpu_ms += float(sum(per_sweep))
            rep.sweep_ms.extend(per_sweep)
            rep.steps += 1
            for slot in in_step:
                resident[slot][1] -= k
            retire_done()
        rep.wall_s = now()
        return rep


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> np.ndarray:
    """Arrival times of a Poisson process (exponential gaps), seconds."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
