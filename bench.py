"""Benchmark of the WMCD sweep on GB300.

Headline workload (one step = one sweep of the whole hot path: slots, bucketing, colour
phases, serial phase, plane waves): the large dilute suspension, 4,000,000 free spheres (WCA
only) and 1,000 self-avoiding chains x 1,024 beads (5,024,000 beads) at volume fraction 1e-3
in a periodic cube (L = 2760.9 a), harmonic bonds k = 100 kT/a^2 with rest length 2a, WCA
sigma = 2a, eps = 1 kT, lambda_min = 2a, lambda_max = L/2, A0 = 0.5, wavelets plus periodic
plane waves (|l| <= 8), mixed precision, the concurrent schedule from the shipped table.
Inputs are synthetic (seeded). The state (5.7 GB) is far larger than L2, and a 256 MiB buffer
is still written on the timed stream before every timed sweep; each sweep is timed with CUDA
events on that stream.

Metric: bead-updates per second (a bead-update = one bead inside an attempted move's
support; N per plane-wave attempt), whole job over all ranks; also simulated time per wall
second. Multi-GPU runs are independent replicas (different seeds), no collective in the data
path. The plain binary64 sweep is timed on the same inputs beside it.

Further legs: the dilute chains (256 x 64, 16,384 beads) and the semi-dilute solution
(4,096 x 256 at volume fraction 0.05); plane-wave moves alone on the suspension; the
uneven-size ensemble (single chains, lengths log-uniform in [16, 2048]) as one batch
(`batched`, one CUDA graph per batched sweep) and through the continuous-batching loop
(`serve`, Poisson arrivals, per-sweep and per-request latency percentiles); and the drift of
mixed precision from plain binary64 on the 32-bead chain and on the dilute chains.

--impl reference times the CPU oracle (the plain sequential FP64 statement of the method)
on the same configuration's 1/64 subsample, on one host core.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bead-updates/s (WMCD sweep)"
UNIT = "bead-updates/s"


SUSPENSION = dict(n_spheres=4_000_000, n_chains=1000, chain_len=1024, phi=1e-3)
SUBSAMPLE = dict(n_spheres=62_500, n_chains=16, chain_len=1024, phi=1e-3)     # N/64 in L/4


def workload_config():
    return {"workload": "suspension 4,000,000 spheres + 1000x1024 chains (5,024,000 beads) phi=1e-3 L=2760.9, "
                        "wavelet+plane-wave lcut 8, A0=0.5, harmonic k=100 r0=2, WCA sigma=2 eps=1, "
                        "lambda 2..L/2, mixed precision",
            "n_beads": 5_024_000, "spheres": 4_000_000, "chains": 1000, "chain_len": 1024, "phi": 1e-3,
            "planewave_lcut": 8,
            "l2": "inputs larger than L2 (5.7 GB of state); L2 also flushed (256 MiB write on the timed stream) "
                  "before each timed sweep"}


def make_system(seed, sample=None):
    from paper_1611_09160_gb300 import inputs as I
    return I.suspension(seed=seed, **(sample or SUSPENSION))


def make_params(system, precision, seed, sim_id=0, scaled=False):
    """The suspension's parameters with the schedule of its shape from the shipped table (the
    table is keyed on the mixed-precision shape; the binary64 run uses the same schedule). A
    scaled-down copy for profiling takes the full size's first candidate without measuring."""
    from paper_1611_09160_gb300 import autotune as A
    from paper_1611_09160_gb300 import wmcd
    base = wmcd.default_params(system.n_beads, system.box_L, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=8,
                               precision=wmcd.MIXED, seed=seed, sim_id=sim_id)
    if scaled:
        return dict(A.Tuner.apply(base, SUSPENSION_CANDIDATES[0]), precision=precision)
    tuner = A.Tuner(path=None, warm=1, sweeps=1, seed_table=A.DEFAULT_TABLE)
    p = tuner.schedule(base, system=system, candidates=SUSPENSION_CANDIDATES)
    return dict(p, precision=precision)


SUSPENSION_CANDIDATES = ({"colour_K": 2, "max_fine": 768, "n_cap": 128, "level2": 1},
                         {"colour_K": 2, "max_fine": 768, "n_cap": 128}, {"colour_K": 2, "max_fine": 768},
                         {"colour_K": 2, "max_fine": 1024}, {"colour_K": 3, "max_fine": 768})


def host_cpu():
    """Host processor model and logical core count (for the CPU-baseline record)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"model": model, "nproc": os.cpu_count()}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 3 + k and r[3 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def profile_traffic(kernel_src_sha):
    """dram bytes per launch of the concurrent kernel from the committed ncu summary, if it
    was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "wavelet_concurrent_suspension.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_sha256") != kernel_src_sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def code_sha(texts):
    """Hash of CUDA sources with // comments and blank lines removed: an edit of comments alone
    leaves the compiled kernels, and so the hash, unchanged."""
    h = hashlib.sha256()
    for t in texts:
        for line in t.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()


def kernel_sha():
    return code_sha(open(os.path.join(ROOT, "paper_1611_09160_gb300", "csrc", f)).read()
                    for f in ["wmcd_kernels.cu", "wmcd_device.cuh", "wmcd_internal.h"])


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0}, "fallback"


def oracle_sample(seconds):
    """The oracle, as it stands, on the suspension's 1/64 subsample (62,500 spheres + 16 chains x
    1,024 beads in L/4, same generator and parameters): the first moves of its first sweep in
    schedule order, as many as take about `seconds` (the oracle needs minutes for a whole sweep
    of this subsample). Returns (bead-updates, seconds, moves, description)."""
    import oracle as O
    from paper_1611_09160_gb300 import wmcd
    sub = make_system(1, SUBSAMPLE)
    p = wmcd.default_params(sub.n_beads, sub.box_L, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=8,
                            precision=wmcd.MIXED, seed=1)
    o = O.Oracle(p, sub.pos, sub.chain_len)
    t0 = time.perf_counter()
    probe = o.sweep_sample(64)
    t_probe = time.perf_counter() - t0
    moves = max(64, int(probe * max(seconds - t_probe, 1.0) / max(t_probe, 1e-6)))
    o2 = O.Oracle(p, sub.pos, sub.chain_len)
    t0 = time.perf_counter()
    done = o2.sweep_sample(moves)
    dt = time.perf_counter() - t0
    st = o2.stats()
    desc = (f"first {done} wavelet moves of the first sweep, in schedule order, of the suspension's 1/64 subsample "
            f"({sub.n_beads:,} beads in L = {sub.box_L:.1f}; sequential C++ oracle in its mixed-precision mode: "
            f"binary32 displacements as the GPU's mixed path, binary64 positions, energies and decisions; "
            f"brute-force neighbour search), {dt:.1f} s")
    return st.bead_updates, dt, done, st.sim_time, desc


def cpu_baseline(seconds=15.0):
    """The oracle on a bounded sample of the headline workload, one host core."""
    bu, dt, moves, simt, desc = oracle_sample(seconds)
    return {"value": bu / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
            "host": host_cpu(), "sim_time_per_s": simt / dt}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle as O
    O.build()
    steps = max(1, args.steps)
    per_step = max(1.0, args.reference_seconds / steps)
    for _ in range(args.warmup):
        oracle_sample(min(2.0, per_step))
    tot_bu, tot_dt, tot_moves, tot_sim = 0, 0.0, 0, 0.0
    for _ in range(steps):
        bu, dt, moves, simt, desc = oracle_sample(per_step)
        tot_bu += bu
        tot_dt += dt
        tot_moves += moves
        tot_sim += simt
    value = tot_bu / tot_dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"{steps} steps, each the first moves (about {per_step:.0f} s of work, "
                                       f"{tot_moves} moves in all) of a sweep of the suspension's 1/64 subsample, "
                                       f"after {args.warmup} warm-up samples; sequential C++ oracle in its mixed-precision mode"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sim_time_per_s": tot_sim / tot_dt}
    print(json.dumps(line), flush=True)


def flush_l2(flush, stream, torch):
    """Write a buffer larger than L2 on the timed stream, so the flush is ordered before the
    next timed sweep on that stream."""
    with torch.cuda.stream(stream):
        flush.zero_()


def alg_bytes(bu, moved, pe):
    """Algorithmic bytes of wavelet moves: 28 B per bead-update (read the bead's 24-byte
    position and its 4-byte list link), 24 B per moved bead (write it back), 28 B per pair
    evaluation with a bead outside the support (read it and its link)."""
    return 28.0 * bu + 24.0 * moved + 28.0 * pe


def roofline_block(kernel, bytes_, ms, launches, peak, pk_kind, traffic=None, **extra):
    achieved = bytes_ / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    out = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_kind": pk_kind, "traffic": traffic,
           "alg_bytes_per_launch": bytes_ / max(launches, 1), "launches": launches,
           "avg_launch_us": 1e3 * ms / max(launches, 1),
           "bytes_model": "28 B per bead-update + 24 B per moved bead + 28 B per partner pair evaluation"}
    out.update(extra)
    return out


def ensemble_leg(args, torch, stream, flush, tuner):
    """The uneven-size ensemble advanced as one batch: mixed precision against plain FP64."""
    from paper_1611_09160_gb300 import autotune as A
    from paper_1611_09160_gb300 import inputs as I
    from paper_1611_09160_gb300 import wmcd
    systems = I.ensemble(args.ensemble, 16, 2048, 1e-3, seed=1)
    t0 = time.perf_counter()
    policy, policy_scores = A.choose_policy(systems, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, tuner)
    params = A.ensemble_params(systems, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, seed=100, tuner=tuner, policy=policy)
    tune_s = time.perf_counter() - t0
    out = {"sims": len(systems), "beads": int(sum(s.n_beads for s in systems)), "tune_s": round(tune_s, 2),
           "policy": policy, "policy_bead_updates_per_s": policy_scores,
           "schedules": {k: v["choice"] for k, v in tuner.table.items()}}
    pk, pk_kind = peaks()
    for name, prec in (("mixed", wmcd.MIXED), ("fp64", wmcd.FP64)):
        ps = [dict(p, precision=prec) for p in params]
        need = sum(wmcd.batch_need(p) for p in ps)
        b = wmcd.Batch(capacity=len(systems), pool_bytes=need + (1 << 24))
        t0 = time.perf_counter()
        slots = [b.admit(p, s.pos, s.chain_len) for p, s in zip(ps, systems)]
        admit_s = time.perf_counter() - t0
        shape = tuner.launch_shape(b, sweeps=1) if name == "mixed" else out["mixed"]["launch_shape"]
        b.set_block(*shape)
        b.step(args.warmup, stream=stream)
        torch.cuda.synchronize()
        st0 = [b.sim(k).stats() for k in slots]
        times = []
        for _ in range(args.ensemble_sweeps):
            flush_l2(flush, stream, torch)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(1, stream=stream)
            e1.record(stream)
            times.append((e0, e1))
        stream.synchronize()
        ms = float(sum(a.elapsed_time(c) for a, c in times))
        st1 = [b.sim(k).stats() for k in slots]
        diff = lambda f: sum(getattr(x, f) - getattr(y, f) for x, y in zip(st1, st0))  # noqa: E731
        bu, simt = diff("bead_updates"), diff("sim_time")
        out[name] = {"bead_updates_per_s": bu / (ms * 1e-3), "sim_time_per_s": simt / (ms * 1e-3),
                     "ms_per_batched_sweep": ms / args.ensemble_sweeps, "sweeps": args.ensemble_sweeps,
                     "launches_per_sweep": b.info()["launches_per_sweep"], "launch_shape": list(shape),
                     "pool_mb": round(need / 2**20, 1), "admit_s": round(admit_s, 2),
                     "error_flags": int(max(x.error_flags for x in st1))}
        if name == "mixed":
            # the whole batched sweep against HBM: one graph launch per sweep, the same byte
            # model over every move of every simulation
            byts = alg_bytes(bu, diff("moved_beads"), diff("partner_evals"))
            out["roofline"] = roofline_block("whole batched sweep (graph)", byts, ms, args.ensemble_sweeps,
                                             float(pk.get("hbm_gbs", 6800.0)), pk_kind)
            b.profile(True)
            b.step(2, stream=stream)
            b.profile(False)
            kt = b.kernel_times(stream=stream)
            out["roofline"]["kernel_ms_per_sweep"] = {k: round(v[1] / 2, 4) for k, v in kt.items()}
        b.close()
    out["speedup_mixed_over_fp64"] = out["mixed"]["bead_updates_per_s"] / out["fp64"]["bead_updates_per_s"]
    return out


def large_leg(args, torch, stream, flush, system, workload, candidates, sweeps):
    """One system, schedule from the shipped table (measured when a shape is missing); mixed
    precision against plain FP64 on the same inputs, L2 flushed on the timed stream before each
    timed sweep."""
    from paper_1611_09160_gb300 import autotune as A
    from paper_1611_09160_gb300 import wmcd
    s = system
    tuner = A.Tuner(path=None, warm=1, sweeps=1, seed_table=A.DEFAULT_TABLE)
    t0 = time.perf_counter()
    base = wmcd.default_params(s.n_beads, s.box_L, seed=1, precision=wmcd.MIXED,
                               planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    p = tuner.schedule(base, system=s, candidates=candidates)
    key = A.shape_key(s.n_beads, s.box_L, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC)
    out = {"workload": workload, "n_beads": s.n_beads,
           "schedule": {"colour_K": p["colour_K"], "grid_f": p["grid_f"], "grid_layer": p["grid_layer"][:10]},
           "tuning": {key: tuner.table[key]}, "tune_s": round(time.perf_counter() - t0, 1)}
    for name, prec in (("mixed", wmcd.MIXED), ("fp64", wmcd.FP64)):
        sim = wmcd.Simulation(dict(p, precision=prec), s.pos, s.chain_len, stream=stream)
        sim.sweep(args.warmup, stream=stream)
        st0 = sim.stats(stream=stream)
        ms = timed_steps(sim, sweeps, flush, stream, torch)
        st1 = sim.stats(stream=stream)
        tot = float(np.sum(ms))
        att = sum(st1.attempts) - sum(st0.attempts)
        out[name] = {"bead_updates_per_s": (st1.bead_updates - st0.bead_updates) / (tot * 1e-3),
                     "sim_time_per_s": (st1.sim_time - st0.sim_time) / (tot * 1e-3), "ms_per_sweep": tot / sweeps,
                     "sweeps": sweeps, "deferred_fraction": (sum(st1.deferred) - sum(st0.deferred)) / max(att, 1),
                     "device_mb": sim.device_bytes() // 2**20, "error_flags": st1.error_flags}
        sim.close()
    out["speedup_mixed_over_fp64"] = out["mixed"]["bead_updates_per_s"] / out["fp64"]["bead_updates_per_s"]
    return out


def semidilute_leg(args, torch, stream, flush):
    """C3: homogeneous semi-dilute solution, 4,096 chains x 256 beads (1,048,576) at volume
    fraction 0.05, wavelets + plane waves."""
    from paper_1611_09160_gb300 import inputs as I
    return large_leg(args, torch, stream, flush, I.semidilute_chains(4096, 256, 0.05, seed=1),
                     "semi-dilute chains 4096x256 beads (1,048,576) phi=0.05 L=444.5, wavelet+plane-wave lcut 8",
                     ({"colour_K": 3}, {"colour_K": 2}), args.semidilute_sweeps)


def dilute_leg(args, torch, stream, flush):
    """C2: dilute chains, 256 x 64 beads (16,384) at volume fraction 1e-3, wavelets + plane waves."""
    from paper_1611_09160_gb300 import inputs as I
    return large_leg(args, torch, stream, flush, I.dilute_chains(256, 64, 1e-3, seed=1),
                     "dilute chains 256x64 beads (16,384) phi=1e-3 L=409.4, wavelet+plane-wave lcut 8",
                     ({"colour_K": 2},), args.dilute_sweeps)


def planewave_leg(args, torch, stream, system, params):
    """Plane-wave moves alone on the suspension (a plane wave moves all 5,024,000 beads: read
    each bead, its bond partner and the beads within reach in the cell lists, write the new
    positions; its energy kernel is the streaming kernel of the path)."""
    from paper_1611_09160_gb300 import wmcd
    sim = wmcd.Simulation(params, system.pos, system.chain_len, stream=stream)
    sim.planewave(2, stream=stream)
    q0 = sim.stats(stream=stream)
    sim.kernel_times(stream=stream)
    sim.profile(True)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.planewave(args.planewave_moves, stream=stream)
    b.record(stream)
    stream.synchronize()
    sim.profile(False)
    kt = sim.kernel_times(stream=stream)
    q1 = sim.stats(stream=stream)
    ms = a.elapsed_time(b)
    sim.close()
    return {"bead_updates_per_s": (q1.bead_updates - q0.bead_updates) / (ms * 1e-3), "moves": args.planewave_moves,
            "ms_per_move": ms / args.planewave_moves, "accepted": int(q1.pw_accepts - q0.pw_accepts),
            "kernel_ms": {k: round(v[1], 3) for k, v in kt.items()}}


def serve_leg(args, torch, tuner, policy):
    """Poisson arrivals through the continuous-batching loop (a bounded sample of the stream)."""
    from paper_1611_09160_gb300 import autotune as A
    from paper_1611_09160_gb300 import inputs as I
    from paper_1611_09160_gb300 import serve, wmcd
    systems = I.ensemble(args.serve_requests, 16, 2048, 1e-3, seed=2)
    params = A.ensemble_params(systems, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, seed=200, tuner=tuner, policy=policy)
    arrivals = serve.poisson_arrivals(len(systems), args.serve_rate, seed=3)
    reqs = [serve.Request(k, p, s.pos, s.chain_len, args.serve_sweeps, float(t))
            for k, (p, s, t) in enumerate(zip(params, systems, arrivals))]
    needs = [wmcd.batch_need(p) for p in params]
    pool = int(np.percentile(needs, 50) * args.serve_capacity)
    srv = serve.Server(capacity=args.serve_capacity, pool_bytes=max(pool, max(needs)), chunk=args.serve_chunk)
    rep = srv.run(reqs, realtime=True)
    srv.close()
    sm = rep.summary()
    sm.update({"policy": policy, "rate_per_s": args.serve_rate, "sweeps_per_request": args.serve_sweeps,
               "capacity": args.serve_capacity, "pool_mb": round(pool / 2**20, 1),
               "latency": "per-sweep: CUDA events around every batched sweep; per-request: arrival to result",
               "sample": f"{len(reqs)} requests of the ensemble shape, {args.serve_sweeps} sweeps each (the full "
                         f"stream is 1,024 requests of 10^3 sweeps)"})
    return sm


def drift_run(system, params_of, sweeps, check_every):
    """Mixed precision against plain binary64 from the same start: the largest position
    difference over the box after `sweeps` sweeps, and the first check beyond 1e-5 L."""
    from paper_1611_09160_gb300 import wmcd
    sims = {prec: wmcd.Simulation(params_of(prec), system.pos, system.chain_len) for prec in (wmcd.FP64, wmcd.MIXED)}
    done, first_beyond, dx = 0, None, 0.0
    while done < sweeps:
        k = min(check_every, sweeps - done)
        for sim in sims.values():
            sim.sweep(k)
        done += k
        dx = float(np.max(np.abs(sims[wmcd.MIXED].positions(unwrapped=True) -
                                 sims[wmcd.FP64].positions(unwrapped=True)))) / system.box_L
        if first_beyond is None and dx > 1e-5:
            first_beyond = done
    acc = {prec: int(sim.stats().accepted_total) for prec, sim in sims.items()}
    for sim in sims.values():
        sim.close()
    return {"sweeps": sweeps, "max_abs_dx_over_L": dx, "first_check_beyond_1e-5_L": first_beyond,
            "check_every": check_every, "accepted_fp64": acc[wmcd.FP64], "accepted_mixed": acc[wmcd.MIXED]}


def drift_leg(args):
    """Mixed precision against plain binary64 from the same start, per configuration: the
    32-bead chain (10^4 sweeps) and the dilute chains (10^3 sweeps), wavelets and plane waves.
    Each run decides exactly as the binary64 definition would on its own positions, so the two
    part once a decision close to its threshold falls differently; until then they differ by
    the binary32 rounding of the displacements."""
    from paper_1611_09160_gb300 import inputs as I
    from paper_1611_09160_gb300 import wmcd
    out = {}
    c1 = I.single_chain(32, 64.0, seed=1)
    out["chain32"] = dict(workload="single chain 32 beads, L = 64, wavelets + plane waves, same seed",
                          **drift_run(c1, lambda prec: wmcd.default_params(
                              c1.n_beads, c1.box_L, seed=1, precision=prec,
                              planewave_mode=wmcd.PLANEWAVE_PERIODIC), args.drift_sweeps, 100))
    if args.drift_dilute_sweeps > 0:
        c2 = I.dilute_chains(256, 64, 1e-3, seed=1)
        out["dilute16k"] = dict(workload="dilute chains 256x64 (16,384 beads), wavelets + plane waves, same seed",
                                **drift_run(c2, lambda prec: wmcd.default_params(
                                    c2.n_beads, c2.box_L, seed=1, precision=prec,
                                    planewave_mode=wmcd.PLANEWAVE_PERIODIC), args.drift_dilute_sweeps, 50))
    return out


def combine_ranks(maxed, summed, world, device):
    """Whole-job figures of independent replicas: the slowest rank's times (max) and the
    units of all ranks (sum). No collective is used for a single rank."""
    if world <= 1:
        return list(maxed), list(summed)
    import torch
    import torch.distributed as dist
    t = torch.tensor(list(maxed), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor(list(summed), dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(x) for x in t], [float(x) for x in u]


def timed_steps(sim, steps, flush, stream, torch):
    """Per-step CUDA-event times (ms) of `steps` sweeps, L2 flushed on the stream before each."""
    times = []
    for _ in range(steps):
        flush_l2(flush, stream, torch)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sim.sweep(1, stream=stream)
        b.record(stream)
        times.append((a, b))
    stream.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_1611_09160_gb300 import wmcd
    import __graft_entry__
    torch.cuda.set_device(local_rank)
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    wmcd.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    seed = 1 + rank
    scale = max(1, args.profile_scale)
    system = make_system(seed, None if scale == 1 else
                         dict(SUSPENSION, n_spheres=SUSPENSION["n_spheres"] // scale, n_chains=SUSPENSION["n_chains"] // scale))
    n_sys = system.n_beads
    pk, pk_kind = peaks()
    peak = float(pk.get("hbm_gbs", 6800.0))

    def measure(precision, profile):
        p = make_params(system, precision, seed, sim_id=rank, scaled=scale > 1)
        sim = wmcd.Simulation(p, system.pos, system.chain_len, stream=stream)
        for _ in range(args.warmup):
            sim.sweep(1, stream=stream)
        st0 = sim.stats(stream=stream)
        sim.kernel_times(stream=stream)
        sim.profile(profile)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ms = timed_steps(sim, args.steps, flush, stream, torch)
        torch.cuda.synchronize()
        sim.profile(False)
        kt = sim.kernel_times(stream=stream)
        st1 = sim.stats(stream=stream)
        return sim, ms, st0, st1, kt, p

    with ClockSampler(local_rank) as clk:
        sim, ms, st0, st1, kt, p_mixed = measure(wmcd.MIXED, True)
    clocks = clk.summary()
    total_ms = float(np.sum(ms))
    bu = st1.bead_updates - st0.bead_updates
    simt = st1.sim_time - st0.sim_time
    launches = st1.kernel_launches - st0.kernel_launches
    (total_ms_all,), (bu_all, simt_all, launches_all) = combine_ranks([total_ms], [float(bu), simt, float(launches)],
                                                                     world, dev)
    launches_all = int(launches_all)
    value = bu_all / (total_ms_all * 1e-3)

    # dominant kernel and its roofline (HBM: the path is gathers and pair energies)
    dom = max(kt, key=lambda k: kt[k][1])
    conc_launches, conc_ms = kt["concurrent_wavelet"]
    cbytes = alg_bytes(st1.conc_bead_updates - st0.conc_bead_updates, st1.conc_moved_beads - st0.conc_moved_beads,
                       st1.conc_partner_evals - st0.conc_partner_evals)
    roofline = roofline_block("k_colour_staged (concurrent wavelet moves)", cbytes, conc_ms, conc_launches, peak,
                              pk_kind, traffic=profile_traffic(kernel_sha()), dominant_by_time=dom,
                              kernel_ms={k: round(v[1], 3) for k, v in kt.items()},
                              kernel_launches={k: v[0] for k, v in kt.items()})
    # the whole sweep against the same byte model (every move of every kind)
    sweep_bytes = alg_bytes(bu, st1.moved_beads - st0.moved_beads, st1.partner_evals - st0.partner_evals)
    roofline["whole_sweep_frac"] = sweep_bytes / (total_ms * 1e-3) / 1e9 / peak
    stats = {"accept_fraction": (st1.accepted_total - st0.accepted_total) /
                                max(1, sum(st1.attempts) - sum(st0.attempts) + st1.pw_attempts - st0.pw_attempts),
             "deferred": int(sum(st1.deferred) - sum(st0.deferred)), "rechecks": int(st1.rechecks - st0.rechecks),
             "error_flags": st1.error_flags, "device_mb": sim.device_bytes() // 2**20,
             "schedule": {"colour_K": p_mixed["colour_K"], "grid_f": p_mixed["grid_f"],
                          "grid_layer": p_mixed["grid_layer"][:st1.n_layers]}}

    # end to end through the public API with host buffers: every step copies the positions in
    # from pinned host memory, runs the sweep and copies them back, L2 flushed as above
    h_in = torch.from_numpy(system.pos.copy()).pin_memory()
    h_out = torch.empty((system.n_beads, 3), dtype=torch.float64).pin_memory()
    for _ in range(args.warmup):
        sim.set_positions(h_in, stream=stream)
        sim.sweep(1, stream=stream)
        sim.positions(out=h_out, stream=stream)
    e0 = sim.stats(stream=stream).bead_updates
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush_l2(flush, stream, torch)
        sim.set_positions(h_in, stream=stream)
        sim.sweep(1, stream=stream)
        sim.positions(out=h_out, stream=stream)
    stream.synchronize()
    e_dt = time.perf_counter() - t0
    e_bu = sim.stats(stream=stream).bead_updates - e0
    (e_dt_all,), (e_bu_all,) = combine_ranks([e_dt], [float(e_bu)], world, dev)
    e2e = {"value": e_bu_all / e_dt_all, "unit": UNIT, "h2d_bytes_per_step": 24 * system.n_beads,
           "d2h_bytes_per_step": 24 * system.n_beads,
           "note": "host positions in (pinned), sweep, positions out, L2 flushed, wall clock per rank, max over ranks"}
    sim.close()

    # plain FP64 GPU sweep on the same inputs (the comparison the method is quoted against)
    sim64, ms64, a64, b64, _, _ = measure(wmcd.FP64, False)
    sim64.close()
    (t64_all,), (bu64_all,) = combine_ranks([float(np.sum(ms64))], [float(b64.bead_updates - a64.bead_updates)],
                                            world, dev)
    fp64_value = bu64_all / (t64_all * 1e-3)

    pw = planewave_leg(args, torch, stream, system, p_mixed) if args.planewave_moves > 0 else None
    del system
    from paper_1611_09160_gb300 import autotune as A
    # schedule per shape, measured among 152 copies of the shape (one per SM); shapes already in
    # the table shipped with the package are not measured again
    tuner = A.Tuner(path=None, warm=1, sweeps=2, copies=152, seed_table=A.DEFAULT_TABLE)
    dil = dilute_leg(args, torch, stream, flush) if args.dilute_sweeps > 0 else None
    semi = semidilute_leg(args, torch, stream, flush) if args.semidilute_sweeps > 0 else None
    ens = ensemble_leg(args, torch, stream, flush, tuner) if args.ensemble > 0 else None
    srv = serve_leg(args, torch, tuner, ens["policy"] if ens else "serial_small") if args.serve_requests > 0 else None
    drift = drift_leg(args) if args.drift_sweeps > 0 and rank == 0 else None

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": dict(workload_config(), parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                           **({} if scale == 1 else {"profile_scale": scale, "n_beads": n_sys,
                                                      "workload": f"suspension scaled down {scale}x for profiling"})),
            "sim_time_per_s": simt_all / (total_ms_all * 1e-3),
            "fp64": {"value": fp64_value, "unit": UNIT, "speedup_mixed_over_fp64": value / fp64_value,
                     "ms_per_step": t64_all / args.steps},
            "e2e": e2e, "gpu_launches": launches_all, "clocks": clocks, "roofline": roofline, "stats": stats,
            "plane_wave": pw, "dilute": dil, "semidilute": semi, "batched": ens, "serve": srv,
            "mixed_vs_fp64": drift}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="bound on the timed part of --impl reference (oracle samples)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--planewave-moves", type=int, default=10, help="plane waves on the suspension (0: skip)")
    ap.add_argument("--dilute-sweeps", type=int, default=20, help="timed sweeps of the 16,384-bead leg (0: skip)")
    ap.add_argument("--semidilute-sweeps", type=int, default=3, help="timed sweeps of the 1M-bead leg (0: skip)")
    ap.add_argument("--ensemble", type=int, default=1024, help="simulations in the batched leg (0: skip)")
    ap.add_argument("--ensemble-sweeps", type=int, default=10)
    ap.add_argument("--serve-requests", type=int, default=1024, help="requests in the serving leg (0: skip)")
    ap.add_argument("--serve-sweeps", type=int, default=100)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-capacity", type=int, default=512)
    ap.add_argument("--serve-chunk", type=int, default=10)
    ap.add_argument("--drift-sweeps", type=int, default=10000,
                    help="sweeps of the mixed-against-binary64 drift check on the 32-bead chain (0: skip)")
    ap.add_argument("--profile-scale", type=int, default=1,
                    help="divide the suspension's spheres and chains by this (same density): profiling only")
    ap.add_argument("--drift-dilute-sweeps", type=int, default=1000,
                    help="sweeps of the same check on the dilute chains (0: skip)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
