"""Validation workloads on the GPU path, at sizes the CPU oracle cannot reach.

Each workload runs through the library's public API and compares what it measures with a
closed form of the paper, or reports the spectra the paper plots:

* ``free_diffusion``: free spheres (no interactions), so every move is accepted. The mean
  squared displacement per accepted move is Eq. 33, (2/105) A0^2 N_lambda (1/lmin - 1/lmax) / N
  (wavelets only), and the bead-updates of a sweep have the exact expectation
  N (1 + (N - 1) (4 pi / 3) <lambda^3> / L^3) with <lambda^3> = N_lambda ln(lmax / lmin)
  (the picked bead plus the others, uniform in the box).
* ``acceptance_spectra``: the acceptance of wavelet moves per octave of lambda (Sec. V.C, the
  paper's Fig. 2) and of plane waves per |k| bin (Sec. VI.A, Fig. 6).
* ``cost_scaling``: bead-updates and wall time per unit simulated time for homogeneous systems
  of growing N at fixed density (Sec. V.F: cost per simulated time ~ N ln N), with the
  algorithmic count against N (1 + c ln(L / (2 lmin))).
* ``chain_relaxation``: the radius of gyration of N_b = 10 chains relaxing from self-avoiding
  walks (Sec. VII.A), and in theta solvent (no WCA), started from the ideal-chain equilibrium,
  its plateau against the exact ideal-chain value (the dynamics must keep that equilibrium).

``python -m paper_1611_09160_gb300.validate --out report.json`` runs them all at full size.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import inputs as I
from . import wmcd

LAMBDA_A = 1.0 / (1.125 - math.log(2.0))      # Eq. 42 for the tapered wavelet


def n_lambda(lmin: float, lmax: float) -> float:
    """Normalisation of P_lambda = N_lambda lambda^-4 on [lmin, lmax] (Eq. 32)."""
    return 3.0 / (lmin ** -3 - lmax ** -3)


def eq33_per_move(A0: float, lmin: float, lmax: float, N: int) -> float:
    """Eq. 33: mean squared displacement of one bead per wavelet move (M4 / (2 pi)^3 = 1/105)."""
    return 2.0 / 105.0 * A0 ** 2 * n_lambda(lmin, lmax) * (1.0 / lmin - 1.0 / lmax) / N


def expected_support(N: int, L: float, lmin: float, lmax: float) -> float:
    """Mean support of a bead-centred move among beads uniform in the box."""
    lam3 = n_lambda(lmin, lmax) * math.log(lmax / lmin)
    return 1.0 + (N - 1) * (4.0 * math.pi / 3.0) * lam3 / L ** 3


def free_diffusion(n: int = 1_000_000, phi: float = 1e-3, sweeps: int = 4, groups: int = 64, seed: int = 1,
                   precision: int = wmcd.MIXED) -> dict:
    """Free spheres at volume fraction phi (WCA off, so no move is rejected): MSD per accepted move
    against Eq. 33 with a standard error from `groups` random groups of beads, and bead-updates
    per sweep against their exact expectation."""
    # beads uniform in the box (no interactions, so overlaps are allowed): the support count then
    # has the closed-form mean of expected_support
    L = I.box_for_volume_fraction(n, phi)
    pos = np.minimum(np.random.default_rng(seed).random((n, 3)) * L, np.nextafter(L, 0.0))
    p = wmcd.default_params(n, L, seed=seed, precision=precision, bond_type=wmcd.BOND_NONE, wca_eps=0.0)
    sim = wmcd.Simulation(p, pos, np.ones(n, dtype=np.int32))
    x0 = sim.positions(unwrapped=True)
    st0 = sim.stats()
    t0 = time.perf_counter()
    sim.sweep(sweeps)
    x1 = sim.positions(unwrapped=True)
    wall = time.perf_counter() - t0
    st1 = sim.stats()
    sim.close()
    acc = st1.accepted_total - st0.accepted_total
    att = sum(st1.attempts) - sum(st0.attempts)
    d2 = np.sum((x1 - x0) ** 2, axis=1)
    g = np.random.default_rng(seed).permutation(len(d2)) % groups
    per = np.array([d2[g == k].mean() for k in range(groups)]) / acc
    want = eq33_per_move(p["A0"], p["lambda_min"], p["lambda_max"], n)
    bu = (st1.bead_updates - st0.bead_updates) / sweeps
    bu_want = (att / sweeps) * expected_support(n, L, p["lambda_min"], p["lambda_max"])
    a = p["lambda_min"] / LAMBDA_A
    # the spread over moves: with E[sum_i dr_i^2 | lambda] = (2/105) A0^2 lambda^2 (Eq. 33 per scale),
    # the relative standard deviation of one move's contribution is about
    # sqrt((lmax - lmin) / N_lambda) / (1/lmin - 1/lmax); over `acc` moves it falls as acc^-1/2
    lmin, lmax = p["lambda_min"], p["lambda_max"]
    rel_move = math.sqrt((lmax - lmin) / n_lambda(lmin, lmax)) / (1.0 / lmin - 1.0 / lmax)
    return {"workload": f"free beads uniform in the box, N = {n:,}, phi = {phi}, L = {L:.1f}, wavelets only",
            "sweeps": sweeps, "accepted": int(acc), "attempted": int(att),
            "msd_per_move": float(per.mean()), "msd_per_move_se": float(per.std(ddof=1) / math.sqrt(groups)),
            "eq33_per_move": want, "ratio": float(per.mean() / want),
            "ratio_rel_se_over_moves": rel_move / math.sqrt(max(acc, 1)),
            "bead_updates_per_sweep": bu, "expected_bead_updates_per_sweep": bu_want,
            "time_step": st1.dt_move, "a2_dt_over_eq33": st1.dt_move * a * a / want, "wall_s": wall}


def acceptance_spectra(system=None, sweeps: int = 3, kbins: int = 8, seed: int = 1,
                       planewave_mode: int = wmcd.PLANEWAVE_PERIODIC_FULL, lcut: int = 15, lambda_max=None,
                       planewaves: int = 1000) -> dict:
    """Acceptance of wavelet moves per octave of lambda and of plane waves per |k| bin on a
    semi-dilute solution (default: 1,024 chains x 64 beads at volume fraction 0.05)."""
    s = system if system is not None else I.semidilute_chains(1024, 64, 0.05, seed=seed)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, precision=wmcd.MIXED, planewave_mode=planewave_mode,
                            lcut=lcut)
    if lambda_max is not None:
        p["lambda_max"] = float(lambda_max)
    sim = wmcd.Simulation(p, s.pos, s.chain_len)
    st0 = sim.stats()
    ks, outs = [], []
    for _ in range(sweeps):
        sim.sweep(1)
        k = sim.trace_pw_k()
        o, _ = sim.trace(-1)
        ks.append(k)
        outs.append(o)
    # plane waves are rare in a sweep: a block of direct plane-wave moves adds to the spectrum
    sim.planewave(planewaves)
    ks.append(sim.trace_pw_k())
    outs.append(sim.trace(-1)[0])
    st1 = sim.stats()
    sim.close()
    nl = int(st1.n_layers)
    lo, hi = [], []
    for l in range(nl):
        lo.append(p["lambda_min"] * 2 ** l)
        hi.append(min(p["lambda_min"] * 2 ** (l + 1), p["lambda_max"]))
    att = np.array([st1.attempts[l] - st0.attempts[l] for l in range(nl)], dtype=float)
    acc = np.array([st1.accepts[l] - st0.accepts[l] for l in range(nl)], dtype=float)
    k = np.concatenate(ks) if ks else np.zeros((0, 3))
    o = np.concatenate(outs) if outs else np.zeros(0)
    kk = np.linalg.norm(k, axis=1) * (2 * math.pi / s.box_L)
    spec = []
    nz = kk > 0
    if nz.any():
        edges = np.geomspace(kk[nz].min(), kk[nz].max() * (1 + 1e-12), kbins + 1)
        for a, b in zip(edges[:-1], edges[1:]):
            m = (kk >= a) & (kk < b)
            if m.any():
                spec.append({"k_lo": float(a), "k_hi": float(b), "moves": int(m.sum()),
                             "p_acc": float(np.mean(o[m] == 1))})
    return {"workload": f"semi-dilute, N = {s.n_beads:,}, L = {s.box_L:.1f}",
            "wavelet": [{"lambda_lo": lo[l], "lambda_hi": hi[l], "moves": int(att[l]),
                         "p_acc": float(acc[l] / att[l]) if att[l] else None} for l in range(nl)],
            "plane_wave": spec, "plane_wave_k0_moves": int(np.sum(~nz))}


def cost_scaling(sizes=(65_536, 262_144, 1_048_576), phi: float = 0.05, sweeps: int = 2, seed: int = 1) -> dict:
    """Bead-updates and wall time per unit simulated time for homogeneous free spheres of growing N
    at fixed volume fraction (WCA on, wavelets and plane waves): Sec. V.F predicts a cost per
    simulated time ~ N ln N. The algorithmic count is fitted to N (a + b ln(L / (2 lmin)))."""
    rows = []
    import torch
    for n in sizes:
        s = I.free_spheres(int(n), phi, seed=seed)
        p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, precision=wmcd.MIXED, bond_type=wmcd.BOND_NONE,
                                planewave_mode=wmcd.PLANEWAVE_PERIODIC_FULL, lcut=15)
        sim = wmcd.Simulation(p, s.pos, s.chain_len)
        sim.sweep(1)
        torch.cuda.synchronize()
        st0 = sim.stats()
        t0 = time.perf_counter()
        sim.sweep(sweeps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st1 = sim.stats()
        sim.close()
        tau = st1.sim_time - st0.sim_time
        rows.append({"N": int(n), "L": s.box_L, "bead_updates_per_tau": (st1.bead_updates - st0.bead_updates) / tau,
                     "wall_s_per_tau": wall / tau, "log_ratio": math.log(s.box_L / (2 * p["lambda_min"]))})
    X = np.array([[r["N"], r["N"] * r["log_ratio"]] for r in rows], dtype=float)
    y = np.array([r["bead_updates_per_tau"] for r in rows])
    coef, *_ = np.linalg.lstsq(X, y, rcond=None)
    fit = X @ coef
    slope = np.polyfit(np.log([r["N"] for r in rows]), np.log([r["wall_s_per_tau"] for r in rows]), 1)[0]
    return {"rows": rows, "fit_a": float(coef[0]), "fit_b": float(coef[1]),
            "fit_max_rel_dev": float(np.max(np.abs(fit - y) / y)), "wall_exponent": float(slope)}


def ideal_bond_msd(k: float, r0: float, kT: float = 1.0) -> float:
    """<b^2> of a harmonic bond U = (k/2)(b - r0)^2 at temperature kT: b has the density
    b^2 exp(-U/kT) on b > 0 (the bond vector's Boltzmann weight in three dimensions)."""
    from scipy import integrate
    w = lambda b: b * b * math.exp(-0.5 * k * (b - r0) ** 2 / kT)
    hi = r0 + 40.0 * math.sqrt(kT / k)
    z = integrate.quad(w, 0.0, hi, epsabs=0.0, epsrel=1e-12, limit=200)[0]
    m2 = integrate.quad(lambda b: b * b * w(b), 0.0, hi, epsabs=0.0, epsrel=1e-12, limit=200)[0]
    return m2 / z


def ideal_chains(n_chains: int, n_b: int, box_L: float, k: float, r0: float, kT: float = 1.0, seed: int = 1):
    """Chains drawn from the ideal-chain equilibrium of harmonic bonds: independent bond vectors,
    isotropic, lengths with density b^2 exp(-(k/2)(b - r0)^2 / kT) (sampled through its tabulated
    distribution function); first beads uniform in the box; positions wrapped into [0, L)."""
    rng = np.random.default_rng(seed)
    sd = math.sqrt(kT / k)
    grid = np.linspace(max(0.0, r0 - 12 * sd), r0 + 12 * sd, 40001)
    w = grid * grid * np.exp(-0.5 * k * (grid - r0) ** 2 / kT)
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (w[1:] + w[:-1]) * np.diff(grid))])
    b = np.interp(rng.random((n_chains, n_b - 1)), cdf / cdf[-1], grid)
    u = rng.normal(size=(n_chains, n_b - 1, 3))
    u /= np.linalg.norm(u, axis=2, keepdims=True)
    x0 = rng.random((n_chains, 1, 3)) * box_L
    x = np.concatenate([x0, x0 + np.cumsum(b[:, :, None] * u, axis=1)], axis=1).reshape(-1, 3)
    return np.minimum(np.mod(x, box_L), np.nextafter(box_L, 0.0))


def chain_relaxation(n_chains: int = 20_000, n_b: int = 10, phi: float = 1e-3, sweeps: int = 600, every: int = 20,
                     seed: int = 1, wca_eps: float = 0.0, start: str = "saw", A0: float = 0.5, **sched) -> dict:
    """Radius of gyration of N_b-bead chains (Sec. VII.A uses N_b = 10) with harmonic bonds
    (k = 100 kT/a^2, rest length 2a), wavelets and plane waves, from self-avoiding walks
    (start="saw": the relaxation curve) or from the ideal-chain equilibrium (start="ideal"). With
    WCA off (theta solvent) the chains are ideal: at equilibrium their bond vectors are independent,
    so the Boltzmann value of <R_g^2> is <b^2> (N_b^2 - 1) / (6 N_b), with <b^2> of one harmonic
    bond; the measured plateau (each chain's average over the last third of the run, the standard
    error from the spread over chains) is compared with it. With WCA on (good solvent) the curve is
    reported."""
    s = I.dilute_chains(n_chains, n_b, phi, seed=seed)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, precision=wmcd.MIXED, wca_eps=wca_eps,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC, A0=A0, **sched)
    pos = s.pos if start == "saw" else ideal_chains(n_chains, n_b, s.box_L, p["bond_k"], p["bond_r0"], p["kT"],
                                                      seed=seed)
    sim = wmcd.Simulation(p, pos, s.chain_len)

    def measure():
        # each chain rebuilt from its bond vectors taken at minimum image (a chain may straddle a
        # face of the periodic box; its bonds are far shorter than L / 2)
        x = sim.positions(unwrapped=True).reshape(n_chains, n_b, 3)
        d = np.diff(x, axis=1)
        d -= s.box_L * np.round(d / s.box_L)
        y = np.concatenate([np.zeros((n_chains, 1, 3)), np.cumsum(d, axis=1)], axis=1)
        c = y - y.mean(axis=1, keepdims=True)
        return (c * c).sum(axis=2).mean(axis=1), float((d * d).sum(axis=2).mean())

    samples, bonds, curve = [], [], []
    r, b2 = measure()
    curve.append({"sweeps": 0, "sim_time": 0.0, "rg2": float(r.mean()), "b2": b2})
    for k in range(sweeps // every):
        sim.sweep(every)
        r, b2 = measure()
        samples.append(r)
        bonds.append(b2)
        curve.append({"sweeps": (k + 1) * every, "sim_time": sim.stats().sim_time, "rg2": float(r.mean()), "b2": b2})
    st = sim.stats()
    sim.close()
    late = np.array(samples[(2 * len(samples)) // 3:])     # last third of the run
    per_chain = late.mean(axis=0)
    out = {"n_chains": n_chains, "n_b": n_b, "box_L": s.box_L, "wca_eps": wca_eps, "start": start, "A0": A0,
           "curve": curve,
           "rg2_initial": curve[0]["rg2"], "rg2_plateau": float(per_chain.mean()),
           "rg2_plateau_se": float(per_chain.std(ddof=1) / math.sqrt(n_chains)),
           "bond_msd_plateau": float(np.mean(bonds[(2 * len(bonds)) // 3:])), "error_flags": st.error_flags,
           "accept_fraction": st.accepted_total / max(1, sum(st.attempts) + st.pw_attempts)}
    if wca_eps == 0.0:
        b2 = ideal_bond_msd(p["bond_k"], p["bond_r0"], p["kT"])
        out["bond_msd_ideal"] = b2
        out["rg2_ideal"] = b2 * (n_b * n_b - 1) / (6.0 * n_b)
        out["ratio"] = out["rg2_plateau"] / out["rg2_ideal"]
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    wmcd.build()
    wmcd.load()
    rep = {"free_diffusion": free_diffusion(), "acceptance_spectra": acceptance_spectra(),
           "cost_scaling": cost_scaling(), "chain_relaxation_theta": chain_relaxation(),
           "chain_equilibrium_theta": chain_relaxation(start="ideal"),
           "chain_relaxation_good": chain_relaxation(wca_eps=1.0)}
    with open(a.out, "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
