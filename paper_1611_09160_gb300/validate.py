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
  its plateau against the exact ideal-chain value (the dynamics must keep that equilibrium); and
  the paper's own FENE + WCA chains in its reduced units from compressed and stretched bonds.
* ``chain_diffusivity``: the centre-of-mass diffusion constant D(N_b) of dilute chains in good
  and theta solvent in the paper's reduced units (Sec. VII.B), with the periodic-image
  correction of Eq. 60, and the exponent of D ~ N_b^-nu.

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
                     seed: int = 1, wca_eps: float = 0.0, start: str = "saw", A0: float = 0.5,
                     paper_units: bool = False, bond0: float = 0.97, chain_gap: float = 25.0, **sched) -> dict:
    """Radius of gyration of N_b-bead chains (Sec. VII.A uses N_b = 10), wavelets and plane waves.

    Bench units (default): harmonic bonds (k = 100 kT/a^2, rest length 2a), from self-avoiding
    walks (start="saw": the relaxation curve) or from the ideal-chain equilibrium (start="ideal").
    With WCA off (theta solvent) the chains are ideal: at equilibrium their bond vectors are
    independent, so the Boltzmann value of <R_g^2> is <b^2> (N_b^2 - 1) / (6 N_b), with <b^2> of one
    harmonic bond; the measured plateau (each chain's average over the last third of the run, the
    standard error from the spread over chains) is compared with it. With WCA on (good solvent)
    the curve is reported.

    paper_units=True: the system of Sec. VII.A in Sec. II's reduced units, FENE bonds and WCA
    between all beads (good solvent), from self-avoiding walks whose bonds start at ``bond0``,
    compressed or stretched against the equilibrium mean of about 0.98, one chain per cube of side
    ``chain_gap``. The curve and the plateau are reported (the paper compares them with a value
    from another study that its text does not give)."""
    if paper_units:
        if start != "saw":
            raise ValueError("in paper units the chains start from self-avoiding walks of bond bond0")
        L = chain_gap * n_chains ** (1.0 / 3.0)
        s = I.make_system([n_b] * n_chains, 0, L, seed, bond=bond0, min_dist=0.999 * min(SIGMA_BAR, bond0))
        p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, precision=wmcd.MIXED,
                                planewave_mode=wmcd.PLANEWAVE_PERIODIC, A0=A0, **paper_unit_params("good"), **sched)
        wca_eps = p["wca_eps"]
    else:
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
           "paper_units": paper_units, "bond0": bond0 if paper_units else p["bond_r0"],
           "curve": curve,
           "rg2_initial": curve[0]["rg2"], "rg2_plateau": float(per_chain.mean()),
           "rg2_plateau_se": float(per_chain.std(ddof=1) / math.sqrt(n_chains)),
           "bond_msd_plateau": float(np.mean(bonds[(2 * len(bonds)) // 3:])), "error_flags": st.error_flags,
           "accept_fraction": st.accepted_total / max(1, sum(st.attempts) + st.pw_attempts)}
    if wca_eps == 0.0 and not paper_units:
        b2 = ideal_bond_msd(p["bond_k"], p["bond_r0"], p["kT"])
        out["bond_msd_ideal"] = b2
        out["rg2_ideal"] = b2 * (n_b * n_b - 1) / (6.0 * n_b)
        out["ratio"] = out["rg2_plateau"] / out["rg2_ideal"]
    return out


# Sec. II's reduced units (length 2^(1/6) sigma, energy eps), chosen there to match the polymer
# systems of the benchmarks the paper compares with
SIGMA_BAR = 2.0 ** (-1.0 / 6.0)
K_FENE_BAR = 7.0 * 2.0 ** (1.0 / 3.0)
R0_FENE_BAR = 2.0 * 2.0 ** (-1.0 / 6.0)
LMIN_BAR = 0.700
KT_BAR = 1.2
R0_THETA_BAR = 0.9691          # Sec. VII.B: the harmonic rest length matching the good solvent's mean bond
BOND_START_BAR = 0.97          # bond length of the generated starting walks, near both solvents' mean
PERIODIC_SELF = 2.837          # Eq. 60: periodic images lower the self-mobility by 2.837 a / L


def paper_unit_params(solvent: str) -> dict:
    """Potential and wavelet parameters of Sec. II in its reduced units. Good solvent: FENE bonds
    (Eq. 1) and WCA (Eq. 2) between all beads. Theta solvent (Sec. VII.B): WCA off and the bond
    (3/2) k_FENE (r - r0)^2, i.e. k = 3 k_FENE in the library's harmonic form (k/2)(r - r0)^2."""
    base = dict(lambda_min=LMIN_BAR, kT=KT_BAR, wca_sigma=SIGMA_BAR)
    if solvent == "good":
        return dict(base, wca_eps=1.0, bond_type=wmcd.BOND_FENE, bond_k=K_FENE_BAR, fene_R0=R0_FENE_BAR)
    if solvent == "theta":
        return dict(base, wca_eps=0.0, bond_type=wmcd.BOND_HARMONIC, bond_k=3.0 * K_FENE_BAR,
                    bond_r0=R0_THETA_BAR)
    raise ValueError(f"solvent must be 'good' or 'theta', not {solvent!r}")


def com_diffusion(com, times, max_lag: int | None = None, groups: int = 8) -> dict:
    """D = <|dR_CoM|^2> / (6 t) (Sec. VII.B) from sampled centre-of-mass trajectories, over every
    time origin. ``com`` is (samples, chains, 3), in coordinates that are continuous in time;
    ``times`` the simulated time of each sample. For each lag of m = 1..max_lag samples: the mean
    square displacement over all origins and chains, and the mean time lag t_m; D is the
    least-squares slope through the origin of MSD against 6 t_m. Its standard error is the spread
    of the same estimate over ``groups`` disjoint sets of chains (motion that one large wavelet
    gives to several chains at once correlates them, which this error does not include)."""
    com = np.asarray(com, dtype=np.float64)
    times = np.asarray(times, dtype=np.float64)
    n_s, n_c = com.shape[0], com.shape[1]
    if n_s < 2 or times.shape != (n_s,):
        raise ValueError("need at least two samples and one time per sample")
    max_lag = n_s - 1 if max_lag is None else max(1, min(int(max_lag), n_s - 1))
    lags = range(1, max_lag + 1)
    t = np.array([float((times[m:] - times[:-m]).mean()) for m in lags])

    def slope(c):
        msd = np.array([float(((c[m:] - c[:-m]) ** 2).sum(axis=2).mean()) for m in lags])
        return float((msd * t).sum() / (6.0 * (t * t).sum())), msd

    D, msd = slope(com)
    parts = [p for p in np.array_split(np.arange(n_c), min(groups, n_c)) if len(p)]
    Dg = np.array([slope(com[:, p])[0] for p in parts])
    se = float(Dg.std(ddof=1) / math.sqrt(len(Dg))) if len(Dg) > 1 else float("nan")
    return {"D": D, "D_se": se, "lag_time": t.tolist(), "msd": msd.tolist()}


def fit_exponent(n, D, se) -> tuple[float, float]:
    """nu and its standard error in D ~ N^-nu: weighted least squares of ln D on ln N, the weight
    of each point (D / se)^2."""
    x = np.log(np.asarray(n, dtype=np.float64))
    y = np.log(np.asarray(D, dtype=np.float64))
    w = (np.asarray(D, dtype=np.float64) / np.asarray(se, dtype=np.float64)) ** 2
    xm = (w * x).sum() / w.sum()
    ym = (w * y).sum() / w.sum()
    sxx = (w * (x - xm) ** 2).sum()
    b = (w * (x - xm) * (y - ym)).sum() / sxx
    return float(-b), float(math.sqrt(1.0 / sxx))


def chain_diffusivity(solvent: str = "good", n_bs=(8, 16, 32), beads: int = 32_768, bead_gap: float = 8.0,
                      sweeps: int = 600, every: int = 20, max_lag: int = 10, seed: int = 1, A0: float = 0.5,
                      **sched) -> dict:
    """Centre-of-mass diffusion of dilute chains of N_b beads (Sec. VII.B) in Sec. II's reduced
    units, wavelets and plane waves, mixed precision. For each N_b, beads / N_b self-avoiding walks
    (bond 0.97, no two beads closer than sigma) in one periodic box of side bead_gap * beads^(1/3)
    for every N_b, so the bead density is the same at every chain length (the wavelet amplitude
    A0 lambda / sqrt(n) of Eq. 29 counts every bead in the ball, the other chains' included). The
    chains' centres of mass are sampled every ``every`` sweeps from the unwrapped positions; D by
    ``com_diffusion``, then corrected for the periodic images by Eq. 60:
    D_inf = D_L + 2.837 D_0 a / L, with D_0 = a^2 / 6 (tau units) the diffusivity of one free sphere
    and a = lambda_min / lambda_a (Eq. 42). D / D_0 is the bracket of the paper's series for D: the
    free-draining (Rouse) value is 1 / N_b; hydrodynamic interactions raise it. nu is fitted to
    D_inf ~ N_b^-nu (Zimm scaling: 0.588 in good, 0.5 in theta solvent; free draining: 1)."""
    a = LMIN_BAR / LAMBDA_A
    D0 = a * a / 6.0
    rows = []
    for n_b in n_bs:
        n_chains = max(2, beads // n_b)
        L = bead_gap * beads ** (1.0 / 3.0)
        s = I.make_system([n_b] * n_chains, 0, L, seed, bond=BOND_START_BAR, min_dist=SIGMA_BAR)
        p = wmcd.default_params(s.n_beads, s.box_L, seed=seed, precision=wmcd.MIXED, A0=A0,
                                planewave_mode=wmcd.PLANEWAVE_PERIODIC, **paper_unit_params(solvent), **sched)
        sim = wmcd.Simulation(p, s.pos, s.chain_len)
        t0 = time.perf_counter()
        com, times = [], []
        for k in range(sweeps // every + 1):
            if k:
                sim.sweep(every)
            com.append(sim.positions(unwrapped=True).reshape(n_chains, n_b, 3).mean(axis=1))
            times.append(sim.stats().sim_time)
        wall = time.perf_counter() - t0
        st = sim.stats()
        sim.close()
        r = com_diffusion(np.stack(com), np.array(times), max_lag=max_lag)
        corr = PERIODIC_SELF * D0 * a / L
        rows.append({"n_b": n_b, "n_chains": n_chains, "box_L": L, "sim_time": times[-1], "wall_s": wall,
                     "D_L": r["D"], "D_se": r["D_se"], "D_inf": r["D"] + corr, "periodic_correction": corr,
                     "D_over_D0": (r["D"] + corr) / D0, "rouse_ratio": n_b * (r["D"] + corr) / D0,
                     "lag_time": r["lag_time"], "msd": r["msd"], "error_flags": st.error_flags,
                     "accept_fraction": st.accepted_total / max(1, sum(st.attempts) + st.pw_attempts)})
    nu, nu_se = fit_exponent([r["n_b"] for r in rows], [r["D_inf"] for r in rows], [r["D_se"] for r in rows])
    return {"solvent": solvent, "a": a, "D0": D0, "A0": A0, "rows": rows, "nu": nu, "nu_se": nu_se,
            "nu_zimm": 0.588 if solvent == "good" else 0.5}


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
           "chain_relaxation_good": chain_relaxation(wca_eps=1.0),
           "chain_relaxation_paper_compressed": chain_relaxation(sweeps=6000, every=100, paper_units=True, bond0=0.8),
           "chain_relaxation_paper_stretched": chain_relaxation(sweeps=6000, every=100, paper_units=True, bond0=1.4),
           "chain_diffusivity_good": chain_diffusivity("good", n_bs=(8, 16, 32, 64), sweeps=2000),
           "chain_diffusivity_theta": chain_diffusivity("theta", n_bs=(8, 16, 32, 64), sweeps=2000)}
    with open(a.out, "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep, indent=1))


if __name__ == "__main__":
    main()
