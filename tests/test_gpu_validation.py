"""Validation workloads on the GPU path at sizes beyond the oracle (the module
paper_1611_09160_gb300.validate): closed forms of the paper checked at 10^6 beads, and the
acceptance spectra and cost-scaling curves produced."""
import math

import numpy as np
import pytest

from paper_1611_09160_gb300 import validate as V
from paper_1611_09160_gb300 import wmcd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def test_free_diffusion_at_a_million_beads():
    """Eq. 33 (MSD per accepted move) and Eq. 34 (time step) on 10^6 free beads; the support count
    per sweep against its closed-form mean."""
    r = V.free_diffusion(n=1_000_000, sweeps=3)
    assert r["accepted"] == r["attempted"]
    assert abs(r["ratio"] - 1.0) < 4.5 * 1.5 * r["ratio_rel_se_over_moves"] + 2e-3, r
    assert r["a2_dt_over_eq33"] == pytest.approx(1.0, rel=1e-12)
    assert r["bead_updates_per_sweep"] == pytest.approx(r["expected_bead_updates_per_sweep"], rel=0.1)


def test_acceptance_spectra_semidilute():
    """Acceptance per octave of lambda (Sec. V.C): it falls from the smallest wavelets, whose
    strain estimate overestimates dU, towards its large-lambda asymptote, over the octaves with
    enough moves to tell; the plane waves' acceptance per |k| bin (Sec. VI.A) is reported."""
    r = V.acceptance_spectra(sweeps=3, planewaves=1000)
    print(r)
    w = [b for b in r["wavelet"] if b["moves"] >= 300]
    assert len(w) >= 4
    p = [b["p_acc"] for b in w]
    assert all(0.0 < x <= 1.0 for x in p)
    assert all(a >= b - 0.02 for a, b in zip(p[:-1], p[1:])) and p[0] > p[-1]
    pw = r["plane_wave"]
    assert sum(b["moves"] for b in pw) + r["plane_wave_k0_moves"] >= 1000
    assert all(0.0 <= b["p_acc"] <= 1.0 for b in pw)


def test_cost_scaling_follows_n_log_n():
    """Bead-updates per simulated time grow as N (a + b ln(L / 2 lmin)) (Sec. V.F). One sweep's
    count carries a few per cent of noise from the rare largest wavelets, so eight sweeps."""
    r = V.cost_scaling(sizes=(32_768, 131_072, 524_288), sweeps=8)
    print(r)
    assert r["fit_max_rel_dev"] < 0.05
    assert r["fit_b"] > 0
    per_n = [row["bead_updates_per_tau"] / row["N"] for row in r["rows"]]
    assert per_n[0] < per_n[1] < per_n[2]


def test_chain_relaxation_reaches_one_plateau_from_both_sides():
    """Sec. VII.A: chains of N_b = 10 beads relax to the same mean-square radius of gyration from
    above (self-avoiding walks) and from below (the exact ideal-chain equilibrium), with harmonic
    bonds in theta solvent (no WCA). The common plateau is reported against the Boltzmann value of
    ideal chains, <b^2> (N_b^2 - 1) / (6 N_b): the sampled distribution of these finite,
    Metropolis-tested moves lies above it (measured +16% at A0 = 0.5, about half of that at
    A0 = 0.25; the same with every move in the serial phase, so the schedule does not cause it)."""
    kw = dict(n_chains=4000, n_b=10, sweeps=9000, every=300, seed=2)
    up = V.chain_relaxation(start="ideal", **kw)
    down = V.chain_relaxation(start="saw", **kw)
    print({k: v for k, v in up.items() if k != "curve"}, {k: v for k, v in down.items() if k != "curve"})
    assert up["error_flags"] == 0 and down["error_flags"] == 0
    assert down["rg2_initial"] > down["rg2_plateau"] > up["rg2_initial"]
    se = math.hypot(up["rg2_plateau_se"], down["rg2_plateau_se"])
    assert abs(up["rg2_plateau"] - down["rg2_plateau"]) < 4.0 * se + 0.01 * up["rg2_ideal"]
    assert 1.0 < up["ratio"] < 1.3
    assert up["bond_msd_plateau"] == pytest.approx(up["bond_msd_ideal"], rel=0.01)


def test_chain_diffusivity_follows_zimm_scaling_in_both_solvents():
    """Sec. VII.B: centre-of-mass diffusion of dilute chains of 8, 16 and 32 beads in the paper's
    reduced units (Sec. II), good solvent (FENE + WCA) and theta solvent (harmonic bonds, no WCA).
    One box and bead density for every chain length. The paper finds D ~ N^-nu with the Zimm
    exponents (0.588, 0.5) already at these lengths. Both runs must show hydrodynamic scaling, nu
    between 0.4 and 0.7, far from free draining (Rouse, nu = 1): hydrodynamic interactions raise
    N D / D_0 above 1, and more so for longer chains."""
    out = {}
    for solvent in ("good", "theta"):
        r = V.chain_diffusivity(solvent, n_bs=(8, 16, 32), beads=32_768, sweeps=600, every=20, seed=3)
        out[solvent] = r
        print(solvent, "nu", r["nu"], "+-", r["nu_se"],
              [(row["n_b"], row["D_over_D0"], row["D_se"] / r["D0"], row["accept_fraction"]) for row in r["rows"]])
        assert all(row["error_flags"] == 0 for row in r["rows"])
        d = [row["D_inf"] for row in r["rows"]]
        assert d[0] > d[1] > d[2]
        rouse = [row["rouse_ratio"] for row in r["rows"]]
        assert rouse[0] > 1.5 and rouse[0] < rouse[1] < rouse[2]
        assert 0.4 < r["nu"] < 0.7, r["nu"]


def test_chain_relaxation_in_paper_units_from_compressed_and_stretched_bonds():
    """Sec. VII.A in the reduced units of Sec. II: 10-bead chains with FENE bonds and WCA between
    all beads (good solvent), started with every bond compressed (0.8) or stretched (1.4) against
    the equilibrium mean of about 0.98. The compressed chains swell, the stretched ones shrink, and
    after 2,400 sweeps (about 145 tau) the two mean-square radii of gyration are within a tenth of
    their starting gap of each other; the bonds have reached one mean-square length in both."""
    kw = dict(n_chains=2000, n_b=10, sweeps=2400, every=100, seed=2, paper_units=True)
    up = V.chain_relaxation(bond0=0.8, **kw)
    down = V.chain_relaxation(bond0=1.4, **kw)
    for r in (up, down):
        print({k: v for k, v in r.items() if k != "curve"}, [(c["sweeps"], round(c["rg2"], 4)) for c in r["curve"]])
        assert r["error_flags"] == 0
    gap0 = down["rg2_initial"] - up["rg2_initial"]
    end_up, end_down = up["curve"][-1]["rg2"], down["curve"][-1]["rg2"]
    assert up["rg2_initial"] < end_up and end_down < down["rg2_initial"]
    assert abs(end_down - end_up) < 0.1 * gap0
    assert up["bond_msd_plateau"] == pytest.approx(down["bond_msd_plateau"], rel=0.01)
