"""Host logic of the validation workloads (no GPU): the centre-of-mass diffusion estimator on
synthetic Brownian trajectories with a known D, the exponent fit, and the reduced units of Sec. II
that the chain-diffusivity workload of Sec. VII.B runs in."""
import math

import numpy as np
import pytest

from paper_1611_09160_gb300 import validate as V
from paper_1611_09160_gb300 import wmcd


def brownian(D, n_chains, n_samples, seed):
    """Free Brownian centres: each step Gaussian with variance 2 D dt per axis, the time steps
    themselves random (the simulated time of a block of sweeps varies)."""
    rng = np.random.default_rng(seed)
    dt = rng.uniform(0.5, 1.5, n_samples - 1)
    steps = rng.normal(size=(n_samples - 1, n_chains, 3)) * np.sqrt(2.0 * D * dt)[:, None, None]
    com = np.concatenate([rng.random((1, n_chains, 3)) * 50.0, steps], axis=0).cumsum(axis=0)
    return com, np.concatenate([[0.0], dt.cumsum()])


def test_com_diffusion_recovers_a_known_diffusivity():
    est = [V.com_diffusion(*brownian(0.3, 512, 31, seed), max_lag=10) for seed in range(40)]
    D = np.array([e["D"] for e in est])
    se = np.array([e["D_se"] for e in est])
    # unbiased: the mean of 40 estimates within 4 standard errors of that mean
    assert abs(D.mean() - 0.3) < 4.0 * D.std(ddof=1) / math.sqrt(len(D))
    # the quoted error is of the size of the actual spread of the estimate
    assert 0.5 < se.mean() / D.std(ddof=1) < 2.0
    e = est[0]
    assert len(e["msd"]) == len(e["lag_time"]) == 10
    assert all(b > a for a, b in zip(e["lag_time"][:-1], e["lag_time"][1:]))


def test_com_diffusion_sees_only_displacements():
    """A constant offset per chain (a chain that straddled a face when its unwrapped coordinates
    started) changes nothing; a uniform drift enters as its square."""
    com, t = brownian(0.2, 64, 21, 3)
    a = V.com_diffusion(com, t)
    b = V.com_diffusion(com + np.random.default_rng(1).integers(-3, 4, (1, 64, 3)) * 97.0, t)
    assert a["D"] == pytest.approx(b["D"], rel=1e-12)
    still = V.com_diffusion(np.zeros((5, 8, 3)), np.arange(5.0))
    assert still["D"] == 0.0
    with pytest.raises(ValueError):
        V.com_diffusion(np.zeros((1, 8, 3)), np.zeros(1))


def test_fit_exponent_of_an_exact_power_law():
    n = np.array([8, 16, 32, 64])
    nu, nu_se = V.fit_exponent(n, 3.0 * n ** -0.588, 0.02 * 3.0 * n ** -0.588)
    assert nu == pytest.approx(0.588, abs=1e-12)
    # weighted least squares with relative errors of 2% on each point over ln N of 1.39 per
    # doubling: nu_se = 0.02 / sqrt(sum (ln N - mean)^2)
    x = np.log(n)
    assert nu_se == pytest.approx(0.02 / math.sqrt(((x - x.mean()) ** 2).sum()), rel=1e-12)


def test_paper_units_of_the_two_solvents():
    """Sec. II: sigma = 2^(-1/6) and R0 = 2 sigma in units of 2^(1/6) sigma, k_FENE = 7 * 2^(1/3),
    kT = 1.2, lambda_min = 0.700; Sec. VII.B: theta solvent without WCA and with the bond
    (3/2) k_FENE (r - 0.9691)^2."""
    g = V.paper_unit_params("good")
    t = V.paper_unit_params("theta")
    assert g["wca_sigma"] * 2 ** (1 / 6) == pytest.approx(1.0, rel=1e-15)
    assert g["fene_R0"] == pytest.approx(2.0 * g["wca_sigma"], rel=1e-15)
    assert g["bond_type"] == wmcd.BOND_FENE and g["wca_eps"] == 1.0
    assert t["bond_type"] == wmcd.BOND_HARMONIC and t["wca_eps"] == 0.0
    # the library's harmonic bond is (k/2)(r - r0)^2, so (3/2) k_FENE means k = 3 k_FENE
    r = 1.1
    assert 0.5 * t["bond_k"] * (r - t["bond_r0"]) ** 2 == pytest.approx(1.5 * g["bond_k"] * (r - 0.9691) ** 2)
    assert g["kT"] == t["kT"] == 1.2 and g["lambda_min"] == t["lambda_min"] == 0.7
    # a = lambda_min / lambda_a (Eq. 42) is the hydrodynamic radius the time unit uses
    assert V.LMIN_BAR / V.LAMBDA_A == pytest.approx(0.3023, abs=1e-4)
    with pytest.raises(ValueError):
        V.paper_unit_params("poor")


class _OracleEngine:
    """The oracle behind the Simulation interface the workloads use (sweep, positions, stats,
    close), so their host code runs on the CPU at a small size."""

    def __init__(self, params, pos, chain_len):
        import oracle
        self.o = oracle.Oracle(params, pos, chain_len)

    def sweep(self, n):
        self.o.sweep(n)

    def positions(self, unwrapped=False):
        return self.o.positions(unwrapped=unwrapped)

    def stats(self):
        import types
        s = self.o.stats()
        ns = types.SimpleNamespace(**{k: getattr(s, k) for k, _ in s._fields_})
        ns.attempts = list(s.attempts)
        ns.error_flags = 0
        return ns

    def close(self):
        self.o.close()


def test_chain_workloads_host_code_on_a_stand_in_engine(monkeypatch):
    monkeypatch.setattr(wmcd, "Simulation", _OracleEngine)
    r = V.chain_diffusivity("theta", n_bs=(4, 8), beads=192, bead_gap=12.0, sweeps=60, every=10, max_lag=3, seed=2)
    assert [row["n_b"] for row in r["rows"]] == [4, 8]
    for row in r["rows"]:
        assert row["n_chains"] == 192 // row["n_b"]
        assert row["sim_time"] > 0 and row["D_L"] > 0 and np.isfinite(row["D_se"])
        assert len(row["msd"]) == 3 and row["D_inf"] > row["D_L"]
        assert row["periodic_correction"] == pytest.approx(V.PERIODIC_SELF * r["D0"] * r["a"] / row["box_L"])
    assert np.isfinite(r["nu"]) and r["nu_zimm"] == 0.5
    up = V.chain_relaxation(n_chains=12, n_b=10, sweeps=60, every=20, seed=2, paper_units=True, bond0=0.8)
    assert up["paper_units"] and up["wca_eps"] == 1.0 and len(up["curve"]) == 4
    # every bond starts at 0.8: the walk's bonds are exactly that long
    assert up["curve"][0]["b2"] == pytest.approx(0.64, rel=1e-9)
    assert up["curve"][-1]["b2"] > 0.64 and "rg2_ideal" not in up
    with pytest.raises(ValueError):
        V.chain_relaxation(n_chains=2, n_b=10, sweeps=10, every=10, paper_units=True, start="ideal")
