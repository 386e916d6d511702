"""GPU tests of the two large workloads: the homogeneous semi-dilute solution (4,096 x 256 =
1,048,576 beads at volume fraction 0.05) and the dilute suspension (4,000,000 free spheres and
1,000 chains of 1,024 beads at volume fraction 1e-3).

At full size the sequential oracle (brute-force neighbour search) would take hours per sweep,
so parity is checked on reduced systems of the same shape, built by the same generator (N/64
for the semi-dilute solution, N/512 for the suspension, in the box that keeps the volume
fraction), slot by slot against the oracle; the full-size runs are checked on properties that
hold at any size: slot counts per layer equal the counter-based counts the oracle computes, no
device error, positions in the box and consistent with the image counters, bonds intact."""
import numpy as np
import pytest

import oracle as O
from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd
from test_gpu_parity import compare_positions, compare_stats, compare_sweep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def test_semidilute_reduced_parity():
    s = I.semidilute_chains(64, 256, 0.05, seed=2)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=3, precision=wmcd.MIXED,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC, colour_K=3)
    gpu, ref = wmcd.Simulation(p, s.pos, s.chain_len), O.Oracle(p, s.pos, s.chain_len)
    gpu.sweep(1)
    ref.sweep(1)
    compare_sweep(gpu, ref, ref.stats().n_layers, "semi-dilute N/64")
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)


def test_suspension_reduced_parity():
    s = I.suspension(n_spheres=7812, n_chains=2, chain_len=1024, seed=2)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=3, precision=wmcd.MIXED,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    gpu, ref = wmcd.Simulation(p, s.pos, s.chain_len), O.Oracle(p, s.pos, s.chain_len)
    for k in range(2):
        gpu.sweep(1)
        ref.sweep(1)
        compare_sweep(gpu, ref, ref.stats().n_layers, f"suspension N/512 sweep {k}")
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)


def full_size_properties(s, p, sweeps):
    gpu = wmcd.Simulation(p, s.pos, s.chain_len)
    ref = O.Oracle(p, s.pos, s.chain_len)           # only for the counter-based slot counts
    want = np.zeros(16, dtype=np.int64)
    want_pw = 0
    for sw in range(sweeps):
        c, pw = ref.slot_counts(sw)
        want[:len(c)] += c
        want_pw += pw
    ref.close()
    gpu.sweep(sweeps)
    st = gpu.stats()
    assert st.error_flags == 0
    nL = st.n_layers
    assert list(st.attempts[:nL]) == list(want[:nL])
    assert st.pw_attempts == want_pw
    x = gpu.positions()
    L = s.box_L
    assert np.all(np.isfinite(x)) and np.all((x >= 0) & (x < L))
    u = gpu.positions(unwrapped=True)
    img = (u - x) / L
    assert np.max(np.abs(img - np.round(img))) < 1e-9
    # bonds of every chain stay near their rest length 2 (harmonic, k = 100 kT); the initial
    # positions are wrapped, so a bond is measured by the minimum image
    starts = np.concatenate([[0], np.cumsum(s.chain_len)[:-1]])
    bonded = np.zeros(len(x), dtype=bool)
    for a, n in zip(starts, s.chain_len):
        bonded[a:a + n - 1] = n > 1
    idx = np.nonzero(bonded)[0]
    d = x[idx + 1] - x[idx]
    d -= L * np.round(d / L)
    r = np.linalg.norm(d, axis=1)
    assert r.min() > 1.0 and r.max() < 3.0
    acc = st.accepted_total / max(1, sum(st.attempts) + st.pw_attempts)
    assert 0.2 < acc < 0.95
    gpu.close()


def test_semidilute_full_size_properties():
    s = I.semidilute_chains(4096, 256, 0.05, seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=1, precision=wmcd.MIXED,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC, colour_K=3)
    full_size_properties(s, p, 2)


def test_suspension_full_size_properties():
    s = I.suspension(seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=1, precision=wmcd.MIXED,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    full_size_properties(s, p, 1)
