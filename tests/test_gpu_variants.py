"""GPU parity of the acceptance and centring variants (Secs. V.C-D, VIII) against the oracle,
slot by slot: Glauber acceptance, and centres uniform in the box with A_w from the mean count,
through every move path (concurrent staged, global-memory fallback, serial, shared-memory
serial), in both precisions."""
import numpy as np
import pytest

from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd

from test_gpu_parity import compare_positions, compare_stats, compare_sweep, pair, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_glauber_dilute_chains_concurrent(precision):
    s = I.dilute_chains(n_chains=24, chain_len=64, phi=1e-3, seed=4)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=13, precision=precision, acceptance=wmcd.ACCEPT_GLAUBER)
    assert sum(1 for g in p["grid_layer"] if g) >= 2
    gpu, ref = run_pair(p, s, 12)
    st = gpu.stats()
    assert 0 < st.accepted_total < sum(st.attempts)


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_glauber_single_chain_serial_and_planewaves(precision):
    s = I.single_chain(32, 64.0, seed=3)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=9, planewave_mode=wmcd.PLANEWAVE_PERIODIC, precision=precision,
                            acceptance=wmcd.ACCEPT_GLAUBER)
    run_pair(p, s, 150, planewaves=30)


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_uniform_centres_dense_coloured(precision):
    """Chains and spheres at volume fraction 0.05: supports of a few beads (and empty balls) with
    centres uniform in the box, coloured layers bucketed by the centre's coarse cell."""
    s = I.make_system([32] * 24, 768, I.box_for_volume_fraction(24 * 32 + 768, 0.05), seed=6)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=21, precision=precision, centring=wmcd.CENTRE_UNIFORM,
                            A0=0.3, min_queues_per_axis=1)
    assert any(p["grid_layer"])
    gpu, ref = run_pair(p, s, 10)
    out, n = gpu.trace(0)
    assert np.any(n == 0) and np.any(n > 1)


def test_uniform_centres_small_system_all_serial():
    """All layers serial in shared memory (a small simulation), Glauber and uniform centres together."""
    s = I.single_chain(48, 30.0, seed=2)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=4, precision=wmcd.MIXED, centring=wmcd.CENTRE_UNIFORM,
                            acceptance=wmcd.ACCEPT_GLAUBER, A0=0.3, serial_only=True)
    assert not any(p["grid_layer"])
    run_pair(p, s, 120)
