"""GPU parity of the second colouring of deferred slots against the oracle, slot by slot: the
slots a coloured layer l (bit l of level2) defers are bucketed again on K floor(G / 2K) coarse
cells (by their bead, or centre, as it is then) and run in that grid's colour phases with
supports up to 256 beads; only what this second colouring defers as well runs serially. Trace
flags: 4 = deferred by the first colouring, 8 = by the second as well."""
import numpy as np
import pytest

from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd

from test_gpu_parity import run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def level_counts(sim, layers):
    """(moves run by the second colouring, moves deferred twice) over the given layers."""
    two = twice = 0
    for l in layers:
        a, _ = sim.trace(l)
        two += int((((a & 4) != 0) & ((a & 8) == 0)).sum())
        twice += int(((a & 8) != 0).sum())
    return two, twice


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_second_colouring_dense_chains(precision):
    """Chains at volume fraction 0.08 with n_cap = 3: nearly every first-colouring move is
    deferred; the second grid (4 cells per axis) runs about half of them concurrently."""
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=12)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=5, precision=precision, n_cap=3, level2=1)
    p["grid_layer"] = [8] + [0] * 15
    gpu, ref = run_pair(p, s, 6)
    two, twice = level_counts(gpu, [0])
    assert two > 0 and twice > 0


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_second_colouring_two_layers_large_regions(precision):
    """4,096 beads at volume fraction 0.15, two coloured layers: the second colouring's regions
    hold hundreds to thousands of beads (staged by whole blocks, or walked in global memory)."""
    s = I.make_system([32] * 128, 0, I.box_for_volume_fraction(4096, 0.15), seed=14)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=8, precision=precision, n_cap=16, level2=3)
    p["grid_layer"] = [12, 8] + [0] * 14
    gpu, ref = run_pair(p, s, 2)
    two, twice = level_counts(gpu, [0, 1])
    assert two > 0 and twice > 0


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_second_colouring_dilute_chains_with_planewaves(precision):
    s = I.dilute_chains(n_chains=128, chain_len=64, phi=1e-3, seed=21)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=17, precision=precision, n_cap=8, level2=0xffff,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    assert any(g >= 8 for g in p["grid_layer"])
    gpu, ref = run_pair(p, s, 4)
    two, _ = level_counts(gpu, range(ref.stats().n_layers))
    assert two > 0


def test_second_colouring_uniform_centres_glauber():
    """Centres uniform in the box: the second colouring buckets by the centre as the first does."""
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=3)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=19, precision=wmcd.MIXED, n_cap=2, level2=1,
                            centring=wmcd.CENTRE_UNIFORM, acceptance=wmcd.ACCEPT_GLAUBER, A0=0.3)
    p["grid_layer"] = [8] + [0] * 15
    gpu, ref = run_pair(p, s, 6)
    two, _ = level_counts(gpu, [0])
    assert two > 0


def test_second_colouring_off_and_too_coarse_change_nothing():
    """level2 = 0, a mask without the layer's bit, or a grid too coarse for a second colouring
    (G < 4K), gives the first colouring's run exactly."""
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=12)
    base = wmcd.default_params(s.n_beads, s.box_L, seed=5, precision=wmcd.MIXED, n_cap=3)
    base["grid_layer"] = [6] + [0] * 15
    runs = []
    for lv, grid in ((0, 6), (1, 6), (0xfffe, 8)):
        sim = wmcd.Simulation(dict(base, level2=lv, grid_layer=[grid] + [0] * 15), s.pos, s.chain_len)
        sim.sweep(5)
        runs.append((sim.positions(unwrapped=True), sim.trace(0)[0]))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert not np.any(runs[1][1] & 8) and not np.any(runs[2][1] & 8)


def test_second_colouring_checkpoint_restores_its_carries():
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=12)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=6, precision=wmcd.MIXED, n_cap=3, level2=1)
    p["grid_layer"] = [8] + [0] * 15
    g = wmcd.Simulation(p, s.pos, s.chain_len)
    g.sweep(3)
    st = g.get_state()
    g.sweep(4)
    a = g.positions(unwrapped=True)
    h = wmcd.Simulation(p, s.pos, s.chain_len)
    h.set_state(st)
    h.sweep(4)
    assert np.array_equal(h.positions(unwrapped=True), a)
    p0 = dict(p, level2=0)
    with pytest.raises(wmcd.WMCDError):          # the state of a run without the second grid differs in size
        wmcd.Simulation(p0, s.pos, s.chain_len).set_state(st)
