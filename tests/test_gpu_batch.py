"""GPU tests of batches: many simulations of uneven size, box, precision and move set advanced
together by one launch per phase (a recorded CUDA graph per batched sweep). Each simulation
must follow the trajectory it follows alone and the oracle's decisions; admission is bounded
by the batch's device-memory pool."""
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


def mixed_systems():
    """(params, system) pairs of different N, L, precision, plane-wave mode and schedule."""
    out = []
    s = I.single_chain(32, 64.0, seed=3)
    out.append((wmcd.default_params(s.n_beads, s.box_L, seed=11, planewave_mode=wmcd.PLANEWAVE_PERIODIC), s))
    s = I.dilute_chains(n_chains=24, chain_len=64, phi=1e-3, seed=4)
    out.append((wmcd.default_params(s.n_beads, s.box_L, seed=12, precision=wmcd.MIXED), s))
    s = I.make_system([100], 0, I.box_for_volume_fraction(100, 1e-3), seed=5)
    out.append((wmcd.default_params(s.n_beads, s.box_L, seed=13, precision=wmcd.MIXED,
                                    planewave_mode=wmcd.PLANEWAVE_PERIODIC), s))
    s = I.make_system([16] * 12, 0, I.box_for_volume_fraction(192, 0.05), seed=6)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=14, n_cap=3, A0=0.8)
    p["grid_layer"] = [4] + [0] * 15
    out.append((p, s))
    s = I.free_spheres(300, 3e-3, seed=7)
    out.append((wmcd.default_params(s.n_beads, s.box_L, seed=15, bond_type=wmcd.BOND_NONE), s))
    s = I.make_system([16] * 12, 0, I.box_for_volume_fraction(192, 0.05), seed=8)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=16, precision=wmcd.MIXED, planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    p["grid_layer"] = [0] * 16
    p["big_support"] = 4          # its largest scales run as whole-GPU moves
    out.append((p, s))
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=12)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=17, precision=wmcd.MIXED, n_cap=3, level2=1)
    p["grid_layer"] = [8] + [0] * 15   # deferred slots get a second colouring on 4 cells per axis
    out.append((p, s))
    return out


def alone(params, system, sweeps):
    sim = wmcd.Simulation(params, system.pos, system.chain_len)
    sim.sweep(sweeps)
    return sim


def pool_for(pairs, extra=0):
    return sum(wmcd.batch_need(p) for p, _ in pairs) + extra


def test_batch_equals_each_simulation_alone():
    pairs = mixed_systems()
    b = wmcd.Batch(capacity=8, pool_bytes=pool_for(pairs, 1 << 20))
    slots = [b.admit(p, s.pos, s.chain_len) for p, s in pairs]
    assert all(x is not None for x in slots)
    b.step(5)
    b.step(7)
    info = b.info()
    assert info["resident"] == len(pairs) and info["launches_per_sweep"] > 0
    for (p, s), slot in zip(pairs, slots):
        ref = alone(p, s, 12)
        got = b.sim(slot)
        x, y = got.positions(unwrapped=True), ref.positions(unwrapped=True)
        assert np.max(np.abs(x - y)) <= 1e-12 * s.box_L
        g, o = got.stats(), ref.stats()
        assert g.error_flags == 0 and g.sweeps == 12
        assert list(g.attempts) == list(o.attempts) and list(g.accepts) == list(o.accepts)
        assert list(g.deferred) == list(o.deferred)
        assert (g.pw_attempts, g.pw_accepts, g.bead_updates) == (o.pw_attempts, o.pw_accepts, o.bead_updates)
        ref.close()
    b.close()


def test_batch_decisions_match_oracle_every_sweep():
    pairs = [mixed_systems()[i] for i in (0, 2, 3, 6)]
    b = wmcd.Batch(capacity=4, pool_bytes=pool_for(pairs))
    slots = [b.admit(p, s.pos, s.chain_len) for p, s in pairs]
    refs = [O.Oracle(p, s.pos, s.chain_len) for p, s in pairs]
    for sweep in range(25):
        b.step(1)
        for slot, ref in zip(slots, refs):
            ref.sweep(1)
            compare_sweep(b.sim(slot), ref, ref.stats().n_layers, f"sweep {sweep} slot {slot}")
    for (p, s), slot, ref in zip(pairs, slots, refs):
        compare_positions(b.sim(slot), ref, s.box_L)
        compare_stats(b.sim(slot), ref)
    b.close()


def test_admission_by_memory_and_continuous_batching():
    """A pool that holds two of three simulations: the third waits until one retires, then
    joins the running batch; every simulation's result equals its run alone."""
    pairs = mixed_systems()
    X, Y, Z = pairs[0], pairs[2], pairs[4]
    needs = [wmcd.batch_need(p) for p, _ in (X, Y, Z)]
    # Y then X fill the pool from the front; the tail left over is smaller than Z, and the
    # block X frees merges with it into room for Z
    pool = needs[1] + max(needs[0], needs[2])
    b = wmcd.Batch(capacity=8, pool_bytes=pool)
    sy = b.admit(Y[0], Y[1].pos, Y[1].chain_len)
    sx = b.admit(X[0], X[1].pos, X[1].chain_len)
    assert sx is not None and sy is not None
    assert b.info()["largest_free"] < needs[2]
    assert b.admit(Z[0], Z[1].pos, Z[1].chain_len) is None
    b.step(3)
    x_pos = b.sim(sx).positions(unwrapped=True)
    free_before = b.info()["pool_free"]
    b.retire(sx)
    assert b.info()["pool_free"] == free_before + needs[0]
    sz = b.admit(Z[0], Z[1].pos, Z[1].chain_len)
    assert sz is not None
    b.step(4)
    b.step(2)
    for (p, s), slot, n in ((Y, sy, 9), (Z, sz, 6)):
        ref = alone(p, s, n)
        assert np.max(np.abs(b.sim(slot).positions(unwrapped=True) - ref.positions(unwrapped=True))) <= 1e-12 * s.box_L
        assert b.sim(slot).stats().sweeps == n
        ref.close()
    ref = alone(X[0], X[1], 3)
    assert np.max(np.abs(x_pos - ref.positions(unwrapped=True))) <= 1e-12 * X[1].box_L
    ref.close()
    b.close()


def test_block_shape_does_not_change_results():
    pairs = [mixed_systems()[i] for i in (1, 3)]
    res = []
    for stage_warps, serial_threads in ((1, 32), (4, 512), (2, 128)):
        b = wmcd.Batch(capacity=2, pool_bytes=pool_for(pairs))
        b.set_block(stage_warps, serial_threads)
        slots = [b.admit(p, s.pos, s.chain_len) for p, s in pairs]
        b.step(6)
        res.append([b.sim(k).positions(unwrapped=True) for k in slots])
        b.close()
    for other in res[1:]:
        for a, c, (_, s) in zip(res[0], other, pairs):
            assert np.max(np.abs(a - c)) <= 1e-12 * s.box_L


def test_batch_owned_handle_is_not_destroyed_directly():
    p, s = mixed_systems()[0]
    b = wmcd.Batch(capacity=1, pool_bytes=wmcd.batch_need(p))
    slot = b.admit(p, s.pos, s.chain_len)
    assert b.admit(p, s.pos, s.chain_len) is None          # no free slot
    lib = wmcd.load()
    assert lib.wmcd_destroy(b.sim(slot).h) == -1           # WMCD_EINVAL: the batch owns it
    b.step(2)
    assert b.sim(slot).stats().sweeps == 2
    b.close()
