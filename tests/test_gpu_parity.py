"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on identical seeded
inputs. Decisions are compared slot by slot (accept / reject / deferred and the support size
n of every wavelet move, the wave vector and outcome of every plane wave); positions must
agree to 1e-12 of the box side (in practice they agree bit for bit: both sides form every
position-changing quantity with the same IEEE operations in the same order)."""
import numpy as np
import pytest

import oracle as O
from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd

pytestmark = pytest.mark.gpu

POS_TOL = 1e-12   # relative to the box side


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def pair(params, system):
    return wmcd.Simulation(params, system.pos, system.chain_len), O.Oracle(params, system.pos, system.chain_len)


def compare_sweep(gpu, ref, n_layers, label=""):
    for l in range(n_layers):
        a, na = gpu.trace(l)
        b, nb = ref.trace_layer(l)
        assert len(a) == len(b), f"{label} layer {l}: slot counts {len(a)} vs {len(b)}"
        bad = np.nonzero((a != b) | (na != nb))[0]
        if bad.size:
            ga, oa = gpu.trace_du(l), ref.trace_du(l)
            detail = "; ".join(f"slot {k}: gpu {a[k]},n={na[k]},dU={ga[k]!r} oracle {b[k]},n={nb[k]},dU={oa[k]!r}"
                               for k in bad[:6])
            raise AssertionError(f"{label} layer {l}: {bad.size} slots differ: {detail}")
        # energy change behind every decision: binary64 paths agree to rounding
        ga, oa = gpu.trace_du(l), ref.trace_du(l)
        exact = (a & 3) != 0
        err = np.abs(ga - oa)[exact]
        # binary32 sums (mixed precision) legitimately differ by up to their error band
        tol = (2e-3 if gpu.params.get("precision", 0) else 1e-9) * (1.0 + np.abs(oa[exact]))
        assert np.all(err <= tol), f"{label} layer {l}: dU differs by up to {err.max()}"
    a, ma = gpu.trace(-1)
    b, mb = ref.trace_pw()
    assert np.array_equal(a, b) and np.array_equal(ma, mb), f"{label} plane-wave trace differs"


def compare_positions(gpu, ref, L, tol=POS_TOL):
    x, y = gpu.positions(unwrapped=True), ref.positions(unwrapped=True)
    err = np.max(np.abs(x - y))
    assert err <= tol * L, f"max position difference {err} > {tol * L}"
    return err


def compare_stats(gpu, ref):
    g, o = gpu.stats(), ref.stats()
    assert g.error_flags == 0
    nL = o.n_layers
    assert list(g.attempts[:nL]) == list(o.attempts[:nL])
    assert list(g.accepts[:nL]) == list(o.accepts[:nL])
    assert list(g.deferred[:nL]) == list(o.deferred[:nL])
    assert (g.pw_attempts, g.pw_accepts) == (o.pw_attempts, o.pw_accepts)
    assert g.bead_updates == o.bead_updates
    assert g.accepted_total == o.accepted_total
    assert g.moved_beads == o.moved_beads
    assert g.sim_time == o.sim_time
    assert g.dt_move == o.dt_move
    assert g.p_fourier == pytest.approx(o.p_fourier, rel=1e-12)


def run_pair(params, system, sweeps, trace_every=1, planewaves=0):
    gpu, ref = pair(params, system)
    nL = ref.stats().n_layers
    for s in range(sweeps):
        gpu.sweep(1)
        ref.sweep(1)
        if s % trace_every == 0:
            compare_sweep(gpu, ref, nL, f"sweep {s}")
    if planewaves:
        gpu.planewave(planewaves)
        ref.planewave(planewaves)
        compare_sweep(gpu, ref, 0, "direct plane waves")
    compare_positions(gpu, ref, system.box_L)
    compare_stats(gpu, ref)
    return gpu, ref


# ---- the 32-bead chain in L = 64 (the small workload) ---------------------------------

def test_single_chain_fp64_all_serial():
    s = I.single_chain(32, 64.0, seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=1)
    assert all(g == 0 for g in p["grid_layer"])
    run_pair(p, s, 300)


def test_single_chain_fp64_10k_sweeps():
    """10^4 sweeps: identical counters and final positions (decisions checked every 500)."""
    s = I.single_chain(32, 64.0, seed=2)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=5, planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    gpu, ref = pair(p, s)
    for block in range(20):
        gpu.sweep(499)
        ref.sweep(499)
        gpu.sweep(1)
        ref.sweep(1)
        compare_sweep(gpu, ref, ref.stats().n_layers, f"block {block}")
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)


def test_single_chain_mixed_10k_sweeps():
    """Mixed precision over 10^4 sweeps, with a coloured layer and plane waves, against the
    oracle's mixed mode (the same binary32 displacements, decisions in binary64): decisions
    checked every 500 sweeps, positions within 1e-5 of the box at each check (in fact equal to
    1e-12 L), identical counters at the end."""
    s = I.single_chain(32, 64.0, seed=6)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=15, planewave_mode=wmcd.PLANEWAVE_PERIODIC,
                            precision=wmcd.MIXED)
    p["grid_layer"] = [2] + [0] * 15
    gpu, ref = pair(p, s)
    for block in range(20):
        gpu.sweep(499)
        ref.sweep(499)
        gpu.sweep(1)
        ref.sweep(1)
        compare_sweep(gpu, ref, ref.stats().n_layers, f"block {block}")
        compare_positions(gpu, ref, s.box_L, tol=1e-5)
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)
    assert gpu.stats().pw_attempts > 0


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_single_chain_coloured_and_planewaves(precision):
    s = I.single_chain(32, 64.0, seed=3)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=9, planewave_mode=wmcd.PLANEWAVE_PERIODIC, precision=precision)
    p["grid_layer"] = [2] + [0] * 15
    gpu, ref = run_pair(p, s, 200, planewaves=40)
    assert gpu.stats().pw_attempts >= 40


# ---- dilute chains with coloured layers and deferrals -----------------------------------

@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_dilute_chains_concurrent(precision):
    s = I.dilute_chains(n_chains=24, chain_len=64, phi=1e-3, seed=4)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=13, precision=precision)
    assert sum(1 for g in p["grid_layer"] if g) >= 2
    gpu, ref = run_pair(p, s, 15)
    st = gpu.stats()
    assert sum(st.attempts) > 10 * s.n_beads


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_dense_small_box_forces_deferrals_and_cell_moves(precision):
    """Semi-dilute chains in a small box, regions barely larger than a move, n_cap small:
    many deferrals, supports above the cap, beads crossing fine cells and box faces. In mixed
    precision the binary32 energy changes decide outside the error band, binary64 inside it."""
    s = I.make_system([16] * 12, 0, I.box_for_volume_fraction(192, 0.05), seed=6)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=21, n_cap=3, A0=0.8, precision=precision)
    p["grid_layer"] = [4] + [0] * 15
    gpu, ref = run_pair(p, s, 25)
    st = ref.stats()
    assert st.deferred[0] > 0 and st.deferred[0] < st.attempts[0]


def test_mixed_precision_many_moves_dense():
    """Thousands of concurrent moves in a dense system: identical decisions to the binary64
    oracle, with some moves re-decided in binary64 (counted)."""
    s = I.make_system([32] * 48, 0, I.box_for_volume_fraction(1536, 0.08), seed=12)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=5, precision=wmcd.MIXED, colour_K=3)
    p["grid_layer"] = [6] + [0] * 15
    gpu, ref = run_pair(p, s, 40, trace_every=4)
    st = gpu.stats()
    assert st.conc_bead_updates > 0


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_whole_gpu_serial_moves(precision):
    """Serial layers of large scale run each move as a sequence of whole-GPU launches (support
    scan over all beads, per-member energies, block partials summed in a fixed order). A small
    threshold on the expected support sends the upper layers of small systems down that path."""
    s = I.make_system([16] * 12, 0, I.box_for_volume_fraction(192, 0.05), seed=9)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=23, precision=precision, planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    p["grid_layer"] = [0] * 16
    p["big_support"] = 4
    run_pair(p, s, 40, planewaves=4)
    c = I.dilute_chains(n_chains=24, chain_len=64, phi=1e-3, seed=10)
    p = wmcd.default_params(c.n_beads, c.box_L, seed=29, precision=precision)
    p["big_support"] = 64
    assert p["grid_layer"][0] > 0 and p["grid_layer"][4] == 0
    gpu, ref = run_pair(p, c, 12)
    assert sum(ref.stats().attempts[4:6]) > 0


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_large_supports_run_concurrently(precision):
    """Chains at volume fraction 0.15 with a coloured layer of scales 4-8 (supports up to about
    100 beads) and n_cap = 256: moves with more than 64 members run in the concurrent phase (the
    whole-box region staged by one block whose warps cooperate) instead of being deferred."""
    s = I.make_system([32] * 64, 0, I.box_for_volume_fraction(2048, 0.15), seed=13)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=7, precision=precision, colour_K=3, n_cap=256)
    p["grid_layer"] = [6, 3] + [0] * 14
    gpu, ref = run_pair(p, s, 3)
    a, na = gpu.trace(1)
    concurrent = ((a & 3) != 0) & ((a & 4) == 0)
    assert (na[concurrent] > 64).any()


def test_large_supports_concurrent_through_global_memory():
    """As above with 4,096 beads: the coloured layer's region (the whole box) is too large to
    stage, so its moves, supports above 64 beads included, run through the global cell lists."""
    s = I.make_system([32] * 128, 0, I.box_for_volume_fraction(4096, 0.15), seed=14)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=8, precision=wmcd.MIXED, colour_K=3, n_cap=256)
    p["grid_layer"] = [9, 3] + [0] * 14
    gpu, ref = run_pair(p, s, 2)
    a, na = gpu.trace(1)
    concurrent = ((a & 3) != 0) & ((a & 4) == 0)
    assert (na[concurrent] > 64).any()


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_coarse_layer_regions_staged_in_blocks_of_their_own(precision):
    """64 chains x 64 beads at volume fraction 1e-3 with colour stride 3: the regions of the
    coarsest coloured layer (about 512 beads each, 27 queues per colour) overflow the base
    staging capacity, so each is staged by a whole block (all its warps stage, one runs the
    moves) with the largest capacity shared memory allows."""
    s = I.dilute_chains(64, 64, 1e-3, seed=7)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=5, precision=precision,
                            planewave_mode=wmcd.PLANEWAVE_PERIODIC, colour_K=3)
    assert p["grid_layer"][2] == 6
    run_pair(p, s, 3)


def test_free_spheres_and_fene():
    s = I.free_spheres(500, 3e-3, seed=7)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=2, bond_type=wmcd.BOND_NONE)
    run_pair(p, s, 10)
    c = I.make_system([20] * 10, 0, 60.0, seed=8, bond=1.9, min_dist=1.9)
    p = wmcd.default_params(c.n_beads, c.box_L, seed=3, bond_type=wmcd.BOND_FENE, bond_k=7.0, fene_R0=2.6,
                            wca_sigma=1.7)
    run_pair(p, c, 20)


def test_one_bead_in_a_well():
    p = wmcd.default_params(1, 64.0, seed=4, ext_kappa=0.3, wca_eps=0.0, bond_type=wmcd.BOND_NONE, lambda_max=16.0)
    s = I.System(np.array([[32.0, 32.0, 32.0]]), np.array([1], np.int32), 64.0)
    run_pair(p, s, 2000, trace_every=97)


# ---- the dilute-chain benchmark system at full size ----------------------------------

@pytest.mark.parametrize("planewave", [wmcd.PLANEWAVE_OFF, wmcd.PLANEWAVE_PERIODIC])
def test_benchmark_system_full_size(planewave):
    """256 chains x 64 beads (16,384) at volume fraction 1e-3, the launch configuration of the
    benchmark: two sweeps compared slot by slot, plus direct plane waves."""
    s = I.dilute_chains(256, 64, 1e-3, seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=1, planewave_mode=planewave, precision=wmcd.MIXED)
    run_pair(p, s, 2, planewaves=2 if planewave else 0)


# ---- state, determinism, errors -----------------------------------------------------------

def test_checkpoint_restores_bit_identically():
    s = I.dilute_chains(n_chains=8, chain_len=32, phi=2e-3, seed=5)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=8, planewave_mode=wmcd.PLANEWAVE_PERIODIC)
    g = wmcd.Simulation(p, s.pos, s.chain_len)
    g.sweep(5)
    st = g.get_state()
    g.sweep(7)
    g.planewave(3)
    a = g.positions(unwrapped=True)
    g.set_state(st)
    g.sweep(7)
    g.planewave(3)
    b = g.positions(unwrapped=True)
    assert np.array_equal(a, b)
    # a second handle from the same inputs repeats the run exactly
    h = wmcd.Simulation(p, s.pos, s.chain_len)
    h.sweep(12)
    h.planewave(3)
    assert np.array_equal(h.positions(unwrapped=True), a)


def test_torch_device_buffers_and_streams():
    import torch
    s = I.single_chain(32, 64.0, seed=9)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=4)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    g = wmcd.Simulation(p, pos, s.chain_len, stream=stream)
    g.sweep(50, stream=stream)
    out = torch.empty((s.n_beads, 3), dtype=torch.float64, device="cuda")
    g.positions(out=out, stream=stream)
    stream.synchronize()
    ref = O.Oracle(p, s.pos, s.chain_len)
    ref.sweep(50)
    assert np.max(np.abs(out.cpu().numpy() - ref.positions())) <= POS_TOL * 64.0


def test_invalid_positions_are_rejected():
    s = I.single_chain(8, 64.0, seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L)
    bad = s.pos.copy()
    bad[3, 1] = 64.0
    with pytest.raises(wmcd.WMCDError):
        wmcd.Simulation(p, bad, s.chain_len)
    bad[3, 1] = np.nan
    with pytest.raises(wmcd.WMCDError):
        wmcd.Simulation(p, bad, s.chain_len)
