"""The allocation-free plane-wave entry point against the handle-based one.

wmcd_planewave_noalloc serves callers that may not allocate device memory (another framework
owns the pool, a real-time loop must not allocate after start-up, or a host forbids allocation
in its callbacks). It keeps its scratch in a static device array. Two calls in a row must give
the positions of two wmcd_planewave calls on a handle created from the same inputs. This file
is collected last so that a failure here stops a run only after every other test has run.
"""
import numpy as np
import pytest

from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd

pytestmark = pytest.mark.gpu

POS_TOL = 1e-12   # relative to the box side, as in the other parity tests


@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_noalloc_planewave_matches_handle_two_calls(precision):
    import torch
    wmcd.build()
    s = I.dilute_chains(n_chains=16, chain_len=32, phi=5e-3, seed=3)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=17, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=6,
                            precision=precision, A0=0.5)
    ref = wmcd.Simulation(p, s.pos, s.chain_len)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    carry = np.zeros(4, dtype=np.int32)
    for call in range(2):
        ref.planewave(8)
        wmcd.planewave_noalloc(p, pos, s.chain_len, call, carry, 8)
        want = ref.positions()
        got = pos.cpu().numpy()
        assert np.max(np.abs(got - want)) <= POS_TOL * s.box_L, f"call {call}"
    st = ref.stats()
    assert st.pw_attempts == 16 and 0 < st.pw_accepts < 16    # both outcomes were exercised
    assert not np.array_equal(pos.cpu().numpy(), s.pos)        # the beads did move


def test_noalloc_rejects_oversized_inputs():
    import torch
    s = I.free_spheres(20000, 1e-3, seed=1)
    p = wmcd.default_params(s.n_beads, s.box_L, planewave_mode=wmcd.PLANEWAVE_PERIODIC, bond_type=wmcd.BOND_NONE)
    pos = torch.tensor(s.pos, dtype=torch.float64, device="cuda")
    with pytest.raises(wmcd.WMCDError):
        wmcd.planewave_noalloc(p, pos, s.chain_len, 0, np.zeros(4, np.int32), 1)


@pytest.mark.parametrize("bad", ["edge", "nan"])
def test_noalloc_error_leaves_caller_buffers_unchanged(bad):
    """A coordinate equal to L (outside [0, L)) or a NaN is refused with WMCD_ESTATE before any
    move runs, and neither the caller's positions nor its carry are touched."""
    import torch
    s = I.dilute_chains(n_chains=4, chain_len=16, phi=5e-3, seed=5)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=3, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=6)
    host = s.pos.copy()
    host[7, 1] = s.box_L if bad == "edge" else float("nan")
    pos = torch.tensor(host, dtype=torch.float64, device="cuda")
    before = pos.cpu().numpy().copy()
    carry = np.array([1, 1, -2, 0], dtype=np.int32)
    with pytest.raises(wmcd.WMCDError) as ei:
        wmcd.planewave_noalloc(p, pos, s.chain_len, 0, carry, 4)
    assert ei.value.code == -5
    after = pos.cpu().numpy()
    assert np.array_equal(after.view(np.uint64), before.view(np.uint64))
    assert carry.tolist() == [1, 1, -2, 0]


def test_noalloc_refuses_host_memory():
    s = I.dilute_chains(n_chains=2, chain_len=8, phi=5e-3, seed=6)
    p = wmcd.default_params(s.n_beads, s.box_L, planewave_mode=wmcd.PLANEWAVE_PERIODIC, lcut=4)
    host = s.pos.copy()
    with pytest.raises(wmcd.WMCDError) as ei:
        wmcd.planewave_noalloc(p, host, s.chain_len, 0, np.zeros(4, np.int32), 1)
    assert ei.value.code == -1
    assert np.array_equal(host, s.pos)
