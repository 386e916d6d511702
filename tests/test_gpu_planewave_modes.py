"""GPU parity of the full periodic plane-wave scheme (discrete cube + quasi-continuous shell,
Appendix D) and of the infinite-system plane waves (Sec. VI.B) against the oracle: every
move's wave vector and outcome, the recycled |k| after rejections, positions to 1e-12 of the
box, and the counters; inside sweeps and as direct plane-wave calls."""
import numpy as np
import pytest

import oracle as O
from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd

from test_gpu_parity import compare_positions, compare_stats, compare_sweep, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def compare_pw(gpu, ref, label):
    a, ma = gpu.trace(-1)
    b, mb = ref.trace_pw()
    assert np.array_equal(a, b), f"{label}: plane-wave outcomes differ"
    assert np.array_equal(ma, mb), f"{label}: packed modes differ"
    ka, kb = gpu.trace_pw_k(), ref.trace_pw_k()
    assert ka.shape == kb.shape
    rel = np.max(np.abs(ka - kb) / np.maximum(np.abs(kb), 1e-300)) if len(ka) else 0.0
    assert np.allclose(ka, kb, rtol=1e-12, atol=0.0), f"{label}: wave vectors differ (largest relative {rel:.3g})"
    return a, ka


@pytest.mark.parametrize("mode,lcut", [(wmcd.PLANEWAVE_PERIODIC_FULL, 15), (wmcd.PLANEWAVE_PERIODIC_FULL, 3),
                                       (wmcd.PLANEWAVE_INFINITE, 0)])
@pytest.mark.parametrize("precision", [wmcd.FP64, wmcd.MIXED])
def test_direct_plane_waves_match_the_oracle(mode, lcut, precision):
    s = I.make_system([24, 24], 16, 24.0, seed=8)             # small dense box: plane waves often reject
    p = wmcd.default_params(s.n_beads, s.box_L, seed=31, planewave_mode=mode, lcut=lcut, precision=precision,
                            A0=0.4)
    gpu, ref = pair(p, s)
    outs, ks = [], []
    for call in range(4):
        gpu.planewave(100)
        ref.planewave(100)
        a, k = compare_pw(gpu, ref, f"call {call}")
        outs.append(a)
        ks.append(k)
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)
    out, k = np.concatenate(outs), np.concatenate(ks)
    assert 0 < np.sum(out == 2) < len(out)                    # both outcomes, so the carry is used
    if mode == wmcd.PLANEWAVE_PERIODIC_FULL:
        assert np.all(k == np.round(k))
        shell = np.any(np.abs(k) > lcut, axis=1)
        assert shell.any() and (~shell).any()                 # both the cube and the shell were drawn
    else:
        assert np.any(np.abs(k - np.round(k)) > 1e-6)           # continuous wave vectors


@pytest.mark.parametrize("mode", [wmcd.PLANEWAVE_PERIODIC_FULL, wmcd.PLANEWAVE_INFINITE])
def test_sweeps_with_the_plane_wave_schemes_match_the_oracle(mode):
    s = I.dilute_chains(n_chains=12, chain_len=32, phi=2e-3, seed=5)
    p = wmcd.default_params(s.n_beads, s.box_L, seed=19, planewave_mode=mode, lcut=15, precision=wmcd.MIXED)
    p["lambda_max"] = 8.0                                     # more plane-wave slots per sweep
    gpu, ref = pair(p, s)
    nL = ref.stats().n_layers
    for sw in range(12):
        gpu.sweep(1)
        ref.sweep(1)
        compare_sweep(gpu, ref, nL, f"sweep {sw}")
        compare_pw(gpu, ref, f"sweep {sw}")
    compare_positions(gpu, ref, s.box_L)
    compare_stats(gpu, ref)
    assert gpu.stats().pw_attempts > 10
