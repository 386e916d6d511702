"""CPU tests of the autotuner's host logic: table keys, lookups that measure nothing, the choice
among measured candidates, the ensemble policies and the shipped table. The timing functions are
replaced by stand-ins (a GPU is needed only to measure)."""
import json

import pytest

from paper_1611_09160_gb300 import autotune as A
from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import wmcd


def _base(n, L, precision=wmcd.MIXED):
    return wmcd.default_params(n, L, seed=1, precision=precision, planewave_mode=wmcd.PLANEWAVE_PERIODIC)


def test_shape_key_rounds_n_and_box():
    assert A.shape_key(16384, 409.4, 1, 1) == "N16384_L8.500_p1_w1"
    assert A.shape_key(12000, 409.4, 1, 1) == A.shape_key(16384, 409.4, 1, 1)   # nearest power of two
    assert A.shape_key(2048, 203.1, 0, 0) == "N2048_L7.500_p0_w0"
    assert A.shape_key(2048, 203.1, 1, 1) != A.shape_key(2048, 290.0, 1, 1)     # half-octave box grid


def test_table_entry_is_used_without_measuring(tmp_path, monkeypatch):
    def no_timing(*a, **k):
        raise AssertionError("a shape in the table must not be measured")
    monkeypatch.setattr(A, "_time_sim", no_timing)
    monkeypatch.setattr(A, "_time_batch", no_timing)
    base = _base(16384, 409.4)
    seed = tmp_path / "seed.json"
    seed.write_text(json.dumps({A.shape_key(16384, 409.4, 1, 1): {"choice": {"colour_K": 3}, "scores": []}}))
    p = A.Tuner(seed_table=str(seed)).schedule(base)
    assert p["colour_K"] == 3 and p["grid_layer"] == A.Tuner.apply(base, {"colour_K": 3})["grid_layer"]


def test_missing_shape_is_measured_and_the_fastest_candidate_kept(tmp_path, monkeypatch):
    seen = []

    def fake_time(params, system, warm, sweeps):
        seen.append(params["colour_K"])
        return {2: 5.0, 3: 9.0, 4: 7.0}[params["colour_K"]]
    monkeypatch.setattr(A, "_time_sim", fake_time)
    path = tmp_path / "table.json"
    base = _base(16384, 409.4)
    cands = ({"colour_K": 2}, {"colour_K": 3}, {"colour_K": 4})
    p = A.Tuner(path=str(path)).schedule(base, chain_lengths=[64] * 256, candidates=cands)
    assert seen == [2, 3, 4] and p["colour_K"] == 3
    saved = json.loads(path.read_text())
    entry = saved[A.shape_key(16384, 409.4, 1, 1)]
    assert entry["choice"] == {"colour_K": 3} and len(entry["scores"]) == 3
    # a second tuner reading the saved table measures nothing
    monkeypatch.setattr(A, "_time_sim", lambda *a, **k: pytest.fail("measured again"))
    assert A.Tuner(path=str(path)).schedule(base)["colour_K"] == 3


def test_serial_small_policy_depends_only_on_each_simulation():
    systems = [I.single_chain(n, I.box_for_volume_fraction(n, 1e-3), seed=n) for n in (16, 300, 2048)]
    ps = A.ensemble_params(systems, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, seed=1, policy="serial_small")
    for p, s in zip(ps, systems):
        assert p["n_beads"] == s.n_beads and all(g == 0 for g in p["grid_layer"])
    # the same simulation gets the same schedule whatever else is in the ensemble
    alone = A.ensemble_params(systems[1:2], wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, seed=1, policy="serial_small")[0]
    assert alone["grid_layer"] == ps[1]["grid_layer"] and alone["colour_K"] == ps[1]["colour_K"]


def test_choose_policy_takes_the_faster_whole_batch(monkeypatch):
    systems = [I.single_chain(n, I.box_for_volume_fraction(n, 1e-3), seed=n) for n in (16, 64, 256)]

    for measured in ((1.0, 2.0), (3.0, 2.0)):        # (per_shape, serial_small), in the order measured
        it = iter(measured)
        monkeypatch.setattr(A, "batch_throughput", lambda params, syss, warm=1, sweeps=3: next(it))
        monkeypatch.setattr(A, "_time_batch", lambda *a, **k: 1.0)
        best, scores = A.choose_policy(systems, wmcd.MIXED, wmcd.PLANEWAVE_PERIODIC, A.Tuner(copies=152), sample=3)
        assert scores == {"per_shape": measured[0], "serial_small": measured[1]}
        assert best == ("serial_small" if measured[1] > measured[0] else "per_shape")


def test_shipped_table_entries_are_valid_schedules():
    with open(A.DEFAULT_TABLE) as f:
        table = json.load(f)
    assert table
    for key, entry in table.items():
        n = int(key.split("_")[0][1:])
        L = 2.0 ** float(key.split("_")[1][1:])
        p = A.Tuner.apply(_base(n, L), entry["choice"])
        K = p["colour_K"]
        assert K in (2, 3, 4) and all(g == 0 or (g % K == 0 and g >= K) for g in p["grid_layer"])
