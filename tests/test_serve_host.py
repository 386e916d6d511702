"""CPU tests of the serving loop's host logic (admission in arrival order, bounded by slots
and pool memory; steps that never run a request past its sweep count; retirement), with a
stand-in batch that records what the loop asks of it."""
import numpy as np
import pytest

from paper_1611_09160_gb300 import serve


class FakeSim:
    def __init__(self, req_pos):
        self.pos = np.array(req_pos, dtype=float)
        self.sweeps = 0

    def positions(self, unwrapped=True):
        return self.pos + self.sweeps

    def stats(self):
        class S:
            pass
        st = S()
        st.bead_updates = 10 * self.sweeps
        st.sim_time = 0.5 * self.sweeps
        st.accepted_total = self.sweeps
        return st


class FakeBatch:
    """Slots and a byte budget; memory need = 100 bytes per bead."""

    def __init__(self, capacity, pool):
        self.capacity, self.pool, self.used = capacity, pool, 0
        self.sims, self.need, self.log = {}, {}, []

    def set_block(self, *a):
        pass

    def admit(self, params, pos, chain_len):
        need = 100 * params["n_beads"]
        if len(self.sims) >= self.capacity or self.used + need > self.pool:
            return None
        slot = min(set(range(self.capacity)) - set(self.sims))
        self.sims[slot], self.need[slot] = FakeSim(pos), need
        self.used += need
        self.log.append(("admit", params["rid"], slot))
        return slot

    def step(self, k):
        assert k >= 1
        for s in self.sims.values():
            s.sweeps += k
        self.log.append(("step", k, tuple(sorted(self.sims))))

    def sim(self, slot):
        return self.sims[slot]

    def retire(self, slot):
        self.used -= self.need.pop(slot)
        del self.sims[slot]
        self.log.append(("retire", slot))

    def close(self):
        pass


class FakeTimer:
    """Stand-in timer: every batched step takes 2 ms, split evenly over its sweeps."""

    def __init__(self):
        self.steps = []                  # sweeps of each batched step, in order

    def start(self):
        self.n = 0

    def mark(self):
        self.n += 1

    def wait_ms(self):
        self.steps.append(self.n)
        return [2.0 / self.n] * self.n


def make_requests(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        nb = int(rng.integers(1, 6))
        reqs.append(serve.Request(i, {"n_beads": nb, "rid": i}, np.full((nb, 3), float(i)), np.array([nb], np.int32),
                                  int(rng.integers(1, 40)), arrival=0.0))
    return reqs


@pytest.mark.parametrize("capacity,pool,chunk", [(3, 10**9, 8), (8, 1000, 5), (1, 10**9, 16), (16, 10**9, 1)])
def test_every_request_runs_exactly_its_sweeps(capacity, pool, chunk):
    reqs = make_requests(40)
    fb = FakeBatch(capacity, pool)
    timer = FakeTimer()
    srv = serve.Server(chunk=chunk, batch=fb, timer=timer)
    rep = srv.run(reqs, realtime=False)
    assert set(rep.results) == {r.rid for r in reqs}
    for r in reqs:
        res = rep.results[r.rid]
        assert np.array_equal(res.positions, r.pos + r.n_sweeps)   # exactly n_sweeps sweeps
        assert res.bead_updates == 10 * r.n_sweeps
    assert rep.bead_updates == sum(10 * r.n_sweeps for r in reqs)
    assert rep.max_resident <= capacity
    assert fb.used == 0 and not fb.sims
    # admission follows arrival order
    admitted = [e[1] for e in fb.log if e[0] == "admit"]
    assert admitted == sorted(admitted)
    assert all(e[1] == 1 for e in fb.log if e[0] == "step")        # one launch per sweep
    s = rep.summary()
    steps = timer.steps
    assert sum(steps) == sum(1 for e in fb.log if e[0] == "step") and max(steps) <= chunk
    assert s["requests"] == 40 and s["steps"] == len(steps) and s["batched_sweeps"] == sum(steps)
    assert s["gpu_ms"] == pytest.approx(2.0 * len(steps))          # the stand-in timer: 2 ms per step
    assert 2.0 / max(steps) <= s["sweep_ms_p50"] <= s["sweep_ms_p99"] <= 2.0


def test_memory_bound_admission_waits_for_retirement():
    reqs = make_requests(12, seed=3)
    fb = FakeBatch(capacity=100, pool=700)       # at most a few small requests at once
    rep = serve.Server(chunk=4, batch=fb, timer=FakeTimer()).run(reqs, realtime=False)
    assert len(rep.results) == 12 and rep.rejected_full > 0


def test_request_larger_than_the_pool_is_an_error():
    reqs = [serve.Request(0, {"n_beads": 50, "rid": 0}, np.zeros((50, 3)), np.array([50], np.int32), 3)]
    with pytest.raises(RuntimeError):
        serve.Server(chunk=4, batch=FakeBatch(4, 100), timer=FakeTimer()).run(reqs, realtime=False)


def test_poisson_arrivals_have_the_requested_rate():
    t = serve.poisson_arrivals(20000, 200.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert t[-1] / 20000 == pytest.approx(1 / 200.0, rel=0.03)
