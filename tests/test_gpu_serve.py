"""GPU test of the serving loop: requests of uneven size arrive over time (Poisson), join
and leave a running batch; each request's result equals the same request run alone."""
import numpy as np
import pytest

from paper_1611_09160_gb300 import inputs as I
from paper_1611_09160_gb300 import serve, wmcd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    wmcd.build()
    wmcd.load()


def requests(n, rate, seed):
    systems = I.ensemble(n, 16, 256, 1e-3, seed=seed)
    arrivals = serve.poisson_arrivals(n, rate, seed)
    rng = np.random.default_rng(seed)
    out = []
    for k, (s, t) in enumerate(zip(systems, arrivals)):
        prec = wmcd.MIXED if k % 2 else wmcd.FP64
        p = wmcd.default_params(s.n_beads, s.box_L, seed=1000 + k, sim_id=k, precision=prec,
                                planewave_mode=wmcd.PLANEWAVE_PERIODIC)
        out.append(serve.Request(k, p, s.pos, s.chain_len, int(rng.integers(5, 40)), arrival=float(t)))
    return out


def test_results_alone_and_in_the_mix_agree():
    reqs = requests(24, rate=400.0, seed=7)
    pool = 6 * max(wmcd.batch_need(r.params) for r in reqs)     # room for about six at once
    srv = serve.Server(capacity=8, pool_bytes=pool, chunk=6)
    rep = srv.run(reqs, realtime=True)
    srv.close()
    s = rep.summary()
    assert s["requests"] == len(reqs) and s["max_resident"] >= 2
    assert s["sweep_ms_p99"] >= s["sweep_ms_p50"] > 0
    for r in reqs:
        sim = wmcd.Simulation(r.params, r.pos, r.chain_len)
        sim.sweep(r.n_sweeps)
        alone = sim.positions(unwrapped=True)
        st = sim.stats()
        sim.close()
        got = rep.results[r.rid]
        L = r.params["box_L"]
        assert np.max(np.abs(got.positions - alone)) <= 1e-12 * L, r.rid
        assert got.bead_updates == st.bead_updates and got.accepted == st.accepted_total
