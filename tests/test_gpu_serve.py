"""Serving loop on the GPU: requests that arrive while others run join the
running batch, and every served result equals the same request computed
alone (bitwise: each job's arithmetic is independent of its neighbours)."""
import numpy as np
import pytest

import syk_inputs as si

pytestmark = pytest.mark.gpu


def test_served_results_equal_alone():
    import paper_2311_00639_b300 as syk
    from paper_2311_00639_b300 import serve

    rng = np.random.default_rng(4)
    reqs = []
    for i in range(10):
        N = int(rng.choice([12, 14, 16, 18, 20, 22]))
        q, J, _ = si.sample_sparse_syk(N, 4, seed=500 + i)
        grid = np.linspace(0.0, 3.0, int(rng.integers(2, 6)))
        reqs.append(serve.Request(i, 0.002 * i, N, q, J, float(rng.choice([0.0, 2.0, 8.0])), grid, seed=77 + i))
    m = 30  # the same Krylov dimension on both sides of the bitwise comparison
    srv = serve.OtocServer(dtype="c64", max_slots=3, hbm_budget_bytes=64 << 20, ticks_per_step=2, m=m)
    served = {r.rid: r for r in srv.run(reqs)}
    srv.close()
    assert sorted(served) == list(range(10))
    s = serve.summarize(list(served.values()), wall=max(r.done for r in served.values()))
    assert s["failed"] == 0 and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    for r in reqs:
        with syk.Terms(r.N, r.quads, r.J, dtype="c64") as h, syk.Batch(dtype="c64", max_slots=1, max_bytes=64 << 20, m=m) as b:
            assert b.submit(h, r.N - 1, r.N - 2, r.beta, r.t_grid, r.seed, 0, 0)
            alone = b.drain()[0]["F"]
        assert np.array_equal(alone, served[r.rid].F), r.rid
