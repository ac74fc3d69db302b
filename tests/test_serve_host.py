"""Host-side scheduling of the OTOC server, driven by a fake batch (no GPU):
FIFO admission without overtaking, admission refused beyond slot/memory
limits, every request completes once, latency accounting."""
import numpy as np

from paper_2311_00639_b300 import serve


class FakeTerms:
    closed = 0

    def __init__(self, r):
        self.N = r.N

    def close(self):
        FakeTerms.closed += 1


class FakeBatch:
    """Admits while slots and 'bytes' allow; a job finishes after `work` ticks."""

    def __init__(self, slots, budget):
        self.slots, self.budget, self.used = slots, budget, 0
        self.live = {}  # tag -> [remaining ticks, bytes]
        self.admitted_order = []
        self.max_live = 0
        self.clock = 0.0

    def submit(self, h, a, b, beta, tg, seed, sid, tag):
        need = 2 ** (h.N // 2)
        if len(self.live) >= self.slots or self.used + need > self.budget:
            return False
        self.live[tag] = [len(tg), need]
        self.used += need
        self.admitted_order.append(tag)
        self.max_live = max(self.max_live, len(self.live))
        return True

    def run(self, max_ticks, ticks_per_sync):
        out = []
        for _ in range(max_ticks):
            self.clock += 1e-3
            for tag in list(self.live):
                self.live[tag][0] -= 1
                if self.live[tag][0] <= 0:
                    self.used -= self.live.pop(tag)[1]
                    F = np.ones(3, dtype=complex)
                    out.append({"tag": tag, "F": F, "otoc": F.real, "matvecs": 1, "status": 0})
            if out:
                break
        return out

    def close(self):
        pass


def test_fifo_admission_limits_and_latency():
    reqs = [serve.Request(i, 0.0005 * i, 10 + 2 * (i % 4), None, None, 1.0, np.zeros(3 + i % 5), seed=i)
            for i in range(40)]
    fb = FakeBatch(slots=3, budget=2 ** 8)
    t = [0.0]

    def clock():
        t[0] += 1e-4
        return t[0]

    srv = serve.OtocServer(batch=fb, make_terms=FakeTerms, ticks_per_step=2)
    res = srv.run(reqs, clock=clock, sleep=lambda s: None)
    assert sorted(r.rid for r in res) == list(range(40))  # each once
    assert fb.admitted_order == sorted(fb.admitted_order)  # FIFO, no overtaking
    assert fb.max_live <= 3 and fb.used == 0
    assert all(r.done >= r.admitted >= r.arrival for r in res)
    assert FakeTerms.closed == 40
    s = serve.summarize(res, wall=t[0])
    assert s["requests"] == 40 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_sjf_admission_prefers_short_requests():
    """With every request waiting at t = 0 and one slot, SJF admits in order of
    estimated work (terms x D x (points + sum |t|)); equal work keeps arrival
    order.  FIFO admits in arrival order."""
    grids = [np.linspace(0, 8, 9), np.linspace(0, 1, 2), np.linspace(0, 4, 5), np.linspace(0, 1, 2)]
    reqs = [serve.Request(i, 0.0, 10, None, np.zeros(5), 1.0, grids[i], seed=i) for i in range(4)]
    order = {}
    for policy in ("fifo", "sjf"):
        fb = FakeBatch(slots=1, budget=2 ** 10)
        t = [0.0]

        def clock():
            t[0] += 1e-4
            return t[0]

        srv = serve.OtocServer(batch=fb, make_terms=FakeTerms, ticks_per_step=2, policy=policy)
        res = srv.run(reqs, clock=clock, sleep=lambda s: None)
        assert sorted(r.rid for r in res) == [0, 1, 2, 3]
        order[policy] = fb.admitted_order
    assert order["fifo"] == [0, 1, 2, 3]
    assert order["sjf"] == [1, 3, 2, 0]


def test_poisson_and_percentiles():
    arr = serve.poisson_arrivals(20000, rate=50.0, seed=1)
    gaps = np.diff(np.concatenate([[0.0], arr]))
    assert abs(gaps.mean() - 1 / 50.0) < 0.05 / 50.0 * 10
    assert np.all(np.diff(arr) > 0)
    assert serve.percentile([1, 2, 3, 4, 5], 50) == 3.0
    assert serve.percentile([1, 2, 3, 4, 5], 100) == 5.0
    assert abs(serve.percentile(np.arange(101), 99) - 99.0) < 1e-12


def test_served_workload_distribution():
    import syk_inputs as si

    reqs = si.served_requests(300, rate=10.0, seed=2, t_max=1.0, dt=0.5)
    Ns = np.array([r["N"] for r in reqs])
    assert Ns.min() >= 28 and Ns.max() <= 48 and np.all(Ns % 2 == 0)
    assert np.mean(Ns == 28) > np.mean(Ns == 34) > 0  # weighted toward small N
    assert {r["beta"] for r in reqs} <= {2.0, 5.0, 10.0, 20.0}
    assert np.allclose(reqs[0]["t_grid"], [0.0, 0.5, 1.0])
    arr = np.array([r["arrival"] for r in reqs])
    assert np.allclose(arr, serve.poisson_arrivals(300, rate=10.0, seed=2))


def _req(rid, N, n_terms, t_max, dt=1.0):
    return serve.Request(rid=rid, arrival=0.0, N=N, quads=np.zeros((n_terms, 4), np.int32), J=np.ones(n_terms),
                         beta=1.0, t_grid=np.arange(0.0, t_max + 1e-9, dt), seed=0)


def test_calibrated_rate_uses_work_not_request_counts():
    """A capacity sample lighter than the served one must lower the rate in
    proportion to the served sample's mean work (the heavy-tailed mix)."""
    light = [_req(i, 28, 100, 2.0) for i in range(10)]
    heavy = [_req(i, 28, 100, 2.0) for i in range(9)] + [_req(9, 36, 100, 2.0)]  # one request 16x heavier
    w = serve.work_estimate(light[0], None)
    assert w == 100 * 2 ** 13 * (3 + 3.0)  # terms x D x (grid points + sum |t|)
    rate_same, cap_same = serve.calibrated_rate(light, 2.0, light, 0.75)
    assert abs(cap_same - 5.0) < 1e-12 and abs(rate_same - 3.75) < 1e-12  # 10 requests in 2 s
    rate, cap = serve.calibrated_rate(light, 2.0, heavy, 0.75)
    assert abs(cap - 5.0 * 10 / (9 + 16)) < 1e-12
    assert abs(rate - 0.75 * cap) < 1e-12
    try:
        serve.calibrated_rate(light, 0.0, heavy, 0.75)
        assert False, "zero wall time accepted"
    except ValueError:
        pass


def test_summarize_windows_report_offered_load():
    res = [serve.Result(rid=i, N=28, F=None, otoc=None, arrival=float(i), admitted=float(i), done=float(i) + 1.0,
                        matvecs=1, status=0) for i in range(8)]
    work = {i: (3.0 if i >= 4 else 1.0) for i in range(8)}
    s = serve.summarize(res, 9.0, windows=2, work=work, capacity_work_per_s=2.0)
    w0, w1 = s["windows"]
    assert abs(w0["offered_load"] - 4 * 1.0 / 4.0 / 2.0) < 1e-12  # 4 units over arrivals 0..4
    assert abs(w1["offered_load"] - 4 * 3.0 / 3.0 / 2.0) < 1e-12  # last window: span 4..7
    assert w0["p50_latency_s"] == 1.0 and s["requests"] == 8
    assert "offered_load" not in serve.summarize(res, 9.0, windows=2)["windows"][0]
