"""Serving runtime: continuous batching under a device-memory budget.
Requests that arrive while others run are admitted as memory frees up, and
each result equals the same request solved alone."""
import numpy as np
import pytest

from paper_1607_00531_gb300 import phantoms as ph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00531_gb300 import build, sac as S
    build.build()
    return S


def requests():
    specs = [((32, 40), 1), ((12, 70, 9), 1), ((24, 150), 1), ((8, 9, 30), 2), ((6, 100, 5), 1),
             ((30, 33), 1), ((10, 48, 12), 1), ((40, 40), 1)]
    out = []
    for i, (m, pe) in enumerate(specs):
        w = ph.small_workload(m, pe, seed=100 + i, peak_px=2.0, max_d=0.5)
        out.append(ph.make_pair(w, dtype=np.float32))
    return out


def params(sac, max_iter=40):
    return sac.params(alpha=1.0, rho=100.0, max_iter=max_iter, eps_abs=0.0, eps_rel=2e-3, prec="mixed")


def solve_alone(sac, d, p):
    srv = sac.Server(p, pool_bytes=64 << 20, max_jobs=1)
    g = sac.grid(d["m"], d["h"], d["pe"])
    t = srv.submit(g, d["I1"], d["I2"])
    while srv.poll(t)["state"] != 2:
        srv.step(10, chunk=5)
    info = srv.poll(t)
    b = srv.fetch(t)
    srv.close()
    return b, info


def test_results_are_the_same_alone_and_in_the_mix(sac):
    reqs = requests()
    p = params(sac)
    srv = sac.Server(p, pool_bytes=256 << 20, max_jobs=16)
    tickets = []
    # staggered arrivals: two requests, a step, three more, a step, the rest
    for batch in (reqs[:2], reqs[2:5], reqs[5:]):
        for d in batch:
            tickets.append(srv.submit(sac.grid(d["m"], d["h"], d["pe"]), d["I1"], d["I2"]))
        srv.step(7, chunk=7)
    while any(srv.poll(t)["state"] != 2 for t in tickets):
        srv.step(10, chunk=5)
    mix = [(srv.poll(t), srv.fetch(t)) for t in tickets]
    srv.close()
    for d, (info, b) in zip(reqs, mix):
        b1, info1 = solve_alone(sac, d, p)
        assert info["iters"] == info1["iters"] and info["converged"] == info1["converged"]
        np.testing.assert_array_equal(b, b1)
        assert np.abs(b).max() > 0


def test_admission_is_bounded_by_the_memory_budget(sac):
    reqs = requests()[:6]
    p = params(sac, max_iter=20)
    # a pool that holds about two of these requests (plus the job table) at a time
    probe = sac.Server(p, pool_bytes=1 << 20, max_jobs=1)
    need = max(probe.request_bytes(sac.grid(d["m"], d["h"], d["pe"])) for d in reqs)
    probe.close()
    budget = int(2.2 * need) + (32 << 10)   # the engine tables of a few small jobs are a few KB
    srv = sac.Server(p, pool_bytes=budget, max_jobs=16)
    tickets = [srv.submit(sac.grid(d["m"], d["h"], d["pe"]), d["I1"], d["I2"]) for d in reqs]
    peak_running, steps = 0, 0
    while any(srv.poll(t)["state"] != 2 for t in tickets) and steps < 200:
        nr, nq = srv.step(5, chunk=5)
        peak_running = max(peak_running, nr)
        assert srv.totals()["pool_used"] <= budget
        steps += 1
    assert all(srv.poll(t)["state"] == 2 for t in tickets)
    assert 1 <= peak_running < len(reqs)            # not everything fit at once
    infos = [srv.poll(t) for t in tickets]
    assert all(i["t_done"] >= i["t_admit"] >= i["t_submit"] for i in infos)
    srv.close()


def test_oversized_request_is_refused(sac):
    d = requests()[0]
    srv = sac.Server(params(sac), pool_bytes=1 << 16, max_jobs=4)
    with pytest.raises(sac.SacError) as e:
        srv.submit(sac.grid(d["m"], d["h"], d["pe"]), d["I1"], d["I2"])
    assert e.value.status == sac.SAC_ENOMEM
    srv.close()
