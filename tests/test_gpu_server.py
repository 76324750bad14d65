"""Continuous-batching server: requests admitted while others run, by device memory;
each result is the same as the request solved alone."""
import numpy as np
import pytest

from paper_2010_06697_gb300 import build, rve, synth

pytestmark = pytest.mark.gpu
PAR = synth.two_phase_params(1.0, 10.0)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    rve.lib()


def request(i, n, kind, dim=3):
    seed = 1000 + i
    Fbar = synth.random_fbar(seed, 54, amp=0.05)
    if kind == "lce":
        ph = np.zeros((n,) * 3, np.uint8)
        return dict(phase=ph, params=np.array([[1.0, 20.0, 4.0, 0.1, (2.0 / n) ** 2]]), Fbar=Fbar, model="lce",
                    n0=synth.director_grf(n, seed, 3.0))
    ph = synth.laminate_phase(n, dim) if kind == "laminate" else synth.inclusion_phase(n, dim, seed, radius=3)
    return dict(phase=ph, params=PAR, Fbar=Fbar, model="neohookean", n0=None)


def alone(req, precision, tol, max_iter):
    s = rve.Rve(req["phase"].ndim, req["phase"].shape[0], req["model"], precision, max_iter=max_iter)
    s.set_material(req["phase"], req["params"], req["n0"])
    info = s.solve(req["Fbar"], 10.0, tol)
    return info, s.stress()


REQS = [(12, "inclusion"), (16, "laminate"), (12, "lce"), (24, "inclusion"), (8, "laminate"), (18, "inclusion"),
        (16, "lce"), (32, "laminate")]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_server_results_equal_alone_with_staggered_arrivals(precision):
    tol, max_iter = (1e-8, 400)
    reqs = [request(i, n, k) for i, (n, k) in enumerate(REQS)]
    srv = rve.Server(64 << 30, precision, max_iter=max_iter, check_every=8)
    tickets = {}
    pending = list(range(len(reqs)))
    results = {}
    step = 0
    while pending or len(results) < len(reqs):
        # two new requests every other tick while others are running
        if pending and step % 2 == 0:
            for _ in range(min(2, len(pending))):
                i = pending.pop(0)
                r = reqs[i]
                tickets[i] = srv.submit(r["phase"], r["params"], r["Fbar"], 10.0, tol, r["model"], r["n0"])
        srv.step()
        for i, t in tickets.items():
            if i not in results:
                out = srv.poll(t)
                if out is not None:
                    results[i] = out
        step += 1
        assert step < 10000
    overlapped = srv.stats()
    for i, r in enumerate(reqs):
        status, S, info, lat, qw = results[i]
        a_info, a_S = alone(r, precision, tol, max_iter)
        d = r["phase"].ndim
        assert info.iterations == a_info.iterations
        assert np.array_equal(S[:d, :d], a_S), (i, S, a_S)
        assert lat >= qw >= 0
    assert overlapped["completed"] == len(reqs)


def test_server_admits_by_memory_budget_and_cancels():
    o = rve.rve_default_options()
    o.precision = rve.RVE_FP64
    one = rve.rve_workspace_bytes(3, 16, rve.RVE_NEOHOOKE, o)
    srv = rve.Server(int(2.5 * one), "fp64", max_iter=200, check_every=8)
    reqs = [request(i, 16, "inclusion") for i in range(5)]
    ts = [srv.submit(r["phase"], r["params"], r["Fbar"], 10.0, 1e-8) for r in reqs]
    a, q = srv.step()
    assert a == 2 and q == 3          # only two workspaces fit
    assert srv.cancel(ts[4]) == rve.RVE_OK   # queued
    assert srv.cancel(ts[0]) == rve.RVE_OK   # running
    assert srv.cancel(ts[0]) == rve.RVE_E_NOT_FOUND
    done = {}
    for _ in range(2000):
        srv.step()
        for t in ts[1:4]:
            if t not in done:
                out = srv.poll(t)
                if out is not None:
                    done[t] = out
        if len(done) == 3:
            break
    assert len(done) == 3 and all(v[0] == rve.RVE_OK for v in done.values())
    assert srv.stats()["bytes"] <= int(2.5 * one)


def test_server_rejects_bad_requests():
    o = rve.rve_default_options()
    one = rve.rve_workspace_bytes(3, 32, rve.RVE_NEOHOOKE, o)
    srv = rve.Server(one // 2, "fp64")
    r = request(0, 32, "inclusion")
    with pytest.raises(rve.RveError) as e:
        srv.submit(r["phase"], r["params"], r["Fbar"], 10.0, 1e-8)
    assert e.value.code == rve.RVE_E_OOM
    with pytest.raises(rve.RveError) as e:
        srv.submit(r["phase"] + 7, r["params"], r["Fbar"], 10.0, 1e-8)
    assert e.value.code == rve.RVE_E_INVALID_ARG
    with pytest.raises(rve.RveError) as e:
        srv.poll(12345)
    assert e.value.code == rve.RVE_E_NOT_FOUND
