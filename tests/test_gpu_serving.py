"""Serving loop (continuous batching) through the C ABI: results are the same
alone and in a mix, requests overlap on the device, admission respects the
memory budget (evicting idle resident plans), and oversized requests fail."""
import numpy as np
import pytest

from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

MIX = [((16, 16), 2, 8, 4, D.DYSON_FP64), ((24, 20), 3, 6, 3, D.DYSON_MIXED),
       ((6, 5, 9), 2, 5, 2, D.DYSON_FP64), ((40, 64), 4, 12, 5, D.DYSON_MIXED),
       ((16, 16), 2, 8, 4, D.DYSON_FP64), ((64, 64), 4, 16, 6, D.DYSON_MIXED)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1102_3137_gb300 import build
    build.build()
    D.load()


def request_inputs(L, p, k, K, seed):
    w = I.Workload("r", tuple(L), -1.0, 0.0, 0.01, 0.5, 10.0, K, p, k, seed)
    omega, V, sigma, q1 = I.make_inputs(w)
    return w, omega, V, sigma, q1


def alone(w, omega, V, sigma, q1, prec):
    pl = D.Plan(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=w.K)
    out = pl.solve(omega, V, sigma, q1)
    pl.close()
    return out


def test_mix_equals_alone_and_overlaps():
    srv = D.dyson_server_create(8 << 30, max_inflight=6)
    jobs = []
    for n, (L, p, k, K, prec) in enumerate(MIX):
        w, omega, V, sigma, q1 = request_inputs(L, p, k, K, 100 + n)
        geom = D.make_geometry(L, w.t, w.mu, p, k, prec, max_freqs=K)
        out = np.zeros((K, w.N), complex)
        st = np.zeros(K, np.int32)
        t = D.dyson_submit(srv, geom, K, omega, V, sigma, q1, out, st)
        jobs.append((t, w, omega, V, sigma, q1, prec, out, st))
    lats = []
    for t, w, omega, V, sigma, q1, prec, out, st in jobs:
        lat, run = D.dyson_wait(srv, t)
        lats.append(lat)
        assert lat >= run >= 0
        ref = alone(w, omega, V, sigma, q1, prec)
        assert np.array_equal(out, ref)
        assert np.all((st & D.DYSON_ST_NO_CONVERGENCE) == 0)
    stats = D.dyson_server_stats(srv)
    assert stats["completed"] == len(MIX) and stats["queued"] == 0 and stats["running"] == 0
    assert stats["peak_running"] >= 2
    # a later request with a resident geometry reuses its plan (no new plan)
    t, w, omega, V, sigma, q1, prec, out, st = jobs[0]
    created = stats["plans_created"]
    out2 = np.zeros_like(out)
    geom = D.make_geometry(w.L, w.t, w.mu, w.p, w.k, prec, max_freqs=w.K)
    D.dyson_wait(srv, D.dyson_submit(srv, geom, w.K, omega, V, sigma, q1, out2))
    assert np.array_equal(out2, out)
    assert D.dyson_server_stats(srv)["plans_created"] == created
    D.dyson_server_destroy(srv)


def test_budget_forces_eviction_and_serialisation():
    geoms = [((40, 64), 4, 8, 3), ((64, 64), 4, 8, 3), ((40, 64), 4, 8, 3)]
    need = max(D.dyson_plan_footprint(D.make_geometry(L, p=p, k_max=k, max_freqs=K))
               for L, p, k, K in geoms)
    srv = D.dyson_server_create(need + need // 2, max_inflight=4)   # room for one plan at a time
    jobs = []
    for n, (L, p, k, K) in enumerate(geoms):
        w, omega, V, sigma, q1 = request_inputs(L, p, k, K, 200 + n)
        geom = D.make_geometry(L, w.t, w.mu, p, k, D.DYSON_FP64, max_freqs=K)
        out = np.zeros((K, w.N), complex)
        jobs.append((D.dyson_submit(srv, geom, K, omega, V, sigma, q1, out), w, omega, V, sigma, q1, out))
    for t, w, omega, V, sigma, q1, out in jobs:
        D.dyson_wait(srv, t)
        assert np.array_equal(out, alone(w, omega, V, sigma, q1, D.DYSON_FP64))
    stats = D.dyson_server_stats(srv)
    assert stats["plans_evicted"] >= 1 and stats["peak_bytes"] <= need + need // 2
    D.dyson_server_destroy(srv)


def test_oversized_request_is_rejected():
    srv = D.dyson_server_create(1 << 20, max_inflight=2)
    w, omega, V, sigma, q1 = request_inputs((64, 64), 4, 16, 4, 7)
    geom = D.make_geometry(w.L, p=4, k_max=16, max_freqs=4)
    with pytest.raises(D.DysonError) as e:
        D.dyson_submit(srv, geom, 4, omega, V, sigma, q1, np.zeros((4, w.N), complex))
    assert e.value.code == -5
    D.dyson_server_destroy(srv)
