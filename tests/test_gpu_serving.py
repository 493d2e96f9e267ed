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


@pytest.mark.parametrize("prec,tol", [(D.DYSON_FP64, 1e-10), (D.DYSON_MIXED, 1e-6)])
def test_request_larger_than_plan_runs_in_chunks_and_matches_oracle(prec, tol):
    """K = 7 frequencies on a plan holding 3: three consecutive chunks on one stream.
    16^2 with p = 2 has m = 16 interface sites; with the cap at 24 the Krylov space closes and
    the served diagonal is the oracle's low-rank diagonal, itself the exact one."""
    from oracle import dyson_oracle as O
    K, cap = 7, 3
    w, omega, V, sigma, q1 = request_inputs((16, 16), 2, 24, K, 31)
    srv = D.dyson_server_create(4 << 30, max_inflight=2)
    geom = D.make_geometry(w.L, w.t, w.mu, 2, 24, prec, max_freqs=cap)
    out = np.zeros((K, w.N), complex)
    st = np.zeros(K, np.int32)
    D.dyson_wait(srv, D.dyson_submit(srv, geom, K, omega, V, sigma, q1, out, st))
    D.dyson_server_destroy(srv)
    assert np.all(st & D.DYSON_ST_TERMINATED)
    ref = alone(w, omega, V, sigma, q1, prec)
    assert np.max(np.abs(out - ref) / np.abs(ref)) <= (1e-12 if prec == D.DYSON_FP64 else 1e-7)
    for k in range(K):
        lr = O.lowrank_diag(w.L, (False,) * 3, w.t, w.mu, V, sigma[k], omega[k], q1, 2, 24)
        ex = O.exact_diag(w.L, (False,) * 3, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]))
        assert np.max(np.abs(lr - ex) / np.abs(ex)) <= 1e-10
        assert np.max(np.abs(out[k] - lr) / np.abs(lr)) <= tol


def test_small_request_backfills_past_one_waiting_for_memory():
    """A large request that must wait for memory (the budget holds one large plan)
    does not hold up a later small request whose plan is resident and idle: the
    small one runs at once, while the large one waits for the running one."""
    small, big_a, big_b = ((16, 16), 2, 8, 2), ((128, 128), 4, 32, 16), ((128, 96), 4, 32, 16)
    need = {g: D.dyson_plan_footprint(D.make_geometry(g[0], p=g[1], k_max=g[2], max_freqs=g[3]))
            for g in (small, big_a, big_b)}
    assert need[big_b] > 2 * need[small]
    srv = D.dyson_server_create(need[big_a] + 2 * need[small], max_inflight=4)

    def submit(g, seed):
        w, omega, V, sigma, q1 = request_inputs(g[0], g[1], g[2], g[3], seed)
        geom = D.make_geometry(w.L, w.t, w.mu, g[1], g[2], D.DYSON_FP64, max_freqs=g[3])
        out = np.zeros((g[3], w.N), complex)
        return D.dyson_submit(srv, geom, g[3], omega, V, sigma, q1, out), (w, omega, V, sigma, q1, out)

    # the host buffers of a request must stay alive until its dyson_wait returns
    t0, keep0 = submit(small, 41)
    D.dyson_wait(srv, t0)                       # the small plan is now resident and idle
    ta, keep_a = submit(big_a, 42)
    tb, keep_b = submit(big_b, 43)              # waits: big_a runs, the budget holds one large plan
    ts, (w, omega, V, sigma, q1, out) = submit(small, 44)
    lat_s, _ = D.dyson_wait(srv, ts)
    lat_b, _ = D.dyson_wait(srv, tb)
    D.dyson_wait(srv, ta)
    del keep0, keep_a, keep_b
    assert lat_s < lat_b
    assert np.array_equal(out, alone(w, omega, V, sigma, q1, D.DYSON_FP64))
    stats = D.dyson_server_stats(srv)
    assert stats["completed"] == 4 and stats["peak_bytes"] <= need[big_a] + 2 * need[small]
    D.dyson_server_destroy(srv)


@pytest.mark.parametrize("prec,tol", [(D.DYSON_FP64, 1e-10), (D.DYSON_MIXED, 1e-6)])
def test_requests_of_one_geometry_fuse_into_one_solve(prec, tol):
    """Four requests of uneven K (3, 5, 2, 6) on one geometry, with the same V and start
    vector, queue behind a running request and then run as one fused solve of 16
    frequencies; each result matches its own solve alone and the exact diagonal (16^2,
    p = 2: m = 16, the cap of 24 closes the Krylov space)."""
    from oracle import dyson_oracle as O
    srv = D.dyson_server_create(8 << 30, max_inflight=1)
    wb, ob, Vb, sb, qb = request_inputs((128, 128), 4, 32, 16, 60)      # runs first, the rest queue
    gb = D.make_geometry(wb.L, wb.t, wb.mu, 4, 32, prec, max_freqs=16)
    outb = np.zeros((16, wb.N), complex)
    tb = D.dyson_submit(srv, gb, 16, ob, Vb, sb, qb, outb)
    _, _, V, _, q1 = request_inputs((16, 16), 2, 24, 1, 70)              # shared V and start vector
    geom = D.make_geometry((16, 16), -1.0, 0.0, 2, 24, prec, max_freqs=16)
    jobs = []
    for n, K in enumerate((3, 5, 2, 6)):
        w, omega, _, sigma, _ = request_inputs((16, 16), 2, 24, K, 71 + n)
        out = np.zeros((K, w.N), complex)
        st = np.zeros(K, np.int32)
        jobs.append((D.dyson_submit(srv, geom, K, omega, V, sigma, q1, out, st), w, omega, sigma, out, st))
    D.dyson_wait(srv, tb)
    for t, w, omega, sigma, out, st in jobs:
        D.dyson_wait(srv, t)
    stats = D.dyson_server_stats(srv)
    D.dyson_server_destroy(srv)
    assert stats["fused"] == 4 and stats["completed"] == 5
    for t, w, omega, sigma, out, st in jobs:
        assert np.all(st & D.DYSON_ST_TERMINATED)
        ref = alone(w, omega, V, sigma, q1, prec)
        assert np.max(np.abs(out - ref) / np.abs(ref)) <= tol
        for k in range(w.K):
            ex = O.exact_diag(w.L, (False,) * 3, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]))
            assert np.max(np.abs(out[k] - ex) / np.abs(ex)) <= tol
