"""Wide slices (3D slabs, slice width W = Ly * h in (64, 320]): the global-memory
factor kernel and the row-chunked sweeps, against the oracle through the C ABI.

Geometries and the paths they take (FP64 / mixed):
  (6, 9, 16)  p = 2: W = 72   row chunks (FP64) / one chunk per block (complex64)
  (4, 16, 17) p = 2: W = 128  chunked / chunked
  (5, 12, 26) p = 2: W = 156  chunked, W not a multiple of the 32-wide tiles
  (3, 16, 33) p = 2: W = 256
  (8, 24, 25), (48, 24, 25) p = 2: W = 288, the slice of 48^3 slabs with p = 8
  (the second with 48 slices, where only the complex64 row buffer stays on chip)
"""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I
from parity_util import (OPEN, TOL_FP64, TOL_MIXED, oracle_parts, plan_for, relerr, rounding_bound,
                         stepwise_check, wl)

pytestmark = pytest.mark.gpu

WIDE = [((6, 9, 16), 2), ((4, 16, 17), 2), ((5, 12, 26), 2), ((3, 16, 33), 2)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1102_3137_gb300 import build
    build.build()
    D.load()


def test_geometries_are_wide():
    for L, p in WIDE:
        heights, m, ndd = D.dyson_partition(D.make_geometry(L, p=p))
        assert 64 < L[1] * max(heights) <= 256


@pytest.mark.parametrize("L,p", WIDE)
def test_wide_subdomain_diag_and_solve_fp64(L, p):
    w = wl(L, p, 4, K=3)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w)
    dB = np.zeros((3, w.N), complex)
    D.dyson_subdomain_diag(pl.handle, 3, omega, V, sigma, dB)
    rng = np.random.default_rng(5)
    q = rng.normal(size=(3, w.N)) + 1j * rng.normal(size=(3, w.N))
    wv = np.zeros_like(q)
    D.dyson_subdomain_solve(pl.handle, 3, omega, V, sigma, q, wv)
    for k in range(3):
        subs = O.Subdomains(w.L, OPEN, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]), p)
        mask = np.ones(w.N, bool)
        mask[np.concatenate(subs.iface)] = False
        assert np.all(dB[k][~mask] == 0)
        assert relerr(dB[k][mask], subs.diagB[mask]) < 1e-12
        ref = subs.solve(q[k])
        assert np.max(np.abs(wv[k] - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("L,p", WIDE[:2])
def test_wide_subdomain_mixed(L, p):
    w = wl(L, p, 4, K=2)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, D.DYSON_MIXED)
    dB = np.zeros((2, w.N), complex)
    D.dyson_subdomain_diag(pl.handle, 2, omega, V, sigma, dB)
    rng = np.random.default_rng(6)
    q = rng.normal(size=(2, w.N)) + 1j * rng.normal(size=(2, w.N))
    wv = np.zeros_like(q)
    D.dyson_subdomain_solve(pl.handle, 2, omega, V, sigma, q, wv)
    for k in range(2):
        subs = O.Subdomains(w.L, OPEN, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]), p)
        mask = subs.diagB != 0
        assert relerr(dB[k][mask], subs.diagB[mask]) < 1e-10      # double-float recursion (R12)
        ref = subs.solve(q[k])
        assert np.max(np.abs(wv[k] - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("L,p", WIDE[:3])
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, 1e-11), (D.DYSON_MIXED, 1e-9)])
def test_wide_xmatvec(L, p, precision, tol):
    w = wl(L, p, 4, K=2)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, precision)
    rng = np.random.default_rng(9)
    q = rng.normal(size=(2, w.N)) + 1j * rng.normal(size=(2, w.N))
    u = np.zeros_like(q)
    D.dyson_xmatvec(pl.handle, 2, omega, V, sigma, q, u)
    for k in range(2):
        ref = O.xmatvec(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], p, q[k])
        assert np.max(np.abs(u[k] - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_wide_solve_terminated(precision, tol):
    """(4, 16, 17), p = 2: one interface layer of m = 64 sites; with the cap at 72
    the Krylov space of X closes and diag(G) is the exact diagonal."""
    w = wl((4, 16, 17), 2, 72, K=3, seed=2)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, precision)
    st = np.zeros(w.K, np.int32)
    out = pl.solve(omega, V, sigma, q1, status=st)
    assert np.all(st & D.DYSON_ST_TERMINATED)
    for k in range(w.K):
        ex = O.exact_diag(w.L, OPEN, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]))
        assert relerr(out[k], ex) <= tol


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_wide_solve_truncated_stepwise(precision, tol):
    w = wl((5, 12, 26), 2, 10, K=2, seed=4)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, precision)
    out = pl.solve(omega, V, sigma, q1)
    info = pl.info(w.K)
    for k in range(w.K):
        subs, X = oracle_parts(w, omega[k], V, sigma[k])
        assert stepwise_check(w, pl, k, subs, X, q1, out[k], info, tol) == w.k


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_cubic32_full_batch_sampled(precision, tol):
    """32^3, K = 128 in one launch, p = 8 (W = 128), k = 48: the 3D workload;
    two sampled frequencies checked step by step against the oracle's X."""
    w = I.WORKLOADS["cubic32_K128_p8_k48"]
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, precision)
    st = np.zeros(w.K, np.int32)
    out = pl.solve(omega, V, sigma, q1, status=st)
    info = pl.info(w.K)
    assert np.all((st & (D.DYSON_ST_NO_CONVERGENCE | D.DYSON_ST_BREAKDOWN)) == 0)
    assert np.all(np.isfinite(out))
    for k in (0, w.K - 1):
        subs, X = oracle_parts(w, omega[k], V, sigma[k])
        stepwise_check(w, pl, k, subs, X, q1, out[k], info, tol)


def test_square512_full_batch_sampled():
    """512^2, K = 32 in one launch, p = 16 (clusters of 16 CTAs), k = 64: the largest
    2D workload and the benchmark's.  Both forms; the lowest frequency (the worst
    conditioned) checked step by step against the oracle's X, and the lowest and the
    highest directly against the oracle's diagonal within max(tol, amplification *
    1e-13) (the amplification of X-matvec rounding, measured on the oracle alone:
    at most ~6e4 here, so the mixed form is held to 1e-6)."""
    name = "square512_K32_p16_k64"
    w = I.WORKLOADS[name]
    omega, V, sigma, q1 = I.make_inputs(w)
    runs = []
    for precision, tol in ((D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)):
        pl = plan_for(w, precision)
        st = np.zeros(w.K, np.int32)
        out = pl.solve(omega, V, sigma, q1, status=st)
        info = pl.info(w.K)
        assert np.all((st & (D.DYSON_ST_NO_CONVERGENCE | D.DYSON_ST_BREAKDOWN)) == 0)
        assert np.all(np.isfinite(out))
        runs.append((pl, out, info, tol))
    for k in (0, 31):
        subs, X = oracle_parts(w, omega[k], V, sigma[k])
        base = subs.diagB + O.cs_lanczos(X, q1, w.k)[0]
        for pl, out, info, tol in runs:
            if k == 0:
                assert stepwise_check(w, pl, 0, subs, X, q1, out[0], info, tol) == w.k
            assert relerr(out[k], base) <= rounding_bound(name, k, tol), (k, tol)
    assert rounding_bound(name, 0, TOL_MIXED) == TOL_MIXED
    for pl, _, _, _ in runs:
        pl.close()


@pytest.mark.parametrize("L,precision,tol", [((8, 24, 25), D.DYSON_FP64, TOL_FP64),
                                             ((48, 24, 25), D.DYSON_MIXED, TOL_MIXED)])
def test_slice_width_288(L, precision, tol):
    """W = 24 * 12 = 288 > 256: diag(B^-1), the subdomain solve, the X-matvec and a
    truncated solve (checked step by step) against the oracle."""
    w = wl(L, 2, 8, K=2, seed=8)
    heights, _, _ = D.dyson_partition(D.make_geometry(L, p=2))
    assert L[1] * max(heights) == 288
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = plan_for(w, precision)
    dB = np.zeros((2, w.N), complex)
    D.dyson_subdomain_diag(pl.handle, 2, omega, V, sigma, dB)
    rng = np.random.default_rng(12)
    q = rng.normal(size=(2, w.N)) + 1j * rng.normal(size=(2, w.N))
    wv = np.zeros_like(q)
    u = np.zeros_like(q)
    D.dyson_subdomain_solve(pl.handle, 2, omega, V, sigma, q, wv)
    D.dyson_xmatvec(pl.handle, 2, omega, V, sigma, q, u)
    sweep_tol, xm_tol = (1e-12, 1e-11) if precision == D.DYSON_FP64 else (1e-5, 1e-9)
    for k in range(2):
        subs = O.Subdomains(w.L, OPEN, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]), 2)
        mask = subs.diagB != 0
        # binary64 recursion in the FP64 form, double-float in the mixed form (R12)
        assert relerr(dB[k][mask], subs.diagB[mask]) < (1e-12 if precision == D.DYSON_FP64 else 1e-10)
        ref = subs.solve(q[k])
        assert np.max(np.abs(wv[k] - ref)) <= sweep_tol * np.max(np.abs(ref))
        ref = O.xmatvec(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], 2, q[k])
        assert np.max(np.abs(u[k] - ref)) <= xm_tol * np.max(np.abs(ref))
    st = np.zeros(w.K, np.int32)
    out = pl.solve(omega, V, sigma, q1, status=st)
    assert np.all((st & (D.DYSON_ST_NO_CONVERGENCE | D.DYSON_ST_BREAKDOWN)) == 0)
    info = pl.info(w.K)
    for k in range(w.K):
        subs, X = oracle_parts(w, omega[k], V, sigma[k])
        assert stepwise_check(w, pl, k, subs, X, q1, out[k], info, tol) == w.k
    pl.close()
