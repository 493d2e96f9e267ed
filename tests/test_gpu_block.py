"""Block Lanczos on X (block size nb = 2..4, not in the paper) against the
oracle's block recurrence: exactness on a degenerate spectrum, the block
recurrence checked step by step on truncated runs, and the single-vector
X-matvec of a block plan."""
import math

import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I
from parity_util import OPEN, TOL_FP64, TOL_MIXED, oracle_parts, plan_for, relerr, wl

pytestmark = pytest.mark.gpu

CUBE = (3, 3, 7)       # the 3 x 3 interface plane gives X an eigenvalue of multiplicity 3


def cube_inputs(K=2):
    N = O.site_count(CUBE)
    omega = np.array([math.pi / 10 * (2 * k + 1) for k in range(K)])
    V = np.zeros(N)
    sigma = np.full((K, N), 0.3 + 0.2j, dtype=np.complex128)
    return omega, V, sigma


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_block_exact_on_degenerate_spectrum(precision, tol):
    K, nb, k = 2, 3, 15     # range(X) (9) + the start block's null-space part (3): 4 block steps, then all deflate
    omega, V, sigma = cube_inputs(K)
    N = O.site_count(CUBE)
    Q1 = I.start_block(np.random.default_rng(11).uniform(-1, 1, N), nb)
    exact = np.stack([O.dense_diag_inverse(CUBE, OPEN, -1.0, O.dyson_diagonal(w, 0.0, V, sigma[kk]))
                      for kk, w in enumerate(omega)])
    pl = D.Plan(CUBE, -1.0, 0.0, 2, k, precision, max_freqs=K, block_size=nb)
    st = np.zeros(K, np.int32)
    out = pl.solve(omega, V, sigma, Q1, status=st)
    assert np.all(st == D.DYSON_ST_TERMINATED)
    assert np.all(pl.info(K)["steps"] == 4)
    assert relerr(out, exact) <= tol
    # the scalar method on the same input stops short of range(X)
    ps = D.Plan(CUBE, -1.0, 0.0, 2, k, precision, max_freqs=K)
    st1 = np.zeros(K, np.int32)
    out1 = ps.solve(omega, V, sigma, np.ascontiguousarray(Q1[0]), status=st1)
    assert np.all(st1 == D.DYSON_ST_TERMINATED)
    assert relerr(out1, exact) > 1e-2
    pl.close()
    ps.close()


def block_stepwise(w, pl, kf, subs, X, Q1, out_k, A, B, nsteps, nb, tol):
    """X Q = Q T + R_last E^T, Q^T Q = I on the kept columns, and Eq. 9 per block."""
    n = nsteps * nb
    Q = D.dyson_lanczos_basis(pl.handle, kf, n + nb, w.N)
    Qk = Q[:n].T
    T = np.zeros((n, n), dtype=complex)
    for j in range(nsteps):
        s = slice(nb * j, nb * j + nb)
        T[s, s] = A[j]
        if j > 0:
            sp = slice(nb * (j - 1), nb * j)
            T[s, sp] = B[j]
            T[sp, s] = B[j].T
    nrm = np.linalg.norm(Qk, axis=0)
    keep = nrm > 0
    G = Qk[:, keep].T @ Qk[:, keep]
    assert np.max(np.abs(G - np.eye(keep.sum())) / np.outer(nrm[keep], nrm[keep])) <= tol
    XQ = np.stack([X(Qk[:, j]) for j in range(n)], 1)
    R = XQ - Qk @ T
    R[:, n - nb:] -= Q[n:n + nb].T             # raw (or deflated) residual block of the last step
    scale = np.abs(XQ) + np.abs(Qk) @ np.abs(T)
    scale[:, n - nb:] += np.abs(Q[n:n + nb].T)
    assert np.max(np.abs(R)) <= tol * np.max(scale)
    ref = subs.diagB + np.einsum("ij,jk,ik->i", Qk, T, Qk)
    assert relerr(out_k, ref) <= tol
    return Q


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
@pytest.mark.parametrize("L,p,k,nb", [((24, 30), 3, 12, 2), ((16, 22), 2, 12, 4), ((6, 5, 13), 3, 8, 2)])
def test_block_truncated_stepwise(L, p, k, nb, precision, tol):
    w = wl(L, p, k, K=3)
    omega, V, sigma, q1 = I.make_inputs(w)
    Q1 = I.start_block(q1, nb)
    pl = plan_for(w, precision, block_size=nb)
    st = np.zeros(w.K, np.int32)
    out = pl.solve(omega, V, sigma, Q1, status=st)
    info = pl.info(w.K)
    assert np.all(st == 0) and np.all(info["steps"] == k // nb)
    for kf in range(w.K):
        subs, X = oracle_parts(w, omega[kf], V, sigma[kf])
        Q = block_stepwise(w, pl, kf, subs, X, Q1, out[kf], info["A"][kf], info["B"][kf],
                           int(info["steps"][kf]), nb, tol)
        # first block and A_0 against the oracle's own start-block QR and first step
        acc, As, Bs, Qo, _ = O.cs_block_lanczos(
            lambda Qb: np.stack([X(Qb[:, c]) for c in range(nb)], 1), Q1.T, nb)
        assert np.max(np.abs(Q[:nb].T - Qo)) <= 1e-12 * np.max(np.abs(Qo))
        assert np.max(np.abs(info["A"][kf, 0] - As[0])) <= tol * np.max(np.abs(As[0]))
    pl.close()


def test_block_plan_single_vector_xmatvec():
    w = wl((20, 23), 3, 8, K=3)
    omega, V, sigma, _ = I.make_inputs(w)
    rng = np.random.default_rng(3)
    q = np.ascontiguousarray(rng.normal(size=(w.K, w.N)) + 1j * rng.normal(size=(w.K, w.N)))
    pl = plan_for(w, D.DYSON_FP64, block_size=2)
    u = np.zeros_like(q)
    D.dyson_xmatvec(pl.handle, w.K, omega, V, sigma, q, u)
    for kf in range(w.K):
        _, X = oracle_parts(w, omega[kf], V, sigma[kf])
        assert relerr(u[kf], X(q[kf])) <= 1e-10
    pl.close()
