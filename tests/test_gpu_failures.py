"""Failure detection on the GPU, with no GPU fault.

* Lanczos breakdown (Sec. 2.1: in the bilinear form a non-zero residual can
  have a vanishing "norm" sqrt(r^T r)).  A self-energy shift c, found on the
  CPU by Newton's method on dense algebra, makes (r, r)_C vanish at the second
  step on a small lattice; the GPU must stop there with DYSON_ST_BREAKDOWN and
  keep the partial sum (Eq. 9 over the two steps taken), as the oracle does.
* The bounded wait of the copy rings: run on an mbarrier nothing arrives on,
  it gives up after its limit and the kernel returns; the device stays usable.
"""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I

from parity_util import OPEN, TOL_FP64, TOL_MIXED, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1102_3137_gb300 import build
    build.build()
    D.load()


def _rr_at_step(L, p, omega0, V, sigma0, q1, c, step):
    """(r^T r / ||r||^2, ||r|| / ||X q||) of the Lanczos residual at `step` (0-based) on the
    dense X = H^-1 - blkdiag(B^-1, 0) of the lattice with Sigma shifted by c."""
    z = O.dyson_diagonal(omega0, 0.0, V, sigma0 + c)
    H = O.dense_H(L, OPEN, -1.0, z)
    _, iface = O.dd_sites(L, p)
    keep = np.setdiff1d(np.arange(H.shape[0]), np.concatenate(iface))
    X = np.linalg.inv(H)
    X[np.ix_(keep, keep)] -= np.linalg.inv(H[np.ix_(keep, keep)])
    Q = [q1 / np.sqrt(q1 @ q1)]
    beta = 0.0
    for j in range(step + 1):
        u = X @ Q[j]
        r = u - (Q[j] @ u) * Q[j] - (beta * Q[j - 1] if j else 0)
        for _ in range(2):
            Qa = np.stack(Q, 1)
            r = r - Qa @ (Qa.T @ r)
        if j == step:
            return (r @ r) / np.vdot(r, r).real, np.linalg.norm(r) / np.linalg.norm(u)
        beta = np.sqrt(r @ r)
        Q.append(r / beta)


def _breakdown_shift(L, p, omega0, V, sigma0, q1, step):
    """Complex shift c of Sigma with r^T r = 0 at `step`: Newton on an analytic function of c."""
    c = 0j
    for _ in range(60):
        f = _rr_at_step(L, p, omega0, V, sigma0, q1, c, step)[0]
        if abs(f) < 1e-16:
            break
        h = 1e-7
        fp = (_rr_at_step(L, p, omega0, V, sigma0, q1, c + h, step)[0] - f) / h
        c -= f / fp
    return c


@pytest.mark.parametrize("precision", [D.DYSON_FP64, D.DYSON_MIXED])
def test_breakdown_reported_with_partial_sum(precision):
    import torch
    L, p, step = (6, 7), 2, 1
    w = I.Workload("t", L, -1.0, 0.0, 0.01, 0.5, 10.0, 1, p, 8, 5)
    omega, V, sigma, q1 = I.make_inputs(w)
    c = _breakdown_shift(L, p, omega[0], V, sigma[0], q1, step)
    f, ratio = _rr_at_step(L, p, omega[0], V, sigma[0], q1, c, step)
    assert abs(f) < 1e-15 and ratio > 0.5          # (r, r)_C = 0 with r well away from 0
    sig = np.ascontiguousarray(sigma + c)
    z = O.dyson_diagonal(omega[0], 0.0, V, sig[0])
    assert np.min(z.imag) > 0.1                     # the factorizations stay pivot-free
    ref, info = O.lowrank_diag(w.L, OPEN, w.t, w.mu, V, sig[0], omega[0], q1, p, w.k,
                               return_info=True)
    assert info["status"] == O.STATUS_BREAKDOWN and info["steps"] == step + 1
    pl = D.Plan(w.L, w.t, w.mu, p, w.k, precision, max_freqs=1, krylov_tol=1e-15 if precision == D.DYSON_FP64 else 0.0)
    dev = torch.device("cuda:0")
    out = torch.zeros((1, w.N), dtype=torch.complex128, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    D.dyson_solve(pl.handle, 1, t(omega[:1]), t(V), t(sig[:1]), t(q1), out, st)
    torch.cuda.synchronize()
    gi = pl.info(1)
    assert int(st.item()) & D.DYSON_ST_BREAKDOWN
    assert int(gi["steps"][0]) == step + 1
    assert relerr(out.cpu().numpy()[0], ref) <= (TOL_FP64 if precision == D.DYSON_FP64 else TOL_MIXED)
    pl.close()


def test_bounded_wait_gives_up_and_returns():
    import torch
    timed_out, waited = D.dyson_wait_selftest(0.002)
    assert timed_out and 0.002 <= waited < 1.0
    # the context is still usable: a small solve afterwards is correct
    w = I.Workload("t", (16, 16), -1.0, 0.0, 0.01, 0.5, 10.0, 1, 2, 24, 1)
    omega, V, sigma, q1 = I.make_inputs(w)
    pl = D.Plan(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=1)
    got = pl.solve(omega, V, sigma, q1)
    ref = O.lowrank_diag(w.L, OPEN, w.t, w.mu, V, sigma[0], omega[0], q1, w.p, w.k)
    assert relerr(got[0], ref) <= TOL_FP64
    pl.close()
    torch.cuda.synchronize()
