"""Real frequency axis (i w_k -> w + i eta, the remark after Eq. 1) through the C ABI:
the same kernels with H_ii = w + i eta + mu - V_i - Sigma_i(w), against the oracle."""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I
from parity_util import OPEN, TOL_FP64, TOL_MIXED, oracle_parts, plan_for, relerr, stepwise_check, wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1102_3137_gb300 import build
    build.build()
    D.load()


def real_inputs(w):
    return I.make_inputs(w, axis="real")


@pytest.mark.parametrize("L", [(16, 16), (5, 4, 6)])
def test_real_axis_stencil(L):
    eta = 0.1
    w = wl(L, 1, 1, K=3)
    omega, V, sigma, q1 = real_inputs(w)
    pl = plan_for(w, eta=eta)
    rng = np.random.default_rng(3)
    x = rng.normal(size=(3, w.N)) + 1j * rng.normal(size=(3, w.N))
    y = np.zeros_like(x)
    D.dyson_apply_H(pl.handle, 3, omega, V, sigma, np.ascontiguousarray(x), y)
    for k in range(3):
        ref = O.apply_H(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], x[k], eta=eta)
        assert np.max(np.abs(y[k] - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", [D.DYSON_FP64, D.DYSON_MIXED])
def test_real_axis_subdomain_diag(precision):
    eta = 0.05
    w = wl((24, 20), 3, 4, K=3)
    omega, V, sigma, q1 = real_inputs(w)
    pl = plan_for(w, precision, eta=eta)
    dB = np.zeros((3, w.N), complex)
    D.dyson_subdomain_diag(pl.handle, 3, omega, V, sigma, dB)
    for k in range(3):
        z = O.dyson_diagonal_real(omega[k], eta, w.mu, V, sigma[k])
        subs = O.Subdomains(w.L, OPEN, w.t, z, w.p)
        mask = subs.diagB != 0
        assert relerr(dB[k][mask], subs.diagB[mask]) < 1e-12


@pytest.mark.parametrize("eta", [0.1, 0.02])
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_real_axis_terminated_is_exact(eta, precision, tol):
    """16x16, p = 2 (m = 16), k cap 24, frequencies across the band: exact diagonal."""
    w = wl((16, 16), 2, 24, K=6, seed=1)
    omega, V, sigma, q1 = real_inputs(w)
    pl = plan_for(w, precision, eta=eta)
    st = np.zeros(w.K, np.int32)
    out = pl.solve(omega, V, sigma, q1, status=st)
    assert np.all(st & D.DYSON_ST_TERMINATED)
    assert np.all((st & D.DYSON_ST_NO_CONVERGENCE) == 0)
    for k in range(w.K):
        ex = O.exact_diag(w.L, OPEN, w.t, O.dyson_diagonal_real(omega[k], eta, w.mu, V, sigma[k]))
        assert relerr(out[k], ex) <= tol
        assert np.all(out[k].imag < 0)          # retarded: spectral weight -Im G / pi > 0


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_real_axis_truncated_stepwise(precision, tol):
    eta = 0.1
    w = wl((40, 64), 4, 12, K=3, seed=17)
    omega, V, sigma, q1 = real_inputs(w)
    pl = plan_for(w, precision, eta=eta)
    out = pl.solve(omega, V, sigma, q1)
    info = pl.info(w.K)
    for k in range(w.K):
        subs, X = oracle_parts(w, omega[k], V, sigma[k], eta=eta)
        stepwise_check(w, pl, k, subs, X, q1, out[k], info, tol)


def test_real_axis_single_domain_is_exact():
    eta = 0.05
    w = wl((30, 20), 1, 4, K=3)
    omega, V, sigma, q1 = real_inputs(w)
    out = plan_for(w, eta=eta).solve(omega, V, sigma, q1)
    for k in range(3):
        ex = O.exact_diag(w.L, OPEN, w.t, O.dyson_diagonal_real(omega[k], eta, w.mu, V, sigma[k]))
        assert relerr(out[k], ex) <= 1e-12
