"""Helpers shared by the GPU parity tests: seeded workloads, the oracle's view
of one frequency, and the step-by-step Lanczos check (Eqs. 9-10)."""
import numpy as np

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I

TOL_FP64 = 1e-10
TOL_MIXED = 1e-6
OPEN = (False, False, False)
# Relative accuracy of an X-matvec of either GPU form: the FP64 form's interface
# solves stop at a relative residual of 1e-13; the mixed form refines in FP64 to it.
EPS_XMATVEC = 1e-13


def rounding_bound(name, k, tol):
    """Fixed bound for a direct GPU-vs-oracle comparison of a truncated (k << m) run at
    frequency k of a full-size workload: max(tol, amplification * EPS_XMATVEC), the
    amplification of X-matvec rounding into the rank-k diagonal measured on the oracle
    alone (tests/golden/make_rounding_spread.py: two exact FP64 forms of Eq. 8)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "rounding_spread.json")) as f:
        amp = json.load(f)[name][str(k)]["amplification"]
    return max(tol, amp * EPS_XMATVEC)


def wl(L, p, k, K=4, seed=11, b_max=0.5, trap=0.01, beta=10.0):
    return I.Workload("t", tuple(L), -1.0, 0.0, trap, b_max, beta, K, p, k, seed)


def relerr(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def plan_for(w, precision=D.DYSON_FP64, K=None, **kw):
    return D.Plan(w.L, w.t, w.mu, w.p, w.k, precision, max_freqs=K or w.K, **kw)


def oracle_parts(w, omega_k, V, sigma_k, eta=0.0):
    z = O.axis_diagonal(omega_k, w.mu, V, sigma_k, eta)
    subs = O.Subdomains(w.L, OPEN, w.t, z, w.p)
    full = O.FullLattice(w.L, OPEN, w.t, z)
    return subs, (lambda q: full.solve(q) - subs.solve(q))


def stepwise_check(w, pl, kf, subs, X, q1, out_k, info, tol):
    n = int(info["steps"][kf])
    Q = D.dyson_lanczos_basis(pl.handle, kf, n + 1, w.N)
    al = info["alpha"][kf, :n]
    be = info["beta"][kf, 1:n]
    Qk = Q[:n].T
    T = np.diag(al) + np.diag(be, 1) + np.diag(be, -1)
    q1n = q1 / np.sqrt(q1 @ q1)
    assert np.max(np.abs(Q[0] - q1n)) <= 1e-14 * np.max(np.abs(q1n))
    nrm = np.linalg.norm(Qk, axis=0)
    G = Qk.T @ Qk
    assert np.max(np.abs(G - np.eye(n)) / np.outer(nrm, nrm)) <= tol
    XQ = np.stack([X(Qk[:, j]) for j in range(n)], 1)
    R = XQ - Qk @ T
    R[:, n - 1] -= Q[n]                       # raw residual beta_{k+1} q_{k+1} of the last step
    scale = np.abs(XQ) + np.abs(Qk) @ np.abs(T)
    scale[:, n - 1] += np.abs(Q[n])
    assert np.max(np.abs(R)) <= tol * np.max(scale)
    ref = subs.diagB + np.einsum("ij,jk,ik->i", Qk, T, Qk)
    assert relerr(out_k, ref) <= tol
    return n
