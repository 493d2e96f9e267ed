"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself:
a library dense inverse, a closed form, an exact identity of Sec. 2.2-2.3,
the paper's worked example (tests/golden/fig1_5x5.json), or an invariant of
the Lanczos recurrence.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_z(N, rng, omega=0.4, spread=3.0):
    """An inhomogeneous Dyson diagonal with Im > 0 (random a_i, b_i, a trap-like real part)."""
    return (rng.uniform(-spread, spread, N) + 1j * (omega + rng.uniform(0, 0.5, N)))


# --------------------------------------------------------------------------- dense LU


def test_hand_lu_inverse_matches_library():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(40, 40)) + 1j * rng.normal(size=(40, 40))
    G = O.lu_inverse(A)
    ref = np.linalg.inv(A)
    assert np.max(np.abs(G - ref)) / np.max(np.abs(ref)) < 1e-12


def test_hand_lu_pivots_on_zero_leading_entry():
    A = np.array([[0, 1, 2], [1, 0, 3], [4, -3, 8]], dtype=complex)
    assert np.allclose(O.lu_inverse(A) @ A, np.eye(3), atol=1e-13)


# ------------------------------------------------------------------ exact recursion


@pytest.mark.parametrize("L,periodic", [
    ((7, 6), (False, False, False)),
    ((5, 6), (False, True, False)),
    ((4, 3, 3), (False, False, False)),
    ((3, 4, 3), (False, True, True)),
    ((1, 9), (False, False, False)),
    ((9, 1), (False, False, False)),
])
def test_exact_recursion_matches_dense_inverse(L, periodic):
    rng = np.random.default_rng(1)
    N = O.site_count(L)
    z = rand_z(N, rng)
    ref = np.diag(np.linalg.inv(O.dense_H(L, periodic, -1.0, z)))
    got = O.exact_diag(L, periodic, -1.0, z)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12
    lu = O.dense_diag_inverse(L, periodic, -1.0, z)
    assert np.max(np.abs(lu - ref) / np.abs(ref)) < 1e-12


def _open_closed_form(L, t, z0):
    """G_ii = sum_q prod_d (2/(L_d+1)) sin^2(q_d x_d) / (z0 + 2t sum_d cos q_d), x_d 1-based."""
    ks = [np.pi * np.arange(1, n + 1) / (n + 1) for n in L]
    xs = [np.arange(1, n + 1) for n in L]
    # mode weights per axis: w_d[x, n] = 2/(L+1) sin^2(q_n x)
    w = [2.0 / (n + 1) * np.sin(np.outer(x, k)) ** 2 for n, x, k in zip(L, xs, ks)]
    out = np.zeros(tuple(reversed(L)), dtype=complex)
    if len(L) == 2:
        E = 2 * t * (np.cos(ks[0])[:, None] + np.cos(ks[1])[None, :])        # [nx, ny]
        R = 1.0 / (z0 + E)
        for y in range(L[1]):
            for x in range(L[0]):
                out[y, x] = np.sum(np.outer(w[0][x], w[1][y]) * R)
    else:
        E = 2 * t * (np.cos(ks[0])[:, None, None] + np.cos(ks[1])[None, :, None]
                     + np.cos(ks[2])[None, None, :])
        R = 1.0 / (z0 + E)
        for zc in range(L[2]):
            for y in range(L[1]):
                for x in range(L[0]):
                    out[zc, y, x] = np.einsum("a,b,c,abc->", w[0][x], w[1][y], w[2][zc], R)
    return out.ravel()


@pytest.mark.parametrize("L", [(7, 5), (4, 3, 5)])
def test_exact_recursion_open_closed_form(L):
    z0 = 0.3 + 0.25j
    got = O.exact_diag(L, (False, False, False), -1.0, np.full(O.site_count(L), z0))
    ref = _open_closed_form(L, -1.0, z0)
    assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-12


def test_periodic_closed_form_dense():
    """Homogeneous periodic lattice: G_ii = (1/N) sum_q 1/(i w + mu - Sigma - eps_q)."""
    L = (6, 5)
    w, mu, sig = math.pi / 10, 0.2, 0.4 - 0.3j
    z0 = 1j * w + mu - sig
    t = -1.0
    qs = [2 * np.pi * np.arange(n) / n for n in L]
    eps = -2 * t * (np.cos(qs[0])[:, None] + np.cos(qs[1])[None, :])
    ref = np.mean(1.0 / (z0 - eps))
    got = O.dense_diag_inverse(L, (True, True, False), t, np.full(30, z0))
    assert np.max(np.abs(got - ref) / abs(ref)) < 1e-12


def test_transverse_periodic_closed_form_recursion():
    """Open along x, periodic along y: sine modes in x times plane waves in y."""
    Lx, Ly = 6, 5
    z0 = -0.2 + 0.3j
    t = -1.0
    kx = np.pi * np.arange(1, Lx + 1) / (Lx + 1)
    ky = 2 * np.pi * np.arange(Ly) / Ly
    R = 1.0 / (z0 + 2 * t * (np.cos(kx)[:, None] + np.cos(ky)[None, :]))   # [nx, ny]
    ref = np.array([np.sum(2.0 / (Lx + 1) * np.sin(kx * (x + 1)) ** 2 * R.mean(1))
                    for x in range(Lx)])
    got = O.exact_diag((Lx, Ly), (False, True, False), t, np.full(Lx * Ly, z0)).reshape(Ly, Lx)
    for y in range(Ly):
        assert np.max(np.abs(got[y] - ref) / np.abs(ref)) < 1e-12


def test_zero_hopping_gives_local_inverse():
    rng = np.random.default_rng(2)
    z = rand_z(48, rng)
    got = O.exact_diag((8, 6), (False, False, False), 0.0, z)
    assert np.max(np.abs(got - 1 / z) / np.abs(1 / z)) < 1e-15


def test_imaginary_part_negative_and_symmetric():
    rng = np.random.default_rng(3)
    L = (6, 6)
    z = rand_z(36, rng)
    G = O.lu_inverse(O.dense_H(L, (False,) * 3, -1.0, z))
    assert np.all(np.diag(G).imag < 0)
    assert np.max(np.abs(G - G.T)) < 1e-13 * np.max(np.abs(G))
    assert np.all(O.exact_diag(L, (False,) * 3, -1.0, z).imag < 0)


def test_large_frequency_limit():
    L = (5, 4)
    w = 1e4
    omega, V, sigma, q1 = I.homogeneous_inputs(L, [w], 0.3 - 0.1j)
    z = O.dyson_diagonal(w, 0.0, V, sigma[0])
    G = O.exact_diag(L, (False,) * 3, -1.0, z)
    assert np.max(np.abs(G * 1j * w - 1)) < 1e-3


def test_stencil_matches_dense():
    rng = np.random.default_rng(4)
    L = (5, 4, 3)
    N = 60
    V = rng.uniform(0, 2, N)
    sig = rng.normal(size=N) + 1j * rng.normal(size=N)
    x = rng.normal(size=N) + 1j * rng.normal(size=N)
    per = (True, False, True)
    y = O.apply_H(L, per, -1.0, 0.1, V, sig, 0.7, x)
    H = O.dense_H(L, per, -1.0, O.dyson_diagonal(0.7, 0.1, V, sig))
    assert np.max(np.abs(y - H @ x)) < 1e-13


# ------------------------------------------------------------------ decomposition


@pytest.mark.parametrize("L,p,heights,m", [
    ((16, 16), 2, [8, 7], 16),
    ((128, 128), 4, [32, 31, 31, 31], 384),
    ((32, 32, 32), 8, [4] + [3] * 7, 7168),
    ((512, 512), 16, [32] + [31] * 15, 7680),
    ((64, 64), 4, [16, 15, 15, 15], 192),
])
def test_partition_sizes(L, p, heights, m):
    starts, h, layers = O.dd_partition(L, p)
    assert h == heights
    A = L[0] * (L[1] if len(L) == 3 else 1)
    assert len(layers) * A == m
    sub, iface = O.dd_sites(L, p)
    allidx = np.concatenate([s.ravel() for s in sub] + list(iface))
    assert np.array_equal(np.sort(allidx), np.arange(O.site_count(L)))


def _dd_dense(L, p, z, t=-1.0):
    sub, iface = O.dd_sites(L, p)
    order = np.concatenate([s.ravel() for s in sub] + list(iface))
    H = O.dense_H(L, (False,) * 3, t, z)[np.ix_(order, order)]
    nb = sum(s.size for s in sub)
    return H, order, nb, sub


@pytest.mark.parametrize("L,p", [((6, 7), 2), ((5, 9), 3), ((3, 3, 5), 2)])
def test_block_inverse_identity_and_rank(L, p):
    """Eq. 5 and Eq. 6: H^-1 = blkdiag(B^-1,0) + [B^-1 E; -I] S^-1 [E^T B^-1, -I]; rank X = m."""
    rng = np.random.default_rng(5)
    z = rand_z(O.site_count(L), rng)
    H, order, nb, sub = _dd_dense(L, p, z)
    B, E, C = H[:nb, :nb], H[:nb, nb:], H[nb:, nb:]
    # B has no coupling between different subdomains (Eq. 3)
    off = 0
    for s in sub:
        n = s.size
        assert np.all(B[off:off + n, :off] == 0) and np.all(B[off:off + n, off + n:] == 0)
        off += n
    Binv = np.linalg.inv(B)
    S = C - E.T @ Binv @ E                                        # Eq. 4
    Y = np.vstack([Binv @ E, -np.eye(C.shape[0])])
    Hinv = np.linalg.inv(H)
    base = np.zeros_like(H)
    base[:nb, :nb] = Binv
    X = Hinv - base                                                # Eq. 6
    assert np.max(np.abs(X - Y @ np.linalg.inv(S) @ Y.T)) < 1e-12 * np.max(np.abs(Hinv))
    sv = np.linalg.svd(X, compute_uv=False)
    m = C.shape[0]
    assert np.sum(sv > 1e-10 * sv[0]) == m
    assert np.max(np.abs(X - X.T)) < 1e-13


def test_subdomain_factors_match_dense_blocks():
    rng = np.random.default_rng(6)
    L, p = (7, 11), 3
    z = rand_z(77, rng)
    subs = O.Subdomains(L, (False,) * 3, -1.0, z, p)
    H = O.dense_H(L, (False,) * 3, -1.0, z)
    iface = np.concatenate(subs.iface)
    mask = np.ones(77, bool)
    mask[iface] = False
    keep = np.where(mask)[0]
    Binv = np.zeros((77, 77), complex)
    Binv[np.ix_(keep, keep)] = np.linalg.inv(H[np.ix_(keep, keep)])
    assert np.max(np.abs(subs.diagB - np.diag(Binv))) < 1e-13
    q = rng.normal(size=77) + 1j * rng.normal(size=77)
    assert np.max(np.abs(subs.solve(q) - Binv @ q)) < 1e-12
    full = O.FullLattice(L, (False,) * 3, -1.0, z)
    assert np.max(np.abs(full.solve(q) - np.linalg.solve(H, q))) < 1e-12


# ------------------------------------------------------------------ Lanczos on X


def _dense_X(H, interface):
    n = H.shape[0]
    keep = np.setdiff1d(np.arange(n), interface)
    base = np.zeros_like(H)
    base[np.ix_(keep, keep)] = np.linalg.inv(H[np.ix_(keep, keep)])
    return np.linalg.inv(H) - base, base


def test_fig1_worked_example():
    """5x5 grid, four 2x2 subdomains, cross-shaped interface of 9 points (Fig. 1)."""
    gold = json.load(open(os.path.join(GOLDEN, "fig1_5x5.json")))
    Lx, Ly = gold["L"]
    rng = np.random.default_rng(7)
    z = rand_z(Lx * Ly, rng)
    H = O.dense_H((Lx, Ly), (False,) * 3, -1.0, z)
    interface = np.array(sorted({x + Lx * 2 for x in range(Lx)} | {2 + Lx * y for y in range(Ly)}))
    assert interface.size == gold["interface_last_label"] - gold["interface_first_label"] + 1
    keep = np.setdiff1d(np.arange(Lx * Ly), interface)
    # the kept sites split into four decoupled 2x2 blocks
    Hk = H[np.ix_(keep, keep)]
    n_comp = 0
    seen = set()
    for a in range(keep.size):
        if a in seen:
            continue
        n_comp += 1
        stack = [a]
        while stack:
            c = stack.pop()
            if c in seen:
                continue
            seen.add(c)
            stack += [d for d in range(keep.size) if d != c and Hk[c, d] != 0]
    assert n_comp == gold["subdomains"]
    X, base = _dense_X(H, interface)
    sv = np.linalg.svd(X, compute_uv=False)
    assert np.sum(sv > 1e-10 * sv[0]) == gold["m"]
    exact = np.diag(np.linalg.inv(H))
    # a start vector inside range(X): the Krylov space closes after m steps
    q1 = X @ rng.normal(size=25)
    acc, al, be, Q, st = O.cs_lanczos(lambda q: X @ q, q1, 25)
    assert st == O.STATUS_TERMINATED and len(al) == gold["lanczos_steps"]
    assert np.max(np.abs(np.diag(base) + acc - exact) / np.abs(exact)) < 1e-11
    # a generic real start vector needs at most one extra step
    acc, al, be, Q, st = O.cs_lanczos(lambda q: X @ q, rng.uniform(-1, 1, 25), 25)
    assert st == O.STATUS_TERMINATED and len(al) <= gold["lanczos_steps"] + 1
    assert np.max(np.abs(np.diag(base) + acc - exact) / np.abs(exact)) < 1e-11


def test_lanczos_invariants_truncated():
    """Q^T Q = I and Q^T X Q = T in the bilinear form; the three-vector sum is diag(Q T Q^T)."""
    rng = np.random.default_rng(8)
    L, p = (10, 12), 3
    z = rand_z(120, rng)
    H, order, nb, sub = _dd_dense(L, p, z)
    X, _ = _dense_X(H, np.arange(nb, 120))
    k = 8
    acc, al, be, Q, st = O.cs_lanczos(lambda q: X @ q, rng.uniform(-1, 1, 120), k)
    assert Q.shape[1] == k and st == O.STATUS_OK
    T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) < 1e-10
    assert np.max(np.abs(Q.T @ X @ Q - T)) < 1e-10 * np.max(np.abs(T))
    assert np.max(np.abs(np.diag(Q @ T @ Q.T) - acc)) < 1e-13 * np.max(np.abs(acc))


def test_lanczos_sqrt_branch_invariance():
    rng = np.random.default_rng(9)
    M = rng.normal(size=(30, 30)) + 1j * rng.normal(size=(30, 30))
    X = M + M.T
    q1 = rng.uniform(-1, 1, 30)
    a1 = O.cs_lanczos(lambda q: X @ q, q1, 10)[0]
    a2 = O.cs_lanczos(lambda q: X @ q, q1, 10, branch=-1)[0]
    assert np.max(np.abs(a1 - a2)) < 1e-11 * np.max(np.abs(a1))


def test_structured_xmatvec_matches_dense_X():
    rng = np.random.default_rng(10)
    L, p = (9, 10), 3
    omega, V, sigma, q1 = I.make_inputs(I.Workload("t", L, -1.0, 0.0, 0.01, 0.5, 10.0, 2, p, 4, 3))
    z = O.dyson_diagonal(omega[0], 0.0, V, sigma[0])
    H = O.dense_H(L, (False,) * 3, -1.0, z)
    _, iface = O.dd_sites(L, p)
    X, _ = _dense_X(H, np.concatenate(iface))
    q = rng.normal(size=90) + 1j * rng.normal(size=90)
    u = O.xmatvec(L, (False,) * 3, -1.0, 0.0, V, sigma[0], omega[0], p, q)
    assert np.max(np.abs(u - X @ q)) < 1e-12 * np.max(np.abs(X @ q))


def test_lowrank_structured_equals_brute_force_truncated():
    """Brute force: Lanczos on the explicitly formed dense X gives the same truncated diagonal."""
    w = I.Workload("t", (12, 12), -1.0, 0.0, 0.01, 0.5, 10.0, 3, 2, 5, 11)
    omega, V, sigma, q1 = I.make_inputs(w)
    for k in range(w.K):
        res, info = O.lowrank_diag(w.L, (False,) * 3, w.t, w.mu, V, sigma[k], omega[k], q1,
                                   w.p, w.k, return_info=True)
        z = O.dyson_diagonal(omega[k], w.mu, V, sigma[k])
        H = O.dense_H(w.L, (False,) * 3, w.t, z)
        _, iface = O.dd_sites(w.L, w.p)
        X, base = _dense_X(H, np.concatenate(iface))
        acc, al, be, Q, st = O.cs_lanczos(lambda q: X @ q, q1, w.k)
        assert np.max(np.abs(al - info["alphas"])) < 1e-11 * np.max(np.abs(al))
        assert np.max(np.abs(np.diag(base) + acc - res) / np.abs(res)) < 1e-11


def test_lowrank_exact_after_termination():
    """k >= m+1 on an inhomogeneous lattice: the correction is exact (Eq. 10, Eq. 9)."""
    w = I.Workload("t", (16, 16), -1.0, 0.0, 0.01, 0.5, 10.0, 2, 2, 24, 1)
    omega, V, sigma, q1 = I.make_inputs(w)
    for k in range(w.K):
        res, info = O.lowrank_diag(w.L, (False,) * 3, w.t, w.mu, V, sigma[k], omega[k], q1,
                                   w.p, w.k, return_info=True)
        z = O.dyson_diagonal(omega[k], w.mu, V, sigma[k])
        ex = O.exact_diag(w.L, (False,) * 3, w.t, z)
        assert info["status"] == O.STATUS_TERMINATED and info["steps"] <= 16 + 3
        assert np.max(np.abs(res - ex) / np.abs(ex)) < 1e-10
        # invariance in k once terminated
        res2 = O.lowrank_diag(w.L, (False,) * 3, w.t, w.mu, V, sigma[k], omega[k], q1, w.p, 40)
        assert np.max(np.abs(res2 - res) / np.abs(res)) < 1e-13


def test_lowrank_single_domain_is_exact():
    w = I.Workload("t", (8, 9), -1.0, 0.0, 0.01, 0.5, 10.0, 2, 1, 4, 5)
    omega, V, sigma, q1 = I.make_inputs(w)
    z = O.dyson_diagonal(omega[0], 0.0, V, sigma[0])
    a = O.lowrank_diag(w.L, (False,) * 3, -1.0, 0.0, V, sigma[0], omega[0], q1, 1, 4)
    assert np.max(np.abs(a - O.exact_diag(w.L, (False,) * 3, -1.0, z))) == 0.0


def test_lowrank_3d_exact_after_termination():
    w = I.Workload("t", (4, 4, 7), -1.0, 0.0, 0.005, 1.0, 40.0, 1, 2, 40, 3)
    omega, V, sigma, q1 = I.make_inputs(w)
    res, info = O.lowrank_diag(w.L, (False,) * 3, -1.0, 0.0, V, sigma[0], omega[0], q1, 2, 40,
                               return_info=True)
    z = O.dyson_diagonal(omega[0], 0.0, V, sigma[0])
    ex = np.diag(np.linalg.inv(O.dense_H(w.L, (False,) * 3, -1.0, z)))
    assert info["status"] == O.STATUS_TERMINATED and info["steps"] <= 16 + 3
    assert np.max(np.abs(res - ex) / np.abs(ex)) < 1e-10


def test_inputs_reproducible_and_physical():
    w = I.WORKLOADS["square16_K8_p2_k16"]
    a = I.make_inputs(w)
    b = I.make_inputs(w)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    omega, V, sigma, q1 = a
    assert omega.shape == (8,) and np.allclose(omega, (2 * np.arange(8) + 1) * np.pi / 10)
    assert V[0] == pytest.approx(0.01 * 2 * 7.5 ** 2)
    z = 1j * omega[:, None] - V[None] - sigma
    assert np.all(z.imag > 0)


# ------------------------------------------------------------------ real frequency axis

def test_real_axis_closed_form_dense():
    """Real axis (i w -> w + i eta): homogeneous periodic lattice,
    G_ii = (1/N) sum_q 1/(w + i eta + mu - Sigma - eps_q)."""
    L = (6, 5)
    w, eta, mu, sig = 0.7, 0.05, 0.2, 0.4 - 0.3j
    z = O.dyson_diagonal_real(w, eta, mu, np.zeros(30), np.full(30, sig))
    t = -1.0
    qs = [2 * np.pi * np.arange(n) / n for n in L]
    eps = -2 * t * (np.cos(qs[0])[:, None] + np.cos(qs[1])[None, :])
    ref = np.mean(1.0 / (w + 1j * eta + mu - sig - eps))
    got = O.dense_diag_inverse(L, (True, True, False), t, z)
    assert np.max(np.abs(got - ref) / abs(ref)) < 1e-12


def test_real_axis_spectral_weight():
    """Retarded G on the real axis: A_i(w) = -Im G_ii(w) / pi >= 0 and, for an open
    lattice with Sigma = 0, integrates to 1 up to the Lorentzian tails outside the
    window: for a level e the weight in [-W, W] is (atan((W-e)/eta) + atan((W+e)/eta)) / pi."""
    L = (5, 4)
    eta, W = 0.05, 30.0
    ws = np.linspace(-W, W, 20001)
    N = O.site_count(L)
    A = np.zeros((ws.size, N))
    for n, w in enumerate(ws):
        z = O.dyson_diagonal_real(w, eta, 0.0, np.zeros(N), np.zeros(N))
        A[n] = -O.exact_diag(L, (False, False, False), -1.0, z).imag / np.pi
    assert A.min() >= 0.0
    weight = np.trapezoid(A, ws, axis=0)
    # eigenvalues of the open-lattice hopping matrix: every site sees all levels
    ks = [np.pi * np.arange(1, n + 1) / (n + 1) for n in L]
    lv = (-2.0 * (np.cos(ks[0])[:, None] + np.cos(ks[1])[None, :])).ravel()
    tails = (np.arctan((W - lv) / eta) + np.arctan((W + lv) / eta)) / np.pi
    lo, hi = tails.min(), tails.max()
    assert np.all(weight > lo - 1e-4) and np.all(weight < hi + 1e-4)


def test_real_axis_lowrank_terminated_is_exact():
    """The low-rank method on the real axis: with k past closure it returns the exact diagonal."""
    w = I.Workload("r", (10, 9), -1.0, 0.0, 0.01, 0.5, 10.0, 2, 2, 12, 5)
    omega, V, sigma, q1 = I.make_inputs(w, axis="real")
    for k in range(2):
        z = O.dyson_diagonal_real(omega[k], 0.1, w.mu, V, sigma[k])
        ex = O.exact_diag(w.L, (False, False, False), w.t, z)
        lr = O.lowrank_diag(w.L, (False, False, False), w.t, w.mu, V, sigma[k], omega[k], q1,
                            w.p, w.k, eta=0.1)
        assert np.max(np.abs(lr - ex) / np.abs(ex)) < 1e-10


# --------------------------------------------------------------------------- block Lanczos


def _homogeneous_cube():
    """3 x 3 x 7 open lattice, constant Sigma, no trap, p = 2: the 3 x 3 interface
    plane has degenerate eigenvalues of X (the x <-> y swap and the accidental
    degeneracy of the plane modes cos(pi n1/4) + cos(pi n2/4) = 0 for
    (1,3), (3,1), (2,2) give an eigenvalue of multiplicity 3)."""
    L = (3, 3, 7)
    N = O.site_count(L)
    V = np.zeros(N)
    sigma = np.full(N, 0.3 + 0.2j)
    return L, N, V, sigma, math.pi / 10


def _dense_X_and_inverse(L, per, t, z, p):
    N = z.shape[0]
    Hinv = np.linalg.inv(O.dense_H(L, per, t, z))
    subs = O.Subdomains(L, per, t, z, p)
    return Hinv - np.stack([subs.solve(e) for e in np.eye(N)], 1), Hinv


def test_block_lanczos_exact_on_degenerate_spectrum():
    """A single start vector spans one direction per eigenspace of X, so on a
    degenerate spectrum the scalar method terminates early and misses part of
    diag(X); a block of size >= the largest multiplicity reaches the exact
    diagonal (dense library inverse) at any start block."""
    L, N, V, sigma, w = _homogeneous_cube()
    per = [False] * 3
    z = O.dyson_diagonal(w, 0.0, V, sigma)
    X, Hinv = _dense_X_and_inverse(L, per, -1.0, z, 2)
    ev = np.linalg.eigvals(X)
    ev = ev[np.abs(ev) > 1e-10]
    assert len(ev) == 9
    mult = max(int(np.sum(np.abs(ev - e) < 1e-8)) for e in ev)
    assert mult == 3
    exact = np.diag(Hinv)
    rng = np.random.default_rng(11)
    Q1 = rng.uniform(-1, 1, (N, 3))
    r1, info1 = O.lowrank_diag(L, per, -1.0, 0.0, V, sigma, w, Q1[:, 0], 2, 12, return_info=True)
    assert info1["status"] == O.STATUS_TERMINATED and info1["steps"] < 9
    assert np.max(np.abs(r1 - exact)) / np.max(np.abs(exact)) > 1e-2
    for seed in (11, 12):
        Q1 = np.random.default_rng(seed).uniform(-1, 1, (N, 3))
        rb, info = O.lowrank_diag_block(L, per, -1.0, 0.0, V, sigma, w, Q1, 2, 12, return_info=True)
        assert np.max(np.abs(rb - exact)) / np.max(np.abs(exact)) < 1e-11


def test_block_lanczos_recurrence_and_orthogonality():
    """X Q_k = Q_k T_k + (last block residual), Q_k^T Q_k = I, A_j = A_j^T,
    and diag(Q T Q^T) from the recurrence equals the product formed densely."""
    L, per, p, nb, k = (6, 11), [False, False], 3, 2, 8
    N = 66
    rng = np.random.default_rng(5)
    V = rng.uniform(0, 0.5, N)
    sigma = rng.uniform(0, 1, N) + 1j * rng.uniform(0.1, 1, N)
    w, mu = math.pi / 10, 0.2
    Q1 = rng.uniform(-1, 1, (N, nb))
    res, info = O.lowrank_diag_block(L, per, -1.0, mu, V, sigma, w, Q1, p, k, return_info=True)
    assert info["status"] == O.STATUS_OK and info["steps"] == k // nb
    z = O.dyson_diagonal(w, mu, V, sigma)
    X, _ = _dense_X_and_inverse(L, per, -1.0, z, p)
    Q, A, B = info["Q"], info["A"], info["B"]
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) < 1e-12
    T = np.zeros((k, k), dtype=complex)
    for j in range(k // nb):
        s = slice(nb * j, nb * j + nb)
        T[s, s] = A[j]
        assert np.max(np.abs(A[j] - A[j].T)) < 1e-12 * np.max(np.abs(A[j]))
        if j > 0:
            sp = slice(nb * (j - 1), nb * j)
            T[s, sp] = B[j]
            T[sp, s] = B[j].T
            assert np.max(np.abs(np.tril(B[j], -1))) == 0.0
    R = X @ Q - Q @ T
    assert np.max(np.abs(R[:, :k - nb])) < 1e-12 * np.max(np.abs(X))
    assert np.max(np.abs(np.diag(Q @ T @ Q.T) + info["diagB"] - res)) < 1e-12


def test_block_lanczos_depends_only_on_start_span():
    """Truncated block runs depend on the start block only through its span:
    Q1 -> Q1 M (M invertible) leaves every block Krylov space, hence the
    rank-k result, unchanged."""
    L, per, p = (6, 11), [False, False], 3
    N = 66
    rng = np.random.default_rng(7)
    V = rng.uniform(0, 0.5, N)
    sigma = rng.uniform(0, 1, N) + 1j * rng.uniform(0.1, 1, N)
    Q1 = rng.uniform(-1, 1, (N, 2))
    M = np.array([[0.7, -1.3], [0.4, 0.9]])
    for k in (4, 8):
        r1 = O.lowrank_diag_block(L, per, -1.0, 0.0, V, sigma, math.pi / 10, Q1, p, k)
        r2 = O.lowrank_diag_block(L, per, -1.0, 0.0, V, sigma, math.pi / 10, Q1 @ M, p, k)
        assert np.max(np.abs(r1 - r2)) / np.max(np.abs(r1)) < 1e-11


def test_block_of_one_is_the_scalar_recurrence():
    L, per, p, N = (6, 11), [False, False], 3, 66
    rng = np.random.default_rng(8)
    V = rng.uniform(0, 0.5, N)
    sigma = rng.uniform(0, 1, N) + 1j * rng.uniform(0.1, 1, N)
    q1 = rng.uniform(-1, 1, N)
    r1 = O.lowrank_diag(L, per, -1.0, 0.0, V, sigma, math.pi / 10, q1, p, 7)
    r2 = O.lowrank_diag_block(L, per, -1.0, 0.0, V, sigma, math.pi / 10, q1[:, None], p, 7)
    assert np.max(np.abs(r1 - r2)) / np.max(np.abs(r1)) < 1e-12


# --------------------------------------------------------------------------- recursive decomposition


def test_recursive_decomposition_exact_past_closure():
    """Sec. 2.3 end: the method applied recursively, cuts alternating between the
    axes, three levels deep on a 12 x 10 lattice; with the rank cap past every
    level's closure it reproduces the dense inverse's diagonal (library inverse),
    whichever axis is cut first."""
    rng = np.random.default_rng(3)
    L, N = (12, 10), 120
    z = rng.uniform(-2, 2, N) + 1j * rng.uniform(0.2, 0.8, N)
    q1 = rng.uniform(-1, 1, N)
    exact = np.diag(np.linalg.inv(O.dense_H(L, (False, False), -1.0, z)))
    for cut in ("x", "y"):
        r = O.recursive_diag(L, -1.0, z, q1, 200, min_sites=20, first_cut=cut)
        assert np.max(np.abs(r - exact)) / np.max(np.abs(exact)) < 1e-11
    # truncated levels are an approximation, not the exact diagonal
    r = O.recursive_diag(L, -1.0, z, q1, 6, min_sites=20)
    assert np.max(np.abs(r - exact)) / np.max(np.abs(exact)) > 1e-3


def test_recursive_one_level_is_the_two_strip_method():
    """One level of the recursion (halves inverted directly) cut along y at the
    middle line is the low-rank method with p = 2 strips, at any rank cap: the
    same X and start vector, reached through dense solves instead of the slice
    recursion and the full-lattice block LU."""
    rng = np.random.default_rng(4)
    L, N = (12, 11), 132
    V = rng.uniform(0, 0.5, N)
    sigma = rng.uniform(-1, 1, N) + 1j * rng.uniform(0.1, 0.6, N)
    w = math.pi / 10
    z = O.dyson_diagonal(w, 0.0, V, sigma)
    q1 = rng.uniform(-1, 1, N)
    for k in (4, 12, 20):
        a = O.recursive_diag(L, -1.0, z, q1, k, min_sites=60, first_cut="y")
        b = O.lowrank_diag(L, (False, False, False), -1.0, 0.0, V, sigma, w, q1, 2, k)
        assert np.max(np.abs(a - b)) / np.max(np.abs(b)) < 1e-11


def test_block_lanczos_partial_deflation_keeps_exactness():
    """4 x 5 lattice, p = 2: X has rank m = 4.  With a block of 3 the third block
    holds the one remaining direction of range(X): two of its columns deflate to
    zero, the block keeps its width, and the diagonal is already exact (dense
    library inverse); one more step finds the whole next block deflated
    (terminated)."""
    rng = np.random.default_rng(9)
    L, N = (4, 5), 20
    V = rng.uniform(0, 0.5, N)
    sigma = rng.uniform(-1, 1, N) + 1j * rng.uniform(0.1, 0.6, N)
    w = math.pi / 10
    exact = np.diag(np.linalg.inv(O.dense_H(L, (False, False), -1.0, O.dyson_diagonal(w, 0.0, V, sigma))))
    Q1 = rng.uniform(-1, 1, (N, 3))
    r, info = O.lowrank_diag_block(L, (False, False, False), -1.0, 0.0, V, sigma, w, Q1, 2, 9,
                                   return_info=True)
    nrm = np.linalg.norm(info["Q"], axis=0)
    assert info["steps"] == 3 and int((nrm == 0).sum()) == 2
    kept = info["Q"][:, nrm > 0]
    assert np.max(np.abs(kept.T @ kept - np.eye(kept.shape[1]))) < 1e-12
    assert np.max(np.abs(r - exact)) / np.max(np.abs(exact)) < 1e-12
    r2, info2 = O.lowrank_diag_block(L, (False, False, False), -1.0, 0.0, V, sigma, w, Q1, 2, 12,
                                     return_info=True)
    assert info2["status"] == O.STATUS_TERMINATED and info2["steps"] == 3
    assert np.max(np.abs(r2 - exact)) / np.max(np.abs(exact)) < 1e-12


# ------------------------------------------------- signs of Eq. 1, breakdown branch


def _degree(L):
    """Neighbours of each site of an open box, from its coordinates (natural order)."""
    idx = np.indices(tuple(reversed(L))).reshape(len(L), -1)[::-1]    # idx[d] = coordinate d
    return sum((idx[d] > 0).astype(int) + (idx[d] < L[d] - 1).astype(int) for d in range(len(L)))


@pytest.mark.parametrize("axis", ["matsubara", "real"])
def test_dyson_diagonal_signs_from_high_frequency_expansion(axis):
    """Eq. 1 fixes H = w I + C + t A with w = i w_k (or w + i eta on the real axis)
    and C_ii = mu - V_i - Sigma_i.  For |w| >> |C + t A| the inverse expands as
    G = 1/w - (C + tA)/w^2 + (C + tA)^2/w^3 - ..., so
        G_ii = 1/w - c_i/w^2 + (c_i^2 + t^2 Z_i)/w^3 + O(|w|^-4),   Z_i neighbours of i.
    At |w| = 1e3 the second term is ~1e-3 of G_ii and the remainder ~1e-7, so the
    signs of mu, V_i and Sigma_i (each O(1) and distinct here) and the t^2 Z_i term
    are held to 1e-6; every single sign flip misses by more than 1e-4."""
    L = (6, 5)
    rng = np.random.default_rng(21)
    N = 30
    V = rng.uniform(0.5, 1.5, N)
    sigma = rng.uniform(-1.0, 1.0, N) - 1j * rng.uniform(0.2, 0.7, N)
    mu, t, wv, eta = 0.7, -1.0, 1e3, 0.05
    if axis == "matsubara":
        z = O.dyson_diagonal(wv, mu, V, sigma)
        W = 1j * wv
    else:
        z = O.dyson_diagonal_real(wv, eta, mu, V, sigma)
        W = wv + 1j * eta
    G = O.exact_diag(L, (False,) * 3, t, z)
    Z = _degree(L)

    def series(m, v, s):
        c = m - v - s
        return 1 / W - c / W ** 2 + (c * c + t * t * Z) / W ** 3

    rel = lambda ser: float(np.max(np.abs(G - ser) / np.abs(G)))
    assert rel(series(mu, V, sigma)) < 1e-6
    for wrong in (series(-mu, V, sigma), series(mu, -V, sigma), series(mu, V, -sigma)):
        assert rel(wrong) > 1e-4


def test_lanczos_breakdown_on_vanishing_bilinear_norm():
    """Sec. 2.1: in the bilinear form the "norm" sqrt(r^T r) of a non-zero vector can
    vanish.  Built by hand: q1 = e1 and X e1 = a e1 + b e2 give alpha_1 = a and
    q2 = e2; X e2 = b e1 + a2 e2 + e3 + i e4 then leaves r = e3 + i e4, with
    r^T r = 1 + i^2 = 0 while ||r||_2^2 = 2.  That is a breakdown (the partial sum
    of the two steps kept, Eq. 9), not an invariant subspace."""
    a, b, a2 = 0.3 + 0.2j, 0.8 - 0.1j, -0.5 + 0.4j
    X = np.array([[a, b, 0, 0],
                  [b, a2, 1, 1j],
                  [0, 1, 0.2, 0.7],
                  [0, 1j, 0.7, -0.3j]], dtype=complex)
    assert np.array_equal(X, X.T)
    q1 = np.array([1.0, 0.0, 0.0, 0.0])
    acc, al, be, Q, st = O.cs_lanczos(lambda q: X @ q, q1, 4)
    assert st == O.STATUS_BREAKDOWN and len(al) == 2
    assert abs(al[0] - a) < 1e-15 and abs(al[1] - a2) < 1e-15
    assert abs(be[0] - b) < 1e-15 or abs(be[0] + b) < 1e-15     # either square-root branch
    beta = be[0]
    want = np.zeros(4, complex)
    want += a * Q[:, 0] ** 2 + a2 * Q[:, 1] ** 2 + 2 * beta * Q[:, 0] * Q[:, 1]
    assert np.max(np.abs(acc - want)) < 1e-15
    assert np.max(np.abs(acc - np.array([a, a2, 0, 0]))) < 1e-15
    # a bilinear norm that does not vanish: the recurrence goes on
    Y = X.copy()
    Y[1, 3] = Y[3, 1] = 0.9j                 # r^T r = 1 - 0.81
    _, al2, _, _, st2 = O.cs_lanczos(lambda q: Y @ q, q1, 4)
    assert st2 != O.STATUS_BREAKDOWN and len(al2) > 2
    # r = 0 after the first step: an invariant subspace, not a breakdown
    Z = np.diag([a, a2, 0.2, 0.1]).astype(complex)
    _, al3, _, _, st3 = O.cs_lanczos(lambda q: Z @ q, q1, 4)
    assert st3 == O.STATUS_TERMINATED and len(al3) == 1


def test_block_qr_breakdown_and_deflation():
    """The block form's column split (R15): a column with r != 0 and r^T r = 0 is a
    breakdown; a column that vanishes in the 2-norm is deflated."""
    R = np.array([[1.0, 1.0], [0.0, 1.0], [0.0, 1j]], dtype=complex)   # column 1 less its e1 part: (0, 1, i)
    _, _, defl, brk = O._bilinear_qr(R, 1.0, 1e-12, 1e-14)
    assert brk and not defl.any()
    R2 = np.array([[1.0, 2.0], [0.5, 1.0], [0.0, 0.0]], dtype=complex)  # column 1 = 2 x column 0
    Q2, B2, defl2, brk2 = O._bilinear_qr(R2, 1.0, 1e-12, 1e-14)
    assert not brk2 and list(defl2) == [False, True] and np.all(Q2[:, 1] == 0)


def test_cancel_free_xmatvec_matches_dense_X():
    """u = H^-1 (q - H w) is the X-matvec of Eqs. 6-8 (w = blkdiag(B^-1, 0) q)."""
    rng = np.random.default_rng(12)
    L, p = (9, 10), 3
    omega, V, sigma, q1 = I.make_inputs(I.Workload("t", L, -1.0, 0.0, 0.01, 0.5, 10.0, 2, p, 4, 3))
    z = O.dyson_diagonal(omega[0], 0.0, V, sigma[0])
    H = O.dense_H(L, (False,) * 3, -1.0, z)
    _, iface = O.dd_sites(L, p)
    X, _ = _dense_X(H, np.concatenate(iface))
    q = rng.normal(size=90) + 1j * rng.normal(size=90)
    u = O.xmatvec_cancel_free(L, (False,) * 3, -1.0, 0.0, V, sigma[0], omega[0], p, q)
    assert np.max(np.abs(u - X @ q)) < 1e-12 * np.max(np.abs(X @ q))


def test_rounding_amplification_record_c2():
    """The stored amplification of X-matvec rounding into the truncated rank-32 diagonal
    (tests/golden/rounding_spread.json, written by make_rounding_spread.py from the
    oracle alone) is what the oracle gives now, within a factor of 3 (it is a ratio of
    rounding-level quantities, so its value moves with the BLAS's summation order)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("mrs", os.path.join(GOLDEN, "make_rounding_spread.py"))
    mrs = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mrs)
    with open(os.path.join(GOLDEN, "rounding_spread.json")) as f:
        rec = json.load(f)["square128_K64_p4_k32"]
    for k in (0, 63):
        now = mrs.spread("square128_K64_p4_k32", k)
        ratio = now["amplification"] / rec[str(k)]["amplification"]
        assert 1 / 3 < ratio < 3, (k, now, rec[str(k)])
        assert now["delta"] < 1e-14                 # both forms of Eq. 8 agree to rounding
