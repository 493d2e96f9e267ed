"""Recursive decomposition (Sec. 2.3, last paragraph: domains alternating
(d_x, d_y) = (2, 1), (1, 2), ...) on the GPU through the C ABI, against the
oracle's recursive_diag (pinned in test_oracle_pins.py: exact past closure, one
level equal to the two-strip method)."""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I
from parity_util import OPEN, TOL_FP64, TOL_MIXED, relerr, wl

pytestmark = pytest.mark.gpu

CUT = {"x": D.DYSON_CUT_X, "y": D.DYSON_CUT_Y}
# Truncated runs (k far below each box's rank) are compared directly.  On these
# cases a relative perturbation of 1e-13 in q1 moves the oracle's own result by
# at most 7.3e-11 (measured on the oracle alone, three draws per frequency);
# 1e-9 leaves a factor of ten over that for the GPU's rounding.
TOL_TRUNC_FP64 = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1102_3137_gb300 import build
    build.build()
    D.load()


def exact(w, omega, V, sigma):
    return np.stack([O.exact_diag(w.L, OPEN[:2], w.t, O.axis_diagonal(omega[k], w.mu, V, sigma[k]))
                     for k in range(len(omega))])


@pytest.mark.parametrize("cut", ["x", "y"])
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_recursive_exact_past_closure(cut, precision, tol):
    """20 x 17, boxes down to 30 sites, rank cap 24 >= every cut line (<= 20 sites):
    every box's Lanczos run closes, so the result is the exact diagonal and every
    frequency reports TERMINATED."""
    w = wl((20, 17), 2, 24, K=4, seed=2)
    omega, V, sigma, q1 = I.make_inputs(w)
    rp = D.RecursivePlan(w.L, w.t, w.mu, 24, precision, max_freqs=4, min_sites=30, first_cut=CUT[cut])
    st = np.zeros(4, dtype=np.int32)
    out = rp.solve(omega, V, sigma, q1, status=st)
    ref = exact(w, omega, V, sigma)
    assert relerr(out, ref) <= tol
    assert np.all(st == D.DYSON_ST_TERMINATED)


@pytest.mark.parametrize("L,ms,k,cut", [((24, 20), 48, 6, "x"), ((23, 18), 40, 8, "y"), ((32, 30), 100, 8, "x")])
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_TRUNC_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_recursive_truncated_matches_oracle(L, ms, k, cut, precision, tol):
    """Rank caps far below the boxes' ranks (truncated at every level), odd and even
    extents (the cut line one site off centre), several boxes per level on
    concurrent streams: element by element against the oracle's recursion."""
    K = 3
    w = wl(L, 2, k, K=4, seed=5)
    omega, V, sigma, q1 = I.make_inputs(w)
    omega, sigma = omega[:K], np.ascontiguousarray(sigma[:K])
    rp = D.RecursivePlan(w.L, w.t, w.mu, k, precision, max_freqs=K, min_sites=ms, first_cut=CUT[cut])
    st = np.zeros(K, dtype=np.int32)
    out = rp.solve(omega, V, sigma, q1, status=st)
    for kf in range(K):
        z = O.axis_diagonal(omega[kf], w.mu, V, sigma[kf])
        ref = O.recursive_diag(w.L, w.t, z, q1, k, min_sites=ms, first_cut=cut)
        assert relerr(out[kf], ref) <= tol, kf
    assert np.all(st == 0)


def test_recursive_single_box_is_exact():
    """A lattice of at most min_sites sites is one leaf: the slice recursion's exact
    diagonal."""
    w = wl((9, 7), 2, 4, K=2, seed=4)
    omega, V, sigma, q1 = I.make_inputs(w)
    rp = D.RecursivePlan(w.L, w.t, w.mu, 4, D.DYSON_FP64, max_freqs=2, min_sites=63)
    info = rp.info()
    assert (info["levels"], info["boxes"], info["leaves"]) == (1, 0, 1)
    st = np.zeros(2, dtype=np.int32)
    out = rp.solve(omega, V, sigma, q1, status=st)
    assert relerr(out, exact(w, omega, V, sigma)) <= 1e-12
    assert np.all(st == D.DYSON_ST_TERMINATED)


def test_recursive_plan_info_matches_tree():
    g = D.make_geometry((40, 36), p=2, k_max=8, max_freqs=2)
    boxes = D.dyson_recursive_boxes(g, 90, D.DYSON_CUT_Y)
    rp = D.RecursivePlan((40, 36), -1.0, 0.0, 8, D.DYSON_MIXED, max_freqs=2, min_sites=90,
                         first_cut=D.DYSON_CUT_Y, streams=3)
    info = rp.info()
    assert info["levels"] == int(boxes[:, 4].max()) + 1
    assert info["boxes"] == int((boxes[:, 5] == 0).sum())
    assert info["leaves"] == int((boxes[:, 5] == 1).sum())
    assert info["bytes"] > 0 and info["plans"] >= 2


def test_recursive_device_buffers_repeat_bitwise():
    """Device-resident inputs and outputs give bit for bit the host call's result,
    and a repeated solve the same bits (levels run in a fixed order; boxes of one
    level are disjoint)."""
    torch = pytest.importorskip("torch")
    w = wl((32, 30), 2, 8, K=4, seed=5)
    omega, V, sigma, q1 = I.make_inputs(w)
    rp = D.RecursivePlan(w.L, w.t, w.mu, 8, D.DYSON_MIXED, max_freqs=4, min_sites=100)
    a = rp.solve(omega, V, sigma, q1)
    b = rp.solve(omega, V, sigma, q1)
    assert np.array_equal(a, b)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.zeros((4, w.N), dtype=torch.complex128, device="cuda")
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    D.dyson_recursive_solve(rp.handle, 4, w.N, dev(omega), dev(V), dev(sigma), dev(q1), out, st)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), a)
    assert int(st.abs().sum()) == 0


@pytest.mark.parametrize("precision,tol_trunc,tol_exact", [(D.DYSON_FP64, TOL_TRUNC_FP64, TOL_FP64),
                                                           (D.DYSON_MIXED, TOL_MIXED, TOL_MIXED)])
def test_recursive_real_axis(precision, tol_trunc, tol_exact):
    """Real frequencies w + i eta (the remark after Eq. 1; eta = 0.1, w across the band):
    every box plan takes eta from the geometry.  Rank 6: against the oracle's recursion
    on the same diagonal (a 1e-13 perturbation of q1 moves it by at most 3.5e-11 here);
    rank 30 (past every box's closure): against the exact diagonal."""
    eta = 0.1
    w = wl((20, 18), 2, 6, K=3, seed=6)
    omega, V, sigma, q1 = I.make_inputs(w, axis="real")
    zs = [O.dyson_diagonal_real(omega[k], eta, w.mu, V, sigma[k]) for k in range(3)]
    for k, tol in ((6, tol_trunc), (30, tol_exact)):
        rp = D.RecursivePlan(w.L, w.t, w.mu, k, precision, max_freqs=3, min_sites=40, eta=eta)
        st = np.zeros(3, dtype=np.int32)
        out = rp.solve(omega, V, sigma, q1, status=st)
        for kf in range(3):
            if k == 6:
                ref = O.recursive_diag(w.L, w.t, zs[kf], q1, k, min_sites=40)
            else:
                ref = O.exact_diag(w.L, OPEN[:2], w.t, zs[kf])
            assert relerr(out[kf], ref) <= tol, (k, kf)
        assert np.all(st == (D.DYSON_ST_TERMINATED if k == 30 else 0))
        rp.close()


def test_recursive_rejects_host_pointers_as_device_buffers():
    """Device-memory calls check every pointer before any work is enqueued."""
    import ctypes
    w = wl((12, 10), 2, 4, K=1, seed=3)
    omega, V, sigma, q1 = I.make_inputs(w)
    rp = D.RecursivePlan(w.L, w.t, w.mu, 4, D.DYSON_FP64, max_freqs=1, min_sites=20)
    out = np.zeros((1, w.N), complex)
    rc = D.load().dyson_recursive_solve(rp.handle, 1, omega.ctypes.data, V.ctypes.data, sigma.ctypes.data,
                                        q1.ctypes.data, out.ctypes.data, None, D.DYSON_MEM_DEVICE, None)
    assert rc == -1 and "device memory" in D.dyson_last_error()
    good = rp.solve(omega, V, sigma, q1)                     # the plan is still usable
    assert np.all(np.isfinite(good)) and np.array_equal(good, rp.solve(omega, V, sigma, q1))
