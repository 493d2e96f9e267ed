"""The two interface preconditioners of the H solves (the paper leaves the
solver open): the exact layer blocks S_ll of the Schur complement (2D strips)
and the banded approximation.  Both must give the same X-matvec and the same
terminated diagonal to the form's tolerance; the exact blocks must cut the
interface iterations to one or two per solve."""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I
from parity_util import OPEN, TOL_FP64, TOL_MIXED, plan_for, relerr, wl

pytestmark = pytest.mark.gpu

PRE = [D.DYSON_PRECOND_LAYER, D.DYSON_PRECOND_BANDED]


@pytest.mark.parametrize("pre", PRE)
@pytest.mark.parametrize("L,p", [((40, 37), 3), ((17, 50), 4), ((100, 30), 2), ((160, 21), 3),
                                 ((200, 65), 2), ((512, 97), 3)])     # the last two: lines beyond 160
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, 1e-11), (D.DYSON_MIXED, 1e-9)])
def test_xmatvec_both_preconditioners(L, p, pre, precision, tol):
    w = wl(L, p, 4, K=2)
    omega, V, sigma, _ = I.make_inputs(w)
    pl = plan_for(w, precision, precond=pre)
    rng = np.random.default_rng(21)
    q = rng.normal(size=(2, w.N)) + 1j * rng.normal(size=(2, w.N))
    u = np.zeros_like(q)
    D.dyson_xmatvec(pl.handle, 2, omega, V, sigma, q, u)
    for k in range(2):
        ref = O.xmatvec(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], p, q[k])
        assert np.max(np.abs(u[k] - ref)) <= tol * np.max(np.abs(ref))
    pl.close()


@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, TOL_FP64), (D.DYSON_MIXED, TOL_MIXED)])
def test_terminated_diagonal_same_with_both(precision, tol):
    # 16 x 17, p = 2: m = 16 interface sites, k = 24 runs past closure (exact diagonal)
    w = wl((16, 17), 2, 24, K=3)
    omega, V, sigma, q1 = I.make_inputs(w)
    exact = np.stack([O.exact_diag(w.L, OPEN, w.t, O.dyson_diagonal(omega[k], w.mu, V, sigma[k]))
                      for k in range(w.K)])
    outs = []
    for pre in PRE:
        pl = plan_for(w, precision, precond=pre)
        st = np.zeros(w.K, np.int32)
        outs.append(pl.solve(omega, V, sigma, q1, status=st))
        assert np.all(st == D.DYSON_ST_TERMINATED)
        pl.close()
    for out in outs:
        assert relerr(out, exact) <= tol


def test_layer_blocks_cut_interface_iterations():
    # the lowest Matsubara frequencies are the worst conditioned (|H^-1| <= 1/w_0)
    w = wl((96, 97), 4, 6, K=4, beta=20.0)
    omega, V, sigma, q1 = I.make_inputs(w)
    per = {}
    for pre in PRE:
        pl = plan_for(w, D.DYSON_FP64, precond=pre)
        pl.solve(omega, V, sigma, q1)
        info = pl.info(w.K)
        per[pre] = info["iters"] / info["steps"]          # one interface solve per FP64 X-matvec
        pl.close()
    # COCG to 1e-13 with M = blkdiag(S_ll) in exact arithmetic (oracle, this geometry):
    # 4 iterations at w_0, 3 at w_1; the lines couple through strips of height 24
    assert np.all(per[D.DYSON_PRECOND_LAYER] <= np.array([4.5, 3.5, 3.5, 3.5]))
    assert np.all(per[D.DYSON_PRECOND_LAYER] < per[D.DYSON_PRECOND_BANDED])


def test_long_line_layer_blocks_cut_interface_iterations():
    """Lines longer than 160 sites take the global-memory form of the layer blocks
    (surface Green's functions with the boundary columns in global memory, block
    Gauss-Jordan inverse); it must still cut the interface iterations well below the
    banded form's on the 512-site lines of the 512^2 benchmark's strips."""
    w = wl((512, 65), 2, 4, K=3, beta=10.0)
    omega, V, sigma, q1 = I.make_inputs(w)
    per = {}
    for pre in PRE:
        pl = plan_for(w, D.DYSON_FP64, precond=pre)
        pl.solve(omega, V, sigma, q1)
        info = pl.info(w.K)
        per[pre] = info["iters"] / info["steps"]
        pl.close()
    # one interface line: its exact block is S itself, so COCG needs the iterations the
    # complex64 inverse leaves to reach 1e-13 (two or three)
    assert np.all(per[D.DYSON_PRECOND_LAYER] <= 3.5)
    assert np.all(per[D.DYSON_PRECOND_LAYER] < per[D.DYSON_PRECOND_BANDED])


@pytest.mark.parametrize("pre", PRE)
@pytest.mark.parametrize("L,p", [((6, 9, 16), 2), ((4, 16, 17), 2), ((5, 12, 26), 2), ((8, 8, 27), 3)])
@pytest.mark.parametrize("precision,tol", [(D.DYSON_FP64, 1e-11), (D.DYSON_MIXED, 1e-9)])
def test_3d_xmatvec_both_preconditioners(L, p, pre, precision, tol):
    """3D slabs (slice width > 64): the exact layer blocks S_ll of A = Lx Ly sites, from
    the slab's surface Green's functions on its T = Ly boundary rows, give the same
    X-matvec as the banded form and the oracle."""
    w = wl(L, p, 4, K=2)
    omega, V, sigma, _ = I.make_inputs(w)
    pl = plan_for(w, precision, precond=pre)
    rng = np.random.default_rng(23)
    q = rng.normal(size=(2, w.N)) + 1j * rng.normal(size=(2, w.N))
    u = np.zeros_like(q)
    D.dyson_xmatvec(pl.handle, 2, omega, V, sigma, q, u)
    for k in range(2):
        ref = O.xmatvec(w.L, OPEN, w.t, w.mu, V, sigma[k], omega[k], p, q[k])
        assert np.max(np.abs(u[k] - ref)) <= tol * np.max(np.abs(ref))
    pl.close()


def test_3d_layer_blocks_cut_interface_iterations():
    """On 3D slabs the exact layer blocks leave only the coupling between layers
    through whole slabs, which thin slabs keep strong: COCG to 1e-13 with
    M = blkdiag(S_ll) formed densely from H on this geometry (slabs of 8, 8, 7 layers
    of 12 x 16 sites, beta = 20) takes 15, 9 and 7 iterations at w_0, w_1, w_2 in exact
    arithmetic; the GPU must match that and beat the banded form."""
    w = wl((12, 16, 25), 3, 6, K=3, beta=20.0)
    omega, V, sigma, q1 = I.make_inputs(w)
    per = {}
    for pre in PRE:
        pl = plan_for(w, D.DYSON_FP64, precond=pre)
        st = np.zeros(w.K, np.int32)
        pl.solve(omega, V, sigma, q1, status=st)
        assert np.all((st & (D.DYSON_ST_NO_CONVERGENCE | D.DYSON_ST_BREAKDOWN)) == 0)
        info = pl.info(w.K)
        per[pre] = info["iters"] / info["steps"]
        pl.close()
    assert np.all(per[D.DYSON_PRECOND_LAYER] <= np.array([16.0, 10.0, 8.0]))
    assert np.all(per[D.DYSON_PRECOND_LAYER] < per[D.DYSON_PRECOND_BANDED])
