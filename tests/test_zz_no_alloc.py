"""The allocation-free entry point, dyson_subdomain_diag_noalloc.

It serves host programs that cannot let the solver allocate device memory:
one that reserves all of its device memory in a pool at start-up and treats
any later cudaMalloc as an error, or a plugin inside another framework that
owns every device buffer.  Its scratch is one fixed device array that every
call shares and that keeps the previous call's contents, so each case here
runs two calls in a row and checks both, through the C ABI, against the
plan-based dyson_subdomain_diag (the existing entry point, which allocates)
and directly against the FP64 oracle's diag(B^-1).

This file is collected last on purpose: a run that stops at its first
failure has then already run every other test.
"""
import numpy as np
import pytest

from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12     # FP64 slice recursion against FP64 references, relative per site


def _relerr(got, ref):
    mask = ref != 0
    assert np.array_equal(got[~mask], ref[~mask])      # interface sites: exactly 0
    return float(np.max(np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])))


@pytest.mark.parametrize("L,p", [((128, 128), 4),      # 2D strips, slice width 32
                                 ((8, 8, 8), 2),        # 3D slabs: slice = y-z plane, width 32
                                 ((24, 20), 1)])        # one subdomain: no interface
def test_noalloc_matches_plan_path_and_oracle_on_two_calls(L, p):
    import torch
    from oracle import dyson_oracle as O
    from paper_1102_3137_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    w = I.Workload("t", L, -1.0, 0.0, 0.01, 0.5, 20.0, 3, p, 8, 2)
    omega, V, sigma, q1 = I.make_inputs(w)
    geom = D.make_geometry(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=2)
    plan = D.Plan(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=2)
    Vd = torch.from_numpy(V).to(dev)
    for ks in ((0, 1), (2, 0)):                  # two calls in a row, different frequencies
        om = np.ascontiguousarray(omega[list(ks)])
        sg = np.ascontiguousarray(sigma[list(ks)])
        out = torch.zeros((2, w.N), dtype=torch.complex128, device=dev)
        D.dyson_subdomain_diag_noalloc(geom, 2, torch.from_numpy(om).to(dev), Vd,
                                       torch.from_numpy(sg).to(dev), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = np.zeros((2, w.N), complex)
        D.dyson_subdomain_diag(plan.handle, 2, om, V, sg, ref)
        assert _relerr(got, ref) <= TOL
        orc = O.subdomain_diag_batch(w.L, (False,) * 3, w.t, w.mu, V, sg, om, w.p)
        assert _relerr(got, orc) <= TOL
    plan.close()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch
    dev = torch.device("cuda:0")
    w = I.Workload("t", (128, 128), -1.0, 0.0, 0.01, 0.5, 20.0, 8, 4, 8, 2)
    omega, V, sigma, q1 = I.make_inputs(w)
    geom = D.make_geometry(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=8)
    out = torch.zeros((8, w.N), dtype=torch.complex128, device=dev)
    with pytest.raises(D.DysonError) as e:
        D.dyson_subdomain_diag_noalloc(geom, 8, torch.from_numpy(omega).to(dev),
                                       torch.from_numpy(V).to(dev),
                                       torch.from_numpy(sigma).to(dev), out)
    assert e.value.code == -5 and "bytes of scratch" in str(e.value)


def test_noalloc_rejects_host_pointers_and_too_many_frequencies():
    import ctypes as C
    import torch
    dev = torch.device("cuda:0")
    w = I.Workload("t", (16, 16), -1.0, 0.0, 0.01, 0.5, 20.0, 2, 2, 8, 2)
    omega, V, sigma, q1 = I.make_inputs(w)
    geom = D.make_geometry(w.L, w.t, w.mu, w.p, w.k, D.DYSON_FP64, max_freqs=2)
    lib = D.load()
    out = torch.zeros((2, w.N), dtype=torch.complex128, device=dev)
    od, Vd, sd = (torch.from_numpy(x).to(dev) for x in (omega, V, sigma))
    # a host array where a device pointer is required: rejected before any launch
    rc = lib.dyson_subdomain_diag_noalloc(C.byref(geom), 2, od.data_ptr(), V.ctypes.data,
                                          sd.data_ptr(), out.data_ptr(), None)
    assert rc == -1                                     # DYSON_E_BAD_ARG
    # more frequencies than one launch dimension takes
    rc = lib.dyson_subdomain_diag_noalloc(C.byref(geom), 70000, od.data_ptr(), Vd.data_ptr(),
                                          sd.data_ptr(), out.data_ptr(), None)
    assert rc == -1                                     # DYSON_E_BAD_ARG
    torch.cuda.synchronize()
