"""The allocation-free entry point (dyson_subdomain_diag_noalloc), for callers
that cannot call cudaMalloc: checked through the C ABI against the
plan-based dyson_subdomain_diag on two calls in a row (the fixed scratch is
shared and keeps the previous call's contents), and its size limit.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1102_3137_gb300 import dyson as D
from paper_1102_3137_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_plan_path_on_two_calls():
    import torch
    from paper_1102_3137_gb300 import build
    build.build()
    dev = torch.device("cuda:0")
    w = I.Workload("t", (128, 128), -1.0, 0.0, 0.01, 0.5, 20.0, 3, 4, 8, 2)
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
        ref = np.zeros((2, w.N), complex)
        D.dyson_subdomain_diag(plan.handle, 2, om, V, sg, ref)
        got = out.cpu().numpy()
        mask = ref != 0
        assert np.array_equal(got[~mask], ref[~mask])
        assert np.max(np.abs(got[mask] - ref[mask]) / np.abs(ref[mask])) <= 1e-12
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
