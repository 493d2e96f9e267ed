"""C-ABI checks that need no GPU: the library loads, exports every symbol that
include/dyson.h declares, validates arguments, and builds the
domain-decomposition ordering (Sec. 2.2, Fig. 1) identical to the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1102_3137_gb300 import build
    build.build()
    return D.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dyson.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dyson_[A-Za-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    out = os.popen(f"nm -D --defined-only {D.LIB_PATH}").read()
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


@pytest.mark.parametrize("L,p", [((16, 16), 2), ((128, 128), 4), ((9, 13), 3), ((4, 5, 9), 3),
                                 ((32, 32, 32), 8), ((7, 5), 3), ((6, 1), 1)])
def test_partition_matches_oracle(lib, L, p):
    g = D.make_geometry(L, p=p, k_max=4, max_freqs=2)
    h, m, dd = D.dyson_partition(g)
    _, hh, _ = O.dd_partition(L, p)
    assert list(h) == hh
    sub, iface = O.dd_sites(L, p)
    W = (max(s.shape[1] for s in sub) + 3) // 4 * 4     # slice width padded to a multiple of 4
    ref = []
    for s in sub:
        blk = -np.ones((L[0], W), dtype=np.int64)
        blk[:, :s.shape[1]] = s
        ref.append(blk.ravel())
    ref = np.concatenate(ref + [np.asarray(x) for x in iface])
    assert np.array_equal(ref, dd)
    assert m == sum(len(x) for x in iface)


@pytest.mark.parametrize("bad", [
    dict(L=(16, 16), p=17), dict(L=(16, 16), p=0), dict(L=(4, 4), p=3), dict(L=(16, 16), k_max=0),
    dict(L=(16, 16), k_max=300), dict(L=(16, 16), max_freqs=0), dict(L=(16, 16), precision=5),
])
def test_bad_geometry_rejected_without_gpu(lib, bad):
    kw = dict(L=(16, 16), p=2, k_max=4, max_freqs=2)
    kw.update(bad)
    g = D.make_geometry(**kw)
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_create(g)
    assert e.value.code == -1
    assert D.dyson_last_error()


def test_wide_slices_reported_unsupported(lib):
    g = D.make_geometry((32, 32, 32), p=2, k_max=4, max_freqs=1)      # W = 32 * 16 = 512
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g)
    assert e.value.code == -4


def test_wide_slices_within_limits(lib):
    # 32^3 with p = 8: W = 128, taken by the global-memory factor and chunked sweeps;
    # the footprint carries the factor workspace (304 CTAs x 2 W x W FP64 matrices)
    g = D.make_geometry((32, 32, 32), p=8, k_max=48, max_freqs=1)
    assert D.dyson_plan_footprint(g) > 304 * 2 * 128 * 128 * 16
    # W = 256 with Lx = 64: the FP64 row buffer (256 KB) cannot stay on chip,
    # the complex64 one (128 KB) can
    g = D.make_geometry((64, 16, 33), p=2, k_max=4, max_freqs=1)
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g)
    assert e.value.code == -4 and "row buffer" in str(e.value)
    g.precision = D.DYSON_MIXED
    assert D.dyson_plan_footprint(g) > 0
    # 48^3 with p = 8: W = 48 * 6 = 288, within the 320 limit; its complex64 row
    # buffer (110 KB) leaves room for the ring, the FP64 one (221 KB) does not
    g = D.make_geometry((48, 48, 48), p=8, k_max=64, max_freqs=1, precision=D.DYSON_MIXED)
    assert D.dyson_plan_footprint(g) > 0
    g.precision = D.DYSON_FP64
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g)
    assert e.value.code == -4 and "row buffer" in str(e.value)


def test_real_axis_eta_validated(lib):
    g = D.make_geometry((16, 16), p=2, k_max=4, max_freqs=1, eta=-0.1)
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g)
    assert e.value.code == -1
    g.eta = 0.05
    assert D.dyson_plan_footprint(g) > 0


def test_block_size_validated(lib):
    for bad in (dict(block_size=2, k_max=9), dict(block_size=5, k_max=10), dict(block_size=-1, k_max=8),
                dict(block_size=2, k_max=8, max_freqs=40000)):
        g = D.make_geometry((16, 16), p=2, **{"max_freqs": 1, **bad})
        with pytest.raises(D.DysonError) as e:
            D.dyson_plan_footprint(g)
        assert e.value.code == -1
    g1 = D.make_geometry((16, 16), p=2, k_max=8, max_freqs=4)
    g2 = D.make_geometry((16, 16), p=2, k_max=8, max_freqs=4, block_size=2)
    # a block plan keeps nb work slots per frequency and k_max + nb basis columns
    assert D.dyson_plan_footprint(g2) > D.dyson_plan_footprint(g1)


def test_precond_choice_validated(lib):
    g = D.make_geometry((128, 128), p=4, k_max=8, max_freqs=2, precond=D.DYSON_PRECOND_LAYER)
    assert D.dyson_plan_footprint(g) > 0
    g3 = D.make_geometry((8, 8, 9), p=2, k_max=8, max_freqs=2, precond=D.DYSON_PRECOND_LAYER)
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g3)                  # 3D slabs of slice width <= 64: only the banded form
    assert e.value.code == -4
    g.precond = 7
    with pytest.raises(D.DysonError) as e:
        D.dyson_plan_footprint(g)
    assert e.value.code == -1
    # the layer blocks add the surface Green's functions and the inverse blocks
    ga = D.make_geometry((128, 128), p=4, k_max=8, max_freqs=2, precond=D.DYSON_PRECOND_AUTO)
    gb = D.make_geometry((128, 128), p=4, k_max=8, max_freqs=2, precond=D.DYSON_PRECOND_BANDED)
    assert D.dyson_plan_footprint(ga) > D.dyson_plan_footprint(gb)


def test_footprint(lib):
    g = D.make_geometry((128, 128), p=4, k_max=32, max_freqs=64)
    b = D.dyson_plan_footprint(g)
    # Lanczos basis alone: 64 freqs x 33 vectors x 16768 slots x 16 B
    assert b > 64 * 33 * 16768 * 16
    g.precision = D.DYSON_MIXED
    assert D.dyson_plan_footprint(g) < b * 1.5     # + complex64 copy of g_s, refinement vectors


def test_null_plan_is_an_error(lib):
    z = np.zeros(4)
    with pytest.raises(D.DysonError):
        D.dyson_solve(None, 1, z[:1], z, np.zeros(4, complex), z, np.zeros(4, complex))


def test_layer_preconditioner_limits(lib):
    # 2D strips with Lx <= 160 and slice width <= 32, or Lx <= 1024 and slice width 32,
    # take the exact layer blocks
    for L in ((160, 33), (200, 65), (1024, 65)):
        ok = D.make_geometry(L, p=2, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_LAYER)
        assert D.dyson_plan_footprint(ok) > 0
    # line beyond 160 with slice width 16; slice width 36 > 32; line beyond 1024
    for L, p in (((161, 33), 2), ((64, 70), 2), ((1025, 65), 2)):
        g = D.make_geometry(L, p=p, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_LAYER)
        with pytest.raises(D.DysonError) as e:
            D.dyson_plan_footprint(g)
        assert e.value.code == -4
        g.precond = D.DYSON_PRECOND_AUTO                 # falls back to the banded form
        auto = D.dyson_plan_footprint(g)
        g.precond = D.DYSON_PRECOND_BANDED
        assert D.dyson_plan_footprint(g) == auto
    g = D.make_geometry((160, 33), p=1, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_LAYER)
    with pytest.raises(D.DysonError):                    # no interface: nothing to precondition
        D.dyson_plan_footprint(g)
    # 3D slabs with slices wider than 64 and layers of Lx Ly <= 1024 sites take them too
    for L, p in (((6, 9, 16), 2), ((4, 16, 17), 2), ((32, 32, 32), 8)):
        ok = D.make_geometry(L, p=p, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_LAYER)
        banded = D.make_geometry(L, p=p, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_BANDED)
        assert D.dyson_plan_footprint(ok) > D.dyson_plan_footprint(banded)
    g = D.make_geometry((33, 32, 32), p=8, k_max=4, max_freqs=1, precond=D.DYSON_PRECOND_LAYER)
    with pytest.raises(D.DysonError) as e:               # layer of 33 x 32 = 1056 sites
        D.dyson_plan_footprint(g)
    assert e.value.code == -4
