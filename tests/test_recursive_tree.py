"""Host side of the recursive decomposition (Sec. 2.3, last paragraph), no GPU:
the box tree the C library builds (origins, extents, levels, leaves and cut
lines, the line derived from the orientation its box plans use) is the one the
oracle's recursive_diag walks, and bad arguments are rejected before any
device work."""
import numpy as np
import pytest

from oracle import dyson_oracle as O
from paper_1102_3137_gb300 import dyson as D


@pytest.fixture(scope="module")
def lib():
    from paper_1102_3137_gb300 import build
    build.build()
    return D.load()


@pytest.mark.parametrize("L,ms,cut", [((12, 11), 20, "x"), ((16, 9), 10, "y"), ((8, 8), 4, "x"),
                                      ((2, 9), 4, "x"), ((5, 1), 2, "y"), ((40, 36), 90, "y"),
                                      ((33, 64), 64, "x"), ((1, 1), 1, "x")])
def test_box_tree_matches_oracle(lib, L, ms, cut):
    N = L[0] * L[1]
    rng = np.random.default_rng(1)
    z = rng.uniform(-1, 1, N) + 1j * rng.uniform(0.5, 1.0, N)
    walked = []
    O.recursive_diag(L, -1.0, z, rng.uniform(-1, 1, N), 1, min_sites=ms, first_cut=cut, boxes=walked)
    g = D.make_geometry(L, p=2, k_max=1, max_freqs=1)
    tree = D.dyson_recursive_boxes(g, ms, D.DYSON_CUT_X if cut == "x" else D.DYSON_CUT_Y)
    assert sorted(map(tuple, tree.tolist())) == sorted(walked)
    # every site lies in exactly one leaf or on exactly one cut line
    cover = np.zeros((L[1], L[0]), dtype=int)
    for x0, y0, nx, ny, lev, leaf, axis, line in tree:
        if leaf:
            cover[y0:y0 + ny, x0:x0 + nx] += 1
        elif axis == 0:
            cover[y0:y0 + ny, line] += 1
        else:
            cover[line, x0:x0 + nx] += 1
    assert cover.min() == 1 and cover.max() == 1


@pytest.mark.parametrize("bad", [dict(dim3=True), dict(min_sites=0), dict(first_cut=2), dict(block_size=2),
                                 dict(streams=17), dict(k_max=0)])
def test_recursive_bad_arguments_rejected_without_gpu(lib, bad):
    L = (4, 5, 6) if bad.get("dim3") else (16, 16)
    g = D.make_geometry(L, p=2, k_max=bad.get("k_max", 4), max_freqs=2, block_size=bad.get("block_size", 1))
    with pytest.raises(D.DysonError) as e:
        D.dyson_recursive_plan_create(g, bad.get("min_sites", 16), bad.get("first_cut", 0), bad.get("streams", 0))
    assert e.value.code == -1
    assert "recursive" in D.dyson_last_error()
