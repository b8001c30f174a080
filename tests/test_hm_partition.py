"""The library's host partition of the compressed form equals the oracle's, integer for integer.

rfcmp_hm_partition runs on the host only (no device), so these run without a GPU: the cluster
order and the symmetric block list (blocks on and above the block diagonal, admissibility by
min(diam) <= eta dist of the support boxes, Sec. 4 compression readings) must equal those of
oracle/lowrank.py on the same items, for point clouds and for the RWG functions and cells of a
mesh.
"""

import numpy as np
import pytest

import paper_1803_08333_gb300 as rf
import synth
from oracle import efie, lowrank as L
from paper_1803_08333_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _oracle_partition(cen, lo, hi, leaf, eta):
    T = L.cluster_tree(cen, lo, hi, leaf)
    blocks = sorted(
        ((a.start, a.stop, b.start, b.stop, int(adm)) for a, b, adm in L.block_tree(T, T, eta) if a.start <= b.start),
        key=lambda t: (t[0], t[2]),
    )
    return T.perm, np.array(blocks, dtype=np.int64).reshape(-1, 5)


def _fib_sphere(n):
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(1.0 - z * z)
    ph = np.pi * (1.0 + 5**0.5) * i
    return np.stack([r * np.cos(ph), r * np.sin(ph), z], axis=1)


@pytest.mark.parametrize("n,leaf,eta", [(800, 16, 0.5), (800, 16, 1.0), (1500, 32, 2.0), (37, 8, 1.0)])
def test_point_cloud_partition_matches_oracle(n, leaf, eta):
    P = _fib_sphere(n)
    h = np.sqrt(4 * np.pi / n)
    lo, hi = P - h / 2, P + h / 2
    perm, blocks = rf.hm_partition(P, lo, hi, leaf, eta)
    perm_o, blocks_o = _oracle_partition(P, lo, hi, leaf, eta)
    assert np.array_equal(perm, perm_o)
    assert np.array_equal(blocks.astype(np.int64), blocks_o)


@pytest.mark.parametrize("eta", [1.0, 2.0])
def test_mesh_partition_matches_oracle(memo, eta):
    def disc():
        m = synth.geodesic_sphere(8)
        return efie.discretize(m.verts, m.tris)

    D = memo(("hm_partition_sphere8",), disc)
    for cen, lo, hi in (L.edge_supports(D), L.cell_supports(D)):
        perm, blocks = rf.hm_partition(cen, lo, hi, 32, eta)
        perm_o, blocks_o = _oracle_partition(cen, lo, hi, 32, eta)
        assert np.array_equal(perm, perm_o)
        assert np.array_equal(blocks.astype(np.int64), blocks_o)
        assert blocks[:, 4].sum() > 0


def test_repeated_coordinates_and_degenerate_sizes():
    # equal centres: the stable sort keeps the input order on both sides
    P = np.repeat(_fib_sphere(40), 5, axis=0)
    perm, blocks = rf.hm_partition(P, P - 0.1, P + 0.1, 8, 1.0)
    perm_o, blocks_o = _oracle_partition(P, P - 0.1, P + 0.1, 8, 1.0)
    assert np.array_equal(perm, perm_o) and np.array_equal(blocks.astype(np.int64), blocks_o)
    perm, blocks = rf.hm_partition(np.zeros((0, 3)), np.zeros((0, 3)), np.zeros((0, 3)), 8, 1.0)
    assert perm.size == 0 and blocks.shape == (0, 5)
    perm, blocks = rf.hm_partition(np.zeros((1, 3)), np.zeros((1, 3)), np.zeros((1, 3)), 8, 1.0)
    assert list(perm) == [0] and blocks.tolist() == [[0, 1, 0, 1, 0]]  # touching boxes: never admissible


def test_partition_argument_errors():
    P = _fib_sphere(50)
    for leaf, eta in ((0, 1.0), (8, -1.0), (8, float("nan"))):
        with pytest.raises(rf.RfcmpError) as ei:
            rf.hm_partition(P, P, P, leaf, eta)
        assert ei.value.status == -1
    bad = P.copy()
    bad[3, 1] = np.inf
    with pytest.raises(rf.RfcmpError):
        rf.hm_partition(bad, P, P, 8, 1.0)
    import ctypes

    perm = np.empty(50, np.int32)
    blocks = np.empty((1, 5), np.int32)
    nb = ctypes.c_int64()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    st = rf.lib().rfcmp_hm_partition(vp(P), vp(P), vp(P), 50, 8, 1.0, vp(perm), vp(blocks), 1, ctypes.byref(nb))
    assert st == -1 and nb.value > 1


def test_hm_opts_defaults_and_layout():
    import ctypes

    o = rf.HmOpts()
    rf.lib().rfcmp_hm_opts_default(ctypes.byref(o))
    assert o.eps == 1e-4 and o.eta == 1.0 and o.leaf == 32 and o.max_rank == 64
    assert ctypes.sizeof(rf.HmOpts) == 8 + 8 + 4 + 4 + 6 * 4
    assert ctypes.sizeof(rf.HmInfo) == 6 * 2 * 8 + 2 * 4 + 6 * 4


def test_compressed_entry_points_refuse_null_handles():
    import ctypes

    L_ = rf.lib()
    out = ctypes.c_void_p()
    assert L_.rfcmp_hm_create(None, None, ctypes.byref(out)) == -1
    assert L_.rfcmp_hm_apply(None, 0, None, None, 1, None) == -1
    assert L_.rfcmp_hm_info_get(None, ctypes.byref(rf.HmInfo())) == -1
    assert L_.rfcmp_hm_destroy(None) == 0
