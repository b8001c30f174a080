"""Compressed T_A and V on the GPU (Sec. 4: ACA at tolerance 1e-4, the vector potential compressed
apart from the scalar one) against the oracle's dense operators.

The ACA pivots are taken in FP32 on the device and in FP64 in the oracle, so the crosses are not
compared one by one; what both must meet is the product error of the compressed matrices against
the dense ones.  Tolerance: the stopping rule bounds each block's remainder near eps times the
block's norm (a heuristic bound), so the relative product error is held to 3 eps.  The block list
is integer work fixed by the geometry and is compared exactly with the oracle's.
"""

import ctypes

import numpy as np
import pytest

import synth
from oracle import efie, lowrank as L

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402

EPS = 1e-4
TOL = 3 * EPS


@pytest.fixture(scope="module")
def ctx():
    from paper_1803_08333_gb300 import build

    build.build()
    return rf.Context(0)


def _case(memo, level, k):
    def make():
        m = synth.geodesic_sphere(level)
        D = efie.discretize(m.verts, m.tris)
        TA, V = efie.assemble(D, k)
        return m, D, TA, V

    return memo(("hm_gpu", level, k), make)


def _rel_cols(y, ref):
    return max(np.linalg.norm(y[c] - ref[c]) / np.linalg.norm(ref[c]) for c in range(ref.shape[0]))


def _rand(n, cols, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((cols, n)) + 1j * rng.standard_normal((cols, n))


def test_compressed_products_match_the_oracle(ctx, memo):
    m, D, TA, V = _case(memo, 8, 1e-3)  # 1920 RWG functions, 1280 cells
    op = rf.Operator(ctx, m.verts, m.tris, 1e-3)
    H = rf.Compressed(op, eps=EPS)
    x = _rand(D.N, 3, 1)
    y = H.apply("T_A", torch.from_numpy(x)).cpu().numpy()
    assert _rel_cols(y, (TA @ x.T).T) <= TOL
    xs = _rand(D.nc, 2, 2)
    ys = H.apply("V", torch.from_numpy(xs)).cpu().numpy()
    assert _rel_cols(ys, (V @ xs.T).T) <= TOL
    inf = H.info()
    for name, (cen, lo, hi), n in (("T_A", L.edge_supports(D), D.N), ("V", L.cell_supports(D), D.nc)):
        T = L.cluster_tree(cen, lo, hi, 32)
        sym = [(a, b, adm) for a, b, adm in L.block_tree(T, T, 1.0) if a.start <= b.start]
        n_adm = sum(1 for _, _, adm in sym if adm)
        i = inf[name]
        assert i["n"] == n
        assert i["lowrank_blocks"] + i["dense_blocks"] == len(sym)
        assert i["lowrank_blocks"] + i["capped_blocks"] + i["small_blocks"] == n_adm and i["capped_blocks"] == 0
        assert 0 < i["max_rank"] <= 64
        assert i["bytes"] < 0.75 * 8 * n * n  # a symmetric half of the dense bytes and less
    H.close()


@pytest.mark.parametrize("k", [1.0, 1e-5])
def test_compressed_products_across_frequency(ctx, memo, k):
    m, D, TA, V = _case(memo, 6, k)  # 1080 RWG functions
    op = rf.Operator(ctx, m.verts, m.tris, k)
    H = rf.Compressed(op, eps=EPS)
    x = _rand(D.N, 1, 3)
    assert _rel_cols(H.apply("T_A", torch.from_numpy(x)).cpu().numpy(), (TA @ x.T).T) <= TOL
    xs = _rand(D.nc, 1, 4)
    assert _rel_cols(H.apply("V", torch.from_numpy(xs)).cpu().numpy(), (V @ xs.T).T) <= TOL


def test_columns_streams_launches_and_the_rank_cap(ctx, memo):
    m, D, TA, V = _case(memo, 6, 1.0)
    op = rf.Operator(ctx, m.verts, m.tris, 1.0)
    H = rf.Compressed(op, eps=EPS)
    x = torch.from_numpy(_rand(D.N, 3, 5))
    y3 = H.apply("T_A", x).cpu().numpy()
    for c in range(3):
        y1 = H.apply("T_A", x[c]).cpu().numpy()[0]
        assert np.linalg.norm(y1 - y3[c]) <= 1e-12 * np.linalg.norm(y3[c])
    s = torch.cuda.Stream()  # a non-blocking caller stream
    with torch.cuda.stream(s):
        ys = H.apply("T_A", x.cuda(), stream=s)
    s.synchronize()
    assert np.linalg.norm(ys.cpu().numpy() - y3) <= 1e-12 * np.linalg.norm(y3)
    before = rf.launch_count()
    H.apply("V", torch.from_numpy(_rand(D.nc, 1, 6)))
    assert rf.launch_count() - before == 3  # gather, blocks, scatter
    # a rank cap of 1 leaves most admissible blocks dense: the product is then closer to dense,
    # and no block takes fewer bytes than under the default cap (the same crosses, or dense)
    Hc = rf.Compressed(op, eps=EPS, max_rank=1)
    ic, i64 = Hc.info()["T_A"], H.info()["T_A"]
    assert ic["capped_blocks"] > 0 and ic["max_rank"] <= 1
    adm = lambda i: i["lowrank_blocks"] + i["capped_blocks"] + i["small_blocks"]  # noqa: E731
    assert adm(ic) == adm(i64)
    assert _rel_cols(Hc.apply("T_A", x).cpu().numpy(), (TA @ x.numpy().T).T) <= TOL
    assert ic["bytes"] >= i64["bytes"]
    Hc.close()
    H.close()


def test_compressed_argument_errors(ctx, memo):
    m, D, _, _ = _case(memo, 6, 1.0)
    op = rf.Operator(ctx, m.verts, m.tris, 1.0)
    for kw in ({"leaf": 4}, {"eps": 0.0}, {"eta": -1.0}, {"max_rank": 0}, {"max_rank": 300}):
        with pytest.raises(rf.RfcmpError) as ei:
            rf.Compressed(op, **kw)
        assert ei.value.status == -1
    H = rf.Compressed(op)
    x = torch.zeros((1, D.N), dtype=torch.complex128, device="cuda")
    y = torch.empty_like(x)
    L_ = rf.lib()
    assert L_.rfcmp_hm_apply(H._h, 2, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 1, None) == -1
    assert L_.rfcmp_hm_apply(H._h, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), 1, None) == -1
    assert L_.rfcmp_hm_apply(H._h, 0, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), 0, None) == -1
    with pytest.raises(ValueError):
        H.apply("V", x)
    H.close()
