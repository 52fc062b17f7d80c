"""The batched workload's generator (no GPU): sizes, kinds, gains and seeding follow the recipe."""
import numpy as np

from paper_2308_07403_gb300 import graphs


def test_workload_batched_recipe():
    kinds, n, As, g = graphs.workload_batched(300, 32, 512)
    assert len(kinds) == len(As) == n.size == g.size == 300
    assert n.min() >= 32 and n.max() <= 512
    assert set(kinds) == set(graphs.BATCH_KINDS)
    for k, m, A, gam in zip(kinds, n, As, g):
        assert A.shape == (m, m) and A.dtype == np.uint8
        assert not A.diagonal().any()
        assert gam == 0.5 / (graphs.max_out_degree(A) + 1)
        if k in ("grid", "ws"):
            assert np.array_equal(A, A.T)
        if k == "grid":
            assert np.array_equal(A, graphs.grid4(m, int(np.ceil(np.sqrt(m)))))


def test_workload_batched_is_seeded():
    a = graphs.workload_batched(20, 32, 128, replica=3)
    b = graphs.workload_batched(20, 32, 128, replica=3)
    c = graphs.workload_batched(20, 32, 128, replica=4)
    assert all(np.array_equal(x, y) for x, y in zip(a[2], b[2]))
    assert not all(x.shape == y.shape and np.array_equal(x, y) for x, y in zip(a[2], c[2]))
