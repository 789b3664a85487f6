"""The library's host-side treecode plan (ibim_treecode_plan, the lists that
ibim_treecode_setup uploads) equals the oracle's tree and lists exactly, entry
by entry and in order, on caller-ordered clouds (no GPU needed)."""
import numpy as np
import pytest

from oracle import treecode as tc
from paper_1709_08070_gb300 import inputs

CENTRES = [(28.0 * i, 28.0 * j, 0.0) for i in range(3) for j in range(3)]


@pytest.mark.parametrize("theta,interp,n_per", [(0.5, 0, 700), (0.7, 1, 1000), (0.9, 1, 1500), (0.8, 0, 333)])
def test_plan_equals_oracle_lists(theta, interp, n_per):
    from paper_1709_08070_gb300 import ibim
    xs, _, _ = inputs.sphere_cluster_cloud(n_per, CENTRES, radius=5.0, seed=4)
    tau = 0.3
    plan = ibim.ibim_treecode_plan(xs, theta, tau, interp)
    tree = tc.TileTree(xs)
    lists = tree.lists(theta, tau, bool(interp))
    assert plan["n_t"] == tree.n_t and plan["clusters"] == len(tree.clusters) and plan["n_real"] >= tree.n_s
    n_real = plan["n_real"]
    for t, entry in enumerate(lists):
        row = plan["steps"][plan["row_ptr"][t]:plan["row_ptr"][t + 1]]
        assert [int(v) for v in row if v < n_real] == list(entry[0])
        assert [int(v) - n_real for v in row if v >= n_real] == list(entry[1])
        ir = plan["isrc"][plan["irow"][t]:plan["irow"][t + 1]]
        assert [int(v) - n_real for v in ir] == (list(entry[2]) if interp else [])


def test_plan_rejects_bad_input():
    from paper_1709_08070_gb300 import ibim
    xs, _, _ = inputs.compact_sphere_cloud(500, radius=4.0, seed=1)
    for theta, tau, ti in ((0.0, 0.3, 0), (1.0, 0.3, 0), (0.5, -1.0, 0), (0.5, 0.3, 3)):
        with pytest.raises(ibim.IbimError) as e:
            ibim.ibim_treecode_plan(xs, theta, tau, ti)
        assert e.value.status == 1
    bad = xs.copy()
    bad[7, 1] = np.nan
    with pytest.raises(ibim.IbimError) as e:
        ibim.ibim_treecode_plan(bad, 0.5, 0.3, 0)
    assert e.value.status == 3


@pytest.mark.parametrize("n", [1, 100, 256, 257, 511, 513, 1500, 2049])
def test_plan_on_tiny_and_ragged_sizes(n):
    """One node, one partial tile, tile boundaries +-1 and a split right above
    2048: lists equal the oracle's and every source tile is covered once."""
    from paper_1709_08070_gb300 import ibim
    xs, _, _ = inputs.compact_sphere_cloud(n, radius=3.0 + n / 300.0, seed=n)
    plan = ibim.ibim_treecode_plan(xs, 0.7, 0.3, 1)
    tree = tc.TileTree(xs)
    lists = tree.lists(0.7, 0.3, True)
    n_real = plan["n_real"]
    assert plan["n_t"] == tree.n_t == -(-n // 512) and plan["clusters"] == len(tree.clusters)
    for t, (near, far, fint) in enumerate(lists):
        row = plan["steps"][plan["row_ptr"][t]:plan["row_ptr"][t + 1]]
        assert [int(v) for v in row if v < n_real] == list(near)
        assert [int(v) - n_real for v in row if v >= n_real] == list(far)
        assert [int(v) - n_real for v in plan["isrc"][plan["irow"][t]:plan["irow"][t + 1]]] == list(fint)
        covered = list(near)
        for ci in list(far) + list(fint):
            c = tree.clusters[ci]
            covered += list(range(c.j0 // 256, -(-c.j1 // 256)))
        assert sorted(covered) == list(range(-(-n // 256)))
