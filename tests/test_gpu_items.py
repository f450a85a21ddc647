"""M2L work items and the row order the M2L kernels take them in.

Items: every box's weak list cut into consecutive pieces of K pairs (K = 192 on
the tensor-core FP32 path, 64 for the one-thread-per-item kernels), a box's
items consecutive, each holding the index of its box's first item when the box
has several (-1 otherwise).  Rows: a permutation of the items with every full
item first (a box's full items on consecutive rows, in item order), then the
shorter last items by non-increasing length, so that threads stepping through
their items in lockstep get about the same number of pairs.  The M2L results
themselves are checked against the oracle by the parity tests."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path,K,batched", [("fp32", 192, False), ("fp64", 64, False), ("fp32", 192, True)])
def test_m2l_items_and_row_order(path, K, batched):
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(21)
    n = 200_000
    xy = W.cluster_mix(n, g)
    X = torch.tensor(xy, device="cuda")
    if batched:  # instances of different depths: many short lists and short last items
        offs = np.array([0, 1000, 21000, 21500, 90000, n])
        t = Tree.build_batched(X, offs, p=17, path=path)
    else:
        t = Tree.build(X, p=17, nlevels=7, path=path)
    nw = t.export("nweak")
    items, rows = t.export("m2l_items"), t.export("m2l_rows")
    t.close()
    m = items.shape[0]
    assert m == int(np.sum((nw + K - 1) // K))
    # items: per box, consecutive pieces of K pairs covering its weak list
    order = np.argsort(items[:, 0], kind="stable")
    boxes, first_idx, counts = np.unique(items[order, 0], return_index=True, return_counts=True)
    assert np.all(nw[boxes] > 0) and np.all(counts == (nw[boxes] + K - 1) // K)
    for b, f, c in zip(boxes, first_idx, counts):
        idx = np.sort(order[f:f + c])
        assert np.all(np.diff(idx) == 1)  # consecutive
        q = np.arange(c)
        assert np.all(items[idx, 1] == q * K) and np.all(items[idx, 2] == np.minimum(nw[b], (q + 1) * K))
        assert np.all(items[idx, 3] == (idx[0] if c > 1 else -1))
    # rows: a permutation; full items first, then non-increasing lengths
    assert np.array_equal(np.sort(rows), np.arange(m))
    lens = items[rows, 2] - items[rows, 1]
    nfull = int(np.sum(lens == K))
    assert np.all(lens[:nfull] == K) and np.all(lens[nfull:] < K)
    assert np.all(np.diff(lens[nfull:]) <= 0)
    assert np.sum(lens) == np.sum(nw)
    # a box's full items sit on consecutive rows, in item order
    full = rows[:nfull]
    pos = np.empty(m, np.int64)
    pos[rows] = np.arange(m)
    for b, f, c in zip(boxes, first_idx, counts):
        idx = np.sort(order[f:f + c])
        fi = idx[items[idx, 2] - items[idx, 1] == K]
        if fi.size > 1:
            assert np.all(np.diff(pos[fi]) == 1)
    assert full.size == nfull


@pytest.mark.parametrize("batched", [False, True])
def test_p2p_items_and_row_order(batched):
    """P2P items: each leaf's strong list cut into consecutive pieces (a leaf's
    items consecutive, each holding the leaf's first item when it has several).
    Rows: a permutation of the items with the full items of split leaves first
    and every leaf's last (or only) item after them."""
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(22)
    n = 300_000
    xy = W.cluster_mix(n, g)
    X = torch.tensor(xy, device="cuda")
    if batched:
        offs = np.array([0, 5000, 150000, 151000, n])
        t = Tree.build_batched(X, offs, p=17, path="fp32")
    else:
        t = Tree.build(X, p=17, nlevels=9, path="fp32")
    ns = t.export("nstrong")
    items, rows = t.export("p2p_items"), t.export("p2p_rows")
    t.close()
    m = items.shape[0]
    assert np.array_equal(np.sort(rows), np.arange(m))
    # every leaf's strong list is covered once, in consecutive pieces
    order = np.argsort(items[:, 0], kind="stable")
    leaves, first_idx, counts = np.unique(items[order, 0], return_index=True, return_counts=True)
    assert np.all(ns[leaves] > 0)
    last = np.zeros(m, bool)
    for b, f, c in zip(leaves, first_idx, counts):
        idx = np.sort(order[f:f + c])
        assert np.all(np.diff(idx) == 1)
        assert items[idx[0], 1] == 0 and items[idx[-1], 2] == ns[b]
        assert np.all(items[idx[1:], 1] == items[idx[:-1], 2])
        assert np.all(items[idx, 3] == (idx[0] if c > 1 else -1))
        last[idx[-1]] = True
    nheavy = int(np.sum(~last))
    assert np.all(~last[rows[:nheavy]]) and np.all(last[rows[nheavy:]])
    if not batched:
        assert nheavy > 0  # the clustered set has leaves whose strong lists are split
