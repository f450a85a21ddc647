"""Slowly tightening point sequences through every evaluation mode.  A tree carried across the sequence (its
list and item capacities, launch grids, captured graphs and persistent stage tables follow the growing lists)
against a tree built fresh for every snapshot: the same kernels on the same lists, so the results agree bit
for bit.  The last snapshot is also checked against the oracle."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L, P, K = 9000, 6, 12, 9


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _sequence(n, seed):
    """Snapshots of three Gaussian clusters with sigma = 0.2 * 0.72^k (clipped to the unit square)."""
    g = np.random.default_rng(seed)
    c = g.uniform(0.35, 0.65, size=(3, 2))
    out = []
    for k in range(K):
        sigma = 0.2 * 0.72 ** k
        xy = np.concatenate([c[i] + sigma * g.normal(size=(n // 3 + (i < n % 3), 2)) for i in range(3)])
        out.append((np.clip(xy, 0.0, 1.0), W.complex_strengths(n, g)))
    return out


@pytest.mark.parametrize("mode", ["plain", "graph", "persistent", "log", "backward"])
def test_carried_tree_equals_fresh_tree(orc, mode):
    import paper_1311_1006_b300 as F

    flags = {"graph": F.FMM_FLAG_GRAPH, "persistent": F.FMM_FLAG_PERSISTENT}.get(mode, 0)
    seq = _sequence(N, 41)
    st = torch.cuda.Stream()  # captured graphs need a stream other than the legacy default one
    with torch.cuda.stream(st):
        carried = F.Tree.build(_dev(W.uniform(N, np.random.default_rng(5))), p=P, nlevels=L, path="fp32",
                               flags=flags)
        for k, (xy, gam) in enumerate(seq):
            X, G = _dev(xy), _dev(gam)
            carried.rebuild(X)
            fresh = F.Tree.build(X, p=P, nlevels=L, path="fp32", flags=flags)
            if mode == "log":
                a, b = carried.eval_log(G), fresh.eval_log(G)
            elif mode == "backward":
                gphi = _dev(W.complex_strengths(N, np.random.default_rng(100 + k)))
                (ga, xa), (gb, xb) = carried.backward(G, gphi), fresh.backward(G, gphi)
                assert torch.equal(ga, gb) and torch.equal(xa, xb), k
                fresh.close()
                continue
            else:
                a, b = carried.eval(G), fresh.eval(G)
            assert torch.equal(a, b), k
            fresh.close()
        st.synchronize()
        if mode in ("plain", "graph", "persistent"):
            ref = orc.fmm(xy, gam, L, 0.5, P)["phi"]
            assert _rel(a.cpu().numpy().astype(np.complex128), ref) <= 1e-5
        elif mode == "log":
            ref = orc.fmm_log(xy, gam, L, 0.5, P)
            assert _rel(a.cpu().numpy().astype(np.complex128), ref) <= 1e-5
        carried.close()


def test_carried_targets_tree_equals_fresh():
    import paper_1311_1006_b300 as F

    seq = _sequence(N, 43)
    g = np.random.default_rng(7)
    tgt = _dev(g.uniform(0.0, 1.0, size=(4000, 2)))
    carried = F.Tree.build_targets(_dev(W.uniform(N, g)), tgt, p=P, nlevels=L, path="fp32")
    for k, (xy, gam) in enumerate(seq):
        X, G = _dev(xy), _dev(gam)
        carried.rebuild_targets(X, tgt)
        fresh = F.Tree.build_targets(X, tgt, p=P, nlevels=L, path="fp32")
        assert torch.equal(carried.eval_targets(G), fresh.eval_targets(G)), k
        fresh.close()
    carried.close()


def test_carried_forest_equals_fresh():
    import paper_1311_1006_b300 as F

    sizes = np.array([3000, 700, 5300, 1200], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    n = int(offs[-1])
    seq = _sequence(n, 47)
    carried = F.Tree.build_batched(_dev(W.uniform(n, np.random.default_rng(9))), offs, p=P, path="fp32")
    for k, (xy, gam) in enumerate(seq):
        X, G = _dev(xy), _dev(gam)
        carried.rebuild(X)
        fresh = F.Tree.build_batched(X, offs, p=P, path="fp32")
        assert torch.equal(carried.eval(G), fresh.eval(G)), k
        fresh.close()
    carried.close()
