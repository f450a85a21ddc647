"""Persistent evaluation (FMM_FLAG_PERSISTENT): the whole evaluation of a tree
or of a forest of uneven instances in one launch over a device work queue.
Every instance against the oracle, the result against the per-phase launches
(same passes; M2L on the CUDA cores instead of the tensor cores), bit-for-bit
repeatability, the captured-graph replay, and the status of the queue waits."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _forest(seed, B, lo, hi):
    g = np.random.default_rng(seed)
    sizes = np.floor(10 ** g.uniform(np.log10(lo), np.log10(hi), size=B)).astype(np.int64)
    pts = [W.batch_instance(int(n), g) for n in sizes]
    gam = [W.real_strengths(int(n), g) for n in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return np.vstack(pts), np.concatenate(gam), offs, sizes


def test_persistent_forest_matches_oracle_and_per_phase(orc):
    import paper_1311_1006_b300 as F

    xy, gam, offs, sizes = _forest(11, 20, 300, 6000)
    levels = [max(1, min(W.leaf_levels(int(n), 20), 6)) for n in sizes]
    levels[2] = 1  # a one-level instance inside the forest
    X, G = _dev(xy), _dev(gam)
    ref_t = F.Tree.build_batched(X, offs, nlevels=levels, p=16, path="fp32")
    ref = ref_t.eval(G).cpu().numpy().astype(np.complex128)
    t = F.Tree.build_batched(X, offs, nlevels=levels, p=16, path="fp32", flags=F.FMM_FLAG_PERSISTENT)
    phi = t.eval(G).cpu().numpy().astype(np.complex128)
    t.eval_status()
    again = t.eval(G).cpu().numpy().astype(np.complex128)
    assert np.array_equal(phi, again)  # the queue order does not change any sum
    for b in range(len(sizes)):
        s, e = offs[b], offs[b + 1]
        o = orc.fmm(xy[s:e], gam[s:e], levels[b], 0.5, 16)["phi"]
        assert _rel(phi[s:e], o) < 1e-5, (b, sizes[b], levels[b])
        assert _rel(phi[s:e], ref[s:e]) < 1e-6, (b, sizes[b], levels[b])
    t.close()
    ref_t.close()


@pytest.mark.parametrize("p", [8, 17, 32])
def test_persistent_single_tree(orc, p):
    import paper_1311_1006_b300 as F

    g = np.random.default_rng(100 + p)
    n = 60_000
    xy, gam = W.cluster_mix(n, g), W.complex_strengths(n, g)
    X, G = _dev(xy), _dev(gam)
    t = F.Tree.build(X, p=p, nlevels=0, path="fp32", flags=F.FMM_FLAG_PERSISTENT)
    L = t.info()["nlevels_max"]
    phi = t.eval(G).cpu().numpy().astype(np.complex128)
    t.eval_status()
    ref = F.Tree.build(X, p=p, nlevels=L, path="fp32").eval(G).cpu().numpy().astype(np.complex128)
    assert _rel(phi, ref) < 1e-6
    tg = np.random.default_rng(1).choice(n, 256, replace=False)
    tol = max(1e-5, 3.0 * 0.5 ** (p / 0.9))
    assert _rel(phi[tg], orc.direct(xy, gam, targets=tg)) < tol
    # a step (rebuild + evaluation) on moved points takes the persistent path too
    xy2 = W.cluster_mix(n, g)
    X2 = _dev(xy2)
    phi2 = t.step(X2, G).cpu().numpy().astype(np.complex128)
    ref2 = F.Tree.build(X2, p=p, nlevels=L, path="fp32").eval(G).cpu().numpy().astype(np.complex128)
    assert _rel(phi2, ref2) < 1e-6
    t.close()


def test_persistent_graph_replay_and_fp64_rejected():
    import paper_1311_1006_b300 as F
    from paper_1311_1006_b300 import _lib

    g = np.random.default_rng(5)
    xy, gam = W.uniform(20_000, g), W.complex_strengths(20_000, g)
    X, G = _dev(xy), _dev(gam)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        t = F.Tree.build(X, p=17, path="fp32", flags=F.FMM_FLAG_PERSISTENT)
        out = torch.empty(20_000, dtype=torch.complex64, device="cuda")
        t.eval(G, out=out, stream=s)
        direct = out.clone()
        t.rebuild(X, flags=F.FMM_FLAG_PERSISTENT | F.FMM_FLAG_GRAPH)
        for _ in range(3):
            out.zero_()
            t.eval(G, out=out, stream=s)
            assert torch.equal(out, direct)
    s.synchronize()
    t.close()
    with pytest.raises(_lib.FMMError):
        t64 = F.Tree.build(X, p=17, path="fp64", flags=F.FMM_FLAG_PERSISTENT)
        try:
            t64.eval(G)
        finally:
            t64.close()
