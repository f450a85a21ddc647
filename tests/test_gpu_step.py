"""fmm_step (rebuild + evaluate in one call, the upward pass overlapping the list
build) against fmm_tree_rebuild + fmm_eval on a second tree: the same kernels in
the same order per stream, so the results must agree bit for bit."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _snapshots(n, seed):
    g = np.random.default_rng(seed)
    out = [W.uniform(n, g)]
    for sigma in (0.05, 0.004):  # ever tighter clusters: longer lists, capacities grow inside the step
        c = g.uniform(0.3, 0.7, size=(2, 2))
        xy = np.concatenate([c[0] + sigma * g.normal(size=(n // 2, 2)),
                             c[1] + sigma * g.normal(size=(n - n // 2, 2))])
        out.append(np.clip(xy, 0.0, 1.0))
    return out, [W.complex_strengths(n, g) for _ in out]


@pytest.mark.parametrize("path", ["fp32", "fp64"])
def test_step_equals_rebuild_then_eval(path):
    from paper_1311_1006_b300 import Tree

    n = 30000
    xs, gs = _snapshots(n, 11)
    a = Tree.build(_dev(xs[0]), p=17, nlevels=6, path=path)  # fmm_step
    b = Tree.build(_dev(xs[0]), p=17, nlevels=6, path=path)  # rebuild + eval
    for xy, gam in zip(xs, gs):
        X, G = _dev(xy), _dev(gam)
        pa = a.step(X, G).cpu().numpy()
        b.rebuild(X)
        pb = b.eval(G).cpu().numpy()
        assert np.array_equal(pa, pb)
        assert a.info()["n_weak"] == b.info()["n_weak"]
    a.close()
    b.close()


def test_step_gradual_clustering_bit_for_bit_and_oracle(orc):
    """A slowly tightening sequence (sigma 0.2 * 0.75^k): most steps reuse the earlier capacities and run the
    evaluation queued behind the lists, some outgrow the list or the item capacities and are redone in the
    checked order.  Every step equals rebuild + eval on a second tree bit for bit; the last one is also checked
    against the oracle FMM."""
    from paper_1311_1006_b300 import Tree

    n, L = 12000, 6
    g = np.random.default_rng(21)
    c = g.uniform(0.35, 0.65, size=(3, 2))
    a = Tree.build(_dev(W.uniform(n, g)), p=12, nlevels=L, path="fp64")
    b = Tree.build(_dev(W.uniform(n, g)), p=12, nlevels=L, path="fp64")
    for k in range(14):
        sigma = 0.2 * 0.75 ** k
        xy = np.clip(np.concatenate([c[i] + sigma * g.normal(size=(n // 3 + (i < n % 3), 2)) for i in range(3)]),
                     0.0, 1.0)
        gam = W.complex_strengths(n, g)
        pa = a.step(_dev(xy), _dev(gam)).cpu().numpy()
        b.rebuild(_dev(xy))
        pb = b.eval(_dev(gam)).cpu().numpy()
        assert np.array_equal(pa, pb), k
        info_a, info_b = a.info(), b.info()
        assert info_a["n_strong"] == info_b["n_strong"] and info_a["p2p_items"] == info_b["p2p_items"], k
    ref = orc.fmm(xy, gam, L, 0.5, 12)["phi"]
    assert np.abs(pa - ref).max() <= 1e-10 * np.abs(ref).max()
    a.close()
    b.close()


def test_step_after_level_changes_equals_fresh_tree():
    """N_levels changing between steps (as the tuner does: a rebuild with another level count, then steps):
    the capacities, grids and counters of the previous shape must not leak into the queued evaluation."""
    from paper_1311_1006_b300 import Tree

    n = 20000
    g = np.random.default_rng(31)
    t = Tree.build(_dev(W.uniform(n, g)), p=12, nlevels=6, path="fp32")
    for L in (7, 5, 8, 6, 7):
        xy, gam = W.cluster_mix(n, g), W.complex_strengths(n, g)
        t.rebuild(_dev(W.uniform(n, g)), nlevels=L)  # the new shape, on other points
        for _ in range(2):
            pa = t.step(_dev(xy), _dev(gam)).cpu().numpy()
            f = Tree.build(_dev(xy), p=12, nlevels=L, path="fp32")
            assert np.array_equal(pa, f.eval(_dev(gam)).cpu().numpy()), L
            f.close()
    t.close()


def test_step_as_the_first_call_and_against_the_oracle(orc):
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(12)
    n, L = 8000, 5
    xy, gam = W.cluster_mix(n, g), W.complex_strengths(n, g)
    t = Tree.build(_dev(W.uniform(n, g)), p=17, nlevels=L, path="fp64")  # no evaluation before the step
    phi = t.step(_dev(xy), _dev(gam)).cpu().numpy()
    ref = orc.fmm(xy, gam, L, 0.5, 17)["phi"]
    assert np.abs(phi - ref).max() <= 1e-10 * np.abs(ref).max()
    t.close()


def test_step_fallbacks_and_argument_checks():
    import paper_1311_1006_b300 as F

    g = np.random.default_rng(13)
    n = 5000
    xy, gam = _dev(W.cluster_mix(n, g)), _dev(W.complex_strengths(n, g))
    ref = F.Tree.build(xy, p=12, nlevels=5, path="fp64")
    r = ref.eval(gam).cpu().numpy()
    for flags in (F.FMM_FLAG_TIMING, F.FMM_FLAG_SERIAL, F.FMM_FLAG_GRAPH):
        t = F.Tree.build(xy, p=12, nlevels=5, path="fp64", flags=flags)
        assert np.array_equal(t.step(xy, gam).cpu().numpy(), r)
        t.close()
    ref.close()
    # batched forest: the two-call sequence
    offs = np.array([0, 2000, n])
    tb = F.Tree.build_batched(xy, offs, p=12, path="fp64")
    ra = tb.eval(gam).cpu().numpy()
    assert np.array_equal(tb.step(xy, gam).cpu().numpy(), ra)
    tb.close()
    # separate evaluation points: not a plain rebuild
    tt = F.Tree.build_targets(xy[:3000], xy[3000:], p=12)
    with pytest.raises(F.FMMError):
        tt.n = 3000
        tt.step(xy[:3000], gam[:3000])
    tt.close()


def test_step_rebuilds_after_a_long_run_of_equal_keys():
    """Coordinates with many exact repeats: the first step's short sort meets a
    run it does not resolve, so fmm_step builds the tree again with the full
    sort (and launches the upward pass again); the result equals a tree built
    and evaluated by the two-call sequence."""
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(14)
    n = 20000
    xy = np.round(W.cluster_mix(n, g) * 50) / 50  # few distinct coordinates
    gam = W.complex_strengths(n, g)
    X, G = _dev(xy), _dev(gam)
    for path in ("fp32", "fp64"):
        a = Tree.build(_dev(W.uniform(n, g)), p=12, nlevels=6, path=path)
        b = Tree.build(X, p=12, nlevels=6, path=path)
        pa = a.step(X, G).cpu().numpy()
        pb = b.eval(G).cpu().numpy()
        assert np.array_equal(pa, pb)
        assert np.array_equal(a.export("perm"), b.export("perm"))
        a.close()
        b.close()
