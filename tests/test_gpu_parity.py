"""GPU path vs the oracle, element by element, through the C ABI.

Bar: the tree (permutation, box ranges, centres, radii) and the coupling lists
are integer / bit exact; the FP64 path is within 1e-10 (relative max-norm) of
the oracle FMM and the FP32 path within 1e-5, both for the whole result and for
the far field alone; per-pass arrays (multipoles, locals, near field) agree
within tolerances derived from the arithmetic (see the design notes)."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _points(kind, n, seed):
    g = np.random.default_rng(seed)
    if kind == "uniform":
        return W.uniform(n, g)
    if kind == "cluster":
        return W.cluster_mix(n, g)
    if kind == "ties":  # many equal coordinates: the input index breaks ties
        return np.round(W.uniform(n, g) * 13) / 13
    if kind == "line":
        s = g.random(n)
        return np.stack([s, 0.5 + 0.3 * s + 1e-3 * g.normal(size=n)], 1)
    if kind == "dup":  # coincident points
        xy = W.uniform(n, g)
        xy[n // 2:] = xy[: n - n // 2]
        return xy
    if kind == "far":  # small clustered set far from the origin: FP32 coordinates must be taken relative to it
        return 1e4 + 1e-2 * W.cluster_mix(n, g)
    if kind == "neg":  # negative and positive coordinates, a wider box than the unit square
        return 4.0 * W.cluster_mix(n, g) - 3.0
    raise ValueError(kind)


def _tree(xy, L, p=17, theta=0.5, path="fp64"):
    from paper_1311_1006_b300 import Tree

    return Tree.build(_dev(xy), p=p, theta=theta, nlevels=L, path=path)


# ---------------------------------------------------------------- tree, lists

@pytest.mark.parametrize("kind,n,L", [("uniform", 1000, 4), ("cluster", 5000, 5), ("ties", 777, 4),
                                      ("line", 3001, 5), ("dup", 640, 4), ("uniform", 1, 1), ("uniform", 5, 2),
                                      ("cluster", 20000, 7), ("uniform", 4096, 7), ("far", 3000, 5), ("neg", 3000, 5),
                                      ("cluster", 300000, 8)])
def test_tree_bit_exact(orc, kind, n, L):
    xy = _points(kind, n, seed=n + L)
    t = _tree(xy, L)
    ref = orc.build_tree(xy, L)
    assert np.array_equal(t.export("perm"), ref["perm"])
    assert np.array_equal(t.export("bstart"), ref["bstart"])
    assert np.array_equal(t.export("bcount"), ref["bcount"])
    assert np.array_equal(t.export("center"), ref["center"])
    assert np.array_equal(t.export("radius"), ref["radius"])


@pytest.mark.parametrize("kind,n,L,theta", [("uniform", 1000, 4, 0.5), ("cluster", 5000, 5, 0.5),
                                            ("line", 3001, 5, 0.35), ("ties", 2000, 5, 0.65),
                                            ("dup", 640, 4, 0.5), ("cluster", 40000, 7, 0.5)])
def test_lists_exact(orc, kind, n, L, theta):
    xy = _points(kind, n, seed=n)
    t = _tree(xy, L, theta=theta)
    ref = orc.build_tree(xy, L)
    li = orc.build_lists(L, ref["center"], ref["radius"], theta)
    strong, weak = t.lists()
    for b in range(orc.num_boxes(L)):
        assert np.array_equal(np.sort(strong[b]), li["s_idx"][li["s_off"][b]: li["s_off"][b + 1]]), b
        assert np.array_equal(np.sort(weak[b]), li["w_idx"][li["w_off"][b]: li["w_off"][b + 1]]), b
    info = t.info()
    assert info["n_weak"] == li["w_off"][-1]


# ------------------------------------------------------------ per-pass arrays

@pytest.mark.parametrize("path,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
def test_expansions_match_oracle(orc, path, tol):
    g = np.random.default_rng(3)
    n, L, p = 6000, 5, 17
    xy = W.cluster_mix(n, g)
    gam = W.complex_strengths(n, g)
    t = _tree(xy, L, p=p, path=path)
    t.eval(_dev(gam))
    torch.cuda.synchronize()
    ref = orc.fmm(xy, gam, L, 0.5, p, parts=True)
    rho = t.export("rho")
    k = np.arange(p)
    # scaled coefficients: a_k / rho^k and b_l rho^l; |a_k/rho^k| <= sum |Gamma| of the box
    with np.errstate(divide="ignore", invalid="ignore"):
        mref = np.where(rho[:, None] > 0, ref["mpole"] / rho[:, None] ** k, ref["mpole"] * (k == 0))
    lref = ref["local"] * rho[:, None] ** k
    mp, lo = t.export("mpole"), t.export("local")
    scale_m = np.abs(mref).max(axis=1, keepdims=True) + 1e-300
    assert np.max(np.abs(mp - mref) / scale_m) < tol * 50
    scale_l = np.abs(lref).max(axis=1, keepdims=True) + 1e-300
    mask = np.abs(lref).max(axis=1) > 0
    assert np.max((np.abs(lo - lref) / scale_l)[mask]) < tol * 50
    near = t.export("near")
    perm = t.export("perm")
    assert _rel(near, ref["near"][perm]) < tol * 10


# --------------------------------------------------------------- end to end

def _check_eval(orc, xy, gam, L, p, theta, path):
    t = _tree(xy, L, p=p, theta=theta, path=path)
    phi = t.eval(_dev(gam)).cpu().numpy().astype(np.complex128)
    near = t.export("near")[np.argsort(t.export("perm"))]
    ref = orc.fmm(xy, gam, L, theta, p, parts=True)
    return _rel(phi, ref["phi"]), _rel(phi - near, ref["far"]) if np.abs(ref["far"]).max() > 0 else 0.0


@pytest.mark.parametrize("kind,n,L,p,theta", [
    ("uniform", 10_000, 5, 20, 0.5),   # plain FP64 workload (35 points per leaf)
    ("cluster", 8000, 5, 17, 0.5),
    ("line", 5000, 5, 12, 0.35),
    ("ties", 3000, 4, 30, 0.65),
    ("dup", 2000, 4, 17, 0.5),
    ("uniform", 5000, 5, 5, 0.5),
    ("uniform", 777, 1, 17, 0.5),      # one level: pure direct sum
    ("uniform", 3, 1, 4, 0.5),
    ("uniform", 4096, 7, 32, 0.5),     # one point per leaf, largest order
    ("cluster", 3001, 5, 1, 0.5),      # p = 1
    ("cluster", 16000, 6, 17, 0.5),    # <= 16 points per leaf: the leaves' parents by a thread per box
    ("far", 6000, 5, 17, 0.5),
    ("neg", 6000, 5, 17, 0.5),
])
@pytest.mark.parametrize("path,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_eval_matches_oracle(orc, kind, n, L, p, theta, path, tol):
    g = np.random.default_rng(n + p)
    xy = _points(kind, n, seed=n)
    gam = W.complex_strengths(n, g)
    err, ferr = _check_eval(orc, xy, gam, L, p, theta, path)
    assert err < tol, (err, ferr)
    assert ferr < tol * (10 if path == "fp32" else 1), (err, ferr)


@pytest.mark.parametrize("kind,n,L", [("uniform", 10_000, 5), ("cluster", 16000, 6), ("dup", 2000, 4),
                                      ("far", 6000, 5), ("uniform", 777, 1)])
@pytest.mark.parametrize("one_complex", [False, True])
def test_fp32_real_strengths(orc, kind, n, L, one_complex):
    """Real strengths take the FP32 P2P's real form (the gather finds no
    nonzero imaginary part); one complex strength among them switches the whole
    evaluation back to the complex form.  Both within 1e-5 of the oracle, the
    near field alone too."""
    g = np.random.default_rng(n + 7)
    xy = _points(kind, n, seed=n + 1)
    gam = W.real_strengths(n, g)
    if one_complex:
        gam[n // 3] += 0.5j
    t = _tree(xy, L, p=17, path="fp32")
    phi = t.eval(_dev(gam)).cpu().numpy().astype(np.complex128)
    near = t.export("near")[np.argsort(t.export("perm"))]
    ref = orc.fmm(xy, gam, L, 0.5, 17, parts=True)
    assert _rel(phi, ref["phi"]) < 1e-5
    assert _rel(near, ref["near"]) < 1e-5


def test_eval_single_point_is_zero():
    from paper_1311_1006_b300 import Tree

    for path in ("fp32", "fp64"):
        t = Tree.build(_dev(np.array([[0.3, 0.7]])), nlevels=1, path=path)
        phi = t.eval(_dev(np.array([2.0 + 1j])))
        assert torch.all(phi == 0)


def test_eval_is_deterministic_and_graph_replay_matches_eager(orc):
    from paper_1311_1006_b300 import FMM_FLAG_GRAPH, FMM_FLAG_NO_GRAPH, Tree

    g = np.random.default_rng(5)
    xy, gam = W.cluster_mix(20000, g), W.complex_strengths(20000, g)
    X, G = _dev(xy), _dev(gam)
    for path in ("fp32", "fp64"):
        t1 = Tree.build(X, nlevels=6, path=path, flags=FMM_FLAG_GRAPH)
        t2 = Tree.build(X, nlevels=6, path=path, flags=FMM_FLAG_NO_GRAPH)
        a = t1.eval(G).clone()
        b = t1.eval(G).clone()
        c = t2.eval(G)
        torch.cuda.synchronize()
        assert torch.equal(a, b) and torch.equal(a, c)


def test_coordinate_sort_runs_and_fallback(orc):
    """The short coordinate sort (high key halves, then the runs of equal high
    halves in place) and its fallback (a run longer than it resolves: the tree
    is rebuilt with the full sort): trees equal the oracle's in both directions."""
    xs = [_points("cluster", 50000, 3), _points("ties", 50000, 4), _points("cluster", 50000, 5)]
    t = _tree(xs[0], 7)
    for xy in xs:
        t.rebuild(_dev(xy))
        ref = orc.build_tree(xy, 7)
        assert np.array_equal(t.export("perm"), ref["perm"])
        assert np.array_equal(t.export("bstart"), ref["bstart"])
        assert np.array_equal(t.export("center"), ref["center"])
    t.close()


def test_rebuild_changes_levels_and_points(orc):
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(6)
    xy1, xy2, gam = W.uniform(5000, g), W.cluster_mix(5000, g), W.complex_strengths(5000, g)
    t = Tree.build(_dev(xy1), nlevels=4, path="fp64")
    G = _dev(gam)
    for xy, L in ((xy2, 5), (xy1, 3), (xy2, 4)):
        t.rebuild(_dev(xy), nlevels=L)
        phi = t.eval(G).cpu().numpy()
        assert _rel(phi, orc.fmm(xy, gam, L, 0.5, 17)["phi"]) < 1e-10


def test_nonfinite_coordinates_rejected():
    from paper_1311_1006_b300 import FMMError, Tree

    xy = W.uniform(100, np.random.default_rng(0))
    xy[17, 1] = np.nan
    with pytest.raises(FMMError) as e:
        Tree.build(_dev(xy), nlevels=3)
    assert e.value.status == 5
    xy[17, 1] = np.inf
    with pytest.raises(FMMError):
        Tree.build(_dev(xy), nlevels=3)


def test_too_many_levels_rejected():
    from paper_1311_1006_b300 import FMMError, Tree

    with pytest.raises(FMMError) as e:
        Tree.build(_dev(W.uniform(10, np.random.default_rng(0))), nlevels=4)
    assert e.value.status == 1


def test_list_capacity_overflow_is_retried(orc):
    # points on a tight line make long strong lists; the library grows its
    # list capacity and rebuilds the lists transparently
    g = np.random.default_rng(9)
    n = 20000
    s = np.sort(g.random(n))
    xy = np.stack([s, 0.5 + 1e-9 * g.normal(size=n)], 1)
    gam = W.real_strengths(n, g)
    t = _tree(xy, 7, path="fp64")
    ref = orc.fmm(xy, gam, 7, 0.5, 17)["phi"]
    assert _rel(t.eval(_dev(gam)).cpu().numpy(), ref) < 1e-10


# ----------------------------------------------------------- full-size checks

@pytest.mark.slow
def test_headline_workload_sampled(orc):
    """1e6-point Gaussian mixture (the headline workload), FP32 and FP64 paths,
    in the launch configuration the benchmark uses: tree bit-exact against the
    oracle and outputs on 2048 sampled points against the exact direct sum."""
    from paper_1311_1006_b300 import Tree

    g = W.rng(W.W_CLUSTER_1M)
    n = 1_000_000
    xy = W.cluster_mix(n, g)
    gam = W.complex_strengths(n, g)
    X, G = _dev(xy), _dev(gam)
    L = 9
    ref_tree = orc.build_tree(xy, L)
    tg = np.random.default_rng(1).choice(n, 2048, replace=False)
    exact = orc.direct(xy, gam, targets=tg)
    for path, tol in (("fp32", 1e-5), ("fp64", 1e-10)):
        t = Tree.build(X, p=17, nlevels=L, path=path)
        if path == "fp32":
            assert np.array_equal(t.export("perm"), ref_tree["perm"])
            assert np.array_equal(t.export("center"), ref_tree["center"])
            assert np.array_equal(t.export("radius"), ref_tree["radius"])
        phi = t.eval(G).cpu().numpy().astype(np.complex128)
        err = _rel(phi[tg], exact)
        assert err < (1e-5 if path == "fp32" else 1e-7), (path, err)
        t.close()
