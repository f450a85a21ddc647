"""Logarithmic potential (Sec. 3.3): Phi_i = sum_{j: z_j != z_i} Gamma_j ln|z_i - z_j|,
GPU library vs the oracle, through the C ABI.

Bar: the FP64 path within 1e-10 (relative max-norm) of the oracle's log-series
FMM on the same tree, lists and order (the same truncation: only rounding
differs); the FP32 path within 1e-5 of the exact sum at p = 17, theta = 0.5, as
for the harmonic kernel."""
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
    if kind == "dup":  # coincident points: their mutual terms are skipped
        xy = W.uniform(n, g)
        xy[n // 2:] = xy[: n - n // 2]
        return xy
    if kind == "origin":  # a point at the origin, where the padding slots of the P2P layout sit
        xy = W.uniform(n, g)
        xy[n // 3] = (0.0, 0.0)
        return xy
    raise ValueError(kind)


def _tree(xy, L, p=17, theta=0.5, path="fp64"):
    from paper_1311_1006_b300 import Tree

    return Tree.build(_dev(xy), p=p, theta=theta, nlevels=L, path=path)


@pytest.mark.parametrize("kind,n,L,p", [("uniform", 1000, 4, 17), ("cluster", 5000, 5, 17), ("dup", 640, 4, 17),
                                        ("origin", 3001, 5, 17), ("uniform", 5, 2, 17), ("uniform", 1, 1, 17),
                                        ("cluster", 20000, 7, 8), ("cluster", 20000, 7, 13),
                                        ("uniform", 4096, 6, 32)])
def test_log_fp64_matches_oracle_fmm(orc, kind, n, L, p):
    xy = _points(kind, n, seed=7 * n + L)
    gam = W.complex_strengths(n, np.random.default_rng(n + p))
    t = _tree(xy, L, p=p)
    phi = t.eval_log(_dev(gam)).cpu().numpy()
    ref = orc.fmm_log(xy, gam, L, 0.5, p)
    if n == 1:
        assert np.all(phi == 0) and np.all(ref == 0)
    else:
        assert _rel(phi, ref) <= 1e-10, _rel(phi, ref)
    t.close()


@pytest.mark.parametrize("kind,n,L", [("cluster", 20000, 7), ("dup", 4000, 5), ("origin", 3001, 5)])
def test_log_fp32_matches_direct_sum(orc, kind, n, L):
    xy = _points(kind, n, seed=11 * n + L)
    gam = W.complex_strengths(n, np.random.default_rng(n))
    t = _tree(xy, L, p=17, path="fp32")
    phi = t.eval_log(_dev(gam)).cpu().numpy().astype(np.complex128)
    exact = orc.direct_log(xy, gam)
    assert _rel(phi, exact) <= 1e-5
    # and against the oracle's FMM with the same truncation
    assert _rel(phi, orc.fmm_log(xy, gam, L, 0.5, 17)) <= 1e-5
    t.close()


def test_log_fp64_truncation_within_table_4_1(orc):
    """p = 17, theta = 0.5 holds the harmonic kernel to about 1e-6 (Table 4.1); the
    log series, one power of the distance ratio faster, stays inside that."""
    xy = _points("cluster", 20000, 3)
    gam = W.complex_strengths(20000, np.random.default_rng(3))
    t = _tree(xy, 7, p=17)
    assert _rel(t.eval_log(_dev(gam)).cpu().numpy(), orc.direct_log(xy, gam)) <= 1e-6
    t.close()


def test_log_real_strengths_give_real_potential(orc):
    """Real Gamma: the imaginary part of the result is exactly zero (the two
    strength sets never mix)."""
    xy = _points("cluster", 5000, 4)
    gam = W.real_strengths(5000, np.random.default_rng(4)).astype(np.complex128)
    for path in ("fp64", "fp32"):
        t = _tree(xy, 5, path=path)
        phi = t.eval_log(_dev(gam)).cpu().numpy()
        assert np.all(phi.imag == 0)
        assert _rel(phi.astype(np.complex128), orc.direct_log(xy, gam)) <= (1e-6 if path == "fp64" else 1e-5)
        t.close()


def test_log_and_harmonic_share_a_tree():
    """eval_log grows the workspace to two strength sets; the harmonic eval on
    the same tree afterwards gives the same bits as before."""
    xy = _points("cluster", 8000, 5)
    gam = _dev(W.complex_strengths(8000, np.random.default_rng(5)))
    for path in ("fp64", "fp32"):
        t = _tree(xy, 6, path=path)
        a = t.eval(gam).cpu().numpy()
        t.eval_log(gam)
        b = t.eval(gam).cpu().numpy()
        assert np.array_equal(a, b)
        t.close()


def test_log_at_separate_evaluation_points(orc):
    """fmm_eval_targets_log: the union tree with zero-strength evaluation points."""
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(31)
    src = W.cluster_mix(12000, g)
    gam = W.complex_strengths(12000, g)
    tgt = np.concatenate([g.random((6000, 2)), src[:100], np.array([[1.5, -0.3], [0.5, 1.25]])])
    allxy = np.concatenate([src, tgt])
    allg = np.concatenate([gam, np.zeros(len(tgt), np.complex128)])
    ref = orc.direct_log(allxy, allg, targets=np.arange(len(src), len(allxy)))
    for path, tol in (("fp64", 1e-6), ("fp32", 1e-5)):
        t = Tree.build_targets(_dev(src), _dev(tgt), p=17, theta=0.5, path=path)
        phi = t.eval_targets_log(_dev(gam)).cpu().numpy().astype(np.complex128)
        assert _rel(phi, ref) <= tol, (path, _rel(phi, ref))
        if path == "fp64":
            L = t.info()["nlevels_max"]
            assert _rel(phi, orc.fmm_log(allxy, allg, L, 0.5, 17)[len(src):]) <= 1e-10
        t.close()


@pytest.mark.slow
def test_log_headline_workload_sampled(orc):
    """1e6-point Gaussian mixture in the benchmark's launch configuration:
    2048 sampled outputs against the exact logarithmic sum."""
    from paper_1311_1006_b300 import Tree

    g = W.rng(W.W_CLUSTER_1M)
    n = 1_000_000
    xy = W.cluster_mix(n, g)
    gam = W.complex_strengths(n, g)
    X, G = _dev(xy), _dev(gam)
    tg = np.random.default_rng(2).choice(n, 2048, replace=False)
    exact = orc.direct_log(xy, gam, targets=tg)
    for path, tol in (("fp32", 1e-5), ("fp64", 1e-7)):
        t = Tree.build(X, p=17, nlevels=9, path=path)
        phi = t.eval_log(G).cpu().numpy().astype(np.complex128)
        err = _rel(phi[tg], exact)
        assert err < tol, (path, err)
        t.close()


def test_log_batched_forest_equals_standalone(orc):
    """fmm_eval_log on a forest of instances: each instance equals its own tree's
    evaluation and the oracle's log-series FMM."""
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(41)
    sizes = [700, 3000, 1, 12000, 2500]
    pts = [W.batch_instance(m, g) for m in sizes]
    gam = np.concatenate([W.complex_strengths(m, g) for m in sizes])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xy = np.vstack(pts)
    t = Tree.build_batched(_dev(xy), offs, p=16, path="fp64")
    phi = t.eval_log(_dev(gam)).cpu().numpy()
    lev = t.export("inst")[:, 2]
    for b, m in enumerate(sizes):
        s, e = offs[b], offs[b + 1]
        tb = Tree.build(_dev(xy[s:e]), p=16, nlevels=int(lev[b]), path="fp64")
        ref = tb.eval_log(_dev(gam[s:e])).cpu().numpy()
        tb.close()
        if m == 1:
            assert np.all(phi[s:e] == 0) and np.all(ref == 0)
            continue
        assert np.abs(phi[s:e] - ref).max() <= 1e-12 * np.abs(ref).max()
        ro = orc.fmm_log(xy[s:e], gam[s:e], int(lev[b]), 0.5, 16)
        assert _rel(phi[s:e], ro) <= 1e-10
    t.close()
