"""The autotuners on real timings (Sec. 4.2, Algorithm 4 "AT3b", and the theta
moves of Algorithms 2-4), on a 2e5-point cluster set: the cost-model seed
(eqs 2.4-2.5) from unit costs measured on the GPU, the N_levels the AT3b walk
accepts against an exhaustive sweep, and the accuracy of the tuned (theta, p)
against the oracle's exact sum."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 200_000
P = 17


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


@pytest.fixture(scope="module")
def data():
    g = np.random.default_rng(77)
    xy = W.cluster_mix(N, g)
    gam = W.complex_strengths(N, g)
    return xy, gam, _dev(xy), _dev(gam)


@pytest.fixture
def keep_cost_model():
    import paper_1311_1006_b300 as F

    saved = F.cost_model("fp32")
    yield
    F.set_cost_model(*saved, "fp32")


def _step_ms(tree, X, G, out, reps, **kw):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        e0.record()
        tree.rebuild(X, **kw)
        tree.eval(G, out=out)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def test_calibrated_seed_and_at3b_against_an_exhaustive_sweep(data, keep_cost_model):
    import paper_1311_1006_b300 as F

    xy, gam, X, G = data
    t = F.Tree.build(X, p=P, theta=0.5, nlevels=0, path="fp32",
                     flags=F.FMM_FLAG_TIMING | F.FMM_FLAG_SERIAL)
    out = torch.empty(N, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        t.eval(G, out=out)
    alpha, beta = t.calibrate_cost_model()
    assert alpha > 0 and beta > 0
    assert F.cost_model("fp32") == (alpha, beta)
    seed = F.default_nlevels(N, P, "fp32")
    assert seed == F.seed_nlevels(N, P, alpha, beta)
    # the seed moves with p under the measured unit costs
    assert F.seed_nlevels(N, 30, alpha, beta) <= F.seed_nlevels(N, 12, alpha, beta)
    # exhaustive sweep: median of 7 rebuild + evaluate steps per level
    t.rebuild(X, flags=0)
    lmax = int(np.floor(np.log(N) / np.log(4))) + 1
    levels = [L for L in range(max(2, seed - 2), min(lmax, seed + 2) + 1)]
    sweep = {}
    for L in levels:
        _step_ms(t, X, G, out, 2, nlevels=L)
        sweep[L] = float(np.median(_step_ms(t, X, G, out, 7, nlevels=L)))
    best = min(sweep, key=sweep.get)
    assert abs(seed - best) <= 1, (seed, sweep)
    # AT3b from the seed
    t.autotune_config(cap=0.2, window=3, period=3)
    L = seed
    t.rebuild(X, nlevels=L)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(60):
        e0.record()
        t.rebuild(X, nlevels=L)
        t.eval(G, out=out)
        e1.record()
        e1.synchronize()
        L = t.autotune_step(e0.elapsed_time(e1) * 1e-3)
    accepted = int(t.info()["autotune_nlevels"])
    assert abs(accepted - best) <= 1, (accepted, sweep)
    t.close()


def test_theta_walk_meets_the_tolerance(data, orc):
    import paper_1311_1006_b300 as F

    xy, gam, X, G = data
    tol = 1e-6
    th = 0.5
    pp = F.p_for_tolerance(tol, th)
    L = F.default_nlevels(N, pp, "fp32")
    t = F.Tree.build(X, p=pp, theta=th, nlevels=L, path="fp32")
    out = torch.empty(N, dtype=torch.complex64, device="cuda")
    t.eval(G, out=out)
    t.autotune_config(cap=0.2, window=3, period=3)
    t.autotune_theta(tol, 0.35, 0.65)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    seen = set()
    for _ in range(80):
        e0.record()
        t.rebuild(X, nlevels=L, theta=th, p=pp)
        t.eval(G, out=out)
        e1.record()
        e1.synchronize()
        seen.add(round(th, 4))
        L, th, pp = t.autotune_params(e0.elapsed_time(e1) * 1e-3)
        assert 0.35 - 1e-9 <= th <= 0.65 + 1e-9 and pp == F.p_for_tolerance(tol, th)
    assert len(seen) > 1  # theta moves were tried
    info = t.info()
    L, th = int(info["autotune_nlevels"]), float(info["autotune_theta"])
    pp = F.p_for_tolerance(tol, th)
    t.rebuild(X, nlevels=L, theta=th, p=pp)
    phi = t.eval(G).cpu().numpy().astype(np.complex128)
    tg = np.random.default_rng(78).choice(N, 256, replace=False)
    exact = orc.direct(xy, gam, targets=tg)
    err = float(np.abs(phi[tg] - exact).max() / np.abs(exact).max())
    assert err <= tol, (th, pp, L, err)
    t.close()
