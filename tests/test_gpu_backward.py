"""Adjoint (fmm_eval_backward) vs the oracle: the FMM gradient with the tree
frozen (fo_fmm_grad), the exact direct-sum gradient, central differences of the
GPU forward, and torch.autograd through FMMFunction."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("kind,n,L,p", [("uniform", 6000, 5, 20), ("cluster", 8000, 5, 17), ("dup", 3000, 4, 12),
                                        ("uniform", 500, 1, 8), ("uniform", 4096, 7, 17)])
@pytest.mark.parametrize("path,tol", [("fp64", 1e-10), ("fp32", 2e-5)])
def test_backward_matches_oracle_fmm_gradient(orc, kind, n, L, p, path, tol):
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(n)
    if kind == "uniform":
        xy = W.uniform(n, g)
    elif kind == "cluster":
        xy = W.cluster_mix(n, g)
    else:
        xy = W.uniform(n, g)
        xy[n // 2:] = xy[: n - n // 2]
    gam = W.complex_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    t = Tree.build(_dev(xy), p=p, nlevels=L, path=path)
    gg, gxy = t.backward(_dev(gam), _dev(gphi))
    rg, rxy = orc.fmm_grad(xy, gam, gphi, L, 0.5, p)
    assert _rel(gg.cpu().numpy(), rg) < tol
    assert _rel(gxy.cpu().numpy(), rxy) < tol


def test_backward_matches_direct_gradient(orc):
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(2)
    n = 20000
    xy, gam = W.uniform(n, g), W.real_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    tg = np.random.default_rng(3).choice(n, 512, replace=False)
    rg, rxy = orc.direct_grad(xy, gam, gphi, targets=tg)
    for path, tol in (("fp64", 1e-7), ("fp32", 1e-5)):
        t = Tree.build(_dev(xy), p=17, nlevels=6, path=path)
        gg, gxy = t.backward(_dev(gam), _dev(gphi))
        assert _rel(gg.cpu().numpy()[tg], rg) < tol
        assert _rel(gxy.cpu().numpy()[tg], rxy) < tol


def test_backward_matches_central_differences_of_the_gpu_forward():
    # FD of L = sum Re(conj(gphi) Phi) through the GPU FP64 path, tree rebuilt
    # at each perturbed position (same ranks, so the same boxes and lists).
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(4)
    n = 3000
    xy, gam = W.uniform(n, g), W.complex_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    t = Tree.build(_dev(xy), p=24, nlevels=4, path="fp64")
    gg, gxy = t.backward(_dev(gam), _dev(gphi))
    gg, gxy = gg.cpu().numpy(), gxy.cpu().numpy()
    G = _dev(gam)

    def loss(x, gm=None):
        t.rebuild(_dev(x))
        phi = t.eval(G if gm is None else _dev(gm)).cpu().numpy()
        return float(np.sum(gphi.real * phi.real + gphi.imag * phi.imag))

    h = 1e-7
    for k in (5, 1234, 2999):
        for d in (0, 1):
            xp, xm = xy.copy(), xy.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (loss(xp) - loss(xm)) / (2 * h)
            assert abs(fd - gxy[k, d]) < 1e-5 * max(1.0, abs(gxy[k, d])), (k, d, fd, gxy[k, d])
        gp, gm = gam.copy(), gam.copy()
        gp[k] += 1e-3
        gm[k] -= 1e-3
        fd = (loss(xy, gp) - loss(xy, gm)) / 2e-3
        assert abs(fd - gg[k].real) < 1e-8 * max(1.0, abs(gg[k].real))


def test_autograd_function_matches_backward():
    import paper_1311_1006_b300 as F

    g = np.random.default_rng(5)
    n = 5000
    xy = _dev(W.uniform(n, g)).requires_grad_(True)
    gam = _dev(W.complex_strengths(n, g)).requires_grad_(True)
    w = _dev(g.normal(size=n) + 1j * g.normal(size=n))
    phi = F.fmm(xy, gam, p=17, nlevels=5, path="fp64")
    loss = (phi * w.conj()).real.sum()
    loss.backward()
    t = F.Tree.build(xy.detach(), p=17, nlevels=5, path="fp64")
    gg, gxy = t.backward(gam.detach(), w)
    assert torch.allclose(gam.grad, gg, rtol=0, atol=1e-12 * gg.abs().max().item())
    assert torch.allclose(xy.grad, gxy, rtol=0, atol=1e-12 * gxy.abs().max().item())
