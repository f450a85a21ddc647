"""The adjoint's gradient convention (dL/dRe + i dL/dIm, upstream w + i v) is the
one torch.autograd uses for complex tensors: checked on the CPU against
autograd of a plain torch direct sum, and against the oracle's closed form."""
import numpy as np
import torch

from paper_1311_1006_b300 import workloads as W


def test_oracle_gradient_matches_torch_autograd_convention(orc):
    g = np.random.default_rng(4)
    n = 50
    xy = W.uniform(n, g)
    gam = W.complex_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    X = torch.tensor(xy, requires_grad=True)
    G = torch.tensor(gam, requires_grad=True)
    z = torch.complex(X[:, 0], X[:, 1])
    d = z[:, None] - z[None, :]
    eye = torch.eye(n, dtype=torch.bool)
    inv = torch.where(eye, torch.zeros_like(d), 1.0 / torch.where(eye, torch.ones_like(d), d))
    phi = inv @ G
    phi.backward(torch.tensor(gphi))
    rg, rxy = orc.direct_grad(xy, gam, gphi)
    np.testing.assert_allclose(G.grad.numpy(), rg, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(X.grad.numpy(), rxy, rtol=1e-9, atol=1e-9)
