"""Cost-model seed of N_levels (Sec. 2.3, eqs 2.4-2.5) on the host: the level
fmm_seed_nlevels picks minimises the modelled time alpha C_P2P + beta C_M2L
over all admissible levels (brute force over the model, not the seed's own
closed form), and the seed moves with p as the model says it must."""
import math

import numpy as np
import pytest


def _model_time(n, p, L, alpha, beta, theta=0.5):
    nf = 4.0 ** (L - 1)
    area = math.pi * ((1 + theta) / theta) ** 2
    return alpha * n * n / (2 * nf) * area + beta * 1.5 * nf * p * p * area


def _levels(n):
    L = 1
    while 4 ** L <= n:
        L += 1
    return range(1, L + 1)


def test_seed_minimises_the_modelled_time():
    import paper_1311_1006_b300 as F

    g = np.random.default_rng(0)
    for _ in range(300):
        n = int(10 ** g.uniform(1, 8))
        p = int(g.integers(1, 33))
        alpha = 10 ** g.uniform(-13, -9)
        beta = 10 ** g.uniform(-13, -10)
        L = F.seed_nlevels(n, p, alpha, beta)
        times = {k: _model_time(n, p, k, alpha, beta) for k in _levels(n)}
        best = min(times.values())
        # ties between neighbouring levels are within rounding of each other
        assert times[L] <= best * (1 + 1e-9), (n, p, alpha, beta, L, times)


def test_seed_moves_with_p():
    import paper_1311_1006_b300 as F

    a, b = F.cost_model("fp32")
    assert a > 0 and b > 0
    n = 2_000_000
    s12, s30 = F.seed_nlevels(n, 12, a, b), F.seed_nlevels(n, 30, a, b)
    assert s12 != s30 and s30 < s12  # higher p: costlier M2L, fewer and larger leaves
    assert F.default_nlevels(n, 12, "fp32") == s12


def test_cost_model_set_get_and_rejects_bad_values():
    import paper_1311_1006_b300 as F
    from paper_1311_1006_b300 import _lib

    a0, b0 = F.cost_model("fp64")
    try:
        F.set_cost_model(1e-10, 1e-12, "fp64")
        assert F.cost_model("fp64") == (1e-10, 1e-12)
        # a cheaper M2L relative to P2P moves the seed to more leaves
        assert F.default_nlevels(10 ** 6, 17, "fp64") >= F.seed_nlevels(10 ** 6, 17, a0, b0)
        for bad in ((0.0, 1.0), (1.0, -1.0), (float("inf"), 1.0), (float("nan"), 1.0)):
            with pytest.raises(_lib.FMMError):
                F.set_cost_model(*bad, "fp64")
    finally:
        F.set_cost_model(a0, b0, "fp64")
    assert F.seed_nlevels(0, 17, 1.0, 1.0) == 0
    assert F.seed_nlevels(100, 17, 0.0, 1.0) == 0
