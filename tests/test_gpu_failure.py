"""Failure detection without a GPU fault: the library's bounded device waits,
run on something that never happens (a predecessor tile that never publishes,
an mbarrier nothing arrives at), give up after their limit and report
FMM_ERR_TIMEOUT through the device status word; the context stays usable."""
import time

import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FMM_ERR_INVALID_ARG, FMM_ERR_TIMEOUT = 1, 4


def test_bounded_waits_time_out_and_the_context_survives(orc):
    from paper_1311_1006_b300 import Tree, _lib

    lib = _lib.load()
    torch.cuda.synchronize()
    for which in (0, 1):  # 0: decoupled look-back, 1: tensor-core M2L mbarrier
        t0 = time.time()
        assert lib.fmm_selftest_bounded_wait(which, None) == FMM_ERR_TIMEOUT
        assert time.time() - t0 < 10.0
    assert lib.fmm_selftest_bounded_wait(2, None) == FMM_ERR_INVALID_ARG
    # the context still works: a normal build and evaluation against the oracle
    g = np.random.default_rng(17)
    xy, gam = W.cluster_mix(3000, g), W.complex_strengths(3000, g)
    t = Tree.build(torch.tensor(xy, device="cuda"), p=12, nlevels=4, path="fp64")
    phi = t.eval(torch.tensor(gam, device="cuda")).cpu().numpy()
    ref = orc.fmm(xy, gam, 4, 0.5, 12)["phi"]
    assert np.abs(phi - ref).max() <= 1e-10 * np.abs(ref).max()
    t.close()
