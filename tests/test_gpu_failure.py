"""Failure detection without a GPU fault: the library's bounded device waits,
run on something that never happens (a predecessor tile that never publishes,
an mbarrier nothing arrives at, a work-queue unit that never completes), give up after their limit and report
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
    # 0: decoupled look-back, 1: tensor-core M2L mbarrier, 2: persistent evaluation's work-queue wait
    for which in (0, 1, 2):
        t0 = time.time()
        assert lib.fmm_selftest_bounded_wait(which, None) == FMM_ERR_TIMEOUT
        assert time.time() - t0 < 10.0
    assert lib.fmm_selftest_bounded_wait(3, None) == FMM_ERR_INVALID_ARG
    # the context still works: a normal build and evaluation against the oracle
    g = np.random.default_rng(17)
    xy, gam = W.cluster_mix(3000, g), W.complex_strengths(3000, g)
    t = Tree.build(torch.tensor(xy, device="cuda"), p=12, nlevels=4, path="fp64")
    phi = t.eval(torch.tensor(gam, device="cuda")).cpu().numpy()
    ref = orc.fmm(xy, gam, 4, 0.5, 12)["phi"]
    assert np.abs(phi - ref).max() <= 1e-10 * np.abs(ref).max()
    t.close()


def test_fp64_reciprocal_within_one_ulp():
    """The FP64 P2P's reciprocal (approximate seed + two Newton-Raphson steps)
    against the correctly rounded 1/x, for inputs whose reciprocal is a normal
    double (squared distances of points: far inside that range)."""
    import ctypes

    from paper_1311_1006_b300 import _lib

    g = np.random.default_rng(19)
    x = np.concatenate([10.0 ** g.uniform(-300, 300, 200000), g.random(100000) * 2.0,
                        np.array([1.0, 2.0, 3.0, 0.5, 1e-300, 2.2250738585072014e-308, 1e300])])
    xd = torch.tensor(x, device="cuda")
    out = torch.empty_like(xd)
    st = _lib.load().fmm_selftest_rcp64(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                        x.size, None)
    assert st == 0
    r = out.cpu().numpy()
    exact = 1.0 / x
    ulp = np.abs(r - exact) / np.spacing(np.abs(exact))
    assert ulp.max() <= 1.0, float(ulp.max())
    # below the smallest normal double: 0 (the pair counts as coincident)
    tiny = torch.tensor([0.0, 1e-310, 4e-320], device="cuda", dtype=torch.float64)
    o2 = torch.empty_like(tiny)
    assert _lib.load().fmm_selftest_rcp64(ctypes.c_void_p(tiny.data_ptr()), ctypes.c_void_p(o2.data_ptr()), 3,
                                          None) == 0
    assert np.all(o2.cpu().numpy() == 0.0)
