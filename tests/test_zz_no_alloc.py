"""fmm_direct_eval_noalloc: the exact pairwise sum for callers that cannot
allocate device memory (their device memory is owned by a host framework's
pool, or their loop may not call cudaMalloc/cudaFree, which can synchronise the
device).  Called through the C ABI and compared with the existing entry point
computing the same sum (fmm_eval on a one-level tree = pure P2P, FP64 path)
and with the oracle's exact sum, within the FP64 tolerance of the other tests,
on two calls in a row; a second call must leave the device's free memory
unchanged.  This file
sorts last so a run that stops at the first failure has run everything else."""
import ctypes

import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _noalloc(lib, X, G, n, out):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.fmm_direct_eval_noalloc(ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(G.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()), s)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_noalloc_direct_sum_matches_fmm_eval_twice(orc):
    from paper_1311_1006_b300 import Tree, _lib

    lib = _lib.load()
    for call, (n, seed) in enumerate(((16384, 1), (3001, 2))):
        g = np.random.default_rng(seed)
        xy = W.cluster_mix(n, g)
        xy[n // 3] = xy[0]  # a coincident pair: excluded on both sides
        gam = W.complex_strengths(n, g)
        X, G = _dev(xy), _dev(gam)
        out = torch.empty(n, dtype=torch.complex128, device="cuda")
        assert _noalloc(lib, X, G, n, out) == 0, lib.fmm_last_error()
        ref = Tree.build(X, p=8, nlevels=1, path="fp64").eval(G)
        torch.cuda.synchronize()
        a = out.cpu().numpy()
        err = _rel(a, ref.cpu().numpy())
        assert err < TOL, (call, n, err)
        if n <= 4000:  # and against the oracle's exact sum (plain FP64 C on the host)
            err = _rel(a, orc.direct(xy, gam))
            assert err < TOL, (call, n, "oracle", err)


def test_noalloc_call_allocates_no_device_memory():
    """After a first call, a second call on the same stream leaves the device's
    free memory unchanged: the entry point allocates nothing."""
    from paper_1311_1006_b300 import _lib

    lib = _lib.load()
    n = 5000
    g = np.random.default_rng(3)
    X, G = _dev(W.uniform(n, g)), _dev(W.complex_strengths(n, g))
    out = torch.empty(n, dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, X, G, n, out) == 0, lib.fmm_last_error()
    first = out.clone()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert _noalloc(lib, X, G, n, out) == 0, lib.fmm_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    assert torch.equal(out, first)  # same inputs, same result bit for bit


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1311_1006_b300 import _lib

    lib = _lib.load()
    X = torch.zeros(16385, 2, dtype=torch.float64, device="cuda")
    G = torch.zeros(16385, dtype=torch.complex128, device="cuda")
    out = torch.empty(16385, dtype=torch.complex128, device="cuda")
    assert _noalloc(lib, X, G, 16385, out) == _lib.FMM_ERR_INVALID_ARG
    assert b"16384" in lib.fmm_last_error()
    assert _noalloc(lib, X, G, 0, out) == _lib.FMM_ERR_INVALID_ARG
