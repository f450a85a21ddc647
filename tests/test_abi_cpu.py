"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/fmm2d.h declares, rejects bad arguments before touching
the device, and the AT3b autotuner (Sec. 4.2, Algorithm 4) behaves as the paper
describes on synthetic cost curves."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1311_1006_b300 import _lib, build

    build.build()
    return _lib.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "fmm2d.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmm_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for s in range(6):
        assert lib.fmm_status_string(s)
    assert lib.fmm_status_string(99) == b"unknown status"


def test_invalid_arguments_rejected_on_host(lib):
    import ctypes

    from paper_1311_1006_b300 import _lib

    h = ctypes.c_void_p()
    dummy = ctypes.c_void_p(0x1000)  # never dereferenced: validation fails first
    bad = [
        (10, _lib.FMMParams(0, 0.5, 0, 0, 0)),      # p < 1
        (10, _lib.FMMParams(33, 0.5, 0, 0, 0)),     # p > 32
        (10, _lib.FMMParams(17, 1.0, 0, 0, 0)),     # theta not in (0,1)
        (10, _lib.FMMParams(17, 0.0, 0, 0, 0)),
        (10, _lib.FMMParams(17, 0.5, 0, 2, 0)),     # unknown path
        (10, _lib.FMMParams(17, 0.5, -1, 0, 0)),    # negative nlevels
        (0, _lib.FMMParams(17, 0.5, 0, 0, 0)),      # n = 0
    ]
    for n, prm in bad:
        st = lib.fmm_build_tree(dummy, n, ctypes.byref(prm), None, ctypes.byref(h))
        assert st == _lib.FMM_ERR_INVALID_ARG, (n, prm.p, prm.theta)
        assert not h.value
    st = lib.fmm_build_tree(None, 10, ctypes.byref(_lib.FMMParams(17, 0.5, 0, 0, 0)), None, ctypes.byref(h))
    assert st == _lib.FMM_ERR_INVALID_ARG
    assert lib.fmm_eval(None, None, None, None) == _lib.FMM_ERR_INVALID_ARG
    assert lib.fmm_eval_backward(None, None, None, None, None, None) == _lib.FMM_ERR_INVALID_ARG
    assert b"NULL" in lib.fmm_last_error()


def test_default_nlevels_keeps_leaves_nonempty(lib):
    for n in (1, 3, 4, 15, 16, 1000, 10_000, 1_000_000):
        for path in (0, 1):
            L = lib.fmm_default_nlevels(n, 17, path)
            assert L >= 1 and 4 ** (L - 1) <= n
    # about 35 points per leaf at N = 1e4 (the plain FP64 workload)
    assert lib.fmm_default_nlevels(10_000, 20, 1) in (5, 6)


def _run_tuner(cost, L0, Lmax, steps, cap=0.1, window=3, period=4, noise=0.0, seed=0):
    from paper_1311_1006_b300 import Autotuner

    g = np.random.default_rng(seed)
    tu = Autotuner(L0, Lmax, cap=cap, window=window, period=period)
    L, hist, total = L0, [], 0.0
    for _ in range(steps):
        t = cost(L) * (1.0 + noise * g.random())
        total += t
        hist.append(L)
        L = tu.step(t)
    return tu, hist, total


def test_autotuner_walks_to_the_minimum(lib):
    cost = lambda L: 1.0 + 0.3 * (L - 7) ** 2  # convex, optimum at 7
    for L0 in (3, 9):
        tu, hist, total = _run_tuner(cost, L0, 10, 200, noise=0.02)
        assert tu.stats()["accepted"] == 7, (L0, hist[-20:])
        assert 7 in hist[:60]  # reached quickly
        # afterwards the probing costs about cap of the run time, not more
        lost = sum(cost(L) - cost(7) for L in hist[100:])
        assert lost <= 2 * 0.1 * sum(cost(L) for L in hist[100:])


def test_autotuner_rejects_a_worse_move_and_respects_the_cap(lib):
    # Optimum already at the start: every move is rejected, and the time lost
    # to rejected moves stays below about cap * total time (AT3b's purpose).
    cost = lambda L: 1.0 + 0.5 * abs(L - 6)
    for cap in (0.05, 0.1, 0.3):
        tu, hist, total = _run_tuner(cost, 6, 10, 600, cap=cap, period=2)
        st = tu.stats()
        assert st["accepted"] == 6 and st["rejected"] >= 2
        lost = sum(cost(L) - cost(6) for L in hist)
        assert lost <= 1.5 * cap * total + 3 * 1.5, (cap, lost, total)


def test_autotuner_follows_a_moving_optimum(lib):
    # Time-marching problems drift (Sec. 4.2): the optimum moves from 5 to 8.
    from paper_1311_1006_b300 import Autotuner

    tu = Autotuner(5, 10, cap=0.2, window=2, period=2)
    L = 5
    for it in range(600):
        opt = 5 if it < 200 else 8
        L = tu.step(1.0 + 0.4 * abs(L - opt))
    assert tu.stats()["accepted"] == 8


def test_autotuner_argument_checks(lib):
    import ctypes

    from paper_1311_1006_b300 import _lib

    h = ctypes.c_void_p()
    assert lib.fmm_autotuner_create(0, 5, 0.1, 3, 4, ctypes.byref(h)) == _lib.FMM_ERR_INVALID_ARG
    assert lib.fmm_autotuner_create(6, 5, 0.1, 3, 4, ctypes.byref(h)) == _lib.FMM_ERR_INVALID_ARG
    assert lib.fmm_autotuner_create(3, 5, 0.0, 3, 4, ctypes.byref(h)) == _lib.FMM_ERR_INVALID_ARG
