"""Theta tuning (the theta moves of Algorithms 2-4, Sec. 4.2) and the p(TOL, theta)
rule of Sec. 4.1, host-only: the standalone tuner is driven by synthetic cost
curves, no GPU involved."""
from __future__ import annotations

import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    rows = []
    with open(os.path.join(HERE, "golden", "table_4_1_p_vs_tol.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                tol, theta, p = ln.split()
                rows.append((float(tol), float(theta), int(p)))
    return rows


def test_p_for_tolerance_follows_table_4_1():
    """p is never below the paper's Table 4.1 and at most one term above it."""
    from paper_1311_1006_b300 import p_for_tolerance

    rows = _table()
    assert len(rows) == 15
    for tol, theta, p in rows:
        q = p_for_tolerance(tol, theta)
        assert p <= q <= p + 1, (tol, theta, p, q)


def test_p_for_tolerance_monotone_and_invalid():
    from paper_1311_1006_b300 import p_for_tolerance

    ths = [0.3 + 0.01 * i for i in range(40)]
    ps = [p_for_tolerance(1e-6, th) for th in ths]
    assert all(a <= b for a, b in zip(ps, ps[1:]))  # larger theta needs more terms
    assert p_for_tolerance(1e-8, 0.5) > p_for_tolerance(1e-6, 0.5)  # tighter tolerance needs more terms
    assert p_for_tolerance(0.0, 0.5) == -1 and p_for_tolerance(1e-6, 1.0) == -1


def _cost(L, theta, L_opt=7, th_opt=0.46):
    # separable cost with its minimum at (L_opt, th_opt): the paper observes the optima in theta and
    # N_levels to be practically independent (Sec. 4.2, "Correlated controls")
    return 1.0 + 0.2 * (L - L_opt) ** 2 + 40.0 * (theta - th_opt) ** 2


def test_theta_walk_finds_the_optimum():
    from paper_1311_1006_b300 import Autotuner

    tu = Autotuner(5, 10, cap=0.5, window=1, period=1)
    tu.enable_theta(0.60, 1e-6, 0.35, 0.65)
    L, th, p = 5, 0.60, None
    for _ in range(400):
        L, th, p = tu.step_params(_cost(L, th))
    st = tu.stats()
    assert int(st["accepted"]) == 7
    assert abs(st["theta"] - 0.46) <= 0.015, st
    # p follows theta through the tolerance rule
    from paper_1311_1006_b300 import p_for_tolerance

    assert p == p_for_tolerance(1e-6, th)


def test_theta_steps_follow_the_fibonacci_sequence():
    """Every theta move is rejected (the start is optimal): each rejection
    reverses the direction and takes the next Fibonacci step (1, 2, 3 x 0.01);
    at the end of the sequence the count restarts and the sequence grows."""
    from paper_1311_1006_b300 import Autotuner

    tu = Autotuner(6, 6, cap=0.5, window=1, period=1)  # N_levels cannot move (1 level range)
    tu.enable_theta(0.50, 1e-6, 0.30, 0.65)
    L, th, _ = 6, 0.50, None
    offsets = []
    for _ in range(80):
        L, th, _ = tu.step_params(1.0 + 50.0 * abs(th - 0.50))
        if abs(th - 0.50) > 1e-9:
            offsets.append(round((th - 0.50) / 0.01))
    # trials in order: +1, -2, +3 (the sequence of length 3 ends: the count restarts and the
    # sequence grows to length 4), then -1, +2, -3, +5; the direction reverses after every rejection
    assert offsets[:3] == [1, -2, 3], offsets[:10]
    assert offsets[3:7] == [-1, 2, -3, 5], offsets[:10]
    st = tu.stats()
    assert abs(st["theta"] - 0.50) < 1e-9 and st["rejected"] >= len(offsets) - 1


def test_theta_stays_in_range_and_p_fits():
    from paper_1311_1006_b300 import Autotuner, FMMError, p_for_tolerance

    tu = Autotuner(6, 6, cap=0.5, window=1, period=1)
    with pytest.raises(FMMError):
        tu.enable_theta(0.60, 1e-8, 0.35, 0.80)  # p(1e-8, 0.60) = 33 > 32: not a valid start
    tu.enable_theta(0.55, 1e-8, 0.35, 0.80)  # p(1e-8, theta) exceeds 32 above theta ~ 0.59
    th = 0.55
    for _ in range(200):
        _, th, p = tu.step_params(1.0 - th)  # always rewards a larger theta
        assert 0.35 - 1e-9 <= th <= 0.80 and p <= 32
    assert p_for_tolerance(1e-8, th) <= 32


def test_theta_tuning_argument_checks():
    from paper_1311_1006_b300 import Autotuner, FMMError

    tu = Autotuner(5, 10)
    with pytest.raises(FMMError):
        tu.enable_theta(0.5, 0.0, 0.35, 0.65)
    with pytest.raises(FMMError):
        tu.enable_theta(0.9, 1e-6, 0.35, 0.65)  # start outside the range
    with pytest.raises(FMMError):
        tu.enable_theta(0.9, 1e-8, 0.85, 0.95)  # p(1e-8, 0.85) > 32
