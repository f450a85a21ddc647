"""Separate evaluation points (eq 2.2): Phi(y_i) = sum_{j: x_j != y_i} Gamma_j / (y_i - x_j),
GPU library vs the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    return torch.tensor(a, device="cuda")


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _case(seed):
    g = np.random.default_rng(seed)
    src = W.cluster_mix(20000, g)
    gam = W.complex_strengths(20000, g)
    tgt = np.concatenate([
        g.random((12000, 2)),                       # uniform in the unit square
        src[g.choice(20000, 300, replace=False)],   # on sources: those sources are skipped
        np.array([[1.5, -0.3], [-0.2, 0.7], [0.5, 1.25]]),  # outside the sources' bounding box
    ])
    return src, gam, tgt


def test_targets_fp64_matches_oracle_fmm_and_direct():
    import oracle
    from paper_1311_1006_b300 import Tree

    src, gam, tgt = _case(21)
    L, p, theta = 6, 17, 0.5
    t = Tree.build_targets(_dev(src), _dev(tgt), p=p, theta=theta, nlevels=L, path="fp64")
    phi = t.eval_targets(_dev(gam)).cpu().numpy()
    # the oracle FMM over the same point set (evaluation points with zero strength)
    allxy = np.concatenate([src, tgt])
    allg = np.concatenate([gam, np.zeros(len(tgt), np.complex128)])
    ref_fmm = oracle.fmm(allxy, allg, L, theta, p)["phi"][len(src):]
    assert _rel(phi, ref_fmm) <= 1e-10
    exact = oracle.direct_points(src, gam, tgt)
    assert _rel(phi, exact) <= 1e-6  # truncation at p = 17, theta = 0.5 (Table 4.1)
    t.close()


def test_targets_fp32_and_rebuild():
    import oracle
    from paper_1311_1006_b300 import Tree

    src, gam, tgt = _case(22)
    t = Tree.build_targets(_dev(src), _dev(tgt), p=17, theta=0.5, path="fp32")
    phi = t.eval_targets(_dev(gam)).cpu().numpy().astype(np.complex128)
    assert _rel(phi, oracle.direct_points(src, gam, tgt)) <= 1e-5
    # new coordinates for both sets, same sizes
    src2, gam2, tgt2 = _case(23)
    t.rebuild_targets(_dev(src2), _dev(tgt2))
    phi2 = t.eval_targets(_dev(gam2)).cpu().numpy().astype(np.complex128)
    assert _rel(phi2, oracle.direct_points(src2, gam2, tgt2)) <= 1e-5
    t.close()


def test_targets_argument_checks():
    from paper_1311_1006_b300 import FMMError, Tree

    g = np.random.default_rng(24)
    xy = _dev(g.random((1000, 2)))
    t = Tree.build(xy, p=8, nlevels=3, path="fp64")
    with pytest.raises(FMMError):
        t.n_src, t.n_tgt = 500, 500
        t.eval_targets(_dev(np.ones(500, np.complex128)))  # not built with separate points
    t.close()


@pytest.mark.parametrize("path", ["fp64", "fp32"])
def test_targets_only_evaluated_against_sources_only(path):
    """Leaves with only sources, only evaluation points, and both: P2P takes a
    leaf's sources as sources and its evaluation points as targets (the slot
    block holds the sources first); the result still equals the oracle FMM
    over the same point set, and the exact sum within the FP32 tolerance."""
    import oracle
    from paper_1311_1006_b300 import Tree

    g = np.random.default_rng(31)
    ns, nt = 30000, 30000
    src = W.cluster_mix(ns, g) * np.array([0.6, 1.0])       # sources in x < 0.6
    tgt = np.concatenate([g.random((nt - 500, 2)), src[g.choice(ns, 500, replace=False)]])
    gam = W.complex_strengths(ns, g)
    L, p = 7, 17
    t = Tree.build_targets(_dev(src), _dev(tgt), p=p, nlevels=L, path=path)
    phi = t.eval_targets(_dev(gam)).cpu().numpy().astype(np.complex128)
    allxy = np.concatenate([src, tgt])
    allg = np.concatenate([gam, np.zeros(nt, np.complex128)])
    ref = oracle.fmm(allxy, allg, L, 0.5, p)["phi"][ns:]
    assert _rel(phi, ref) <= (1e-10 if path == "fp64" else 1e-5)
    pick = g.choice(nt, 512, replace=False)
    exact = oracle.direct_points(src, gam, tgt[pick])
    assert _rel(phi[pick], exact) <= 1e-5
    # the log kernel at the same points
    phl = t.eval_targets_log(_dev(gam)).cpu().numpy().astype(np.complex128)
    refl = oracle.fmm_log(allxy, allg, L, 0.5, p)[ns:]
    assert _rel(phl, refl) <= (1e-10 if path == "fp64" else 1e-5)
    t.close()
