"""Batched instances (one forest, one set of launches) vs standalone trees and
the oracle: every instance must equal its own evaluation."""
import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda")


def _batch(seed, B, lo=200, hi=3000):
    g = np.random.default_rng(seed)
    sizes = np.floor(10 ** g.uniform(np.log10(lo), np.log10(hi), size=B)).astype(np.int64)
    pts = [W.batch_instance(int(n), g) for n in sizes]
    gam = [W.real_strengths(int(n), g) for n in sizes]
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return np.vstack(pts), np.concatenate(gam), offs, sizes


@pytest.mark.parametrize("path,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_batched_matches_oracle_per_instance(orc, path, tol):
    from paper_1311_1006_b300 import Tree

    xy, gam, offs, sizes = _batch(1, 24)
    levels = [max(1, min(W.leaf_levels(int(n), 35), 6)) for n in sizes]
    levels[3] = 1  # a one-level instance inside the forest
    t = Tree.build_batched(_dev(xy), offs, nlevels=levels, p=16, path=path)
    phi = t.eval(_dev(gam)).cpu().numpy().astype(np.complex128)
    for b in range(len(sizes)):
        s, e = offs[b], offs[b + 1]
        ref = orc.fmm(xy[s:e], gam[s:e], levels[b], 0.5, 16)["phi"]
        err = np.abs(phi[s:e] - ref).max() / np.abs(ref).max()
        assert err < tol, (b, sizes[b], levels[b], err)


def test_batched_equals_standalone_trees():
    from paper_1311_1006_b300 import Tree

    xy, gam, offs, sizes = _batch(2, 12, lo=1000, hi=20000)
    t = Tree.build_batched(_dev(xy), offs, p=16, path="fp64")
    phi = t.eval(_dev(gam)).cpu().numpy()
    lev = t.export("inst")[:, 2]
    for b in range(len(sizes)):
        s, e = offs[b], offs[b + 1]
        tb = Tree.build(_dev(xy[s:e]), p=16, nlevels=int(lev[b]), path="fp64")
        ref = tb.eval(_dev(gam[s:e])).cpu().numpy()
        assert np.abs(phi[s:e] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_batched_tree_matches_oracle_trees(orc):
    from paper_1311_1006_b300 import Tree

    xy, gam, offs, sizes = _batch(3, 9)
    levels = [max(1, min(W.leaf_levels(int(n), 35), 5)) for n in sizes]
    t = Tree.build_batched(_dev(xy), offs, nlevels=levels, path="fp64")
    perm = t.export("perm")
    inst = t.export("inst")
    center = t.export("center")
    for b in range(len(sizes)):
        s, e = offs[b], offs[b + 1]
        ref = orc.build_tree(xy[s:e], levels[b])
        assert np.array_equal(perm[s:e] - s, ref["perm"])
        bo = inst[b, 1]
        nb = orc.num_boxes(levels[b])
        assert np.array_equal(center[bo:bo + nb], ref["center"])
