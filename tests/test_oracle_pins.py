"""Pins for the oracle: each test checks the oracle against something the paper
or the mathematics fixes (closed forms, invariants, brute force on tiny inputs,
the paper's Table 4.1 and complexity estimates), never against a retyped copy
of its own formulas.  CPU only."""
import os

import numpy as np
import pytest

from paper_1311_1006_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cz(xy):
    return xy[:, 0] + 1j * xy[:, 1]


# ----------------------------------------------------------------- direct sum

def test_direct_roots_of_unity_closed_form(orc):
    # Points at the n-th roots of unity with unit strengths: for p(z) = z^n - 1,
    # sum_{j!=k} 1/(z_k - z_j) = p''(z_k) / (2 p'(z_k)) = (n-1) / (2 z_k).
    for n in (2, 3, 7, 64):
        z = np.exp(2j * np.pi * np.arange(n) / n)
        xy = np.stack([z.real, z.imag], 1)
        phi = orc.direct(xy, np.ones(n))
        np.testing.assert_allclose(phi, (n - 1) / (2 * z), rtol=1e-12, atol=1e-12)


def test_direct_two_points_values(orc):
    # Phi(z_1) = Gamma_2/(z_1 - z_2) with the + sign of the kernel: z_1 = 0,
    # z_2 = 1, Gamma_2 = 2 -> Phi_1 = -2;  Phi_2 = Gamma_1/(1 - 0) = Gamma_1.
    xy = np.array([[0.0, 0.0], [1.0, 0.0]])
    phi = orc.direct(xy, np.array([3.0 + 1j, 2.0]))
    np.testing.assert_allclose(phi, [-2.0, 3.0 + 1j], atol=1e-15)
    # a purely imaginary offset: 1/(0 - i) = i
    xy = np.array([[0.0, 0.0], [0.0, 1.0]])
    np.testing.assert_allclose(orc.direct(xy, np.array([0.0, 1.0]))[0], 1j, atol=1e-15)


def test_direct_pairwise_antisymmetry(orc):
    # sum_i Gamma_i Phi_i = sum_{i != j} Gamma_i Gamma_j / (z_i - z_j) = 0 (pairs cancel).
    g = np.random.default_rng(1)
    xy = W.uniform(500, g)
    gam = W.complex_strengths(500, g)
    phi = orc.direct(xy, gam)
    assert abs(np.sum(gam * phi)) < 1e-10 * np.sum(np.abs(gam * phi))


def test_direct_coincident_points_excluded(orc):
    # Two coincident sources a, b at z0 and a third point z2: the pair at z0 is
    # excluded (eq 2.2), so Phi(z0) = c/(z0 - z2) for both, Phi(z2) = (a+b)/(z2-z0).
    xy = np.array([[0.25, 0.5], [0.25, 0.5], [0.75, 0.25]])
    a, b, c = 1.5, -0.5 + 2j, 0.25
    phi = orc.direct(xy, np.array([a, b, c]))
    z0, z2 = 0.25 + 0.5j, 0.75 + 0.25j
    np.testing.assert_allclose(phi, [c / (z0 - z2), c / (z0 - z2), (a + b) / (z2 - z0)], rtol=1e-14)


def test_direct_derivative_matches_finite_difference(orc):
    # Phi is holomorphic in the target, so dPhi/dz = dPhi/dx.
    g = np.random.default_rng(2)
    xy = W.uniform(40, g)
    gam = W.complex_strengths(40, g)
    _, dphi = orc.direct(xy, gam, targets=np.arange(40), deriv=True)
    h = 1e-6
    for t in (0, 7, 39):
        src = np.delete(np.arange(40), t)
        zt = xy[t, 0] + 1j * xy[t, 1]
        zs = _cz(xy[src])
        f = lambda z: np.sum(gam[src] / (z - zs))  # field of the other points
        fd = (f(zt + h) - f(zt - h)) / (2 * h)
        assert abs(fd - dphi[t]) < 1e-6 * abs(dphi[t])


def _loss(orc, xy, gam, gphi):
    phi = orc.direct(xy, gam)
    return float(np.sum(gphi.real * phi.real + gphi.imag * phi.imag))


def test_direct_gradient_matches_central_differences(orc):
    # L = sum_i w_i Re Phi_i + v_i Im Phi_i; compare the closed-form gradient
    # with central differences of the direct sum in x, y, Re Gamma, Im Gamma.
    g = np.random.default_rng(3)
    n = 60
    xy = W.uniform(n, g)
    gam = W.complex_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    gg, gxy = orc.direct_grad(xy, gam, gphi)
    h = 1e-6
    for k in (0, 13, 59):
        for d in (0, 1):
            xp, xm = xy.copy(), xy.copy()
            xp[k, d] += h
            xm[k, d] -= h
            fd = (_loss(orc, xp, gam, gphi) - _loss(orc, xm, gam, gphi)) / (2 * h)
            assert abs(fd - gxy[k, d]) < 2e-5 * max(1.0, abs(gxy[k, d])), (k, d, fd, gxy[k, d])
        for comp, unit in ((0, 1.0), (1, 1j)):
            gp, gm = gam.copy(), gam.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            fd = (_loss(orc, xy, gp, gphi) - _loss(orc, xy, gm, gphi)) / (2 * h)
            ref = gg[k].real if comp == 0 else gg[k].imag
            assert abs(fd - ref) < 1e-6 * max(1.0, abs(ref))


# ----------------------------------------------------------------------- tree

def _lex_less_all(a_key, a_idx, b_key, b_idx):
    """max over set A of (key, idx) < min over set B, lexicographically."""
    if len(a_key) == 0 or len(b_key) == 0:
        return True
    ia = np.lexsort((a_idx, a_key))[-1]
    ib = np.lexsort((b_idx, b_key))[0]
    return (a_key[ia], a_idx[ia]) < (b_key[ib], b_idx[ib])


@pytest.mark.parametrize("n,levels,ties", [(37, 3, False), (100, 4, True), (1000, 5, True), (64, 4, False)])
def test_tree_median_split_invariants(orc, n, levels, ties):
    g = np.random.default_rng(n)
    xy = W.uniform(n, g)
    if ties:  # many equal x and y values: the original index decides
        xy = np.round(xy * 7) / 7
    t = orc.build_tree(xy, levels)
    perm, bs, bc = t["perm"], t["bstart"], t["bcount"]
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert bs[0] == 0 and bc[0] == n
    for l in range(levels - 1):
        off, coff = orc.num_boxes(l), orc.num_boxes(l + 1)
        for b in range(4 ** l):
            G = off + b
            par = perm[bs[G]: bs[G] + bc[G]]
            kids = [perm[bs[coff + 4 * b + c]: bs[coff + 4 * b + c] + bc[coff + 4 * b + c]] for c in range(4)]
            assert np.array_equal(np.sort(np.concatenate(kids)), np.sort(par))
            nl = len(par) // 2
            left, right = np.concatenate(kids[:2]), np.concatenate(kids[2:])
            assert len(left) == nl and len(right) == len(par) - nl
            assert len(kids[0]) == nl // 2 and len(kids[2]) == (len(par) - nl) // 2
            # x-split by (x, index); y-split of each half by (y, index)
            assert _lex_less_all(xy[left, 0], left, xy[right, 0], right)
            assert _lex_less_all(xy[kids[0], 1], kids[0], xy[kids[1], 1], kids[1])
            assert _lex_less_all(xy[kids[2], 1], kids[2], xy[kids[3], 1], kids[3])
    # leaves are non-empty and ordered by (y, index)
    l0 = orc.num_boxes(levels - 1)
    for G in range(l0, orc.num_boxes(levels)):
        ids = perm[bs[G]: bs[G] + bc[G]]
        assert len(ids) >= 1
        assert np.array_equal(ids, ids[np.lexsort((ids, xy[ids, 1]))])


def test_tree_geometry_encloses_and_is_tight(orc):
    g = np.random.default_rng(11)
    xy = W.cluster_mix(3000, g)
    t = orc.build_tree(xy, 5)
    for G in range(orc.num_boxes(5)):
        ids = t["perm"][t["bstart"][G]: t["bstart"][G] + t["bcount"][G]]
        c, r = t["center"][G], t["radius"][G]
        d = np.hypot(xy[ids, 0] - c[0], xy[ids, 1] - c[1])
        assert np.all(d <= r * (1 + 1e-14) + 1e-300)
        # tight: the bbox edges are touched and the radius is the half diagonal
        lo, hi = xy[ids].min(0), xy[ids].max(0)
        np.testing.assert_allclose(c, (lo + hi) / 2, rtol=0, atol=1e-16)
        assert abs(r - 0.5 * np.hypot(*(hi - lo))) <= 4e-16 * max(1.0, r)


def test_tree_rejects_empty_leaves(orc):
    with pytest.raises(ValueError):
        orc.build_tree(W.uniform(10, np.random.default_rng(0)), 4)  # 16 leaves > 10 points


# --------------------------------------------------------------------- lists

@pytest.mark.parametrize("dist,levels,theta", [("uniform", 4, 0.5), ("cluster", 4, 0.5), ("uniform", 5, 0.35),
                                               ("cluster", 5, 0.65), ("line", 4, 0.5)])
def test_lists_cover_every_leaf_pair_exactly_once(orc, dist, levels, theta):
    g = np.random.default_rng(levels * 10 + int(theta * 100))
    n = 4 ** (levels - 1) * 5
    if dist == "uniform":
        xy = W.uniform(n, g)
    elif dist == "cluster":
        xy = W.cluster_mix(n, g)
    else:  # points near a line, a distribution the paper also tunes for (Sec. 4.1)
        s = g.random(n)
        xy = np.stack([s, 0.5 + 0.3 * s + 1e-3 * g.normal(size=n)], 1)
    t = orc.build_tree(xy, levels)
    li = orc.build_lists(levels, t["center"], t["radius"], theta)
    so, si, wo, wi = li["s_off"], li["s_idx"], li["w_off"], li["w_idx"]
    nf = 4 ** (levels - 1)
    l0 = orc.num_boxes(levels - 1)
    cover = np.zeros((nf, nf), np.int64)
    for a in range(nf):
        for s in si[so[l0 + a]: so[l0 + a + 1]]:
            cover[a, s - l0] += 1
    for l in range(1, levels):
        off = orc.num_boxes(l)
        span = 4 ** (levels - 1 - l)  # leaves per box at level l
        for A in range(4 ** l):
            for B in wi[wo[off + A]: wo[off + A + 1]]:
                Bi = B - off
                cover[A * span:(A + 1) * span, Bi * span:(Bi + 1) * span] += 1
    assert np.all(cover == 1), np.argwhere(cover != 1)[:5]
    # weak pairs satisfy eq (2.3) and are symmetric; strong pairs are symmetric
    C, R = t["center"], t["radius"]
    for G in range(orc.num_boxes(levels)):
        for B in wi[wo[G]: wo[G + 1]]:
            d = np.hypot(*(C[G] - C[B]))
            assert max(R[G], R[B]) + theta * min(R[G], R[B]) <= theta * d and d > 0
            assert G in wi[wo[B]: wo[B + 1]]
        for B in si[so[G]: so[G + 1]]:
            assert G in si[so[B]: so[B + 1]]
            if B != G:
                d = np.hypot(*(C[G] - C[B]))
                assert not (max(R[G], R[B]) + theta * min(R[G], R[B]) <= theta * d and d > 0)
    assert list(si[so[0]: so[1]]) == [0] and wo[1] == 0


@pytest.mark.parametrize("levels", [5, 6])
def test_lists_match_complexity_estimates(orc, levels):
    # eq (2.4): C_P2P ~ N^2/(2 N_f) pi ((1+theta)/theta)^2 interactions;
    # eq (2.5): finest-level M2L pairs ~ (3 N_f / 2) pi ((1+theta)/theta)^2.
    g = np.random.default_rng(7)
    n, theta = 20000, 0.5
    xy = W.uniform(n, g)
    t = orc.build_tree(xy, levels)
    li = orc.build_lists(levels, t["center"], t["radius"], theta)
    nb, l0 = orc.num_boxes(levels), orc.num_boxes(levels - 1)
    nf = nb - l0
    inter = sum(int(t["bcount"][b]) * int(t["bcount"][li["s_idx"][li["s_off"][b]:li["s_off"][b + 1]]].sum())
                for b in range(l0, nb))
    k = np.pi * ((1 + theta) / theta) ** 2
    assert 0.5 < inter / (n * n / (2 * nf) * k) < 1.5
    assert 0.5 < (li["w_off"][nb] - li["w_off"][l0]) / (1.5 * nf * k) < 1.5


# -------------------------------------------------------------- expansions

def _setup(orc, n=3000, levels=4, seed=21, dist="uniform"):
    g = np.random.default_rng(seed)
    xy = W.uniform(n, g) if dist == "uniform" else W.cluster_mix(n, g)
    gam = W.complex_strengths(n, g)
    t = orc.build_tree(xy, levels)
    return xy, gam, t


def _far_point(c, r, factor):
    return complex(c[0], c[1]) + factor * r * np.exp(0.7j)


def test_p2m_and_m2m_series_converge_to_the_kernel(orc):
    # sum_k a_k/(z-c)^(k+1) equals the box's exact field at a point with
    # |z-c| = rho > r, up to sum|Gamma| (r/rho)^p / (rho - r).
    xy, gam, t = _setup(orc)
    p = 20
    mp = orc.m2m(t, orc.p2m(t, xy, gam, p))
    for G in (0, 1, 3, 7, 20, orc.num_boxes(3) + 5, orc.num_boxes(4) - 1):
        ids = t["perm"][t["bstart"][G]: t["bstart"][G] + t["bcount"][G]]
        c, r = t["center"][G], t["radius"][G]
        for factor in (2.0, 3.0):
            z = _far_point(c, r, factor)
            rho = factor * r
            exact = np.sum(gam[ids] / (z - _cz(xy[ids])))
            series = np.sum(mp[G] / (z - complex(*c)) ** (np.arange(p) + 1))
            bound = np.sum(np.abs(gam[ids])) * (r / rho) ** p / (rho - r)
            assert abs(series - exact) <= 1.01 * bound + 1e-12 * abs(exact)


def test_m2l_l2p_single_pair_within_truncation_bound(orc):
    # One weakly coupled leaf pair: local expansion of the source's field at the
    # target leaf, evaluated at the target's points, vs the exact field.  The
    # error must fall geometrically in p.
    xy, gam, t = _setup(orc, levels=4)
    li = orc.build_lists(4, t["center"], t["radius"], 0.5)
    l0, nb = orc.num_boxes(3), orc.num_boxes(4)
    G = next(b for b in range(l0, nb) if li["w_off"][b + 1] > li["w_off"][b])
    H = li["w_idx"][li["w_off"][G]]
    errs = []
    for p in (6, 12, 18, 24):
        mp = orc.p2m(t, xy, gam, p)
        one = dict(w_off=np.zeros(nb + 1, np.int64), w_idx=np.array([H], np.int32))
        one["w_off"][G + 1:] = 1
        lo = orc.m2l(t, one, mp)
        far = orc.l2p(t, xy, lo)
        ti = t["perm"][t["bstart"][G]: t["bstart"][G] + t["bcount"][G]]
        si = t["perm"][t["bstart"][H]: t["bstart"][H] + t["bcount"][H]]
        exact = np.array([np.sum(gam[si] / (complex(*xy[i]) - _cz(xy[si]))) for i in ti])
        errs.append(np.abs(far[ti] - exact).max() / np.abs(exact).max())
    assert errs[-1] < 1e-7
    assert all(errs[i + 1] < 0.2 * errs[i] for i in range(len(errs) - 1)), errs


def test_l2l_is_an_exact_polynomial_shift(orc):
    # L2L re-centres the polynomial sum_l b_l (z-c)^l: with random coefficients
    # on the parents of the leaves only, the leaves' shifted coefficients
    # evaluated by L2P at the leaf points equal the parent polynomial there.
    xy, gam, t = _setup(orc, levels=4)
    p = 15
    g = np.random.default_rng(5)
    lp, l0, nb = orc.num_boxes(2), orc.num_boxes(3), orc.num_boxes(4)
    lo = np.zeros((nb, p), np.complex128)
    lo[lp:l0] = g.normal(size=(l0 - lp, p)) + 1j * g.normal(size=(l0 - lp, p))
    vals = orc.l2p(t, xy, orc.l2l(t, lo))
    for G in range(l0, nb):
        P = lp + (G - l0) // 4
        ids = t["perm"][t["bstart"][G]: t["bstart"][G] + t["bcount"][G]]
        w = _cz(xy[ids]) - complex(*t["center"][P])
        want = sum(lo[P, k] * w ** k for k in range(p))
        assert np.abs(vals[ids] - want).max() <= 1e-12 * np.abs(lo[P]).sum()


# ------------------------------------------------------------- whole method

def test_fmm_single_level_is_the_direct_sum(orc):
    g = np.random.default_rng(8)
    xy, gam = W.uniform(700, g), W.complex_strengths(700, g)
    ref = orc.direct(xy, gam)
    out = orc.fmm(xy, gam, 1, 0.5, 10)["phi"]
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


def test_fmm_error_falls_geometrically_in_p(orc):
    # p ~ log TOL / log theta (Sec. 2.3): each extra term gains about a factor
    # theta; the far-field error must shrink by > 10x over every 6 terms.
    g = np.random.default_rng(9)
    xy, gam = W.cluster_mix(4000, g), W.complex_strengths(4000, g)
    ref = orc.direct(xy, gam)
    errs = []
    for p in (4, 10, 16, 22, 28):
        o = orc.fmm(xy, gam, 4, 0.5, p, parts=True)
        farref = ref - o["near"]
        errs.append(np.abs(o["far"] - farref).max() / np.abs(farref).max())
    assert errs[-1] < 1e-9
    assert all(errs[i + 1] < 0.1 * errs[i] for i in range(len(errs) - 1)), errs


def test_fmm_table_4_1_tolerances(orc):
    # Table 4.1: at the printed (TOL, theta) the printed p reaches TOL.  The
    # far-field relative max-norm error of the oracle must be <= TOL.
    rows = [r.split() for r in open(os.path.join(GOLDEN, "table_4_1_p_vs_tol.txt")) if not r.startswith("#")]
    g = np.random.default_rng(5)
    xy, gam = W.uniform(4000, g), W.real_strengths(4000, g)
    ref = orc.direct(xy, gam)
    for tol, theta, p in rows:
        o = orc.fmm(xy, gam, 4, float(theta), int(p), parts=True)
        farref = ref - o["near"]
        err = np.abs(o["far"] - farref).max() / np.abs(farref).max()
        assert err <= float(tol), (tol, theta, p, err)


def test_fmm_linear_in_strengths(orc):
    g = np.random.default_rng(10)
    xy = W.uniform(2000, g)
    a, b = W.complex_strengths(2000, g), W.complex_strengths(2000, g)
    fa, fb = orc.fmm(xy, a, 4, 0.5, 12)["phi"], orc.fmm(xy, b, 4, 0.5, 12)["phi"]
    fab = orc.fmm(xy, 2.0 * a - 3j * b, 4, 0.5, 12)["phi"]
    assert np.abs(fab - (2.0 * fa - 3j * fb)).max() <= 1e-12 * np.abs(fab).max()


def test_fmm_permutation_invariant(orc):
    g = np.random.default_rng(12)
    xy, gam = W.uniform(2000, g), W.complex_strengths(2000, g)
    out = orc.fmm(xy, gam, 4, 0.5, 14)["phi"]
    q = g.permutation(2000)
    outq = orc.fmm(xy[q], gam[q], 4, 0.5, 14)["phi"]
    assert np.abs(outq - out[q]).max() <= 1e-12 * np.abs(out).max()


def test_fmm_antisymmetry_within_tolerance(orc):
    g = np.random.default_rng(13)
    xy, gam = W.uniform(3000, g), W.real_strengths(3000, g)
    phi = orc.fmm(xy, gam, 4, 0.5, 20)["phi"]
    assert abs(np.sum(gam * phi)) <= 1e-8 * np.sum(np.abs(gam * phi))


def test_fmm_gradient_matches_direct_gradient(orc):
    g = np.random.default_rng(14)
    n = 3000
    xy, gam = W.uniform(n, g), W.real_strengths(n, g)
    gphi = g.normal(size=n) + 1j * g.normal(size=n)
    gg, gxy = orc.fmm_grad(xy, gam, gphi, 4, 0.5, 20)
    rg, rxy = orc.direct_grad(xy, gam, gphi)
    assert np.abs(gg - rg).max() <= 1e-8 * np.abs(rg).max()
    assert np.abs(gxy - rxy).max() <= 1e-8 * np.abs(rxy).max()


# ---------------------------------------------------------------- separate evaluation points (eq 2.2)

def test_direct_points_closed_form():
    """Two sources and two evaluation points, summed by hand; an evaluation
    point on a source skips that source (x_j != y_t)."""
    import oracle

    src = np.array([[0.0, 0.0], [1.0, 0.0]])
    gam = np.array([2.0 + 1.0j, -1.0 + 0.5j])
    tgt = np.array([[0.0, 1.0], [1.0, 0.0]])
    y0 = 0.0 + 1.0j
    want0 = (2.0 + 1.0j) / (y0 - 0.0) + (-1.0 + 0.5j) / (y0 - 1.0)
    want1 = (2.0 + 1.0j) / (1.0 - 0.0)  # the second source coincides with the point
    got = oracle.direct_points(src, gam, tgt)
    assert abs(got[0] - want0) < 1e-15 and abs(got[1] - want1) < 1e-15


def test_direct_points_equals_direct_on_the_sources():
    """With the evaluation points equal to the sources, eq (2.2) is eq (2.1)."""
    import oracle

    g = np.random.default_rng(11)
    xy = g.random((300, 2))
    gam = g.standard_normal(300) + 1j * g.standard_normal(300)
    a = oracle.direct_points(xy, gam, xy)
    b = oracle.direct(xy, gam)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))


# ---------------------------------------------------------------- logarithmic kernel

def test_direct_log_closed_form():
    import oracle

    xy = np.array([[0.0, 0.0], [3.0, 4.0], [0.0, 1.0]])
    gam = np.array([1.0 + 2.0j, -0.5, 2.0j])
    got = oracle.direct_log(xy, gam)
    want0 = -0.5 * np.log(5.0) + 2.0j * np.log(1.0)
    want1 = (1.0 + 2.0j) * np.log(5.0) + 2.0j * np.log(np.hypot(3.0, 3.0))
    want2 = (1.0 + 2.0j) * np.log(1.0) - 0.5 * np.log(np.hypot(3.0, 3.0))
    assert np.allclose(got, [want0, want1, want2], rtol=0, atol=1e-15)


def test_direct_log_gradient_is_the_harmonic_field():
    """d/dx sum_j q_j ln|y - x_j| = Re sum_j q_j / (y - x_j) and d/dy = -Im of it
    (real q): central differences of the log sum against the harmonic direct sum."""
    import oracle

    g = np.random.default_rng(31)
    src = g.random((200, 2))
    q = g.standard_normal(200).astype(np.complex128)
    y = np.array([0.37, 0.61])
    h = 1e-6

    def pot(pt):
        xy = np.vstack([src, pt[None, :]])
        return oracle.direct_log(xy, np.concatenate([q, [0.0]]), targets=[200])[0].real

    dx = (pot(y + [h, 0]) - pot(y - [h, 0])) / (2 * h)
    dy = (pot(y + [0, h]) - pot(y - [0, h])) / (2 * h)
    hm = oracle.direct_points(src, q, y[None, :])[0]
    assert abs(dx - hm.real) <= 1e-6 * abs(hm) and abs(dy + hm.imag) <= 1e-6 * abs(hm)


def test_fmm_log_converges_geometrically_and_one_level_is_direct():
    import oracle

    g = np.random.default_rng(32)
    xy = g.random((3000, 2))
    gam = g.standard_normal(3000) + 1j * g.standard_normal(3000)
    ex = oracle.direct_log(xy, gam)
    errs = [np.max(np.abs(oracle.fmm_log(xy, gam, 5, 0.5, p) - ex)) / np.max(np.abs(ex)) for p in (6, 10, 14, 18)]
    assert all(b < 0.2 * a for a, b in zip(errs, errs[1:])), errs  # geometric in p (theta = 0.5)
    assert errs[-1] < 1e-8
    assert np.max(np.abs(oracle.fmm_log(xy, gam, 1, 0.5, 6) - ex)) <= 1e-13 * np.max(np.abs(ex))
