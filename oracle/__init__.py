"""The oracle: plain FP64 CPU statement of the balanced adaptive 2D FMM.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The library (``paper_1311_1006_b300``) never imports it and shares no
code with it; the C source is ``fmm_oracle.c`` (see its header for the
formulas, each tied to the paper's Sec. 2 / eq 2.1-2.5, and for the readings of
the points the paper leaves open).

All complex arrays are numpy ``complex128``; points are an ``(n, 2)`` float64
array of (x, y).  Outputs are in the caller's (original) point order.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_fmm.so")
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (FP contraction off)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.fo_num_boxes.restype = _I64
        lib.fo_num_boxes.argtypes = [ctypes.c_int]
        lib.fo_set_threads.argtypes = [ctypes.c_int]
        lib.fo_max_threads.restype = ctypes.c_int
        lib.fo_direct.argtypes = [_I64, _P, _P, _I64, _P, _P, _P]
        lib.fo_direct_grad.argtypes = [_I64, _P, _P, _P, _I64, _P, _P, _P]
        lib.fo_direct_points.argtypes = [_I64, _P, _P, _I64, _P, _P]
        lib.fo_direct_log.argtypes = [_I64, _P, _P, _I64, _P, _P]
        lib.fo_fmm_log.restype = ctypes.c_int
        lib.fo_fmm_log.argtypes = [_I64, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P]
        lib.fo_build_tree.restype = ctypes.c_int
        lib.fo_build_tree.argtypes = [_I64, _P, ctypes.c_int, _P, _P, _P, _P, _P]
        lib.fo_build_lists.restype = ctypes.c_int
        lib.fo_build_lists.argtypes = [ctypes.c_int, _P, _P, ctypes.c_double, _P, _P, _P, _P]
        lib.fo_fmm.restype = ctypes.c_int
        lib.fo_fmm.argtypes = [_I64, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                               _P, _P, _P, _P, _P, _P]
        lib.fo_fmm_grad.restype = ctypes.c_int
        lib.fo_fmm_grad.argtypes = [_I64, _P, _P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, _P]
        for name in ("fo_p2m", "fo_m2m", "fo_m2l", "fo_l2l", "fo_l2p", "fo_p2p"):
            getattr(lib, name).restype = None
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _xy(xy):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    assert xy.ndim == 2 and xy.shape[1] == 2
    return xy


def _cx(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if n is not None:
        assert a.shape == (n,)
    return a


def set_threads(t: int) -> None:
    _load().fo_set_threads(int(t))


def max_threads() -> int:
    return int(_load().fo_max_threads())


def num_boxes(nlevels: int) -> int:
    return int(_load().fo_num_boxes(int(nlevels)))


def direct(xy, gamma, targets=None, deriv: bool = False):
    """Exact eq (2.2) sum at ``targets`` (all points when None); optional d/dz."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    m = n if tg is None else tg.shape[0]
    phi = np.zeros(m, np.complex128)
    dphi = np.zeros(m, np.complex128) if deriv else None
    lib.fo_direct(n, _ptr(xy), _ptr(gamma), m, _ptr(tg), _ptr(phi), _ptr(dphi))
    return (phi, dphi) if deriv else phi


def direct_points(src_xy, gamma, tgt_xy):
    """Exact eq (2.2) sum at separate evaluation points ``tgt_xy`` (M x 2):
    Phi(y_t) = sum_{j: x_j != y_t} Gamma_j / (y_t - x_j)."""
    lib = _load()
    sxy, txy = _xy(src_xy), _xy(tgt_xy)
    n, m = sxy.shape[0], txy.shape[0]
    gamma = _cx(gamma, n)
    phi = np.zeros(m, np.complex128)
    lib.fo_direct_points(n, _ptr(sxy), _ptr(gamma), m, _ptr(txy), _ptr(phi))
    return phi


def direct_log(xy, gamma, targets=None):
    """Exact logarithmic potential sum_{j: z_j != z_t} Gamma_j ln|z_t - z_j| at ``targets``."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    m = n if tg is None else tg.shape[0]
    phi = np.zeros(m, np.complex128)
    lib.fo_direct_log(n, _ptr(xy), _ptr(gamma), m, _ptr(tg), _ptr(phi))
    return phi


def fmm_log(xy, gamma, nlevels: int, theta: float, p: int):
    """One oracle FMM evaluation of the logarithmic potential (complex strengths
    on the real kernel ln|z - z_j|)."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    phi = np.zeros(n, np.complex128)
    rc = lib.fo_fmm_log(n, _ptr(xy), _ptr(gamma), int(nlevels), float(theta), int(p), _ptr(phi))
    if rc != 0:
        raise ValueError(f"oracle fmm_log failed ({rc})")
    return phi


def direct_grad(xy, gamma, gphi, targets=None):
    """Exact gradient of L = sum_i Re(conj(gphi_i) Phi_i) at ``targets``.

    Returns (dL/dRe Gamma + i dL/dIm Gamma, dL/d(x, y)) for the target points."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    gphi = _cx(gphi, n)
    tg = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    m = n if tg is None else tg.shape[0]
    gg = np.zeros(m, np.complex128)
    gxy = np.zeros((m, 2), np.float64)
    lib.fo_direct_grad(n, _ptr(xy), _ptr(gamma), _ptr(gphi), m, _ptr(tg), _ptr(gg), _ptr(gxy))
    return gg, gxy


def build_tree(xy, nlevels: int):
    """Pyramid tree by exact median splits; see fo_build_tree."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    nb = num_boxes(nlevels)
    perm = np.zeros(n, np.int64)
    bstart = np.zeros(nb, np.int64)
    bcount = np.zeros(nb, np.int64)
    center = np.zeros((nb, 2), np.float64)
    radius = np.zeros(nb, np.float64)
    rc = lib.fo_build_tree(n, _ptr(xy), int(nlevels), _ptr(perm), _ptr(bstart), _ptr(bcount),
                           _ptr(center), _ptr(radius))
    if rc != 0:
        raise ValueError(f"oracle tree build failed ({rc}) for n={n}, nlevels={nlevels}")
    return dict(perm=perm, bstart=bstart, bcount=bcount, center=center, radius=radius, nlevels=int(nlevels))


def build_lists(nlevels: int, center, radius, theta: float):
    """Strong / weak CSR lists of every box (global box ids, sorted per box)."""
    lib = _load()
    nb = num_boxes(nlevels)
    center = np.ascontiguousarray(center, dtype=np.float64)
    radius = np.ascontiguousarray(radius, dtype=np.float64)
    s_off = np.zeros(nb + 1, np.int64)
    w_off = np.zeros(nb + 1, np.int64)
    rc = lib.fo_build_lists(int(nlevels), _ptr(center), _ptr(radius), float(theta), _ptr(s_off), _ptr(w_off),
                            None, None)
    if rc != 0:
        raise MemoryError("oracle list build failed")
    s_idx = np.zeros(max(int(s_off[-1]), 1), np.int32)
    w_idx = np.zeros(max(int(w_off[-1]), 1), np.int32)
    lib.fo_build_lists(int(nlevels), _ptr(center), _ptr(radius), float(theta), _ptr(s_off), _ptr(w_off),
                       _ptr(s_idx), _ptr(w_idx))
    return dict(s_off=s_off, s_idx=s_idx[: s_off[-1]], w_off=w_off, w_idx=w_idx[: w_off[-1]])


def fmm(xy, gamma, nlevels: int, theta: float, p: int, deriv: bool = False, parts: bool = False):
    """One oracle FMM evaluation.  Returns a dict with ``phi`` (and ``dphi``,
    ``near``, ``far``, unscaled ``mpole`` / ``local`` of shape (nbox, p) when
    asked)."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    nb = num_boxes(nlevels)
    phi = np.zeros(n, np.complex128)
    dphi = np.zeros(n, np.complex128) if deriv else None
    mp = np.zeros((nb, p), np.complex128) if parts else None
    lo = np.zeros((nb, p), np.complex128) if parts else None
    ne = np.zeros(n, np.complex128) if parts else None
    fa = np.zeros(n, np.complex128) if parts else None
    rc = lib.fo_fmm(n, _ptr(xy), _ptr(gamma), int(nlevels), float(theta), int(p), _ptr(phi), _ptr(dphi),
                    _ptr(mp), _ptr(lo), _ptr(ne), _ptr(fa))
    if rc != 0:
        raise ValueError(f"oracle fmm failed ({rc})")
    out = dict(phi=phi)
    if deriv:
        out["dphi"] = dphi
    if parts:
        out.update(mpole=mp, local=lo, near=ne, far=fa)
    return out


def fmm_grad(xy, gamma, gphi, nlevels: int, theta: float, p: int):
    """Gradient of L = sum_i Re(conj(gphi_i) Phi_i) through the oracle FMM."""
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    gphi = _cx(gphi, n)
    gg = np.zeros(n, np.complex128)
    gxy = np.zeros((n, 2), np.float64)
    rc = lib.fo_fmm_grad(n, _ptr(xy), _ptr(gamma), _ptr(gphi), int(nlevels), float(theta), int(p), _ptr(gg),
                         _ptr(gxy))
    if rc != 0:
        raise ValueError(f"oracle fmm_grad failed ({rc})")
    return gg, gxy


# Per-pass entry points for the per-kernel parity tests.

def p2m(tree, xy, gamma, p):
    lib = _load()
    xy = _xy(xy)
    gamma = _cx(gamma, xy.shape[0])
    nb = num_boxes(tree["nlevels"])
    mp = np.zeros((nb, p), np.complex128)
    lib.fo_p2m(ctypes.c_int(tree["nlevels"]), ctypes.c_int(p), _ptr(xy), _ptr(gamma), _ptr(tree["perm"]),
               _ptr(tree["bstart"]), _ptr(tree["bcount"]), _ptr(tree["center"]), _ptr(mp))
    return mp


def m2m(tree, mpole):
    """In place on a copy: fills every non-leaf box from its children."""
    lib = _load()
    mp = np.ascontiguousarray(mpole, dtype=np.complex128).copy()
    lib.fo_m2m(ctypes.c_int(tree["nlevels"]), ctypes.c_int(mp.shape[1]), _ptr(tree["center"]), _ptr(mp))
    return mp


def m2l(tree, lists, mpole):
    lib = _load()
    mp = np.ascontiguousarray(mpole, dtype=np.complex128)
    lo = np.zeros_like(mp)
    lib.fo_m2l(ctypes.c_int(tree["nlevels"]), ctypes.c_int(mp.shape[1]), _ptr(tree["center"]),
               _ptr(lists["w_off"]), _ptr(np.ascontiguousarray(lists["w_idx"])), _ptr(mp), _ptr(lo))
    return lo


def l2l(tree, local):
    lib = _load()
    lo = np.ascontiguousarray(local, dtype=np.complex128).copy()
    lib.fo_l2l(ctypes.c_int(tree["nlevels"]), ctypes.c_int(lo.shape[1]), _ptr(tree["center"]), _ptr(lo))
    return lo


def l2p(tree, xy, local, deriv=False):
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    lo = np.ascontiguousarray(local, dtype=np.complex128)
    phi = np.zeros(n, np.complex128)
    dphi = np.zeros(n, np.complex128) if deriv else None
    lib.fo_l2p(ctypes.c_int(tree["nlevels"]), ctypes.c_int(lo.shape[1]), _ptr(xy), _ptr(tree["perm"]),
               _ptr(tree["bstart"]), _ptr(tree["bcount"]), _ptr(tree["center"]), _ptr(lo), _ptr(phi), _ptr(dphi))
    return (phi, dphi) if deriv else phi


def p2p(tree, lists, xy, gamma, deriv=False):
    lib = _load()
    xy = _xy(xy)
    n = xy.shape[0]
    gamma = _cx(gamma, n)
    phi = np.zeros(n, np.complex128)
    dphi = np.zeros(n, np.complex128) if deriv else None
    lib.fo_p2p(ctypes.c_int(tree["nlevels"]), _ptr(xy), _ptr(gamma), _ptr(tree["perm"]), _ptr(tree["bstart"]),
               _ptr(tree["bcount"]), _ptr(lists["s_off"]), _ptr(np.ascontiguousarray(lists["s_idx"])), _ptr(phi),
               _ptr(dphi))
    return (phi, dphi) if deriv else phi
