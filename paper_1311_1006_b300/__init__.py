"""B300 (sm_103a) balanced adaptive 2D FMM for the harmonic potential.

    Phi(z_i) = sum_{j : z_j != z_i} Gamma_j / (z_i - z_j)      (eq 2.1 / 2.2)

The method is the balanced adaptive FMM of Holm, Engblom, Goude, Holmgren
(arXiv:1311.1006): a pyramid tree with median splits (Sec. 2.2-2.3), coupling by
the theta-criterion (eq 2.3), P2M / M2M / M2L / L2L / L2P / P2P passes
(Sec. 2.1), an N_levels autotuner (Sec. 4.2, Algorithm 4) and, added here, a
hand-written adjoint and batched instances.

This module is a thin binding over the C ABI of ``libfmm2d.so`` (same names,
argument marshalling only).  PyTorch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (FMM_FLAG_GRAPH, FMM_FLAG_NO_GRAPH, FMM_FLAG_PERSISTENT, FMM_FLAG_SERIAL, FMM_FLAG_TIMING,
                   FMM_PATH_FP32, FMM_PATH_FP64, FMMError, FMMParams)

__all__ = ["Tree", "FMMFunction", "fmm", "default_nlevels", "seed_nlevels", "cost_model", "set_cost_model",
           "p_for_tolerance", "Autotuner", "FMMError", "FMM_PATH_FP32",
           "FMM_PATH_FP64", "FMM_FLAG_GRAPH", "FMM_FLAG_NO_GRAPH", "FMM_FLAG_PERSISTENT", "FMM_FLAG_SERIAL",
           "FMM_FLAG_TIMING"]


def _torch():
    import torch

    return torch


def _path(path) -> int:
    if path in (FMM_PATH_FP32, "fp32", "mixed"):
        return FMM_PATH_FP32
    if path in (FMM_PATH_FP64, "fp64"):
        return FMM_PATH_FP64
    raise ValueError(f"unknown path {path!r}")


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, shape=None, name="tensor"):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def default_nlevels(n: int, p: int = 17, path="fp32") -> int:
    """fmm_default_nlevels: the cost-model seed with the library's unit costs of `path`."""
    return int(_lib.load().fmm_default_nlevels(int(n), int(p), _path(path)))


def seed_nlevels(n: int, p: int, alpha: float, beta: float) -> int:
    """fmm_seed_nlevels: N_levels whose N_f is closest to (N/p) sqrt(alpha/(3 beta))."""
    return int(_lib.load().fmm_seed_nlevels(int(n), int(p), float(alpha), float(beta)))


def cost_model(path="fp32") -> tuple:
    """fmm_cost_model_get: the library's unit costs (alpha, beta) of `path`."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _lib.check(_lib.load().fmm_cost_model_get(_path(path), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def set_cost_model(alpha: float, beta: float, path="fp32") -> None:
    """fmm_cost_model_set."""
    _lib.check(_lib.load().fmm_cost_model_set(_path(path), float(alpha), float(beta)))


class Tree:
    """A device-resident FMM tree (tree + coupling lists + workspace)."""

    def __init__(self, handle, n, params: FMMParams, batched=False, ninst=1, n_src=0, n_tgt=0):
        self._h = handle
        self.n = int(n)
        self.params = params
        self.batched = batched
        self.ninst = ninst
        self.n_src, self.n_tgt = int(n_src), int(n_tgt)

    # -- construction -------------------------------------------------------
    @classmethod
    def build(cls, xy, p=17, theta=0.5, nlevels=0, path="fp32", flags=0, stream=None) -> "Tree":
        """fmm_build_tree: xy is an (N, 2) float64 CUDA tensor."""
        torch = _torch()
        lib = _lib.load()
        n = xy.shape[0]
        ptr = _dev(xy, torch.float64, (n, 2), "xy")
        prm = FMMParams(int(p), float(theta), int(nlevels), _path(path), int(flags))
        h = ctypes.c_void_p()
        _lib.check(lib.fmm_build_tree(ptr, n, ctypes.byref(prm), _stream(stream), ctypes.byref(h)))
        return cls(h, n, prm)

    @classmethod
    def build_targets(cls, src_xy, tgt_xy, p=17, theta=0.5, nlevels=0, path="fp32", flags=0,
                      stream=None) -> "Tree":
        """fmm_build_tree_targets: sources (N, 2) and separate evaluation points (M, 2), float64 CUDA."""
        torch = _torch()
        lib = _lib.load()
        ns, nt = src_xy.shape[0], tgt_xy.shape[0]
        ps = _dev(src_xy, torch.float64, (ns, 2), "src_xy")
        pt = _dev(tgt_xy, torch.float64, (nt, 2), "tgt_xy")
        prm = FMMParams(int(p), float(theta), int(nlevels), _path(path), int(flags))
        h = ctypes.c_void_p()
        _lib.check(lib.fmm_build_tree_targets(ps, ns, pt, nt, ctypes.byref(prm), _stream(stream), ctypes.byref(h)))
        return cls(h, ns + nt, prm, n_src=ns, n_tgt=nt)

    def rebuild_targets(self, src_xy, tgt_xy, nlevels=None, p=None, theta=None, path=None, flags=None,
                        stream=None) -> None:
        """fmm_tree_rebuild_targets for new source / evaluation-point coordinates."""
        torch = _torch()
        ps = _dev(src_xy, torch.float64, (self.n_src, 2), "src_xy")
        pt = _dev(tgt_xy, torch.float64, (self.n_tgt, 2), "tgt_xy")
        prm = FMMParams(self.params.p if p is None else int(p),
                        self.params.theta if theta is None else float(theta),
                        0 if nlevels is None else int(nlevels),
                        self.params.path if path is None else _path(path),
                        self.params.flags if flags is None else int(flags))
        _lib.check(_lib.load().fmm_tree_rebuild_targets(self._h, ps, pt, ctypes.byref(prm), _stream(stream)))
        self.params = prm

    @classmethod
    def build_batched(cls, xy, offsets, nlevels=None, p=17, theta=0.5, path="fp32", flags=0,
                      stream=None) -> "Tree":
        """fmm_build_tree_batched: instance b owns xy[offsets[b]:offsets[b+1]]."""
        torch = _torch()
        lib = _lib.load()
        n = xy.shape[0]
        ptr = _dev(xy, torch.float64, (n, 2), "xy")
        offs = np.ascontiguousarray(offsets, dtype=np.int64)
        B = offs.shape[0] - 1
        if offs[-1] != n:
            raise ValueError("offsets[-1] must equal the number of points")
        prm = FMMParams(int(p), float(theta), 0, _path(path), int(flags))
        nl = None
        if nlevels is not None:
            nl = np.ascontiguousarray(nlevels, dtype=np.int32)
            if nl.shape[0] != B:
                raise ValueError("one nlevels entry per instance")
        h = ctypes.c_void_p()
        _lib.check(lib.fmm_build_tree_batched(
            ptr, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), B, ctypes.byref(prm),
            None if nl is None else nl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _stream(stream),
            ctypes.byref(h)))
        return cls(h, n, prm, batched=True, ninst=B)

    def rebuild(self, xy, nlevels=None, p=None, theta=None, path=None, flags=None, stream=None) -> None:
        """fmm_tree_rebuild for new coordinates (and optionally new parameters)."""
        torch = _torch()
        ptr = _dev(xy, torch.float64, (self.n, 2), "xy")
        prm = FMMParams(self.params.p if p is None else int(p),
                        self.params.theta if theta is None else float(theta),
                        0 if nlevels is None else int(nlevels),
                        self.params.path if path is None else _path(path),
                        self.params.flags if flags is None else int(flags))
        _lib.check(_lib.load().fmm_tree_rebuild(self._h, ptr, ctypes.byref(prm), _stream(stream)))
        self.params = prm

    # -- evaluation ---------------------------------------------------------
    @property
    def out_dtype(self):
        torch = _torch()
        return torch.complex64 if self.params.path == FMM_PATH_FP32 else torch.complex128

    def eval(self, gamma, out=None, stream=None):
        """fmm_eval: gamma is an (N,) complex128 CUDA tensor; returns Phi."""
        torch = _torch()
        g = _dev(gamma, torch.complex128, (self.n,), "gamma")
        if out is None:
            out = torch.empty(self.n, dtype=self.out_dtype, device=gamma.device)
        o = _dev(out, self.out_dtype, (self.n,), "out")
        fn = _lib.load().fmm_eval_batched if self.batched else _lib.load().fmm_eval
        _lib.check(fn(self._h, g, o, _stream(stream)))
        return out

    def step(self, xy, gamma, out=None, stream=None):
        """fmm_step: rebuild for new coordinates and evaluate in one call (the upward
        pass overlaps the list build); same result as rebuild() + eval()."""
        torch = _torch()
        p = _dev(xy, torch.float64, (self.n, 2), "xy")
        g = _dev(gamma, torch.complex128, (self.n,), "gamma")
        if out is None:
            out = torch.empty(self.n, dtype=self.out_dtype, device=gamma.device)
        o = _dev(out, self.out_dtype, (self.n,), "out")
        _lib.check(_lib.load().fmm_step(self._h, p, g, o, _stream(stream)))
        return out

    def eval_log(self, gamma, out=None, stream=None):
        """fmm_eval_log: the logarithmic potential sum_j Gamma_j ln|z_i - z_j| (Sec. 3.3)."""
        torch = _torch()
        g = _dev(gamma, torch.complex128, (self.n,), "gamma")
        if out is None:
            out = torch.empty(self.n, dtype=self.out_dtype, device=gamma.device)
        o = _dev(out, self.out_dtype, (self.n,), "out")
        _lib.check(_lib.load().fmm_eval_log(self._h, g, o, _stream(stream)))
        return out

    def _eval_targets(self, fn, gamma, out, stream):
        torch = _torch()
        g = _dev(gamma, torch.complex128, (self.n_src,), "gamma")
        if out is None:
            out = torch.empty(self.n_tgt, dtype=self.out_dtype, device=gamma.device)
        o = _dev(out, self.out_dtype, (self.n_tgt,), "out")
        _lib.check(fn(self._h, g, o, _stream(stream)))
        return out

    def eval_targets(self, gamma, out=None, stream=None):
        """fmm_eval_targets: gamma = (N_src,) complex128 source strengths; returns Phi at the evaluation points."""
        return self._eval_targets(_lib.load().fmm_eval_targets, gamma, out, stream)

    def eval_targets_log(self, gamma, out=None, stream=None):
        """fmm_eval_targets_log: the logarithmic potential at the evaluation points."""
        return self._eval_targets(_lib.load().fmm_eval_targets_log, gamma, out, stream)

    def backward(self, gamma, gphi, stream=None):
        """fmm_eval_backward: returns (dL/dGamma complex128, dL/d(x,y) float64 (N,2))."""
        torch = _torch()
        g = _dev(gamma, torch.complex128, (self.n,), "gamma")
        gp = gphi.to(torch.complex128).contiguous()
        gpp = _dev(gp, torch.complex128, (self.n,), "gphi")
        gg = torch.empty(self.n, dtype=torch.complex128, device=gamma.device)
        gxy = torch.empty(self.n, 2, dtype=torch.float64, device=gamma.device)
        _lib.check(_lib.load().fmm_eval_backward(self._h, g, gpp, ctypes.c_void_p(gg.data_ptr()),
                                                 ctypes.c_void_p(gxy.data_ptr()), _stream(stream)))
        return gg, gxy

    # -- diagnostics --------------------------------------------------------
    def info(self) -> dict:
        inf = _lib.FMMTreeInfo()
        _lib.check(_lib.load().fmm_get_tree_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in _lib.FMMTreeInfo._fields_}

    def export(self, what: str, stream=None) -> np.ndarray:
        """fmm_tree_export into a numpy array (tests, diagnostics)."""
        inf = self.info()
        nb, n, p = inf["nboxes"], inf["n"], inf["p"]
        spec = {
            "perm": (np.int32, n), "bstart": (np.int32, nb), "bcount": (np.int32, nb),
            "center": (np.float64, 2 * nb), "radius": (np.float64, nb), "rho": (np.float64, nb),
            "nstrong": (np.int32, nb), "strong": (np.int32, max(inf["n_strong"], 1)),
            "nweak": (np.int32, nb), "weak": (np.int32, max(inf["n_weak"], 1)),
            "soff": (np.int32, nb), "woff": (np.int32, nb),
            "mpole": (np.float64, 2 * nb * p), "local": (np.float64, 2 * nb * p),
            "near": (np.float64, 2 * n), "inst": (np.int64, 3 * inf["ninst"]),
            "m2l_items": (np.int32, max(4 * inf["m2l_items"], 1)), "m2l_rows": (np.int32, max(inf["m2l_items"], 1)),
            "p2p_items": (np.int32, max(4 * inf["p2p_items"], 1)), "p2p_rows": (np.int32, max(inf["p2p_items"], 1)),
        }[what]
        buf = np.zeros(spec[1], dtype=spec[0])
        _lib.check(_lib.load().fmm_tree_export(self._h, _lib.EXPORT[what], ctypes.c_void_p(buf.ctypes.data),
                                               buf.shape[0], _stream(stream)))
        if what == "center":
            return buf.reshape(nb, 2)
        if what in ("mpole", "local"):
            return buf.view(np.complex128).reshape(nb, p)
        if what == "near":
            return buf.view(np.complex128)
        if what == "inst":
            return buf.reshape(-1, 3)
        if what == "m2l_items":
            return buf[: 4 * inf["m2l_items"]].reshape(-1, 4)
        if what == "m2l_rows":
            return buf[: inf["m2l_items"]]
        if what == "p2p_items":
            return buf[: 4 * inf["p2p_items"]].reshape(-1, 4)
        if what == "p2p_rows":
            return buf[: inf["p2p_items"]]
        return buf

    def lists(self):
        """Strong and weak lists of every box as (list of arrays, list of arrays)."""
        ns, so, si = self.export("nstrong"), self.export("soff"), self.export("strong")
        nw, wo, wi = self.export("nweak"), self.export("woff"), self.export("weak")
        strong = [si[so[b]: so[b] + ns[b]] for b in range(ns.shape[0])]
        weak = [wi[wo[b]: wo[b] + nw[b]] for b in range(nw.shape[0])]
        return strong, weak

    def eval_status(self, stream=None) -> None:
        """fmm_eval_status: raises FMMError (timeout) if a bounded wait of the last evaluation ran out."""
        _lib.check(_lib.load().fmm_eval_status(self._h, _stream(stream)))

    def phase_times(self) -> dict:
        out = (ctypes.c_double * 7)()
        _lib.check(_lib.load().fmm_phase_times(self._h, out, 7))
        keys = ["gather", "p2m_m2m", "m2l", "l2l", "p2p", "l2p", "total"]
        return dict(zip(keys, list(out)))

    def calibrate_cost_model(self) -> tuple:
        """fmm_cost_model_calibrate: unit costs (alpha, beta) from the last timed
        evaluation, which become the library's cost model for this tree's path."""
        a, b = ctypes.c_double(), ctypes.c_double()
        _lib.check(_lib.load().fmm_cost_model_calibrate(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def autotune_config(self, cap=0.1, window=3, period=8) -> None:
        _lib.check(_lib.load().fmm_autotune_config(self._h, float(cap), int(window), int(period)))

    def autotune_step(self, seconds: float) -> int:
        prm = FMMParams(self.params.p, self.params.theta, 0, self.params.path, self.params.flags)
        _lib.check(_lib.load().fmm_autotune_step(self._h, float(seconds), ctypes.byref(prm)))
        return int(prm.nlevels)

    def autotune_theta(self, tol: float, theta_min=0.35, theta_max=0.65) -> None:
        """Tune theta as well (p follows from tol); see autotune_params."""
        _lib.check(_lib.load().fmm_autotune_theta(self._h, float(tol), float(theta_min), float(theta_max)))

    def autotune_params(self, seconds: float) -> tuple:
        """One tuner step; returns (nlevels, theta, p) to rebuild with."""
        prm = FMMParams(self.params.p, self.params.theta, 0, self.params.path, self.params.flags)
        _lib.check(_lib.load().fmm_autotune_step(self._h, float(seconds), ctypes.byref(prm)))
        return int(prm.nlevels), float(prm.theta), int(prm.p)

    def close(self) -> None:
        if getattr(self, "_h", None):
            _lib.load().fmm_tree_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def p_for_tolerance(tol: float, theta: float) -> int:
    """fmm_p_for_tolerance: expansion terms for tolerance tol at separation theta."""
    return int(_lib.load().fmm_p_for_tolerance(float(tol), float(theta)))


class Autotuner:
    """Standalone AT3b autotuner (fmm_autotuner_*): N_levels, optionally theta."""

    def __init__(self, nlevels: int, max_levels: int, cap=0.1, window=3, period=8):
        lib = _lib.load()
        self._h = ctypes.c_void_p()
        _lib.check(lib.fmm_autotuner_create(int(nlevels), int(max_levels), float(cap), int(window), int(period),
                                            ctypes.byref(self._h)))

    def step(self, seconds: float) -> int:
        out = ctypes.c_int()
        _lib.check(_lib.load().fmm_autotuner_step(self._h, float(seconds), ctypes.byref(out)))
        return int(out.value)

    def enable_theta(self, theta: float, tol: float, theta_min=0.35, theta_max=0.65) -> None:
        _lib.check(_lib.load().fmm_autotuner_theta(self._h, float(theta), float(tol), float(theta_min),
                                                   float(theta_max)))

    def step_params(self, seconds: float) -> tuple:
        """(nlevels, theta, p) to use next."""
        nl, th, pp = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _lib.check(_lib.load().fmm_autotuner_step_params(self._h, float(seconds), ctypes.byref(nl), ctypes.byref(th),
                                                         ctypes.byref(pp)))
        return int(nl.value), float(th.value), int(pp.value)

    def stats(self) -> dict:
        out = (ctypes.c_double * 8)()
        _lib.check(_lib.load().fmm_autotuner_stats(self._h, out, 8))
        return dict(zip(["accepted", "steps", "rejected", "tuning_cost", "basetime", "trial", "theta",
                         "theta_trial"], list(out)))

    def __del__(self):
        try:
            if self._h:
                _lib.load().fmm_autotuner_destroy(self._h)
                self._h = None
        except Exception:
            pass


def _make_function():
    torch = _torch()

    class FMMFunction(torch.autograd.Function):
        """Phi = FMM(xy, gamma) with the tree frozen; backward = fmm_eval_backward."""

        @staticmethod
        def forward(ctx, xy, gamma, tree):
            ctx.tree = tree
            ctx.xy_dtype = xy.dtype
            ctx.save_for_backward(gamma)
            return tree.eval(gamma.detach().contiguous())

        @staticmethod
        def backward(ctx, gphi):
            (gamma,) = ctx.saved_tensors
            gg, gxy = ctx.tree.backward(gamma.detach().contiguous(), gphi)
            # gradients in the dtypes of the inputs they belong to
            return gxy.to(ctx.xy_dtype), gg.to(gamma.dtype), None

    return FMMFunction


class _Lazy:
    _fn = None

    def __getattr__(self, k):
        if _Lazy._fn is None:
            _Lazy._fn = _make_function()
        return getattr(_Lazy._fn, k)


FMMFunction = _Lazy()


def fmm(xy, gamma, p=17, theta=0.5, nlevels=0, path="fp32"):
    """Differentiable one-shot evaluation: builds a tree for xy (frozen under
    autograd) and returns Phi with gradients for xy and gamma."""
    tree = Tree.build(xy.detach().contiguous(), p=p, theta=theta, nlevels=nlevels, path=path)
    return FMMFunction.apply(xy, gamma, tree)
