"""ctypes wrapper of the plain FP64 CPU oracle of the VEGAS+ iteration loop.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference leg may import this package; the product path
(paper_2408_09229_gb300) never does.  The oracle shares no code with the CUDA
library.  Every routine cites the passage of cuVegas (arXiv 2408.09229) it
follows in oracle_vegas.h / oracle_vegas.c.
"""
import ctypes
import math
import os

import numpy as np

from . import build_oracle

_lib = None

GAUSS_SUM, PRODUCT_PEAK, OSCILLATORY, SIN_EXP, LINEAR, COSINE, EXPONENTIAL, \
    ROOS_ARNOLD, MOROKOFF_CAFLISCH, MAP_DENSITY = range(10)


class _Config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nbins", ctypes.c_int),
                ("nstrat", ctypes.POINTER(ctypes.c_int)),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("points_f32", ctypes.c_int), ("problem_id", ctypes.c_uint32)]


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_integrand.argtypes = [i32, i32, P, i64, P, P]
        L.orc_integrand.restype = i32
        L.orc_log2r.argtypes = [f64]
        L.orc_log2r.restype = ctypes.c_float
        L.orc_exp2r.argtypes = [ctypes.c_float]
        L.orc_exp2r.restype = ctypes.c_float
        L.orc_cube_ell.argtypes = [f64, i64, f64]
        L.orc_cube_ell.restype = ctypes.c_float
        L.orc_quant_weight.argtypes = [ctypes.c_float, ctypes.c_float]
        L.orc_quant_weight.restype = ctypes.c_uint32
        L.orc_allocate.argtypes = [P, i64, i64, f64, P]
        L.orc_allocate.restype = i32
        L.orc_refine_axis.argtypes = [i32, f64, P, P, P]
        L.orc_refine_axis.restype = i32
        L.orc_combine.argtypes = [P, P, i32, i32, P]
        L.orc_combine_lagged.argtypes = [P, P, i32, i32, P]
        L.orc_ncubes.argtypes = [ctypes.POINTER(_Config)]
        L.orc_ncubes.restype = i64
        L.orc_default_nstrat.argtypes = [i64, i32]
        L.orc_default_nstrat.restype = i32
        L.orc_fill_range.argtypes = [ctypes.POINTER(_Config), i32, P, i64, i64, i32, ctypes.c_uint64,
                                     P, P, i64, i64, P, P, P, P]
        L.orc_fill_range.restype = i32
        L.orc_cube_stats.argtypes = [ctypes.POINTER(_Config), i32, P, i64, i32, ctypes.c_uint64, P, i64, i64, i64,
                                     P, P]
        L.orc_cube_stats.restype = i32
        L.orc_finish_cubes.argtypes = [ctypes.POINTER(_Config), P, P, P, P, P, P]
        L.orc_iteration.argtypes = [ctypes.POINTER(_Config), i32, P, i64, i64, i32, ctypes.c_uint64,
                                    P, P, P, P, P, P, P, P, P, P]
        L.orc_iteration.restype = i32
        L.orc_integrate.argtypes = [ctypes.POINTER(_Config), i32, P, i64, i64, i32, i32, ctypes.c_uint64,
                                    P, P, P, P]
        L.orc_integrate.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def philox4x32_10(counter, key):
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def integrand(iid, x, params=()):
    x = np.ascontiguousarray(x, dtype=np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(1)
    out = np.zeros(1)
    rc = lib().orc_integrand(iid, x.size, _ptr(p), len(params), _ptr(x), _ptr(out))
    if rc != 0:
        raise ValueError("bad integrand id or parameter count")
    return float(out[0])


def log2r(x):
    return lib().orc_log2r(float(x))


def exp2r(y):
    return lib().orc_exp2r(float(y))


def cube_ell(m2, n, beta):
    return lib().orc_cube_ell(float(m2), int(n), float(beta))


def quant_weight(ell, ell_max):
    return lib().orc_quant_weight(float(ell), float(ell_max))


def allocate(ell, ncubes, neval, beta):
    off = np.zeros(ncubes + 1, dtype=np.int64)
    e = None if ell is None else np.ascontiguousarray(ell, dtype=np.float32)
    rc = lib().orc_allocate(_ptr(e), ncubes, neval, beta, _ptr(off))
    if rc != 0:
        raise ValueError(f"orc_allocate failed: {rc}")
    return off


def refine_axis(w, edges, alpha):
    w = np.ascontiguousarray(w, dtype=np.float64)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    out = np.zeros_like(e)
    unchanged = lib().orc_refine_axis(w.size, alpha, _ptr(w), _ptr(e), _ptr(out))
    return out, bool(unchanged)


def combine(it_est, it_sig, skip=0, lagged=False):
    """Eqs. (8)-(9) (R9), or with lagged=True the weights of the previous iteration (R20)"""
    I = np.ascontiguousarray(it_est, dtype=np.float64)
    S = np.ascontiguousarray(it_sig, dtype=np.float64)
    out = np.zeros(4)
    (lib().orc_combine_lagged if lagged else lib().orc_combine)(_ptr(I), _ptr(S), I.size, skip, _ptr(out))
    return {"estimate": out[0], "sigma": out[1], "chi2_dof": out[2], "n_used": int(out[3])}


def default_nstrat(neval, dim):
    return lib().orc_default_nstrat(int(neval), int(dim))


class Config:
    """dim, nbins, per-axis nstrat, alpha, beta, point precision, problem id."""

    def __init__(self, dim, nbins, nstrat, alpha, beta, points_f32=False, problem_id=0):
        if isinstance(nstrat, int):
            nstrat = [nstrat] * dim
        self.dim, self.nbins, self.alpha, self.beta = dim, nbins, alpha, beta
        self.nstrat = np.ascontiguousarray(nstrat, dtype=np.int32)
        self.points_f32, self.problem_id = bool(points_f32), problem_id
        self._c = _Config(dim, nbins, self.nstrat.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                          alpha, beta, int(points_f32), problem_id)

    @property
    def ncubes(self):
        return int(np.prod(self.nstrat.astype(np.int64)))

    def uniform_edges(self):
        e = np.arange(self.nbins + 1, dtype=np.float64) / self.nbins
        return np.tile(e, (self.dim, 1))


def fill_range(cfg, iid, params, neval, t, seed, edges, offsets, j_begin, j_end):
    p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(1)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    nh = cfg.ncubes
    cnt = np.zeros(nh, dtype=np.int64)
    mean = np.zeros(nh)
    m2 = np.zeros(nh)
    bins = np.zeros(cfg.dim * cfg.nbins)
    rc = lib().orc_fill_range(ctypes.byref(cfg._c), iid, _ptr(p), len(params), neval, t, seed, _ptr(e), _ptr(o),
                              j_begin, j_end, _ptr(cnt), _ptr(mean), _ptr(m2), _ptr(bins))
    if rc not in (0, -2):
        raise ValueError(f"orc_fill_range failed: {rc}")
    return cnt, mean, m2, bins.reshape(cfg.dim, cfg.nbins)


def cube_stats(cfg, iid, params, t, seed, edges, h, off_h, n_h):
    """mean and M2 of J f over the evaluations of one cube (Algorithm 2 on one cube)"""
    p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(1)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    mean, m2 = np.zeros(1), np.zeros(1)
    rc = lib().orc_cube_stats(ctypes.byref(cfg._c), iid, _ptr(p), len(params), t, seed, _ptr(e), int(h), int(off_h),
                              int(n_h), _ptr(mean), _ptr(m2))
    if rc not in (0, -2):
        raise ValueError(f"orc_cube_stats failed: {rc}")
    return float(mean[0]), float(m2[0])


def finish_cubes(cfg, offsets, mean, m2):
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    ell = np.zeros(cfg.ncubes, dtype=np.float32)
    I = np.zeros(1)
    V = np.zeros(1)
    lib().orc_finish_cubes(ctypes.byref(cfg._c), _ptr(o), _ptr(np.ascontiguousarray(mean)),
                           _ptr(np.ascontiguousarray(m2)), _ptr(ell), _ptr(I), _ptr(V))
    return float(I[0]), float(V[0]), ell


def iteration(cfg, iid, params, neval, t, seed, edges, offsets):
    """One Algorithm-1 iteration; returns a dict of every intermediate."""
    p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(1)
    e = np.ascontiguousarray(edges, dtype=np.float64)
    o = np.ascontiguousarray(offsets, dtype=np.int64)
    nh = cfg.ncubes
    mean, m2 = np.zeros(nh), np.zeros(nh)
    ell = np.zeros(nh, dtype=np.float32)
    bins = np.zeros(cfg.dim * cfg.nbins)
    e_next = np.zeros_like(e)
    o_next = np.zeros(nh + 1, dtype=np.int64)
    I, V = np.zeros(1), np.zeros(1)
    rc = lib().orc_iteration(ctypes.byref(cfg._c), iid, _ptr(p), len(params), neval, t, seed, _ptr(e), _ptr(o),
                             _ptr(mean), _ptr(m2), _ptr(ell), _ptr(bins), _ptr(e_next), _ptr(o_next),
                             _ptr(I), _ptr(V))
    if rc not in (0, -2):
        raise ValueError(f"orc_iteration failed: {rc}")
    return {"mean": mean, "m2": m2, "ell": ell, "bins": bins.reshape(cfg.dim, cfg.nbins),
            "edges_next": e_next, "offsets_next": o_next, "est": float(I[0]), "var": float(V[0]),
            "nonfinite": rc == -2}


def integrate(cfg, iid, params, neval, nitn, seed=0, skip=0):
    p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(1)
    it_est = np.zeros(nitn)
    it_sig = np.zeros(nitn)
    edges = np.zeros((cfg.dim, cfg.nbins + 1))
    out = np.zeros(4)
    rc = lib().orc_integrate(ctypes.byref(cfg._c), iid, _ptr(p), len(params), neval, nitn, skip, seed,
                             _ptr(it_est), _ptr(it_sig), _ptr(edges), _ptr(out))
    if rc not in (0, -2):
        raise ValueError(f"orc_integrate failed: {rc}")
    return {"estimate": out[0], "sigma": out[1], "chi2_dof": out[2], "n_used": int(out[3]),
            "it_est": it_est, "it_sig": it_sig, "edges": edges, "nonfinite": rc == -2}
