"""GB300 (sm_103a) VEGAS+ iteration loop: thin Python binding of the C ABI.

Every function here marshals arguments to the entry point of the same name
in libvegas_gb300.so (declared in include/vegas.h).  The compute runs only in
the library's CUDA kernels.  Importing this package fails loudly when the
library is missing; there is no CPU fallback.  Build the library with
``python -c "import __graft_entry__ as g; g.build()"`` or with
``python paper_2408_09229_gb300/build_lib.py``.

Device buffers for the step entry points are torch CUDA tensors.  torch is
used only for device memory and streams; the pointers go to the library.
"""
import ctypes
import os

import numpy as np

from .workloads import (GAUSS_SUM, PRODUCT_PEAK, OSCILLATORY, SIN_EXP, LINEAR, COSINE, EXPONENTIAL,  # noqa: F401
                        ROOS_ARNOLD, MOROKOFF_CAFLISCH, MAP_DENSITY)

HERE = os.path.dirname(os.path.abspath(__file__))
# VEGAS_GB300_LIB selects another build of the library, e.g. the bounds-checking libvegas_gb300_check.so
LIB_PATH = os.environ.get("VEGAS_GB300_LIB") or os.path.join(HERE, "libvegas_gb300.so")

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, ENOSPACE = 0, -1, -2, -3, -4, -5, -6, -7
FP64, FP32 = 0, 1
RESULT_CHI2_HIGH, RESULT_FLOW_OFF, RESULT_FLOW_KEPT, RESULT_FP32_FLOOR = 1, 2, 4, 8

# device memory hooks (vegas_alloc_fn, vegas_free_fn)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
WEIGHT_AUTO, WEIGHT_INVERSE_VARIANCE, WEIGHT_LAGGED = 0, 1, 2


class VegasError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})" if where else strerror(status))


class Result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
                ("neval_total", ctypes.c_int64), ("nitn_run", ctypes.c_int32), ("n_used", ctypes.c_int32),
                ("it_est", ctypes.POINTER(ctypes.c_double)), ("it_sigma", ctypes.POINTER(ctypes.c_double)),
                ("it_cap", ctypes.c_int32), ("flags", ctypes.c_int32), ("nitn_judge", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("judge_ratio", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("integrand", ctypes.c_int32), ("params", ctypes.c_void_p),
                ("nparams", ctypes.c_int64), ("neval", ctypes.c_int64), ("nstrat", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


class ProblemResult(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("sigma", ctypes.c_double), ("chi2_dof", ctypes.c_double),
                ("n_used", ctypes.c_int32), ("nitn_run", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("flags", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Geometry(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nbins", ctypes.c_int32), ("nstrat", ctypes.POINTER(ctypes.c_int32)),
                ("tile_log2", ctypes.c_int32), ("pad", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (paper_2408_09229_gb300/build_lib.py); "
                          "the VEGAS+ loop has no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64, f64, u64, u32 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                  ctypes.c_uint64, ctypes.c_uint32)
    sz = ctypes.c_size_t
    sig = {
        "vegas_create": ([i32, i32, i32, f64, f64, ctypes.POINTER(P)], i32),
        "vegas_destroy": ([P], i32),
        "vegas_set_nstrat_axes": ([P, P, i32], i32),
        "vegas_set_skip": ([P, i32], i32),
        "vegas_set_weighting": ([P, i32], i32),
        "vegas_set_precision": ([P, i32], i32),
        "vegas_set_stream": ([P, P], i32),
        "vegas_set_rtol": ([P, f64], i32),
        "vegas_reset_map": ([P], i32),
        "vegas_set_allocator": ([P, ALLOC_FN, FREE_FN, P], i32),
        "vegas_set_chi2_bound": ([P, f64], i32),
        "vegas_set_flow_judge": ([P, i32], i32),
        "vegas_integrate": ([P, i32, P, i64, i64, i32, u64, ctypes.POINTER(Result)], i32),
        "vegas_get_timings": ([P, P, P, i32, ctypes.POINTER(i32)], i32),
        "vegas_get_state": ([P, P, ctypes.POINTER(sz)], i32),
        "vegas_set_state": ([P, P, sz], i32),
        "vegas_get_edges": ([P, P, sz], i32),
        "vegas_strerror": ([i32], ctypes.c_char_p),
        "vegas_allocate_scratch_bytes": ([i64], sz),
        "vegas_allocate": ([P, i64, i64, i32, P, P, sz, P], i32),
        "vegas_allocate_static": ([P, i64, i64, i32, P, P], i32),
        "vegas_fill_scratch_bytes": ([ctypes.POINTER(Geometry), i64], sz),
        "vegas_fill": ([ctypes.POINTER(Geometry), i32, i32, P, i64, i64, u64, i32, u32, f64, P, P, P, P, P, P, P,
                        P, P, sz, P], i32),
        "vegas_refine": ([i32, i32, f64, P, P, P, P], i32),
        "vegas_combine": ([P, P, i32, i32, P, P], i32),
        "vegas_combine_weighted": ([P, P, i32, i32, i32, P, P], i32),
        "vegas_probe_pipes": ([P], i32),
        "vegas_probe_shared_atomics": ([P], i32),
        "vegas_probe_exp64": ([P], i32),
        "vegas_exp64_eval": ([P, P, i64, i32, P], i32),
        "vegas_batch_create": ([ctypes.POINTER(Problem), i32, i32, f64, f64, u64, ctypes.POINTER(P)], i32),
        "vegas_batch_create_ex": ([ctypes.POINTER(Problem), i32, i32, f64, f64, u64, ALLOC_FN, FREE_FN, P,
                                   ctypes.POINTER(P)], i32),
        "vegas_batch_destroy": ([P], i32),
        "vegas_batch_set_chi2_bound": ([P, f64], i32),
        "vegas_batch_set_stream": ([P, P], i32),
        "vegas_batch_set_skip": ([P, i32], i32),
        "vegas_batch_set_launch": ([P, i32, i32, i32], i32),
        "vegas_batch_set_tile": ([P, i32], i32),
        "vegas_batch_tune": ([P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                              ctypes.POINTER(ctypes.c_float)], i32),
        "vegas_batch_reset": ([P], i32),
        "vegas_batch_integrate": ([P, i32, f64, ctypes.POINTER(ProblemResult), ctypes.POINTER(i32),
                                   ctypes.POINTER(ctypes.c_float)], i32),
        "vegas_batch_get": ([P, i32, i32, P, i64], i32),
        "vegas_flow_param_count": ([i32], i64),
        "vegas_set_flow": ([P, P, i64], i32),
        "vegas_set_flow_training": ([P, i32, i32, i32, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float], i32),
        "vegas_get_flow": ([P, P, i64, P], i32),
        "vegas_flow_explore": ([P, i32, P, i64, i64, i32, i32, i64, i32, i32, ctypes.c_float, ctypes.c_float, i32,
                                u64], i32),
        "vegas_explore_points": ([i32, i32, i32, P, i64, u64, P, P, P], i32),
        "vegas_flow_apply": ([i32, i32, P, P, P, P, i64, P], i32),
        "vegas_flow_check": ([P], i32),
        "vegas_flow_wait_selftest": ([i32, i32, P], i32),
        "vegas_flow_grad_scratch_bytes": ([i32, i64], sz),
        "vegas_flow_grad": ([i32, P, P, P, i64, P, P, P, sz, P], i32),
        "vegas_flow_adam": ([i64, P, P, P, P, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


def strerror(status):
    return lib.vegas_strerror(status).decode()


def _check(status, where):
    if status != OK:
        raise VegasError(status, where)


def _ptr(t):
    """device pointer of a torch tensor (or None)"""
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def hooks(alloc, free):
    """ctypes function pointers for the device memory hooks: alloc(nbytes, stream) -> device address or 0,
    free(address, nbytes, stream).  Keep the returned pair alive while a handle or batch uses it."""
    if alloc is None and free is None:
        return ALLOC_FN(), FREE_FN()

    def _alloc(ctx, nbytes, stream):
        try:
            return int(alloc(int(nbytes), stream or 0)) or None
        except Exception:
            return None

    def _free(ctx, ptr, nbytes, stream):
        free(int(ptr), int(nbytes), stream or 0)

    return ALLOC_FN(_alloc), FREE_FN(_free)


def torch_hooks():
    """(alloc, free) through torch's CUDA caching allocator on the current device"""
    import torch

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, free


def _stream_ptr(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---------------------------------------------------------------------------
# Level 1: handle
# ---------------------------------------------------------------------------
class Vegas:
    """A VEGAS+ integrator on the current CUDA device (vegas_create ... vegas_destroy)."""

    def __init__(self, dim, nbins=50, nstrat=0, alpha=0.5, beta=0.75, precision=FP64, skip=0, rtol=0.0,
                 nstrat_axes=None, stream=None):
        h = ctypes.c_void_p()
        _check(lib.vegas_create(dim, nbins, nstrat, alpha, beta, ctypes.byref(h)), "vegas_create")
        self._h = h
        self.dim, self.nbins = dim, nbins
        self.set_precision(precision)
        self.set_skip(skip)
        self.set_rtol(rtol)
        if nstrat_axes is not None:
            self.set_nstrat_axes(nstrat_axes)
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            lib.vegas_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_precision(self, precision):
        _check(lib.vegas_set_precision(self._h, precision), "vegas_set_precision")

    def set_skip(self, skip):
        _check(lib.vegas_set_skip(self._h, skip), "vegas_set_skip")

    def set_weighting(self, weighting):
        """WEIGHT_AUTO (lagged with a flow, else Eq. (8)), WEIGHT_INVERSE_VARIANCE or WEIGHT_LAGGED"""
        _check(lib.vegas_set_weighting(self._h, weighting), "vegas_set_weighting")

    def set_rtol(self, rtol):
        _check(lib.vegas_set_rtol(self._h, rtol), "vegas_set_rtol")

    def set_stream(self, stream):
        _check(lib.vegas_set_stream(self._h, _stream_ptr(stream)), "vegas_set_stream")

    def set_nstrat_axes(self, nstrat):
        a = np.ascontiguousarray(nstrat, dtype=np.int32)
        _check(lib.vegas_set_nstrat_axes(self._h, a.ctypes.data_as(ctypes.c_void_p), a.size), "vegas_set_nstrat_axes")

    def reset_map(self):
        _check(lib.vegas_reset_map(self._h), "vegas_reset_map")

    def set_allocator(self, alloc=None, free=None):
        """vegas_set_allocator: alloc(nbytes, stream) -> device address (0 when it cannot), free(address, nbytes,
        stream); both None returns to cudaMalloc / cudaFree"""
        fa, ff = hooks(alloc, free)
        _check(lib.vegas_set_allocator(self._h, fa, ff, None), "vegas_set_allocator")
        self._hooks = (fa, ff)

    def set_chi2_bound(self, bound):
        _check(lib.vegas_set_chi2_bound(self._h, float(bound)), "vegas_set_chi2_bound")

    def set_flow_judge(self, window):
        """vegas_set_flow_judge: plain VEGAS+ beside the learned proposal until a decision over `window`
        iterations after training; 0 turns it off"""
        _check(lib.vegas_set_flow_judge(self._h, int(window)), "vegas_set_flow_judge")

    def integrate(self, integrand, params, neval, nitn, seed=0, check=True):
        p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(0)
        it_est = np.zeros(nitn)
        it_sig = np.zeros(nitn)
        r = Result()
        r.it_est = it_est.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.it_sigma = it_sig.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.it_cap = nitn
        st = lib.vegas_integrate(self._h, integrand, p.ctypes.data_as(ctypes.c_void_p) if p.size else None, p.size,
                                 int(neval), int(nitn), int(seed), ctypes.byref(r))
        if check and st not in (OK, ENONFINITE):
            raise VegasError(st, "vegas_integrate")
        n = r.nitn_run
        return {"estimate": r.estimate, "sigma": r.sigma, "chi2_dof": r.chi2_dof, "n_used": r.n_used,
                "nitn_run": n, "neval_total": r.neval_total, "it_est": it_est[:n], "it_sig": it_sig[:n],
                "status": st, "flags": r.flags, "nitn_judge": r.nitn_judge, "judge_ratio": r.judge_ratio}

    def timings(self, cap=4096):
        it = np.zeros(cap, dtype=np.float32)
        fl = np.zeros(cap, dtype=np.float32)
        n = ctypes.c_int32()
        _check(lib.vegas_get_timings(self._h, it.ctypes.data_as(ctypes.c_void_p), fl.ctypes.data_as(ctypes.c_void_p),
                                     cap, ctypes.byref(n)), "vegas_get_timings")
        m = min(n.value, cap)
        return it[:m].copy(), fl[:m].copy()

    def get_state(self):
        size = ctypes.c_size_t()
        _check(lib.vegas_get_state(self._h, None, ctypes.byref(size)), "vegas_get_state")
        buf = ctypes.create_string_buffer(size.value)
        _check(lib.vegas_get_state(self._h, buf, ctypes.byref(size)), "vegas_get_state")
        return buf.raw[:size.value]

    def state_arrays(self):
        """the checkpoint's contents as arrays: edges [dim][nbins+1], the stratification weights ell (float32
        [ncubes], or None before the first iteration), the strata and the iteration counter"""
        blob = self.get_state()
        ell_valid = int(np.frombuffer(blob, np.int32, 1, 20)[0])
        ncubes, iteration = (int(x) for x in np.frombuffer(blob, np.int64, 2, 24))
        nstrat = np.frombuffer(blob, np.int32, self.dim, 40).copy()
        head = 40 + 4 * 32
        ne = self.dim * (self.nbins + 1)
        edges = np.frombuffer(blob, np.float64, ne, head).reshape(self.dim, self.nbins + 1).copy()
        ell = np.frombuffer(blob, np.float32, ncubes, head + 8 * ne).copy() if ell_valid else None
        return {"edges": edges, "ell": ell, "nstrat": nstrat if ell_valid else None, "iteration": iteration}

    def set_state(self, blob):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib.vegas_set_state(self._h, buf, len(blob)), "vegas_set_state")

    def set_flow(self, params):
        """the learned proposal's flow parameters (FP32 vector), or None to turn it off"""
        if params is None:
            _check(lib.vegas_set_flow(self._h, None, 0), "vegas_set_flow")
            return
        p = np.ascontiguousarray(params, dtype=np.float32)
        self._flow = p
        _check(lib.vegas_set_flow(self._h, p.ctypes.data_as(ctypes.c_void_p), p.size), "vegas_set_flow")

    def set_flow_training(self, iterations, steps_per_iteration, samples, batch=4096, lr=1e-3, temper=1.0,
                          floor=0.03):
        """train the flow after each of the next `iterations` iterations (vegas_set_flow_training); floor is the
        weight of the uniform points mixed into the training set, 0 for none"""
        _check(lib.vegas_set_flow_training(self._h, iterations, steps_per_iteration, samples, batch, lr, temper,
                                           floor), "vegas_set_flow_training")

    def flow_explore(self, integrand, params, neval, iterations=10, maps=8, samples_per_map=32768, steps=2000,
                     batch=4096, lr=1e-3, floor=0.03, rounds=3, seed=0):
        """vegas_flow_explore: adapt `maps` VEGAS+ maps with seeds seed, seed + 1, ..., pool their samples by the
        balance heuristic and train the flow on them, then rounds - 1 times on samples of the flow itself; the map
        is uniform again afterwards"""
        p = np.ascontiguousarray(params, dtype=np.float64) if len(params) else np.zeros(0)
        _check(lib.vegas_flow_explore(self._h, integrand, p.ctypes.data_as(ctypes.c_void_p) if p.size else None,
                                      p.size, int(neval), int(iterations), int(maps), int(samples_per_map),
                                      int(steps), int(batch), float(lr), float(floor), int(rounds), int(seed)),
               "vegas_flow_explore")

    def get_flow(self):
        n = lib.vegas_flow_param_count(self.dim)
        p = np.zeros(n, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib.vegas_get_flow(self._h, p.ctypes.data_as(ctypes.c_void_p), n, ctypes.byref(loss)), "vegas_get_flow")
        return p, loss.value

    def edges(self):
        e = np.zeros((self.dim, self.nbins + 1))
        _check(lib.vegas_get_edges(self._h, e.ctypes.data_as(ctypes.c_void_p), e.size), "vegas_get_edges")
        return e


# ---------------------------------------------------------------------------
# Level 3: a batch of independent integrals
# ---------------------------------------------------------------------------
BATCH_EDGES, BATCH_OFFSETS, BATCH_ELL, BATCH_BINS, BATCH_ITER_EST, BATCH_ITER_SIG, BATCH_INFO = range(7)


class Batch:
    """Independent integrals run together (vegas_batch_create ... vegas_batch_destroy).

    problems: a list of dicts with keys dim, integrand, params, neval and
    optionally nstrat (0: automatic)."""

    def __init__(self, problems, nbins=50, alpha=0.5, beta=0.75, seed=0, skip=0, stream=None, alloc=None,
                 free=None):
        n = len(problems)
        arr = (Problem * n)()
        self._params = []
        for i, q in enumerate(problems):
            prm = np.ascontiguousarray(q.get("params", []), dtype=np.float64)
            self._params.append(prm)
            arr[i] = Problem(int(q["dim"]), int(q["integrand"]), prm.ctypes.data if prm.size else None, prm.size,
                             int(q["neval"]), int(q.get("nstrat", 0)), 0)
        h = ctypes.c_void_p()
        self._hooks = hooks(alloc, free)
        _check(lib.vegas_batch_create_ex(arr, n, nbins, alpha, beta, int(seed), self._hooks[0], self._hooks[1], None,
                                         ctypes.byref(h)), "vegas_batch_create_ex")
        self._h = h
        self.n, self.nbins = n, nbins
        self.dims = [int(q["dim"]) for q in problems]
        if skip:
            _check(lib.vegas_batch_set_skip(self._h, skip), "vegas_batch_set_skip")
        if stream is not None:
            _check(lib.vegas_batch_set_stream(self._h, _stream_ptr(stream)), "vegas_batch_set_stream")

    def close(self):
        if getattr(self, "_h", None):
            lib.vegas_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_chi2_bound(self, bound):
        _check(lib.vegas_batch_set_chi2_bound(self._h, float(bound)), "vegas_batch_set_chi2_bound")

    def set_launch(self, variant, ctas_per_sm=0, chunk_tiles=4):
        _check(lib.vegas_batch_set_launch(self._h, variant, ctas_per_sm, chunk_tiles), "vegas_batch_set_launch")

    def set_tile(self, tile_log2):
        """tiles of 2^tile_log2 evaluations (10 or 11) for every integral"""
        _check(lib.vegas_batch_set_tile(self._h, int(tile_log2)), "vegas_batch_set_tile")

    def tune(self):
        v, c, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        ms = ctypes.c_float()
        _check(lib.vegas_batch_tune(self._h, ctypes.byref(v), ctypes.byref(c), ctypes.byref(k), ctypes.byref(ms)),
               "vegas_batch_tune")
        return {"variant": v.value, "ctas_per_sm": c.value, "chunk_tiles": k.value, "ms": ms.value,
                "tile_log2": self.info(0)["tile_log2"]}

    def reset(self):
        _check(lib.vegas_batch_reset(self._h), "vegas_batch_reset")

    def integrate(self, nitn, rtol=0.0):
        res = (ProblemResult * self.n)()
        nrun = ctypes.c_int32()
        ms = ctypes.c_float()
        _check(lib.vegas_batch_integrate(self._h, int(nitn), float(rtol), res, ctypes.byref(nrun), ctypes.byref(ms)),
               "vegas_batch_integrate")
        out = [{"estimate": r.estimate, "sigma": r.sigma, "chi2_dof": r.chi2_dof, "n_used": r.n_used,
                "nitn_run": r.nitn_run, "converged": bool(r.converged), "status": r.status, "flags": r.flags}
               for r in res]
        return out, nrun.value, ms.value

    def info(self, p):
        o = np.zeros(5, dtype=np.int64)
        _check(lib.vegas_batch_get(self._h, p, BATCH_INFO, o.ctypes.data_as(ctypes.c_void_p), 5), "vegas_batch_get")
        return {"dim": int(o[0]), "nstrat": int(o[1]), "ncubes": int(o[2]), "nitn_run": int(o[3]),
                "tile_log2": int(o[4])}

    def get(self, p, what):
        inf = self.info(p)
        d, nh, nrec, G = inf["dim"], inf["ncubes"], inf["nitn_run"], self.nbins
        shape, dt = {BATCH_EDGES: ((d, G + 1), np.float64), BATCH_OFFSETS: ((nh + 1,), np.int64),
                     BATCH_ELL: ((nh,), np.float32), BATCH_BINS: ((d, G), np.float64),
                     BATCH_ITER_EST: ((nrec,), np.float64), BATCH_ITER_SIG: ((nrec,), np.float64)}[what]
        a = np.zeros(shape, dtype=dt)
        _check(lib.vegas_batch_get(self._h, p, what, a.ctypes.data_as(ctypes.c_void_p), a.size), "vegas_batch_get")
        return a


# ---------------------------------------------------------------------------
# Level 2: step entry points on torch CUDA tensors
# ---------------------------------------------------------------------------
def _geometry(dim, nbins, nstrat, tile_log2=0):
    ns = np.ascontiguousarray(nstrat if not isinstance(nstrat, int) else [nstrat] * dim, dtype=np.int32)
    g = Geometry(dim, nbins, ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), int(tile_log2), 0)
    g._keep = ns
    return g


def allocate_scratch_bytes(ncubes):
    return lib.vegas_allocate_scratch_bytes(int(ncubes))


def allocate(ell, ncubes, neval, uniform, offsets, scratch, stream=None):
    """vegas_allocate: ell (float32 [ncubes] or None), offsets (int64 [ncubes+1]), scratch (uint8)."""
    _check(lib.vegas_allocate(_ptr(ell), int(ncubes), int(neval), int(bool(uniform)), _ptr(offsets), _ptr(scratch),
                              scratch.numel(), _stream_ptr(stream)), "vegas_allocate")


ALLOCATE_STATIC_MAX_CUBES = 1 << 28


def allocate_static(ell, ncubes, neval, uniform, offsets, stream=None):
    """vegas_allocate_static: as allocate(), with the library's fixed device scratch instead of a caller area."""
    _check(lib.vegas_allocate_static(_ptr(ell), int(ncubes), int(neval), int(bool(uniform)), _ptr(offsets),
                                     _stream_ptr(stream)), "vegas_allocate_static")


def fill_scratch_bytes(dim, nbins, nstrat, neval):
    g = _geometry(dim, nbins, nstrat)
    return lib.vegas_fill_scratch_bytes(ctypes.byref(g), int(neval))


def fill(dim, nbins, nstrat, precision, integrand, params, neval, seed, iteration, beta, edges, offsets, ell, bins,
         result, flags, scratch, cube_mean=None, cube_m2=None, problem_id=0, stream=None, tile_log2=0):
    """vegas_fill on torch CUDA tensors: params/edges/bins/result/cube_* float64, offsets int64,
    ell float32, flags int32, scratch uint8; tile_log2 0 (the library's choice), 10 or 11."""
    g = _geometry(dim, nbins, nstrat, tile_log2)
    _check(lib.vegas_fill(ctypes.byref(g), precision, integrand, _ptr(params) if params is not None and
                          params.numel() else None, 0 if params is None else params.numel(), int(neval), int(seed),
                          int(iteration), int(problem_id), float(beta), _ptr(edges), _ptr(offsets), _ptr(ell),
                          _ptr(bins), _ptr(result), _ptr(cube_mean), _ptr(cube_m2), _ptr(flags), _ptr(scratch),
                          scratch.numel(), _stream_ptr(stream)), "vegas_fill")


def refine(dim, nbins, alpha, bins, edges_in, edges_out, stream=None):
    _check(lib.vegas_refine(dim, nbins, float(alpha), _ptr(bins), _ptr(edges_in), _ptr(edges_out),
                            _stream_ptr(stream)), "vegas_refine")


def combine(it_est, it_sig, skip, out, stream=None):
    _check(lib.vegas_combine(_ptr(it_est), _ptr(it_sig), it_est.numel(), int(skip), _ptr(out), _stream_ptr(stream)),
           "vegas_combine")


def combine_weighted(it_est, it_sig, skip, weighting, out, stream=None):
    _check(lib.vegas_combine_weighted(_ptr(it_est), _ptr(it_sig), it_est.numel(), int(skip), int(weighting), _ptr(out),
                                      _stream_ptr(stream)), "vegas_combine_weighted")


# ---------------------------------------------------------------------------
# Level 4: the learned proposal's coupling flow, on torch CUDA tensors (FP32)
# ---------------------------------------------------------------------------
FLOW_NORMALISE, FLOW_SAMPLE = 0, 1


def explore_points(dim, nbins, maps, samples_per_map, seed, x, q, stream=None):
    """vegas_explore_points: maps a float64 CUDA tensor [nmaps][dim][nbins + 1]; x float32 [nmaps * samples][dim]
    and q float64 [nmaps * samples] receive the points and the mixture density"""
    import torch
    if not (maps.is_cuda and maps.dtype == torch.float64 and q.dtype == torch.float64 and x.dtype == torch.float32):
        raise TypeError("explore_points: maps and q float64, x float32, all CUDA tensors")
    _check(lib.vegas_explore_points(int(dim), int(nbins), int(maps.shape[0]), _ptr(maps), int(samples_per_map),
                                    int(seed), _ptr(x), _ptr(q), _stream_ptr(stream)), "vegas_explore_points")


def flow_param_count(dim):
    return lib.vegas_flow_param_count(dim)


def _f32_device(name, *tensors):
    """the flow entry points take contiguous FP32 device buffers: refuse anything else before the call"""
    for t in tensors:
        if t is None:
            continue
        if not (getattr(t, "is_cuda", False) and str(t.dtype) == "torch.float32" and t.is_contiguous()):
            raise TypeError(f"{name}: buffers must be contiguous float32 CUDA tensors, got "
                            f"{getattr(t, 'dtype', type(t))} on {getattr(t, 'device', '?')}")


def flow_apply(dim, direction, params, x_in, x_out, logdet, stream=None):
    """vegas_flow_apply: x_in / x_out [n][dim], logdet [n], params [flow_param_count(dim)]"""
    _f32_device("flow_apply", params, x_in, x_out, logdet)
    _check(lib.vegas_flow_apply(dim, direction, _ptr(params), _ptr(x_in), _ptr(x_out), _ptr(logdet),
                                x_in.shape[0], _stream_ptr(stream)), "vegas_flow_apply")


def flow_check(stream=None):
    """vegas_flow_check: synchronise and raise if a bounded wait of an earlier flow_apply ran out"""
    _check(lib.vegas_flow_check(_stream_ptr(stream)), "vegas_flow_check")


def flow_wait_selftest(polls, arrive, stream=None):
    """vegas_flow_wait_selftest: the status code (ETIMEOUT when nothing arrived within `polls` polls)"""
    return lib.vegas_flow_wait_selftest(int(polls), int(arrive), _stream_ptr(stream))


def flow_grad_scratch_bytes(dim, n):
    return lib.vegas_flow_grad_scratch_bytes(dim, int(n))


def flow_grad(dim, params, x, w, grad, loss, scratch, stream=None):
    """vegas_flow_grad: the weighted negative log-likelihood of samples x [n][dim] with weights w [n]"""
    _f32_device("flow_grad", params, x, w, grad, loss)
    _check(lib.vegas_flow_grad(dim, _ptr(params), _ptr(x), _ptr(w), x.shape[0], _ptr(grad), _ptr(loss),
                               _ptr(scratch), scratch.numel(), _stream_ptr(stream)), "vegas_flow_grad")


def flow_adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _f32_device("flow_adam", params, grad, m, v)
    _check(lib.vegas_flow_adam(params.numel(), _ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), lr, beta1,
                               beta2, eps, _stream_ptr(stream)), "vegas_flow_adam")


def probe_pipes():
    """(FP32 FMA, FP64 FMA, MUFU ex2, IMAD.HI) issue rates in operations per SM per clock"""
    r = np.zeros(4)
    _check(lib.vegas_probe_pipes(r.ctypes.data_as(ctypes.c_void_p)), "vegas_probe_pipes")
    return r


def probe_exp64():
    """FP64 exp() calls per SM per clock (vegas_probe_exp64)"""
    r = ctypes.c_double()
    _check(lib.vegas_probe_exp64(ctypes.byref(r)), "vegas_probe_exp64")
    return r.value


def exp64_eval(x, y, which=0, stream=None):
    """vegas_exp64_eval on float64 CUDA tensors: which 0 the table-driven e^x, 1 the library exp(), 2 the
    table-driven 2^(x/64) of the FP64 Gaussian sum"""
    _check(lib.vegas_exp64_eval(_ptr(x), _ptr(y), x.numel(), int(which), _stream_ptr(stream)), "vegas_exp64_eval")


def probe_shared_atomics():
    """shared-memory 32-bit atomic adds per SM per clock, lanes on distinct banks"""
    r = ctypes.c_double()
    _check(lib.vegas_probe_shared_atomics(ctypes.byref(r)), "vegas_probe_shared_atomics")
    return r.value
