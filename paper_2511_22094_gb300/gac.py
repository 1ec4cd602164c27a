"""ctypes binding of libgac.so (include/gac.h) -- argument marshalling only.

Every function here has the name of the C entry point it calls and only
converts arguments: numpy arrays and host tensors become host pointers, CUDA
tensors become device pointers, a torch.cuda.Stream becomes a cudaStream_t.
All arithmetic runs in libgac.so.  There is no fallback: if the library is
missing, importing this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgac.so")

GAC_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNKNOWN_MODEL", 3: "BUDGET", 4: "OOM", 5: "CUDA",
          6: "TIMEOUT", 7: "NOT_READY", 8: "CANCELLED", 9: "UNKNOWN_JOB"}
MONOEXP, MWI3, SMT, LINEAR_TEST = 1, 2, 3, 100
PREC_MIXED, PREC_FP32, PREC_FP64 = 0, 1, 2
MOMENTS_THINNED, MOMENTS_ALL_POSTBURNIN = 0, 1
MAX_PAR = 12


class GacError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class ModelDesc(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("n_acq", ct.c_int), ("acq", ct.POINTER(ct.c_double)),
                ("n_par", ct.c_int), ("lb", ct.POINTER(ct.c_double)),
                ("ub", ct.POINTER(ct.c_double)), ("step", ct.POINTER(ct.c_double))]


class McmcOpts(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("burnin", ct.c_int), ("thin", ct.c_int),
                ("n_chains", ct.c_int), ("seed", ct.c_uint64), ("voxel_base", ct.c_uint64),
                ("precision", ct.c_int), ("moments_mode", ct.c_int), ("trace_n_vox", ct.c_int),
                ("adapt_window", ct.c_int), ("adapt_target", ct.c_double), ("lanes_per_chain", ct.c_int)]


class TraceRec(ct.Structure):
    _fields_ = [("theta", ct.c_double * MAX_PAR), ("prop", ct.c_double * MAX_PAR),
                ("L", ct.c_double), ("Lp", ct.c_double), ("w_acc", ct.c_uint32),
                ("accepted", ct.c_int32)]


TRACE_DTYPE = np.dtype([("theta", np.float64, MAX_PAR), ("prop", np.float64, MAX_PAR),
                        ("L", np.float64), ("Lp", np.float64), ("w_acc", np.uint32),
                        ("accepted", np.int32)])
assert TRACE_DTYPE.itemsize == ct.sizeof(TraceRec)


FIT_L1, FIT_L2 = 1, 2


class FitOpts(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("loss", ct.c_int),
                ("iterations", ct.c_int), ("learning_rate", ct.c_double), ("beta1", ct.c_double),
                ("beta2", ct.c_double), ("epsilon", ct.c_double), ("tol", ct.c_double),
                ("convergence_value", ct.c_double), ("convergence_window", ct.c_int),
                ("tv_lambda", ct.c_double), ("tv_params", ct.c_uint32), ("tv_dims", ct.c_int),
                ("precision", ct.c_int)]


RESULT_KEYS = ("mean", "std", "samples", "accept_rate", "nonfinite", "trace", "rhat", "step_scale")


class Result(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in RESULT_KEYS]


class ServerStats(ct.Structure):
    _fields_ = [("queued", ct.c_int64), ("resident", ct.c_int64), ("finished", ct.c_int64),
                ("rounds", ct.c_int64), ("bytes_in_use", ct.c_size_t), ("budget", ct.c_size_t),
                ("gpu_s", ct.c_double), ("round_host_s", ct.c_double), ("admit_s", ct.c_double)]


EXPORTS = ["gac_model_register", "gac_model_info", "gac_result_sizes", "gac_mcmc_run",
           "gac_forward", "gac_loglik", "gac_philox_words", "gac_normals", "gac_last_error",
           "gac_version", "gac_server_create", "gac_server_job_bytes", "gac_server_submit",
           "gac_server_poll", "gac_server_wait", "gac_server_cancel", "gac_server_get_stats",
           "gac_server_destroy", "gac_mcmc_run_noalloc", "gac_ensemble_run", "gac_fit_run",
           "gac_pipe_rate"]
NOALLOC_STATE_BYTES = 64 << 20


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libgac.so is not built ({LIB_PATH}); run paper_2511_22094_gb300.build.build()")
    L = ct.CDLL(LIB_PATH)
    vp, i64, u64 = ct.c_void_p, ct.c_int64, ct.c_uint64
    L.gac_last_error.restype = ct.c_char_p
    L.gac_version.restype = ct.c_char_p
    sig = {
        "gac_model_register": [ct.POINTER(ModelDesc), ct.POINTER(ct.c_int)],
        "gac_model_info": [ct.c_int, ct.POINTER(ct.c_int), ct.POINTER(ct.c_int)],
        "gac_result_sizes": [ct.c_int, i64, ct.POINTER(McmcOpts), ct.POINTER(ct.c_size_t * len(RESULT_KEYS))],
        "gac_mcmc_run": [ct.c_int, vp, i64, vp, ct.c_float, vp, ct.POINTER(McmcOpts),
                         ct.POINTER(Result), vp],
        "gac_forward": [ct.c_int, vp, i64, ct.c_int, vp, vp],
        "gac_loglik": [ct.c_int, vp, i64, vp, vp, ct.c_int, vp, vp],
        "gac_philox_words": [u64, vp, vp, vp, i64, ct.c_int, vp, vp],
        "gac_normals": [u64, vp, vp, vp, i64, ct.c_int, ct.c_int, vp, vp, vp],
        "gac_ensemble_run": [ct.c_int, vp, i64, vp, ct.c_float, vp, ct.POINTER(McmcOpts), ct.c_double,
                             ct.POINTER(Result), vp],
        "gac_mcmc_run_noalloc": [ct.c_int, vp, i64, vp, ct.c_float, vp, ct.POINTER(McmcOpts), ct.c_int,
                                 ct.POINTER(Result), vp],
        "gac_fit_run": [ct.c_int, vp, vp, vp, ct.POINTER(FitOpts), vp, vp, ct.POINTER(ct.c_int), vp],
        "gac_pipe_rate": [ct.c_int, ct.POINTER(ct.c_double), vp],
        "gac_server_create": [ct.c_size_t, ct.c_int, ct.POINTER(vp)],
        "gac_server_job_bytes": [ct.c_int, i64, ct.POINTER(McmcOpts), ct.c_int, ct.c_int,
                                 ct.POINTER(ct.c_size_t)],
        "gac_server_submit": [vp, ct.c_int, vp, i64, vp, ct.c_float, ct.POINTER(McmcOpts), ct.c_int,
                              ct.POINTER(u64)],
        "gac_server_poll": [vp, u64, ct.POINTER(ct.c_int), ct.POINTER(Result),
                            ct.POINTER(ct.c_double)],
        "gac_server_wait": [vp, u64, ct.c_double, ct.POINTER(Result), ct.POINTER(ct.c_double)],
        "gac_server_cancel": [vp, u64],
        "gac_server_get_stats": [vp, ct.POINTER(ServerStats)],
        "gac_server_destroy": [vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ct.c_int
    return L


_lib = _load()


def lib():
    return _lib


def last_error() -> str:
    return _lib.gac_last_error().decode()


def version() -> str:
    return _lib.gac_version().decode()


def _check(st: int, where: str):
    if st != GAC_OK:
        raise GacError(st, where, last_error())


def _ptr(x):
    """Host (numpy / CPU tensor) or device (CUDA tensor) address, or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot pass {type(x)} as a buffer")


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


# ------------------------------------------------------------- models ------
def gac_model_register(kind: int, acq, lb, ub, step) -> int:
    arrs = [np.ascontiguousarray(a, np.float64) for a in (acq, lb, ub, step)]
    p = [a.ctypes.data_as(ct.POINTER(ct.c_double)) for a in arrs]
    d = ModelDesc(kind, len(arrs[0]), p[0], len(arrs[1]), p[1], p[2], p[3])
    mid = ct.c_int(0)
    _check(_lib.gac_model_register(ct.byref(d), ct.byref(mid)), "gac_model_register")
    return mid.value


def gac_model_info(model_id: int):
    P, M = ct.c_int(), ct.c_int()
    _check(_lib.gac_model_info(model_id, ct.byref(P), ct.byref(M)), "gac_model_info")
    return P.value, M.value


def make_opts(iterations, burnin, thin, n_chains, seed, voxel_base=0, precision=PREC_MIXED,
              moments_mode=MOMENTS_THINNED, trace_n_vox=0, adapt_window=0,
              adapt_target=0.0, lanes_per_chain=0) -> McmcOpts:
    return McmcOpts(iterations, burnin, thin, n_chains, seed, voxel_base, precision, moments_mode,
                    trace_n_vox, adapt_window, adapt_target, lanes_per_chain)


def gac_result_sizes(model_id: int, n_vox: int, opts: McmcOpts):
    b = (ct.c_size_t * len(RESULT_KEYS))()
    _check(_lib.gac_result_sizes(model_id, n_vox, ct.byref(opts), ct.byref(b)), "gac_result_sizes")
    return dict(zip(RESULT_KEYS, list(b)))


def gac_mcmc_run(model_id: int, data, n_vox: int, sigma, sigma_scalar: float, x0,
                 opts: McmcOpts, out: dict, stream=None):
    """out: dict with any of RESULT_KEYS (caller-allocated numpy arrays or
    tensors, host or device)."""
    r = _result(out)
    _check(_lib.gac_mcmc_run(model_id, _ptr(data), n_vox, _ptr(sigma), sigma_scalar, _ptr(x0),
                             ct.byref(opts), ct.byref(r), _stream(stream)), "gac_mcmc_run")


def gac_ensemble_run(model_id: int, data, n_vox: int, sigma, sigma_scalar: float, x0,
                     opts: McmcOpts, stretch: float, out: dict, stream=None):
    """Affine-invariant ensemble sampler; opts.n_chains = walkers."""
    r = _result(out)
    _check(_lib.gac_ensemble_run(model_id, _ptr(data), n_vox, _ptr(sigma), sigma_scalar, _ptr(x0),
                                 ct.byref(opts), stretch, ct.byref(r), _stream(stream)),
           "gac_ensemble_run")


def gac_mcmc_run_noalloc(model_id: int, data, n_vox: int, sigma, sigma_scalar: float, x0,
                         opts: McmcOpts, slice_iterations: int, out: dict, stream=None):
    """Allocation-free sampler run (device buffers only); see include/gac.h."""
    r = _result(out)
    _check(_lib.gac_mcmc_run_noalloc(model_id, _ptr(data), n_vox, _ptr(sigma), sigma_scalar,
                                     _ptr(x0), ct.byref(opts), slice_iterations, ct.byref(r),
                                     _stream(stream)), "gac_mcmc_run_noalloc")


def make_fit_opts(shape, *, loss=FIT_L1, iterations=100, learning_rate=0.01, beta1=0.9, beta2=0.999,
                  epsilon=1e-8, tol=0.0, convergence_value=0.0, convergence_window=20, tv_lambda=0.0,
                  tv_params=0, tv_dims=3, precision=PREC_FP32) -> FitOpts:
    return FitOpts(shape[0], shape[1], shape[2], loss, iterations, learning_rate, beta1, beta2, epsilon, tol,
                   convergence_value, convergence_window, tv_lambda, tv_params, tv_dims, precision)


def gac_fit_run(model_id: int, data, mask, weight, opts: FitOpts, theta, loss_history=None, stream=None) -> int:
    """Whole-volume Adam fit; theta [N][P] float64 is updated in place.
    Returns the number of updates taken."""
    done = ct.c_int(0)
    _check(_lib.gac_fit_run(model_id, _ptr(data), _ptr(mask), _ptr(weight), ct.byref(opts), _ptr(theta),
                            _ptr(loss_history), ct.byref(done), _stream(stream)), "gac_fit_run")
    return done.value


def fit_host(model_id: int, data, theta0, *, shape, mask=None, weight=None, **kw):
    """gac_fit_run on host numpy arrays: returns (theta, loss history, updates)."""
    th = np.array(theta0, np.float64, copy=True, order="C")
    it = kw.get("iterations", 100)
    hist = np.full(max(it, 1), np.nan)
    opts = make_fit_opts(shape, **kw)
    d = np.ascontiguousarray(data, np.float32)
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    wt = None if weight is None else np.ascontiguousarray(weight, np.float32)
    done = gac_fit_run(model_id, d, mk, wt, opts, th, hist)
    return th, hist[:done], done


def gac_forward(model_id: int, theta, n: int, precision: int, s, stream=None):
    _check(_lib.gac_forward(model_id, _ptr(theta), n, precision, _ptr(s), _stream(stream)),
           "gac_forward")


def gac_loglik(model_id: int, theta, n: int, data, sigma, precision: int, L, stream=None):
    _check(_lib.gac_loglik(model_id, _ptr(theta), n, _ptr(data), _ptr(sigma), precision, _ptr(L),
                           _stream(stream)), "gac_loglik")


def gac_philox_words(seed: int, t, v, c, n: int, n_words: int, out, stream=None):
    _check(_lib.gac_philox_words(seed, _ptr(t), _ptr(v), _ptr(c), n, n_words, _ptr(out),
                                 _stream(stream)), "gac_philox_words")


def gac_normals(seed: int, t, v, c, n: int, n_par: int, precision: int, z, w_acc, stream=None):
    _check(_lib.gac_normals(seed, _ptr(t), _ptr(v), _ptr(c), n, n_par, precision, _ptr(z),
                            _ptr(w_acc), _stream(stream)), "gac_normals")


PIPE_OPS = {"ffma": 0, "ffma2": 1, "ex2": 2, "sin": 3, "lg2": 4, "rsqrt": 5, "rcp": 6, "sqrt": 7,
            "dfma": 8, "imad_hi": 9, "lop3": 10}


def gac_pipe_rate(op, stream=None) -> float:
    """Results per SM clock of one arithmetic pipe operation (name or code)."""
    code = PIPE_OPS[op] if isinstance(op, str) else int(op)
    r = ct.c_double()
    _check(_lib.gac_pipe_rate(code, ct.byref(r), _stream(stream)), "gac_pipe_rate")
    return r.value


# ------------------------------------------------------------- serving -----
def _result(out):
    out = out or {}
    return Result(*(_ptr(out.get(k)) for k in RESULT_KEYS))


def gac_server_create(hbm_budget_bytes: int, max_resident_jobs: int):
    h = ct.c_void_p()
    _check(_lib.gac_server_create(hbm_budget_bytes, max_resident_jobs, ct.byref(h)),
           "gac_server_create")
    return h


def gac_server_job_bytes(model_id: int, n_vox: int, opts: McmcOpts, keep_samples: bool,
                         has_sigma: bool) -> int:
    b = ct.c_size_t()
    _check(_lib.gac_server_job_bytes(model_id, n_vox, ct.byref(opts), int(keep_samples),
                                     int(has_sigma), ct.byref(b)), "gac_server_job_bytes")
    return b.value


def gac_server_submit(srv, model_id: int, data, n_vox: int, sigma, sigma_scalar: float,
                      opts: McmcOpts, keep_samples: bool = False) -> int:
    jid = ct.c_uint64()
    _check(_lib.gac_server_submit(srv, model_id, _ptr(data), n_vox, _ptr(sigma), sigma_scalar,
                                  ct.byref(opts), int(keep_samples), ct.byref(jid)),
           "gac_server_submit")
    return jid.value


def gac_server_poll(srv, job_id: int, out: dict | None = None):
    """Returns (done, latency_s); raises GacError for a failed/cancelled job."""
    done, lat = ct.c_int(), ct.c_double()
    r = _result(out)
    _check(_lib.gac_server_poll(srv, job_id, ct.byref(done), ct.byref(r), ct.byref(lat)),
           "gac_server_poll")
    return bool(done.value), lat.value


def gac_server_wait(srv, job_id: int, timeout_s: float, out: dict | None = None) -> float:
    lat = ct.c_double()
    r = _result(out)
    _check(_lib.gac_server_wait(srv, job_id, timeout_s, ct.byref(r), ct.byref(lat)),
           "gac_server_wait")
    return lat.value


def gac_server_cancel(srv, job_id: int):
    _check(_lib.gac_server_cancel(srv, job_id), "gac_server_cancel")


def gac_server_get_stats(srv) -> dict:
    st = ServerStats()
    _check(_lib.gac_server_get_stats(srv, ct.byref(st)), "gac_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def gac_server_destroy(srv):
    _check(_lib.gac_server_destroy(srv), "gac_server_destroy")


# --------------------------------------------------- numpy conveniences ----
def n_samples(iterations: int, burnin: int, thin: int) -> int:
    return (iterations - burnin) // thin if iterations > burnin and thin > 0 else 0


def run_host(model_id: int, data: np.ndarray, sigma, *, iterations, burnin, thin, n_chains, seed,
             x0=None, sigma_scalar=0.0, voxel_base=0, precision=PREC_MIXED,
             moments_mode=MOMENTS_THINNED, trace_n_vox=0, want_samples=True, adapt_window=0,
             adapt_target=0.0, lanes_per_chain=0):
    """Runs the sampler on host numpy inputs (the library stages them through
    device memory) and returns host numpy outputs."""
    P, M = gac_model_info(model_id)
    data = np.ascontiguousarray(data, np.float32)
    N = data.shape[0]
    S = n_samples(iterations, burnin, thin)
    C = n_chains
    out = dict(mean=np.full((P, N), np.nan), std=np.full((P, N), np.nan),
               samples=np.full((S, C, P, N), np.nan, np.float32) if (want_samples and S) else None,
               accept_rate=np.zeros((C, N), np.float32), nonfinite=np.zeros((C, N), np.int32),
               trace=np.zeros((trace_n_vox, C, iterations), TRACE_DTYPE) if trace_n_vox else None,
               rhat=np.full((P, N), np.nan), step_scale=np.zeros((C, N), np.float32))
    sig = None if sigma is None else np.ascontiguousarray(sigma, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    opts = make_opts(iterations, burnin, thin, n_chains, seed, voxel_base, precision, moments_mode,
                     trace_n_vox, adapt_window, adapt_target, lanes_per_chain)
    gac_mcmc_run(model_id, data, N, sig, sigma_scalar, x0a, opts, out)
    return out


def run_ensemble_host(model_id: int, data: np.ndarray, sigma, *, iterations, burnin, thin,
                      n_walkers, seed, stretch=2.0, x0=None, sigma_scalar=0.0, voxel_base=0,
                      precision=PREC_MIXED, moments_mode=MOMENTS_THINNED, trace_n_vox=0,
                      want_samples=True):
    """Ensemble sampler on host numpy inputs; host numpy outputs."""
    P, M = gac_model_info(model_id)
    data = np.ascontiguousarray(data, np.float32)
    N = data.shape[0]
    S = n_samples(iterations, burnin, thin)
    L = n_walkers
    out = dict(mean=np.full((P, N), np.nan), std=np.full((P, N), np.nan),
               samples=np.full((S, L, P, N), np.nan, np.float32) if (want_samples and S) else None,
               accept_rate=np.zeros((L, N), np.float32), nonfinite=np.zeros((L, N), np.int32),
               trace=np.zeros((trace_n_vox, L, iterations), TRACE_DTYPE) if trace_n_vox else None)
    sig = None if sigma is None else np.ascontiguousarray(sigma, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    opts = make_opts(iterations, burnin, thin, n_walkers, seed, voxel_base, precision, moments_mode,
                     trace_n_vox)
    gac_ensemble_run(model_id, data, N, sig, sigma_scalar, x0a, opts, stretch, out)
    return out


def forward_host(model_id: int, theta, precision=PREC_MIXED) -> np.ndarray:
    P, M = gac_model_info(model_id)
    th = np.ascontiguousarray(np.atleast_2d(theta), np.float64)
    s = np.zeros((th.shape[0], M), np.float64)
    gac_forward(model_id, th, th.shape[0], precision, s)
    return s


def loglik_host(model_id: int, theta, data, sigma, precision=PREC_MIXED) -> np.ndarray:
    th = np.ascontiguousarray(np.atleast_2d(theta), np.float64)
    n = th.shape[0]
    y = np.ascontiguousarray(np.asarray(data, np.float32).reshape(n, -1))
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.float32), (n,)))
    L = np.zeros(n, np.float64)
    gac_loglik(model_id, th, n, y, sg, precision, L)
    return L
