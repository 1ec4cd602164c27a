"""FP64 CPU oracle for the voxel-wise Metropolis-Hastings sampler (GACELLE
mcmc.m, Sec. 2.2.2) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library
(``paper_2511_22094_gb300``) never imports it, and the two share no code: the
C source ``gac_oracle.c`` re-implements Philox4x32-10, the forward models, the
Gaussian likelihood, the sampler and the moments in plain double precision.

This module only compiles that C file with gcc/OpenMP and marshals numpy
arrays through ctypes; all arithmetic of the method lives in ``gac_oracle.c``.
"""
from __future__ import annotations

import contextlib
import ctypes as ct
import os
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MONOEXP, MWI3, SMT, LINEAR = 1, 2, 3, 100
MOMENTS_THINNED, MOMENTS_ALL_POSTBURNIN = 0, 1


def _compile(src: str, out: str) -> None:
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
           "-ffp-contract=off", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile gac_oracle.c into liboracle.so (portable flags: x86 and Arm)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        _compile(_SRC, _LIB)
    return _LIB


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def build_variant(src_text: str, tag: str) -> str:
    """Compile a modified copy of the oracle source (the tests plant mistakes
    in such copies to show that the pins catch them); returns the .so path."""
    d = tempfile.mkdtemp(prefix=f"orc_{tag}_")
    src = os.path.join(d, "gac_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    out = os.path.join(d, "liboracle.so")
    _compile(src, out)
    return out


@contextlib.contextmanager
def variant(so_path: str):
    """Route every call of this module to another build of the oracle."""
    global _lib
    lib()
    with _lock:
        saved = _lib
        _lib = None
    try:
        with _lock:
            _lib = _declare(ct.CDLL(so_path))
        yield
    finally:
        with _lock:
            _lib = saved


class _Model(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("n_acq", ct.c_int), ("acq", ct.POINTER(ct.c_double)),
                ("n_par", ct.c_int), ("lb", ct.POINTER(ct.c_double)),
                ("ub", ct.POINTER(ct.c_double)), ("step", ct.POINTER(ct.c_double))]


class _Opts(ct.Structure):
    _fields_ = [("iterations", ct.c_int), ("burnin", ct.c_int), ("thin", ct.c_int),
                ("n_chains", ct.c_int), ("seed", ct.c_uint64), ("voxel_base", ct.c_uint64),
                ("moments_mode", ct.c_int), ("n_threads", ct.c_int), ("adapt_window", ct.c_int),
                ("adapt_target", ct.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(ct.CDLL(_LIB))
    return _lib


def _declare(L):
    P = np.ctypeslib.ndpointer
    u32 = P(np.uint32, flags="C_CONTIGUOUS")
    f64 = P(np.float64, flags="C_CONTIGUOUS")
    L.orc_philox4x32_10.argtypes = [u32, u32, u32]
    L.orc_philox4x32_10.restype = None
    L.orc_words.argtypes = [ct.c_uint64, ct.c_uint32, ct.c_uint32, ct.c_uint32, ct.c_int, u32]
    L.orc_words.restype = None
    L.orc_u01.argtypes = [ct.c_uint32]
    L.orc_u01.restype = ct.c_double
    L.orc_n_words.argtypes = [ct.c_int]
    L.orc_n_words.restype = ct.c_int
    L.orc_normals_from_words.argtypes = [u32, ct.c_int, f64]
    L.orc_normals_from_words.restype = None
    L.orc_n_par.argtypes = [ct.c_int]
    L.orc_n_par.restype = ct.c_int
    L.orc_n_meas.argtypes = [ct.c_int, ct.c_int]
    L.orc_n_meas.restype = ct.c_int
    L.orc_g.argtypes = [ct.c_double]
    L.orc_g.restype = ct.c_double
    L.orc_n_samples.argtypes = [ct.c_int, ct.c_int, ct.c_int]
    L.orc_n_samples.restype = ct.c_int
    L.orc_stretch_z.argtypes = [ct.c_uint32, ct.c_double]
    L.orc_stretch_z.restype = ct.c_double
    L.orc_j1p_zero.argtypes = [ct.c_int]
    L.orc_j1p_zero.restype = ct.c_double
    L.orc_cyl_kappa.argtypes = [ct.c_double] * 5
    L.orc_cyl_kappa.restype = ct.c_double
    L.orc_dg.argtypes = [ct.c_double]
    L.orc_dg.restype = ct.c_double
    L.orc_window_slope.argtypes = [ct.POINTER(ct.c_double), ct.c_int]
    L.orc_window_slope.restype = ct.c_double
    L.orc_jacobian.restype = ct.c_int
    L.orc_fit_run.restype = ct.c_int
    L.orc_rhat.argtypes = [f64, ct.c_int, ct.c_int, ct.c_size_t]
    L.orc_rhat.restype = ct.c_double
    L.orc_max_threads.argtypes = []
    L.orc_max_threads.restype = ct.c_int
    for name in ("orc_forward_many", "orc_loglik_many", "orc_mcmc_run", "orc_chain_path",
                 "orc_lockstep", "orc_words_many", "orc_normals_many", "orc_ensemble_run",
                 "orc_ensemble_path"):
        getattr(L, name).restype = ct.c_int
    return L


def _dptr(a):
    return a.ctypes.data_as(ct.POINTER(ct.c_double)) if a is not None else None


def _vp(a):
    return ct.c_void_p(a.ctypes.data) if a is not None else ct.c_void_p(0)


# ---------------------------------------------------------------- RNG -----
def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32),
                            np.ascontiguousarray(key, np.uint32), out)
    return out


def words(seed: int, t: int, v: int, c: int, n: int) -> np.ndarray:
    w = np.zeros(n, np.uint32)
    lib().orc_words(seed, t & 0xFFFFFFFF, v, c, n, w)
    return w


def words_many(seed: int, t, v, c, nw: int) -> np.ndarray:
    """Words of draws (t[i], v[i], c[i]) -> [n][nw] uint32."""
    t, v, c = (np.ascontiguousarray(a, np.uint32) for a in (t, v, c))
    out = np.zeros((t.size, nw), np.uint32)
    lib().orc_words_many(ct.c_uint64(seed), _vp(t), _vp(v), _vp(c), ct.c_int64(t.size), nw, _vp(out))
    return out


def normals_many(words, n_par: int) -> np.ndarray:
    """Proposal normals of draws whose words are words [n][nw] -> [n][P]."""
    w = np.ascontiguousarray(words, np.uint32)
    z = np.zeros((w.shape[0], n_par))
    lib().orc_normals_many(_vp(w), ct.c_int64(w.shape[0]), w.shape[1], n_par, _vp(z))
    return z


def u01(w: int) -> float:
    return lib().orc_u01(int(w))


def n_words(n_par: int) -> int:
    return lib().orc_n_words(n_par)


def normals_from_words(w, n_par: int) -> np.ndarray:
    z = np.zeros(max(n_par, 1) + 1, np.float64)
    lib().orc_normals_from_words(np.ascontiguousarray(w, np.uint32), n_par, z)
    return z[:n_par]


# ------------------------------------------------------------- models -----
def n_par(kind: int) -> int:
    return lib().orc_n_par(kind)


def n_meas(kind: int, n_acq: int) -> int:
    return lib().orc_n_meas(kind, n_acq)


def g(x: float) -> float:
    return lib().orc_g(float(x))


def n_samples(iterations: int, burnin: int, thin: int) -> int:
    return lib().orc_n_samples(iterations, burnin, thin)


def forward(kind: int, acq, theta) -> np.ndarray:
    """theta [n][P] (or [P]) -> signals [n][M] float64."""
    acq = np.ascontiguousarray(acq, np.float64)
    th = np.ascontiguousarray(np.atleast_2d(theta), np.float64)
    M = n_meas(kind, len(acq))
    out = np.zeros((th.shape[0], M), np.float64)
    rc = lib().orc_forward_many(kind, _dptr(acq), len(acq), th.shape[0], _dptr(th), _dptr(out))
    assert rc == 0
    return out if np.ndim(theta) == 2 else out[0]


def loglik(kind: int, acq, theta, y, sigma) -> np.ndarray:
    """theta [n][P], y [n][M] float32, sigma [n] float32 -> L [n] float64."""
    acq = np.ascontiguousarray(acq, np.float64)
    th = np.ascontiguousarray(np.atleast_2d(theta), np.float64)
    n = th.shape[0]
    yy = np.ascontiguousarray(np.asarray(y, np.float32).reshape(n, -1))
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma, np.float32), (n,)))
    out = np.zeros(n, np.float64)
    rc = lib().orc_loglik_many(kind, _dptr(acq), len(acq), n, _dptr(th), _vp(yy), _vp(sg), _dptr(out))
    assert rc == 0
    return out


# ------------------------------------------------------------ sampler -----
class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""

    def __init__(self, **kw):
        self.__dict__.update(kw)


def _model(kind, acq, lb, ub, step):
    keep = _Keep(acq=np.ascontiguousarray(acq, np.float64), lb=np.ascontiguousarray(lb, np.float64),
                 ub=np.ascontiguousarray(ub, np.float64), step=np.ascontiguousarray(step, np.float64))
    m = _Model(kind, len(keep.acq), _dptr(keep.acq), len(keep.lb), _dptr(keep.lb), _dptr(keep.ub),
               _dptr(keep.step))
    return m, keep


def mcmc_run(kind, acq, lb, ub, step, data, sigma, *, iterations, burnin, thin, n_chains, seed,
             x0=None, sigma_scalar=0.0, voxel_base=0, moments_mode=0, n_threads=0,
             want_samples=True, adapt_window=0, adapt_target=0.0):
    """Runs the oracle sampler; returns a dict of numpy arrays (float64)."""
    m, keep = _model(kind, acq, lb, ub, step)
    P = len(keep.lb)
    data = np.ascontiguousarray(data, np.float32)
    n_vox = data.shape[0]
    sig = None if sigma is None else np.ascontiguousarray(sigma, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    S = n_samples(iterations, burnin, thin)
    C = n_chains
    mean = np.full((P, n_vox), np.nan)
    std = np.full((P, n_vox), np.nan)
    samples = np.full((S, C, P, n_vox), np.nan) if want_samples else None
    acc = np.zeros((C, n_vox))
    bad = np.zeros((C, n_vox), np.int32)
    rhat = np.full((P, n_vox), np.nan)
    scale = np.zeros((C, n_vox))
    used = ct.c_int(0)
    o = _Opts(iterations, burnin, thin, n_chains, seed, voxel_base, moments_mode, n_threads,
              adapt_window, adapt_target)
    rc = lib().orc_mcmc_run(ct.byref(m), _vp(data), ct.c_int64(n_vox), _vp(sig),
                            ct.c_float(sigma_scalar), _vp(x0a), ct.byref(o), _vp(mean), _vp(std),
                            _vp(samples), _vp(acc), _vp(bad), _vp(rhat), _vp(scale), ct.byref(used))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dict(mean=mean, std=std, samples=samples, accept_rate=acc, nonfinite=bad, rhat=rhat,
                step_scale=scale, threads=used.value)


class _FitOpts(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("nz", ct.c_int), ("loss", ct.c_int),
                ("iterations", ct.c_int), ("lr", ct.c_double), ("beta1", ct.c_double),
                ("beta2", ct.c_double), ("eps", ct.c_double), ("tol", ct.c_double),
                ("conv_value", ct.c_double), ("conv_window", ct.c_int), ("lam", ct.c_double),
                ("tv_params", ct.c_uint32), ("tv_dims", ct.c_int)]


def dg(x):
    """d/dx of g(x) = int_0^1 exp(-x u^2) du."""
    return lib().orc_dg(x)


def jacobian(kind, acq, theta):
    """theta [P] -> (s [M], J [M][P])."""
    acq = np.ascontiguousarray(acq, np.float64)
    th = np.ascontiguousarray(theta, np.float64)
    M, P = n_meas(kind, len(acq)), n_par(kind)
    s, J = np.zeros(M), np.zeros((M, P))
    if lib().orc_jacobian(kind, _dptr(acq), len(acq), _dptr(th), _dptr(s), _dptr(J)) != 0:
        raise ValueError("no Jacobian for this kind")
    return s, J


def window_slope(y):
    y = np.ascontiguousarray(y, np.float64)
    return lib().orc_window_slope(_dptr(y), len(y))


def fit_run(kind, acq, lb, ub, data, theta0, *, shape, mask=None, weight=None, loss=1, iterations=100,
            lr=0.01, beta1=0.9, beta2=0.999, eps=1e-8, tol=0.0, conv_value=0.0, conv_window=20,
            lam=0.0, tv_params=0, tv_dims=3):
    """Whole-volume Adam fit; returns (theta [N][P], loss history, updates done)."""
    m, keep = _model(kind, acq, lb, ub, np.zeros(len(lb)))
    data = np.ascontiguousarray(data, np.float32)
    th = np.array(theta0, np.float64, copy=True, order="C")
    mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
    wt = None if weight is None else np.ascontiguousarray(weight, np.float32)
    hist = np.full(max(iterations, 1), np.nan)
    done = ct.c_int(0)
    o = _FitOpts(shape[0], shape[1], shape[2], loss, iterations, lr, beta1, beta2, eps, tol, conv_value,
                 conv_window, lam, tv_params, tv_dims)
    rc = lib().orc_fit_run(ct.byref(m), _vp(data), _vp(mk), _vp(wt), ct.byref(o), _dptr(th), _dptr(hist),
                           ct.byref(done))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return th, hist[:done.value], done.value


def j1p_zero(m):
    """m-th positive zero of J1' (m >= 1)."""
    return lib().orc_j1p_zero(m)


def cyl_kappa(b, Delta, delta, R, D):
    """-ln of the perpendicular signal of a cylinder (Gaussian phase approximation)."""
    return lib().orc_cyl_kappa(b, Delta, delta, R, D)


def rhat(chains):
    """R-hat of chains [C][n] (float64)."""
    x = np.ascontiguousarray(chains, np.float64)
    return lib().orc_rhat(x.reshape(-1) if x.size else np.zeros(1), x.shape[0], x.shape[1], x.shape[1])


def chain_path(kind, acq, lb, ub, step, y, sigma, *, iterations, burnin=0, thin=1, seed,
               voxel=0, chain=0, x0=None, voxel_base=0, adapt_window=0, adapt_target=0.0,
               want_scale=False):
    """State after each iteration t = 0..I of one chain, [I+1][P] float64, and
    the acceptance rate (and the final step multiplier if want_scale)."""
    m, keep = _model(kind, acq, lb, ub, step)
    P = len(keep.lb)
    y = np.ascontiguousarray(y, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    path = np.zeros((iterations + 1, P))
    acc = ct.c_double(0)
    scale = ct.c_double(0)
    o = _Opts(iterations, burnin, thin, chain + 1, seed, voxel_base, 0, 1, adapt_window, adapt_target)
    rc = lib().orc_chain_path(ct.byref(m), _vp(y), ct.c_double(sigma), _vp(x0a), ct.byref(o),
                              ct.c_uint64(voxel), ct.c_int(chain), _vp(path), ct.byref(acc),
                              ct.byref(scale))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return (path, acc.value, scale.value) if want_scale else (path, acc.value)


def ensemble_run(kind, acq, lb, ub, data, sigma, *, iterations, burnin, thin, n_walkers, seed,
                 stretch=2.0, x0=None, sigma_scalar=0.0, voxel_base=0, moments_mode=0,
                 n_threads=0, want_samples=True):
    """Affine-invariant ensemble sampler; outputs as mcmc_run, walkers as chains."""
    P = len(lb)
    m, keep = _model(kind, acq, lb, ub, np.zeros(P))
    data = np.ascontiguousarray(data, np.float32)
    n_vox = data.shape[0]
    sig = None if sigma is None else np.ascontiguousarray(sigma, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    S = n_samples(iterations, burnin, thin)
    L = n_walkers
    mean = np.full((P, n_vox), np.nan)
    std = np.full((P, n_vox), np.nan)
    samples = np.full((S, L, P, n_vox), np.nan) if want_samples else None
    acc = np.zeros((L, n_vox))
    bad = np.zeros((L, n_vox), np.int32)
    used = ct.c_int(0)
    o = _Opts(iterations, burnin, thin, L, seed, voxel_base, moments_mode, n_threads, 0, 0.0)
    rc = lib().orc_ensemble_run(ct.byref(m), _vp(data), ct.c_int64(n_vox), _vp(sig),
                                ct.c_float(sigma_scalar), _vp(x0a), ct.byref(o), ct.c_double(stretch),
                                _vp(mean), _vp(std), _vp(samples), _vp(acc), _vp(bad), ct.byref(used))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return dict(mean=mean, std=std, samples=samples, accept_rate=acc, nonfinite=bad,
                threads=used.value)


def ensemble_path(kind, acq, lb, ub, y, sigma, *, iterations, n_walkers, seed, stretch=2.0,
                  voxel=0, x0=None, voxel_base=0):
    """All walkers after each iteration of one voxel: [I+1][L][P] float64."""
    P = len(lb)
    m, keep = _model(kind, acq, lb, ub, np.zeros(P))
    y = np.ascontiguousarray(y, np.float32)
    x0a = None if x0 is None else np.ascontiguousarray(x0, np.float32)
    path = np.zeros((iterations + 1, n_walkers, P))
    acc = np.zeros((n_walkers, 1))
    o = _Opts(iterations, 0, 1, n_walkers, seed, voxel_base, 0, 1, 0, 0.0)
    rc = lib().orc_ensemble_path(ct.byref(m), _vp(y), ct.c_double(sigma), _vp(x0a), ct.byref(o),
                                 ct.c_double(stretch), ct.c_uint64(voxel), _vp(path), _vp(acc))
    if rc != 0:
        raise ValueError("oracle rejected the arguments")
    return path, acc[:, 0]


def stretch_z(w: int, a: float) -> float:
    return lib().orc_stretch_z(int(w), float(a))


def lockstep(kind, acq, lb, ub, step, y, sigma, theta, prop, w_acc):
    """FP64 likelihoods and decisions for recorded steps of one voxel."""
    m, keep = _model(kind, acq, lb, ub, step)
    th = np.ascontiguousarray(theta, np.float64)
    pr = np.ascontiguousarray(prop, np.float64)
    w = np.ascontiguousarray(w_acc, np.uint32)
    n = th.shape[0]
    L = np.zeros(n)
    Lp = np.zeros(n)
    acc = np.zeros(n, np.int32)
    rc = lib().orc_lockstep(ct.byref(m), _vp(np.ascontiguousarray(y, np.float32)),
                            ct.c_double(sigma), ct.c_int64(n), _vp(th), _vp(pr), _vp(w), _vp(L),
                            _vp(Lp), _vp(acc))
    assert rc == 0
    return L, Lp, acc.astype(bool)


def max_threads() -> int:
    return lib().orc_max_threads()
