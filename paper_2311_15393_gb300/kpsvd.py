"""ctypes binding of libkpsvd.so (include/kpsvd.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device images are torch CUDA tensors holding vec(X), i.e. the
column-major n_r x n_c image (``to_device`` / ``from_device`` convert numpy
arrays).  The library must have been built (``paper_2311_15393_gb300.build``);
importing this module raises if it is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libkpsvd.so")

KP_OK, KP_EINVAL, KP_ENOMEM, KP_ECUDA, KP_ENOTSUP, KP_ENOCONV, KP_EBREAKDOWN, KP_ENUMERIC, KP_ENOROOT, \
    KP_ETIMEOUT, KP_ESTATE = range(11)
BC = {"zero": 0, "reflexive": 1}
PREC = {"f64": 0, "f32": 1, "bf16": 2, "bf16x3": 3, "f16": 4, "e4m3": 5}
SIGMA = {"product": 0, "projected": 1}
LAMBDA = {"gcv": 0, "wgcv": 1, "discrepancy": 2, "opt": 3}
N_FEAT = 256  # spectral features per problem (kp_lambda_features, the MLP's input width)

# every function declared in include/kpsvd.h
EXPORTS = ["kp_create", "kp_destroy", "kp_setup", "kp_forward", "tik_pcg", "choose_lambda", "kp_apply_A",
           "kp_apply_K", "kp_apply_Minv", "kp_get_spectrum", "kp_get_terms", "kp_get_kpsvd", "kp_get_rank",
           "kp_set_option", "kp_launch_count", "kp_time_parts", "kp_test_bounded_wait", "kp_status_str", "kp_last_error", "kp_apply_Minv_noalloc",
           "kp_solve_batch", "kp_batch_release", "kp_batch_grouped", "kp_lambda_features", "kp_mlp_create", "kp_mlp_destroy", "kp_mlp_param_count",
           "kp_mlp_set_params", "kp_mlp_get_params", "kp_mlp_forward", "kp_mlp_gradients", "kp_mlp_train_step"]


class KpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("replacements", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("status", ctypes.c_int), ("ms_solve", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("res_hist", ctypes.POINTER(ctypes.c_double)), ("res_hist_len", ctypes.c_int)]


class Problem(ctypes.Structure):
    """kp_problem: one problem of a batch."""
    _fields_ = [("psf", ctypes.c_void_p), ("n_r", ctypes.c_int), ("n_c", ctypes.c_int),
                ("center_r", ctypes.c_int), ("center_c", ctypes.c_int), ("bc", ctypes.c_int),
                ("op_rank", ctypes.c_int), ("b", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("lambda_", ctypes.c_double), ("lambda_param", ctypes.c_double), ("info", SolveInfo)]


class BatchOpts(ctypes.Structure):
    """kp_batch_opts."""
    _fields_ = [("op_prec", ctypes.c_int), ("pc_prec", ctypes.c_int), ("vec_prec", ctypes.c_int),
                ("sigma", ctypes.c_int), ("method", ctypes.c_int), ("tol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("flexible", ctypes.c_int), ("workers", ctypes.c_int),
                ("autotune", ctypes.c_int)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libkpsvd.so not built ({path}); run python -m paper_2311_15393_gb300.build")
    lib = ctypes.CDLL(path)
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "kp_create": ([ctypes.POINTER(vp), i, vp], i),
        "kp_destroy": ([vp], None),
        "kp_setup": ([vp, vp, i, i, i, i, i, i, i, i, i, i, i], i),
        "kp_forward": ([vp, vp, vp, d, vp, dp], i),
        "tik_pcg": ([vp, vp, d, d, i, i, vp, i, ctypes.POINTER(SolveInfo)], i),
        "choose_lambda": ([vp, vp, i, d, vp, dp], i),
        "kp_apply_A": ([vp, vp, vp, i], i),
        "kp_apply_K": ([vp, vp, vp, d], i),
        "kp_apply_Minv": ([vp, vp, vp, d], i),
        "kp_get_spectrum": ([vp, dp], i),
        "kp_get_terms": ([vp, dp, dp, dp], i),
        "kp_get_kpsvd": ([vp, dp, dp, dp, dp, dp, dp], i),
        "kp_get_rank": ([vp, ctypes.POINTER(i)], i),
        "kp_set_option": ([vp, ctypes.c_char_p, d], i),
        "kp_launch_count": ([vp, i], ctypes.c_longlong),
        "kp_time_parts": ([vp, d, i, dp, ctypes.POINTER(ctypes.c_longlong)], i),
        "kp_test_bounded_wait": ([vp, d], i),
        "kp_status_str": ([i], ctypes.c_char_p),
        "kp_last_error": ([], ctypes.c_char_p),
        "kp_apply_Minv_noalloc": ([vp, vp, vp, i, i, d, vp, vp, vp], i),
        "kp_solve_batch": ([i, ctypes.POINTER(Problem), i, ctypes.POINTER(BatchOpts), dp], i),
        "kp_batch_release": ([i], None),
        "kp_batch_grouped": ([i, ctypes.POINTER(i), dp, ctypes.POINTER(i)], i),
        "kp_lambda_features": ([vp, vp, vp], i),
        "kp_mlp_create": ([ctypes.POINTER(vp), i, vp, i, i, i], i),
        "kp_mlp_destroy": ([vp], None),
        "kp_mlp_param_count": ([vp], ctypes.c_longlong),
        "kp_mlp_set_params": ([vp, vp], i),
        "kp_mlp_get_params": ([vp, vp], i),
        "kp_mlp_forward": ([vp, vp, i, vp], i),
        "kp_mlp_gradients": ([vp, vp, vp, i, vp, dp], i),
        "kp_mlp_train_step": ([vp, vp, vp, i, ctypes.c_float, dp], i),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


_lib = load_library()


_VEC_DTYPE = {"f64": "float64", "f32": "float32"}


def _dev(t, dtype: str | None, numel: int, device: int, what: str) -> int | None:
    """Device address of tensor ``t`` after the checks the C library cannot
    make on a raw pointer: ``t`` must be a contiguous CUDA tensor of
    ``dtype`` ("float64" / "float32"; None: any) on cuda:``device`` with at
    least ``numel`` elements.  None stays None (the C call decides whether it
    is allowed); an int is taken as a device address the caller vouches for."""
    if t is None or isinstance(t, int):
        return t
    dev = getattr(t, "device", None)
    if dev is None or getattr(dev, "type", None) != "cuda" or dev.index != device:
        raise KpError(KP_EINVAL, f"{what}: needs a CUDA tensor on cuda:{device}, got one on {dev}")
    if dtype is not None and str(t.dtype) != "torch." + dtype:
        raise KpError(KP_EINVAL, f"{what}: needs {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise KpError(KP_EINVAL, f"{what}: needs a contiguous tensor")
    if t.numel() < numel:
        raise KpError(KP_EINVAL, f"{what}: needs at least {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _check(status: int):
    if status != KP_OK:
        msg = _lib.kp_last_error().decode()
        raise KpError(status, f"{_lib.kp_status_str(status).decode()}: {msg}")


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def to_device(X: np.ndarray, dtype=None, device: str = "cuda:0"):
    """numpy n_r x n_c image -> torch CUDA vector vec(X) (column stacking)."""
    import torch
    dtype = dtype or torch.float64
    v = np.ascontiguousarray(np.asarray(X, dtype=np.float64).reshape(-1, order="F"))
    return torch.from_numpy(v).to(device=device, dtype=dtype)


def from_device(t, n_r: int, n_c: int) -> np.ndarray:
    return t.detach().to("cpu").double().numpy().reshape((n_r, n_c), order="F")


def kp_apply_Minv_noalloc(Vc, Vr, sigma, n_r: int, n_c: int, lam: float, r, z, stream: int | None = None):
    """Preconditioner solve without any device allocation (see include/kpsvd.h):
    Vc, Vr float32 column-major factors, sigma float64 spectrum, r, z float32."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    d = torch.cuda.current_device()
    N = max(n_r, 0) * max(n_c, 0)
    _check(_lib.kp_apply_Minv_noalloc(
        _dev(Vc, "float32", max(n_r, 0) ** 2, d, "Vc"), _dev(Vr, "float32", max(n_c, 0) ** 2, d, "Vr"),
        _dev(sigma, "float64", N, d, "sigma"), n_r, n_c, lam, _dev(r, "float32", N, d, "r"),
        _dev(z, "float32", N, d, "z"), stream))


@dataclass
class Info:
    iters: int
    replacements: int
    rel_res: float
    status: int
    ms_solve: float
    res_hist: np.ndarray
    ms_setup: float = 0.0


class KpContext:
    """Owns one kp_ctx.  All methods mirror the C ABI.  Image arguments are
    checked to be contiguous CUDA tensors on the context's device with the
    element type and size of the problem set up (before kp_setup only the
    device is checked; the C call then returns KP_ESTATE)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        _check(_lib.kp_create(ctypes.byref(h), device, stream))
        self._h = h
        self.device = device
        self.n_r = self.n_c = 0
        self.vec = "f64"

    def _img(self, t, what: str):
        if self.n_r == 0:
            return _dev(t, None, 0, self.device, what)
        return _dev(t, _VEC_DTYPE[self.vec], self.n_r * self.n_c, self.device, what)

    def close(self):
        if getattr(self, "_h", None):
            _lib.kp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- setup / solve -------------------------------------------------------------
    def kp_setup(self, psf_dev, n_r: int, n_c: int, center, bc: str = "reflexive", op_rank: int = 0,
                 op_prec: str = "f64", pc_prec: str = "f64", vec_prec: str = "f64", sigma: str = "projected",
                 pc_rank: int = 1):
        psf = _dev(psf_dev, "float64", max(n_r, 0) * max(n_c, 0), self.device, "psf")
        _check(_lib.kp_setup(self._h, psf, n_r, n_c, int(center[0]), int(center[1]), BC[bc], op_rank, pc_rank,
                             PREC[op_prec], PREC[pc_prec], PREC[vec_prec], SIGMA[sigma]))
        self.n_r, self.n_c, self.vec = n_r, n_c, vec_prec

    def kp_forward(self, x, g, noise_level: float, b) -> float:
        nn = ctypes.c_double(0.0)
        _check(_lib.kp_forward(self._h, self._img(x, "x"), self._img(g, "g"), noise_level, self._img(b, "b"),
                               ctypes.byref(nn)))
        return nn.value

    def tik_pcg(self, b, lam: float, tol: float, maxit: int, flexible: bool, x, warm_start: bool = False,
                hist_len: int = 0, check: bool = True) -> Info:
        info = SolveInfo()
        hist = np.zeros(max(hist_len, 0), dtype=np.float64)
        if hist_len > 0:
            info.res_hist = _dptr(hist)
            info.res_hist_len = hist_len
        st = _lib.tik_pcg(self._h, self._img(b, "b"), lam, tol, maxit, 1 if flexible else 0, self._img(x, "x"),
                          1 if warm_start else 0, ctypes.byref(info))
        if check and st not in (KP_OK,):
            _check(st)
        n = min(hist_len, info.iters + 1) if hist_len > 0 else 0
        return Info(info.iters, info.replacements, info.rel_res, st, info.ms_solve, hist[:n], info.ms_setup)

    def choose_lambda(self, b, method: str, param: float = 0.0, x_true=None) -> float:
        lam = ctypes.c_double(0.0)
        _check(_lib.choose_lambda(self._h, self._img(b, "b"), LAMBDA[method], param, self._img(x_true, "x_true"),
                                  ctypes.byref(lam)))
        return lam.value

    # -- hooks ---------------------------------------------------------------------
    def kp_lambda_features(self, b, out):
        """256 spectral features of b (device float32 tensor ``out``)."""
        _check(_lib.kp_lambda_features(self._h, self._img(b, "b"), _dev(out, "float32", N_FEAT, self.device, "out")))

    def kp_apply_A(self, x, y, transpose: bool = False):
        _check(_lib.kp_apply_A(self._h, self._img(x, "x"), self._img(y, "y"), 1 if transpose else 0))

    def kp_apply_K(self, x, y, lam: float):
        _check(_lib.kp_apply_K(self._h, self._img(x, "x"), self._img(y, "y"), lam))

    def kp_apply_Minv(self, r, z, lam: float):
        _check(_lib.kp_apply_Minv(self._h, self._img(r, "r"), self._img(z, "z"), lam))

    def kp_get_rank(self) -> int:
        r = ctypes.c_int(0)
        _check(_lib.kp_get_rank(self._h, ctypes.byref(r)))
        return r.value

    def kp_get_spectrum(self) -> np.ndarray:
        s = np.zeros(self.n_r * self.n_c)
        _check(_lib.kp_get_spectrum(self._h, _dptr(s)))
        return s.reshape((self.n_r, self.n_c), order="F")

    def kp_get_terms(self):
        r = self.kp_get_rank()
        s, u, v = np.zeros(r), np.zeros(self.n_r * r), np.zeros(self.n_c * r)
        _check(_lib.kp_get_terms(self._h, _dptr(s), _dptr(u), _dptr(v)))
        return s, u.reshape((self.n_r, r), order="F"), v.reshape((self.n_c, r), order="F")

    def kp_get_kpsvd(self):
        nr, nc = self.n_r, self.n_c
        sr, Ur, Vr = np.zeros(nc), np.zeros(nc * nc), np.zeros(nc * nc)
        sc, Uc, Vc = np.zeros(nr), np.zeros(nr * nr), np.zeros(nr * nr)
        _check(_lib.kp_get_kpsvd(self._h, _dptr(sr), _dptr(Ur), _dptr(Vr), _dptr(sc), _dptr(Uc), _dptr(Vc)))
        f = lambda a, n: a.reshape((n, n), order="F")  # noqa: E731
        return dict(sr=sr, Ur=f(Ur, nc), Vr=f(Vr, nc), sc=sc, Uc=f(Uc, nr), Vc=f(Vc, nr))

    def kp_set_option(self, name: str, value: float):
        _check(_lib.kp_set_option(self._h, name.encode(), float(value)))

    def kp_launch_count(self, reset: bool = False) -> int:
        return int(_lib.kp_launch_count(self._h, 1 if reset else 0))

    def kp_test_bounded_wait(self, limit_ms: float) -> int:
        """Status of one bounded device wait that nothing releases (KP_ETIMEOUT)."""
        return int(_lib.kp_test_bounded_wait(self._h, limit_ms))

    def kp_time_parts(self, lam: float, reps: int = 20):
        """Device ms per launch and kernels per launch of the iteration's parts:
        K application, preconditioner solve, vector phase, residual replacement."""
        ms = np.zeros(4)
        ln = (ctypes.c_longlong * 4)()
        _check(_lib.kp_time_parts(self._h, lam, reps, _dptr(ms), ln))
        return ms, [int(v) for v in ln]


def kp_solve_batch(problems, op_prec: str = "bf16", pc_prec: str = "f16", vec_prec: str = "f32",
                   sigma: str = "projected", method: str = "gcv", tol: float = 1e-7, maxit: int = 500,
                   flexible: bool = True, workers: int = 0, device: int = 0, check: bool = True,
                   autotune: int = 0):
    """Solve a batch of independent problems (kp_solve_batch).  ``problems``:
    dicts with psf, b, x (torch CUDA tensors), n_r, n_c, center, bc, op_rank and
    optionally lam (> 0: fixed) and lambda_param.  ``workers`` 0: the grouped
    form (one launch per iteration step over all problems); > 0: host
    threads.  Returns (status, ms_total, [(lambda, Info), ...]) in the order
    given.  ``autotune`` (grouped form): 0 one tile shape for all problems,
    1 shapes chosen by timing, 2 the size rule of single solves."""
    arr = (Problem * len(problems))()
    vt = _VEC_DTYPE.get(vec_prec, "float32")
    for k, p in enumerate(problems):
        q = arr[k]
        N = max(p["n_r"], 0) * max(p["n_c"], 0)
        q.psf = _dev(p["psf"], "float64", N, device, f"problem {k} psf")
        q.b = _dev(p["b"], vt, N, device, f"problem {k} b")
        q.x = _dev(p["x"], vt, N, device, f"problem {k} x")
        q.n_r, q.n_c = p["n_r"], p["n_c"]
        q.center_r, q.center_c = int(p["center"][0]), int(p["center"][1])
        q.bc, q.op_rank = BC[p["bc"]], p["op_rank"]
        q.lambda_ = p.get("lam") or 0.0
        q.lambda_param = p.get("lambda_param", 0.0)
    o = BatchOpts(PREC[op_prec], PREC[pc_prec], PREC[vec_prec], SIGMA[sigma], LAMBDA[method], tol, maxit,
                  1 if flexible else 0, workers, int(autotune))
    ms = ctypes.c_double(0.0)
    st = _lib.kp_solve_batch(device, arr, len(problems), ctypes.byref(o), ctypes.byref(ms))
    if check and st != KP_OK:
        _check(st)
    out = [(q.lambda_, Info(q.info.iters, q.info.replacements, q.info.rel_res, q.info.status, q.info.ms_solve,
                            np.zeros(0))) for q in arr]
    return st, ms.value, out


def kp_batch_grouped(device: int = 0):
    """(problems the last grouped kp_solve_batch ran in its grouped loop, the
    loop's passes, [ms before the loop, ms building it, ms running it],
    [launches per problem iteration, grouped launches per pass, the same
    for the residual replacement, setups ran as fibers, fiber yields])."""
    passes = ctypes.c_int(0)
    ms = (ctypes.c_double * 3)()
    shape = (ctypes.c_int * 6)()
    n = _lib.kp_batch_grouped(device, ctypes.byref(passes), ms, shape)
    return n, passes.value, list(ms), list(shape)


class Mlp:
    """Owns one kp_mlp (learned lambda); methods mirror the C ABI.  Parameter
    vectors are float32 numpy arrays of param_count entries."""

    def __init__(self, width: int = 256, depth: int = 3, max_batch: int = 1024, device: int = 0,
                 stream: int | None = None):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        _check(_lib.kp_mlp_create(ctypes.byref(h), device, stream, width, depth, max_batch))
        self._h = h
        self.device = device
        self.param_count = int(_lib.kp_mlp_param_count(h))

    def _batch(self, X, what: str = "X"):
        """(batch, device address) of a contiguous float32 batch x 256 CUDA tensor."""
        if getattr(X, "dim", None) is None or X.dim() != 2 or X.shape[1] != N_FEAT:
            raise KpError(KP_EINVAL, f"{what}: needs a batch x {N_FEAT} tensor")
        return X.shape[0], _dev(X, "float32", X.shape[0] * N_FEAT, self.device, what)

    def close(self):
        if getattr(self, "_h", None):
            _lib.kp_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, params: np.ndarray):
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.param_count
        _check(_lib.kp_mlp_set_params(self._h, a.ctypes.data))

    def get_params(self) -> np.ndarray:
        a = np.empty(self.param_count, dtype=np.float32)
        _check(_lib.kp_mlp_get_params(self._h, a.ctypes.data))
        return a

    def forward(self, X, y):
        n, xp = self._batch(X)
        _check(_lib.kp_mlp_forward(self._h, xp, n, _dev(y, "float32", n, self.device, "y")))

    def gradients(self, X, labels):
        n, xp = self._batch(X)
        g = np.empty(self.param_count, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        _check(_lib.kp_mlp_gradients(self._h, xp, _dev(labels, "float32", n, self.device, "labels"), n,
                                     g.ctypes.data, ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, X, labels, lr: float) -> float:
        n, xp = self._batch(X)
        loss = ctypes.c_double(0.0)
        _check(_lib.kp_mlp_train_step(self._h, xp, _dev(labels, "float32", n, self.device, "labels"), n, lr,
                                      ctypes.byref(loss)))
        return loss.value

