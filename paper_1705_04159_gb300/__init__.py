"""GB300 BPMF Gibbs sampler: Python binding of the C ABI in include/bpmf.h.

The functions here carry the same names as the C entry points and only
marshal arguments (numpy arrays for host buffers, CUDA torch tensors for
device buffers, which select BPMF_DEVPTR).  Every step of the sampler runs in
the CUDA library ``_build/libbpmf_gb300.so``; there is no other backend, and
loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "BpmfError", "Config", "lib", "build", "bpmf_config_default", "bpmf_init", "bpmf_set_test",
    "bpmf_sample_hyper", "bpmf_sweep", "bpmf_step", "bpmf_predict", "bpmf_test_rmse",
    "bpmf_get_state", "bpmf_set_state", "bpmf_get_structure", "bpmf_get_hyper_stats",
    "bpmf_get_sweep_info", "bpmf_set_timing", "bpmf_get_timing", "bpmf_destroy", "bpmf_strerror",
    "bpmf_hyper_stats_noalloc", "bpmf_set_graph", "bpmf_get_thresholds", "bpmf_set_thresholds",
    "bpmf_set_test_hold", "bpmf_server_create", "bpmf_server_submit", "bpmf_server_poll",
    "bpmf_server_wait", "bpmf_server_stats", "bpmf_server_clock", "bpmf_server_destroy",
    "Sampler", "Server", "Job", "JobResult", "TIMERS",
    "USERS", "MOVIES", "PATH_PLAIN", "PATH_BINNED", "PATH_MIXED", "DEVPTR",
]

OK, EINVAL, ENOMEM, ECUDA, ENOTPD, ERNG, ESTATE, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
USERS, MOVIES = 0, 1
PATH_PLAIN, PATH_BINNED, PATH_MIXED = 0, 1, 2
DEVPTR = 1

SYMBOLS = [
    "bpmf_config_default", "bpmf_init", "bpmf_set_test", "bpmf_sample_hyper", "bpmf_sweep",
    "bpmf_step", "bpmf_predict", "bpmf_test_rmse", "bpmf_get_state", "bpmf_set_state",
    "bpmf_get_structure", "bpmf_get_hyper_stats", "bpmf_get_sweep_info", "bpmf_destroy",
    "bpmf_strerror", "bpmf_last_error", "bpmf_set_timing", "bpmf_get_timing",
    "bpmf_hyper_stats_noalloc", "bpmf_set_graph", "bpmf_get_thresholds", "bpmf_set_thresholds",
    "bpmf_set_test_hold", "bpmf_server_create", "bpmf_server_submit", "bpmf_server_poll",
    "bpmf_server_wait", "bpmf_server_stats", "bpmf_server_clock", "bpmf_server_destroy",
]
TIMERS = ["hyper_reduce", "hyper_draw", "rows_users", "rows_movies", "fp64_redo", "predict"]


class BpmfError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = f"{where}: {bpmf_strerror(code)} ({code})"
        detail = lib().bpmf_last_error().decode() if _lib is not None else ""
        if detail:
            msg += f": {detail}"
        super().__init__(msg)


class Config(C.Structure):
    _fields_ = [
        ("K", C.c_int32), ("path", C.c_int32), ("alpha", C.c_double), ("beta0", C.c_double),
        ("nu0", C.c_double), ("mu0", C.c_void_p), ("W0", C.c_void_p), ("seed", C.c_uint64),
        ("order", C.c_int32), ("burnin", C.c_int32), ("light_max", C.c_int32),
        ("hub_min", C.c_int32), ("tiny_max", C.c_int32), ("heavy_kernel", C.c_int32),
        ("autotune", C.c_int32), ("pivot_rel", C.c_double),
    ]


class Job(C.Structure):
    """bpmf_job: one server job (host arrays are copied at submission)."""
    _fields_ = [
        ("M", C.c_int64), ("N", C.c_int64), ("nnz", C.c_int64),
        ("row", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
        ("n_test", C.c_int64), ("test_row", C.c_void_p), ("test_col", C.c_void_p),
        ("test_val", C.c_void_p), ("cfg", Config), ("iterations", C.c_int32),
        ("U_out", C.c_void_p), ("V_out", C.c_void_p),
    ]


class JobResult(C.Structure):
    """bpmf_job_result."""
    _fields_ = [
        ("status", C.c_int32), ("iterations", C.c_int32), ("rmse_sample", C.c_double),
        ("rmse_mean", C.c_double), ("t_submit", C.c_double), ("t_start", C.c_double),
        ("t_end", C.c_double), ("device_bytes", C.c_int64),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (nvcc) if it is missing or stale."""
    return _build.build(force=force)


def lib():
    """The loaded CUDA library.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"CUDA library {path} is not built; call paper_1705_04159_gb300.build()")
        L = C.CDLL(path)
        P, i64, i32, u32 = C.c_void_p, C.c_int64, C.c_int32, C.c_uint32
        L.bpmf_config_default.argtypes = [C.POINTER(Config), i32]
        L.bpmf_config_default.restype = None
        L.bpmf_init.argtypes = [C.POINTER(C.c_void_p), i64, i64, i64, P, P, P, C.POINTER(Config),
                                P, u32]
        L.bpmf_set_test.argtypes = [P, i64, P, P, P, u32]
        L.bpmf_sample_hyper.argtypes = [P, C.c_int]
        L.bpmf_sweep.argtypes = [P, C.c_int]
        L.bpmf_step.argtypes = [P]
        L.bpmf_predict.argtypes = [P, i64, P, P, P, u32]
        L.bpmf_test_rmse.argtypes = [P, P, P]
        L.bpmf_get_state.argtypes = [P, P, P, P, P, u32]
        L.bpmf_set_state.argtypes = [P, P, P, P, i64, u32]
        L.bpmf_get_structure.argtypes = [P, C.c_int, P, P, P, P, P]
        L.bpmf_get_hyper_stats.argtypes = [P, C.c_int, P, P]
        L.bpmf_get_sweep_info.argtypes = [P, C.c_int, P, P]
        L.bpmf_set_timing.argtypes = [P, C.c_int]
        L.bpmf_set_graph.argtypes = [P, C.c_int]
        L.bpmf_set_limits.argtypes = [P, i32, i64]
        L.bpmf_set_test_hold.argtypes = [P, i32]
        L.bpmf_get_thresholds.argtypes = [P, C.c_int, P]
        L.bpmf_set_thresholds.argtypes = [P, C.c_int, P]
        L.bpmf_get_timing.argtypes = [P, P, P, P]
        L.bpmf_hyper_stats_noalloc.argtypes = [P, i64, i32, P, P, P]
        L.bpmf_destroy.argtypes = [P]
        L.bpmf_destroy.restype = None
        L.bpmf_server_create.argtypes = [C.POINTER(C.c_void_p), i64, i32]
        L.bpmf_server_submit.argtypes = [P, C.POINTER(Job), C.POINTER(C.c_int64)]
        L.bpmf_server_poll.argtypes = [P, i64, C.POINTER(JobResult)]
        L.bpmf_server_wait.argtypes = [P, i64, C.POINTER(JobResult)]
        L.bpmf_server_stats.argtypes = [P, P]
        L.bpmf_server_clock.argtypes = [P]
        L.bpmf_server_clock.restype = C.c_double
        L.bpmf_server_trace.argtypes = [P, i64, i32, P, P, P]
        L.bpmf_server_destroy.argtypes = [P]
        L.bpmf_server_destroy.restype = None
        L.bpmf_strerror.argtypes = [C.c_int]
        L.bpmf_strerror.restype = C.c_char_p
        L.bpmf_last_error.argtypes = []
        L.bpmf_last_error.restype = C.c_char_p
        _lib = L
    return _lib


# ------------------------------------------------------------ marshalling --

def _is_cuda_tensor(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x, dtype):
    """(pointer, keepalive, is_device) for a numpy array or a CUDA tensor."""
    if x is None:
        return None, None, False
    if _is_cuda_tensor(x):
        import torch
        want = {np.int32: torch.int32, np.float32: torch.float32, np.int64: torch.int64,
                np.float64: torch.float64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"device tensor must be contiguous {want}")
        return x.data_ptr(), x, True
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a, False


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def _check(rc, where):
    if rc != OK:
        raise BpmfError(rc, where)


# ------------------------------------------------------- C-named wrappers --

def bpmf_strerror(code: int) -> str:
    return lib().bpmf_strerror(code).decode()


def bpmf_config_default(K: int) -> Config:
    cfg = Config()
    lib().bpmf_config_default(C.byref(cfg), K)
    return cfg


def bpmf_init(M, N, row, col, val, cfg: Config, stream=None, mu0=None, W0=None):
    """Returns an opaque handle (int).  Device tensors select BPMF_DEVPTR."""
    pr, kr, dr = _ptr(row, np.int32)
    pc, kc, dc = _ptr(col, np.int32)
    pv, kv, dv = _ptr(val, np.float32)
    if len({dr, dc, dv}) != 1:
        raise TypeError("row, col and val must all be host arrays or all device tensors")
    nnz = int(len(row))
    keep = []
    if mu0 is not None:
        m = np.ascontiguousarray(mu0, np.float64)
        keep.append(m)
        cfg.mu0 = m.ctypes.data
    if W0 is not None:
        w = np.ascontiguousarray(W0, np.float64)
        keep.append(w)
        cfg.W0 = w.ctypes.data
    h = C.c_void_p()
    rc = lib().bpmf_init(C.byref(h), int(M), int(N), nnz, pr, pc, pv, C.byref(cfg),
                         _stream_ptr(stream), DEVPTR if dr else 0)
    cfg.mu0 = None
    cfg.W0 = None
    _check(rc, "bpmf_init")
    return h.value


def bpmf_set_test(h, row, col, val):
    pr, kr, dr = _ptr(row, np.int32)
    pc, kc, dc = _ptr(col, np.int32)
    pv, kv, dv = _ptr(val, np.float32)
    _check(lib().bpmf_set_test(h, int(len(row)), pr, pc, pv, DEVPTR if dr else 0), "bpmf_set_test")


def bpmf_sample_hyper(h, side):
    _check(lib().bpmf_sample_hyper(h, side), "bpmf_sample_hyper")


def bpmf_sweep(h, side):
    _check(lib().bpmf_sweep(h, side), "bpmf_sweep")


def bpmf_step(h):
    _check(lib().bpmf_step(h), "bpmf_step")


def bpmf_predict(h, row, col, out=None):
    n = int(len(row))
    pr, kr, dr = _ptr(row, np.int32)
    pc, kc, dc = _ptr(col, np.int32)
    if out is None:
        if dr:
            import torch
            out = torch.empty(n, dtype=torch.float32, device=row.device)
        else:
            out = np.empty(n, np.float32)
    po, ko, do = _ptr(out, np.float32)
    _check(lib().bpmf_predict(h, n, pr, pc, po, DEVPTR if dr else 0), "bpmf_predict")
    return out


def bpmf_test_rmse(h):
    a = C.c_double()
    b = C.c_double()
    _check(lib().bpmf_test_rmse(h, C.byref(a), C.byref(b)), "bpmf_test_rmse")
    return a.value, b.value


def bpmf_get_state(h, M, N, K, U=None, V=None):
    """Returns (U, V, hyper, iter); U/V may be given as CUDA tensors (DEVPTR)."""
    dev = _is_cuda_tensor(U)
    if U is None:
        U = np.empty((M, K), np.float32)
    if V is None:
        V = np.empty((N, K), np.float32)
    hyper = np.empty(2 * (K * K + K), np.float64)
    it = C.c_int64()
    pu, ku, _ = _ptr(U, np.float32)
    pv, kv, _ = _ptr(V, np.float32)
    _check(lib().bpmf_get_state(h, pu, pv, hyper.ctypes.data, C.byref(it), DEVPTR if dev else 0),
           "bpmf_get_state")
    return U, V, hyper, it.value


def bpmf_set_state(h, U=None, V=None, hyper=None, it=0):
    dev = _is_cuda_tensor(U) or _is_cuda_tensor(V)
    pu, ku, _ = _ptr(U, np.float32)
    pv, kv, _ = _ptr(V, np.float32)
    hy = None if hyper is None else np.ascontiguousarray(hyper, np.float64)
    _check(lib().bpmf_set_state(h, pu, pv, None if hy is None else hy.ctypes.data, int(it),
                                DEVPTR if dev else 0), "bpmf_set_state")


def bpmf_get_structure(h, side, R, nnz):
    ptr = np.empty(R + 1, np.int64)
    idx = np.empty(max(nnz, 1), np.int32)
    val = np.empty(max(nnz, 1), np.float32)
    perm = np.empty(R, np.int32)
    mean = C.c_double()
    _check(lib().bpmf_get_structure(h, side, ptr.ctypes.data, idx.ctypes.data, val.ctypes.data,
                                    perm.ctypes.data, C.byref(mean)), "bpmf_get_structure")
    return ptr, idx[:nnz], val[:nnz], perm, mean.value


def bpmf_get_hyper_stats(h, side, K):
    xbar = np.empty(K)
    S = np.empty((K, K))
    _check(lib().bpmf_get_hyper_stats(h, side, xbar.ctypes.data, S.ctypes.data),
           "bpmf_get_hyper_stats")
    return xbar, S


def bpmf_get_sweep_info(h, side):
    bins = np.zeros(4, np.int64)
    f = C.c_int64()
    _check(lib().bpmf_get_sweep_info(h, side, bins.ctypes.data, C.byref(f)), "bpmf_get_sweep_info")
    return bins, f.value


def bpmf_set_timing(h, enable=True):
    _check(lib().bpmf_set_timing(h, 1 if enable else 0), "bpmf_set_timing")


def bpmf_get_thresholds(h, side):
    """(tiny_max, light_max, hub_min, heavy kernel, persistent consumers) of `side`."""
    t = np.zeros(5, np.int64)
    _check(lib().bpmf_get_thresholds(h, side, t.ctypes.data), "bpmf_get_thresholds")
    return tuple(int(x) for x in t)


def bpmf_set_thresholds(h, side, thresholds):
    """Applies five values in bpmf_get_thresholds' order to `side`."""
    t = np.ascontiguousarray(thresholds, dtype=np.int64)
    if t.shape != (5,):
        raise ValueError("thresholds: five integers")
    _check(lib().bpmf_set_thresholds(h, side, t.ctypes.data), "bpmf_set_thresholds")


def bpmf_set_graph(h, enable=True):
    _check(lib().bpmf_set_graph(h, 1 if enable else 0), "bpmf_set_graph")


def bpmf_set_limits(h, gamma_cap=-1, wait_ns=0):
    """Failure-path limits: Gamma attempts per draw (negative: default 64) and
    the bound of each persistent-kernel wait in ns (0: default 2 s)."""
    _check(lib().bpmf_set_limits(h, int(gamma_cap), int(wait_ns)), "bpmf_set_limits")


def bpmf_set_test_hold(h, hold):
    """Failure-path testing: 1 makes the persistent kernel withhold one
    arrive, so that its bounded wait runs out; 0 restores normal operation."""
    _check(lib().bpmf_set_test_hold(h, int(hold)), "bpmf_set_test_hold")


def bpmf_get_timing(h):
    """({timer: ms}, {timer: phases}, kernels launched) since timing was enabled."""
    ms = np.zeros(len(TIMERS))
    cnt = np.zeros(len(TIMERS), np.int64)
    k = C.c_int64()
    _check(lib().bpmf_get_timing(h, ms.ctypes.data, cnt.ctypes.data, C.byref(k)),
           "bpmf_get_timing")
    return dict(zip(TIMERS, ms.tolist())), dict(zip(TIMERS, cnt.tolist())), k.value


def _check_noalloc_args(X, R, K, xbar, S):
    """Argument checks of bpmf_hyper_stats_noalloc that the C call cannot make
    (it sees bare pointers): device tensors on one device, each large enough
    for R x K, K and K x K elements.  Raises TypeError or ValueError."""
    if not (_is_cuda_tensor(X) and _is_cuda_tensor(xbar) and _is_cuda_tensor(S)):
        raise TypeError("bpmf_hyper_stats_noalloc takes device tensors only")
    if not (X.device == xbar.device == S.device):
        raise ValueError("bpmf_hyper_stats_noalloc: X, xbar and S must be on one device")
    R, K = int(R), int(K)
    if R < 1 or K < 1:
        raise ValueError("bpmf_hyper_stats_noalloc: R and K must be positive")
    if X.numel() < R * K or xbar.numel() < K or S.numel() < K * K:
        raise ValueError(f"bpmf_hyper_stats_noalloc: buffers too small for R={R}, K={K} "
                         f"(X {X.numel()}, xbar {xbar.numel()}, S {S.numel()} elements)")


def bpmf_hyper_stats_noalloc(X, R, K, xbar, S, stream=None):
    """Row mean and centred scatter of the device factor matrix X (R x K float32)
    into the device tensors xbar (K float64) and S (K*K float64), with no
    allocation (scratch compiled into the library; see include/bpmf.h).  The
    call runs with X's device current, on `stream` (default: that device's
    current stream)."""
    _check_noalloc_args(X, R, K, xbar, S)
    import torch
    with torch.cuda.device(X.device):
        px, kx, _ = _ptr(X, np.float32)
        pm, km, _ = _ptr(xbar, np.float64)
        ps, ks, _ = _ptr(S, np.float64)
        _check(lib().bpmf_hyper_stats_noalloc(px, int(R), int(K), pm, ps, _stream_ptr(stream)),
               "bpmf_hyper_stats_noalloc")


def bpmf_destroy(h):
    if h:
        lib().bpmf_destroy(h)


def bpmf_server_create(budget_bytes=0, max_resident=0):
    h = C.c_void_p()
    _check(lib().bpmf_server_create(C.byref(h), int(budget_bytes), int(max_resident)),
           "bpmf_server_create")
    return h


def bpmf_server_submit(srv, job):
    jid = C.c_int64()
    _check(lib().bpmf_server_submit(srv, C.byref(job), C.byref(jid)), "bpmf_server_submit")
    return jid.value


def bpmf_server_poll(srv, jid):
    """The JobResult once job `jid` is done, else None."""
    r = JobResult()
    rc = lib().bpmf_server_poll(srv, int(jid), C.byref(r))
    if rc == EBUSY:
        return None
    _check(rc, "bpmf_server_poll")
    return r


def bpmf_server_wait(srv, jid):
    r = JobResult()
    _check(lib().bpmf_server_wait(srv, int(jid), C.byref(r)), "bpmf_server_wait")
    return r


def bpmf_server_stats(srv):
    st = np.zeros(6, np.int64)
    _check(lib().bpmf_server_stats(srv, st.ctypes.data), "bpmf_server_stats")
    return dict(zip(("queued", "resident", "done", "peak_resident", "peak_bytes", "budget"),
                    st.tolist()))


def bpmf_server_clock(srv):
    return lib().bpmf_server_clock(srv)


def bpmf_server_trace(srv, jid, n=256):
    """(start_ms, end_ms) arrays of the device interval of each traced
    iteration of finished job `jid`, on the server's shared clock."""
    a = np.empty(n)
    b = np.empty(n)
    m = C.c_int32()
    _check(lib().bpmf_server_trace(srv, int(jid), int(n), a.ctypes.data, b.ctypes.data,
                                   C.byref(m)), "bpmf_server_trace")
    k = min(n, m.value)
    return a[:k], b[:k]


def bpmf_server_destroy(srv):
    if srv:
        lib().bpmf_server_destroy(srv)


# -------------------------------------------------------------- wrapper --

class Sampler:
    """A BPMF sampler on the current CUDA device (one handle of the C ABI)."""

    def __init__(self, M, N, row, col, val, K, alpha=2.0, beta0=2.0, nu0=None, mu0=None, W0=None,
                 seed=0, path=PATH_MIXED, order=0, burnin=0, light_max=-1, hub_min=-1,
                 tiny_max=-1, heavy_kernel=0, autotune=0, stream=None, pivot_rel=None):
        cfg = bpmf_config_default(K)
        cfg.alpha = float(alpha)
        cfg.beta0 = float(beta0)
        cfg.nu0 = float(K if nu0 is None else nu0)
        cfg.seed = int(seed)
        cfg.path = int(path)
        cfg.order = int(order)
        cfg.burnin = int(burnin)
        cfg.light_max = int(light_max)
        cfg.hub_min = int(hub_min)
        cfg.tiny_max = int(tiny_max)
        cfg.heavy_kernel = int(heavy_kernel)
        cfg.autotune = int(autotune)
        if pivot_rel is not None:
            cfg.pivot_rel = float(pivot_rel)
        self.M, self.N, self.K = int(M), int(N), int(K)
        self.nnz = int(len(row))
        self.h = bpmf_init(M, N, row, col, val, cfg, stream=stream, mu0=mu0, W0=W0)

    def close(self):
        if self.h:
            bpmf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_test(self, row, col, val):
        bpmf_set_test(self.h, row, col, val)

    def sample_hyper(self, side):
        bpmf_sample_hyper(self.h, side)

    def sweep(self, side):
        bpmf_sweep(self.h, side)

    def step(self):
        bpmf_step(self.h)

    def predict(self, row, col, out=None):
        return bpmf_predict(self.h, row, col, out)

    def test_rmse(self):
        return bpmf_test_rmse(self.h)

    def get_state(self, U=None, V=None):
        return bpmf_get_state(self.h, self.M, self.N, self.K, U, V)

    def set_state(self, U=None, V=None, hyper=None, it=0):
        bpmf_set_state(self.h, U, V, hyper, it)

    def structure(self, side):
        R = self.M if side == USERS else self.N
        return bpmf_get_structure(self.h, side, R, self.nnz)

    def hyper_stats(self, side):
        return bpmf_get_hyper_stats(self.h, side, self.K)

    def sweep_info(self, side):
        return bpmf_get_sweep_info(self.h, side)

    def set_timing(self, enable=True):
        bpmf_set_timing(self.h, enable)

    def timing(self):
        return bpmf_get_timing(self.h)

    def set_graph(self, enable=True):
        bpmf_set_graph(self.h, enable)

    def set_limits(self, gamma_cap=-1, wait_ns=0):
        bpmf_set_limits(self.h, gamma_cap, wait_ns)

    def set_test_hold(self, hold):
        bpmf_set_test_hold(self.h, hold)

    def thresholds(self, side):
        return bpmf_get_thresholds(self.h, side)

    def set_thresholds(self, side, thresholds):
        bpmf_set_thresholds(self.h, side, thresholds)

    def hyper(self):
        """(Lambda_U, mu_U, Lambda_V, mu_V) from the packed state."""
        K = self.K
        _, _, hy, _ = self.get_state(U=np.empty((self.M, K), np.float32),
                                     V=np.empty((self.N, K), np.float32))
        o = K * K + K
        return (hy[:K * K].reshape(K, K), hy[K * K:o], hy[o:o + K * K].reshape(K, K),
                hy[o + K * K:])


class Server:
    """Continuous-batching job server on the current CUDA device (bpmf_server_*)."""

    def __init__(self, budget_bytes=0, max_resident=0):
        self.h = bpmf_server_create(budget_bytes, max_resident)
        self._outs = {}

    def submit(self, M, N, row, col, val, K, iterations, test=None, alpha=2.0, seed=0,
               path=PATH_MIXED, burnin=0, want_factors=False, **cfg_kw):
        """Queues a job; returns its id.  Arrays are host numpy arrays, copied
        by the call.  With want_factors the final U, V come back from result()."""
        cfg = bpmf_config_default(K)
        cfg.alpha = float(alpha)
        cfg.seed = int(seed)
        cfg.path = int(path)
        cfg.burnin = int(burnin)
        for k, v in cfg_kw.items():
            setattr(cfg, k, v)
        row = np.ascontiguousarray(row, np.int32)
        col = np.ascontiguousarray(col, np.int32)
        val = np.ascontiguousarray(val, np.float32)
        j = Job()
        j.M, j.N, j.nnz = int(M), int(N), len(row)
        j.row, j.col, j.val = row.ctypes.data, col.ctypes.data, val.ctypes.data
        keep = [row, col, val]
        if test is not None:
            tr, tc, tv = (np.ascontiguousarray(test[0], np.int32),
                          np.ascontiguousarray(test[1], np.int32),
                          np.ascontiguousarray(test[2], np.float32))
            j.n_test = len(tr)
            j.test_row, j.test_col, j.test_val = tr.ctypes.data, tc.ctypes.data, tv.ctypes.data
            keep += [tr, tc, tv]
        j.cfg = cfg
        j.iterations = int(iterations)
        outs = None
        if want_factors:
            outs = (np.empty((M, K), np.float32), np.empty((N, K), np.float32))
            j.U_out, j.V_out = outs[0].ctypes.data, outs[1].ctypes.data
        jid = bpmf_server_submit(self.h, j)
        del keep  # copied by the call
        self._outs[jid] = outs
        return jid

    def poll(self, jid):
        return bpmf_server_poll(self.h, jid)

    def result(self, jid):
        """(JobResult, (U, V) or None), waiting for the job."""
        r = bpmf_server_wait(self.h, jid)
        return r, self._outs.pop(jid, None)

    def stats(self):
        return bpmf_server_stats(self.h)

    def trace(self, jid, n=256):
        return bpmf_server_trace(self.h, jid, n)

    def clock(self):
        return bpmf_server_clock(self.h)

    def close(self):
        if getattr(self, "h", None):
            bpmf_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
