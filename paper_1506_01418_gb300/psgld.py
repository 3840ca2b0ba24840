"""Thin ctypes binding of the C ABI in include/psgld.h.

Argument marshalling only: every step of the sampler runs in the CUDA library
``libpsgld.so``.  There is no CPU fallback -- if the library cannot be loaded,
importing a function from here raises.

Array arguments may be torch tensors (on the context's GPU or on the host) or
numpy arrays (host); they are passed to the library as raw pointers, so they
must be C-contiguous with the documented dtype.  ``stream`` defaults to the
current torch CUDA stream.
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref
import os

import numpy as np

from . import _build

_lib = None


class PsgldError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"psgld status {status}: {msg}")
        self.status = status


PSGLD_OK, PSGLD_ERR_ARG, PSGLD_ERR_OOM, PSGLD_ERR_CUDA, PSGLD_ERR_STATE, PSGLD_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5
PSGLD_ERR_SIZE = -6
PSGLD_STATIC_MAX_NNZ = 4096 * 4096
PSGLD_PRIOR_EXPONENTIAL, PSGLD_PRIOR_GAUSSIAN = 0, 1
PSGLD_EPS_FIXED, PSGLD_EPS_POLY = 0, 1
PSGLD_SCALE_N_OVER_PART, PSGLD_SCALE_B = 0, 1


class psgld_prior(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lambda_w", C.c_double), ("lambda_h", C.c_double),
                ("sigma_w", C.c_double), ("sigma_h", C.c_double)]


class psgld_options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("eps_mode", C.c_int32), ("eps", C.c_double),
                ("eps_a", C.c_double), ("eps_b", C.c_double), ("scale_mode", C.c_int32),
                ("mu_min", C.c_double), ("freeze_W", C.c_int32), ("freeze_H", C.c_int32),
                ("burn_in_sweeps", C.c_int64), ("use_graphs", C.c_int32),
                ("profile", C.c_int32), ("dense_path", C.c_int32),
                ("dense_v_bf16", C.c_int32), ("part_mode", C.c_int32),
                ("dense_fp8", C.c_int32), ("gather_bf16", C.c_int32), ("max_sms", C.c_int32),
                ("batch_ctas", C.c_int32), ("batch_update_blocks", C.c_int32),
                ("debug_wait_polls", C.c_int32), ("wide_col_blocks", C.c_int32),
                ("dense_share_e", C.c_int32)]


class psgld_job(C.Structure):
    _fields_ = [("I", C.c_int64), ("J", C.c_int64), ("K", C.c_int32), ("B", C.c_int32),
                ("tweedie_p", C.c_double), ("phi", C.c_double), ("prior", psgld_prior),
                ("options", psgld_options), ("sweeps", C.c_int32), ("V_dev", C.c_void_p),
                ("ldv", C.c_int64), ("W0_dev", C.c_void_p), ("Ht0_dev", C.c_void_p),
                ("Wmean_host", C.c_void_p), ("Hmean_host", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class psgld_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


EXPORTS = [
    "psgld_default_options", "psgld_create", "psgld_set_options", "psgld_set_data_coo",
    "psgld_set_data_dense", "psgld_set_factors", "psgld_get_factors", "psgld_part_step",
    "psgld_sweep", "psgld_posterior_mean", "psgld_log_lik", "psgld_rmse", "psgld_piece_bounds",
    "psgld_part_schedule", "psgld_part_layout", "psgld_profile_read", "psgld_profile_read_split",
    "psgld_iterations_done", "psgld_estimate_device_bytes", "psgld_set_allocator",
    "psgld_batch_sweep", "psgld_get_state", "psgld_set_state",
    "psgld_log_lik_static", "psgld_last_error",
    "psgld_destroy",
    "psgld_server_create", "psgld_server_submit", "psgld_server_poll", "psgld_server_wait_idle",
    "psgld_server_stats", "psgld_server_last_error", "psgld_server_destroy",
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpsgld.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path}")
    L = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    st = C.c_int
    sig = {
        "psgld_default_options": (None, [C.POINTER(psgld_options)]),
        "psgld_create": (st, [i64, i64, i32, i32, f64, f64, C.POINTER(psgld_prior), C.POINTER(vp)]),
        "psgld_set_options": (st, [vp, C.POINTER(psgld_options)]),
        "psgld_set_data_coo": (st, [vp, i64, vp, vp, vp, vp]),
        "psgld_set_data_dense": (st, [vp, vp, i64, vp]),
        "psgld_set_factors": (st, [vp, vp, vp, vp]),
        "psgld_get_factors": (st, [vp, vp, vp, vp]),
        "psgld_part_step": (st, [vp, i64, vp]),
        "psgld_sweep": (st, [vp, i32, vp]),
        "psgld_posterior_mean": (st, [vp, vp, vp, vp, vp, vp]),
        "psgld_log_lik": (st, [vp, vp, vp]),
        "psgld_rmse": (st, [vp, i32, vp, vp]),
        "psgld_get_state": (st, [vp, vp, vp, vp, vp, vp]),
        "psgld_set_state": (st, [vp, vp, vp, vp, vp, vp]),
        "psgld_piece_bounds": (st, [vp, vp, vp]),
        "psgld_part_schedule": (st, [vp, i64, vp]),
        "psgld_part_layout": (st, [vp, i32, vp, vp, vp]),
        "psgld_profile_read": (st, [vp, vp, vp]),
        "psgld_profile_read_split": (st, [vp, vp, vp, vp]),
        "psgld_estimate_device_bytes": (i64, [i64, i64, i32, i32, i64, i32, i32]),
        "psgld_set_allocator": (st, [C.POINTER(psgld_allocator)]),
        "psgld_batch_sweep": (st, [vp, i32, i32, vp]),
        "psgld_iterations_done": (i64, [vp]),
        "psgld_log_lik_static": (st, [i64, vp, vp, vp, vp, vp, i64, i64, i32, f64, f64, f64, vp, vp]),
        "psgld_last_error": (C.c_char_p, [vp]),
        "psgld_destroy": (None, [vp]),
        "psgld_server_create": (st, [C.c_size_t, i32, C.POINTER(vp)]),
        "psgld_server_submit": (st, [vp, C.POINTER(psgld_job), C.POINTER(i64)]),
        "psgld_server_poll": (i32, [vp, vp, vp, i32]),
        "psgld_server_wait_idle": (st, [vp, f64]),
        "psgld_server_stats": (st, [vp, C.POINTER(i64), C.POINTER(f64), C.POINTER(C.c_size_t)]),
        "psgld_server_last_error": (C.c_char_p, [vp]),
        "psgld_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _ptr(x, dtype=None):
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if dtype is not None and x.dtype != dtype[0]:
                raise TypeError(f"expected {dtype[0]}, got {x.dtype}")
            return C.c_void_p(x.data_ptr())
    except ImportError:
        pass
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != dtype[1]:
            raise TypeError(f"expected {dtype[1]}, got {x.dtype}")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _dt(kind):
    import torch
    return {"i32": (torch.int32, np.int32), "f32": (torch.float32, np.float32),
            "f64": (torch.float64, np.float64)}[kind]


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(0)


def _check(ctx, status):
    if status != PSGLD_OK:
        msg = load().psgld_last_error(ctx).decode() if ctx else ""
        raise PsgldError(status, msg)


# ---------------------------------------------------------------------------
# the ABI, one function per entry point
# ---------------------------------------------------------------------------

def psgld_default_options() -> psgld_options:
    o = psgld_options()
    load().psgld_default_options(C.byref(o))
    return o


def psgld_create(I, J, K, B, tweedie_p, phi, prior: psgld_prior):
    h = C.c_void_p()
    st = load().psgld_create(int(I), int(J), int(K), int(B), float(tweedie_p), float(phi),
                             C.byref(prior), C.byref(h))
    if st != PSGLD_OK:
        raise PsgldError(st, "psgld_create rejected its arguments or ran out of memory")
    return h


def psgld_set_options(ctx, opt: psgld_options):
    _check(ctx, load().psgld_set_options(ctx, C.byref(opt)))


def psgld_set_data_coo(ctx, i, j, v, stream=None):
    _check(ctx, load().psgld_set_data_coo(ctx, len(i), _ptr(i, _dt("i32")), _ptr(j, _dt("i32")),
                                          _ptr(v, _dt("f32")), _stream(stream)))


def psgld_set_data_dense(ctx, V, ld=None, stream=None):
    ld = V.shape[1] if ld is None else ld
    _check(ctx, load().psgld_set_data_dense(ctx, _ptr(V, _dt("f32")), int(ld), _stream(stream)))


def psgld_set_factors(ctx, W, Ht, stream=None):
    _check(ctx, load().psgld_set_factors(ctx, _ptr(W, _dt("f32")), _ptr(Ht, _dt("f32")),
                                         _stream(stream)))


def psgld_get_factors(ctx, W, Ht, stream=None):
    _check(ctx, load().psgld_get_factors(ctx, _ptr(W, _dt("f32")), _ptr(Ht, _dt("f32")),
                                         _stream(stream)))


def psgld_part_step(ctx, t, stream=None):
    _check(ctx, load().psgld_part_step(ctx, int(t), _stream(stream)))


def psgld_sweep(ctx, n_sweeps=1, stream=None):
    _check(ctx, load().psgld_sweep(ctx, int(n_sweeps), _stream(stream)))


def psgld_posterior_mean(ctx, Wmean, Wvar, Hmean, Hvar):
    n = C.c_int64(0)
    f = _dt("f64")
    _check(ctx, load().psgld_posterior_mean(ctx, _ptr(Wmean, f), _ptr(Wvar, f), _ptr(Hmean, f),
                                            _ptr(Hvar, f), C.byref(n)))
    return n.value


def psgld_get_state(ctx, I, J, K):
    """(sum W, sum W^2, sum H^T, sum (H^T)^2, counters [t, sweeps, samples])
    as numpy arrays (FP64 I x K / J x K, int64 [3])."""
    out = [np.zeros((n, K)) for n in (I, I, J, J)]
    cnt = np.zeros(3, np.int64)
    f = _dt("f64")
    _check(ctx, load().psgld_get_state(ctx, *[_ptr(x, f) for x in out], C.c_void_p(cnt.ctypes.data)))
    return (*out, cnt)


def psgld_set_state(ctx, sW, sW2, sH, sH2, counters):
    f = _dt("f64")
    arrs = [np.ascontiguousarray(x, np.float64) for x in (sW, sW2, sH, sH2)]
    cnt = np.ascontiguousarray(counters, np.int64)
    _check(ctx, load().psgld_set_state(ctx, *[_ptr(x, f) for x in arrs], C.c_void_p(cnt.ctypes.data)))


def psgld_log_lik(ctx, stream=None) -> float:
    out = C.c_double(0.0)
    _check(ctx, load().psgld_log_lik(ctx, C.byref(out), _stream(stream)))
    return out.value


def psgld_rmse(ctx, use_posterior_mean=False, stream=None) -> float:
    out = C.c_double(0.0)
    _check(ctx, load().psgld_rmse(ctx, int(bool(use_posterior_mean)), C.byref(out),
                                  _stream(stream)))
    return out.value


def psgld_piece_bounds(ctx, B):
    rs = np.zeros(B + 1, dtype=np.int64)
    cs = np.zeros(B + 1, dtype=np.int64)
    _check(ctx, load().psgld_piece_bounds(ctx, _ptr(rs), _ptr(cs)))
    return rs, cs


def psgld_part_schedule(ctx, t, B):
    cp = np.zeros(B, dtype=np.int32)
    _check(ctx, load().psgld_part_schedule(ctx, int(t), _ptr(cp)))
    return cp


def psgld_part_layout(ctx, s, I):
    n = C.c_int64(0)
    _check(ctx, load().psgld_part_layout(ctx, int(s), None, None, C.byref(n)))
    ptr = np.zeros(I + 1, dtype=np.int32)
    cols = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(ctx, load().psgld_part_layout(ctx, int(s), _ptr(ptr), _ptr(cols), C.byref(n)))
    return ptr, cols[:n.value]


def psgld_profile_read(ctx):
    """(summed part-step kernel milliseconds, number of launches) since the last read."""
    ms = C.c_double(0.0)
    n = C.c_int64(0)
    _check(ctx, load().psgld_profile_read(ctx, C.byref(ms), C.byref(n)))
    return ms.value, n.value


# Every allocator handed to the library stays alive for the whole process:
# contexts keep a copy of its function pointers and call them when they free
# memory, possibly long after another allocator (or none) was set.
_allocator_keepalive = []


def psgld_set_allocator(alloc_fn=None, free_fn=None):
    """Device memory for contexts created from now on: alloc_fn(bytes, stream)
    -> device pointer (int) or 0, free_fn(ptr, stream); None restores
    cudaMalloc / cudaFree (contexts created before keep what they had)."""
    if alloc_fn is None:
        _check(None, load().psgld_set_allocator(None))
        return

    def _a(nbytes, stream, user):
        try:
            return int(alloc_fn(int(nbytes), stream)) or None
        except Exception:
            return None

    def _f(ptr, stream, user):
        free_fn(int(ptr), stream)

    a = psgld_allocator(ALLOC_FN(_a), FREE_FN(_f), None)
    _allocator_keepalive.append((a, _a, _f))
    _check(None, load().psgld_set_allocator(C.byref(a)))


def use_torch_allocator(device=None):
    """Hand the library PyTorch's caching allocator (no device-wide wait when
    a context frees its memory)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)

    def alloc_fn(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, dev)

    def free_fn(ptr, stream):
        torch.cuda.caching_allocator_delete(ptr)

    psgld_set_allocator(alloc_fn, free_fn)


def psgld_batch_sweep(chains, n_sweeps=1, stream=None):
    """n_sweeps sweeps of every chain (PSGLD objects), part-steps in shared launches."""
    arr = (C.c_void_p * len(chains))(*[ch.ctx for ch in chains])
    st = load().psgld_batch_sweep(arr, len(chains), int(n_sweeps), _stream(stream))
    if st != PSGLD_OK:
        msgs = [load().psgld_last_error(ch.ctx).decode() for ch in chains]
        raise PsgldError(st, "; ".join(m for m in msgs if m))


def psgld_estimate_device_bytes(I, J, K, B, nnz=0, dense_path=0, dense_v_bf16=0):
    """Device bytes a context of these sizes holds once its data is set."""
    return int(load().psgld_estimate_device_bytes(int(I), int(J), int(K), int(B), int(nnz),
                                                   int(dense_path), int(dense_v_bf16)))


def psgld_profile_read_split(ctx):
    """(gradient-kernel ms, update-kernel ms, number of part-steps) since the last read."""
    g = C.c_double(0.0)
    u = C.c_double(0.0)
    n = C.c_int64(0)
    _check(ctx, load().psgld_profile_read_split(ctx, C.byref(g), C.byref(u), C.byref(n)))
    return g.value, u.value, n.value


def psgld_log_lik_static(i, j, v, W, Ht, tweedie_p, phi, out, mu_min=1e-10, stream=None):
    """Log-likelihood of factors W (I x K), Ht (J x K) on entries (i, j, v),
    written to `out` (a one-element float64 CUDA tensor); allocates nothing."""
    I, K = W.shape
    J = Ht.shape[0]
    st = load().psgld_log_lik_static(
        len(i), _ptr(i, _dt("i32")), _ptr(j, _dt("i32")), _ptr(v, _dt("f32")),
        _ptr(W, _dt("f32")), _ptr(Ht, _dt("f32")), int(I), int(J), int(K), float(tweedie_p),
        float(phi), float(mu_min), _ptr(out, _dt("f64")), _stream(stream))
    if st == PSGLD_ERR_SIZE:
        raise PsgldError(st, f"nnz {len(i)} exceeds PSGLD_STATIC_MAX_NNZ {PSGLD_STATIC_MAX_NNZ}")
    if st != PSGLD_OK:
        raise PsgldError(st, "psgld_log_lik_static failed")


def psgld_iterations_done(ctx) -> int:
    return load().psgld_iterations_done(ctx)


def psgld_last_error(ctx) -> str:
    return load().psgld_last_error(ctx).decode()


def psgld_destroy(ctx):
    if ctx:
        load().psgld_destroy(ctx)


# ---------------------------------------------------------------------------
# convenience wrapper (still marshalling only)
# ---------------------------------------------------------------------------

_live_chains = weakref.WeakSet()


@atexit.register
def _close_live_chains():
    """Destroy the contexts still open at interpreter exit, while the
    allocator callbacks they may call can still run."""
    for ch in list(_live_chains):
        try:
            ch.close()
        except Exception:
            pass


class PSGLD:
    """One PSGLD chain held by a library context."""

    def __init__(self, I, J, K, B, tweedie_p, phi, prior_kind=PSGLD_PRIOR_EXPONENTIAL,
                 lambda_w=1.0, lambda_h=1.0, sigma_w=1.0, sigma_h=1.0, **options):
        self.I, self.J, self.K, self.B = int(I), int(J), int(K), int(B)
        pr = psgld_prior(int(prior_kind), float(lambda_w), float(lambda_h), float(sigma_w),
                         float(sigma_h))
        self.ctx = psgld_create(I, J, K, B, tweedie_p, phi, pr)
        _live_chains.add(self)
        self.options = psgld_default_options()
        if options:
            self.set_options(**options)

    def set_options(self, **kw):
        for k, v in kw.items():
            if not hasattr(self.options, k):
                raise AttributeError(k)
            setattr(self.options, k, v)
        psgld_set_options(self.ctx, self.options)

    def close(self):
        if getattr(self, "ctx", None):
            psgld_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_data_coo(self, i, j, v, stream=None):
        psgld_set_data_coo(self.ctx, i, j, v, stream)

    def set_data_dense(self, V, stream=None):
        psgld_set_data_dense(self.ctx, V, None, stream)

    def set_factors(self, W, Ht, stream=None):
        psgld_set_factors(self.ctx, W, Ht, stream)

    def get_factors(self, stream=None):
        import torch
        W = torch.empty((self.I, self.K), dtype=torch.float32, device="cuda")
        Ht = torch.empty((self.J, self.K), dtype=torch.float32, device="cuda")
        psgld_get_factors(self.ctx, W, Ht, stream)
        return W, Ht

    def part_step(self, t, stream=None):
        psgld_part_step(self.ctx, t, stream)

    def sweep(self, n=1, stream=None):
        psgld_sweep(self.ctx, n, stream)

    def posterior_mean(self):
        Wm = np.zeros((self.I, self.K)); Wv = np.zeros((self.I, self.K))
        Hm = np.zeros((self.J, self.K)); Hv = np.zeros((self.J, self.K))
        n = psgld_posterior_mean(self.ctx, Wm, Wv, Hm, Hv)
        return Wm, Wv, Hm, Hv, n

    def get_state(self):
        """The chain's state beside its factors: FP64 posterior sums and the
        counters (t, sweeps, samples); with get_factors, a checkpoint."""
        return psgld_get_state(self.ctx, self.I, self.J, self.K)

    def set_state(self, state):
        psgld_set_state(self.ctx, *state)

    def log_lik(self, stream=None):
        return psgld_log_lik(self.ctx, stream)

    def rmse(self, use_posterior_mean=False, stream=None):
        return psgld_rmse(self.ctx, use_posterior_mean, stream)

    def profile_read(self):
        return psgld_profile_read(self.ctx)

    def profile_read_split(self):
        return psgld_profile_read_split(self.ctx)

    @property
    def iterations_done(self):
        return psgld_iterations_done(self.ctx)


class NativeServer:
    """The library's serving loop (psgld_server_*): submit dense jobs with
    device inputs; a worker thread in the library admits them by memory,
    batches their sweeps and writes their posterior means to host arrays."""

    def __init__(self, hbm_budget: int, max_inflight: int = 1):
        h = C.c_void_p()
        st = load().psgld_server_create(int(hbm_budget), int(max_inflight), C.byref(h))
        if st != PSGLD_OK:
            raise PsgldError(st, "psgld_server_create")
        self.h = h
        self._keep = {}          # job id -> the arrays the library reads or writes
        self._done = {}          # job id -> (W mean, H^T mean, latency s)

    def submit(self, I, J, K, B, tweedie_p, phi, V, W0, Ht0, sweeps, prior_kind=PSGLD_PRIOR_EXPONENTIAL,
               lambda_w=1.0, lambda_h=1.0, sigma_w=1.0, sigma_h=1.0, **options):
        """V (I x J), W0 (I x K), Ht0 (J x K): contiguous FP32 CUDA tensors,
        ready (their stream synchronised).  Returns the job id; results()
        gives the posterior means once the job is reported done."""
        opts = psgld_default_options()
        for k, v in options.items():
            setattr(opts, k, v)
        Wm = np.zeros((I, K))
        Hm = np.zeros((J, K))
        job = psgld_job(I=I, J=J, K=K, B=B, tweedie_p=float(tweedie_p), phi=float(phi),
                        prior=psgld_prior(int(prior_kind), float(lambda_w), float(lambda_h),
                                          float(sigma_w), float(sigma_h)),
                        options=opts, sweeps=int(sweeps), V_dev=V.data_ptr(), ldv=V.stride(0),
                        W0_dev=W0.data_ptr(), Ht0_dev=Ht0.data_ptr(),
                        Wmean_host=Wm.ctypes.data, Hmean_host=Hm.ctypes.data)
        jid = C.c_int64()
        st = load().psgld_server_submit(self.h, C.byref(job), C.byref(jid))
        if st != PSGLD_OK:
            raise PsgldError(st, "psgld_server_submit")
        self._keep[jid.value] = (V, W0, Ht0, Wm, Hm)
        return jid.value

    def poll(self, max_n: int = 1024):
        """[(job id, latency s)] of jobs finished since the last poll; their
        inputs are released and their results kept for results()."""
        ids = np.zeros(max_n, np.int64)
        lat = np.zeros(max_n, np.float64)
        n = load().psgld_server_poll(self.h, ids.ctypes.data, lat.ctypes.data, max_n)
        out = []
        for k in range(n):
            jid = int(ids[k])
            V, W0, Ht0, Wm, Hm = self._keep.pop(jid)
            self._done[jid] = (Wm, Hm, float(lat[k]))
            out.append((jid, float(lat[k])))
        return out

    def results(self, jid):
        """(W posterior mean, H^T posterior mean, latency s) of a finished job."""
        return self._done.pop(jid)

    def wait_idle(self, timeout_s: float = 600.0):
        st = load().psgld_server_wait_idle(self.h, float(timeout_s))
        if st != PSGLD_OK:
            raise PsgldError(st, "psgld_server_wait_idle")

    def stats(self):
        n, jps, peak = C.c_int64(), C.c_double(), C.c_size_t()
        load().psgld_server_stats(self.h, C.byref(n), C.byref(jps), C.byref(peak))
        return {"sweeps": n.value, "jobs_per_sweep": jps.value, "peak_bytes": peak.value}

    def last_error(self) -> str:
        return load().psgld_server_last_error(self.h).decode()

    def close(self):
        if getattr(self, "h", None):
            load().psgld_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
