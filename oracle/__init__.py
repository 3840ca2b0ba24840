"""FP64 CPU oracle of PSGLD (Simsekli et al. 2015) -- ctypes wrapper.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
(``paper_1506_01418_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``psgld_oracle.c`` (plain C99, FP64); this module only
compiles it on demand and marshals numpy arrays.  Layouts follow the paper:
W is I x K and H is K x J, both row-major.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# The mutation tests (tests/test_oracle_mutants.py) point the loader at a
# copy of the source with one planted mistake, built into a library of its
# own, through these two variables; unset, the loader uses this directory.
_SRC = os.environ.get("PSGLD_ORACLE_SOURCE") or os.path.join(_HERE, "psgld_oracle.c")
_HDR = os.path.join(os.path.dirname(_SRC), "psgld_oracle.h")
_LIB = os.environ.get("PSGLD_ORACLE_LIB") or os.path.join(_HERE, "liboracle_psgld.so")

PRIOR_EXPONENTIAL, PRIOR_GAUSSIAN = 0, 1
EPS_FIXED, EPS_POLY = 0, 1
SCALE_N_OVER_PART, SCALE_B = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
            "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        i64, i32, u64, f64 = C.c_int64, C.c_int32, C.c_uint64, C.c_double
        vp = C.c_void_p
        sig = {
            "or_create": (vp, [i64, i64, i32, i32, f64, f64, i32, f64, f64, f64, f64]),
            "or_destroy": (None, [vp]),
            "or_set_options": (None, [vp, u64, i32, f64, f64, f64, i32, f64, i32, i32, i64]),
            "or_set_data": (C.c_int, [vp, i64, vp, vp, vp]),
            "or_set_factors": (None, [vp, vp, vp]),
            "or_get_factors": (None, [vp, vp, vp]),
            "or_piece_start": (i64, [i64, i64, i32]),
            "or_piece_of": (i32, [i64, i64, i32]),
            "or_part_col_piece": (i32, [i64, i32, i32]),
            "or_block_entries": (i64, [vp, i32, i32, i64, vp, vp]),
            "or_part_size": (i64, [vp, i64]),
            "or_philox4x32_10": (None, [vp, vp, vp]),
            "or_noise": (f64, [u64, i64, i32, i64, i32]),
            "or_noise_matrix": (None, [u64, i64, i32, i64, i32, vp]),
            "or_eps": (f64, [vp, i64]),
            "or_scale": (f64, [vp, i64]),
            "or_drift": (None, [vp, i64, vp, vp]),
            "or_part_step": (None, [vp, i64]),
            "or_sweep": (C.c_int, [vp, i32]),
            "or_iterations_done": (i64, [vp]),
            "or_posterior": (None, [vp, vp, vp, vp, vp, vp]),
            "or_beta_div": (f64, [f64, f64, f64]),
            "or_log_lik": (f64, [vp]),
            "or_log_lik_part": (f64, [vp, i64]),
            "or_log_post": (f64, [vp]),
            "or_rmse": (f64, [vp, i32]),
            "or_set_threads": (i32, [i32]),
            "or_set_part_mode": (None, [vp, i32]),
            "or_part_index": (i32, [vp, i64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads the oracle uses for the blocks of a part (n <= 0: query)."""
    return int(lib().or_set_threads(int(n)))


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# free functions
# --------------------------------------------------------------------------

def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def noise(seed: int, t: int, mat: int, row: int, k: int) -> float:
    return lib().or_noise(seed, t, mat, row, k)


def noise_matrix(seed: int, t: int, mat: int, nrows: int, K: int) -> np.ndarray:
    out = np.zeros((nrows, K), dtype=np.float64)
    lib().or_noise_matrix(seed, t, mat, nrows, K, _p(out))
    return out


def piece_start(r: int, n: int, B: int) -> int:
    return lib().or_piece_start(r, n, B)


def piece_of(x: int, n: int, B: int) -> int:
    return lib().or_piece_of(x, n, B)


def part_col_piece(t: int, B: int, r: int) -> int:
    return lib().or_part_col_piece(t, B, r)


def beta_div(v: float, mu: float, p: float) -> float:
    return lib().or_beta_div(v, mu, p)


# --------------------------------------------------------------------------
# model
# --------------------------------------------------------------------------

class Oracle:
    """One PSGLD chain in FP64 (Algorithm 1)."""

    def __init__(self, I, J, K, B, p, phi, prior_kind=PRIOR_EXPONENTIAL,
                 lambda_w=1.0, lambda_h=1.0, sigma_w=1.0, sigma_h=1.0):
        self.I, self.J, self.K, self.B = int(I), int(J), int(K), int(B)
        self.p, self.phi = float(p), float(phi)
        self._h = lib().or_create(self.I, self.J, self.K, self.B, self.p, self.phi,
                                  int(prior_kind), float(lambda_w), float(lambda_h),
                                  float(sigma_w), float(sigma_h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def set_options(self, seed=0, eps_mode=EPS_FIXED, eps=1e-4, eps_a=0.01,
                    eps_b=0.51, scale_mode=SCALE_N_OVER_PART, mu_min=1e-10,
                    freeze_W=False, freeze_H=False, burn_in=0):
        lib().or_set_options(self._h, int(seed), int(eps_mode), float(eps),
                             float(eps_a), float(eps_b), int(scale_mode),
                             float(mu_min), int(bool(freeze_W)),
                             int(bool(freeze_H)), int(burn_in))

    def set_part_mode(self, mode):
        """0: cyclic part order (Sec. 4.1); 1: size-proportional draw (C2)."""
        lib().or_set_part_mode(self._h, int(mode))

    def part_index(self, t):
        return int(lib().or_part_index(self._h, int(t)))

    def set_data(self, i, j, v):
        i = np.ascontiguousarray(i, dtype=np.int32)
        j = np.ascontiguousarray(j, dtype=np.int32)
        v = np.ascontiguousarray(v, dtype=np.float64)
        rc = lib().or_set_data(self._h, len(i), _p(i), _p(j), _p(v))
        if rc != 0:
            raise ValueError("oracle: duplicate or out-of-range entry")

    def set_factors(self, W, H):
        W = np.ascontiguousarray(W, dtype=np.float64).reshape(self.I, self.K)
        H = np.ascontiguousarray(H, dtype=np.float64).reshape(self.K, self.J)
        lib().or_set_factors(self._h, _p(W), _p(H))

    def get_factors(self):
        W = np.zeros((self.I, self.K))
        H = np.zeros((self.K, self.J))
        lib().or_get_factors(self._h, _p(W), _p(H))
        return W, H

    def block_entries(self, r, c):
        n = lib().or_block_entries(self._h, r, c, 0, None, None)
        i = np.zeros(max(n, 1), dtype=np.int32)
        j = np.zeros(max(n, 1), dtype=np.int32)
        lib().or_block_entries(self._h, r, c, n, _p(i), _p(j))
        return i[:n], j[:n]

    def part_size(self, t):
        return lib().or_part_size(self._h, t)

    def eps(self, t):
        return lib().or_eps(self._h, t)

    def scale(self, t):
        return lib().or_scale(self._h, t)

    def drift(self, t):
        dW = np.zeros((self.I, self.K))
        dH = np.zeros((self.K, self.J))
        lib().or_drift(self._h, t, _p(dW), _p(dH))
        return dW, dH

    def part_step(self, t):
        lib().or_part_step(self._h, int(t))

    def sweep(self, n=1):
        if lib().or_sweep(self._h, int(n)) != 0:
            raise RuntimeError("oracle: sweep must start at a sweep boundary")

    @property
    def iterations_done(self):
        return lib().or_iterations_done(self._h)

    def posterior(self):
        Wm = np.zeros((self.I, self.K)); Wv = np.zeros((self.I, self.K))
        Hm = np.zeros((self.K, self.J)); Hv = np.zeros((self.K, self.J))
        n = C.c_int64(0)
        lib().or_posterior(self._h, _p(Wm), _p(Wv), _p(Hm), _p(Hv), C.byref(n))
        return Wm, Wv, Hm, Hv, n.value

    def log_lik(self):
        return lib().or_log_lik(self._h)

    def log_lik_part(self, t):
        return lib().or_log_lik_part(self._h, t)

    def log_post(self):
        return lib().or_log_post(self._h)

    def rmse(self, use_mean=False):
        return lib().or_rmse(self._h, int(bool(use_mean)))
