"""The C-ABI library loads and exports every entry point include/*.h declares.

CPU only: no compute call runs.  psgld_create validates its arguments before
touching the GPU, so argument rejection is host logic and is checked here too.
"""
import ctypes as C
import glob
import os
import re

import pytest

from paper_1506_01418_gb300 import psgld as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"PSGLD_API\s+[\w\s\*]*?\b(psgld_\w+)\s*\(", text))
    return names


def test_header_declares_the_abi():
    names = declared_symbols()
    for required in ("psgld_create", "psgld_part_step", "psgld_sweep",
                     "psgld_posterior_mean", "psgld_log_lik", "psgld_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = P.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(P.EXPORTS) == declared_symbols()


def test_default_options():
    o = P.psgld_default_options()
    assert o.eps == 1e-4 and o.eps_a == 0.01 and o.eps_b == 0.51
    assert o.scale_mode == P.PSGLD_SCALE_N_OVER_PART and o.mu_min == 1e-10
    assert o.use_graphs == 1 and o.burn_in_sweeps == 0


@pytest.mark.parametrize("I,J,K,B,p,phi,kind", [
    (0, 10, 4, 1, 1.0, 1.0, 0),       # empty I
    (10, 10, 0, 2, 1.0, 1.0, 0),      # K = 0
    (10, 10, 513, 2, 1.0, 1.0, 0),    # K too large
    (10, 5, 4, 6, 1.0, 1.0, 0),       # B > min(I, J)
    (10, 10, 4, 0, 1.0, 1.0, 0),      # B = 0
    (10, 10, 4, 2, 0.5, 1.0, 0),      # no Tweedie model for 0 < p < 1
    (10, 10, 4, 2, 1.0, 0.0, 0),      # phi = 0
    (10, 10, 4, 2, 1.0, 1.0, 7),      # unknown prior
    (1 << 31, 10, 4, 2, 1.0, 1.0, 0),  # I too large
])
def test_create_rejects_bad_arguments(I, J, K, B, p, phi, kind):
    pr = P.psgld_prior(kind, 1.0, 1.0, 1.0, 1.0)
    with pytest.raises(P.PsgldError) as e:
        P.psgld_create(I, J, K, B, p, phi, pr)
    assert e.value.status == P.PSGLD_ERR_ARG


def test_create_rejects_bad_prior_parameters():
    with pytest.raises(P.PsgldError):
        P.psgld_create(10, 10, 4, 2, 1.0, 1.0, P.psgld_prior(0, 0.0, 1.0, 1.0, 1.0))
    with pytest.raises(P.PsgldError):
        P.psgld_create(10, 10, 4, 2, 0.0, 1.0, P.psgld_prior(1, 1.0, 1.0, -1.0, 1.0))


def test_null_context_is_rejected():
    lib = P.load()
    assert lib.psgld_part_step(None, 1, None) == P.PSGLD_ERR_ARG
    assert lib.psgld_sweep(None, 1, None) == P.PSGLD_ERR_ARG
    assert lib.psgld_iterations_done(None) == -1
    assert lib.psgld_get_state(None, None, None, None, None, None) == P.PSGLD_ERR_ARG
    assert lib.psgld_set_state(None, None, None, None, None, None) == P.PSGLD_ERR_ARG
    lib.psgld_destroy(None)


def test_server_rejects_bad_arguments_before_touching_the_gpu():
    lib = P.load()
    h = C.c_void_p()
    assert lib.psgld_server_create(0, 1, C.byref(h)) == P.PSGLD_ERR_ARG
    assert lib.psgld_server_create(1 << 20, 0, C.byref(h)) == P.PSGLD_ERR_ARG
    assert lib.psgld_server_create(1 << 20, 1, None) == P.PSGLD_ERR_ARG
    job = P.psgld_job()
    jid = C.c_int64()
    assert lib.psgld_server_submit(None, C.byref(job), C.byref(jid)) == P.PSGLD_ERR_ARG
    assert lib.psgld_server_poll(None, None, None, 4) == 0
    assert lib.psgld_server_wait_idle(None, 0.0) == P.PSGLD_ERR_ARG
    assert lib.psgld_server_last_error(None) == b""
    lib.psgld_server_destroy(None)


def test_batch_sweep_rejects_bad_arguments():
    lib = P.load()
    assert lib.psgld_batch_sweep(None, 1, 1, None) == P.PSGLD_ERR_ARG
    arr = (C.c_void_p * 1)(None)
    assert lib.psgld_batch_sweep(arr, 1, 1, None) == P.PSGLD_ERR_ARG
    assert lib.psgld_batch_sweep(arr, 0, 1, None) == P.PSGLD_ERR_ARG
