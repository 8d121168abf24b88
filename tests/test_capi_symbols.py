"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/euler_hyp.h declares. CPU only: no compute call is made."""
import ctypes
import os
import re

import pytest

from paper_2106_02159_gb300 import binding

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "euler_hyp.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(eh_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    binding.build()
    return binding.load()


def test_header_and_binding_agree():
    assert declared_functions() == sorted(binding.EXPORTS)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_host_only_calls(lib):
    cfg = binding.Config()
    lib.eh_config_default(ctypes.byref(cfg))
    assert (cfg.dim, cfg.gamma, cfg.cfl, cfg.limiter_passes, cfg.bound_relaxation) == (2, 1.4, 0.5, 2, 0)
    assert lib.eh_status_string(binding.EH_ERR_CFL) == b"EH_ERR_CFL"
    assert lib.eh_status_string(99) == b"EH_UNKNOWN"
    assert lib.eh_last_error(None) == b"null context"
    out = ctypes.c_void_p(1)
    assert lib.eh_create(None, ctypes.byref(out)) == binding.EH_ERR_INVALID_ARG and not out.value
    bad = binding.Config()
    lib.eh_config_default(ctypes.byref(bad))
    assert lib.eh_batch_last_error(None) == b"null batch"
    lib.eh_batch_destroy(None)
    assert lib.eh_batch_create(None, 1 << 30, ctypes.byref(out)) == binding.EH_ERR_INVALID_ARG and not out.value
    ticket, done = ctypes.c_int64(0), ctypes.c_int32(0)
    assert lib.eh_batch_admit(None, 10, 10, None, None, None, None, None, 0, None, None, None, None, None, 1.0,
                              ctypes.byref(ticket)) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_batch_advance(None, 1, None) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_batch_poll(None, 1, ctypes.byref(done), None, None, None) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_batch_active(None, None, None) == binding.EH_ERR_INVALID_ARG
    nbytes = ctypes.c_uint64(0)
    assert lib.eh_estimate_device_bytes(2, 0, 1000, 9000, ctypes.byref(nbytes)) == binding.EH_OK
    small = nbytes.value
    assert lib.eh_estimate_device_bytes(2, 0, 2000, 18000, ctypes.byref(nbytes)) == binding.EH_OK
    assert (1 << 20) < small < nbytes.value
    for args in ((4, 0, 10, 10), (2, 5, 10, 10), (2, 0, 0, 10), (2, 0, 10, 5)):
        assert lib.eh_estimate_device_bytes(*args, ctypes.byref(nbytes)) == binding.EH_ERR_INVALID_ARG, args
    for field, value in (("dim", 4), ("gamma", 2.0), ("cfl", 1.5), ("limiter_passes", 0)):
        b2 = binding.Config.from_buffer_copy(bad)
        setattr(b2, field, value)
        assert lib.eh_create(ctypes.byref(b2), ctypes.byref(out)) == binding.EH_ERR_INVALID_ARG, field


def test_request_bytes_by_batch_mode(lib):
    """Merged mode counts a request's resident copy of its mesh on top of the
    per-context estimate; bad sizes or modes are refused (host only)."""
    est, merged, streams = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    assert lib.eh_estimate_device_bytes(2, 0, 5000, 45000, ctypes.byref(est)) == binding.EH_OK
    assert lib.eh_estimate_request_bytes(2, 0, binding.EH_BATCH_PER_REQUEST_STREAMS, 5000, 45000, 300,
                                         ctypes.byref(streams)) == binding.EH_OK
    assert lib.eh_estimate_request_bytes(2, 0, binding.EH_BATCH_MERGED, 5000, 45000, 300,
                                         ctypes.byref(merged)) == binding.EH_OK
    assert streams.value == est.value
    assert est.value < merged.value < 2 * est.value
    for args in ((2, 0, 7, 5000, 45000, 300), (2, 0, 0, 5000, 45000, -1), (3, 9, 0, 10, 10, 0)):
        assert lib.eh_estimate_request_bytes(*args, ctypes.byref(merged)) == binding.EH_ERR_INVALID_ARG, args
    assert lib.eh_batch_set_mode(None, 0) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_batch_repacks(None, None) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_get_instance_steps(None, None) == binding.EH_ERR_INVALID_ARG
    assert lib.eh_get_mesh_index(None, None, None, None) == binding.EH_ERR_INVALID_ARG
