"""The C ABI without a GPU: the library builds, loads, exports every symbol the
header declares, and its host-side checks answer without touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "varlingam_gb300.h")
LIB = os.path.join(ROOT, "paper_2409_05500_gb300", "libvarlingam_gb300.so")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__

        __graft_entry__._load_build_module().build()
    return ctypes.CDLL(LIB)


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(
        r"^\s*(?:vl_status|const char\*|unsigned long long)\s+(vl_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("vl_var_fit", "vl_pairwise_measure", "vl_causal_order", "vl_fit_b",
              "vl_fit_batched", "vl_create", "vl_destroy", "vl_sync", "vl_last_error"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_null_handle_is_rejected_on_the_host(lib):
    P = ctypes.c_void_p
    lib.vl_var_fit.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_int, P, P]
    assert lib.vl_var_fit(None, None, 10, 3, 10, 1, 1, None, None) == 1
    lib.vl_sync.argtypes = [P]
    assert lib.vl_sync(None) == 1
    lib.vl_causal_order_standard.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, P, P]
    assert lib.vl_causal_order_standard(None, None, 10, 3, 10, 1, None, None) == 1
    lib.vl_last_error.restype = ctypes.c_char_p
    lib.vl_last_error.argtypes = [P]
    assert lib.vl_last_error(None) == b"null handle"
    lib.vl_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_size_t]
    assert lib.vl_create(None, 0, None, 0) == 1


def test_create_fails_cleanly_without_device(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    P = ctypes.c_void_p
    h = P()
    lib.vl_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P, ctypes.c_size_t]
    assert lib.vl_create(ctypes.byref(h), 0, None, 0) == 6  # VL_ERR_CUDA
    assert not h.value


def test_every_handle_call_rejects_a_null_handle_on_the_host(lib):
    """Each declared entry point that takes a handle answers VL_ERR_ARG (1) for
    a NULL handle before touching a device; the handle-free ordering entry
    point answers its argument, shape and size errors the same way."""
    P, I, I64, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    calls = {
        "vl_destroy": ([P], [None]),
        "vl_set_stream": ([P, P], [None, None]),
        "vl_reserve": ([P, I, I, I], [None, 10, 100, 1]),
        "vl_sync": ([P], [None]),
        "vl_profile_events": ([P, P, P], [None, None, None]),
        "vl_var_fit": ([P, P, I64, I, I, I, I, P, P], [None, None, 100, 10, 100, 1, 1, None, None]),
        "vl_var_select": ([P, P, I64, I, I, I, I, I, P, P],
                          [None, None, 100, 10, 100, 2, 1, 1, None, None]),
        "vl_pairwise_measure": ([P, P, I64, I, I, I, P, P, P],
                                [None, None, 100, 10, 100, 1, None, None, None]),
        "vl_causal_order": ([P, P, I, P, P], [None, None, 10, None, None]),
        "vl_causal_order_certified": ([P, P, P, I64, I, I, P, P, P],
                                      [None, None, None, 100, 10, 100, None, None, None]),
        "vl_causal_order_standard": ([P, P, I64, I, I, I, P, P],
                                     [None, None, 100, 10, 100, 1, None, None]),
        "vl_fit_b": ([P, P, I64, I, I, P, P, I, I, P, P],
                     [None, None, 100, 10, 100, None, None, 1, 1, None, None]),
        "vl_fit": ([P, P, I64, I, I, I, I, P, P, P, P, P],
                   [None, None, 100, 10, 100, 1, 1, None, None, None, None, None]),
        "vl_fit_batched": ([P, P, I, I, P], [None, None, 1, 1, None]),
        "vl_fit_batched_async": ([P, P, I, I, P], [None, None, 1, 1, None]),
        "vl_bootstrap_resample": ([P, P, I64, I, I, I, ctypes.c_uint64, I64, I, P],
                                  [None, None, 100, 10, 100, 10, 1, 0, 1, None]),
        "vl_bootstrap": ([P, P, I64, I, I, I, I, I, ctypes.c_uint64, ctypes.c_double, I, P, P],
                         [None, None, 100, 10, 100, 1, 4, 10, 1, 0.1, 1, None, None]),
    }
    handle_calls = [n for n in declared_functions()
                    if n not in ("vl_create", "vl_kernel_launches", "vl_last_error",
                                 "vl_causal_order_noalloc", "vl_sfu_rate")]
    assert sorted(handle_calls) == sorted(calls)
    lib.vl_kernel_launches.restype = ctypes.c_ulonglong
    lib.vl_kernel_launches.argtypes = []
    launches0 = lib.vl_kernel_launches()
    for name, (argtypes, args) in calls.items():
        f = getattr(lib, name)
        f.argtypes = argtypes
        f.restype = I
        assert f(*args) == 1, name
    f = lib.vl_causal_order_noalloc
    f.argtypes = [P, P, I, P, P]
    f.restype = I
    buf = (ctypes.c_double * 4)()
    order = (ctypes.c_int32 * 4)()
    assert f(None, None, 4, None, None) == 1              # VL_ERR_ARG
    assert f(None, ctypes.addressof(buf), 0, ctypes.addressof(order), None) == 2   # VL_ERR_SHAPE
    assert f(None, ctypes.addressof(buf), 513, ctypes.addressof(order), None) == 9  # UNSUPPORTED
    f = lib.vl_sfu_rate
    f.argtypes = [I, P, P]
    f.restype = I
    assert f(0, None, None) == 1                          # VL_ERR_ARG
    assert lib.vl_kernel_launches() == launches0          # none of these launched anything
