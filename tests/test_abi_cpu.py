"""Host-side checks of libhom that need no GPU: it builds, loads, exports every
function include/hom.h declares, sizes buffers, and rejects bad arguments
before touching the device."""

import ctypes

import pytest

from paper_1903_02581_gb300 import binding as H
from paper_1903_02581_gb300 import build as Bd
from paper_1903_02581_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    Bd.build()
    return H.lib()


def test_exports_every_declared_function(lib):
    names = H.declared_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_state_and_workspace_sizes(lib):
    p = H.make_params(W.tiny())
    n = 16 * 16
    assert H.hom_state_bytes(p) == n * n * 16
    p64 = H.make_params(W.fullscale())
    assert H.hom_state_bytes(p64) == (256 * 64) ** 2 * 8
    ws = H.hom_workspace_bytes(p64)
    state = (256 * 64) ** 2 * 8
    assert state < ws < state + 64 * 2 ** 20      # one transposed state plus tables and partials
    p64.ckpt_slots = 2
    assert H.hom_workspace_bytes(p64) >= ws + 2 * (256 * 64) ** 2 * 8


@pytest.mark.parametrize("field,value", [("nx", 24), ("nx", 8), ("ny", 128), ("batch", 0),
                                         ("dx", 0.0), ("dt", 0.0), ("coul_soft", 0.0),
                                         ("qpc_w", -1.0), ("prec", 7), ("ckpt_slots", -1)])
def test_invalid_params_rejected(lib, field, value):
    p = H.make_params(W.tiny())
    setattr(p, field, value)
    assert H.hom_state_bytes(p) == 0
    assert H.hom_workspace_bytes(p) == 0
    ctx = ctypes.c_void_p()
    st = lib.hom_create(ctypes.byref(p), 256, 256, 1 << 30, None, ctypes.byref(ctx))
    assert st == H.HOM_ERR_ARG and not ctx.value
    assert lib.hom_last_error(None)


def test_complex128_plane_limit(lib):
    p = H.make_params(W.fullscale())
    p.prec = H.HOM_C128
    assert H.hom_state_bytes(p) == 0


def test_create_rejects_null_and_small_workspace(lib):
    p = H.make_params(W.tiny())
    ctx = ctypes.c_void_p()
    assert lib.hom_create(ctypes.byref(p), None, 256, 1 << 30, None, ctypes.byref(ctx)) == H.HOM_ERR_ARG
    assert lib.hom_create(ctypes.byref(p), 256, 256, 16, None, ctypes.byref(ctx)) == H.HOM_ERR_NOMEM
    assert b"workspace" in lib.hom_last_error(None)
    assert lib.hom_create(ctypes.byref(p), 255, 256, 1 << 30, None, ctypes.byref(ctx)) == H.HOM_ERR_ARG


def test_null_context_calls(lib):
    assert lib.hom_step(None, 1) == H.HOM_ERR_ARG
    assert lib.hom_observables(None, None) == H.HOM_ERR_ARG
    lib.hom_destroy(None)
