"""Host-side checks of libhom that need no GPU: it builds, loads, exports every
function include/hom.h declares, sizes buffers, rejects bad arguments before
touching the device, and computes slice entropies on the host (the one
entry point with no device work)."""

import ctypes

import numpy as np
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
                                         ("qpc_w", -1.0), ("prec", 7), ("ckpt_slots", -1),
                                         ("coul_screen", -0.5), ("coul_screen", float("inf")),
                                         ("split", 2), ("reserved", 1), ("fermi_xa", float("nan")),
                                         ("fermi_vb", float("inf"))])
def test_invalid_params_rejected(lib, field, value):
    p = H.make_params(W.tiny())
    setattr(p, field, value)
    if field == "fermi_vb":
        p.fermi_tau = 0.5
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


# --- host-side entropy of a slice (no GPU) -----------------------------------

def test_vn_entropy_closed_forms_and_oracle(lib):
    import math

    from oracle import hom_oracle as O

    rng = np.random.default_rng(3)
    for probs in [(1.0,), (0.5, 0.5), (0.6, 0.3, 0.1)]:
        u, _ = np.linalg.qr(rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7)))
        v, _ = np.linalg.qr(rng.standard_normal((11, 11)) + 1j * rng.standard_normal((11, 11)))
        phi = 0.8 * sum(math.sqrt(p) * np.outer(u[:, k], v[:, k]) for k, p in enumerate(probs))
        for a in (phi, phi.T.copy()):
            s, w = H.hom_vn_entropy(a)
            assert abs(s + sum(p * math.log(p) for p in probs)) <= 1e-12
            assert abs(w - 0.64) <= 1e-13
    # a generic slice: the same entropy as the oracle (numpy eigvalsh of rho_T)
    psi = W.random_state((12, 3, 12, 3), seed=9)
    s_ref, w_ref = O.entanglement_entropy(psi, 1, 2, (2, 10), (0, 12))
    s, w = H.hom_vn_entropy(psi[2:10, 1, 0:12, 2])
    assert abs(s - s_ref) <= 1e-12 and abs(w - w_ref) <= 1e-12 * w_ref


def test_vn_entropy_errors(lib):
    with pytest.raises(H.HomError) as e:
        H.hom_vn_entropy(np.zeros((4, 5), dtype=np.complex128))
    assert e.value.status == H.HOM_ERR_NUMERIC
    s = ctypes.c_double()
    assert lib.hom_vn_entropy(None, 2, 2, ctypes.byref(s), None) == H.HOM_ERR_ARG


def test_fermi_tau_needed_only_with_blocks(lib):
    p = H.make_params(W.tiny())
    p.fermi_tau = 0.0
    assert H.hom_state_bytes(p) > 0                 # no blocks: tau unused
    p.fermi_vb = 2.0
    assert H.hom_state_bytes(p) == 0
