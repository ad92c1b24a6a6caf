"""GPU probability maps and entanglement (hom_marginal, hom_conditional,
hom_entanglement) against the FP64 oracle (captions of Fig. 2 and Fig. 3(b),
Sec. V).

Both sides read the same state values (the GPU state copied to the host), so
the only differences are summation order and the eigen-solver:
- maps: 1e-12 relative;
- entropies: 1e-10 absolute.
At full scale the marginal is checked on sampled rows and against the norm,
and the entropy of a 256 x 256 slice against the oracle on the same slice.
"""

import math

import numpy as np
import pytest

from oracle import adapter as A
from oracle import hom_oracle as O
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import build

    build.build()


def H():
    from paper_1903_02581_gb300 import binding

    return binding


def scattered(prec):
    """The tiny workload after 60 steps (packets at the saddle), two simulations."""
    w = W.tiny()
    w["prec"] = prec
    s2 = dict(w["sims"][0], lam=0.0, exch=1)
    w["sims"] = [w["sims"][0], s2]
    w["batch"] = 2
    pr = H().Propagator(w)
    pr.step(60)
    return w, pr


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_maps_match_oracle(prec):
    w, pr = scattered(prec)
    mg = pr.marginal()
    for b in range(2):
        psi = pr.get_state(b).astype(np.complex128)
        m = A.model_for(w, w["sims"][b])
        ref = O.marginal(psi, m)
        assert np.max(np.abs(mg[b] - ref)) <= 1e-12 * np.max(ref)
        # hom_observables squares complex64 values in FP32 (two roundings per
        # point, 1.2e-7 relative at most), hom_marginal in FP64
        tol = 1e-12 if prec == "c128" else 2e-7
        assert abs(np.sum(mg[b]) * m.dx * m.dy - pr.observables()[b]["norm"]) <= tol
        for ix2, iy2 in [(3, 4), (12, 9), (0, 15)]:
            c = pr.conditional(b, ix2, iy2)
            cref = O.conditional(psi, ix2, iy2)
            assert np.max(np.abs(c - cref)) <= 1e-12 * max(np.max(cref), 1e-300)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_entanglement_matches_oracle(prec):
    w, pr = scattered(prec)
    nx = w["nx"]
    for b in range(2):
        psi = pr.get_state(b).astype(np.complex128)
        for iy1, iy2, r1, r2 in [(4, 11, (0, nx // 2), (nx // 2, nx)), (8, 8, (0, nx), (0, nx)), (2, 13, (3, 9), (5, 16))]:
            s, wt = pr.entanglement(b, iy1, iy2, r1, r2)
            s_ref, wt_ref = O.entanglement_entropy(psi, iy1, iy2, r1, r2)
            assert abs(s - s_ref) <= 1e-10, (b, iy1, iy2, s, s_ref)
            assert abs(wt - wt_ref) <= 1e-12 * wt_ref
            assert s >= -1e-12


def test_entanglement_product_state_and_errors():
    w = W.tiny()
    w["sims"][0]["exch"] = 0                       # product state: every slice is separable
    pr = H().Propagator(w)
    s, _ = pr.entanglement(0, 5, 10, (0, 16), (0, 16))
    assert abs(s) <= 1e-10
    with pytest.raises(H().HomError) as e:
        pr.entanglement(0, 5, 10, (4, 4), (0, 16))
    assert e.value.status == H().HOM_ERR_ARG
    with pytest.raises(H().HomError) as e:
        pr.conditional(0, 16, 0)
    assert e.value.status == H().HOM_ERR_ARG
    pr.set_state(0, np.zeros((16, 16, 16, 16), dtype=np.complex128))
    with pytest.raises(H().HomError) as e:
        pr.entanglement(0, 5, 10, (0, 16), (0, 16))
    assert e.value.status == H().HOM_ERR_NUMERIC


def test_fullscale_marginal_and_entanglement():
    w = W.fullscale()
    pr = H().Propagator(w)
    pr.step(2)
    nx, ny = w["nx"], w["ny"]
    n = nx * ny
    mg = pr.marginal()[0]
    dxdy = w["dx"] * w["dy"]
    assert abs(np.sum(mg) * dxdy - pr.observables()[0]["norm"]) <= 2e-7
    psi = pr.get_state(0).reshape(n, n)
    rows = np.random.default_rng(W.SEED).choice(n, size=48, replace=False)
    for r in rows:
        ref = float(np.sum(np.abs(psi[r].astype(np.complex128)) ** 2)) * dxdy
        assert abs(mg.reshape(-1)[r] - ref) <= 1e-12 * max(ref, 1e-300) + 1e-300
    # the packets sit on opposite edges: the slice through both edge maxima
    iy1, iy2 = ny // 2 + 5, ny // 2 - 6
    s, wt = pr.entanglement(0, iy1, iy2, (0, nx), (0, nx))
    psi4 = psi.reshape(nx, ny, nx, ny)
    sl = psi4[:, iy1:iy1 + 1, :, iy2:iy2 + 1].astype(np.complex128)
    s_ref, wt_ref = O.entanglement_entropy(sl, 0, 0, (0, nx), (0, nx))
    assert abs(s - s_ref) <= 1e-10 and abs(wt - wt_ref) <= 1e-10 * wt_ref
    assert 0.0 <= s <= math.log(nx)
