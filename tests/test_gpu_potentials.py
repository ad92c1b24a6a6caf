"""The screened Coulomb interaction (Eq. screenedCoulomb), the paper's
first-order Lie product (Eq. evoloperat as printed), the barrier blocks of
Eq. pot_xy and numerical edge-state packets (Eq. H_effective) on the GPU,
against the FP64 oracle.

Tolerances are those of the Strang path: complex128 1e-10 and complex64 2e-5
relative to the l2 norm of the state, observables 1e-11 (complex128).
"""

import numpy as np
import pytest

from oracle import adapter as A
from oracle import hom_oracle as O
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 2e-5}


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


def rel_err(gpu, ora):
    return float(np.max(np.abs(gpu.astype(np.complex128) - ora)) / np.linalg.norm(ora.ravel()))


def small_w(nx, ny, prec, **kw):
    w = W.shrink(W.tiny(), nx=nx, ny=ny)
    w["dx"] = w["dy"] = 0.5
    w["prec"] = prec
    w["dt"] = 0.03
    w["sims"][0]["qpc_h"] = 1.2
    w["sims"][0]["lam"] = 1.3
    w.update(kw)
    return w


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("nx,ny", [(32, 16), (16, 32)])
def test_screened_coulomb_steps_and_energy(prec, nx, ny):
    w = small_w(nx, ny, prec, screen=0.8)
    pr = H().Propagator(w, init=False)
    psi = W.random_state((nx, ny, nx, ny), seed=3 * nx + ny)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * (w["dx"] * w["dy"]) ** 2)
    pr.set_state(0, psi)
    m = A.model_for(w, w["sims"][0])
    assert m.screen == 0.8
    s0 = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
    got = pr.observables()[0]["e_coul"]
    ref = O.observables(s0, m)["e_coul"]
    assert abs(got - ref) <= (1e-11 if prec == "c128" else 2e-6) * abs(ref)
    unscreened = O.observables(s0, A.model_for(dict(w, screen=0.0), w["sims"][0]))["e_coul"]
    assert ref < 0.9 * unscreened
    pr.step(3)
    assert rel_err(pr.get_state(0), O.propagate(s0, m, 3)) <= TOL[prec] * 0.1


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("nsteps", [1, 4, 5])
def test_lie_product_all_strategies(prec, nsteps):
    w = small_w(32, 16, prec, split="lie")
    psi = W.random_state((32, 16, 32, 16), seed=70 + nsteps)
    m = A.model_for(w, w["sims"][0])
    s0 = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
    ref = O.propagate(s0, m, nsteps, order="lie")
    strang = O.propagate(s0, m, nsteps)
    out = []
    for strategy in (0, 1, 2):
        pr = H().Propagator(w, init=False)
        H().hom_autotune_set(pr.ctx, 0, 0, strategy)
        pr.set_state(0, psi)
        pr.step(nsteps)
        out.append(pr.get_state(0))
        assert rel_err(out[-1], ref) <= TOL[prec] * 0.1
        pr.close()
    assert all(np.array_equal(o.view(np.uint8), out[0].view(np.uint8)) for o in out[1:])
    # the Lie and Strang products really differ at this dt, by far more than
    # the GPU differs from the Lie oracle
    assert rel_err(out[0], strang) > max(1e-4, 20 * rel_err(out[0], ref))


def test_lie_rejects_adjoint():
    w = small_w(16, 16, "c128", split="lie")
    pr = H().Propagator(w, ckpt_slots=2)
    with pytest.raises(H().HomError) as e:
        pr.backward(4, 2)
    assert e.value.status == H().HOM_ERR_ARG


# --- the barrier blocks of Eq. pot_xy and numerical edge states (Eq. H_effective)

FERMI = dict(fermi_vb=2.5, fermi_tau=0.4, fermi_xa=-1.0, fermi_ya=-0.75, fermi_xb=1.0, fermi_yb=0.75)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_fermi_blocks_steps_and_energy(prec):
    w = small_w(32, 16, prec, **FERMI)
    pr = H().Propagator(w, init=False)
    psi = W.random_state((32, 16, 32, 16), seed=91)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * (w["dx"] * w["dy"]) ** 2)
    pr.set_state(0, psi)
    m = A.model_for(w, w["sims"][0])
    assert m.fermi_vb == 2.5
    s0 = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
    got = pr.observables()[0]["e_pot"]
    ref = O.observables(s0, m)["e_pot"]
    assert abs(got - ref) <= (1e-11 if prec == "c128" else 2e-6) * abs(ref)
    pr.step(3)
    assert rel_err(pr.get_state(0), O.propagate(s0, m, 3)) <= TOL[prec] * 0.1


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_numeric_edge_packets(prec):
    w = small_w(32, 16, prec, **FERMI)
    w["dt"] = 0.01
    a = dict(W.packet(-3.0, 1.2, k0=1.5, by_k0=True), numeric=True, wall_y=-2.0, wall_side=1)
    b = dict(W.packet(3.0, 1.2, k0=-1.5, by_k0=True), numeric=True, wall_y=2.0, wall_side=-1)
    w["sims"][0].update(alpha=a, beta=b, exch=-1)
    pr = H().Propagator(w)
    ref0 = A.initial_state(w, w["sims"][0])
    assert rel_err(pr.get_state(0), ref0) <= (1e-12 if prec == "c128" else 2e-7)
    # the walls really change the packets
    plain = dict(w["sims"][0], alpha=dict(a, numeric=False), beta=dict(b, numeric=False))
    assert rel_err(pr.get_state(0), A.initial_state(w, plain)) > 1e-4
    pr.step(5)
    m = A.model_for(w, w["sims"][0])
    # complex64: start the oracle from the rounded initial state
    s0 = ref0 if prec == "c128" else H().Propagator(w).get_state(0).astype(np.complex128)
    assert rel_err(pr.get_state(0), O.propagate(s0, m, 5)) <= TOL[prec] * 0.1


def test_numeric_packet_errors():
    w = small_w(16, 16, "c128", **FERMI)
    pr = H().Propagator(w, init=False)
    bad = H().make_packet(dict(W.packet(0.0, 1.0, 2.5, 1), numeric=True))      # numeric needs k0
    good = H().make_packet(dict(W.packet(2.0, 1.0, k0=-1.0, by_k0=True), numeric=True, wall_side=1))
    with pytest.raises(H().HomError) as e:
        H().hom_init_packets(pr.ctx, 0, bad, good, -1)
    assert e.value.status == H().HOM_ERR_ARG
    side = H().make_packet(dict(W.packet(2.0, 1.0, k0=-1.0, by_k0=True), numeric=True, wall_side=0))
    with pytest.raises(H().HomError):
        H().hom_init_packets(pr.ctx, 0, good, side, -1)
