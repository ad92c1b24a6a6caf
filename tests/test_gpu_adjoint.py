"""Adjoint gradient of the bunching probability (hom_backward) against the
oracle's adjoint and against central finite differences of the CUDA path."""

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


def grad_w(prec, dt=0.05, sims=None):
    w = W.tiny()
    w["prec"] = prec
    w["dt"] = dt
    if sims is not None:
        w["sims"] = sims
        w["batch"] = len(sims)
    else:
        w["sims"][0]["alpha"] = W.packet(-2.0, 1.0, 2.5, +1)
        w["sims"][0]["beta"] = W.packet(2.0, 1.0, 2.5, -1)
    return w


def oracle_grad(w, sim, nsteps):
    m, a, b = A.packets(w, sim)
    psi0 = O.two_particle(a, b, sim["exch"], m.dV)
    kb = A.packet_k0(m, sim["beta"])
    db = O.edge_packet_dx0(m, sim["beta"]["x0"], sim["beta"]["sigma"], kb)
    dpsi = O.slater_dstate(a, b, db, sim["exch"], m.dV)
    return O.loss_and_gradient(psi0, dpsi, m, nsteps)


@pytest.mark.parametrize("prec,K", [("c128", 4), ("c128", 5), ("c64", 4)])
def test_adjoint_matches_oracle(prec, K):
    nsteps = 12
    w = grad_w(prec)
    pr = H().Propagator(w, ckpt_slots=-(-nsteps // K))
    loss, grad = pr.backward(nsteps, K)
    ref_loss, ref = oracle_grad(w, w["sims"][0], nsteps)
    tol = 1e-9 if prec == "c128" else 2e-4
    assert abs(loss[0] - ref_loss) <= (1e-12 if prec == "c128" else 2e-6)
    for i, k in enumerate(("h", "w", "delay")):
        assert abs(grad[0, i] - ref[k]) <= tol * max(abs(ref[k]), 1e-2), (k, grad[0, i], ref[k])
    # the state is back at step 0
    assert np.allclose(pr.get_state(0), A.initial_state(w, w["sims"][0]), rtol=0,
                       atol=(1e-12 if prec == "c128" else 1e-5) * np.abs(pr.get_state(0)).max())


def test_adjoint_batch_and_finite_differences():
    nsteps, K = 10, 5
    sims = [dict(qpc_h=1.0, qpc_w=1.5, lam=1.0, alpha=W.packet(-2, 1.0, 2.5, 1), beta=W.packet(2, 1.0, 2.5, -1), exch=-1),
            dict(qpc_h=0.8, qpc_w=1.2, lam=0.0, alpha=W.packet(-2, 1.2, 2.5, 1), beta=W.packet(2.3, 1.0, 2.5, -1), exch=0)]
    w = grad_w("c128", sims=sims)
    pr = H().Propagator(w, ckpt_slots=2)
    loss, grad = pr.backward(nsteps, K)
    for b, s in enumerate(sims):
        ref_loss, ref = oracle_grad(w, s, nsteps)
        assert abs(loss[b] - ref_loss) < 1e-12
        for i, k in enumerate(("h", "w", "delay")):
            assert abs(grad[b, i] - ref[k]) <= 1e-9 * max(abs(ref[k]), 1e-2), (b, k)

    # central finite differences of the CUDA forward path, h = 1e-4
    eps = 1e-4

    def loss_at(dh=0.0, dw=0.0, dd=0.0):
        s2 = [dict(s) for s in sims]
        for s in s2:
            s["qpc_h"] += dh
            s["qpc_w"] += dw
            s["beta"] = dict(s["beta"], x0=s["beta"]["x0"] + dd)
        q = H().Propagator(grad_w("c128", sims=s2))
        q.step(nsteps)
        return np.array([o["p_bunch"] for o in q.observables()])

    fd = np.stack([(loss_at(dh=eps) - loss_at(dh=-eps)) / (2 * eps),
                   (loss_at(dw=eps) - loss_at(dw=-eps)) / (2 * eps),
                   (loss_at(dd=eps) - loss_at(dd=-eps)) / (2 * eps)], axis=1)
    assert np.all(np.abs(grad - fd) <= 1e-6 * np.maximum(np.abs(fd), 1e-3)), (grad, fd)


def test_adjoint_errors():
    w = grad_w("c128")
    pr = H().Propagator(w, ckpt_slots=1)
    with pytest.raises(H().HomError) as e:
        pr.backward(10, 5)                      # needs 2 checkpoints
    assert e.value.status == H().HOM_ERR_ARG
    pr.set_state(0, pr.get_state(0))            # state no longer from packets
    with pytest.raises(H().HomError) as e:
        pr.backward(4, 4)
    assert e.value.status == H().HOM_ERR_STATE


def test_autograd_function():
    import torch

    from paper_1903_02581_gb300.autograd import BunchingProbability

    nsteps, K = 8, 4
    w = grad_w("c128")
    pr = H().Propagator(w, ckpt_slots=2)
    h = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    wd = torch.tensor([1.5], dtype=torch.float64, requires_grad=True)
    d = torch.tensor([0.0], dtype=torch.float64, requires_grad=True)
    pb = BunchingProbability.apply(h, wd, d, pr, nsteps, K)
    (3.0 * pb.sum()).backward()
    ref_loss, ref = oracle_grad(w, w["sims"][0], nsteps)
    assert abs(pb.item() - ref_loss) < 1e-12
    assert abs(h.grad.item() - 3 * ref["h"]) <= 1e-9 * max(abs(ref["h"]), 1e-2)
    assert abs(wd.grad.item() - 3 * ref["w"]) <= 1e-9 * max(abs(ref["w"]), 1e-2)
    assert abs(d.grad.item() - 3 * ref["delay"]) <= 1e-9 * max(abs(ref["delay"]), 1e-2)


def test_adjoint_with_screening_barriers_and_numeric_packets():
    """The adjoint composes with the potential-family options: screened
    Coulomb, barrier blocks added to V1 and numerical edge-state packets (with
    a wall); it still matches the oracle's adjoint and central differences."""
    nsteps, K = 8, 4
    w = grad_w("c128")
    w.update(screen=0.9, fermi_vb=1.5, fermi_tau=0.5, fermi_xa=-2.5, fermi_ya=-2.0, fermi_xb=2.5, fermi_yb=2.0)
    s = w["sims"][0]
    s["alpha"] = dict(W.packet(-2.0, 1.0, k0=1.4, by_k0=True), numeric=True, wall_y=-2.5, wall_side=1)
    s["beta"] = dict(W.packet(2.0, 1.0, k0=-1.4, by_k0=True), numeric=True, wall_y=2.5, wall_side=-1)
    pr = H().Propagator(w, ckpt_slots=2)
    loss, grad = pr.backward(nsteps, K)
    m, a, b = A.packets(w, s)
    psi0 = O.two_particle(a, b, s["exch"], m.dV)
    # d psi0 / d(beta centre): the packet is a sum of plane waves in x, so the
    # derivative is the same sum with weights -i k
    x = O.coords(m.nx, m.dx)
    k = O.wavenumbers(m.nx, m.dx)
    wk = np.exp(-(s["beta"]["sigma"] ** 2) * (k - s["beta"]["k0"]) ** 2)
    chi = np.array([O.edge_state_numeric(m, float(kk), s["beta"]["wall_y"], s["beta"]["wall_side"])[1]
                    if wk[i] >= 1e-300 else np.zeros(m.ny) for i, kk in enumerate(k)])
    plane = np.exp(1j * np.outer(x - s["beta"]["x0"], k))
    raw = plane @ (wk[:, None] * chi)
    db = (plane @ ((-1j * k * wk)[:, None] * chi)) / np.sqrt(np.sum(np.abs(raw) ** 2) * m.dx * m.dy)
    ref_loss, ref = O.loss_and_gradient(psi0, O.slater_dstate(a, b, db, s["exch"], m.dV), m, nsteps)
    assert abs(loss[0] - ref_loss) <= 1e-12
    for i, key in enumerate(("h", "w", "delay")):
        assert abs(grad[0, i] - ref[key]) <= 1e-9 * max(abs(ref[key]), 1e-2), (key, grad[0, i], ref[key])
