"""The gradient and batched workloads at their full sizes, checked by properties.

The FP64 oracle cannot run these sizes in a test (the 64x32 adjoint would
store 800 FP64 states of 67 MB; the batch is 537M points per step), so the
checks are the ones the method fixes at any size:

- gradient (64x32 per electron, 800 steps, checkpoints every 50): the FP64
  adjoint gradient equals central finite differences (h = 1e-4, FP64) of the
  forward path; FP32 and FP64 adjoint gradients agree to the FP32 state
  precision.  The oracle's own adjoint is compared with the CUDA adjoint at
  small sizes in test_gpu_adjoint.py.
- batched sweep (32 simulations of 128x32 per electron, 1500 steps): one
  simulation of the batch equals the same simulation run alone, bit for bit;
  for a sample of the simulations (one without and one with Coulomb), the
  FP32 run matches an FP64 run of the same simulation in the bunching
  probability (the raw sum) to 1e-6, with the norm within 2e-6 of 1 and the
  energy drift within 2e-5.

Tolerances:
- FD: 1e-6 relative.  The truncation error of a central difference with
  h = 1e-4 is O(h^2) ~ 1e-8 relative for these smooth losses, and the
  rounding is ~1e-16 / h.
- FP32 against FP64 gradients: 1e-4 relative, the FP32 rounding of 800
  steps forward and back.
- FP32 losses: 2e-5 absolute, the FP32 state tolerance relative to the norm.
"""

import copy

import numpy as np
import pytest

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


def test_gradient_fullsize_finite_differences_and_precision():
    w = W.gradient()
    nsteps, K = w["nsteps"], w["ckpt_every"]
    res = {}
    for prec in ("c64", "c128"):
        wp = copy.deepcopy(w)
        wp["prec"] = prec
        pr = H().Propagator(wp, ckpt_slots=-(-nsteps // K))
        loss, grad = pr.backward(nsteps, K)
        res[prec] = (loss[0], grad[0])
        pr.close()

    eps = 1e-4

    def loss_at(dh=0.0, dw=0.0, dd=0.0):
        wp = copy.deepcopy(w)
        wp["prec"] = "c128"
        s = wp["sims"][0]
        s["qpc_h"] += dh
        s["qpc_w"] += dw
        s["beta"] = dict(s["beta"], x0=s["beta"]["x0"] + dd)
        q = H().Propagator(wp)
        q.step(nsteps)
        r = q.observables()[0]["p_bunch"]
        q.close()
        return r

    fd = np.array([(loss_at(dh=eps) - loss_at(dh=-eps)) / (2 * eps),
                   (loss_at(dw=eps) - loss_at(dw=-eps)) / (2 * eps),
                   (loss_at(dd=eps) - loss_at(dd=-eps)) / (2 * eps)])
    g128 = res["c128"][1]
    g64 = res["c64"][1]
    assert np.all(np.abs(g128 - fd) <= 1e-6 * np.abs(fd)), (g128, fd)
    assert np.all(np.abs(g64 - g128) <= 1e-4 * np.abs(g128)), (g64, g128)
    assert abs(res["c64"][0] - res["c128"][0]) <= 2e-5


def test_batched_fullsize_sampled_against_fp64():
    wb = W.batched()
    nsteps = wb["nsteps"]
    pr = H().Propagator(wb)
    before = pr.observables()
    pr.step(nsteps)
    after = pr.observables()
    s0 = pr.get_state(0)
    pr.close()
    for b in (0, len(wb["sims"]) - 1):
        assert wb["sims"][b]["lam"] == (0.0 if b == 0 else 1.0)
        one = copy.deepcopy(wb)
        one["sims"] = [wb["sims"][b]]
        one["batch"] = 1
        if b == 0:
            q = H().Propagator(copy.deepcopy(one))
            q.step(nsteps)
            assert np.array_equal(q.get_state(0).view(np.uint8), s0.view(np.uint8))
            q.close()
        one["prec"] = "c128"
        q = H().Propagator(one)
        q.step(nsteps)
        r = q.observables()[0]
        q.close()
        a, e0 = after[b], before[b]["energy"]
        assert abs(a["p_bunch"] - r["p_bunch"]) <= 1e-6, (b, a, r)
        assert abs(a["norm"] - 1.0) <= 2e-6
        assert abs(r["norm"] - 1.0) <= 1e-10
        assert abs(a["energy"] - e0) <= 2e-5 * abs(e0)
        assert abs(a["energy"] - r["energy"]) <= 2e-5 * abs(r["energy"])
