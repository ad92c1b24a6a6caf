"""Step strategies and kernel variants of libhom give bitwise-identical states.

Strategy 0 runs a transposing pass and an in-place pass per Strang step,
strategy 1 an in-place pass, a plain transpose and an in-place pass, and
strategy 2 a transpose and a double in-place pass (the end of one step, the
potential between steps and the start of the next); each kinetic pass has
two launch variants.  All of them apply the same arithmetic
to every element, so the states after any number of steps must agree bit for
bit, and one of them is checked against the FP64 oracle.
"""

import itertools

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


def small_w(nx, ny, prec):
    w = W.shrink(W.tiny(), nx=nx, ny=ny)
    w["dx"] = w["dy"] = 0.5
    w["prec"] = prec
    w["dt"] = 0.02
    w["sims"][0]["qpc_h"] = 1.1
    w["sims"][0]["lam"] = 0.8
    return w


CHOICES = list(itertools.product((0, 1), (0, 1), (0, 1, 2)))


@pytest.mark.parametrize("prec", ["c128", "c64"])
# (128, 32): the grid of the batched sweep, whose in-place pass runs its x
# stages in column groups while its transposing pass does not
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16), (64, 32), (128, 16), (16, 64), (128, 32)])
@pytest.mark.parametrize("nsteps", [1, 2, 5])
def test_choices_bitwise_identical(prec, nx, ny, nsteps):
    w = small_w(nx, ny, prec)
    psi = W.random_state((nx, ny, nx, ny), seed=nx + 7 * ny + nsteps)
    out = {}
    for ch in CHOICES:
        pr = H().Propagator(w, init=False)
        H().hom_autotune_set(pr.ctx, *ch)
        pr.set_state(0, psi)
        pr.step(nsteps)
        out[ch] = pr.get_state(0)
        assert H().hom_autotune_info(pr.ctx)["strategy"] == ch[2]
        pr.close()
    base = out[CHOICES[0]]
    for ch in CHOICES[1:]:
        assert np.array_equal(out[ch].view(np.uint8), base.view(np.uint8)), ch
    if nx * ny <= 512:
        m = A.model_for(w, w["sims"][0])
        s0 = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
        ref = O.propagate(s0, m, nsteps)
        err = np.max(np.abs(base.astype(np.complex128) - ref)) / np.linalg.norm(ref.ravel())
        assert err <= (1e-11 if prec == "c128" else 2e-6)


def test_choices_bitwise_identical_fullscale():
    """The full-scale grid (256x64 per electron, complex64, a 2 GiB state),
    where every kinetic pass runs its x stages in column groups and the
    in-place pass is persistent: three steps under every strategy and variant
    give the same bits.  The states are compared on the device."""
    import torch

    w = W.fullscale()
    ref = None
    for ch in CHOICES:
        pr = H().Propagator(w)
        H().hom_autotune_set(pr.ctx, *ch)
        pr.step(3)
        assert H().hom_autotune_info(pr.ctx)["strategy"] == ch[2]
        bits = torch.view_as_real(pr.state).view(torch.int32)
        if ref is None:
            ref = bits.clone()
            assert bool(torch.isfinite(torch.view_as_real(pr.state)).all())
        else:
            assert torch.equal(bits, ref), ch
        pr.close()
        del pr, bits
    del ref
    torch.cuda.empty_cache()


def test_strategy_one_batched_profile_counts():
    w = small_w(32, 16, "c64")
    w["sims"] = w["sims"] * 3
    w["batch"] = 3
    pr = H().Propagator(w)
    H().hom_autotune_set(pr.ctx, 0, 0, 1)
    H().hom_profile(pr.ctx, 1)
    pr.step(3)
    prof = H().hom_profile_read(pr.ctx)
    # steps 0 and 1: in-place, transpose, in-place; step 2 (ends off the
    # caller's layout): in-place, transpose, transposing pass
    assert prof["n_in_place"] == 5
    assert prof["n_transpose"] == 3
    assert prof["n_transposing"] == 1
    assert prof["ms_transpose"] > 0.0
    H().hom_profile(pr.ctx, 0)


def test_strategy_two_profile_counts():
    w = small_w(32, 16, "c64")
    pr = H().Propagator(w)
    H().hom_autotune_set(pr.ctx, 1, 1, 2)
    H().hom_profile(pr.ctx, 1)
    pr.step(3)
    prof = H().hom_profile_read(pr.ctx)
    # in-place (opening phase); then per step a transpose and a double pass,
    # the last step a single in-place pass and (odd count) a transpose back
    assert prof["n_in_place"] == 2
    assert prof["n_double"] == 2
    assert prof["n_transpose"] == 4
    assert prof["n_transposing"] == 0
    pr.step(4)
    prof = H().hom_profile_read(pr.ctx)
    assert (prof["n_in_place"], prof["n_double"], prof["n_transpose"]) == (4, 5, 8)
    H().hom_profile(pr.ctx, 0)


@pytest.mark.parametrize("strategy", [0, 1, 2])
def test_graph_replay_matches_plain_launches(strategy):
    """hom_step captures its launches into a CUDA graph per step count and
    replays it; with profiling on it launches the same kernels one by one
    instead.  Both give the same state bit for bit, including the second call
    of a step count, which replays the graph the first call captured."""
    w = small_w(64, 32, "c64")
    psi = W.random_state((64, 32, 64, 32), seed=31 + strategy)
    out = []
    for profile in (False, True):
        pr = H().Propagator(w, init=False)
        H().hom_autotune_set(pr.ctx, 0, 0, strategy)
        pr.set_state(0, psi)
        if profile:
            H().hom_profile(pr.ctx, 1)
        pr.step(5)
        pr.step(5)
        out.append(pr.get_state(0))
        if profile:
            assert sum(H().hom_profile_read(pr.ctx)[k] for k in ("n_transposing", "n_in_place", "n_transpose",
                                                                "n_double")) > 0
            H().hom_profile(pr.ctx, 0)
        pr.close()
    assert np.array_equal(out[0].view(np.uint8), out[1].view(np.uint8))


def test_autotune_set_rejects_bad_choice():
    w = small_w(16, 16, "c64")
    pr = H().Propagator(w)
    with pytest.raises(H().HomError) as e:
        H().hom_autotune_set(pr.ctx, 0, 2, 0)
    assert e.value.status == H().HOM_ERR_ARG
    with pytest.raises(H().HomError):
        H().hom_autotune_set(pr.ctx, 0, 0, 3)


def test_autotune_reports_both_strategies():
    w = small_w(32, 32, "c64")
    pr = H().Propagator(w)
    before = pr.get_state(0)
    pr.step(24)
    info = H().hom_autotune_info(pr.ctx)
    assert info["strategy"] in (0, 1, 2)
    assert all(v in (0, 1) for v in info["variants"])
    assert len(info["step_ms"]) == 3 and min(info["step_ms"]) > 0.0
    assert info["step_ms"][info["strategy"]] == min(info["step_ms"])
    # the tuner's 12 steps (six calls of 2) are part of the 24
    ref = H().Propagator(w)
    H().hom_autotune_set(ref.ctx, 0, 0, 0)
    assert np.array_equal(ref.get_state(0), before)
    for _ in range(6):
        ref.step(2)
    ref.step(12)
    assert np.array_equal(ref.get_state(0).view(np.uint8), pr.get_state(0).view(np.uint8))


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_choices_bitwise_identical_batched(prec):
    """Three simulations with different potentials: every choice gives the
    same bits, and each simulation matches the oracle."""
    from oracle import adapter as A
    from oracle import hom_oracle as O

    w = small_w(32, 16, prec)
    w["sims"] = [dict(w["sims"][0], qpc_h=0.7 + 0.3 * b, lam=0.5 * b) for b in range(3)]
    w["batch"] = 3
    states = [W.random_state((32, 16, 32, 16), seed=200 + b) for b in range(3)]
    out = {}
    for ch in CHOICES:
        pr = H().Propagator(w, init=False)
        H().hom_autotune_set(pr.ctx, *ch)
        for b in range(3):
            pr.set_state(b, states[b])
        pr.step(3)
        out[ch] = [pr.get_state(b) for b in range(3)]
        pr.close()
    base = out[CHOICES[0]]
    for ch in CHOICES[1:]:
        for b in range(3):
            assert np.array_equal(out[ch][b].view(np.uint8), base[b].view(np.uint8)), (ch, b)
    for b in range(3):
        m = A.model_for(w, w["sims"][b])
        s0 = states[b].astype(np.complex64).astype(np.complex128) if prec == "c64" else states[b]
        ref = O.propagate(s0, m, 3)
        err = np.max(np.abs(base[b].astype(np.complex128) - ref)) / np.linalg.norm(ref.ravel())
        assert err <= (1e-11 if prec == "c128" else 2e-6), (b, err)
