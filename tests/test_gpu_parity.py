"""GPU parity of libhom against the FP64 oracle, through the C ABI.

Tolerances (stated by the requirements of the method's precision study):
  complex128: max |psi_gpu - psi_oracle| / ||psi_oracle||_2 <= 1e-10
  complex64:  same ratio <= 2e-5
  bunching probability: |dP_b| <= 1e-6 (both precisions)
||.||_2 is the discrete l2 norm of the whole 4D array.
"""

import math

import numpy as np
import pytest

from oracle import adapter as A
from oracle import hom_oracle as O
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 2e-5}
PB_TOL = 1e-6


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


def small_w(nx=16, ny=16, prec="c128", **kw):
    w = W.tiny()
    w = W.shrink(w, nx=nx, ny=ny)
    w["dx"] = w["dy"] = 0.5
    w["prec"] = prec
    w.update(kw)
    return w


# --- initial state -----------------------------------------------------------

@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("exch", [-1, 0, 1])
def test_init_packets_matches_oracle(prec, exch):
    w = small_w(32, 16, prec)
    w["sims"][0]["exch"] = exch
    w["sims"][0]["alpha"] = W.packet(-2.0, 1.2, 2.5, +1)
    w["sims"][0]["beta"] = W.packet(1.5, 1.0, 2.8, -1)
    pr = H().Propagator(w)
    got = pr.get_state(0)
    ref = A.initial_state(w, w["sims"][0])
    assert rel_err(got, ref) <= (1e-13 if prec == "c128" else 2e-7)


def test_init_by_k0_and_errors():
    w = small_w(16, 16)
    w["sims"][0]["alpha"] = W.packet(-2.0, 1.0, k0=1.5, by_k0=True)
    w["sims"][0]["beta"] = W.packet(2.0, 1.0, k0=-0.5, by_k0=True)
    pr = H().Propagator(w)
    assert rel_err(pr.get_state(0), A.initial_state(w, w["sims"][0])) <= 1e-13
    bad = H().make_packet(W.packet(0.0, 1.0, 0.1, +1))        # below the lowest level
    with pytest.raises(H().HomError) as e:
        H().hom_init_packets(pr.ctx, 0, bad, bad, -1)
    assert e.value.status == H().HOM_ERR_ARG
    same = H().make_packet(W.packet(0.0, 1.0, 2.5, +1))       # Slater of identical packets vanishes
    with pytest.raises(H().HomError):
        H().hom_init_packets(pr.ctx, 0, same, same, -1)


# --- one Strang step on a random state (every index path) --------------------

@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16), (16, 32), (64, 16), (16, 64), (32, 32), (128, 16), (256, 16)])
def test_one_step_random_state(prec, nx, ny):
    w = small_w(nx, ny, prec, dt=0.03)
    w["sims"][0]["qpc_h"] = 1.3
    w["sims"][0]["lam"] = 0.7
    pr = H().Propagator(w, init=False)
    psi = W.random_state((nx, ny, nx, ny), seed=nx * 100 + ny)
    pr.set_state(0, psi)
    pr.step(1)
    got = pr.get_state(0)
    m = A.model_for(w, w["sims"][0])
    ref = O.strang_step(psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi, m)
    assert rel_err(got, ref) <= TOL[prec] * 0.05


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_three_steps_batch_of_three(prec):
    w = small_w(32, 16, prec, dt=0.02)
    w["sims"] = [dict(qpc_h=0.8, qpc_w=1.5, lam=0.0, alpha=W.packet(-2, 1, 2.5, 1), beta=W.packet(2, 1, 2.5, -1), exch=-1),
                 dict(qpc_h=1.2, qpc_w=1.0, lam=1.0, alpha=W.packet(-2, 1, 2.5, 1), beta=W.packet(2, 1, 2.5, -1), exch=0),
                 dict(qpc_h=1.0, qpc_w=2.0, lam=2.0, alpha=W.packet(-1, 1, 2.5, 1), beta=W.packet(2, 1.5, 2.5, -1), exch=1)]
    w["batch"] = 3
    pr = H().Propagator(w, init=False)
    states = [W.random_state((32, 16, 32, 16), seed=40 + b) for b in range(3)]
    for b in range(3):
        pr.set_state(b, states[b])
    pr.step(3)
    for b in range(3):
        m = A.model_for(w, w["sims"][b])
        s0 = states[b].astype(np.complex64).astype(np.complex128) if prec == "c64" else states[b]
        ref = O.propagate(s0, m, 3)
        assert rel_err(pr.get_state(b), ref) <= TOL[prec] * 0.1, b


@pytest.mark.parametrize("prec,tol", [("c128", 1e-12), ("c64", 2e-6)])
def test_time_reversal(prec, tol):
    """S(-dt) S(dt) = I for the Strang product (Eq. evoloperat, symmetric
    order): five steps forward, then five steps of a context with -dt on the
    result, give back the starting state.  Exercises the negative-dt tables."""
    w = small_w(64, 16, prec, dt=0.03)
    w["sims"][0]["lam"] = 1.1
    fwd = H().Propagator(w, init=False)
    psi = W.random_state((64, 16, 64, 16), seed=77)
    fwd.set_state(0, psi)
    start = fwd.get_state(0).astype(np.complex128)
    fwd.step(5)
    mid = fwd.get_state(0)
    back = H().Propagator(dict(w, dt=-w["dt"]), init=False)
    back.set_state(0, mid)
    back.step(5)
    assert rel_err(back.get_state(0), start) <= tol
    # the five steps did move the state (relative l2 change)
    assert np.linalg.norm((mid - start).ravel()) > 0.1 * np.linalg.norm(start.ravel())


@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("field", ["free", "no_field"])
def test_degenerate_hamiltonians(prec, field):
    """Degenerate cases of the Hamiltonian: a free particle (B = 0, no
    confinement, no saddle, no interaction) and confinement without a
    magnetic field (B = 0, where T_x loses its y dependence)."""
    kw = dict(B=0.0, omega=0.0) if field == "free" else dict(B=0.0)
    w = small_w(32, 16, prec, dt=0.03, **kw)
    if field == "free":
        w["sims"][0].update(qpc_h=0.0, lam=0.0)
    pr = H().Propagator(w, init=False)
    psi = W.random_state((32, 16, 32, 16), seed=5 if field == "free" else 6)
    pr.set_state(0, psi)
    pr.step(2)
    m = A.model_for(w, w["sims"][0])
    assert m.B == 0.0 and (m.omega == 0.0) == (field == "free")
    s0 = psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi
    assert rel_err(pr.get_state(0), O.propagate(s0, m, 2)) <= TOL[prec] * 0.05


def test_zero_steps_is_identity():
    w = small_w(16, 32, "c64")
    pr = H().Propagator(w)
    before = pr.get_state(0)
    pr.step(0)
    assert np.array_equal(before, pr.get_state(0))


def test_deterministic_and_batch_independent():
    w = small_w(32, 16, "c64", dt=0.02)
    w3 = dict(w)
    w3["sims"] = [w["sims"][0]] * 3
    w3["batch"] = 3
    p1 = H().Propagator(w)
    p3 = H().Propagator(w3)
    p1.step(7)
    p3.step(7)
    a = p1.get_state(0)
    for b in range(3):
        assert np.array_equal(a, p3.get_state(b))
    p1b = H().Propagator(w)
    p1b.step(7)
    assert np.array_equal(a, p1b.get_state(0))


# --- observables ---------------------------------------------------------------

@pytest.mark.parametrize("prec", ["c128", "c64"])
@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 64), (64, 16)])
def test_observables_random_state(prec, nx, ny):
    w = small_w(nx, ny, prec)
    pr = H().Propagator(w, init=False)
    m = A.model_for(w, w["sims"][0])
    psi = W.random_state((nx, ny, nx, ny), seed=7)
    psi /= math.sqrt(np.sum(np.abs(psi) ** 2) * m.dV)
    pr.set_state(0, psi)
    got = pr.observables()[0]
    ref = O.observables(psi.astype(np.complex64).astype(np.complex128) if prec == "c64" else psi, m)
    tol = 1e-11 if prec == "c128" else 2e-6
    for k in ("norm", "energy", "e_kin", "e_pot", "e_coul", "p_bunch"):
        assert abs(got[k] - ref[k]) <= tol * max(1.0, abs(ref[k])), (k, got[k], ref[k])


# --- the tiny configuration end to end ----------------------------------------

@pytest.fixture(scope="module")
def tiny_oracle():
    w = W.tiny()
    psi0 = A.initial_state(w, w["sims"][0])
    m = A.model_for(w, w["sims"][0])
    return w, m, O.propagate(psi0, m, w["nsteps"])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_tiny_full_run(tiny_oracle, prec):
    w, m, ref = tiny_oracle
    w = dict(w, prec=prec)
    pr = H().Propagator(w)
    pr.step(w["nsteps"])
    got = pr.get_state(0)
    assert rel_err(got, ref) <= TOL[prec]
    o = pr.observables()[0]
    r = O.observables(ref, m)
    assert abs(o["p_bunch"] - r["p_bunch"]) <= PB_TOL
    etol = 1e-10 if prec == "c128" else 1e-5
    for k in ("norm", "energy", "e_kin", "e_pot", "e_coul"):
        assert abs(o[k] - r[k]) <= etol * max(1.0, abs(r[k])), (k, o[k], r[k])
    # exchange antisymmetry holds on the device result
    assert np.max(np.abs(got + np.transpose(got, (2, 3, 0, 1)))) <= TOL[prec] * np.linalg.norm(got.ravel())


# --- full-scale grid (256 x 64 per electron, complex64), the bench's launch config

@pytest.fixture(scope="module")
def full_zero_coulomb():
    w = W.fullscale(sigma=2.0)
    w["sims"][0]["lam"] = 0.0
    nsteps = 20
    pr = H().Propagator(w)
    pr.step(nsteps)
    m, a, b = A.packets(w, w["sims"][0])
    a_t = O.propagate_2d(a, m, nsteps)
    b_t = O.propagate_2d(b, m, nsteps)
    return w, m, pr, a_t, b_t


def test_fullscale_zero_coulomb_rows_match_factorised_oracle(full_zero_coulomb):
    w, m, pr, a_t, b_t = full_zero_coulomb
    n = w["nx"] * w["ny"]
    a_f, b_f = a_t.ravel(), b_t.ravel()
    ab = np.vdot(a_f, b_f) * m.dx * m.dy
    # sum |a(r1) b(r2) - b(r1) a(r2)|^2 dV = 2 (1 - |<a|b>|^2) for unit packets
    c = 1.0 / math.sqrt(2.0 * (1.0 - abs(ab) ** 2))
    l2 = 1.0 / math.sqrt(m.dV)                       # ||psi||_2 of a normalised state
    rng = np.random.default_rng(W.SEED)
    rows = rng.choice(n, size=12, replace=False)
    worst = 0.0
    for r1 in rows:
        got = pr.state[0, int(r1), :].cpu().numpy().astype(np.complex128)
        ref = c * (a_f[r1] * b_f - b_f[r1] * a_f)
        worst = max(worst, float(np.max(np.abs(got - ref))) / l2)
    assert worst <= TOL["c64"], worst


def test_c128_maximum_plane_zero_coulomb_rows_match_factorised_oracle():
    """complex128 at its largest plane (128 x 64 per electron, nx*ny = 8192,
    a 1 GiB state): with lam = 0 the evolved state is the antisymmetrised
    product of the two single-particle evolutions, so sampled rows are checked
    against the FP64 2D oracle at the FP64 tolerance."""
    w = W.shrink(W.fullscale(sigma=2.0), nx=128)
    w["prec"] = "c128"
    w["sims"][0]["lam"] = 0.0
    nsteps = 20
    pr = H().Propagator(w)
    pr.step(nsteps)
    m, a, b = A.packets(w, w["sims"][0])
    a_f = O.propagate_2d(a, m, nsteps).ravel()
    b_f = O.propagate_2d(b, m, nsteps).ravel()
    ab = np.vdot(a_f, b_f) * m.dx * m.dy
    c = 1.0 / math.sqrt(2.0 * (1.0 - abs(ab) ** 2))
    l2 = 1.0 / math.sqrt(m.dV)
    n = w["nx"] * w["ny"]
    rows = np.random.default_rng(W.SEED + 1).choice(n, size=12, replace=False)
    worst = 0.0
    for r1 in rows:
        got = pr.state[0, int(r1), :].cpu().numpy()
        ref = c * (a_f[r1] * b_f - b_f[r1] * a_f)
        worst = max(worst, float(np.max(np.abs(got - ref))) / l2)
    assert worst <= TOL["c128"], worst
    o = pr.observables()[0]
    assert abs(o["norm"] - 1.0) < 1e-10
    pr.close()


def test_fullscale_invariants_with_coulomb():
    import torch

    w = W.fullscale(sigma=2.0)
    pr = H().Propagator(w)
    o0 = pr.observables()[0]
    pr.step(10)
    o1 = pr.observables()[0]
    assert abs(o0["norm"] - 1.0) < 1e-6 and abs(o1["norm"] - 1.0) < 1e-5
    assert abs(o1["energy"] - o0["energy"]) < 1e-3 * abs(o0["energy"])
    n = w["nx"] * w["ny"]
    rng = np.random.default_rng(5)
    r1 = torch.as_tensor(rng.integers(0, n, 4096), device="cuda")
    r2 = torch.as_tensor(rng.integers(0, n, 4096), device="cuda")
    a = pr.state[0, r1, r2]
    b = pr.state[0, r2, r1]
    scale = math.sqrt(1.0 / ((w["dx"] * w["dy"]) ** 2))
    assert float(torch.max(torch.abs(a + b))) <= 2e-5 * scale
