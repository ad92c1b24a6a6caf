"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Each test fixes something the paper or the mathematics determines, chosen so
that a plausible mistake in the oracle (a dropped term, a wrong sign, a
transposed axis, a wrong normalisation) fails at least one of them.  None of
them compares the oracle with itself.
"""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import hom_oracle as O
from paper_1903_02581_gb300 import workloads as W


def small(**kw):
    base = dict(nx=16, ny=16, dx=0.5, dy=0.5, B=1.0, omega=1.0, dt=0.02,
                qpc_h=1.0, qpc_w=1.5, lam=1.0, soft=0.5)
    base.update(kw)
    return O.Model(**base)


def ip(a, b, m):
    return np.sum(np.conj(a) * b) * m.dV


# --- I1: the discrete Fourier transform -------------------------------------

def test_dft_matches_library_fft():
    a = W.random_state((8, 16, 4, 32), seed=1)
    for ax in range(4):
        got = O.dft_axis(a, ax)
        ref = np.fft.fft(a, axis=ax)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
        back = O.dft_axis(got, ax, inverse=True)
        assert np.max(np.abs(back - a)) <= 1e-13 * np.max(np.abs(a))


def test_grid_and_wavenumber_conventions():
    x = O.coords(16, 0.5)
    assert np.allclose(x, -x[::-1], atol=0, rtol=0) and abs(x[0] + 3.75) < 1e-15
    k = O.wavenumbers(16, 0.5)
    assert np.allclose(k, 2 * np.pi * np.fft.fftfreq(16, d=0.5), rtol=0, atol=1e-14)
    assert k[8] < 0                       # Nyquist mode taken negative (R4)


# --- I2 / I3 / I9: unitarity, exchange antisymmetry, time reversal ----------

def test_norm_conserved_on_random_state():
    m = small()
    psi = W.random_state((16, 16, 16, 16), seed=2)
    n0 = np.sum(np.abs(psi) ** 2)
    out = O.propagate(psi, m, 10)
    assert abs(np.sum(np.abs(out) ** 2) / n0 - 1.0) <= 1e-12


def slater_pair(m, exch=-1, sigma=1.0, xs=2.0, energy=2.5):
    ka = O.k0_from_energy(energy, m.B, m.omega, +1)
    kb = O.k0_from_energy(energy, m.B, m.omega, -1)
    a = O.edge_packet(m, -xs, sigma, ka)
    b = O.edge_packet(m, +xs, sigma, kb)
    return a, b, O.two_particle(a, b, exch, m.dV)


def test_exchange_antisymmetry_preserved():
    m = small()
    _, _, psi = slater_pair(m)
    out = O.propagate(psi, m, 20)
    swapped = np.transpose(out, (2, 3, 0, 1))
    assert np.max(np.abs(out + swapped)) <= 1e-13 * np.max(np.abs(out))
    assert np.max(np.abs(out)) > 0.01


def test_time_reversal():
    m = small()
    psi = W.random_state((16, 16, 16, 16), seed=3)
    back = O.strang_step(O.strang_step(psi, m), m, dt=-m.dt)
    assert np.max(np.abs(back - psi)) <= 1e-12 * np.max(np.abs(psi))


# --- I4: zero Coulomb factorises into independently propagated packets ------

def test_zero_coulomb_is_slater_of_propagated_packets():
    m = small(lam=0.0)
    a, b, psi = slater_pair(m)
    out = O.propagate(psi, m, 25)
    a_t = O.propagate_2d(a, m, 25)
    b_t = O.propagate_2d(b, m, 25)
    ref = O.two_particle(a_t, b_t, -1, m.dV)
    # same normalisation constant at t and at 0 (unitary, swap-symmetric)
    scale = np.sum(np.abs(ref) ** 2) / np.sum(np.abs(out) ** 2)
    assert abs(scale - 1.0) < 1e-12
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


# --- I5: free Gaussian spreading (B = 0, V = 0: the splitting is exact) -----

def test_free_gaussian_spreading_closed_form():
    m = O.Model(nx=32, ny=8, dx=0.4, dy=0.5, B=0.0, omega=0.0, dt=0.25,
                qpc_h=0.0, lam=0.0)
    s0 = 0.5
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)
    gx = np.exp(-x ** 2 / (4 * s0 ** 2))
    gy = np.exp(-y ** 2 / 2.0)
    phi = np.outer(gx, gy).astype(np.complex128)
    phi /= math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)
    psi = np.einsum("ab,cd->abcd", phi, phi)
    t = 0.5
    out = O.propagate(psi, m, 2)                     # two steps of 0.25
    rho_x1 = np.sum(np.abs(out) ** 2, axis=(1, 2, 3)) * m.dV / m.dx
    mean = np.sum(x * rho_x1) * m.dx
    var = np.sum((x - mean) ** 2 * rho_x1) * m.dx
    exact = s0 ** 2 * (1.0 + t ** 2 / (4.0 * s0 ** 4))
    assert abs(mean) < 1e-12
    assert abs(var - exact) <= 1e-10


# --- I7: Landau levels, cyclotron motion, hybrid edge levels ----------------

def eigen_product(m, k1, k2):
    """Product of two single-k lowest hybrid states e^{ikx} phi_k(y)."""
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)
    om = O.hybrid_omega(m.B, m.omega)

    def one(k):
        phi = np.exp(1j * k * x)[:, None] * np.exp(-0.5 * om * (y - k * m.B / om ** 2) ** 2)[None, :]
        return phi / math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)

    return np.einsum("ab,cd->abcd", one(k1), one(k2))


def level_energy(m, k):
    om = O.hybrid_omega(m.B, m.omega)
    return 0.5 * om + k * k * m.omega ** 2 / (2 * om ** 2)


@pytest.mark.parametrize("B,omega", [(1.0, 0.0), (1.0, 1.0), (1.5, 0.5)])
def test_level_phase_converges_at_second_order(B, omega):
    m = O.Model(nx=8, ny=32, dx=0.5, dy=0.4, B=B, omega=omega, qpc_h=0.0, lam=0.0)
    k = O.wavenumbers(m.nx, m.dx)
    k1, k2 = k[1], k[7]                               # +pi/4 and -pi/4
    psi0 = eigen_product(m, k1, k2)
    E = level_energy(m, k1) + level_energy(m, k2)
    # exact energy of the discrete state (spectral accuracy)
    obs = O.observables(psi0, m)
    assert abs(obs["energy"] - E) <= 1e-10
    T = 1.0
    errs = []
    for n in (20, 40):
        out = O.propagate(psi0, m, n, dt=T / n)
        errs.append(abs(ip(psi0, out, m) - np.exp(-1j * E * T)))
    ratio = errs[0] / errs[1]
    assert 3.6 < ratio < 4.4, (errs, ratio)
    assert errs[1] < 1e-3


def test_cyclotron_half_period():
    m = O.Model(nx=8, ny=32, dx=0.5, dy=0.4, B=1.0, omega=0.0, qpc_h=0.0, lam=0.0)
    y = O.coords(m.ny, m.dy)
    A = 1.0
    shifted = np.ones((m.nx, 1)) * np.exp(-0.5 * (y - A) ** 2)[None, :]
    ground = np.ones((m.nx, 1)) * np.exp(-0.5 * y ** 2)[None, :]
    psi0 = np.einsum("ab,cd->abcd", shifted, ground).astype(np.complex128)
    psi0 /= math.sqrt(np.sum(np.abs(psi0) ** 2) * m.dV)
    # <y1>(t) = A cos(B t).  At the quarter period the splitting's O(dt^2)
    # frequency shift shows at first order; at the half period only at second.
    def y1_at(t, n):
        out = O.propagate(psi0, m, n, dt=t / n)
        rho_y1 = np.sum(np.abs(out) ** 2, axis=(0, 2, 3)) * m.dV
        return np.sum(y * rho_y1)

    errs = [abs(y1_at(math.pi / 2, n)) for n in (12, 24)]
    assert errs[1] < 2e-3
    assert 3.5 < errs[0] / errs[1] < 4.5, errs
    half = [abs(y1_at(math.pi, n) + A) for n in (24, 48)]
    assert half[1] < 1e-5 and half[0] / half[1] > 12.0, half


# --- I8: Strang is second order, the printed (Lie) product first order ------

def test_splitting_orders():
    m = small(dt=0.04)
    _, _, psi = slater_pair(m)
    T = 0.32
    ref = O.propagate(psi, m, 64, dt=T / 64)
    e = {}
    for order in ("strang", "lie"):
        e[order] = [np.max(np.abs(O.propagate(psi, m, n, order=order, dt=T / n) - ref))
                    for n in (4, 8)]
    rs = e["strang"][0] / e["strang"][1]
    rl = e["lie"][0] / e["lie"][1]
    assert 3.5 < rs < 4.5, e
    assert 1.7 < rl < 2.3, e


# --- energy conservation ties the propagator's V and T to the observable ----

def test_energy_conserved_to_second_order():
    m = small()
    _, _, psi = slater_pair(m)
    e0 = O.observables(psi, m)["energy"]
    T = 0.4
    drifts = []
    for n in (10, 20):
        out = O.propagate(psi, m, n, dt=T / n)
        drifts.append(abs(O.observables(out, m)["energy"] - e0))
    assert drifts[1] < 1e-3
    assert 3.0 < drifts[0] / drifts[1] < 5.0, drifts


def test_energy_terms_change_sign_with_coulomb_strength():
    m = small()
    _, _, psi = slater_pair(m)
    o1 = O.observables(psi, m)
    o2 = O.observables(psi, small(lam=-1.0))
    assert o1["e_coul"] > 0 and abs(o1["e_coul"] + o2["e_coul"]) < 1e-14
    assert abs(o1["e_pot"] - o2["e_pot"]) < 1e-14


# --- Coulomb expectation by independent quadrature (Eq. coulomb) ------------

@pytest.mark.parametrize("screen", [0.0, 0.7])
def test_coulomb_expectation_matches_quadrature(screen):
    m = O.Model(nx=32, ny=32, dx=0.25, dy=0.25, lam=1.0, soft=1.2, screen=screen)
    s = 0.35
    # with screening the integrand has a cusp at r1 = r2, which the grid sum
    # resolves only to O(dx^2); the centres are far enough apart that the
    # relative-coordinate density there is ~1e-8
    ca, cb = (-0.6, 0.0), (0.6, 0.3)
    if screen > 0:
        ca, cb = (-1.5, 0.0), (1.5, 0.3)
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)

    def g(c):
        phi = np.exp(-((x[:, None] - c[0]) ** 2 + (y[None, :] - c[1]) ** 2) / (4 * s * s))
        return (phi / math.sqrt(np.sum(phi ** 2) * m.dx * m.dy)).astype(np.complex128)

    psi = np.einsum("ab,cd->abcd", g(ca), g(cb))
    got = O.observables(psi, m)["e_coul"]
    # relative coordinate R = r1 - r2 ~ N(ca - cb, 2 s^2 I)
    mu = (ca[0] - cb[0], ca[1] - cb[1])
    v = 2 * s * s

    def f(ry, rx):
        pdf = math.exp(-((rx - mu[0]) ** 2 + (ry - mu[1]) ** 2) / (2 * v)) / (2 * math.pi * v)
        damp = math.exp(-math.hypot(rx, ry) / screen) if screen > 0 else 1.0
        return pdf * damp / math.sqrt(rx * rx + ry * ry + m.soft ** 2)

    L = 8 * math.sqrt(v)
    ref, _ = integrate.dblquad(f, mu[0] - L, mu[0] + L, mu[1] - L, mu[1] + L,
                               epsabs=1e-13, epsrel=1e-12)
    assert abs(got - ref) <= (1e-9 if screen == 0 else 1e-8) * ref


# --- packet construction (Eq. singlepwp, R6) --------------------------------

def test_packet_energy_closed_form():
    m = O.Model(nx=64, ny=32, dx=0.5, dy=0.4, B=1.0, omega=1.0, qpc_h=0.0, lam=0.0)
    sigma = 1.5
    k0 = O.k0_from_energy(2.5, m.B, m.omega, +1)
    assert abs(level_energy(m, k0) - 2.5) < 1e-14
    phi = O.edge_packet(m, -3.0, sigma, k0)
    om = O.hybrid_omega(m.B, m.omega)
    exact = 0.5 * om + m.omega ** 2 / (2 * om ** 2) * (k0 ** 2 + 1.0 / (4 * sigma ** 2))
    assert abs(O.energy_2d(phi, m) - exact) <= 1e-9
    # centre of the x-marginal
    x = O.coords(m.nx, m.dx)
    rho = np.sum(np.abs(phi) ** 2, axis=1) * m.dy
    assert abs(np.sum(x * rho) * m.dx + 3.0) < 1e-9


def test_packet_direction_and_edge():
    m = O.Model(nx=64, ny=32, dx=0.5, dy=0.4)
    y = O.coords(m.ny, m.dy)
    for d in (+1, -1):
        k0 = O.k0_from_energy(2.5, m.B, m.omega, d)
        phi = O.edge_packet(m, 0.0, 1.5, k0)
        rho_y = np.sum(np.abs(phi) ** 2, axis=0) * m.dx
        yc = np.sum(y * rho_y) * m.dy
        assert np.sign(yc) == d and abs(yc - k0 / 2.0) < 0.05


def test_two_particle_slater_vanishes_on_diagonal():
    m = small()
    _, _, psi = slater_pair(m)
    n = m.nx * m.ny
    flat = psi.reshape(n, n)
    assert np.max(np.abs(np.diag(flat))) <= 1e-15 * np.max(np.abs(flat))
    assert abs(np.sum(np.abs(psi) ** 2) * m.dV - 1.0) < 1e-13


# --- I6: exchange-sum identity with Coulomb on ------------------------------

def test_exchange_sum_identity():
    m = small()
    a, b, _ = slater_pair(m)
    prod = O.two_particle(a, b, 0, m.dV)
    ov = abs(np.sum(np.conj(a) * b) * m.dx * m.dy) ** 2
    n = 15
    pp = O.bunching(O.propagate(prod, m, n), m)
    total = 0.0
    for s in (+1, -1):
        st = O.two_particle(a, b, s, m.dV)
        total += (1 + s * ov) * O.bunching(O.propagate(st, m, n), m)
    assert abs(total - 2 * pp) <= 1e-12


def test_bunching_counts_same_side_pairs():
    m = small()
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)

    def blob(xc):
        phi = np.exp(-((x[:, None] - xc) ** 2 + y[None, :] ** 2) / 0.1).astype(np.complex128)
        return phi / math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)

    left, right = blob(-2.0), blob(2.0)
    assert O.bunching(O.two_particle(left, left, 0, m.dV), m) > 1 - 1e-12
    assert O.bunching(O.two_particle(right, right, 0, m.dV), m) > 1 - 1e-12
    assert O.bunching(O.two_particle(left, right, 0, m.dV), m) < 1e-12
    # half of a particle on each side, the other one left: P_b = 1/2
    both = (left + right) / math.sqrt(2.0)
    assert abs(O.bunching(O.two_particle(both, left, 0, m.dV), m) - 0.5) < 1e-12


def test_bunching_is_half_for_uniform_density():
    m = small()
    psi = np.ones((16, 16, 16, 16), dtype=np.complex128)
    psi /= math.sqrt(np.sum(np.abs(psi) ** 2) * m.dV)
    assert abs(O.bunching(psi, m) - 0.5) < 1e-14


# --- I10: adjoint ------------------------------------------------------------

def test_adjoint_dot_product():
    m = small()
    u = W.random_state((16, 16, 16, 16), seed=4)
    v = W.random_state((16, 16, 16, 16), seed=5)
    lhs = np.sum(np.conj(O.strang_step(u, m)) * v)
    rhs = np.sum(np.conj(u) * O.strang_step(v, m, dt=-m.dt))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_gradient_matches_finite_differences():
    m = small(dt=0.05)
    n = 12
    xs, sig, delay = 2.0, 1.0, 0.0
    ka = O.k0_from_energy(2.5, m.B, m.omega, +1)
    kb = O.k0_from_energy(2.5, m.B, m.omega, -1)

    def state(dl):
        a = O.edge_packet(m, -xs, sig, ka)
        b = O.edge_packet(m, xs + dl, sig, kb)
        return a, b, O.two_particle(a, b, -1, m.dV)

    a, b, psi0 = state(delay)
    db = O.edge_packet_dx0(m, xs + delay, sig, kb)
    dpsi = O.slater_dstate(a, b, db, -1, m.dV)
    loss, grad = O.loss_and_gradient(psi0, dpsi, m, n)

    def L(mm, p0):
        return O.bunching(O.propagate(p0, mm, n), mm)

    h = 1e-4
    fd = {
        "h": (L(small(dt=0.05, qpc_h=1.0 + h), psi0) - L(small(dt=0.05, qpc_h=1.0 - h), psi0)) / (2 * h),
        "w": (L(small(dt=0.05, qpc_w=1.5 + h), psi0) - L(small(dt=0.05, qpc_w=1.5 - h), psi0)) / (2 * h),
        "delay": (L(m, state(delay + h)[2]) - L(m, state(delay - h)[2])) / (2 * h),
    }
    assert abs(loss - L(m, psi0)) < 1e-14
    for k, v in fd.items():
        assert abs(grad[k] - v) <= 1e-6 * max(abs(v), 1e-3), (k, grad[k], v)


# --- observables beyond P_b: maps and entanglement (Fig. 2, Fig. 3(b), Sec. V) --

def _orthonormal_pair(m, seed):
    """Two single-particle functions on the grid, orthonormal in sum(conj(a) b) dx dy."""
    a = W.random_state((m.nx, m.ny), seed=seed)
    b = W.random_state((m.nx, m.ny), seed=seed + 1)
    d1 = m.dx * m.dy
    a = a / math.sqrt(np.sum(np.abs(a) ** 2) * d1)
    b = b - a * (np.sum(np.conj(a) * b) * d1)
    b = b / math.sqrt(np.sum(np.abs(b) ** 2) * d1)
    return a, b


def test_marginal_and_conditional_closed_forms():
    m = small(nx=16, ny=8)
    a, b = _orthonormal_pair(m, 11)
    prod = np.einsum("ab,cd->abcd", a, b)
    # product state: particle 1 is a, particle 2 is b
    assert np.max(np.abs(O.marginal(prod, m) - np.abs(a) ** 2)) <= 1e-12 * np.max(np.abs(a) ** 2)
    cond = O.conditional(prod, 3, 5)
    assert np.max(np.abs(cond - np.abs(a) ** 2 * abs(b[3, 5]) ** 2)) <= 1e-12 * np.max(cond)
    # Slater determinant of orthonormal a, b: each particle sees (|a|^2 + |b|^2)/2
    sl = (prod - np.einsum("ab,cd->abcd", b, a)) / math.sqrt(2.0)
    mg = O.marginal(sl, m)
    assert np.max(np.abs(mg - 0.5 * (np.abs(a) ** 2 + np.abs(b) ** 2))) <= 1e-12 * np.max(mg)
    assert abs(np.sum(mg) * m.dx * m.dy - 1.0) <= 1e-12
    # Pauli: the conditional probability vanishes where particle 1 sits on particle 2
    assert O.conditional(sl, 4, 6)[4, 6] <= 1e-30


def _slice_state(m, iy1, iy2, x1r, x2r, probs, scale, seed):
    """A 4D array whose slice (x1 in x1r, y1*, x2 in x2r, y2*) is
    scale * sum_k sqrt(p_k) u_k(x1) v_k(x2) with orthonormal u_k, v_k, and
    whose every other entry is unrelated noise."""
    rng = np.random.default_rng(seed)
    psi = W.random_state((m.nx, m.ny, m.nx, m.ny), seed=seed)
    n1, n2 = x1r[1] - x1r[0], x2r[1] - x2r[0]
    u, _ = np.linalg.qr(rng.standard_normal((n1, n1)) + 1j * rng.standard_normal((n1, n1)))
    v, _ = np.linalg.qr(rng.standard_normal((n2, n2)) + 1j * rng.standard_normal((n2, n2)))
    phi = sum(math.sqrt(p) * np.outer(u[:, k], v[:, k]) for k, p in enumerate(probs))
    psi[x1r[0]:x1r[1], iy1, x2r[0]:x2r[1], iy2] = scale * phi
    return psi


@pytest.mark.parametrize("probs", [(1.0,), (0.5, 0.5), (0.5, 0.3, 0.2), (0.4, 0.3, 0.2, 0.1)])
def test_entropy_of_known_schmidt_spectra(probs):
    m = small(nx=16, ny=8)
    x1r, x2r = (2, 9), (6, 16)                        # T and B of different sizes
    psi = _slice_state(m, 2, 5, x1r, x2r, probs, scale=0.37, seed=21)
    s, weight = O.entanglement_entropy(psi, 2, 5, x1r, x2r)
    exact = -sum(p * math.log(p) for p in probs)
    assert abs(s - exact) <= 1e-12
    assert abs(weight - 0.37 ** 2) <= 1e-14
    # the same state read on other y rows has a different (generic) entropy
    s_other, _ = O.entanglement_entropy(psi, 3, 5, x1r, x2r)
    assert abs(s_other - exact) > 1e-3


def test_entropy_of_slater_slice_is_ln2():
    m = small(nx=16, ny=8)
    rng = np.random.default_rng(5)
    q, _ = np.linalg.qr(rng.standard_normal((m.nx, 2)) + 1j * rng.standard_normal((m.nx, 2)))
    u, v = q[:, 0], q[:, 1]
    psi = np.zeros((m.nx, m.ny, m.nx, m.ny), dtype=np.complex128)
    psi[:, 1, :, 1] = (np.outer(u, v) - np.outer(v, u)) / math.sqrt(2.0)
    s, _ = O.entanglement_entropy(psi, 1, 1, (0, m.nx), (0, m.nx))
    assert abs(s - math.log(2.0)) <= 1e-12


# --- the paper's barrier family and numerical edge states (R10, R11) ---------

def test_fermi_function_closed_forms():
    tau = 0.7
    assert abs(O.fermi(0.0, tau) - 0.5) <= 1e-15
    assert abs(O.fermi(tau * math.log(3.0), tau) - 0.25) <= 1e-15      # tau is a length
    u = np.linspace(-9, 9, 37)
    assert np.max(np.abs(O.fermi(u, tau) + O.fermi(-u, tau) - 1.0)) <= 1e-15
    assert O.fermi(-50.0, tau) == pytest.approx(1.0) and O.fermi(50.0, tau) < 1e-30


def test_barrier_blocks_of_pot_xy():
    m = O.Model(nx=64, ny=32, dx=0.25, dy=0.25, omega=0.0, qpc_h=0.0, fermi_vb=3.0, fermi_tau=0.1,
                fermi_xa=-1.0, fermi_ya=-0.5, fermi_xb=1.5, fermi_yb=1.0)
    v = O.v1(m)
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)
    ix = lambda val: int(np.argmin(np.abs(x - val)))
    iy = lambda val: int(np.argmin(np.abs(y - val)))
    assert v[ix(-6.0), iy(-3.75)] == pytest.approx(3.0, rel=1e-9)         # inside block A
    assert v[ix(6.0), iy(3.75)] == pytest.approx(3.0, rel=1e-9)           # inside block B
    assert v[ix(-6.0), iy(3.75)] < 1e-9 and v[ix(6.0), iy(-3.75)] < 1e-9    # open quadrants
    assert v[ix(0.25), iy(0.25)] < 1e-3                                   # the QPC gap
    # a corner of a block sits at a quarter of the height
    m2 = O.Model(nx=16, ny=16, dx=0.5, dy=0.5, omega=0.0, qpc_h=0.0, fermi_vb=2.0, fermi_tau=0.3,
                 fermi_xa=O.coords(16, 0.5)[5], fermi_ya=O.coords(16, 0.5)[7], fermi_xb=99.0, fermi_yb=99.0)
    assert O.v1(m2)[5, 7] == pytest.approx(0.5, rel=1e-12)


@pytest.mark.parametrize("k", [-1.5, 0.0, 2.0])
def test_numerical_edge_state_matches_closed_form(k):
    m = O.Model(nx=32, ny=64, dx=0.5, dy=0.25, B=1.0, omega=1.0)
    e, phi = O.edge_state_numeric(m, k)
    om = math.sqrt(2.0)
    assert abs(e - (0.5 * om + k * k / (2 * om ** 2))) <= 1e-12
    y = O.coords(m.ny, m.dy)
    chi = (om / math.pi) ** 0.25 * np.exp(-0.5 * om * (y - k / om ** 2) ** 2)
    assert np.max(np.abs(phi - chi)) <= 1e-10


def test_numerical_edge_state_pure_landau_level():
    m = O.Model(nx=32, ny=64, dx=0.5, dy=0.25, B=1.5, omega=0.0)
    for k in (-2.0, 0.5, 3.0):                                            # centre k/B inside the box
        assert abs(O.edge_state_numeric(m, k)[0] - 0.75) <= 1e-11       # B/2


def test_wall_side_convention():
    m = O.Model(nx=32, ny=64, dx=0.5, dy=0.25, B=1.0, omega=1.0, fermi_vb=5.0, fermi_tau=0.2)
    k = 2.0                                                               # centre y_k = 1
    om = math.sqrt(2.0)
    free = 0.5 * om + k * k / 4.0
    y = O.coords(m.ny, m.dy)
    chi = (om / math.pi) ** 0.25 * np.exp(-0.5 * om * (y - k / om ** 2) ** 2)
    # first-order shift of the closed-form level by the smooth tail of a wall
    # at y = -3: exp(-(y + 3)/tau) reaches the state; the second-order
    # remainder is a few 1e-10, three orders below the shift itself
    tail = float(np.sum(chi ** 2 * 5.0 / (np.exp((y + 3.0) / 0.2) + 1.0)) * m.dy)
    assert 1e-7 < tail < 1e-5
    # barrier below y = -3: the level rises by the tail only
    assert abs(O.edge_state_numeric(m, k, wall_y=-3.0, wall_side=1)[0] - (free + tail)) <= 2e-9
    # the same wall facing up covers the state: V_b minus the same tail
    assert abs(O.edge_state_numeric(m, k, wall_y=-3.0, wall_side=-1)[0] - (free + 5.0 - tail)) <= 2e-9
    # a wall through the state pushes the level up (variational bound)
    assert O.edge_state_numeric(m, k, wall_y=1.0, wall_side=1)[0] > free + 0.05


def test_numerical_packet_without_wall_is_the_closed_form_packet():
    m = O.Model(nx=32, ny=64, dx=0.5, dy=0.25, B=1.0, omega=1.0)
    a = O.edge_packet(m, -2.0, 1.3, 1.1)
    b = O.edge_packet_numeric(m, -2.0, 1.3, 1.1)
    assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(a))


# --- R3: the Gaussian saddle standing in for the QPC, by value and moments ---

def test_qpc_saddle_height_and_width_by_value():
    # cell-centred grid x_j = (j - 7.5) * 0.5: x0 = 0.25 is x_8, and x0 -+ w with
    # w = 1 are x_6 and x_10.  With omega = 0 the potential is the saddle alone.
    h, w, x0 = 1.3, 1.0, 0.25
    m = O.Model(nx=16, ny=16, dx=0.5, dy=0.5, omega=0.0, lam=0.0, qpc_h=h, qpc_w=w, qpc_x0=x0)
    x = O.coords(m.nx, m.dx)
    assert x[8] == x0 and x[6] == x0 - w and x[10] == x0 + w
    v = O.v1(m)
    assert np.max(np.abs(v - v[:, :1])) == 0.0                # no y dependence without confinement
    assert abs(v[8, 0] - h) <= 1e-15                           # the height at the centre
    # w is the standard deviation: one width away the saddle is down by e^{-1/2}
    for j in (6, 10):
        assert abs(v[j, 0] - h * math.exp(-0.5)) <= 1e-15
    assert abs(v[0, 0] - h * math.exp(-0.5 * ((x[0] - x0) / w) ** 2)) <= 1e-15 * h
    assert v[0, 0] < 1e-3 * h                                   # far away: nothing left


def test_qpc_saddle_moments_on_a_fine_grid():
    # integral h w sqrt(2 pi), mean x0 and variance w^2 of the saddle profile:
    # the moments that make w a standard deviation and h a height
    h, w, x0 = 0.8, 0.9, 0.37
    m = O.Model(nx=1024, ny=16, dx=0.02, dy=0.5, omega=0.0, lam=0.0, qpc_h=h, qpc_w=w, qpc_x0=x0)
    x = O.coords(m.nx, m.dx)
    v = O.v1(m)[:, 0]
    area = np.sum(v) * m.dx
    mean = np.sum(x * v) * m.dx / area
    var = np.sum((x - mean) ** 2 * v) * m.dx / area
    assert abs(area - h * w * math.sqrt(2 * math.pi)) <= 1e-12
    assert abs(mean - x0) <= 1e-12
    assert abs(var - w * w) <= 1e-12


def test_qpc_saddle_expectation_of_gaussian_packets():
    # <V1(r1) + V1(r2)> of a product of two normalised Gaussians with x
    # densities N(mu_i, s_i^2): the Gaussian convolution
    #   E[h exp(-(X - x0)^2 / 2w^2)] = h w / sqrt(w^2 + s^2) exp(-(mu - x0)^2 / 2(w^2 + s^2)),
    # checked against scipy quad of the same expectation first
    h, w, x0 = 1.7, 0.8, 0.3
    m = O.Model(nx=128, ny=16, dx=0.125, dy=0.5, omega=0.0, lam=0.0, qpc_h=h, qpc_w=w, qpc_x0=x0)
    x = O.coords(m.nx, m.dx)
    y = O.coords(m.ny, m.dy)
    parts = [(-0.9, 0.45), (1.2, 0.6)]

    def packet(mu, s):
        phi = np.exp(-((x[:, None] - mu) ** 2) / (4 * s * s) - y[None, :] ** 2 / 2.0).astype(np.complex128)
        return phi / math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)

    psi = np.einsum("ab,cd->abcd", packet(*parts[0]), packet(*parts[1]))
    got = O.observables(psi, m)["e_pot"]
    closed = sum(h * w / math.sqrt(w * w + s * s) * math.exp(-((mu - x0) ** 2) / (2 * (w * w + s * s)))
                 for mu, s in parts)
    for mu, s in parts:
        q, _ = integrate.quad(lambda t: math.exp(-((t - mu) ** 2) / (2 * s * s)) / math.sqrt(2 * math.pi * s * s)
                              * h * math.exp(-((t - x0) ** 2) / (2 * w * w)), -np.inf, np.inf,
                              epsabs=1e-14, epsrel=1e-13)
        one = h * w / math.sqrt(w * w + s * s) * math.exp(-((mu - x0) ** 2) / (2 * (w * w + s * s)))
        assert abs(q - one) <= 1e-12
    assert abs(got - closed) <= 1e-12


def test_dv_dtheta_is_the_derivative_of_the_potential():
    m = O.Model(nx=32, ny=16, dx=0.5, dy=0.5, qpc_h=1.2, qpc_w=1.4, qpc_x0=0.3)
    eps = 1e-5

    def four_d(a):
        return a[:, :, None, None] + a[None, None, :, :]

    fd = {"h": four_d(O.v1(m, h=m.qpc_h + eps) - O.v1(m, h=m.qpc_h - eps)) / (2 * eps),
          "w": four_d(O.v1(m, w=m.qpc_w + eps) - O.v1(m, w=m.qpc_w - eps)) / (2 * eps)}
    for k, ref in fd.items():
        got = O.dv_dtheta(m, k)
        assert np.max(np.abs(got - ref)) <= 1e-9 * np.max(np.abs(ref)), k


# --- R2 and the printed product: factor order against dense exponentials ----

def _dense_factors(m):
    """T_x, T_y (sums over both particles) and V as dense Hermitian matrices on
    the 4D index (x1, y1, x2, y2), built from numpy's FFT of the identity and
    numpy's fftfreq, so that their exponentials (scipy.linalg.expm) give the
    factors of a split step with no code of the oracle but v_total."""
    nx, ny = m.nx, m.ny
    n = nx * ny
    y = (np.arange(ny) - (ny - 1) / 2.0) * m.dy
    kx = 2 * np.pi * np.fft.fftfreq(nx, d=m.dx)
    ky = 2 * np.pi * np.fft.fftfreq(ny, d=m.dy)
    Fx, Fy = np.fft.fft(np.eye(nx), axis=0), np.fft.fft(np.eye(ny), axis=0)
    t1x = np.zeros((n, n), dtype=np.complex128)
    t1y = np.zeros((n, n), dtype=np.complex128)
    for j in range(ny):
        blk = np.linalg.inv(Fx) @ np.diag(0.5 * (kx - m.B * y[j]) ** 2) @ Fx
        t1x[j::ny, j::ny] = blk
    tyb = np.linalg.inv(Fy) @ np.diag(0.5 * ky ** 2) @ Fy
    for i in range(nx):
        t1y[i * ny:(i + 1) * ny, i * ny:(i + 1) * ny] = tyb
    eye = np.eye(n)
    Tx = np.kron(t1x, eye) + np.kron(eye, t1x)
    Ty = np.kron(t1y, eye) + np.kron(eye, t1y)
    V = np.diag(O.v_total(m).reshape(-1)).astype(np.complex128)
    return Tx, Ty, V


def test_step_factor_orders_against_dense_exponentials():
    from scipy.linalg import expm
    m = O.Model(nx=8, ny=4, dx=0.6, dy=0.7, B=1.3, omega=0.9, dt=0.3, qpc_h=1.1, qpc_w=1.2,
                qpc_x0=0.2, lam=0.8, soft=0.5)
    Tx, Ty, V = _dense_factors(m)
    dt = m.dt
    E = lambda A, s: expm(-1j * s * A)
    psi = W.random_state((m.nx, m.ny, m.nx, m.ny), seed=21)
    v = psi.reshape(-1)
    strang = E(V, dt / 2) @ E(Tx, dt / 2) @ E(Ty, dt) @ E(Tx, dt / 2) @ E(V, dt / 2) @ v
    lie = E(V, dt) @ E(Ty, dt) @ E(Tx, dt) @ v             # Eq. evoloperat: T_x first, then T_y, then V
    got_s = O.strang_step(psi, m).reshape(-1)
    got_l = O.lie_step(psi, m).reshape(-1)
    scale = np.max(np.abs(v))
    assert np.max(np.abs(got_s - strang)) <= 1e-12 * scale
    assert np.max(np.abs(got_l - lie)) <= 1e-12 * scale
    # the orders are distinguishable at this dt: every other order of the
    # printed product misses by far more than the tolerance
    for other in (E(V, dt) @ E(Tx, dt) @ E(Ty, dt), E(Ty, dt) @ E(Tx, dt) @ E(V, dt),
                  E(Tx, dt) @ E(V, dt) @ E(Ty, dt)):
        assert np.max(np.abs(got_l - other @ v)) > 1e-3 * scale
