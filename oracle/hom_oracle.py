"""Plain FP64 CPU oracle of the two-electron split-step Fourier propagation.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this module: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code, header, table or helper with the CUDA library; it is written
from the paper, slowly and literally, so that a reader can check it by eye.

Paper: Bellentani, Bordone, Oriols, Bertoni, "Coulomb and exchange
interaction effects on the exact two-electron dynamics in the Hong-Ou-Mandel
interferometer based on Hall edge states" (arXiv:1903.02581).

What is followed, by passage
----------------------------
* Sec. II.C, Eq. (evoloperat) and Appendix A (Eq. 2PTB and the regrouping
  T_{x1,y1}+T_{x2,y2} = T_{x1,x2} + T_{y1,y2}): split-step Fourier propagation
  of the 4D two-particle wavefunction with 2D Fourier transforms over the axis
  pairs (x1,x2) and (y1,y2), kinetic phases diagonal in the transformed
  representation and the potential phase diagonal in real space.
* Eq. (coulomb): V12 = lambda / sqrt(|r1-r2|^2 + a^2), and its screened form
  Eq. (screenedCoulomb) with the damping exp(-|r1-r2| / sigma_c).
* Eq. (twopstate): Slater determinant of two single-particle packets.
* Eq. (singlepwp) and Eq. (H_effective): a packet is a Gaussian-weighted sum
  of edge eigenstates e^{ik x} phi_k(y) of the confined Landau problem, in
  closed form for the parabolic edge (R6) or numerically (R11).
* Eqs. (pot_x) and (pot_xy): Fermi-function barriers (R10).
* Eq. (p_bunching): bunching probability = probability that both particles
  are found on the same side of the beam splitter.
* Captions of Fig. 2 and Fig. 3(b): conditional probability
  |psi(x1,y1,x2*,y2*)|^2 and unconditional probability of particle 1,
  P(x1,y1) = integral over (x2,y2) of |psi|^2.
* Sec. V, Eq. (reduced_density) and the entropy below it: von Neumann entropy
  of a 1D slice of the two-particle state (reading R9).

Readings of the paper used here (silent, garbled or inconsistent passages)
--------------------------------------------------------------------------
R1  Axes are relabelled x<->y with respect to the paper: propagation runs
    along x and the edge confinement acts along y.  Units hbar = m* = |e| = 1.
    The magnetic kinetic term is 1/2 (k_x - B y)^2, diagonal in the mixed
    representation (k_x, y); the y kinetic term is 1/2 k_y^2, diagonal in k_y.
    (Appendix A, Eq. 2PTB; its printed "(p_y + eB x^2)/2m" is read as
    (p_y + eBx)^2/2m, which is what the expansion printed below it gives.)
R2  The time step is the symmetric (Strang) product
        S(dt) = V/2 . Fx^-1 Tx/2 Fy^-1 Ty Fy Tx/2 Fx . V/2,
    built from the same factors as Eq. (evoloperat); the paper's first-order
    order of Eq. (evoloperat) is kept as ``lie_step`` for the order test.
R3  Single-particle potential V1(x,y) = 1/2 omega^2 y^2 + h exp(-(x-x0)^2/2w^2)
    (parabolic edge confinement plus a Gaussian saddle standing in for the
    QPC of Eq. pot_xy, whose corner parameters the paper does not give).  It
    sits in the real-space phase, not in the kinetic phase.
R4  Grid: cell-centred, x_j = (j - (N-1)/2) dx; k_m = 2 pi m / (N dx) with m
    taken in [-N/2, N/2) (the Nyquist mode negative); forward DFT sums
    e^{-2 pi i j m / N}, inverse has the 1/N.  Coulomb uses plain coordinate
    differences (no minimum image).
R5  Regions of Eq. (p_bunching): "left" x < 0 and "right" x > 0.  P_b is the
    probability that x1 and x2 have the same sign.
R6  Edge packet (Eq. singlepwp with the closed-form lowest hybrid level of the
    parabolic edge): phi_k(y) = (Omega/pi)^(1/4) exp(-Omega (y - y_k)^2 / 2),
    Omega^2 = B^2 + omega^2, y_k = k B / Omega^2, E(k) = Omega/2 +
    k^2 omega^2 / (2 Omega^2); weights exp(-sigma^2 (k - k0)^2) over the grid
    wavenumbers; k0 from E(k0) = energy, sign from the direction.
R7  The combined two-particle state is renormalised numerically (the 1/sqrt2
    of Eq. twopstate assumes orthogonal packets).
R9  Spatial entanglement (Sec. V): the 1D slice phi(x1,x2) = psi(x1, y1*, x2, y2*)
    with x1 in a region T and x2 in a region B is renormalised (discrete sum of
    |phi|^2 = 1); rho_T(x1,x1') = sum_{x2 in B} phi(x1,x2) conj(phi(x1',x2)) (the
    printed phi*(x2,x1') of Eq. reduced_density is read as phi*(x1',x2), the
    only form that is a density matrix); S = -Tr rho_T ln rho_T (the printed
    formula lacks the minus sign; S >= 0 is the von Neumann entropy).
R10 Barriers of Eqs. (pot_x) and (pot_xy): F_tau(u) = 1 / (exp(u / tau) + 1)
    with tau a length (the paper quotes tau = 3 nm).  With the axes of R1 the
    QPC is two blocks, A = V_b F(x - xa) F(y - ya) (filling x < xa, y < ya)
    and B = V_b F(xb - x) F(yb - y) (filling x > xb, y > yb); the factors at
    -infinity of Eq. (pot_xy) are 1.  They add to the potential of R3.
R11 Numerical edge states (Eq. H_effective, relabelled): phi_k(y) is the
    lowest eigenvector of H_eff(k) = -1/2 d^2/dy^2 + 1/2 (k - B y)^2 +
    1/2 omega^2 y^2 + V_wall(y) on the y grid, the second derivative being the
    spectral one of the periodic grid (the operator the split step
    propagates), V_wall(y) = V_b F_tau(s (y - y_w)) the one-sided barrier of
    Eq. (pot_x) (s = +1: barrier below y_w, s = -1: above), normalised to
    sum |phi|^2 dy = 1 with its largest component positive.  The packet of
    Eq. (singlepwp) is then built as in R6 with these phi_k, from a given k0.
R8  Adjoint: the Strang product is palindromic and each factor unitary, so
    S(dt)^dagger = S(-dt); the gradient of L = <psi_N|M|psi_N> with respect
    to a potential parameter theta is
        dL/dtheta = 2 dt Im sum'_n <lambda_n| dV/dtheta |psi_n>,
    with trapezoid weights (1/2 at n = 0 and n = N), lambda_n the adjoint
    state at integer step n.

Parity pins: ``tests/test_oracle_pins.py`` checks this module against closed
forms and invariants (DFT vs numpy.fft, unitarity, exchange symmetry,
factorisation at zero Coulomb, free Gaussian spreading, Landau / hybrid level
phases, cyclotron motion, Strang/Lie convergence orders, time reversal,
energy conservation, Coulomb expectation by quadrature, packet energy,
adjoint dot-product test and finite differences, marginals and conditional
slices of product and Slater states in closed form, entropies of states with
known Schmidt coefficients, the saddle of R3 by its height, its value one
width away, its moments on a fine grid and its expectation in Gaussian
packets, dV/dtheta against differences of the potential, and the factor order
of the Strang and printed first-order steps against dense matrix
exponentials built from numpy's FFT).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

AXIS_X1, AXIS_Y1, AXIS_X2, AXIS_Y2 = 0, 1, 2, 3


@dataclasses.dataclass
class Model:
    """Physical and numerical parameters of one simulation (units hbar=m*=e=1)."""

    nx: int
    ny: int
    dx: float
    dy: float
    B: float = 1.0
    omega: float = 1.0          # parabolic edge confinement (R3)
    dt: float = 0.01
    qpc_h: float = 1.0          # saddle height (R3)
    qpc_w: float = 1.5          # saddle width, standard deviation (R3)
    qpc_x0: float = 0.0
    lam: float = 1.0            # Coulomb strength, Eq. (coulomb)
    soft: float = 0.5           # Coulomb softening (the paper's thickness d)
    screen: float = 0.0         # screening length sigma_c of Eq. (screenedCoulomb); 0: none
    fermi_vb: float = 0.0       # height V_b of the barrier blocks of Eq. (pot_xy); 0: none (R10)
    fermi_tau: float = 1.0      # smoothness tau of F_tau, a length (R10)
    fermi_xa: float = 0.0       # block A fills x < xa, y < ya
    fermi_ya: float = 0.0
    fermi_xb: float = 0.0       # block B fills x > xb, y > yb
    fermi_yb: float = 0.0

    @property
    def dV(self) -> float:
        return (self.dx * self.dy) ** 2


# ----------------------------------------------------------------------------
# Grids and discrete Fourier transform (R4)
# ----------------------------------------------------------------------------

def coords(n: int, d: float) -> np.ndarray:
    j = np.arange(n, dtype=np.float64)
    return (j - (n - 1) / 2.0) * d


def wavenumbers(n: int, d: float) -> np.ndarray:
    m = np.arange(n)
    m = np.where(m < n // 2, m, m - n).astype(np.float64)
    return 2.0 * np.pi * m / (n * d)


def dft_matrix(n: int, inverse: bool = False) -> np.ndarray:
    """Matrix [m, j] of the length-n DFT: e^{-2 pi i jm/n} (inverse: e^{+...}/n)."""
    j = np.arange(n)
    jm = np.outer(j, j) % n                      # exact integer reduction
    ang = 2.0 * np.pi * jm / n
    if inverse:
        return np.exp(1j * ang) / n
    return np.exp(-1j * ang)


def dft_axis(a: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """Apply the length-n DFT along one axis by a plain matrix product."""
    f = dft_matrix(a.shape[axis], inverse)
    out = np.tensordot(f, a, axes=([1], [axis]))
    return np.moveaxis(out, 0, axis)


def dft_pair(a: np.ndarray, axes: tuple[int, int], inverse: bool = False) -> np.ndarray:
    """2D DFT over an axis pair: the F_{x1,x2} / F_{y1,y2} of Eq. (evoloperat)."""
    return dft_axis(dft_axis(a, axes[0], inverse), axes[1], inverse)


# ----------------------------------------------------------------------------
# Operators (Appendix A with readings R1, R3; Eq. coulomb)
# ----------------------------------------------------------------------------

def fermi(u: np.ndarray, tau: float) -> np.ndarray:
    """F_tau(u) = 1 / (exp(u / tau) + 1) of Eq. (pot_x) (R10), via the
    library logistic function, which does not overflow."""
    from scipy.special import expit
    return expit(-np.asarray(u, dtype=np.float64) / tau)


def v_fermi(m: Model) -> np.ndarray:
    """The two barrier blocks of Eq. (pot_xy) on [x, y] (R10)."""
    x = coords(m.nx, m.dx)[:, None]
    y = coords(m.ny, m.dy)[None, :]
    t = m.fermi_tau
    return m.fermi_vb * (fermi(x - m.fermi_xa, t) * fermi(y - m.fermi_ya, t)
                         + fermi(m.fermi_xb - x, t) * fermi(m.fermi_yb - y, t))


def v1(m: Model, h: float | None = None, w: float | None = None) -> np.ndarray:
    """Single-particle potential V1[x, y] (R3, plus the blocks of R10)."""
    h = m.qpc_h if h is None else h
    w = m.qpc_w if w is None else w
    x = coords(m.nx, m.dx)[:, None]
    y = coords(m.ny, m.dy)[None, :]
    v = 0.5 * m.omega ** 2 * y ** 2 + h * np.exp(-((x - m.qpc_x0) ** 2) / (2.0 * w ** 2))
    if m.fermi_vb != 0.0:
        v = v + v_fermi(m)
    return v


def v12(m: Model, lam: float | None = None) -> np.ndarray:
    """Coulomb interaction V12[x1, y1, x2, y2], Eq. (coulomb) with thickness a;
    with m.screen = sigma_c > 0 the exponential damping exp(-|r1 - r2| / sigma_c)
    of Eq. (screenedCoulomb), whose exponent has no thickness term."""
    lam = m.lam if lam is None else lam
    x = coords(m.nx, m.dx)
    y = coords(m.ny, m.dy)
    ddx = x[:, None, None, None] - x[None, None, :, None]
    ddy = y[None, :, None, None] - y[None, None, None, :]
    r2 = ddx ** 2 + ddy ** 2
    v = lam / np.sqrt(r2 + m.soft ** 2)
    if m.screen > 0.0:
        v = v * np.exp(-np.sqrt(r2) / m.screen)
    return v


def v_total(m: Model, h=None, w=None, lam=None) -> np.ndarray:
    """V1(r1) + V1(r2) + V12(r1, r2) on the 4D real-space grid."""
    a = v1(m, h, w)
    return a[:, :, None, None] + a[None, None, :, :] + v12(m, lam)


def tx_single(m: Model) -> np.ndarray:
    """1/2 (k_x - B y)^2 on [k_x, y] (R1)."""
    k = wavenumbers(m.nx, m.dx)[:, None]
    y = coords(m.ny, m.dy)[None, :]
    return 0.5 * (k - m.B * y) ** 2


def ty_single(m: Model) -> np.ndarray:
    """1/2 k_y^2 on [k_y]."""
    return 0.5 * wavenumbers(m.ny, m.dy) ** 2


def tx_total(m: Model) -> np.ndarray:
    """T_{x1,x2} on the mixed representation [k_x1, y1, k_x2, y2]."""
    t = tx_single(m)
    return t[:, :, None, None] + t[None, None, :, :]


def ty_total(m: Model) -> np.ndarray:
    """T_{y1,y2} on [., k_y1, ., k_y2] (broadcast over the x axes)."""
    t = ty_single(m)
    return t[None, :, None, None] + t[None, None, None, :]


# ----------------------------------------------------------------------------
# Time step (Eq. evoloperat, Appendix A; R2)
# ----------------------------------------------------------------------------

def strang_phases(m: Model, dt: float | None = None,
                  vtot: np.ndarray | None = None) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """The three diagonal factors of one Strang step as arrays:
    e^{-i V dt/2} (real space), e^{-i T_x dt/2} (k_x, y) and e^{-i T_y dt} (k_y).
    They are the same every step, so a long run may compute them once."""
    dt = m.dt if dt is None else dt
    V = v_total(m) if vtot is None else vtot
    return (np.exp(-0.5j * dt * V), np.exp(-0.5j * dt * tx_total(m)), np.exp(-1j * dt * ty_total(m)))


def strang_step(psi: np.ndarray, m: Model, dt: float | None = None,
                vtot: np.ndarray | None = None, phases=None) -> np.ndarray:
    """One symmetric split step, factor by factor, right to left."""
    pv, ptx, pty = strang_phases(m, dt, vtot) if phases is None else phases
    X, Y = (AXIS_X1, AXIS_X2), (AXIS_Y1, AXIS_Y2)
    psi = pv * psi                                      # e^{-i V dt/2}      (real space)
    psi = dft_pair(psi, X)                              # F_{x1,x2}: -> (k_x, y)
    psi = ptx * psi                                     # e^{-i T_x dt/2}
    psi = dft_pair(psi, Y)                              # F_{y1,y2}: -> (k_x, k_y)
    psi = pty * psi                                     # e^{-i T_y dt}
    psi = dft_pair(psi, Y, inverse=True)                # F^-1_{y1,y2}
    psi = ptx * psi                                     # e^{-i T_x dt/2}
    psi = dft_pair(psi, X, inverse=True)                # F^-1_{x1,x2}: -> real space
    psi = pv * psi                                      # e^{-i V dt/2}
    return psi


def lie_step(psi: np.ndarray, m: Model, dt: float | None = None,
             vtot: np.ndarray | None = None) -> np.ndarray:
    """The first-order product exactly as printed in Eq. (evoloperat)."""
    dt = m.dt if dt is None else dt
    V = v_total(m) if vtot is None else vtot
    X, Y = (AXIS_X1, AXIS_X2), (AXIS_Y1, AXIS_Y2)
    psi = dft_pair(psi, X)
    psi = np.exp(-1j * dt * tx_total(m)) * psi
    psi = dft_pair(psi, X, inverse=True)
    psi = dft_pair(psi, Y)
    psi = np.exp(-1j * dt * ty_total(m)) * psi
    psi = dft_pair(psi, Y, inverse=True)
    psi = np.exp(-1j * dt * V) * psi
    return psi


def propagate(psi: np.ndarray, m: Model, nsteps: int, order: str = "strang",
              dt: float | None = None) -> np.ndarray:
    V = v_total(m)
    if order == "strang":
        ph = strang_phases(m, dt, V)
        for _ in range(nsteps):
            psi = strang_step(psi, m, dt, phases=ph)
        return psi
    for _ in range(nsteps):
        psi = lie_step(psi, m, dt, vtot=V)
    return psi


# ----------------------------------------------------------------------------
# Single-particle 2D propagation (used only by the zero-Coulomb factorisation
# pin and by sampled checks of large product states)
# ----------------------------------------------------------------------------

def strang_step_2d(phi: np.ndarray, m: Model, dt: float | None = None) -> np.ndarray:
    """The one-particle restriction of ``strang_step`` on phi[x, y]."""
    dt = m.dt if dt is None else dt
    V = v1(m)
    phi = np.exp(-0.5j * dt * V) * phi
    phi = dft_axis(phi, 0)
    phi = np.exp(-0.5j * dt * tx_single(m)) * phi
    phi = dft_axis(phi, 1)
    phi = np.exp(-1j * dt * ty_single(m))[None, :] * phi
    phi = dft_axis(phi, 1, inverse=True)
    phi = np.exp(-0.5j * dt * tx_single(m)) * phi
    phi = dft_axis(phi, 0, inverse=True)
    phi = np.exp(-0.5j * dt * V) * phi
    return phi


def propagate_2d(phi: np.ndarray, m: Model, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        phi = strang_step_2d(phi, m)
    return phi


# ----------------------------------------------------------------------------
# Initial state (Eq. singlepwp, Eq. H_effective, Eq. twopstate; R6, R7)
# ----------------------------------------------------------------------------

def hybrid_omega(B: float, omega: float) -> float:
    return math.sqrt(B * B + omega * omega)


def k0_from_energy(energy: float, B: float, omega: float, direction: int) -> float:
    """Solve E(k0) = energy for the lowest hybrid level (R6)."""
    om = hybrid_omega(B, omega)
    if omega <= 0.0 or energy < 0.5 * om:
        raise ValueError("energy below the lowest level, or no confinement")
    return float(np.sign(direction)) * om * math.sqrt(2.0 * (energy - 0.5 * om)) / omega


def edge_packet(m: Model, x0: float, sigma: float, k0: float,
                normalise: bool = True) -> np.ndarray:
    """Gaussian packet of lowest-level edge states on the grid, phi[x, y] (R6)."""
    x = coords(m.nx, m.dx)
    y = coords(m.ny, m.dy)
    k = wavenumbers(m.nx, m.dx)
    om = hybrid_omega(m.B, m.omega)
    yk = k * m.B / om ** 2
    chi = (om / np.pi) ** 0.25 * np.exp(-0.5 * om * (y[None, :] - yk[:, None]) ** 2)   # [k, y]
    wk = np.exp(-(sigma ** 2) * (k - k0) ** 2)                                          # [k]
    plane = np.exp(1j * np.outer(x - x0, k))                                            # [x, k]
    phi = plane @ (wk[:, None] * chi)                                                   # [x, y]
    if normalise:
        phi = phi / math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)
    return phi


def edge_packet_dx0(m: Model, x0: float, sigma: float, k0: float) -> np.ndarray:
    """d(edge_packet)/d(x0) of the normalised packet (the norm does not depend on x0)."""
    x = coords(m.nx, m.dx)
    y = coords(m.ny, m.dy)
    k = wavenumbers(m.nx, m.dx)
    om = hybrid_omega(m.B, m.omega)
    yk = k * m.B / om ** 2
    chi = (om / np.pi) ** 0.25 * np.exp(-0.5 * om * (y[None, :] - yk[:, None]) ** 2)
    wk = np.exp(-(sigma ** 2) * (k - k0) ** 2)
    plane = np.exp(1j * np.outer(x - x0, k))
    phi = plane @ (wk[:, None] * chi)
    dphi = plane @ ((-1j * k * wk)[:, None] * chi)
    nrm = math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)
    return dphi / nrm


def edge_hamiltonian(m: Model, k: float, wall_y: float = 0.0, wall_side: int = 1) -> np.ndarray:
    """H_eff(k) on the y grid (R11), a real symmetric ny x ny matrix."""
    y = coords(m.ny, m.dy)
    ky = wavenumbers(m.ny, m.dy)
    t = dft_matrix(m.ny, inverse=True) @ np.diag(0.5 * ky ** 2) @ dft_matrix(m.ny)
    t = np.real(0.5 * (t + t.conj().T))
    diag = 0.5 * (k - m.B * y) ** 2 + 0.5 * m.omega ** 2 * y ** 2
    if m.fermi_vb != 0.0:
        diag = diag + m.fermi_vb * fermi(wall_side * (y - wall_y), m.fermi_tau)
    return t + np.diag(diag)


def edge_state_numeric(m: Model, k: float, wall_y: float = 0.0, wall_side: int = 1) -> tuple[float, np.ndarray]:
    """Lowest eigenpair of H_eff(k) by numpy.linalg.eigh (R11)."""
    e, v = np.linalg.eigh(edge_hamiltonian(m, k, wall_y, wall_side))
    phi = v[:, 0] / math.sqrt(np.sum(v[:, 0] ** 2) * m.dy)
    if phi[np.argmax(np.abs(phi))] < 0:
        phi = -phi
    return float(e[0]), phi


def edge_packet_numeric(m: Model, x0: float, sigma: float, k0: float,
                        wall_y: float = 0.0, wall_side: int = 1) -> np.ndarray:
    """Packet of Eq. (singlepwp) from numerical edge states (R11): weights
    exp(-sigma^2 (k - k0)^2) over the grid wavenumbers, normalised.  Modes
    whose weight is below 1e-300 are left out, as they cannot contribute."""
    x = coords(m.nx, m.dx)
    k = wavenumbers(m.nx, m.dx)
    wk = np.exp(-(sigma ** 2) * (k - k0) ** 2)
    chi = np.zeros((m.nx, m.ny))
    for i in range(m.nx):
        if wk[i] >= 1e-300:
            chi[i] = edge_state_numeric(m, float(k[i]), wall_y, wall_side)[1]
    plane = np.exp(1j * np.outer(x - x0, k))
    phi = plane @ (wk[:, None] * chi)
    return phi / math.sqrt(np.sum(np.abs(phi) ** 2) * m.dx * m.dy)


def two_particle(alpha: np.ndarray, beta: np.ndarray, exch: int, dV: float) -> np.ndarray:
    """psi[x1,y1,x2,y2] = alpha(r1) beta(r2) + exch * beta(r1) alpha(r2), renormalised.

    exch = -1 is the Slater determinant of Eq. (twopstate); +1 the symmetric
    combination; 0 the product (distinguishable) state.
    """
    psi = np.einsum("ab,cd->abcd", alpha, beta)
    if exch != 0:
        psi = psi + exch * np.einsum("ab,cd->abcd", beta, alpha)
    return psi / math.sqrt(np.sum(np.abs(psi) ** 2) * dV)


# ----------------------------------------------------------------------------
# Observables (Eq. p_bunching; energy terms of the Hamiltonian of Sec. II.C)
# ----------------------------------------------------------------------------

def same_side_mask(m: Model) -> np.ndarray:
    """Indicator of x1, x2 on the same side of the beam splitter (R5), 4D-broadcast."""
    left = coords(m.nx, m.dx) < 0.0
    same = left[:, None] == left[None, :]
    return same[:, None, :, None].astype(np.float64)


def observables(psi: np.ndarray, m: Model) -> dict:
    """norm, energy, e_kin, e_pot (V1+V2), e_coul (V12), p_bunch."""
    dV = m.dV
    rho = np.abs(psi) ** 2
    norm = float(np.sum(rho) * dV)
    a = v1(m)
    e_pot = float(np.sum(rho * (a[:, :, None, None] + a[None, None, :, :])) * dV)
    e_coul = float(np.sum(rho * v12(m)) * dV)
    p_b = float(np.sum(rho * same_side_mask(m)) * dV)
    psi_m = dft_pair(psi, (AXIS_X1, AXIS_X2))                 # (k_x, y), Parseval 1/Nx^2
    e_tx = float(np.sum(np.abs(psi_m) ** 2 * tx_total(m)) * dV / m.nx ** 2)
    psi_k = dft_pair(psi_m, (AXIS_Y1, AXIS_Y2))               # (k_x, k_y), 1/(Nx Ny)^2
    e_ty = float(np.sum(np.abs(psi_k) ** 2 * ty_total(m)) * dV / (m.nx * m.ny) ** 2)
    e_kin = e_tx + e_ty
    return dict(norm=norm, energy=e_kin + e_pot + e_coul, e_kin=e_kin,
                e_pot=e_pot, e_coul=e_coul, p_bunch=p_b)


def energy_2d(phi: np.ndarray, m: Model) -> float:
    """Single-particle <1/2 (k_x - B y)^2 + 1/2 k_y^2 + V1> of phi[x, y] (Parseval)."""
    w = np.sum(np.abs(phi) ** 2)
    pm = dft_axis(phi, 0)
    e_tx = np.sum(np.abs(pm) ** 2 * tx_single(m)) / m.nx
    pk = dft_axis(phi, 1)
    e_ty = np.sum(np.abs(pk) ** 2 * ty_single(m)[None, :]) / m.ny
    e_v = np.sum(np.abs(phi) ** 2 * v1(m))
    return float((e_tx + e_ty + e_v) / w)


def bunching(psi: np.ndarray, m: Model) -> float:
    return float(np.sum(np.abs(psi) ** 2 * same_side_mask(m)) * m.dV)


# ----------------------------------------------------------------------------
# Adjoint gradient of the final bunching probability (R8)
# ----------------------------------------------------------------------------

def dv_dtheta(m: Model, which: str) -> np.ndarray:
    """d V / d theta on the 4D grid for theta in {h, w} (R3)."""
    x = coords(m.nx, m.dx)
    g = np.exp(-((x - m.qpc_x0) ** 2) / (2.0 * m.qpc_w ** 2))
    if which == "h":
        d1 = g
    elif which == "w":
        d1 = m.qpc_h * g * (x - m.qpc_x0) ** 2 / m.qpc_w ** 3
    else:
        raise ValueError(which)
    d1 = np.broadcast_to(d1[:, None], (m.nx, m.ny))
    return d1[:, :, None, None] + d1[None, None, :, :]


def loss_and_gradient(psi0: np.ndarray, dpsi0_ddelay: np.ndarray | None,
                      m: Model, nsteps: int) -> tuple[float, dict]:
    """L = P_b(psi_N) and dL/d(h, w[, delay]) by the adjoint of R8, all states kept."""
    V = v_total(m)
    states = [psi0]
    for _ in range(nsteps):
        states.append(strang_step(states[-1], m, vtot=V))
    mask = same_side_mask(m)
    loss = float(np.sum(np.abs(states[-1]) ** 2 * mask) * m.dV)
    lam = mask * states[-1]                                   # lambda_N = M psi_N
    dvs = {k: dv_dtheta(m, k) for k in ("h", "w")}
    acc = {k: 0.0 for k in dvs}
    for n in range(nsteps, -1, -1):
        wgt = 0.5 if n in (0, nsteps) else 1.0
        for k, dv in dvs.items():
            acc[k] += wgt * float(np.imag(np.sum(np.conj(lam) * dv * states[n])))
        if n > 0:
            lam = strang_step(lam, m, dt=-m.dt, vtot=V)       # S(dt)^dagger = S(-dt)
    grad = {k: 2.0 * m.dt * v * m.dV for k, v in acc.items()}
    if dpsi0_ddelay is not None:
        grad["delay"] = 2.0 * float(np.real(np.sum(np.conj(lam) * dpsi0_ddelay))) * m.dV
    return loss, grad


def slater_dstate(alpha: np.ndarray, beta: np.ndarray, dbeta: np.ndarray,
                  exch: int, dV: float) -> np.ndarray:
    """d/d(beta centre) of ``two_particle(alpha, beta, exch)`` including the norm."""
    u = np.einsum("ab,cd->abcd", alpha, beta)
    du = np.einsum("ab,cd->abcd", alpha, dbeta)
    if exch != 0:
        u = u + exch * np.einsum("ab,cd->abcd", beta, alpha)
        du = du + exch * np.einsum("ab,cd->abcd", dbeta, alpha)
    nn = np.sum(np.abs(u) ** 2) * dV
    dnn = 2.0 * np.real(np.sum(np.conj(u) * du)) * dV
    c = 1.0 / math.sqrt(nn)
    dc = -0.5 * c * dnn / nn
    return dc * u + c * du


# ----------------------------------------------------------------------------
# Observables beyond P_b: maps and entanglement (Fig. 2, Fig. 3(b), Sec. V)
# ----------------------------------------------------------------------------

def marginal(psi: np.ndarray, m: Model) -> np.ndarray:
    """Unconditional probability density of particle 1, P(x1, y1) = sum over
    (x2, y2) of |psi|^2 dx dy (caption of Fig. 3(b)); integrates to the norm."""
    return np.sum(np.abs(psi) ** 2, axis=(AXIS_X2, AXIS_Y2)) * m.dx * m.dy


def conditional(psi: np.ndarray, ix2: int, iy2: int) -> np.ndarray:
    """Conditional probability |psi(x1, y1, x2*, y2*)|^2 at the grid point
    (ix2, iy2) of particle 2 (caption of Fig. 2), unnormalised."""
    return np.abs(psi[:, :, ix2, iy2]) ** 2


def entanglement_entropy(psi: np.ndarray, iy1: int, iy2: int,
                         x1_range: tuple[int, int], x2_range: tuple[int, int]) -> tuple[float, float]:
    """Von Neumann entropy of the slice phi(x1, x2) = psi(x1, y1*, x2, y2*),
    x1 in the index range x1_range (region T), x2 in x2_range (region B), as
    in Sec. V with reading R9.  Returns (S, sum |phi|^2 before renormalising).
    The eigenvalues of the Hermitian rho_T come from numpy.linalg.eigvalsh;
    rounding leaves some at -1e-17, which count as 0 (0 ln 0 = 0)."""
    a0, a1 = x1_range
    b0, b1 = x2_range
    phi = psi[a0:a1, iy1, b0:b1, iy2]
    weight = float(np.sum(np.abs(phi) ** 2))
    phi = phi / math.sqrt(weight)
    rho = phi @ np.conj(phi).T                       # rho_T(x1, x1') = sum_x2 phi(x1,x2) phi*(x1',x2)
    lam = np.linalg.eigvalsh(rho)
    lam = lam[lam > 0.0]
    return float(-np.sum(lam * np.log(lam))), weight
