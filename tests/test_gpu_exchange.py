"""Exchange symmetry and the Hong-Ou-Mandel dip of the whole propagation on
the GPU, through a full scattering event at the saddle.

The Hamiltonian and the bunching mask are symmetric under the swap of the
particles, so for the antisymmetrised (-), symmetrised (+) and product
states built from the same two normalised packets (Eq. twopstate),

    (1 + |s|^2) P_+ + (1 - |s|^2) P_- = 2 P_prod,     s = <alpha|beta>,

at every time, P being the bunching probability (Eq. p_bunching) of each
renormalised state.  A kernel that treated the two particles differently, or
an exchange sign applied wrongly, breaks it.  Checked in complex128 on a
64 x 32 grid per electron, with and without Coulomb, at two delays.

Without interaction the antisymmetric state shows the Hong-Ou-Mandel dip and
the symmetric one the peak (Sec. IV), and a sweep of the delay follows the
1D scattering model of Eq. bunching, which the paper fits to its own
simulations; wider packets antibunch more, Coulomb repulsion adds its own
antibunching (Sec. III), and the entanglement between the output arms
follows the trends of Sec. V.  Those runs use a 256 x 32 grid (dx = dy = 0.5:
a 128 x 16 box) in complex64, packets of energy 2.5 and width 1.5 (1 to 3
for the width scan) started at x = -(x_s - delay/2) and x_s + delay/2 (beta
travels `delay` further; x_s = 15, more for wider packets, so that they start
clear of the saddle, which has width 1.5, and the delay changes only the
arrival times: a single packet is transmitted with probability 0.5093 from
every start used), a saddle of height 1.85, and stop at t = 26, when the
packets have left the saddle (P_b changes by less than 3e-4 after that) and
none has come near the periodic edge."""

import numpy as np
import pytest

from oracle import adapter as A
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _binding():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding as H
    from paper_1903_02581_gb300 import build

    build.build()
    return H


def _run(w, keys, make, extra=None):
    H = _binding()
    w["sims"] = [make(*k) for k in keys]
    w["batch"] = len(keys)
    pr = H.Propagator(w)
    pr.step(round(w["t_end"] / w["dt"]))
    obs = pr.observables()
    if extra is not None:
        for b, o in enumerate(obs):
            o.update(extra(pr, b))
    pr.close()
    return w, obs


def _arm_entropy(pr, b):
    """Von Neumann entropy (Sec. V) of the slice that joins the two output
    arms: x1 > 0 on the right-moving edge (y1 = +1.25) and x2 < 0 on the
    left-moving edge (y2 = -1.25), for the 256 x 32 grid below."""
    s, weight = pr.entanglement(b, 18, 13, (128, 256), (0, 128))
    return {"entropy": s, "arm_weight": weight}


@pytest.fixture(scope="module")
def identity_runs():
    w = W.sweep32(prec="c128")
    w.update(nx=64, ny=32, dx=0.5, dy=0.5, dt=0.01, t_end=9.0)

    def make(lam, delay, exch):
        return dict(qpc_h=2.25, qpc_w=1.5, lam=lam, exch=exch,
                    alpha=W.packet(-3.0, 1.5, 2.5, +1), beta=W.packet(3.0 + delay, 1.5, 2.5, -1))

    keys = [(lam, delay, exch) for lam in (1.0, 0.0) for delay in (0.0, 4.0) for exch in (-1, 0, 1)]
    w, obs = _run(w, keys, make)
    out = {}
    for k, o, s in zip(keys, obs, w["sims"]):
        assert abs(o["norm"] - 1.0) < 1e-11
        m, a, b = A.packets(w, s)
        out[k] = (o["p_bunch"], abs(np.vdot(a.ravel(), b.ravel()) * m.dx * m.dy) ** 2)
    return out


@pytest.mark.parametrize("lam,delay", [(1.0, 0.0), (1.0, 4.0), (0.0, 0.0), (0.0, 4.0)])
def test_exchange_sum_identity(identity_runs, lam, delay):
    pm, s2 = identity_runs[(lam, delay, -1)]
    p0, _ = identity_runs[(lam, delay, 0)]
    pp, _ = identity_runs[(lam, delay, 1)]
    assert abs((1 + s2) * pp + (1 - s2) * pm - 2 * p0) <= 1e-11, (pm, p0, pp, s2)


SWEEP = (0.0, 1.0, 2.0, 3.0, 4.0, 6.0, 8.0)
SIGMAS = (1.0, 1.5, 2.0, 2.5, 3.0)


@pytest.fixture(scope="module")
def hom_batch():
    """One batch of 28 simulations, keyed (sigma, delay, exch, lam): their
    stationary P_b and the entropy of their output-arm slice."""
    w = W.sweep32(prec="c64")
    w.update(nx=256, ny=32, dx=0.5, dy=0.5, dt=0.01, t_end=26.0)

    def make(sigma, delay, exch, lam):
        xs = 15.0 + 3.0 * max(0.0, sigma - 1.5)   # wider packets start further out
        return dict(qpc_h=1.85, qpc_w=1.5, lam=lam, exch=exch,
                    alpha=W.packet(-xs + delay / 2, sigma, 2.5, +1), beta=W.packet(xs + delay / 2, sigma, 2.5, -1))

    keys = [(1.5, d, -1, 0.0) for d in SWEEP] + [(1.5, 0.0, 1, 0.0), (1.5, 8.0, 1, 0.0), (1.5, 8.0, 0, 0.0)]
    keys += [(s, 0.0, 0, 0.0) for s in SIGMAS] + [(s, 0.0, -1, 0.0) for s in SIGMAS if s != 1.5]
    keys += [(1.5, d, -1, 1.0) for d in SWEEP] + [(1.5, 0.0, 0, 1.0), (1.5, 8.0, 0, 1.0)]
    _, obs = _run(w, keys, make, extra=_arm_entropy)
    return ({k: o["p_bunch"] / o["norm"] for k, o in zip(keys, obs)},
            {k: o["entropy"] for k, o in zip(keys, obs)})


@pytest.fixture(scope="module")
def hom_runs(hom_batch):
    return hom_batch[0]


@pytest.fixture(scope="module")
def arm_entropy(hom_batch):
    return hom_batch[1]


def test_hong_ou_mandel_dip_and_peak(hom_runs):
    anti0, sym0, prod0 = hom_runs[(1.5, 0.0, -1, 0.0)], hom_runs[(1.5, 0.0, 1, 0.0)], hom_runs[(1.5, 0.0, 0, 0.0)]
    antid, symd, prodd = hom_runs[(1.5, 8.0, -1, 0.0)], hom_runs[(1.5, 8.0, 1, 0.0)], hom_runs[(1.5, 8.0, 0, 0.0)]
    print("P_b: antisymmetric", anti0, antid, "symmetric", sym0, symd, "product", prod0, prodd)
    assert 0.4 < prod0 < 0.6                       # the saddle splits the packets about evenly
    assert abs(prod0 - prodd) < 1e-3               # distinguishable: the delay does not matter
    assert anti0 < antid - 0.01                    # dip
    assert sym0 > symd + 0.01                      # peak
    assert anti0 < prod0 < sym0


def test_delay_sweep_follows_the_1d_model(hom_runs):
    """The antisymmetric sweep fitted with Eq. bunching, as the paper fits its
    simulations: the dip fills in monotonically with the delay, the fit
    leaves residuals of a few percent of the dip depth, and the fitted packet
    width is within 20 % of the width the packets were built with (1.5; the
    model's width is the same standard deviation of |psi|^2 along the edge)."""
    from paper_1903_02581_gb300 import analysis as AN

    d = np.array(SWEEP)
    pb = np.array([hom_runs[(1.5, x, -1, 0.0)] for x in SWEEP])
    sigma, a = AN.fit_bunching_1d(d, pb, sigma0=1.5, a0=5.0)
    fit = AN.bunching_1d(d, sigma, a)
    depth = 0.5 - pb[0]
    print("P_b(delay):", pb, "fit sigma, a:", sigma, a, "residuals:", pb - fit)
    assert np.all(np.diff(pb) > 0)
    assert depth > 0.03
    assert np.max(np.abs(pb - fit)) <= 0.05 * depth
    assert 1.2 < sigma < 1.8


def test_bunching_falls_with_packet_width(hom_runs):
    """Sec. III(A): without interaction the antisymmetric state's stationary
    P_b decreases about linearly as the packets get wider (full antibunching
    is the plane-wave limit), while the product state stays at the classical
    value 2 T (1 - T), here 1/2."""
    anti = np.array([hom_runs[(s, 0.0, -1, 0.0)] for s in SIGMAS])
    prod = np.array([hom_runs[(s, 0.0, 0, 0.0)] for s in SIGMAS])
    print("P_b(sigma): antisymmetric", anti, "product", prod)
    assert np.all(np.abs(prod - 0.5) < 2e-3)
    slope = np.diff(anti)
    assert np.all(slope < -0.02)
    assert np.max(np.abs(np.diff(slope))) < 0.25 * np.mean(np.abs(slope))


def test_coulomb_antibunching_and_effective_parameters(hom_runs):
    """Sec. III(B): Coulomb repulsion alone antibunches a product state (P_b
    below 1/2, less so when the delay keeps the packets apart, and not down to
    0 in 2D); with exchange as well, P_b is shifted lower still; and a fit of
    Eq. bunching to the interacting delay sweep needs an effective width and
    range larger than the non-interacting ones."""
    from paper_1903_02581_gb300 import analysis as AN

    prod0, prodd = hom_runs[(1.5, 0.0, 0, 1.0)], hom_runs[(1.5, 8.0, 0, 1.0)]
    anti0 = hom_runs[(1.5, 0.0, -1, 1.0)]
    free_anti0 = hom_runs[(1.5, 0.0, -1, 0.0)]
    print("Coulomb: product", prod0, prodd, "antisymmetric", anti0, "(no Coulomb", free_anti0, ")")
    assert 0.1 < prod0 < prodd < 0.5 - 0.02
    assert anti0 < prod0 and anti0 < free_anti0
    d = np.array(SWEEP)
    pb_int = np.array([hom_runs[(1.5, x, -1, 1.0)] for x in SWEEP])
    pb_free = np.array([hom_runs[(1.5, x, -1, 0.0)] for x in SWEEP])
    assert np.all(np.diff(pb_int) > 0)
    s_int, a_int = AN.fit_bunching_1d(d, pb_int, sigma0=1.5, a0=10.0)
    s_free, a_free = AN.fit_bunching_1d(d, pb_free, sigma0=1.5, a0=10.0)
    print("fits: interacting", s_int, a_int, "free", s_free, a_free)
    assert np.max(np.abs(pb_int - AN.bunching_1d(d, s_int, a_int))) <= 0.05 * (0.5 - pb_int[0])
    assert s_int > 1.3 * s_free and a_int > a_free


def test_screening_restores_exchange_driven_bunching(hom_runs):
    """Sec. III(B), Eq. screenedCoulomb: damping the repulsion over a range
    sigma_c brings the interacting antisymmetric P_b back towards its value
    without interaction, the more so the shorter the range."""
    w = W.sweep32(prec="c64")
    w.update(nx=256, ny=32, dx=0.5, dy=0.5, dt=0.01, t_end=26.0)
    make = lambda: dict(qpc_h=1.85, qpc_w=1.5, lam=1.0, exch=-1,  # noqa: E731
                        alpha=W.packet(-15.0, 1.5, 2.5, +1), beta=W.packet(15.0, 1.5, 2.5, -1))
    screened = {}
    for sc in (3.0, 1.0):
        _, obs = _run(dict(w, screen=sc), [()], make)
        screened[sc] = obs[0]["p_bunch"] / obs[0]["norm"]
    free, full = hom_runs[(1.5, 0.0, -1, 0.0)], hom_runs[(1.5, 0.0, -1, 1.0)]
    print("P_b: free", free, "screened 1.0", screened[1.0], "screened 3.0", screened[3.0], "unscreened", full)
    assert abs(screened[1.0] - free) < abs(screened[3.0] - free) < abs(full - free)


def test_output_arm_entanglement(arm_entropy):
    """Sec. V: the spatial entanglement between the two output arms, from the
    slice that joins them.  A product state without interaction has none;
    with exchange alone it falls as the packets get wider (it vanishes in the
    plane-wave limit); Coulomb repulsion quenches the antisymmetric state's
    entanglement, and entangles a product state on its own."""
    S = arm_entropy
    anti = np.array([S[(s, 0.0, -1, 0.0)] for s in SIGMAS])
    print("S: antisymmetric by sigma", anti, "product", S[(1.5, 0.0, 0, 0.0)], "with Coulomb: antisymmetric",
          S[(1.5, 0.0, -1, 1.0)], "product", S[(1.5, 0.0, 0, 1.0)])
    assert S[(1.5, 0.0, 0, 0.0)] < 1e-5
    assert np.all(np.diff(anti) < -0.02)
    assert S[(1.5, 0.0, -1, 1.0)] < 0.7 * S[(1.5, 0.0, -1, 0.0)]
    assert S[(1.5, 0.0, 0, 1.0)] > 0.05


def test_coulomb_softening_saturates():
    """Sec. III(B), Fig. 5(b): for a product state (no exchange) the Coulomb
    repulsion alone antibunches.  A weak interaction (large softening d of
    Eq. coulomb) leaves P_b at the classical 1/2.  As d shrinks P_b falls,
    but each halving of d lowers it less: in 2D the electrons find paths
    around each other, so P_b saturates above 0 instead of vanishing."""
    p = {}
    for soft in (8.0, 1.0, 0.5, 0.25, 0.125):
        w = W.sweep32(prec="c64")
        w.update(nx=256, ny=32, dx=0.5, dy=0.5, dt=0.01, t_end=26.0, soft=soft)
        _, obs = _run(w, [()], lambda: dict(qpc_h=1.85, qpc_w=1.5, lam=1.0, exch=0,
                                            alpha=W.packet(-15.0, 1.5, 2.5, +1), beta=W.packet(15.0, 1.5, 2.5, -1)))
        p[soft] = obs[0]["p_bunch"] / obs[0]["norm"]
    print("P_b(softening):", p)
    assert p[8.0] > 0.49
    steps = [p[1.0] - p[0.5], p[0.5] - p[0.25], p[0.25] - p[0.125]]
    assert p[8.0] > p[1.0] and all(d > 0 for d in steps)
    assert steps[0] > steps[1] > steps[2]
    assert p[0.125] > 0.3


def test_bunching_dynamics():
    """Sec. III(A): P_b(t) of the antisymmetric state is 0 while the packets
    are apart, peaks while they meet at the saddle, then falls to a
    stationary value that does not vanish.  The product state has no such
    peak: it rises to its stationary 1/2, so the overshoot is an exchange
    effect.  Sampled every 100 steps (one time unit) to t = 26."""
    H = _binding()
    w = W.sweep32(prec="c64")
    w.update(nx=256, ny=32, dx=0.5, dy=0.5, dt=0.01)
    w["sims"] = [dict(qpc_h=1.85, qpc_w=1.5, lam=0.0, exch=e, alpha=W.packet(-15.0, 1.5, 2.5, +1),
                      beta=W.packet(15.0, 1.5, 2.5, -1)) for e in (-1, 0)]
    w["batch"] = 2
    pr = H.Propagator(w)
    pb = []
    for _ in range(27):
        pb.append([o["p_bunch"] / o["norm"] for o in pr.observables()])
        pr.step(100)
    pr.close()
    anti, prod = np.array(pb).T
    print("P_b(t) antisymmetric", np.round(anti, 4), "product", np.round(prod, 4))
    assert np.all(anti[:6] < 1e-4) and np.all(prod[:6] < 1e-4)
    assert abs(anti[-1] - anti[-3]) < 1e-4 and abs(prod[-1] - prod[-3]) < 1e-4      # stationary
    assert anti.max() > anti[-1] + 0.03 and anti[-1] > 0.3                          # peak, no vanishing
    assert 5 < int(np.argmax(anti)) < 20
    assert prod.max() < prod[-1] + 1e-3                                             # no overshoot
