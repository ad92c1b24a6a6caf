"""Exchange symmetry of the whole propagation on the GPU (complex128), with
Coulomb repulsion, through a full scattering event at the saddle.

The Hamiltonian and the bunching mask are symmetric under the swap of the
particles, so for the antisymmetrised (-), symmetrised (+) and product
states built from the same two normalised packets (Eq. twopstate),

    (1 + |s|^2) P_+ + (1 - |s|^2) P_- = 2 P_prod,     s = <alpha|beta>,

at every time, P being the bunching probability (Eq. p_bunching) of each
renormalised state.  A kernel that treated the two particles differently, or
an exchange sign applied wrongly, breaks it.  Without interaction the
antisymmetric state also shows the Hong-Ou-Mandel dip and the symmetric one
the peak (Sec. IV): at zero delay P_- is below, and P_+ above, their values
at a delay where the packets barely overlap.

Grid 64 x 32 per electron (dx = dy = 0.5: a 32 x 16 box), packets of width
1.5 and energy 2.5 from x = -3 and x = 3 + delay, a saddle of height 2.25
(about half of a single packet is transmitted), run to t = 10, after both
packets have passed the saddle."""

import numpy as np
import pytest

from oracle import adapter as A
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T_END, DT = 10.0, 0.01


@pytest.fixture(scope="module")
def runs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding as H
    from paper_1903_02581_gb300 import build

    build.build()
    w = W.sweep32(prec="c128")
    w.update(nx=64, ny=32, dx=0.5, dy=0.5, dt=DT)

    def sim(lam, delay, exch):
        return dict(qpc_h=2.25, qpc_w=1.5, lam=lam, exch=exch,
                    alpha=W.packet(-3.0, 1.5, 2.5, +1), beta=W.packet(3.0 + delay, 1.5, 2.5, -1))

    keys = [(lam, delay, exch) for lam, delay in ((1.0, 0.0), (1.0, 4.0), (0.0, 0.0), (0.0, 6.0))
            for exch in (-1, 0, 1)]
    w["sims"] = [sim(*k) for k in keys]
    w["batch"] = len(keys)
    pr = H.Propagator(w)
    pr.step(round(T_END / DT))
    obs = pr.observables()
    pr.close()
    out = {}
    for k, o, s in zip(keys, obs, w["sims"]):
        assert abs(o["norm"] - 1.0) < 1e-11
        m, a, b = A.packets(w, s)
        ov = np.vdot(a.ravel(), b.ravel()) * m.dx * m.dy
        out[k] = (o["p_bunch"], abs(ov) ** 2)
    return out


@pytest.mark.parametrize("lam,delay", [(1.0, 0.0), (1.0, 4.0), (0.0, 0.0), (0.0, 6.0)])
def test_exchange_sum_identity(runs, lam, delay):
    pm, s2 = runs[(lam, delay, -1)]
    p0, _ = runs[(lam, delay, 0)]
    pp, _ = runs[(lam, delay, 1)]
    assert abs((1 + s2) * pp + (1 - s2) * pm - 2 * p0) <= 1e-11, (pm, p0, pp, s2)


def test_hong_ou_mandel_dip_and_peak(runs):
    anti0, sym0 = runs[(0.0, 0.0, -1)][0], runs[(0.0, 0.0, 1)][0]
    antid, symd = runs[(0.0, 6.0, -1)][0], runs[(0.0, 6.0, 1)][0]
    prod = runs[(0.0, 0.0, 0)][0]
    print("P_b: antisymmetric", anti0, antid, "symmetric", sym0, symd, "product", prod)
    assert 0.1 < prod < 0.9                        # the saddle splits the packets
    # The saddle's transmission varies over the energy spread of these narrow
    # packets (the parameter a of Eq. bunching), so the dip and the peak are
    # shallow; they still exceed FP64 noise by ten orders of magnitude.
    assert anti0 < antid - 0.01                    # dip
    assert sym0 > symd + 0.01                      # peak
    assert anti0 < prod < sym0
