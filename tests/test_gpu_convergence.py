"""Convergence of the interacting bunching probability, through the CUDA path
in complex128: the paper prints no P_b for a comparable geometry, so its
absolute value is otherwise pinned only by agreement with the oracle.  Two
properties hold whatever the value:

- the symmetric (Strang) product of Eq. evoloperat is second order in dt:
  at a fixed time, successive differences of P_b shrink by 4 as dt halves;
- the Fourier representation of App. A converges faster than any power of
  the grid spacing for smooth packets and potentials: refining the grid at a
  fixed box changes P_b by far less than the coarser refinement did.

Geometry: the 32x32 sweep's simulation with QPC height 1 and Coulomb strength
1 (packets of energy 2.5 at x = -3 and +3 + jitter, on a 16 x 16 box), run to
t = 4, past the packets' meeting at the saddle."""

import pytest

from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu

T_END = 4.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import build

    build.build()


def p_bunch(nx, ny, dt):
    from paper_1903_02581_gb300 import binding as H

    w = W.sweep32(prec="c128")
    w["sims"] = [w["sims"][3]]                   # qpc_h = 1.0, lam = 1.0
    w["batch"] = 1
    assert w["sims"][0]["qpc_h"] == 1.0 and w["sims"][0]["lam"] == 1.0
    w = W.shrink(w, nx=nx, ny=ny)                # same 16 x 16 box
    w["dt"] = dt
    pr = H.Propagator(w)
    pr.step(round(T_END / dt))
    o = pr.observables()[0]
    pr.close()
    assert abs(o["norm"] - 1.0) < 1e-11
    return o["p_bunch"]


def test_pb_is_second_order_in_dt():
    dts = (0.04, 0.02, 0.01, 0.005)
    p = [p_bunch(32, 32, dt) for dt in dts]
    d = [abs(p[i] - p[i + 1]) for i in range(3)]
    print("P_b(dt):", p, "differences:", d)
    assert 0.05 < p[-1] < 0.95                   # the packets have met and scattered
    assert 3.4 < d[1] / d[2] < 4.6, d
    assert 3.0 < d[0] / d[1] < 5.0, d


def test_pb_converges_fast_in_dx():
    p = {n: p_bunch(n, n, 0.01) for n in (16, 32, 64)}
    coarse, fine = abs(p[16] - p[32]), abs(p[32] - p[64])
    print("P_b(grid):", p, "differences:", coarse, fine)
    assert fine < coarse / 4, (coarse, fine)
