"""The tensor-core form of the y sandwich (hom_ysandwich_tc, a measured design
trial of the short-axis DFT as a dense product on tcgen05 with bf16 operands
split three ways): each 64-point line times F_y^-1 e^{-i dt T_y} F_y, against
the oracle's DFT and kinetic phase in FP64 on seeded random lines.

Tolerance: 48 x 2^-23 = 5.7e-6 of the largest output value.  The split keeps
the products down to 2^-16 of the leading one, so the dropped terms are
~2^-24 relative (2.6e-8 on the CPU with exact accumulation); what remains is
the tensor core's FP32 accumulation, at most one accumulator ulp (2^-23) per
accumulation step of the 6 x 8 = 48 steps.  The mean change of a line's norm
(the operator is unitary) is reported and bounded by twice that: a bias
there, the same every step, is what decides the trial for the propagator
(on a GB300 it is -1.6e-6 per application, against +1e-10 for the same split
with exact accumulation, so the FFT form stays in the kinetic passes).
"""

import numpy as np
import pytest

from oracle import hom_oracle as O
from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_tensor_core_y_sandwich_matches_oracle_operator():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding as H
    from paper_1903_02581_gb300 import build

    build.build()
    nlines, dt, dy = 2048, 0.002, 0.25
    x = W.random_state((nlines, 64), seed=31).astype(np.complex64)
    d_in = torch.from_numpy(x).cuda()
    d_out = torch.empty_like(d_in)
    wb = H.lib().hom_ysandwich_tc_work_bytes()
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    H.hom_ysandwich_tc(d_in.data_ptr(), d_out.data_ptr(), nlines, dt, dy, work.data_ptr(), wb, 1)
    got = d_out.cpu().numpy().astype(np.complex128)
    m = O.Model(nx=16, ny=64, dx=0.25, dy=dy, dt=dt)
    g = np.exp(-1j * dt * O.ty_single(m))
    x64 = x.astype(np.complex128)
    ref = O.dft_axis(g[None, :] * O.dft_axis(x64, 1), 1, inverse=True)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    n0 = np.sum(np.abs(x64) ** 2, axis=1)
    bias = float(np.mean((np.sum(np.abs(got) ** 2, axis=1) - n0) / n0))
    print(f"tensor-core y sandwich: max error {err:.3e} of max|y|, mean norm change per line {bias:+.3e}")
    assert err <= 48 * 2.0 ** -23, err
    assert abs(bias) <= 2 * 48 * 2.0 ** -23, bias


def test_tensor_core_y_sandwich_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding as H

    buf = torch.zeros(64 * 2 * 256, dtype=torch.float32, device="cuda")
    wb = H.lib().hom_ysandwich_tc_work_bytes()
    work = torch.empty(wb, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HomError):
        H.hom_ysandwich_tc(buf.data_ptr(), buf.data_ptr(), 100, 0.002, 0.25, work.data_ptr(), wb, 1)
    with pytest.raises(H.HomError):
        H.hom_ysandwich_tc(buf.data_ptr(), buf.data_ptr(), 128, 0.002, 0.25, work.data_ptr(), wb - 1, 1)
