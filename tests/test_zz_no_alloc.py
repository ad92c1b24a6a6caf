"""hom_bunching_static: the observables' norm and bunching probability for
callers that cannot allocate device memory (their partial sums live in a fixed
array inside the library).  Checked through the C ABI against hom_observables
on the same states, on two calls in a row with different inputs, so that the
second call cannot pass on what the first one left in the shared array.
This file is collected last so that a failure here stops a run only after
every other test has run."""

import ctypes

import numpy as np
import pytest

from paper_1903_02581_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_02581_gb300 import binding, build

    build.build()
    L = binding.lib()
    f = L.hom_bunching_static
    f.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                  ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return L


def run_static(L, prop, out):
    import torch

    w = prop.w
    st = L.hom_bunching_static(prop.state.data_ptr(), prop.params.prec, w["nx"], w["ny"], prop.batch,
                               w["dx"], w["dy"], out.data_ptr(), prop.stream.cuda_stream)
    assert st == 0, st
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(prop.batch, 2)


def batch_of(prec, batch):
    """The 32x32 sweep shrunk to 32x16, its simulations repeated up to batch
    with the second packet moved by 0.05 per repetition (distinct states)."""
    import copy

    w = W.shrink(W.sweep32(prec=prec), nx=32, ny=16)
    w["dx"] = w["dy"] = 0.5
    base = w["sims"]
    sims = []
    for i in range(batch):
        s = copy.deepcopy(base[i % len(base)])
        s["beta"]["x0"] += 0.05 * (i // len(base))
        sims.append(s)
    w["sims"] = sims
    w["batch"] = batch
    return w


# Both entry points sum the exact FP64 squares of the same stored values; only
# the order of the FP64 additions differs, so 1e-12 relative separates a
# rounding difference from a missing or doubled stripe of elements.
@pytest.mark.parametrize("prec,batch", [("c128", 3), ("c64", 3), ("c64", 64)])
def test_static_matches_observables_on_two_calls(lib, prec, batch):
    import torch

    from paper_1903_02581_gb300 import binding as H

    tol = 1e-12
    prop = H.Propagator(batch_of(prec, batch))
    out = torch.full((2 * prop.batch,), float("nan"), dtype=torch.float64, device="cuda")
    for nsteps in (0, 25):                       # second call on a different state
        prop.step(nsteps)
        ref = prop.observables()
        got = run_static(lib, prop, out)
        for b in range(prop.batch):
            assert abs(got[b, 0] - ref[b]["norm"]) <= tol * abs(ref[b]["norm"]), (b, got[b], ref[b])
            assert abs(got[b, 1] - ref[b]["p_bunch"]) <= tol * abs(ref[b]["p_bunch"]), (b, got[b], ref[b])
    assert np.all(np.isfinite(got))
    prop.close()


def test_static_rejects_sizes_beyond_the_array(lib):
    import torch

    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    # 65 simulations exceed the fixed array: rejected before any launch
    st = lib.hom_bunching_static(buf.data_ptr(), 0, 16, 16, 65, 0.5, 0.5, buf.data_ptr(), None)
    assert st == 1
    st = lib.hom_bunching_static(buf.data_ptr(), 0, 24, 16, 1, 0.5, 0.5, buf.data_ptr(), None)
    assert st == 1
    assert float(buf.abs().sum()) == 0.0
