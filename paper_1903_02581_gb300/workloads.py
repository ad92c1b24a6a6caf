"""Seeded synthetic workloads shared by the tests, the bench and the oracle legs.

This module holds parameters and random draws only: no step of the method's
arithmetic lives here, so the CUDA path and the oracle stay independent.  All
random numbers the method needs (packet-centre jitter, sweep draws, random
test states) are drawn here with numpy ``default_rng`` and passed on as plain
numbers or arrays.

The five workloads follow the paper's physical setting (Sec. II and III:
two counter-propagating edge packets at a beam splitter, with and without
Coulomb repulsion, with antisymmetrised states) on synthetic geometries,
because the paper gives neither its device geometry nor its grid or time
step.  Units hbar = m* = |e| = 1, magnetic length 1.
"""

from __future__ import annotations

import copy

import numpy as np

SEED = 20190306

# One packet: centre x0, width sigma, energy (or k0 when by_k0), direction.
def packet(x0, sigma, energy=0.0, direction=1, k0=0.0, by_k0=False):
    return dict(x0=float(x0), sigma=float(sigma), energy=float(energy),
                k0=float(k0), dir=int(direction), by_k0=bool(by_k0))


def _base(nx, ny, dx, dy, **kw):
    p = dict(nx=nx, ny=ny, dx=dx, dy=dy, B=1.0, omega=1.0, dt=0.01,
             qpc_h=1.0, qpc_w=1.5, qpc_x0=0.0, lam=1.0, soft=0.5,
             batch=1, prec="c128", nsteps=1, observe_every=0)
    p.update(kw)
    return p


def tiny():
    """16x16 per electron (65,536 points, complex128), 200 Strang steps at dt=0.01."""
    p = _base(16, 16, 0.5, 0.5, dt=0.01, nsteps=200, prec="c128")
    p["sims"] = [dict(qpc_h=1.0, qpc_w=1.5, lam=1.0,
                      alpha=packet(-3.0, 1.5, 2.5, +1), beta=packet(3.0, 1.5, 2.5, -1),
                      exch=-1)]
    return p


def sweep32(prec="c64"):
    """32x32 per electron: QPC height {0.8,1.0,1.2} x Coulomb {0,1}, 1000 steps at dt=0.005."""
    rng = np.random.default_rng(SEED)
    p = _base(32, 32, 0.5, 0.5, dt=0.005, nsteps=1000, prec=prec)
    sims = []
    for h in (0.8, 1.0, 1.2):
        for lam in (0.0, 1.0):
            ja, jb = rng.uniform(-0.1, 0.1, size=2)
            sims.append(dict(qpc_h=h, qpc_w=1.5, lam=lam,
                             alpha=packet(-3.0 + ja, 2.0, 2.5, +1),
                             beta=packet(3.0 + jb, 2.0, 2.5, -1), exch=-1))
    p["sims"] = sims
    p["batch"] = len(sims)
    return p


def fullscale(sigma=2.0):
    """256x64 per electron (268,435,456 points, complex64, 2 GiB), dt=0.002, 2000 steps."""
    p = _base(256, 64, 0.25, 0.25, dt=0.002, nsteps=2000, prec="c64",
              qpc_h=1.0, qpc_w=2.0, lam=1.0, soft=0.25, observe_every=100)
    p["sims"] = [dict(qpc_h=1.0, qpc_w=2.0, lam=1.0,
                      alpha=packet(-24.0, sigma, 3.0, +1),
                      beta=packet(24.0, sigma, 3.0, -1), exch=-1)]
    return p


def gradient():
    """64x32 per electron (4,194,304 points, complex64): final P_b after 800 steps at dt=0.005."""
    p = _base(64, 32, 0.5, 0.5, dt=0.005, nsteps=800, prec="c64",
              qpc_h=1.0, qpc_w=1.5, lam=1.0, soft=0.5)
    p["sims"] = [dict(qpc_h=1.0, qpc_w=1.5, lam=1.0,
                      alpha=packet(-3.0, 2.0, 2.5, +1), beta=packet(3.0, 2.0, 2.5, -1),
                      exch=-1)]
    p["ckpt_every"] = 50
    return p


def batched(nsim=32, shard=0):
    """nsim x 128x32 per electron (16,777,216 points each, complex64), dt=0.004, 1500 steps.

    ``shard`` selects one block of nsim simulations of a larger sweep (one
    block per process when the sweep is spread over several GPUs): shard 0 is
    this sweep itself, and every other shard draws its delays and widths from
    a stream of its own."""
    rng = np.random.default_rng(SEED + 5 if shard == 0 else [SEED + 5, int(shard)])
    p = _base(128, 32, 0.5, 0.5, dt=0.004, nsteps=1500, prec="c64", soft=0.5)
    delay = rng.uniform(-4.0, 4.0, size=nsim)
    sigma = rng.uniform(1.0, 3.0, size=nsim)
    sims = []
    for i in range(nsim):
        lam = 0.0 if i < nsim // 2 else 1.0
        sims.append(dict(qpc_h=1.0, qpc_w=1.5, lam=lam,
                         alpha=packet(-3.0, sigma[i], 2.5, +1),
                         beta=packet(3.0 + delay[i], sigma[i], 2.5, -1), exch=-1))
    p["sims"] = sims
    p["batch"] = nsim
    return p


WORKLOADS = dict(tiny=tiny, sweep32=sweep32, fullscale=fullscale,
                 gradient=gradient, batched=batched)


def shrink(p, nx=None, ny=None, nsteps=None, batch=None):
    """A copy of workload ``p`` on a smaller grid / shorter run (same physics family)."""
    q = copy.deepcopy(p)
    if nx is not None:
        q["dx"] = q["dx"] * q["nx"] / nx
        q["nx"] = nx
    if ny is not None:
        q["dy"] = q["dy"] * q["ny"] / ny
        q["ny"] = ny
    if nsteps is not None:
        q["nsteps"] = nsteps
    if batch is not None:
        q["sims"] = q["sims"][:batch]
        q["batch"] = len(q["sims"])
    return q


def random_state(shape, seed, dtype=np.complex128):
    """Complex Gaussian random array (unnormalised), for operator-level parity."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return a.astype(dtype)
