"""Write the golden observables and sampled states used by the precision
study and the GPU tests.

Calls only the FP64 oracle (oracle/); every stored value is the oracle's.
Usage:
  python tests/golden/make_golden.py sweep32     -> sweep32_oracle.json
  python tests/golden/make_golden.py fullscale2  -> fullscale2_oracle.json + .npz
      the full-scale workload (256x64 per electron, Coulomb strength 1,
      softening 0.25, packets of width 2) after 2 Strang steps: observables
      and 12 sampled rows psi[r1, :] (r1 = x1*ny + y1 fixed, all r2)
  python tests/golden/make_golden.py batched     -> batched_oracle.json + .npz
      simulations 0 and 31 of the batched sweep (128x32 per electron) over
      all 1500 steps: observables every few hundred steps and 8 sampled rows
      of each final state
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import adapter as A  # noqa: E402
from oracle import hom_oracle as O  # noqa: E402
from paper_1903_02581_gb300 import workloads as W  # noqa: E402


def sweep32():
    w = W.sweep32(prec="c128")
    out = {"workload": "sweep32", "nx": w["nx"], "ny": w["ny"], "dt": w["dt"], "nsteps": w["nsteps"],
           "checkpoints": [0, 100, 500, 1000], "sims": []}
    for i, sim in enumerate(w["sims"]):
        t0 = time.time()
        m = A.model_for(w, sim)
        psi = A.initial_state(w, sim)
        V = O.v_total(m)
        rec = {"qpc_h": sim["qpc_h"], "lam": sim["lam"], "alpha_x0": sim["alpha"]["x0"],
               "beta_x0": sim["beta"]["x0"], "obs": {}}
        done = 0
        for c in out["checkpoints"]:
            for _ in range(c - done):
                psi = O.strang_step(psi, m, vtot=V)
            done = c
            rec["obs"][str(c)] = O.observables(psi, m)
        out["sims"].append(rec)
        print(f"sim {i} done in {time.time() - t0:.0f}s: P_b(1000) = {rec['obs']['1000']['p_bunch']:.12f}", flush=True)
    return out


def sampled_rows(psi, nrand, seed, extra=()):
    """Row indices r1 of psi[r1, r2] to store: the rows of largest norm (where
    the state is), nrand seeded random rows and any extra ones, sorted."""
    n = psi.shape[0] * psi.shape[1]
    flat = psi.reshape(n, n)
    norms = np.sum(np.abs(flat) ** 2, axis=1)
    top = list(np.argsort(norms)[::-1][:8])
    rng = np.random.default_rng(seed)
    rows = set(int(r) for r in top) | set(int(r) for r in rng.choice(n, size=nrand, replace=False)) | set(extra)
    rows = sorted(rows)
    return rows, flat[rows]


def fullscale2():
    """Two Strang steps of the full-scale workload from the oracle's own
    initial state (the state the library builds from the same packets)."""
    w = W.fullscale(sigma=2.0)
    sim = w["sims"][0]
    m = A.model_for(w, sim)
    t0 = time.time()
    psi = A.initial_state(w, sim)
    obs = {"0": O.observables(psi, m)}
    print(f"initial state and observables: {time.time() - t0:.0f}s", flush=True)
    ph = O.strang_phases(m)
    for i in range(2):
        psi = O.strang_step(psi, m, phases=ph)
        print(f"step {i + 1}: {time.time() - t0:.0f}s", flush=True)
    del ph
    obs["2"] = O.observables(psi, m)
    ny = w["ny"]
    # the periodic x edge (x1 = 0 and nx - 1) and the saddle (x1 = nx/2) at the
    # packets' edge row y1 = 37 besides the largest and random rows
    rows, vals = sampled_rows(psi, 4, 3, extra=(0 * ny + 37, (w["nx"] - 1) * ny + 37, (w["nx"] // 2) * ny + 37))
    print(f"done: {time.time() - t0:.0f}s, P_b = {obs['2']['p_bunch']:.15f}", flush=True)
    np.savez(os.path.join(HERE, "fullscale2_oracle.npz"), rows=np.array(rows), psi_rows=vals)
    return {"workload": "fullscale", "sigma": 2.0, "nx": w["nx"], "ny": w["ny"], "dt": w["dt"], "nsteps": 2,
            "rows": rows, "obs": obs}


def fullscale_lie2():
    """Two steps of the paper's printed first-order product (Eq. evoloperat,
    the Lie order: T_x, T_y, then V, each over a full step) on the full-scale
    workload, from the oracle's own initial state."""
    w = W.fullscale(sigma=2.0)
    w["split"] = "lie"
    sim = w["sims"][0]
    m = A.model_for(w, sim)
    t0 = time.time()
    psi = A.initial_state(w, sim)
    V = O.v_total(m)
    for i in range(2):
        psi = O.lie_step(psi, m, vtot=V)
        print(f"step {i + 1}: {time.time() - t0:.0f}s", flush=True)
    del V
    obs = {"2": O.observables(psi, m)}
    ny = w["ny"]
    rows, vals = sampled_rows(psi, 4, 5, extra=(0 * ny + 37, (w["nx"] - 1) * ny + 37, (w["nx"] // 2) * ny + 37))
    print(f"done: {time.time() - t0:.0f}s, P_b = {obs['2']['p_bunch']:.15f}", flush=True)
    np.savez(os.path.join(HERE, "fullscale_lie2_oracle.npz"), rows=np.array(rows), psi_rows=vals)
    return {"workload": "fullscale", "split": "lie", "sigma": 2.0, "nx": w["nx"], "ny": w["ny"], "dt": w["dt"],
            "nsteps": 2, "rows": rows, "obs": obs}


def batched():
    """Simulations 0 (Coulomb off) and 31 (Coulomb on) of the batched sweep."""
    w = W.batched()
    out = {"workload": "batched", "nx": w["nx"], "ny": w["ny"], "dt": w["dt"], "nsteps": w["nsteps"],
           "checkpoints": [0, 100, 500, 1000, 1500], "sims": {}}
    arrays = {}
    for b in (0, 31):
        sim = w["sims"][b]
        m = A.model_for(w, sim)
        t0 = time.time()
        psi = A.initial_state(w, sim)
        ph = O.strang_phases(m)
        rec = {"lam": sim["lam"], "sigma": sim["alpha"]["sigma"], "beta_x0": sim["beta"]["x0"], "obs": {}}
        done = 0
        for c in out["checkpoints"]:
            for _ in range(c - done):
                psi = O.strang_step(psi, m, phases=ph)
            done = c
            rec["obs"][str(c)] = O.observables(psi, m)
            print(f"sim {b} step {c}: {time.time() - t0:.0f}s P_b = {rec['obs'][str(c)]['p_bunch']:.15f}",
                  flush=True)
        rows, vals = sampled_rows(psi, 0, 7 + b)
        rec["rows"] = rows
        arrays[f"rows_{b}"] = np.array(rows)
        arrays[f"psi_rows_{b}"] = vals
        out["sims"][str(b)] = rec
    np.savez(os.path.join(HERE, "batched_oracle.npz"), **arrays)
    return out


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "sweep32"
    res = {"sweep32": sweep32, "fullscale2": fullscale2, "fullscale_lie2": fullscale_lie2, "batched": batched}[which]()
    with open(os.path.join(HERE, f"{which}_oracle.json"), "w") as f:
        json.dump(res, f, indent=1)
