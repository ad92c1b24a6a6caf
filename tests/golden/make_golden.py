"""Write the golden observables used by the precision study and GPU tests.

Calls only the FP64 oracle (oracle/); every stored value is the oracle's.
Usage: python tests/golden/make_golden.py sweep32   (writes sweep32_oracle.json)
"""

import json
import os
import sys
import time

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


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "sweep32"
    res = {"sweep32": sweep32}[which]()
    with open(os.path.join(HERE, f"{which}_oracle.json"), "w") as f:
        json.dump(res, f, indent=1)
