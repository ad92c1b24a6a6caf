"""Turn a plain workload dictionary into oracle inputs (test infrastructure only).

A workload is plain data (grid, time step, and per-simulation QPC, Coulomb
and packet parameters); this module reads it and calls ``hom_oracle`` only.
"""

from __future__ import annotations

from . import hom_oracle as O


def model_for(w: dict, sim: dict | None = None) -> O.Model:
    sim = sim or {}
    return O.Model(nx=w["nx"], ny=w["ny"], dx=w["dx"], dy=w["dy"], B=w["B"], omega=w["omega"],
                   dt=w["dt"], qpc_h=sim.get("qpc_h", w["qpc_h"]), qpc_w=sim.get("qpc_w", w["qpc_w"]),
                   qpc_x0=w.get("qpc_x0", 0.0), lam=sim.get("lam", w["lam"]), soft=w["soft"],
                   screen=w.get("screen", 0.0), fermi_vb=w.get("fermi_vb", 0.0),
                   fermi_tau=w.get("fermi_tau", 1.0), fermi_xa=w.get("fermi_xa", 0.0),
                   fermi_ya=w.get("fermi_ya", 0.0), fermi_xb=w.get("fermi_xb", 0.0),
                   fermi_yb=w.get("fermi_yb", 0.0))


def packet_k0(m: O.Model, pk: dict) -> float:
    if pk.get("by_k0", False):
        return pk["k0"]
    return O.k0_from_energy(pk["energy"], m.B, m.omega, pk["dir"])


def one_packet(m: O.Model, pk: dict):
    if pk.get("numeric", False):
        return O.edge_packet_numeric(m, pk["x0"], pk["sigma"], packet_k0(m, pk),
                                     pk.get("wall_y", 0.0), pk.get("wall_side", 1))
    return O.edge_packet(m, pk["x0"], pk["sigma"], packet_k0(m, pk))


def packets(w: dict, sim: dict):
    m = model_for(w, sim)
    return m, one_packet(m, sim["alpha"]), one_packet(m, sim["beta"])


def initial_state(w: dict, sim: dict):
    m, a, b = packets(w, sim)
    return O.two_particle(a, b, sim["exch"], m.dV)
