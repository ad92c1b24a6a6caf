"""ctypes binding of libhom (include/hom.h): argument marshalling only.

Every step of the propagation runs in the CUDA library; this module converts
Python values to the C structures, passes raw device pointers owned by
PyTorch, and turns a non-OK status into an exception.  There is no fallback:
if the library is missing, ``lib()`` raises.
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import re

import numpy as np

from . import build as _build

HOM_OK, HOM_ERR_ARG, HOM_ERR_STATE, HOM_ERR_CUDA, HOM_ERR_NOMEM, HOM_ERR_TIMEOUT, HOM_ERR_NUMERIC = range(7)
HOM_C64, HOM_C128 = 0, 1
HOM_STRANG, HOM_LIE = 0, 1
STATUS_NAMES = ["HOM_OK", "HOM_ERR_ARG", "HOM_ERR_STATE", "HOM_ERR_CUDA", "HOM_ERR_NOMEM",
                "HOM_ERR_TIMEOUT", "HOM_ERR_NUMERIC"]


class hom_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("prec", ctypes.c_int32),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("B", ctypes.c_double),
                ("omega_y", ctypes.c_double), ("dt", ctypes.c_double),
                ("qpc_h", ctypes.c_double), ("qpc_w", ctypes.c_double), ("qpc_x0", ctypes.c_double),
                ("coul_lambda", ctypes.c_double), ("coul_soft", ctypes.c_double),
                ("observe_every", ctypes.c_int32), ("ckpt_slots", ctypes.c_int32),
                ("coul_screen", ctypes.c_double), ("split", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("fermi_vb", ctypes.c_double), ("fermi_tau", ctypes.c_double), ("fermi_xa", ctypes.c_double),
                ("fermi_ya", ctypes.c_double), ("fermi_xb", ctypes.c_double), ("fermi_yb", ctypes.c_double)]


class hom_packet(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("sigma", ctypes.c_double), ("energy", ctypes.c_double),
                ("k0", ctypes.c_double), ("dir", ctypes.c_int32), ("by_k0", ctypes.c_int32),
                ("numeric", ctypes.c_int32), ("wall_side", ctypes.c_int32), ("wall_y", ctypes.c_double)]


class hom_obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("energy", ctypes.c_double), ("e_kin", ctypes.c_double),
                ("e_pot", ctypes.c_double), ("e_coul", ctypes.c_double), ("p_bunch", ctypes.c_double)]


OBS_KEYS = [f for f, _ in hom_obs._fields_]


class HomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


_LIB = None


def declared_functions() -> list[str]:
    """Names of the functions include/hom.h declares."""
    with open(os.path.join(_build.INCLUDE, "hom.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hom_[a-z_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libhom.so (built in-tree by ``build.build()``); raise if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libhom is not built ({_build.LIB} missing): run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    L.hom_state_bytes.argtypes = [P(hom_params)]
    L.hom_state_bytes.restype = ctypes.c_size_t
    L.hom_workspace_bytes.argtypes = [P(hom_params)]
    L.hom_workspace_bytes.restype = ctypes.c_size_t
    L.hom_create.argtypes = [P(hom_params), vp, vp, ctypes.c_size_t, vp, P(vp)]
    L.hom_create.restype = ctypes.c_int
    L.hom_set_sim_params.argtypes = [vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double]
    L.hom_set_sim_params.restype = ctypes.c_int
    L.hom_init_packets.argtypes = [vp, ctypes.c_int32, P(hom_packet), P(hom_packet), ctypes.c_int32]
    L.hom_init_packets.restype = ctypes.c_int
    L.hom_step.argtypes = [vp, ctypes.c_int32]
    L.hom_step.restype = ctypes.c_int
    L.hom_observables.argtypes = [vp, P(hom_obs)]
    L.hom_observables.restype = ctypes.c_int
    L.hom_backward.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double), P(ctypes.c_double)]
    L.hom_backward.restype = ctypes.c_int
    L.hom_copy_state.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_size_t, ctypes.c_int32]
    L.hom_copy_state.restype = ctypes.c_int
    L.hom_profile.argtypes = [vp, ctypes.c_int32]
    L.hom_profile.restype = ctypes.c_int
    L.hom_profile_read.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int64)]
    L.hom_profile_read.restype = ctypes.c_int
    L.hom_autotune_info.argtypes = [vp, P(ctypes.c_int32), P(ctypes.c_double)]
    L.hom_autotune_info.restype = ctypes.c_int
    L.hom_autotune_set.argtypes = [vp, P(ctypes.c_int32)]
    L.hom_autotune_set.restype = ctypes.c_int
    L.hom_marginal.argtypes = [vp, P(ctypes.c_double)]
    L.hom_marginal.restype = ctypes.c_int
    L.hom_conditional.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double)]
    L.hom_conditional.restype = ctypes.c_int
    L.hom_entanglement.argtypes = [vp] + [ctypes.c_int32] * 7 + [P(ctypes.c_double), P(ctypes.c_double)]
    L.hom_entanglement.restype = ctypes.c_int
    L.hom_vn_entropy.argtypes = [P(ctypes.c_double), ctypes.c_int32, ctypes.c_int32, P(ctypes.c_double),
                                 P(ctypes.c_double)]
    L.hom_vn_entropy.restype = ctypes.c_int
    L.hom_alu_peak.argtypes = [ctypes.c_int32, vp, vp, P(ctypes.c_double)]
    L.hom_alu_peak.restype = ctypes.c_int
    L.hom_ysandwich_tc_work_bytes.argtypes = []
    L.hom_ysandwich_tc_work_bytes.restype = ctypes.c_size_t
    L.hom_ysandwich_tc.argtypes = [vp, vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, vp, ctypes.c_size_t,
                                   ctypes.c_int32, P(ctypes.c_float), vp]
    L.hom_ysandwich_tc.restype = ctypes.c_int
    L.hom_last_error.argtypes = [vp]
    L.hom_last_error.restype = ctypes.c_char_p
    L.hom_destroy.argtypes = [vp]
    L.hom_destroy.restype = None
    _LIB = L
    return L


def _check(status, ctx):
    if status != HOM_OK:
        msg = lib().hom_last_error(ctx)
        raise HomError(status, msg.decode() if msg else "")


# --- thin wrappers with the C names ----------------------------------------

def hom_state_bytes(p: hom_params) -> int:
    return lib().hom_state_bytes(ctypes.byref(p))


def hom_workspace_bytes(p: hom_params) -> int:
    return lib().hom_workspace_bytes(ctypes.byref(p))


def hom_create(p: hom_params, d_state: int, d_workspace: int, workspace_bytes: int, stream: int):
    ctx = ctypes.c_void_p()
    _check(lib().hom_create(ctypes.byref(p), d_state, d_workspace, workspace_bytes, stream, ctypes.byref(ctx)), None)
    return ctx


def hom_set_sim_params(ctx, b, qpc_h, qpc_w, coul_lambda):
    _check(lib().hom_set_sim_params(ctx, b, qpc_h, qpc_w, coul_lambda), ctx)


def hom_init_packets(ctx, b, alpha: hom_packet, beta: hom_packet, exch: int):
    _check(lib().hom_init_packets(ctx, b, ctypes.byref(alpha), ctypes.byref(beta), exch), ctx)


def hom_step(ctx, nsteps: int):
    _check(lib().hom_step(ctx, nsteps), ctx)


def hom_observables(ctx, batch: int) -> list[dict]:
    out = (hom_obs * batch)()
    _check(lib().hom_observables(ctx, out), ctx)
    return [{k: getattr(o, k) for k in OBS_KEYS} for o in out]


def hom_backward(ctx, batch: int, nsteps: int, K: int):
    loss = (ctypes.c_double * batch)()
    grad = (ctypes.c_double * (3 * batch))()
    _check(lib().hom_backward(ctx, nsteps, K, loss, grad), ctx)
    return np.array(loss[:]), np.array(grad[:]).reshape(batch, 3)


def hom_marginal(ctx, batch: int, nx: int, ny: int) -> np.ndarray:
    out = np.empty((batch, nx, ny), dtype=np.float64)
    _check(lib().hom_marginal(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return out


def hom_conditional(ctx, b: int, ix2: int, iy2: int, nx: int, ny: int) -> np.ndarray:
    out = np.empty((nx, ny), dtype=np.float64)
    _check(lib().hom_conditional(ctx, b, ix2, iy2, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)
    return out


def hom_entanglement(ctx, b: int, iy1: int, iy2: int, x1_range, x2_range) -> tuple[float, float]:
    s = ctypes.c_double()
    w = ctypes.c_double()
    _check(lib().hom_entanglement(ctx, b, iy1, iy2, x1_range[0], x1_range[1], x2_range[0], x2_range[1],
                                  ctypes.byref(s), ctypes.byref(w)), ctx)
    return s.value, w.value


def hom_vn_entropy(phi: np.ndarray) -> tuple[float, float]:
    a = np.ascontiguousarray(phi, dtype=np.complex128)
    if a.ndim != 2:
        raise ValueError("phi must be a 2D array")
    s = ctypes.c_double()
    w = ctypes.c_double()
    st = lib().hom_vn_entropy(a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), a.shape[0], a.shape[1],
                              ctypes.byref(s), ctypes.byref(w))
    if st != HOM_OK:
        raise HomError(st, "hom_vn_entropy failed")
    return s.value, w.value


def hom_copy_state(ctx, b: int, host: np.ndarray, to_device: bool):
    if not host.flags.c_contiguous:
        raise ValueError("host array must be C-contiguous")
    _check(lib().hom_copy_state(ctx, b, host.ctypes.data, host.nbytes, 1 if to_device else 0), ctx)


def hom_profile(ctx, enable: bool):
    _check(lib().hom_profile(ctx, 1 if enable else 0), ctx)


HOM_PROFILE_KINDS = 4
PROFILE_KINDS = ("transposing", "in_place", "transpose", "double")


def hom_profile_read(ctx) -> dict:
    """Summed device ms and launch counts per kind: keys ms_<kind>, n_<kind>."""
    ms = (ctypes.c_double * HOM_PROFILE_KINDS)()
    n = (ctypes.c_int64 * HOM_PROFILE_KINDS)()
    _check(lib().hom_profile_read(ctx, ms, n), ctx)
    out = {}
    for i, k in enumerate(PROFILE_KINDS):
        out["ms_" + k] = ms[i]
        out["n_" + k] = n[i]
    return out


def hom_autotune_info(ctx) -> dict:
    v = (ctypes.c_int32 * 3)()
    ms = (ctypes.c_double * 7)()
    _check(lib().hom_autotune_info(ctx, v, ms), ctx)
    return dict(variants=list(v[:2]), strategy=v[2], pass_ms=list(ms[:4]), step_ms=list(ms[4:]))


def hom_autotune_set(ctx, variant_transposing: int, variant_in_place: int, strategy: int) -> None:
    ch = (ctypes.c_int32 * 3)(variant_transposing, variant_in_place, strategy)
    _check(lib().hom_autotune_set(ctx, ch), ctx)


def hom_alu_peak(kind: int, d_sink: int, stream: int = 0) -> float:
    """Measured FMA rate of the current GPU in flops/s: kind 0 FP32, 1 FP64.
    d_sink: a device buffer of at least 16 bytes (never written in practice)."""
    out = ctypes.c_double(0.0)
    st = lib().hom_alu_peak(kind, d_sink, stream or None, ctypes.byref(out))
    if st != HOM_OK:
        raise HomError(st, "hom_alu_peak failed")
    return out.value


def hom_ysandwich_tc(d_in: int, d_out: int, nlines: int, dt: float, dy: float, d_work: int, work_bytes: int,
                     nrep: int = 1, stream: int = 0) -> float:
    """Tensor-core y sandwich of nlines 64-point lines (design trial); returns
    the average device ms of nrep launches."""
    ms = ctypes.c_float(0.0)
    st = lib().hom_ysandwich_tc(d_in, d_out, nlines, dt, dy, d_work, work_bytes, nrep, ctypes.byref(ms),
                                stream or None)
    if st != HOM_OK:
        raise HomError(st, "hom_ysandwich_tc failed")
    return ms.value


def hom_last_error(ctx) -> str:
    return lib().hom_last_error(ctx).decode()


def hom_destroy(ctx):
    if ctx:
        lib().hom_destroy(ctx)


# --- convenience: parameters from a workload description -------------------

def make_params(w: dict, batch: int | None = None, ckpt_slots: int = 0, dt: float | None = None) -> hom_params:
    p = hom_params()
    p.nx, p.ny = w["nx"], w["ny"]
    p.batch = batch if batch is not None else w.get("batch", 1)
    p.prec = HOM_C128 if w.get("prec", "c128") == "c128" else HOM_C64
    p.dx, p.dy = w["dx"], w["dy"]
    p.B, p.omega_y = w["B"], w["omega"]
    p.dt = w["dt"] if dt is None else dt
    p.qpc_h, p.qpc_w, p.qpc_x0 = w["qpc_h"], w["qpc_w"], w.get("qpc_x0", 0.0)
    p.coul_lambda, p.coul_soft = w["lam"], w["soft"]
    p.observe_every = w.get("observe_every", 0)
    p.ckpt_slots = ckpt_slots
    p.coul_screen = w.get("screen", 0.0)
    p.split = HOM_LIE if w.get("split", "strang") == "lie" else HOM_STRANG
    p.reserved = 0
    p.fermi_vb, p.fermi_tau = w.get("fermi_vb", 0.0), w.get("fermi_tau", 1.0)
    p.fermi_xa, p.fermi_ya = w.get("fermi_xa", 0.0), w.get("fermi_ya", 0.0)
    p.fermi_xb, p.fermi_yb = w.get("fermi_xb", 0.0), w.get("fermi_yb", 0.0)
    return p


def make_packet(d: dict) -> hom_packet:
    pk = hom_packet()
    pk.x0, pk.sigma, pk.energy, pk.k0 = d["x0"], d["sigma"], d.get("energy", 0.0), d.get("k0", 0.0)
    pk.dir, pk.by_k0 = d.get("dir", 1), 1 if d.get("by_k0", False) else 0
    pk.numeric = 1 if d.get("numeric", False) else 0
    pk.wall_side, pk.wall_y = d.get("wall_side", 1), d.get("wall_y", 0.0)
    return pk


class Propagator:
    """Device state + workspace (PyTorch tensors) and a libhom context.

    ``w`` is a workload description (see ``workloads``): grid, time step,
    default potential, and a list ``sims`` of per-simulation QPC / Coulomb
    parameters and packets.  The state is initialised from the packets
    unless ``init=False``.
    """

    def __init__(self, w: dict, device: str = "cuda", ckpt_slots: int = 0, init: bool = True, stream=None):
        import torch

        self.w = w
        self.batch = len(w["sims"]) if "sims" in w else w.get("batch", 1)
        self.params = make_params(w, self.batch, ckpt_slots)
        sb = hom_state_bytes(self.params)
        wb = hom_workspace_bytes(self.params)
        if sb == 0 or wb == 0:
            raise HomError(HOM_ERR_ARG, "invalid parameters")
        self.dtype = torch.complex128 if self.params.prec == HOM_C128 else torch.complex64
        self.np_dtype = np.complex128 if self.params.prec == HOM_C128 else np.complex64
        n = w["nx"] * w["ny"]
        self.n = n
        self.device = torch.device(device)
        self.state = torch.empty((self.batch, n, n), dtype=self.dtype, device=self.device)
        self.workspace = torch.empty(wb, dtype=torch.uint8, device=self.device)
        # A stream of its own: hom_step captures its launches into CUDA graphs,
        # which the legacy default stream cannot hold.  Streams from torch's
        # pool do not synchronise with the default stream, so every call below
        # runs between two cross-stream waits (_ordered): the library sees what
        # torch wrote to the state before the call, and torch work issued after
        # it sees what the library wrote.
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.state.record_stream(self.stream)
        self.workspace.record_stream(self.stream)
        with self._ordered():
            self.ctx = hom_create(self.params, self.state.data_ptr(), self.workspace.data_ptr(), wb,
                                  self.stream.cuda_stream)
            if "sims" in w:
                for b, s in enumerate(w["sims"]):
                    hom_set_sim_params(self.ctx, b, s["qpc_h"], s["qpc_w"], s["lam"])
                    if init:
                        hom_init_packets(self.ctx, b, make_packet(s["alpha"]), make_packet(s["beta"]),
                                         s["exch"])

    @contextlib.contextmanager
    def _ordered(self):
        import torch

        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream == self.stream.cuda_stream:
            yield
            return
        self.stream.wait_stream(cur)
        try:
            yield
        finally:
            cur.wait_stream(self.stream)

    def step(self, nsteps: int):
        with self._ordered():
            hom_step(self.ctx, nsteps)

    def observables(self) -> list[dict]:
        with self._ordered():
            return hom_observables(self.ctx, self.batch)

    def backward(self, nsteps: int, K: int):
        with self._ordered():
            return hom_backward(self.ctx, self.batch, nsteps, K)

    def marginal(self) -> np.ndarray:
        """Unconditional probability density of particle 1, [batch][nx][ny]."""
        with self._ordered():
            return hom_marginal(self.ctx, self.batch, self.w["nx"], self.w["ny"])

    def conditional(self, b: int, ix2: int, iy2: int) -> np.ndarray:
        """|psi(x1, y1, x2*, y2*)|^2 of simulation b, [nx][ny]."""
        with self._ordered():
            return hom_conditional(self.ctx, b, ix2, iy2, self.w["nx"], self.w["ny"])

    def entanglement(self, b: int, iy1: int, iy2: int, x1_range, x2_range) -> tuple[float, float]:
        """(von Neumann entropy, slice weight) of the slice at (y1*, y2*)."""
        with self._ordered():
            return hom_entanglement(self.ctx, b, iy1, iy2, x1_range, x2_range)

    def get_state(self, b: int = 0) -> np.ndarray:
        nx, ny = self.w["nx"], self.w["ny"]
        out = np.empty((nx, ny, nx, ny), dtype=self.np_dtype)
        with self._ordered():
            hom_copy_state(self.ctx, b, out, to_device=False)
        return out

    def set_state(self, b: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, dtype=self.np_dtype)
        with self._ordered():
            hom_copy_state(self.ctx, b, a, to_device=True)

    def close(self):
        if getattr(self, "ctx", None):
            self.stream.synchronize()
            hom_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
