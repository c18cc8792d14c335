"""Thin Python binding of the C ABI in include/fnn.h (argument marshalling only).

Every step of the path runs in libfnn.so's CUDA kernels; torch is used only to
own device memory and to name the current stream.  Importing this module loads
the library and raises if it is missing: there is no CPU fallback.

Names follow the C entry points: build_neighbors, nlist_nnz, nlist_export, aev,
aev_jvp, energy_forces, energy_forces_host, param_grads, md_run, Server, sync,
load_weights, save_weights; energy_forces_autograd wraps energy_forces and
param_grads as a torch.autograd.Function for training.
"""
from __future__ import annotations

import ctypes
import os
import struct
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfnn.so")

FNN_OK, FNN_PENDING = 0, 1
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "E_INVALID", -2: "E_SPECIES", -3: "E_CELL", -4: "E_CAPACITY",
                -5: "E_OOM", -6: "E_TIMEOUT", -7: "E_NONFINITE", -8: "E_CUDA", -9: "E_STATE"}
PRECISION = {"fp32": 0, "bf16": 1, "fp8": 2, "fp32x3": 3, "bf16_fused": 4}


class FnnError(RuntimeError):
    def __init__(self, code: int, msg: str, info: int = 0):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg} (info={info})")
        self.code = code
        self.info = info


class Config(ctypes.Structure):
    _fields_ = [("rc_rad", ctypes.c_double), ("rc_ang", ctypes.c_double), ("eta_rad", ctypes.c_double),
                ("eta_ang", ctypes.c_double), ("zeta", ctypes.c_double), ("shift_rad0", ctypes.c_double),
                ("shift_ang0", ctypes.c_double), ("skin", ctypes.c_double), ("n_members", ctypes.c_int32),
                ("switch_kind", ctypes.c_int32), ("switch_p", ctypes.c_double)]


SWITCH = {"cosine": 0, "polynomial": 1, "exponential": 2}


class CWeights(ctypes.Structure):
    _fields_ = [("n_members", ctypes.c_int32)] + [(n, ctypes.c_void_p) for n in
                                                   ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")]


PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")


def param_shapes(M: int) -> dict:
    """Shapes of the network parameters of an M-member ensemble (row-major W[out][in], element axis 7)."""
    return {"W1": (M, 7, 256, 1008), "b1": (M, 7, 256), "W2": (M, 7, 192, 256), "b2": (M, 7, 192),
            "W3": (M, 7, 160, 192), "b3": (M, 7, 160), "w4": (M, 7, 160), "b4": (M, 7)}


class CGrads(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in PARAM_NAMES]


class CRequest(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("Z", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("cell", ctypes.c_void_p), ("n_steps", ctypes.c_int32), ("dt_fs", ctypes.c_double)]


class CResult(ctypes.Structure):
    _fields_ = [("energies", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("forces", ctypes.c_void_p), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("n_steps_done", ctypes.c_int32)]


class CServeCounters(ctypes.Structure):
    _fields_ = [("atom_evals", ctypes.c_int64), ("batch_steps", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("max_batch_atoms", ctypes.c_int64), ("pending", ctypes.c_int64), ("bytes_per_atom", ctypes.c_double),
                ("host_ms", ctypes.c_double), ("step_ms", ctypes.c_double), ("failed", ctypes.c_int64),
                ("rebuilds", ctypes.c_int64), ("guard_rebuilds", ctypes.c_int64)]


class CMdOptions(ctypes.Structure):
    _fields_ = [("n_steps", ctypes.c_int32), ("dt_fs", ctypes.c_double), ("rebuild_every", ctypes.c_int32),
                ("skin_guard", ctypes.c_int32), ("integrator", ctypes.c_int32), ("temperature_K", ctypes.c_double),
                ("friction_per_fs", ctypes.c_double), ("seed", ctypes.c_uint64), ("step0", ctypes.c_uint64)]


class CMdCounters(ctypes.Structure):
    _fields_ = [("rebuilds", ctypes.c_int32), ("guard_rebuilds", ctypes.c_int32), ("graph_blocks", ctypes.c_int32),
                ("max_displacement", ctypes.c_double)]


class CRpmdOptions(ctypes.Structure):
    _fields_ = [("n_beads", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("dt_fs", ctypes.c_double),
                ("temperature_K", ctypes.c_double), ("rebuild_every", ctypes.c_int32), ("skin_guard", ctypes.c_int32)]


class CSystem(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int32), ("n_mol", ctypes.c_int32), ("mol_offsets", ctypes.c_void_p),
                ("Z", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("cell", ctypes.c_void_p), ("pbc", ctypes.c_void_p)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2405_01491_b300.build` "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "fnn_config_default": (None, [P]),
        "fnn_create": (I32, [P, P]),
        "fnn_destroy": (I32, [P]),
        "fnn_load_weights": (I32, [P, ctypes.c_char_p, P]),
        "fnn_nlist_create": (I32, [P, P, I64]),
        "fnn_nlist_destroy": (I32, [P]),
        "fnn_nlist_reserve": (I32, [P, I32, I32, I64]),
        "fnn_build_neighbors": (I32, [P, P, P, P]),
        "fnn_nlist_nnz": (I32, [P, P]),
        "fnn_nlist_export": (I32, [P, P, P, P, I64, P]),
        "fnn_aev": (I32, [P, P, P, P, P]),
        "fnn_aev_jvp": (I32, [P, P, P, P, P, P]),
        "fnn_param_grads": (I32, [P, P, P, I32, P, P, P, P]),
        "fnn_calibrate_fp8": (I32, [P, P, P, P]),
        "fnn_graph_create": (I32, [P, P, P, I32, P, P, P, I32, P, P]),
        "fnn_graph_launch": (I32, [P, P]),
        "fnn_graph_kernels": (I32, [P, P]),
        "fnn_graph_destroy": (I32, [P]),
        "fnn_energy_forces": (I32, [P, P, P, I32, P, P, P, P]),
        "fnn_energy_forces_host": (I32, [P, I32, I32, P, P, P, P, P, I32, P, P, P, P]),
        "fnn_sync": (I32, [P, P, P]),
        "fnn_last_error": (ctypes.c_char_p, [P]),
        "fnn_profile_enable": (I32, [P, I32]),
        "fnn_profile_read": (I32, [P, P, P, P, I32, P]),
        "fnn_launch_count": (I32, [P, P]),
        "fnn_selftest_lookback": (I32, [P, I32, P]),
        "fnn_crate_angular": (I32, [P, P, P, P, P, P]),
        "fnn_crate_angular_vjp": (I32, [P, P, P, P, P, P, P, P]),
        "fnn_build_neighbors_static": (I32, [P, ctypes.c_double, P, P, P, I64, P, P]),
        "fnn_md_run": (I32, [P, P, P, P, P, I32, I32, ctypes.c_double, I32, P, P, P]),
        "fnn_md_run_ex": (I32, [P, P, P, P, P, I32, P, P, P, P, P, P]),
        "fnn_rpmd_run": (I32, [P, P, P, P, P, I32, P, P, P, P, P, P]),
        "fnn_serve_create": (I32, [P, P, ctypes.c_size_t, I32, I32]),
        "fnn_serve_submit": (I32, [P, P, P]),
        "fnn_serve_poll": (I32, [P, ctypes.c_uint64, P, I64]),
        "fnn_serve_stats": (I32, [P, P]),
        "fnn_serve_destroy": (I32, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """fnn_ctx: constants, ensemble size, device parameters and workspaces."""

    def __init__(self, n_members: int = 1, skin: float = 0.0, **overrides):
        cfg = Config()
        lib.fnn_config_default(ctypes.byref(cfg))
        cfg.n_members = n_members
        cfg.skin = skin
        if "switch" in overrides:   # by name: "cosine", "polynomial", "exponential"
            cfg.switch_kind = SWITCH[overrides.pop("switch")]
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        self.h = None
        h = ctypes.c_void_p()
        code = lib.fnn_create(ctypes.byref(h), ctypes.byref(cfg))
        if code != FNN_OK:
            raise FnnError(code, "fnn_create")
        self.h = h

    def _check(self, code, what):
        if code != FNN_OK:
            raise FnnError(code, f"{what}: {lib.fnn_last_error(self.h).decode()}")

    def close(self):
        if getattr(self, "h", None):
            lib.fnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def load_weights(ctx: Context, weights=None, path: str | None = None):
    """fnn_load_weights from a synth.Weights-like object (float32 arrays) or a file."""
    ctx.param_stamp = None
    if path is not None:
        ctx._check(lib.fnn_load_weights(ctx.h, path.encode(), None), "fnn_load_weights")
        return
    arrs = [np.ascontiguousarray(getattr(weights, k), np.float32) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")]
    cw = CWeights(int(arrs[0].shape[0]), *(a.ctypes.data for a in arrs))
    ctx._check(lib.fnn_load_weights(ctx.h, None, ctypes.byref(cw)), "fnn_load_weights")


def save_weights(path: str, weights):
    """Write the flat weight file fnn_load_weights reads ("FNNW", version 1, M, eight float32 arrays)."""
    arrs = [np.ascontiguousarray(getattr(weights, k), np.float32) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "w4", "b4")]
    with open(path, "wb") as f:
        f.write(b"FNNW" + struct.pack("<ii", 1, int(arrs[0].shape[0])))
        for a in arrs:
            f.write(a.astype("<f4").tobytes())


@dataclass
class DeviceSystem:
    """Device copies of a structure batch in the layout of fnn_system (positions as float4)."""
    n_atoms: int
    n_mol: int
    mol_offsets: object
    Z: object
    pos: object
    cell: object
    pbc: object

    @classmethod
    def from_structures(cls, s, device="cuda"):
        import torch
        pos4 = torch.zeros((s.n_atoms, 4), dtype=torch.float32)
        pos4[:, :3] = torch.from_numpy(np.asarray(s.pos, np.float32))
        periodic = bool(np.any(s.pbc))
        return cls(s.n_atoms, s.n_mol,
                   torch.from_numpy(np.asarray(s.mol_offsets, np.int32)).to(device),
                   torch.from_numpy(np.asarray(s.Z, np.int32)).to(device),
                   pos4.to(device),
                   torch.from_numpy(np.asarray(s.cell, np.float32).reshape(-1, 9)).to(device) if periodic else None,
                   torch.from_numpy(np.asarray(s.pbc, np.uint8)).to(device) if periodic else None)

    def c(self):
        return CSystem(self.n_atoms, self.n_mol, self.mol_offsets.data_ptr(), self.Z.data_ptr(),
                       self.pos.data_ptr(), self.cell.data_ptr() if self.cell is not None else None,
                       self.pbc.data_ptr() if self.pbc is not None else None)


class NeighborList:
    """fnn_nlist handle."""

    def __init__(self, ctx: Context, capacity: int = 0):
        self.ctx = ctx
        self.h = None
        h = ctypes.c_void_p()
        ctx._check(lib.fnn_nlist_create(ctx.h, ctypes.byref(h), int(capacity)), "fnn_nlist_create")
        self.h = h

    def reserve(self, n_atoms: int, n_mol: int, capacity: int):
        self.ctx._check(lib.fnn_nlist_reserve(self.h, n_atoms, n_mol, int(capacity)), "fnn_nlist_reserve")

    def close(self):
        if getattr(self, "h", None):
            lib.fnn_nlist_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sync(ctx: Context, stream=None):
    """fnn_sync: (status code, info); clears the sticky status."""
    info = ctypes.c_int64(0)
    code = lib.fnn_sync(ctx.h, _stream(stream), ctypes.byref(info))
    return code, info.value


def check(ctx: Context, what: str = "device status", stream=None):
    code, info = sync(ctx, stream)
    if code != FNN_OK:
        raise FnnError(code, f"{what}: {lib.fnn_last_error(ctx.h).decode()}", info)


def build_neighbors(ctx: Context, system: DeviceSystem, nl: NeighborList, stream=None, checked: bool = False):
    """fnn_build_neighbors; with checked=True synchronise, and on overflow grow the list and rebuild once."""
    cs = system.c()
    ctx._check(lib.fnn_build_neighbors(ctx.h, ctypes.byref(cs), nl.h, _stream(stream)), "fnn_build_neighbors")
    if checked:
        code, info = sync(ctx, stream)
        if code == -4 and info > 0:
            nl.reserve(system.n_atoms, system.n_mol, info + info // 4)
            ctx._check(lib.fnn_build_neighbors(ctx.h, ctypes.byref(cs), nl.h, _stream(stream)), "fnn_build_neighbors")
            code, info = sync(ctx, stream)
        if code != FNN_OK:
            raise FnnError(code, "fnn_build_neighbors", info)


def nlist_nnz(nl: NeighborList) -> int:
    n = ctypes.c_int64(0)
    nl.ctx._check(lib.fnn_nlist_nnz(nl.h, ctypes.byref(n)), "fnn_nlist_nnz")
    return n.value


def nlist_export(nl: NeighborList, n_atoms: int):
    """CSR copy of the list on the host: row_ptr [N+1], nbr [nnz], shift [nnz, 3] (int8)."""
    nnz = nlist_nnz(nl)
    row_ptr = np.zeros(n_atoms + 1, np.int32)
    nbr = np.zeros(max(nnz, 1), np.int32)
    shift = np.zeros((max(nnz, 1), 3), np.int8)
    got = ctypes.c_int64(0)
    nl.ctx._check(lib.fnn_nlist_export(nl.h, row_ptr.ctypes.data, nbr.ctypes.data, shift.ctypes.data, max(nnz, 1),
                                       ctypes.byref(got)), "fnn_nlist_export")
    return row_ptr, nbr[:nnz], shift[:nnz]


def aev(ctx: Context, system: DeviceSystem, nl: NeighborList, out=None, stream=None):
    """fnn_aev into a float32 device tensor [N, 1008]."""
    import torch
    if out is None:
        out = torch.empty((system.n_atoms, 1008), dtype=torch.float32, device="cuda")
    cs = system.c()
    ctx._check(lib.fnn_aev(ctx.h, ctypes.byref(cs), nl.h, _ptr(out), _stream(stream)), "fnn_aev")
    return out


def aev_jvp(ctx: Context, system: DeviceSystem, nl: NeighborList, V, out=None, stream=None):
    """fnn_aev_jvp: directional derivative [N, 1008] of the AEVs along the displacement field V [N, 3] (device)."""
    import torch
    if out is None:
        out = torch.empty((system.n_atoms, 1008), dtype=torch.float32, device="cuda")
    cs = system.c()
    ctx._check(lib.fnn_aev_jvp(ctx.h, ctypes.byref(cs), nl.h, _ptr(V), _ptr(out), _stream(stream)), "fnn_aev_jvp")
    return out


def param_grads(ctx: Context, system: DeviceSystem, nl: NeighborList, dLdE, dLdF, grads: dict | None = None,
                stream=None, precision: str = "fp32") -> dict:
    """fnn_param_grads: ADDS dL/dtheta into grads (float32 device tensors shaped like the weights; zeros
    when None) for the loss gradients dL/dE [n_mol] float64 and dL/dF [N,3] float32; returns grads.
    precision "fp32" (SIMT) or "bf16" (tensor cores)."""
    import torch
    if grads is None:
        grads = {k: torch.zeros(v, dtype=torch.float32, device="cuda")
                 for k, v in param_shapes(ctx.cfg.n_members).items()}
    dLdE = dLdE.to(torch.float64).contiguous()
    dLdF = dLdF.to(torch.float32).contiguous()
    cg = CGrads(*(grads[k].data_ptr() for k in PARAM_NAMES))
    cs = system.c()
    ctx._check(lib.fnn_param_grads(ctx.h, ctypes.byref(cs), nl.h, PRECISION[precision], _ptr(dLdE), _ptr(dLdF),
                                   ctypes.byref(cg), _stream(stream)), "fnn_param_grads")
    return grads


_FUNCTION = None


def _function():
    """torch.autograd.Function over fnn_energy_forces (forward) and fnn_param_grads (backward)."""
    global _FUNCTION
    if _FUNCTION is not None:
        return _FUNCTION
    import torch

    class EnergyForces(torch.autograd.Function):
        @staticmethod
        def forward(fctx, ctx, system, nl, precision, *params):
            _load_params(ctx, params)
            E, F, _ = energy_forces(ctx, system, nl, precision, virial=False)
            fctx.ctx, fctx.system, fctx.nl, fctx.precision = ctx, system, nl, precision
            fctx.stamp = ctx.param_stamp
            return E, F

        @staticmethod
        def backward(fctx, gE, gF):
            ctx = fctx.ctx
            if ctx.param_stamp != fctx.stamp:
                raise RuntimeError("the context's parameters changed between forward and backward")
            system = fctx.system
            if gE is None:
                gE = torch.zeros(system.n_mol, dtype=torch.float64, device="cuda")
            if gF is None:
                gF = torch.zeros((system.n_atoms, 3), dtype=torch.float32, device="cuda")
            g = param_grads(ctx, system, fctx.nl, gE, gF, precision=fctx.precision)
            return (None, None, None, None) + tuple(g[k] for k in PARAM_NAMES)

    _FUNCTION = EnergyForces
    return _FUNCTION


def _load_params(ctx: Context, params):
    """Upload the parameter tensors to the context when they differ from what it holds."""
    stamp = tuple((p.data_ptr(), p._version) for p in params)
    if getattr(ctx, "param_stamp", None) == stamp:
        return
    host = type("W", (), {k: p.detach().float().cpu().numpy() for k, p in zip(PARAM_NAMES, params)})
    load_weights(ctx, host)
    ctx.param_stamp = stamp


def energy_forces_autograd(ctx: Context, system: DeviceSystem, nl: NeighborList, params, precision: str = "fp32"):
    """(E [n_mol] float64, F [N,3] float32) as differentiable functions of params (the eight weight
    tensors in PARAM_NAMES order, float32): a loss built from E and F back-propagates into the
    parameters through fnn_param_grads (section IV).  precision "fp32" or "bf16" (networks on the
    tensor cores for both the forward evaluation and the gradients)."""
    return _function().apply(ctx, system, nl, precision, *params)


def crate_angular(ctx: Context, system: DeviceSystem, nl: NeighborList, V, out=None, stream=None):
    """fnn_crate_angular: the CRATE angular resource g [N, 4, 32] (float32, device) from V [7, 8, 32]."""
    import torch
    if out is None:
        out = torch.empty((system.n_atoms, 4, 32), dtype=torch.float32, device="cuda")
    cs = system.c()
    ctx._check(lib.fnn_crate_angular(ctx.h, ctypes.byref(cs), nl.h, _ptr(V), _ptr(out), _stream(stream)),
               "fnn_crate_angular")
    return out


def crate_angular_vjp(ctx: Context, system: DeviceSystem, nl: NeighborList, V, G, grad_V: bool = True,
                      stream=None):
    """fnn_crate_angular_vjp: (dL/dx [N, 3], dL/dV [7, 8, 32] or None) from G = dL/dg [N, 4, 32]."""
    import torch
    gx = torch.empty((system.n_atoms, 3), dtype=torch.float32, device="cuda")
    gV = torch.empty((7, 8, 32), dtype=torch.float32, device="cuda") if grad_V else None
    cs = system.c()
    ctx._check(lib.fnn_crate_angular_vjp(ctx.h, ctypes.byref(cs), nl.h, _ptr(V), _ptr(G), _ptr(gx), _ptr(gV),
                                         _stream(stream)), "fnn_crate_angular_vjp")
    return gx, gV


def calibrate_fp8(ctx: Context, system: DeviceSystem, nl: NeighborList, stream=None):
    """fnn_calibrate_fp8: per-layer activation scales of the FP8 form from an FP32 evaluation of system."""
    cs = system.c()
    ctx._check(lib.fnn_calibrate_fp8(ctx.h, ctypes.byref(cs), nl.h, _stream(stream)), "fnn_calibrate_fp8")


def energy_forces(ctx: Context, system: DeviceSystem, nl: NeighborList, precision: str = "fp32", virial: bool = True,
                  out=None, stream=None):
    """fnn_energy_forces: (E [n_mol] float64, F [N,3] float32, virial [n_mol,3,3] float64 or None)."""
    import torch
    if out is None:
        E = torch.empty(system.n_mol, dtype=torch.float64, device="cuda")
        F = torch.empty((system.n_atoms, 3), dtype=torch.float32, device="cuda")
        W = torch.empty((system.n_mol, 3, 3), dtype=torch.float64, device="cuda") if virial else None
    else:
        E, F, W = out
    cs = system.c()
    ctx._check(lib.fnn_energy_forces(ctx.h, ctypes.byref(cs), nl.h, PRECISION[precision], _ptr(E), _ptr(F), _ptr(W),
                                     _stream(stream)), "fnn_energy_forces")
    return E, F, W


def energy_forces_host(ctx: Context, s, precision: str = "fp32", virial: bool = True, stream=None, out=None):
    """fnn_energy_forces_host from host arrays (numpy); returns host (E, F, virial)."""
    Z = np.ascontiguousarray(s.Z, np.int32)
    pos = np.ascontiguousarray(s.pos, np.float32)
    mo = np.ascontiguousarray(s.mol_offsets, np.int32)
    periodic = bool(np.any(s.pbc))
    cell = np.ascontiguousarray(s.cell, np.float32) if periodic else None
    pbc = np.ascontiguousarray(s.pbc, np.uint8) if periodic else None
    if out is None:
        out = (np.zeros(s.n_mol), np.zeros((s.n_atoms, 3), np.float32), np.zeros((s.n_mol, 3, 3)) if virial else None)
    E, F, W = out
    code = lib.fnn_energy_forces_host(ctx.h, s.n_atoms, s.n_mol, mo.ctypes.data, Z.ctypes.data, pos.ctypes.data,
                                      None if cell is None else cell.ctypes.data,
                                      None if pbc is None else pbc.ctypes.data, PRECISION[precision],
                                      E.ctypes.data, F.ctypes.data, None if W is None else W.ctypes.data,
                                      _stream(stream))
    ctx._check(code, "fnn_energy_forces_host")
    return E, F, W


def profile_enable(ctx: Context, on: bool = True):
    """fnn_profile_enable: bracket every kernel of this context with CUDA events on its stream."""
    ctx._check(lib.fnn_profile_enable(ctx.h, int(on)), "fnn_profile_enable")


def profile_read(ctx: Context) -> dict:
    """fnn_profile_read: {kernel name: (device ms summed, launches)} since the previous read."""
    cap = 128
    names = ctypes.create_string_buffer(48 * cap)
    ms = (ctypes.c_double * cap)()
    n = (ctypes.c_int64 * cap)()
    count = ctypes.c_int32(0)
    ctx._check(lib.fnn_profile_read(ctx.h, names, ms, n, cap, ctypes.byref(count)), "fnn_profile_read")
    out = {}
    for k in range(min(count.value, cap)):
        name = names.raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
        out[name] = (ms[k], n[k])
    return out


def launch_count(ctx: Context) -> int:
    """fnn_launch_count: kernels this context has launched since it was created."""
    n = ctypes.c_int64(0)
    ctx._check(lib.fnn_launch_count(ctx.h, ctypes.byref(n)), "fnn_launch_count")
    return n.value


def md_run(ctx: Context, system: DeviceSystem, vel, nl: NeighborList, precision: str, n_steps: int, dt_fs: float,
           rebuild_every: int = 10, E_hist=None, F=None, stream=None):
    """fnn_md_run: NVE velocity Verlet on the device; system.pos and vel ([N,4] float32) advance in place.
    Returns (E_hist [n_steps, n_mol] float64, F [N,3] of the last evaluation)."""
    import torch
    if E_hist is None:
        E_hist = torch.empty((n_steps, system.n_mol), dtype=torch.float64, device="cuda")
    if F is None:
        F = torch.empty((system.n_atoms, 3), dtype=torch.float32, device="cuda")
    cs = system.c()
    ctx._check(lib.fnn_md_run(ctx.h, ctypes.byref(cs), _ptr(system.pos), _ptr(vel), nl.h, PRECISION[precision],
                              int(n_steps), float(dt_fs), int(rebuild_every), _ptr(E_hist), _ptr(F), _stream(stream)),
               "fnn_md_run")
    return E_hist, F


def bead_system(s, x, device="cuda"):
    """The P beads of structure s at positions x [P, N, 3] as one batch of P structures (bead-major)."""
    from . import synth
    P, N = x.shape[0], s.n_atoms
    b = synth.Structures(np.tile(np.asarray(s.Z, np.int32), P), np.asarray(x, np.float32).reshape(P * N, 3),
                         np.arange(P + 1, dtype=np.int32) * N,
                         np.repeat(np.asarray(s.cell, np.float32).reshape(1, 9), P, 0),
                         np.repeat(np.asarray(s.pbc, np.uint8), P))
    return DeviceSystem.from_structures(b, device)


def rpmd_run(ctx: Context, beads: DeviceSystem, vel, nl: NeighborList, precision: str, n_beads: int, n_steps: int,
             dt_fs: float, temperature_K: float = 300.0, rebuild_every: int = 10, skin_guard: bool = True,
             counters: bool = False, stream=None):
    """fnn_rpmd_run: ring-polymer MD of the beads (a batch of n_beads structures, bead-major); beads.pos and
    vel ([P N, 4] float32) advance in place.  Returns (E_hist [n_steps, P], H_hist [n_steps], F, counters)."""
    import torch
    E_hist = torch.empty((n_steps, n_beads), dtype=torch.float64, device="cuda")
    H_hist = torch.empty((n_steps,), dtype=torch.float64, device="cuda")
    F = torch.empty((beads.n_atoms, 3), dtype=torch.float32, device="cuda")
    o = CRpmdOptions(int(n_beads), int(n_steps), float(dt_fs), float(temperature_K), int(rebuild_every),
                     int(bool(skin_guard)))
    c = CMdCounters()
    cs = beads.c()
    ctx._check(lib.fnn_rpmd_run(ctx.h, ctypes.byref(cs), _ptr(beads.pos), _ptr(vel), nl.h, PRECISION[precision],
                                ctypes.byref(o), _ptr(E_hist), _ptr(H_hist), _ptr(F),
                                ctypes.byref(c) if counters else None, _stream(stream)), "fnn_rpmd_run")
    cnt = {f: getattr(c, f) for f, _ in CMdCounters._fields_} if counters else None
    return E_hist, H_hist, F, cnt


def md_run_ex(ctx: Context, system: DeviceSystem, vel, nl: NeighborList, precision: str, n_steps: int, dt_fs: float,
              rebuild_every: int = 10, integrator: str = "nve", temperature_K: float = 300.0,
              friction_per_fs: float = 0.0, seed: int = 0, step0: int = 0, skin_guard: bool = True,
              kinetic: bool = False, counters: bool = False, stream=None):
    """fnn_md_run_ex: NVE velocity Verlet or BAOAB Langevin on the device, rebuilds on schedule and by the
    skin guard; system.pos and vel ([N,4] float32) advance in place.  Returns (E_hist [n_steps, n_mol],
    K_hist [n_steps, n_mol] or None, F [N,3] of the last evaluation, counters dict or None)."""
    import torch
    E_hist = torch.empty((n_steps, system.n_mol), dtype=torch.float64, device="cuda")
    K_hist = torch.empty((n_steps, system.n_mol), dtype=torch.float64, device="cuda") if kinetic else None
    F = torch.empty((system.n_atoms, 3), dtype=torch.float32, device="cuda")
    o = CMdOptions(int(n_steps), float(dt_fs), int(rebuild_every), int(bool(skin_guard)),
                   {"nve": 0, "langevin": 1}[integrator], float(temperature_K), float(friction_per_fs), int(seed),
                   int(step0))
    c = CMdCounters()
    cs = system.c()
    ctx._check(lib.fnn_md_run_ex(ctx.h, ctypes.byref(cs), _ptr(system.pos), _ptr(vel), nl.h, PRECISION[precision],
                                 ctypes.byref(o), _ptr(E_hist), _ptr(K_hist) if kinetic else None, _ptr(F),
                                 ctypes.byref(c) if counters else None, _stream(stream)), "fnn_md_run_ex")
    cnt = {f: getattr(c, f) for f, _ in CMdCounters._fields_} if counters else None
    return E_hist, K_hist, F, cnt


class Graph:
    """fnn_graph_*: one step (list rebuild when rebuild, then energies and forces) captured as a CUDA graph
    on a non-default stream; replays read the system's buffers at replay time."""

    def __init__(self, ctx: Context, system: DeviceSystem, nl: NeighborList, precision: str = "fp32x3",
                 virial: bool = True, rebuild: bool = True, stream=None):
        import torch
        self.ctx, self.system, self.nl = ctx, system, nl
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.E = torch.empty(system.n_mol, dtype=torch.float64, device="cuda")
        self.F = torch.empty((system.n_atoms, 3), dtype=torch.float32, device="cuda")
        self.W = torch.empty((system.n_mol, 3, 3), dtype=torch.float64, device="cuda") if virial else None
        self._cs = system.c()
        h = ctypes.c_void_p()
        self.h = None
        code = lib.fnn_graph_create(ctx.h, ctypes.byref(self._cs), nl.h, PRECISION[precision], _ptr(self.E),
                                    _ptr(self.F), _ptr(self.W), int(bool(rebuild)),
                                    ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        ctx._check(code, "fnn_graph_create")
        self.h = h
        k = ctypes.c_int64(0)
        lib.fnn_graph_kernels(self.h, ctypes.byref(k))
        self.kernels = k.value

    def launch(self):
        self.ctx._check(lib.fnn_graph_launch(self.h, ctypes.c_void_p(self.stream.cuda_stream)), "fnn_graph_launch")

    def close(self):
        if getattr(self, "h", None):
            lib.fnn_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """fnn_serve_*: continuous-batching MD service on a context (used exclusively while it lives)."""

    def __init__(self, ctx: Context, budget_bytes: int, precision: str = "bf16", rebuild_every: int = 10):
        self.ctx = ctx
        self.h = None
        h = ctypes.c_void_p()
        ctx._check(lib.fnn_serve_create(ctypes.byref(h), ctx.h, int(budget_bytes), PRECISION[precision],
                                        int(rebuild_every)), "fnn_serve_create")
        self.h = h
        self.n = {}

    def submit(self, s, vel=None, n_steps: int = 10, dt_fs: float = 0.5) -> int:
        """Queue one structure (a single-molecule synth.Structures); returns its ticket."""
        Z = np.ascontiguousarray(s.Z, np.int32)
        pos = np.ascontiguousarray(s.pos, np.float32)
        v = None if vel is None else np.ascontiguousarray(vel, np.float32)
        cell = np.ascontiguousarray(s.cell[0], np.float32) if bool(s.pbc[0]) else None
        rq = CRequest(s.n_atoms, Z.ctypes.data, pos.ctypes.data, None if v is None else v.ctypes.data,
                      None if cell is None else cell.ctypes.data, int(n_steps), float(dt_fs))
        t = ctypes.c_uint64(0)
        code = lib.fnn_serve_submit(self.h, ctypes.byref(rq), ctypes.byref(t))
        if code != FNN_OK:
            raise FnnError(code, "fnn_serve_submit")
        self.n[t.value] = (s.n_atoms, int(n_steps))
        return t.value

    def poll(self, ticket: int, timeout_s: float = 0.0, arrays: bool = True):
        """The result dict once done, else None (after waiting up to timeout_s).  With arrays=False only the
        timings and step count come back (nothing of the structure is copied)."""
        n, k = self.n[ticket]
        if arrays:
            out = {"energies": np.zeros(k), "pos": np.zeros((n, 3), np.float32),
                   "vel": np.zeros((n, 3), np.float32), "forces": np.zeros((n, 3), np.float32)}
            r = CResult(out["energies"].ctypes.data, out["pos"].ctypes.data, out["vel"].ctypes.data,
                        out["forces"].ctypes.data, 0.0, 0.0, 0)
        else:
            out = {}
            r = CResult(None, None, None, None, 0.0, 0.0, 0)
        code = lib.fnn_serve_poll(self.h, ticket, ctypes.byref(r), int(timeout_s * 1e6))
        if code == FNN_PENDING:
            return None
        if code != FNN_OK:
            del self.n[ticket]
            raise FnnError(code, "fnn_serve_poll")
        del self.n[ticket]
        out.update(latency_ms=r.latency_ms, queue_ms=r.queue_ms, n_steps_done=r.n_steps_done)
        return out

    def stats(self) -> dict:
        c = CServeCounters()
        code = lib.fnn_serve_stats(self.h, ctypes.byref(c))
        d = {f: getattr(c, f) for f, _ in CServeCounters._fields_}
        d["status"] = code
        return d

    def close(self):
        if getattr(self, "h", None):
            lib.fnn_serve_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
