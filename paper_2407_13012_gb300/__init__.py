"""GB300-native MaxCut-QAOA statevector simulator (arXiv 2407.13012, CUAOA) — Python binding.

A thin ctypes layer over ``libqaoa_gb300.so`` (declared in
``include/qaoa_gb300.h``).  It only marshals arguments: torch supplies device
memory and the current CUDA stream; every step of the computation runs in the
library's CUDA kernels.  There is no CPU fallback: if the library cannot be
loaded, importing this package raises.

Conventions (see the header): qubit j is bit j of the amplitude index;
C(z) = sum over edges of w_uv [z_u != z_v]; a layer is
psi *= exp(-i gamma C) followed by RX(2 beta) on every qubit.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import dataclass
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
_LIB_PATH = _PKG / "libqaoa_gb300.so"

QAOA_OK, QAOA_ERR_INVALID_ARG, QAOA_ERR_UNSUPPORTED, QAOA_ERR_CUDA, QAOA_ERR_TIMEOUT, QAOA_ERR_WORKSPACE = range(6)
C128, C64 = 0, 1
COST_I32, COST_F64 = 0, 1
WEIGHT_INT, WEIGHT_F64 = 0, 1
OP_COST, OP_LAYERS, OP_EXPECTATION, OP_SAMPLE, OP_GRADIENT, OP_OPTIMIZE, OP_LBFGS = range(7)
LBFGS_MAX_M = 16
MAX_N, MAX_P, MAX_TABLE_SPAN = 32, 64, 16384
BATCH_MAX_N, BATCH_MAX_P, BATCH_MAX_EDGES = 26, 12, 512

EXPORTS = [
    "qaoa_version", "qaoa_strerror", "qaoa_graph_check", "qaoa_workspace_size", "qaoa_cost_vector",
    "qaoa_apply_layers", "qaoa_expectation", "qaoa_expectation_host", "qaoa_sample", "qaoa_sample_host",
    "qaoa_gradient", "qaoa_gradient_host", "qaoa_launch_count", "qaoa_launch_count_reset",
    "qaoa_timing_enable", "qaoa_timing_read", "qaoa_gradient_dev", "qaoa_optimize_adam", "qaoa_expectation_noalloc",
    "qaoa_batch_workspace_size", "qaoa_batch_gradient", "qaoa_batch_autotune_workspace_size", "qaoa_batch_autotune",
    "qaoa_cost_vector_pubo", "qaoa_optimize_lbfgs", "qaoa_proposer_param_count", "qaoa_propose_workspace_size",
    "qaoa_propose_angles", "qaoa_xy_dim", "qaoa_xy_workspace_size", "qaoa_xy_cost_vector", "qaoa_xy_apply_layers",
    "qaoa_xy_expectation",
]


class QaoaError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_lib.qaoa_strerror(status).decode()} (status {status})")
        self.status = status


class GraphT(ct.Structure):
    _fields_ = [("n", ct.c_int32), ("m", ct.c_int64), ("uv", ct.POINTER(ct.c_int32)),
                ("w", ct.POINTER(ct.c_double)), ("weight_kind", ct.c_int32)]


class CostT(ct.Structure):
    _fields_ = [("C_dev", ct.c_void_p), ("dtype", ct.c_int32), ("cmin", ct.c_int64), ("cmax", ct.c_int64)]


def _load() -> ct.CDLL:
    from . import _build
    _build.build()  # no-op when the library matches the sources; raises if nvcc is missing
    lib = ct.CDLL(str(_LIB_PATH))
    vp, i32, i64, u64, dp, szp = ct.c_void_p, ct.c_int, ct.c_int64, ct.c_uint64, ct.POINTER(ct.c_double), ct.POINTER(ct.c_size_t)
    sig = {
        "qaoa_version": ([], i32),
        "qaoa_strerror": ([i32], ct.c_char_p),
        "qaoa_graph_check": ([ct.POINTER(GraphT), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64)], i32),
        "qaoa_workspace_size": ([i32, i32, i32, i32, i64, i64, szp], i32),
        "qaoa_cost_vector": ([ct.POINTER(GraphT), vp, i32, ct.POINTER(CostT), vp], i32),
        "qaoa_apply_layers": ([i32, i32, vp, ct.POINTER(CostT), dp, dp, i32, i32, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_expectation": ([i32, i32, vp, ct.POINTER(CostT), vp, vp, ct.c_size_t, vp], i32),
        "qaoa_expectation_host": ([i32, i32, vp, ct.POINTER(CostT), dp, vp, ct.c_size_t, vp], i32),
        "qaoa_expectation_noalloc": ([i32, i32, vp, ct.POINTER(CostT), vp, vp], i32),
        "qaoa_sample": ([i32, i32, vp, ct.POINTER(CostT), i64, u64, vp, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_sample_host": ([i32, i32, vp, ct.POINTER(CostT), i64, u64, vp, vp, vp, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_gradient": ([i32, i32, vp, vp, ct.POINTER(CostT), dp, dp, i32, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_gradient_host": ([i32, i32, vp, vp, ct.POINTER(CostT), dp, dp, i32, vp, dp, vp, ct.c_size_t, vp], i32),
        "qaoa_gradient_dev": ([i32, i32, vp, vp, ct.POINTER(CostT), vp, i32, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_optimize_adam": ([i32, i32, vp, vp, ct.POINTER(CostT), vp, i32, i64, ct.c_double, ct.c_double,
                                ct.c_double, ct.c_double, vp, vp, i32, vp, ct.c_size_t, vp], i32),
        "qaoa_optimizer_state_size": ([i32, i32, szp], i32),
        "qaoa_optimize_lbfgs": ([i32, i32, vp, vp, ct.POINTER(CostT), vp, i32, i64, i32, ct.c_double, vp, vp, vp,
                                 i32, vp, ct.c_size_t, vp], i32),
        "qaoa_proposer_param_count": ([i32], i64),
        "qaoa_propose_workspace_size": ([i32, ct.POINTER(GraphT), szp], i32),
        "qaoa_propose_angles": ([i32, ct.POINTER(GraphT), i32, vp, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_cost_vector_pubo": ([i32, i64, vp, dp, i32, vp, i32, ct.POINTER(CostT), vp], i32),
        "qaoa_batch_workspace_size": ([i32, i32, i32, ct.POINTER(GraphT), vp, szp], i32),
        "qaoa_batch_gradient": ([i32, i32, ct.POINTER(GraphT), dp, i32, vp, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_batch_autotune_workspace_size": ([i32, i32, i32, i32, szp], i32),
        "qaoa_batch_autotune": ([i32, i32, i32, i32, i32, vp, dp, vp, ct.c_size_t, vp], i32),
        "qaoa_xy_dim": ([i32, i32, ct.POINTER(ct.c_int64)], i32),
        "qaoa_xy_workspace_size": ([i32, i32, i32, i32, i64, szp], i32),
        "qaoa_xy_cost_vector": ([ct.POINTER(GraphT), i32, vp, i32, ct.POINTER(CostT), vp], i32),
        "qaoa_xy_apply_layers": ([i32, i32, i32, vp, ct.POINTER(CostT), dp, dp, i32, i32, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_xy_expectation": ([i32, i32, i32, vp, ct.POINTER(CostT), vp, vp, ct.c_size_t, vp], i32),
        "qaoa_xy_gradient_workspace_size": ([i32, i32, i32, i32, i64, szp], i32),
        "qaoa_xy_sample_workspace_size": ([i32, i32, szp], i32),
        "qaoa_xy_sample": ([i32, i32, i32, vp, ct.POINTER(CostT), i64, u64, vp, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_xy_gradient": ([i32, i32, i32, vp, vp, ct.POINTER(CostT), dp, dp, i32, vp, vp, ct.c_size_t, vp], i32),
        "qaoa_launch_count": ([], i64),
        "qaoa_launch_count_reset": ([], None),
        "qaoa_timing_enable": ([i32], i32),
        "qaoa_timing_read": ([dp, ct.POINTER(ct.c_int64), dp, ct.POINTER(ct.c_int64)], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


_lib = _load()
lib = _lib


def _check(status: int, where: str) -> None:
    if status != QAOA_OK:
        raise QaoaError(status, where)


def version() -> int:
    return _lib.qaoa_version()


# ---------------------------------------------------------------- graphs


@dataclass
class Graph:
    """MaxCut instance: n vertices, int32 edges (m, 2), float64 weights, integer flag."""
    n: int
    edges: np.ndarray
    weights: np.ndarray | None = None
    integer: bool = True

    def __post_init__(self):
        self.edges = np.ascontiguousarray(np.asarray(self.edges, dtype=np.int32).reshape(-1, 2))
        if self.weights is not None:
            self.weights = np.ascontiguousarray(np.asarray(self.weights, dtype=np.float64))

    @property
    def m(self) -> int:
        return len(self.edges)

    def as_struct(self) -> GraphT:
        """The C descriptor.  It points into this graph's edge and weight arrays, so it is kept
        (with references to those arrays) until one of the fields is replaced."""
        key = (self.edges, self.weights, self.n, self.integer)
        c = self.__dict__.get("_struct")
        if c is None or any(a is not b for a, b in zip(c[0][:2], key[:2])) or c[0][2:] != key[2:]:
            uv = self.edges.ctypes.data_as(ct.POINTER(ct.c_int32))
            w = self.weights.ctypes.data_as(ct.POINTER(ct.c_double)) if self.weights is not None else None
            c = (key, GraphT(self.n, self.m, uv, w, WEIGHT_INT if self.integer else WEIGHT_F64))
            self.__dict__["_struct"] = c
        return c[1]

    def check(self) -> tuple[int, int]:
        """Host-side validation; returns integer bounds (cmin, cmax) on C(z)."""
        lo, hi = ct.c_int64(), ct.c_int64()
        g = self.as_struct()
        _check(_lib.qaoa_graph_check(ct.byref(g), ct.byref(lo), ct.byref(hi)), "graph_check")
        return lo.value, hi.value


def workspace_size(n: int, dtype: int, op: int, p: int = 0, shots: int = 0, cost_span: int = 0) -> int:
    out = ct.c_size_t()
    _check(_lib.qaoa_workspace_size(n, dtype, op, p, shots, cost_span, ct.byref(out)), "workspace_size")
    return out.value


# ------------------------------------------------------------------ torch side

def _torch():
    import torch
    return torch


def _stream(device=None) -> int:
    torch = _torch()
    return torch.cuda.current_stream(device).cuda_stream


_ws_cache: dict = {}


def _workspace(nbytes: int, device):
    """A cached device scratch buffer of at least nbytes (torch-allocated).  One buffer per
    device serves every call of this binding on that device, so those calls must be ordered
    on one stream (the current stream, which the binding uses throughout)."""
    torch = _torch()
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise TypeError(f"state must be complex128 or complex64, got {t.dtype}")


def _require_cuda(*ts):
    for t in ts:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("tensors must be contiguous CUDA tensors")


@dataclass
class CostVector:
    """A device cost vector C(z) with its descriptor (dtype, integer bounds)."""
    C: object          # torch tensor int32 or float64, 2^n entries
    n: int
    cmin: int = 1
    cmax: int = 0

    @property
    def code(self) -> int:
        torch = _torch()
        return COST_I32 if self.C.dtype == torch.int32 else COST_F64

    @property
    def span(self) -> int:
        return self.cmax - self.cmin + 1 if self.cmax >= self.cmin else 0

    def struct(self) -> CostT:
        return CostT(self.C.data_ptr(), self.code, self.cmin, self.cmax)


def _cost_out(out, entries: int, tdt, device):
    """The caller's cost-vector buffer, or a new one: `entries` elements of dtype tdt (the
    kernels write exactly that many)."""
    torch = _torch()
    if out is None:
        return torch.empty(entries, dtype=tdt, device=device)
    if out.numel() != entries or out.dtype != tdt or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous {tdt} tensor of {entries} entries")
    return out


def cost_vector(graph: Graph, dtype: str = "i32", device="cuda", out=None) -> CostVector:
    """S1: C(z) for all z on the device (int32 exact, or float64)."""
    torch = _torch()
    tdt = torch.int32 if dtype == "i32" else torch.float64
    C = _cost_out(out, 1 << graph.n, tdt, device)
    _require_cuda(C)
    desc = CostT()
    g = graph.as_struct()
    code = COST_I32 if tdt == torch.int32 else COST_F64
    _check(_lib.qaoa_cost_vector(ct.byref(g), ct.c_void_p(C.data_ptr()), code, ct.byref(desc),
                                 ct.c_void_p(_stream(C.device))), "cost_vector")
    return CostVector(C, graph.n, desc.cmin, desc.cmax)


def _angles(gammas, betas):
    g = np.ascontiguousarray(np.asarray(gammas, dtype=np.float64).reshape(-1))
    b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64).reshape(-1))
    if len(g) != len(b):
        raise ValueError("gammas and betas must have the same length")
    return g, b, g.ctypes.data_as(ct.POINTER(ct.c_double)), b.ctypes.data_as(ct.POINTER(ct.c_double))


def cost_vector_pubo(n: int, masks, weights, integer: bool = True, dtype: str = "i32", device="cuda",
                     out=None) -> CostVector:
    """General PUBO cost (Eq. 3) on the device: C(z) = sum_t w_t [z & masks[t] == masks[t]]."""
    torch = _torch()
    m = np.ascontiguousarray(np.asarray(masks, dtype=np.uint32).reshape(-1))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(-1))
    if len(m) != len(w):
        raise ValueError("masks and weights must have the same length")
    tdt = torch.int32 if dtype == "i32" else torch.float64
    C = _cost_out(out, 1 << n, tdt, device)
    _require_cuda(C)
    desc = CostT()
    _check(_lib.qaoa_cost_vector_pubo(n, len(m), ct.c_void_p(m.ctypes.data), w.ctypes.data_as(ct.POINTER(ct.c_double)),
                                      WEIGHT_INT if integer else WEIGHT_F64, ct.c_void_p(C.data_ptr()),
                                      COST_I32 if tdt == torch.int32 else COST_F64, ct.byref(desc),
                                      ct.c_void_p(_stream(C.device))), "cost_vector_pubo")
    return CostVector(C, n, desc.cmin, desc.cmax)


def new_state(n: int, dtype: str = "c128", device="cuda"):
    torch = _torch()
    return torch.empty(1 << n, dtype=torch.complex128 if dtype == "c128" else torch.complex64, device=device)


def _state_qubits(psi, cost: CostVector | None = None, *others) -> int:
    """n of a 2^n-amplitude state.  The C ABI takes plain pointers, so check here that the
    state is a power-of-two length >= 2 and that the cost vector and any second state
    hold as many entries."""
    m = psi.numel()
    n = m.bit_length() - 1
    if m < 2 or m != 1 << n:
        raise ValueError(f"a state holds 2^n amplitudes (n >= 1), got {m}")
    if cost is not None:
        _check_cost_tensor(cost)
    for t in [psi] + ([cost.C] if cost is not None else []) + list(others):
        if t.numel() != m or not t.is_contiguous():
            raise ValueError(f"every buffer must be contiguous with 2^{n} = {m} entries, got {t.numel()}")
    return n


def _check_cost_tensor(cost: CostVector) -> None:
    torch = _torch()
    if cost.C.dtype not in (torch.int32, torch.float64):
        raise ValueError(f"cost vectors are int32 or float64, got {cost.C.dtype}")


def apply_layers(psi, cost: CostVector, gammas, betas, init: bool = True, expect: bool = False):
    """S2+S3 in place; returns the device tensor [<C>, norm] when expect=True."""
    torch = _torch()
    _require_cuda(psi)
    n = _state_qubits(psi, cost)
    g, b, gp, bp = _angles(gammas, betas)
    dt = _dtype_code(psi)
    ws_n = workspace_size(n, dt, OP_LAYERS, len(g), 0, cost.span)
    ws = _workspace(ws_n, psi.device)
    out = torch.empty(2, dtype=torch.float64, device=psi.device) if expect else None
    cs = cost.struct()
    _check(_lib.qaoa_apply_layers(n, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), gp, bp, len(g), int(init),
                                  ct.c_void_p(out.data_ptr() if out is not None else 0),
                                  ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))),
           "apply_layers")
    return out


def expectation(psi, cost: CostVector):
    """S4: device tensor [<C>, <psi|psi>]."""
    torch = _torch()
    _require_cuda(psi)
    n = _state_qubits(psi, cost)
    dt = _dtype_code(psi)
    ws = _workspace(workspace_size(n, dt, OP_EXPECTATION), psi.device)
    out = torch.empty(2, dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_expectation(n, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), ct.c_void_p(out.data_ptr()),
                                 ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))),
           "expectation")
    return out


def sample(psi, cost: CostVector, shots: int, seed: int):
    """S5+S6: (z uint64 as int64 tensor, cost float64 tensor) on the device, in draw order."""
    torch = _torch()
    _require_cuda(psi)
    n = _state_qubits(psi, cost)
    dt = _dtype_code(psi)
    ws = _workspace(workspace_size(n, dt, OP_SAMPLE, 0, shots), psi.device)
    z = torch.empty(max(shots, 1), dtype=torch.int64, device=psi.device)
    cz = torch.empty(max(shots, 1), dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_sample(n, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), shots, ct.c_uint64(seed & (2**64 - 1)),
                            ct.c_void_p(z.data_ptr()), ct.c_void_p(cz.data_ptr()), ct.c_void_p(ws.data_ptr()),
                            ws.numel(), ct.c_void_p(_stream(psi.device))), "sample")
    return z[:shots], cz[:shots]


def gradient(psi, lam, cost: CostVector, gammas, betas):
    """S7: device tensor [E, norm, dE/dgamma_1..p, dE/dbeta_1..p] (psi ends uncomputed)."""
    torch = _torch()
    _require_cuda(psi, lam)
    n = _state_qubits(psi, cost, lam)
    g, b, gp, bp = _angles(gammas, betas)
    dt = _dtype_code(psi)
    if lam.dtype != psi.dtype or lam.numel() != psi.numel():
        raise ValueError("lambda buffer must match psi")
    ws = _workspace(workspace_size(n, dt, OP_GRADIENT, len(g), 0, cost.span), psi.device)
    out = torch.empty(2 * len(g) + 2, dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_gradient(n, dt, ct.c_void_p(psi.data_ptr()), ct.c_void_p(lam.data_ptr()), ct.byref(cs), gp, bp,
                              len(g), ct.c_void_p(out.data_ptr()), ct.c_void_p(ws.data_ptr()), ws.numel(),
                              ct.c_void_p(_stream(psi.device))), "gradient")
    return out


def gradient_dev(psi, lam, cost: CostVector, angles):
    """S7 with device-resident angles [gamma_1..p, beta_1..p] (float64 CUDA tensor)."""
    torch = _torch()
    _require_cuda(psi, lam, angles)
    _check_angles(angles)
    n = _state_qubits(psi, cost, lam)
    p = angles.numel() // 2
    dt = _dtype_code(psi)
    ws = _workspace(workspace_size(n, dt, OP_GRADIENT, p, 0, cost.span), psi.device)
    out = torch.empty(2 * p + 2, dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_gradient_dev(n, dt, ct.c_void_p(psi.data_ptr()), ct.c_void_p(lam.data_ptr()), ct.byref(cs),
                                  ct.c_void_p(angles.data_ptr()), p, ct.c_void_p(out.data_ptr()),
                                  ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))),
           "gradient_dev")
    return out


class QAOAExpectation:
    """E(angles) = <C> of the depth-p state as a differentiable torch function.

    Forward runs the adjoint pass once (qaoa_gradient_dev) and keeps dE/dangles for the
    backward; angles = [gamma_1..p, beta_1..p] on the device (float64).  The state and
    lambda buffers are scratch owned by this object.
    """

    def __init__(self, cost: CostVector, dtype: str = "c128"):
        self.cost = cost
        self.psi = new_state(cost.n, dtype, cost.C.device)
        self.lam = new_state(cost.n, dtype, cost.C.device)
        torch = _torch()

        class _Fn(torch.autograd.Function):
            @staticmethod
            def forward(ctx, angles):
                out = gradient_dev(self.psi, self.lam, self.cost, angles.detach().contiguous())
                ctx.save_for_backward(out[2:].clone())
                return out[0].clone()

            @staticmethod
            def backward(ctx, grad_out):
                (g,) = ctx.saved_tensors
                return grad_out * g

        self._fn = _Fn

    def __call__(self, angles):
        return self._fn.apply(angles)


OPTIMIZER_ADAM, OPTIMIZER_LBFGS = 0, 1


def optimizer_state(kind: str, p: int, device="cuda"):
    """A zeroed device buffer for an optimiser's state ("adam" or "lbfgs"), for checkpoints:
    pass it as `state`, copy it (and the angles) to save, pass it back with resume=True."""
    torch = _torch()
    nbytes = ct.c_size_t()
    _check(_lib.qaoa_optimizer_state_size(OPTIMIZER_ADAM if kind == "adam" else OPTIMIZER_LBFGS, p,
                                          ct.byref(nbytes)), "optimizer_state_size")
    return torch.zeros(nbytes.value // 8, dtype=torch.float64, device=device)


def _check_angles(angles) -> None:
    torch = _torch()
    if angles.dtype != torch.float64 or angles.numel() < 2 or angles.numel() % 2 or not angles.is_contiguous():
        raise ValueError("angles must be a contiguous float64 tensor of length 2p, p >= 1")


def _check_optimizer_args(kind: str, cost: CostVector, angles, state) -> None:
    """Device buffers of the optimiser loops: the angles, the cost vector (2^n entries) and
    an optional state buffer at least optimizer_state(kind, p) long."""
    torch = _torch()
    _check_angles(angles)
    _check_cost_tensor(cost)
    if cost.C.numel() != 1 << cost.n or not cost.C.is_contiguous():
        raise ValueError(f"the cost vector must hold 2^{cost.n} entries")
    if state is not None:
        nbytes = ct.c_size_t()
        _check(_lib.qaoa_optimizer_state_size(OPTIMIZER_ADAM if kind == "adam" else OPTIMIZER_LBFGS,
                                              angles.numel() // 2, ct.byref(nbytes)), "optimizer_state_size")
        if state.dtype != torch.float64 or not state.is_contiguous() or state.numel() * 8 < nbytes.value:
            raise ValueError(f"state must be a contiguous float64 tensor of at least {nbytes.value // 8} values")


def optimize_adam(cost: CostVector, angles, steps: int, lr: float = 0.01, betas=(0.9, 0.999), eps: float = 1e-8,
                  dtype: str = "c128", history: bool = True, state=None, resume: bool = False):
    """Adam ascent on <C> for `steps` steps, entirely on the device (one CUDA graph per
    step replayed).  angles: float64 CUDA tensor [gamma, beta] updated in place.  state /
    resume: see optimizer_state.
    Returns the history tensor (steps x (4p + 2)): [E, norm, dE/dgamma, dE/dbeta, gamma, beta]."""
    torch = _torch()
    _require_cuda(angles)
    _check_optimizer_args("adam", cost, angles, state)
    p = angles.numel() // 2
    n = cost.n
    dt = C128 if dtype == "c128" else C64
    psi = new_state(n, dtype, angles.device)
    lam = new_state(n, dtype, angles.device)
    ws = _workspace(workspace_size(n, dt, OP_OPTIMIZE, p, 0, cost.span), angles.device)
    hist = torch.empty((max(steps, 1), 4 * p + 2), dtype=torch.float64, device=angles.device) if history else None
    cs = cost.struct()
    _check(_lib.qaoa_optimize_adam(n, dt, ct.c_void_p(psi.data_ptr()), ct.c_void_p(lam.data_ptr()), ct.byref(cs),
                                   ct.c_void_p(angles.data_ptr()), p, steps, lr, betas[0], betas[1], eps,
                                   ct.c_void_p(hist.data_ptr() if hist is not None else 0),
                                   ct.c_void_p(state.data_ptr() if state is not None else 0), int(resume),
                                   ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(angles.device))),
           "optimize_adam")
    return hist[:steps] if hist is not None else None


def _tiles_arg(tiles):
    if tiles is None:
        return None, None
    arr = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1))
    if len(arr) != MAX_N + 1:
        raise ValueError(f"tiles must have {MAX_N + 1} entries (indexed by n)")
    return arr, arr.ctypes.data_as(ct.c_void_p)


def batch_gradient(graphs, angles, dtype: str = "c128", tiles=None, device="cuda"):
    """Batched S7 for many small graphs (grouped sweeps per size, one persistent launch for the rest).

    graphs: sequence of Graph; angles: (ngraphs, 2p) host array, row i = [gamma | beta] of
    graph i.  Returns a (ngraphs, 2p + 2) float64 device tensor, row i = [E, norm,
    dE/dgamma_1..p, dE/dbeta_1..p] of graph i."""
    torch = _torch()
    ng = len(graphs)
    ang = np.ascontiguousarray(np.asarray(angles, dtype=np.float64).reshape(ng, -1))
    p = ang.shape[1] // 2
    dt = C128 if dtype == "c128" else C64
    structs = (GraphT * max(ng, 1))(*[g.as_struct() for g in graphs])
    tarr, tptr = _tiles_arg(tiles)
    nbytes = ct.c_size_t()
    _check(_lib.qaoa_batch_workspace_size(dt, p, ng, structs, tptr, ct.byref(nbytes)), "batch_workspace_size")
    ws = _workspace(nbytes.value, device)
    out = torch.empty((max(ng, 1), 2 * p + 2), dtype=torch.float64, device=device)
    _check(_lib.qaoa_batch_gradient(dt, ng, structs, ang.ctypes.data_as(ct.POINTER(ct.c_double)), p, tptr,
                                    ct.c_void_p(out.data_ptr()), ct.c_void_p(ws.data_ptr()), ws.numel(),
                                    ct.c_void_p(_stream(device))), "batch_gradient")
    return out[:ng]


def batch_autotune(dtype: str = "c128", p: int = 3, n_lo: int = 8, n_hi: int = 20, graphs_per_n: int = 304,
                   device="cuda"):
    """Measured tile choice per qubit count for batch_gradient: (tiles[MAX_N + 1], ms[(MAX_N + 1), 2])."""
    dt = C128 if dtype == "c128" else C64
    nbytes = ct.c_size_t()
    _check(_lib.qaoa_batch_autotune_workspace_size(dt, p, n_hi, graphs_per_n, ct.byref(nbytes)),
           "batch_autotune_workspace_size")
    ws = _workspace(nbytes.value, device)
    tiles = np.zeros(MAX_N + 1, dtype=np.int32)
    ms = np.zeros(2 * (MAX_N + 1), dtype=np.float64)
    _check(_lib.qaoa_batch_autotune(dt, p, n_lo, n_hi, graphs_per_n, ct.c_void_p(tiles.ctypes.data),
                                    ms.ctypes.data_as(ct.POINTER(ct.c_double)), ct.c_void_p(ws.data_ptr()),
                                    ws.numel(), ct.c_void_p(_stream(device))), "batch_autotune")
    return tiles, ms.reshape(MAX_N + 1, 2)


def optimize_lbfgs(cost: CostVector, angles, max_evals: int = 200, m: int = 10, gtol: float = 1e-6,
                   dtype: str = "c128", state=None, resume: bool = False):
    """L-BFGS ascent on <C>, on the device (graph replay; the host polls a stop flag every 16
    evaluations).  angles: float64 CUDA tensor [gamma, beta], updated in place to the best
    accepted point.  state / resume: see optimizer_state.  Returns (history of this call's
    evaluations (rows x (4p + 2)) device tensor, info dict with running totals)."""
    torch = _torch()
    _require_cuda(angles)
    _check_optimizer_args("lbfgs", cost, angles, state)
    p = angles.numel() // 2
    n = cost.n
    dt = C128 if dtype == "c128" else C64
    psi = new_state(n, dtype, angles.device)
    lam = new_state(n, dtype, angles.device)
    ws = _workspace(workspace_size(n, dt, OP_LBFGS, p, 0, cost.span), angles.device)
    hist = torch.zeros((max(max_evals, 1), 4 * p + 2), dtype=torch.float64, device=angles.device)
    info = torch.zeros(4, dtype=torch.float64, device=angles.device)
    cs = cost.struct()
    before = int(state[3].item()) if (resume and state is not None) else 0
    _check(_lib.qaoa_optimize_lbfgs(n, dt, ct.c_void_p(psi.data_ptr()), ct.c_void_p(lam.data_ptr()), ct.byref(cs),
                                    ct.c_void_p(angles.data_ptr()), p, max_evals, m, gtol,
                                    ct.c_void_p(hist.data_ptr()), ct.c_void_p(info.data_ptr()),
                                    ct.c_void_p(state.data_ptr() if state is not None else 0), int(resume),
                                    ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(angles.device))),
           "optimize_lbfgs")
    i = info.cpu().numpy()
    res = {"E": float(i[0]), "iterations": int(i[1]), "evaluations": int(i[2]),
           "status": ("evaluations used up", "converged", "no progress")[int(i[3])]}
    return hist[:res["evaluations"] - before], res


def proposer_param_count(p: int) -> int:
    return int(_lib.qaoa_proposer_param_count(p))


def propose_angles(graphs, params, p: int, device="cuda"):
    """Learned starting angles for each graph from the fused network kernel: a (ngraphs, 2p)
    float64 device tensor, rows [gamma | beta].  params: float32 CUDA tensor of
    proposer_param_count(p) values."""
    torch = _torch()
    _require_cuda(params)
    if params.dtype != torch.float32 or params.numel() != proposer_param_count(p):
        raise ValueError("params must be a float32 tensor of proposer_param_count(p) values")
    ng = len(graphs)
    structs = (GraphT * max(ng, 1))(*[g.as_struct() for g in graphs])
    nbytes = ct.c_size_t()
    _check(_lib.qaoa_propose_workspace_size(ng, structs, ct.byref(nbytes)), "propose_workspace_size")
    ws = _workspace(nbytes.value, device)
    out = torch.empty((max(ng, 1), 2 * p), dtype=torch.float64, device=device)
    _check(_lib.qaoa_propose_angles(ng, structs, p, ct.c_void_p(params.data_ptr()), ct.c_void_p(out.data_ptr()),
                                    ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(device))),
           "propose_angles")
    return out[:ng]


# ------------------------------------------- Hamming-weight subspace, ring XY mixer


def xy_dim(n: int, k: int) -> int:
    """binom(n, k): amplitudes of a state on F_k = {z : popcount(z) = k}."""
    d = ct.c_int64()
    _check(_lib.qaoa_xy_dim(n, k, ct.byref(d)), "xy_dim")
    return d.value


def xy_cost_vector(graph: Graph, k: int, dtype: str = "i32", device="cuda", out=None) -> CostVector:
    """C(z) of every z in F_k, in rank order (increasing z), on the device."""
    torch = _torch()
    tdt = torch.int32 if dtype == "i32" else torch.float64
    C = _cost_out(out, xy_dim(graph.n, k), tdt, device)
    _require_cuda(C)
    desc = CostT()
    g = graph.as_struct()
    _check(_lib.qaoa_xy_cost_vector(ct.byref(g), k, ct.c_void_p(C.data_ptr()), COST_I32 if tdt == torch.int32 else COST_F64,
                                    ct.byref(desc), ct.c_void_p(_stream(C.device))), "xy_cost_vector")
    return CostVector(C, graph.n, desc.cmin, desc.cmax)


def xy_new_state(n: int, k: int, dtype: str = "c128", device="cuda"):
    torch = _torch()
    return torch.empty(xy_dim(n, k), dtype=torch.complex128 if dtype == "c128" else torch.complex64, device=device)


def _xy_workspace(n: int, k: int, dt: int, p: int, span: int, device):
    b = ct.c_size_t()
    _check(_lib.qaoa_xy_workspace_size(n, k, dt, p, span, ct.byref(b)), "xy_workspace_size")
    return _workspace(b.value, device)


def _xy_sizes(n: int, k: int, psi, cost: CostVector) -> None:
    """The C ABI takes plain pointers: check here that both buffers hold binom(n, k) entries."""
    d = xy_dim(n, k)
    _check_cost_tensor(cost)
    if psi.numel() != d or cost.C.numel() != d or not psi.is_contiguous() or not cost.C.is_contiguous():
        raise ValueError(f"state and cost vector must hold binom({n}, {k}) = {d} entries, "
                         f"got {psi.numel()} and {cost.C.numel()}")


def xy_apply_layers(psi, n: int, k: int, cost: CostVector, gammas, betas, init: bool = True, expect: bool = False):
    """p layers of phase + ring XY mixer in place on a subspace state; returns the device
    tensor [<C>, norm] when expect=True."""
    torch = _torch()
    _xy_sizes(n, k, psi, cost)
    _require_cuda(psi)
    g, b, gp, bp = _angles(gammas, betas)
    dt = _dtype_code(psi)
    ws = _xy_workspace(n, k, dt, len(g), cost.span, psi.device)
    out = torch.empty(2, dtype=torch.float64, device=psi.device) if expect else None
    cs = cost.struct()
    _check(_lib.qaoa_xy_apply_layers(n, k, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), gp, bp, len(g), int(init),
                                     ct.c_void_p(out.data_ptr() if out is not None else 0),
                                     ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))),
           "xy_apply_layers")
    return out


def xy_expectation(psi, n: int, k: int, cost: CostVector):
    """Device tensor [<C>, <psi|psi>] of a subspace state."""
    torch = _torch()
    _xy_sizes(n, k, psi, cost)
    _require_cuda(psi)
    dt = _dtype_code(psi)
    ws = _xy_workspace(n, k, dt, 0, 0, psi.device)
    out = torch.empty(2, dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_xy_expectation(n, k, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), ct.c_void_p(out.data_ptr()),
                                    ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))),
           "xy_expectation")
    return out


def xy_gradient(psi, lam, n: int, k: int, cost: CostVector, gammas, betas):
    """Adjoint gradient on the Hamming-weight subspace: runs the forward layers from the Dicke
    state in psi, lambda in lam (both binom(n, k) entries, same dtype), and returns the device
    tensor [E, norm, dE/dgamma_1..p, dE/dbeta_1..p]."""
    torch = _torch()
    _xy_sizes(n, k, psi, cost)
    _require_cuda(psi, lam)
    if lam.dtype != psi.dtype or lam.numel() != psi.numel() or not lam.is_contiguous():
        raise ValueError("lambda buffer must match psi")
    if lam.data_ptr() == psi.data_ptr():
        raise ValueError("psi and lambda must be distinct buffers")
    g, b, gp, bp = _angles(gammas, betas)
    dt = _dtype_code(psi)
    nb = ct.c_size_t()
    _check(_lib.qaoa_xy_gradient_workspace_size(n, k, dt, len(g), cost.span, ct.byref(nb)),
           "xy_gradient_workspace_size")
    ws = _workspace(nb.value, psi.device)
    out = torch.empty(2 * len(g) + 2, dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_xy_gradient(n, k, dt, ct.c_void_p(psi.data_ptr()), ct.c_void_p(lam.data_ptr()), ct.byref(cs),
                                 gp, bp, len(g), ct.c_void_p(out.data_ptr()), ct.c_void_p(ws.data_ptr()), ws.numel(),
                                 ct.c_void_p(_stream(psi.device))), "xy_gradient")
    return out


def xy_sample(psi, n: int, k: int, cost: CostVector, shots: int, seed: int):
    """Samples of a subspace state: (z bitstrings with k ones as an int64 tensor, cost float64
    tensor) on the device, in draw order."""
    torch = _torch()
    _xy_sizes(n, k, psi, cost)
    _require_cuda(psi)
    dt = _dtype_code(psi)
    nb = ct.c_size_t()
    _check(_lib.qaoa_xy_sample_workspace_size(n, k, ct.byref(nb)), "xy_sample_workspace_size")
    ws = _workspace(nb.value, psi.device)
    z = torch.empty(max(shots, 1), dtype=torch.int64, device=psi.device)
    cz = torch.empty(max(shots, 1), dtype=torch.float64, device=psi.device)
    cs = cost.struct()
    _check(_lib.qaoa_xy_sample(n, k, dt, ct.c_void_p(psi.data_ptr()), ct.byref(cs), shots,
                               ct.c_uint64(seed & (2**64 - 1)), ct.c_void_p(z.data_ptr()), ct.c_void_p(cz.data_ptr()),
                               ct.c_void_p(ws.data_ptr()), ws.numel(), ct.c_void_p(_stream(psi.device))), "xy_sample")
    return z[:shots], cz[:shots]


def launch_count() -> int:
    return _lib.qaoa_launch_count()


def launch_count_reset() -> None:
    _lib.qaoa_launch_count_reset()


def timing_enable(on: bool) -> None:
    _check(_lib.qaoa_timing_enable(int(on)), "timing_enable")


def timing_read():
    """Per kernel class [sweep, cost, sample, other]: (ms, launches, algorithmic bytes), dropped."""
    ms = (ct.c_double * 4)()
    la = (ct.c_int64 * 4)()
    by = (ct.c_double * 4)()
    dr = ct.c_int64()
    _check(_lib.qaoa_timing_read(ms, la, by, ct.byref(dr)), "timing_read")
    return list(ms), list(la), list(by), dr.value


def linear_ramp(p: int):
    """Constant-speed schedule (Sec. II-A): gamma_i = i/p, beta_i = 1 - i/p for i = 1..p."""
    i = np.arange(1, p + 1, dtype=np.float64)
    return i / p, 1.0 - i / p
