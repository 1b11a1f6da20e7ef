"""GB300-native Friends-of-Friends hot path (jFoF, arXiv 2510.26851).

Thin Python binding over the C ABI in ``include/jfof.h`` (``_build/libjfof.so``,
hand-written sm_103a kernels).  This module only marshals arguments: every step
of the path runs in the library's CUDA kernels.  There is no CPU fallback: if
the library is missing or no GPU is present, calls raise.

PyTorch supplies device memory (tensors) and the current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libjfof.so")

JFOF_OK, JFOF_EINVAL, JFOF_ERANGE, JFOF_ENOMEM, JFOF_ECUDA, JFOF_ETIMEOUT, JFOF_EOVERFLOW = range(7)
JFOF_WRAP = 1

# Every symbol the header declares (checked by the tests).
EXPORTED = [
    "jfof_create", "jfof_destroy", "jfof_set_stream", "jfof_sync", "jfof_strerror",
    "jfof_set_loop_budget", "jfof_set_cell_classes", "jfof_set_cta_shape", "jfof_trace_enable", "jfof_trace_read", "jfof_max_cells_per_axis", "jfof_default_cells_per_axis",
    "jfof_fof_bytes", "jfof_bin_cells", "jfof_link", "jfof_groups_bytes", "jfof_groups",
    "jfof_halo_props", "jfof_halo_props_backward", "jfof_fof_all_bytes", "jfof_fof",
    "jfof_prob_coef", "jfof_pairs_bytes", "jfof_pairs", "jfof_reinforce_sample_bytes",
    "jfof_reinforce_sample", "jfof_reinforce_grad_bytes", "jfof_reinforce_grad", "jfof_eval_exp",
    "jfof_eval_edge_uniform", "jfof_batch_bytes", "jfof_fof_batched", "jfof_autotune",
    "jfof_fof_static", "jfof_fof_host", "jfof_slab_select", "jfof_merge_labels", "jfof_fof_stream_bytes",
    "jfof_fof_stream", "jfof_halo_decoration", "jfof_halo_decoration_backward", "jfof_soft_hmf_bytes",
    "jfof_soft_hmf", "jfof_soft_hmf_backward", "jfof_subhalos_bytes", "jfof_subhalos",
]


class JfofError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


class Cells(ctypes.Structure):
    """Mirror of ``jfof_cells`` (views into the caller's workspace)."""
    _fields_ = [("n", ctypes.c_int64), ("n_axis", ctypes.c_int32), ("brick", ctypes.c_int32),
                ("L", ctypes.c_float), ("b", ctypes.c_float), ("flags", ctypes.c_uint32),
                ("small_threshold", ctypes.c_int32), ("dense_threshold", ctypes.c_int32),
                ("spos", ctypes.c_void_p),
                ("cell_start", ctypes.c_void_p), ("n_cells_table", ctypes.c_int64),
                ("workspace", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None
_ctx = {}


def _declare(lib):
    c = ctypes
    vp, i32, i64, u32, f32, sz = c.c_void_p, c.c_int32, c.c_int64, c.c_uint32, c.c_float, c.c_size_t
    P = c.POINTER
    sig = {
        "jfof_create": [P(vp), c.c_int, vp],
        "jfof_destroy": [vp],
        "jfof_set_stream": [vp, vp],
        "jfof_sync": [vp],
        "jfof_set_loop_budget": [vp, i64],
        "jfof_set_cell_classes": [vp, i32, i32],
        "jfof_set_cta_shape": [vp, i32],
        "jfof_trace_enable": [vp, c.c_int],
        "jfof_trace_read": [vp, c.c_char_p, sz, P(sz)],
        "jfof_max_cells_per_axis": [f32, f32, P(i32)],
        "jfof_default_cells_per_axis": [i64, f32, f32, P(i32)],
        "jfof_fof_bytes": [i64, i32, P(sz)],
        "jfof_bin_cells": [vp, vp, i64, f32, f32, i32, u32, vp, sz, P(Cells)],
        "jfof_link": [vp, P(Cells), vp],
        "jfof_groups_bytes": [i64, P(sz)],
        "jfof_groups": [vp, vp, i64, i32, vp, sz, vp, vp, vp, vp, vp],
        "jfof_halo_props": [vp, vp, vp, i64, f32, u32, vp, vp, vp, i64, f32, vp, vp, vp, vp],
        "jfof_halo_props_backward": [vp, vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp],
        "jfof_fof_all_bytes": [i64, i32, P(sz)],
        "jfof_fof": [vp, vp, i64, f32, f32, i32, u32, i32, vp, sz, vp, vp, vp, vp, vp, vp],
        "jfof_prob_coef": [f32, i32, f32, f32, P(f32)],
        "jfof_pairs_bytes": [i64, f32, f32, P(sz)],
        "jfof_pairs": [vp, vp, i64, f32, f32, f32, i32, f32, u32, vp, sz, i64, vp, vp, vp, vp, vp],
        "jfof_reinforce_sample_bytes": [i64, P(sz)],
        "jfof_reinforce_sample": [vp, i64, vp, vp, vp, i64, i32, c.c_uint64, i32, vp, sz, vp, vp],
        "jfof_reinforce_grad_bytes": [i64, i64, P(sz)],
        "jfof_reinforce_grad": [vp, vp, i64, f32, u32, vp, vp, vp, vp, i64, i32, c.c_uint64, vp, i32,
                                f32, vp, sz, vp],
        "jfof_eval_exp": [vp, vp, vp, i64],
        "jfof_eval_edge_uniform": [vp, c.c_uint64, vp, vp, vp, vp, i64],
        "jfof_batch_bytes": [vp, i32, vp, vp, vp, i32, P(sz)],
        "jfof_fof_batched": [vp, vp, vp, i32, vp, vp, vp, vp, vp, vp, u32, i32, vp, sz, vp, vp, vp, i32],
        "jfof_autotune": [vp, vp, i64, f32, f32, u32, i32, vp, sz, vp, vp, vp, i32, i32, vp, sz, P(i32),
                          P(i32), P(i32), P(i32), P(f32)],
        "jfof_fof_static": [vp, vp, i64, f32, f32, i32, u32, i32, vp, vp, vp, vp, vp, vp],
        "jfof_fof_host": [vp, vp, vp, i64, f32, f32, i32, u32, i32, f32, vp, vp, vp, sz, vp, vp, vp, vp, vp,
                          vp, vp, vp, vp, vp],
        "jfof_slab_select": [vp, i64, f32, f32, i32, i32, i32, vp, vp, P(i64)],
        "jfof_merge_labels": [i64, vp, i64, vp, vp, vp],
        "jfof_fof_stream_bytes": [vp, i64, f32, f32, i32, i32, P(sz)],
        "jfof_fof_stream": [vp, vp, i64, f32, f32, i32, i32, i32, vp, sz, vp, vp, P(i64)],
        "jfof_halo_decoration": [vp, vp, i64, f32, u32, vp, vp, vp, i64, vp, vp],
        "jfof_halo_decoration_backward": [vp, vp, vp, vp, i64, f32, u32, vp, vp, vp, vp],
        "jfof_soft_hmf_bytes": [i64, i32, P(sz)],
        "jfof_soft_hmf": [vp, vp, vp, i64, f32, vp, i32, f32, vp, sz, vp],
        "jfof_soft_hmf_backward": [vp, vp, vp, i64, f32, vp, vp, i32, f32, f32, vp, vp],
        "jfof_subhalos_bytes": [i64, P(sz)],
        "jfof_subhalos": [vp, vp, vp, i64, f32, u32, vp, vp, vp, i64, f32, f32, vp, sz, vp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = c.c_int
    lib.jfof_strerror.argtypes = [c.c_int]
    lib.jfof_strerror.restype = c.c_char_p
    return lib


def library():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libjfof.so not built ({LIB_PATH}); run "
                                   "python -m paper_2510_26851_gb300.build")
            _lib = _declare(ctypes.CDLL(LIB_PATH))
        return _lib


def strerror(code: int) -> str:
    try:
        return library().jfof_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def _check(code: int, where: str):
    if code != JFOF_OK:
        raise JfofError(code, where)


def context(device=None):
    """Per-device library context bound to torch's current stream."""
    if not torch.cuda.is_available():
        raise RuntimeError("jfof needs a CUDA GPU; there is no CPU fallback")
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    dev = 0 if dev is None else dev
    lib = library()
    with _lock:
        h = _ctx.get(dev)
        if h is None:
            h = ctypes.c_void_p()
            _check(lib.jfof_create(ctypes.byref(h), dev, None), "jfof_create")
            _ctx[dev] = h
    stream = torch.cuda.current_stream(dev).cuda_stream
    _check(lib.jfof_set_stream(h, ctypes.c_void_p(stream)), "jfof_set_stream")
    return h


def sync(device=None):
    """Wait for queued work; raise the latched device error, if any."""
    h = context(device)
    _check(library().jfof_sync(h), "device status")


def set_loop_budget(iterations: int, device=None):
    _check(library().jfof_set_loop_budget(context(device), int(iterations)), "jfof_set_loop_budget")


def set_cell_classes(small_max: int = 16, dense_over: int = -1, device=None):
    """Link-step cell classes: <= small_max particles "small", > dense_over
    "dense" (sub-cell path; 0 disables it; -1: 160 above 2^23 particles, 96
    below), the rest "medium"."""
    _check(library().jfof_set_cell_classes(context(device), int(small_max), int(dense_over)),
           "jfof_set_cell_classes")


def trace_enable(on: bool = True, device=None):
    """Record CUDA events around every library kernel launch."""
    _check(library().jfof_trace_enable(context(device), 1 if on else 0), "jfof_trace_enable")


def trace_read(device=None) -> dict:
    """Synchronise and return {kernel: (launches, total_ms)} since the last read."""
    buf = ctypes.create_string_buffer(1 << 16)
    n = ctypes.c_size_t()
    _check(library().jfof_trace_read(context(device), buf, len(buf), ctypes.byref(n)),
           "jfof_trace_read")
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, shape=None, name="tensor"):
    if t is None:
        return
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")


def max_cells_per_axis(L: float, b: float) -> int:
    n = ctypes.c_int32()
    _check(library().jfof_max_cells_per_axis(L, b, ctypes.byref(n)), "jfof_max_cells_per_axis")
    return n.value


def default_cells_per_axis(N: int, L: float, b: float) -> int:
    n = ctypes.c_int32()
    _check(library().jfof_default_cells_per_axis(N, L, b, ctypes.byref(n)),
           "jfof_default_cells_per_axis")
    return n.value


def fof_bytes(N: int, n_axis: int) -> int:
    s = ctypes.c_size_t()
    _check(library().jfof_fof_bytes(N, n_axis, ctypes.byref(s)), "jfof_fof_bytes")
    return s.value


def groups_bytes(N: int) -> int:
    s = ctypes.c_size_t()
    _check(library().jfof_groups_bytes(N, ctypes.byref(s)), "jfof_groups_bytes")
    return s.value


def _ws(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


@dataclass
class CellGrid:
    cells: Cells
    workspace: torch.Tensor  # keeps the memory the views point into alive


def bin_cells(pos: torch.Tensor, L: float, b: float, n_axis: int = 0, wrap: bool = False,
              workspace: torch.Tensor | None = None) -> CellGrid:
    """a1-a3: wrap (optional), cell binning and counting sort by cell."""
    _need(pos, torch.float32, None, "pos")
    N = pos.shape[0]
    n = default_cells_per_axis(N, L, b) if n_axis == 0 else int(n_axis)
    need = fof_bytes(N, n)
    ws = workspace if workspace is not None else _ws(need, pos.device)
    cells = Cells()
    h = context(pos.device)
    _check(library().jfof_bin_cells(h, _ptr(pos), N, L, b, n, JFOF_WRAP if wrap else 0,
                                    _ptr(ws), ws.numel(), ctypes.byref(cells)), "jfof_bin_cells")
    return CellGrid(cells, ws)


def link(grid: CellGrid, label: torch.Tensor | None = None) -> torch.Tensor:
    """a4-a6: neighbour scan + union-find; raw labels (smallest member index)."""
    N = grid.cells.n
    dev = grid.workspace.device
    if label is None:
        label = torch.empty(N, dtype=torch.int32, device=dev)
    _need(label, torch.int32, (N,), "label")
    _check(library().jfof_link(context(dev), ctypes.byref(grid.cells), _ptr(label)), "jfof_link")
    return label


@dataclass
class Groups:
    halo_id: torch.Tensor     # [N] int32, -1 below the cut
    count: torch.Tensor       # [H_cap] int32 (first H valid)
    halo_start: torch.Tensor  # [H_cap+1] int32
    members: torch.Tensor     # [N] int32 (first halo_start[H] valid)
    n_halos_dev: torch.Tensor # [1] int32 on the device
    H_cap: int

    @property
    def n_halos(self) -> int:
        return int(self.n_halos_dev.item())


def _alloc_groups(N: int, min_size: int, dev) -> Groups:
    H_cap = max(N // min_size, 1)
    return Groups(torch.empty(N, dtype=torch.int32, device=dev),
                  torch.empty(H_cap, dtype=torch.int32, device=dev),
                  torch.empty(H_cap + 1, dtype=torch.int32, device=dev),
                  torch.empty(N, dtype=torch.int32, device=dev),
                  torch.empty(1, dtype=torch.int32, device=dev), H_cap)


def groups(label: torch.Tensor, min_size: int = 20, workspace: torch.Tensor | None = None) -> Groups:
    """a7: compaction, histogram, minimum-size cut, CSR members."""
    _need(label, torch.int32, None, "label")
    N = label.shape[0]
    dev = label.device
    g = _alloc_groups(N, min_size, dev)
    ws = workspace if workspace is not None else _ws(groups_bytes(N), dev)
    _check(library().jfof_groups(context(dev), _ptr(label), N, min_size, _ptr(ws), ws.numel(),
                                 _ptr(g.halo_id), _ptr(g.count), _ptr(g.halo_start),
                                 _ptr(g.members), _ptr(g.n_halos_dev)), "jfof_groups")
    return g


@dataclass
class FofResult:
    label: torch.Tensor
    groups: Groups
    n_axis: int


def fof_all_bytes(N: int, n_axis: int) -> int:
    s = ctypes.c_size_t()
    _check(library().jfof_fof_all_bytes(N, n_axis, ctypes.byref(s)), "jfof_fof_all_bytes")
    return s.value


def fof(pos: torch.Tensor, L: float, b: float, min_size: int = 20, n_axis: int = 0,
        wrap: bool = False, workspace: torch.Tensor | None = None,
        out: FofResult | None = None) -> FofResult:
    """a1-a7 in one call: labels, halo ids, counts and CSR members.  ``out``
    (from a previous call with the same N and min_size) is reused in place."""
    _need(pos, torch.float32, None, "pos")
    N = pos.shape[0]
    dev = pos.device
    n = default_cells_per_axis(N, L, b) if n_axis == 0 else int(n_axis)
    ws = workspace if workspace is not None else _ws(fof_all_bytes(N, n), dev)
    if out is not None:
        label, g = out.label, out.groups
    else:
        label = torch.empty(N, dtype=torch.int32, device=dev)
        g = _alloc_groups(N, min_size, dev)
    _check(library().jfof_fof(context(dev), _ptr(pos), N, L, b, n, JFOF_WRAP if wrap else 0,
                              min_size, _ptr(ws), ws.numel(), _ptr(label), _ptr(g.halo_id),
                              _ptr(g.count), _ptr(g.halo_start), _ptr(g.members),
                              _ptr(g.n_halos_dev)), "jfof_fof")
    return FofResult(label, g, n)


@dataclass
class Props:
    mass: torch.Tensor   # [H_cap]
    com: torch.Tensor    # [H_cap, 3]
    vmean: torch.Tensor  # [H_cap, 3]
    sigv: torch.Tensor   # [H_cap]


def halo_props(pos: torch.Tensor, vel: torch.Tensor | None, L: float, g: Groups,
               particle_mass: float = 1.0, wrap: bool = False, out: Props | None = None) -> Props:
    """a8: mass, periodic COM, velocity mean and dispersion (first H rows valid)."""
    _need(pos, torch.float32, None, "pos")
    _need(vel, torch.float32, tuple(pos.shape), "vel")
    dev = pos.device
    H = g.H_cap
    if out is None:
        out = Props(torch.zeros(H, device=dev), torch.zeros(H, 3, device=dev),
                    torch.zeros(H, 3, device=dev), torch.zeros(H, device=dev))
    _check(library().jfof_halo_props(context(dev), _ptr(pos), _ptr(vel), pos.shape[0], L,
                                     JFOF_WRAP if wrap else 0, _ptr(g.halo_start), _ptr(g.members),
                                     _ptr(g.n_halos_dev), g.H_cap, particle_mass, _ptr(out.mass),
                                     _ptr(out.com), _ptr(out.vmean), _ptr(out.sigv)),
           "jfof_halo_props")
    return out


def fof_host(h_pos: torch.Tensor, h_vel: torch.Tensor | None, L: float, b: float, min_size: int = 20,
             n_axis: int = 0, wrap: bool = False, particle_mass: float = 1.0, device=None,
             d_pos: torch.Tensor | None = None, d_vel: torch.Tensor | None = None,
             workspace: torch.Tensor | None = None, out: FofResult | None = None,
             props_out: Props | None = None):
    """a1-a8 from host tensors (page-locked for asynchronous uploads): the
    positions are uploaded, the velocity upload overlaps the FoF kernels, then
    labels, groups and halo properties as ``fof`` + ``halo_props``.  Returns
    (FofResult, Props, d_pos, d_vel); pass them back to reuse the buffers."""
    if h_pos.device.type != "cpu" or (h_vel is not None and h_vel.device.type != "cpu"):
        raise ValueError("fof_host takes host tensors")
    if h_pos.dtype != torch.float32 or not h_pos.is_contiguous() or h_pos.dim() != 2 or h_pos.shape[1] != 3:
        raise ValueError("h_pos must be contiguous float32 [N, 3]")
    if h_vel is not None and (h_vel.dtype != torch.float32 or not h_vel.is_contiguous()
                              or tuple(h_vel.shape) != tuple(h_pos.shape)):
        raise ValueError("h_vel must be contiguous float32 [N, 3]")
    dev = torch.device(device if device is not None else "cuda")
    N = h_pos.shape[0]
    n = default_cells_per_axis(N, L, b) if n_axis == 0 else int(n_axis)
    if d_pos is None:
        d_pos = torch.empty(N, 3, dtype=torch.float32, device=dev)
    if h_vel is not None and d_vel is None:
        d_vel = torch.empty(N, 3, dtype=torch.float32, device=dev)
    ws = workspace if workspace is not None else _ws(fof_all_bytes(N, n), dev)
    if out is not None:
        label, g = out.label, out.groups
    else:
        label = torch.empty(N, dtype=torch.int32, device=dev)
        g = _alloc_groups(N, min_size, dev)
    H = g.H_cap
    p = props_out if props_out is not None else Props(
        torch.zeros(H, device=dev), torch.zeros(H, 3, device=dev), torch.zeros(H, 3, device=dev),
        torch.zeros(H, device=dev))
    _check(library().jfof_fof_host(
        context(dev), _ptr(h_pos), _ptr(h_vel), N, L, b, n, JFOF_WRAP if wrap else 0, min_size,
        particle_mass, _ptr(d_pos), _ptr(d_vel if h_vel is not None else None), _ptr(ws), ws.numel(),
        _ptr(label), _ptr(g.halo_id), _ptr(g.count), _ptr(g.halo_start), _ptr(g.members),
        _ptr(g.n_halos_dev), _ptr(p.mass), _ptr(p.com), _ptr(p.vmean), _ptr(p.sigv)), "jfof_fof_host")
    return FofResult(label, g, n), p, d_pos, d_vel


def halo_props_backward(vel, g: Groups, vmean, sigv, g_com=None, g_vmean=None, g_sigv=None):
    """a9: frozen-assignment adjoint -> (g_pos[N,3], g_vel[N,3])."""
    dev = g.halo_id.device
    N = g.halo_id.shape[0]
    g_pos = torch.empty(N, 3, device=dev)
    g_vel = torch.empty(N, 3, device=dev)
    _check(library().jfof_halo_props_backward(
        context(dev), _ptr(vel), _ptr(g.halo_id), _ptr(g.count), N, _ptr(vmean), _ptr(sigv),
        _ptr(g_com), _ptr(g_vmean), _ptr(g_sigv), _ptr(g_pos), _ptr(g_vel)),
        "jfof_halo_props_backward")
    return g_pos, g_vel


class HaloProps(torch.autograd.Function):
    """Differentiable halo properties with frozen memberships (Sec. 3.1).

    forward(pos, vel, groups, L) -> (com[H,3], vmean[H,3], sigv[H]) for the H
    halos of ``groups``; backward runs the adjoint kernel.  Memberships (the
    FoF labels) are not differentiated.
    """

    @staticmethod
    def forward(ctx, pos, vel, g: Groups, L: float, wrap: bool = False):
        H = g.n_halos
        p = halo_props(pos.detach().contiguous(), vel.detach().contiguous(), L, g, wrap=wrap)
        ctx.g = g
        vm, sg = p.vmean[:H].contiguous(), p.sigv[:H].contiguous()
        ctx.save_for_backward(vel.detach(), p.vmean, p.sigv)
        ctx.H = H
        return p.com[:H].clone(), vm, sg

    @staticmethod
    def backward(ctx, g_com, g_vmean, g_sigv):
        vel, vmean, sigv = ctx.saved_tensors
        g = ctx.g
        H, Hc = ctx.H, g.H_cap

        def pad(t, shape):
            if t is None:
                return None
            out = torch.zeros(shape, device=vel.device, dtype=torch.float32)
            out[:H] = t
            return out.contiguous()
        gp, gv = halo_props_backward(vel, g, vmean, sigv, pad(g_com, (Hc, 3)),
                                     pad(g_vmean, (Hc, 3)), pad(g_sigv, (Hc,)))
        return gp, gv, None, None, None


# ---------------------------------------------------------------------------
# REINFORCE topological mode (Sec. 3.2)

def prob_coef(b: float, prob_form: int = 0, tau: float = 0.0, alpha: float = 0.5) -> float:
    """Edge-probability constant: 1/tau (form 0, tau <= 0 -> 0.05 b) or alpha/b^2 (form 1)."""
    c = ctypes.c_float()
    _check(library().jfof_prob_coef(b, prob_form, tau, alpha, ctypes.byref(c)), "jfof_prob_coef")
    return c.value


@dataclass
class Pairs:
    i: torch.Tensor  # [E] int32, sorted by (i, j), i < j
    j: torch.Tensor  # [E] int32
    d: torch.Tensor  # [E] float32
    p: torch.Tensor  # [E] float32
    N: int
    L: float
    b: float
    prob_form: int
    coef: float
    wrap: bool

    @property
    def E(self) -> int:
        return int(self.i.shape[0])


def pairs(pos: torch.Tensor, L: float, b: float, r_cut: float | None = None, prob_form: int = 0,
          coef: float | None = None, wrap: bool = False) -> Pairs:
    """a11: fixed candidate pairs within r_cut (default 1.5 b) with d and p.
    Counts first, then allocates exactly and fills (one host sync)."""
    _need(pos, torch.float32, None, "pos")
    N = pos.shape[0]
    dev = pos.device
    if r_cut is None:
        r_cut = float(torch.tensor(1.5 * float(torch.tensor(b, dtype=torch.float32)),
                                   dtype=torch.float32).item())
    if coef is None:
        coef = prob_coef(b, prob_form)
    s = ctypes.c_size_t()
    _check(library().jfof_pairs_bytes(N, L, r_cut, ctypes.byref(s)), "jfof_pairs_bytes")
    ws = _ws(s.value, dev)
    nE = torch.zeros(1, dtype=torch.int64, device=dev)
    h = context(dev)
    flags = JFOF_WRAP if wrap else 0
    _check(library().jfof_pairs(h, _ptr(pos), N, L, b, r_cut, prob_form, coef, flags, _ptr(ws),
                                ws.numel(), 0, None, None, None, None, _ptr(nE)), "jfof_pairs")
    sync(dev)
    E = int(nE.item())
    out = Pairs(torch.empty(E, dtype=torch.int32, device=dev), torch.empty(E, dtype=torch.int32, device=dev),
                torch.empty(E, device=dev), torch.empty(E, device=dev), N, L, b, prob_form, coef, wrap)
    if E:
        _check(library().jfof_pairs(h, _ptr(pos), N, L, b, r_cut, prob_form, coef, flags, _ptr(ws),
                                    ws.numel(), E, _ptr(out.i), _ptr(out.j), _ptr(out.d), _ptr(out.p),
                                    _ptr(nE)), "jfof_pairs")
    return out


def reinforce_sample(pr: Pairs, K: int, seed: int, min_size: int = 20,
                     labels: torch.Tensor | None = None):
    """a12: labels [K, N] (smallest member index per sample) and n_halos [K]."""
    dev = pr.i.device
    N = pr.N
    if labels is None:
        labels = torch.empty(K, N, dtype=torch.int32, device=dev)
    _need(labels, torch.int32, (K, N), "labels")
    nh = torch.empty(K, dtype=torch.int32, device=dev)
    s = ctypes.c_size_t()
    _check(library().jfof_reinforce_sample_bytes(N, ctypes.byref(s)), "jfof_reinforce_sample_bytes")
    ws = _ws(s.value, dev)
    _check(library().jfof_reinforce_sample(context(dev), N, _ptr(pr.i), _ptr(pr.j), _ptr(pr.p), pr.E, K,
                                           ctypes.c_uint64(seed), min_size, _ptr(ws), ws.numel(),
                                           _ptr(labels), _ptr(nh)), "jfof_reinforce_sample")
    return labels, nh


def reinforce_grad(pos: torch.Tensor, pr: Pairs, K: int, seed: int, advantage: torch.Tensor) -> torch.Tensor:
    """a13: score-function gradient w.r.t. positions, [N,3]."""
    _need(pos, torch.float32, None, "pos")
    _need(advantage, torch.float32, (K,), "advantage")
    dev = pos.device
    N = pos.shape[0]
    s = ctypes.c_size_t()
    _check(library().jfof_reinforce_grad_bytes(N, pr.E, ctypes.byref(s)), "jfof_reinforce_grad_bytes")
    ws = _ws(s.value, dev)
    g = torch.empty(N, 3, device=dev)
    _check(library().jfof_reinforce_grad(context(dev), _ptr(pos), N, pr.L, JFOF_WRAP if pr.wrap else 0,
                                         _ptr(pr.i), _ptr(pr.j), _ptr(pr.d), _ptr(pr.p), pr.E, K,
                                         ctypes.c_uint64(seed), _ptr(advantage), pr.prob_form, pr.coef,
                                         _ptr(ws), ws.numel(), _ptr(g)), "jfof_reinforce_grad")
    return g


def eval_exp(x: torch.Tensor) -> torch.Tensor:
    _need(x, torch.float32, None, "x")
    y = torch.empty_like(x)
    _check(library().jfof_eval_exp(context(x.device), _ptr(x), _ptr(y), x.numel()), "jfof_eval_exp")
    return y


def eval_edge_uniform(seed: int, i: torch.Tensor, j: torch.Tensor, k: torch.Tensor) -> torch.Tensor:
    for t, nm in ((i, "i"), (j, "j"), (k, "k")):
        _need(t, torch.int32, None, nm)
    u = torch.empty(i.shape, device=i.device)
    _check(library().jfof_eval_edge_uniform(context(i.device), ctypes.c_uint64(seed), _ptr(i), _ptr(j),
                                            _ptr(k), _ptr(u), i.numel()), "jfof_eval_edge_uniform")
    return u


class ReinforceFoF(torch.autograd.Function):
    """Expected loss over stochastic FoF topologies (Sec. 3.2, Eqs. 6-8).

    forward(pos, pairs, losses, seed) -> mean of the per-sample losses
    ``losses`` [K] (computed by the caller from the labels of
    ``reinforce_sample(pairs, K, seed)``); backward returns the REINFORCE
    gradient with the batch-mean baseline, A_k = L_k - mean(L).  The pair
    list (the neighbour structure) is fixed, as in the paper.
    """

    @staticmethod
    def forward(ctx, pos, pr: Pairs, losses, seed: int):
        lo = losses.detach().to(torch.float32).contiguous()
        ctx.pr, ctx.seed = pr, seed
        ctx.save_for_backward(pos.detach(), lo)
        return lo.mean()

    @staticmethod
    def backward(ctx, grad_out):
        pos, lo = ctx.saved_tensors
        adv = (lo - lo.mean()).contiguous()
        g = reinforce_grad(pos.contiguous(), ctx.pr, lo.shape[0], ctx.seed, adv)
        return g * grad_out, None, None, None


# ---------------------------------------------------------------------------
# Batched boxes and the autotuner

class Batch:
    """Many independent boxes through one CUDA-graph launch (or the per-box
    loop with ``use_graph=False``).  Host-side sizes and parameters are fixed
    at construction; inputs and outputs are device tensors over the
    concatenated particles."""

    def __init__(self, box_offset, L, b, min_size: int = 20, n_axis=None, small=None, dense=None,
                 shape=None, device=None):
        import numpy as _np
        self.off = _np.ascontiguousarray(box_offset, _np.int64)
        self.B = len(self.off) - 1
        self.L = _np.ascontiguousarray(L, _np.float32)
        self.b = _np.ascontiguousarray(b, _np.float32)
        self.n = None if n_axis is None else _np.ascontiguousarray(n_axis, _np.int32)
        self.small = None if small is None else _np.ascontiguousarray(small, _np.int32)
        self.dense = None if dense is None else _np.ascontiguousarray(dense, _np.int32)
        self.shape = None if shape is None else _np.ascontiguousarray(shape, _np.int32)
        self.min_size = min_size
        dev = torch.device("cuda") if device is None else torch.device(device)
        s = ctypes.c_size_t()
        _check(library().jfof_batch_bytes(self.off.ctypes.data, self.B, self.L.ctypes.data,
                                          self.b.ctypes.data, None if self.n is None else self.n.ctypes.data,
                                          min_size, ctypes.byref(s)), "jfof_batch_bytes")
        self.ws = _ws(s.value, dev)
        N = int(self.off[-1])
        self.label = torch.empty(N, dtype=torch.int32, device=dev)
        self.halo_id = torch.empty(N, dtype=torch.int32, device=dev)
        self.n_halos = torch.empty(self.B, dtype=torch.int32, device=dev)

    def run(self, pos: torch.Tensor, use_graph: bool = True, wrap: bool = False):
        _need(pos, torch.float32, (int(self.off[-1]), 3), "pos")
        arr = lambda a: None if a is None else a.ctypes.data  # noqa: E731
        _check(library().jfof_fof_batched(
            context(pos.device), _ptr(pos), self.off.ctypes.data, self.B, self.L.ctypes.data,
            self.b.ctypes.data, arr(self.n), arr(self.small), arr(self.dense), arr(self.shape),
            JFOF_WRAP if wrap else 0,
            self.min_size, _ptr(self.ws), self.ws.numel(), _ptr(self.label), _ptr(self.halo_id),
            _ptr(self.n_halos), 1 if use_graph else 0), "jfof_fof_batched")
        return self.label, self.halo_id, self.n_halos

    @classmethod
    def tuned(cls, pos: torch.Tensor, box_offset, L, b, min_size: int = 20, reps: int = 2, use_cache: bool = True,
              wrap: bool = False):
        """A batch whose boxes each run with the autotuner's choice of grid,
        cell classes and CTA shape (boxes of one size bucket share a choice
        through the context's cache).  Returns (batch, per-box choices)."""
        import numpy as _np
        off = _np.ascontiguousarray(box_offset, _np.int64)
        picks = []
        for k in range(len(off) - 1):
            sl = pos[int(off[k]):int(off[k + 1])]
            picks.append(autotune(sl, float(L[k]), float(b[k]), min_size, reps=reps, wrap=wrap,
                                  use_cache=use_cache))
        n, S, T, W = (list(c) for c in zip(*[p[:4] for p in picks]))
        return cls(off, L, b, min_size, n_axis=n, small=S, dense=T, shape=W, device=pos.device), picks


def _graph_ms(bt: "Batch", pos: torch.Tensor, reps: int = 3) -> float:
    bt.run(pos, use_graph=True)
    sync(pos.device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        bt.run(pos, use_graph=True)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune_batch(pos: torch.Tensor, box_offset, L, b, min_size: int = 20, reps: int = 3, min_gain: float = 0.01):
    """Autotune a batch as a whole: boxes are grouped by the autotuner's size
    bucket (round(2 log2 N), round(4 log2(L/b))) and, bucket by bucket, a
    few candidate choices (grid, cell classes, CTA shape) are applied to all
    of the bucket's boxes and kept only when the whole batch graph runs
    faster.  Unlike per-box tuning this sees the boxes share the GPU and its
    L2.  Returns (batch, per-box choices (n, S, T, shape), ms per graph)."""
    import math

    import numpy as _np
    off = _np.ascontiguousarray(box_offset, _np.int64)
    B = len(off) - 1
    Ns = _np.diff(off)
    n0 = [default_cells_per_axis(int(Ns[k]), float(L[k]), float(b[k])) for k in range(B)]
    nmax = [max_cells_per_axis(float(L[k]), float(b[k])) for k in range(B)]
    choice = [[n0[k], 16, -1, 0] for k in range(B)]
    buckets = {}
    for k in range(B):
        key = (round(2 * math.log2(int(Ns[k]))), round(4 * math.log2(float(L[k]) / float(b[k]))))
        buckets.setdefault(key, []).append(k)

    def build(ch):
        n, S, T, W = (list(c) for c in zip(*ch))
        return Batch(off, L, b, min_size, n_axis=n, small=S, dense=T, shape=W, device=pos.device)

    best = _graph_ms(build(choice), pos, reps)
    cands = [(1.0, 8, 96, 0), (1.0, 16, 128, 0), (1.0, 8, 64, 0), (1.0, 24, 96, 0), (0.8, 16, -1, 0),
             (1.0, 16, -1, 1), (1.0, 16, -1, 2)]
    for key in sorted(buckets, reverse=True):  # largest boxes first
        for f, S, T, W in cands:
            trial = [list(c) for c in choice]
            for k in buckets[key]:
                n = max(3, min(nmax[k], int(round(n0[k] * f))))
                trial[k] = [n, S, T, W]
            ms = _graph_ms(build(trial), pos, reps)
            if ms < best * (1.0 - min_gain):
                best, choice = ms, trial
    return build(choice), [tuple(c) for c in choice], best


def set_cta_shape(shape: int = 0, device=None):
    """CTA shape of the list-driven link kernels: 0 = (4, 8, 4, 8) warps, 1 = all 8, 2 = all 4."""
    _check(library().jfof_set_cta_shape(context(device), shape), "jfof_set_cta_shape")


_flush = {}


def _flush_buffer(dev) -> torch.Tensor:
    """A 256 MiB device buffer (twice the L2) the autotuner overwrites before
    each timed run."""
    key = str(dev)
    if key not in _flush:
        _flush[key] = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    return _flush[key]


def autotune(pos: torch.Tensor, L: float, b: float, min_size: int = 20, reps: int = 2,
             wrap: bool = False, use_cache: bool = False):
    """Fastest (n_axis, small, dense, cta_shape, ms) for this box among the
    candidates; ``use_cache`` returns a choice already made for the same size
    bucket without timing."""
    _need(pos, torch.float32, None, "pos")
    N = pos.shape[0]
    dev = pos.device
    n0 = default_cells_per_axis(N, L, b)
    nmax = max_cells_per_axis(L, b)
    n_big = min(nmax, int(n0 * 1.26))
    size = max(fof_all_bytes(N, n0), fof_all_bytes(N, max(3, n_big))) + 3 * 4 * N + (1 << 20)
    ws = _ws(size, dev)
    label = torch.empty(N, dtype=torch.int32, device=dev)
    hid = torch.empty(N, dtype=torch.int32, device=dev)
    nh = torch.empty(1, dtype=torch.int32, device=dev)
    bn, bs, bd, bw, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    flush = _flush_buffer(dev)
    _check(library().jfof_autotune(context(dev), _ptr(pos), N, L, b, JFOF_WRAP if wrap else 0, min_size,
                                   _ptr(ws), ws.numel(), _ptr(label), _ptr(hid), _ptr(nh), reps,
                                   1 if use_cache else 0, _ptr(flush), flush.numel(), ctypes.byref(bn),
                                   ctypes.byref(bs), ctypes.byref(bd), ctypes.byref(bw), ctypes.byref(ms)),
           "jfof_autotune")
    return bn.value, bs.value, bd.value, bw.value, ms.value


def fof_static(pos: torch.Tensor, L: float, b: float, min_size: int = 20, n_axis: int = 0,
               wrap: bool = False, out: FofResult | None = None) -> FofResult:
    """a1-a7 like :func:`fof`, with the library's fixed 16 MiB device scratch
    instead of a workspace (for callers that must not allocate device memory).
    Limit: ``fof_all_bytes(N, n) <= 16 MiB``, about 1.9e5 particles at the
    default grid.  Calls sharing a GPU must not overlap."""
    _need(pos, torch.float32, None, "pos")
    N = pos.shape[0]
    dev = pos.device
    n = default_cells_per_axis(N, L, b) if n_axis == 0 else int(n_axis)
    if out is not None:
        label, g = out.label, out.groups
    else:
        label = torch.empty(N, dtype=torch.int32, device=dev)
        g = _alloc_groups(N, min_size, dev)
    _check(library().jfof_fof_static(context(dev), _ptr(pos), N, L, b, n, JFOF_WRAP if wrap else 0,
                                     min_size, _ptr(label), _ptr(g.halo_id), _ptr(g.count),
                                     _ptr(g.halo_start), _ptr(g.members), _ptr(g.n_halos_dev)),
           "jfof_fof_static")
    return FofResult(label, g, n)


# ---------------------------------------------------------------------------
# Slabs of cell layers: streaming FoF with bounded device memory and the
# union-find fusion of slabs (include/jfof.h).  Host arrays are CPU tensors.

def _host(t, dtype, name):
    if t.device.type != "cpu" or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CPU {dtype} tensor")
    return t


def slab_select(h_pos: torch.Tensor, L: float, b: float, n_slabs: int, slab: int, n_axis: int = 0):
    """Host only: ascending global indices (int64) of slab ``slab``'s subset
    (its cell layers plus one layer on each side) and its core flags (uint8)."""
    _host(h_pos, torch.float32, "h_pos")
    N = h_pos.shape[0]
    lib = library()
    cnt = ctypes.c_int64()
    _check(lib.jfof_slab_select(_ptr(h_pos), N, L, b, n_axis, n_slabs, slab, None, None, ctypes.byref(cnt)),
           "jfof_slab_select")
    idx = torch.empty(cnt.value, dtype=torch.int64)
    core = torch.empty(cnt.value, dtype=torch.uint8)
    _check(lib.jfof_slab_select(_ptr(h_pos), N, L, b, n_axis, n_slabs, slab, _ptr(idx), _ptr(core),
                                ctypes.byref(cnt)), "jfof_slab_select")
    return idx, core


def merge_labels(pre: torch.Tensor, a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Host only: union-find fusion over global indices (smaller index wins):
    classes joined pairwise by (a[k], b[k]); returns the root of pre[i]."""
    for t, nm in ((pre, "pre"), (a, "a"), (b, "b")):
        _host(t, torch.int32, nm)
    if a.numel() != b.numel():
        raise ValueError("a and b must have the same length")
    out = torch.empty_like(pre)
    _check(library().jfof_merge_labels(pre.numel(), _ptr(pre), a.numel(), _ptr(a) if a.numel() else None,
                                       _ptr(b) if b.numel() else None, _ptr(out)), "jfof_merge_labels")
    return out


def fof_stream(h_pos: torch.Tensor, L: float, b: float, n_slabs: int, min_size: int = 20, n_axis: int = 0,
               device=None):
    """FoF of positions kept in host memory, one slab of cell layers at a
    time on the GPU: returns host (label, halo_id, n_halos), equal to
    :func:`fof`'s labels and halo ids."""
    _host(h_pos, torch.float32, "h_pos")
    N = h_pos.shape[0]
    lib = library()
    nb = ctypes.c_size_t()
    _check(lib.jfof_fof_stream_bytes(_ptr(h_pos), N, L, b, n_axis, n_slabs, ctypes.byref(nb)),
           "jfof_fof_stream_bytes")
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index)
    ws = _ws(nb.value, dev)
    label = torch.empty(N, dtype=torch.int32)
    hid = torch.empty(N, dtype=torch.int32)
    nh = ctypes.c_int64()
    _check(lib.jfof_fof_stream(context(dev), _ptr(h_pos), N, L, b, n_axis, n_slabs, min_size, _ptr(ws), ws.numel(),
                               _ptr(label), _ptr(hid), ctypes.byref(nh)), "jfof_fof_stream")
    return label, hid, nh.value


def _link_slab_on_gpu(pos_s: torch.Tensor, L: float, b: float, n_axis: int) -> torch.Tensor:
    """Raw labels of one slab subset (host positions in, host labels out):
    jfof_bin_cells + jfof_link on the current GPU with the box's grid."""
    dev = torch.device("cuda", torch.cuda.current_device())
    grid = bin_cells(pos_s.to(dev), L, b, n_axis=n_axis)
    lab = link(grid)
    sync(dev)
    return lab.cpu()


def fof_slabs(h_pos: torch.Tensor, L: float, b: float, min_size: int = 20, n_axis: int = 0, group=None,
              link_slab=None):
    """Slab decomposition with union-find fusion over the ranks of a
    torch.distributed group (Sec. 2.3): rank r of W links slab r of W (its
    cell layers plus one layer on each side) on its own GPU; the ranks then
    exchange the labels of the particles two slabs share (two all-gathers of
    small records) and fuse them with :func:`merge_labels`.  Every rank holds
    the host positions.  Returns, for this rank's own particles, their global
    indices (int64), raw labels (smallest index of the group) and halo ids
    (ascending with the raw label, -1 below min_size), all on the host, and
    the number of halos.  ``link_slab(pos_s, L, b, n) -> labels`` replaces the
    GPU link of a slab (the CPU tests pass the oracle)."""
    import torch.distributed as dist

    _host(h_pos, torch.float32, "h_pos")
    N = h_pos.shape[0]
    W = dist.get_world_size(group) if dist.is_initialized() else 1
    r = dist.get_rank(group) if dist.is_initialized() else 0
    n = default_cells_per_axis(N, L, b) if n_axis == 0 else int(n_axis)
    idx, core = slab_select(h_pos, L, b, W, r, n_axis=n)
    linker = link_slab or _link_slab_on_gpu
    lab = linker(h_pos[idx].contiguous(), L, b, n).to(torch.int64) if idx.numel() else torch.empty(0, dtype=torch.int64)
    R = idx[lab] if idx.numel() else idx  # global smallest index of each slab component
    is_core = core.bool()
    g_own, r_own = idx[is_core], R[is_core]
    ghosts = (idx[~is_core], R[~is_core])

    def gather(obj):
        if W == 1:
            return [obj]
        out = [None] * W
        dist.all_gather_object(out, obj, group=group)
        return out

    # particles of an extra layer: their label in this slab against their
    # label in their own slab (known to the rank that owns them)
    own_label = torch.full((N,), -1, dtype=torch.int64)
    own_label[g_own] = r_own
    pa, pb = [], []
    for gg, rr in gather(ghosts):
        mine = own_label[gg] >= 0
        pa.append(own_label[gg][mine])
        pb.append(rr[mine])
    pairs = gather((torch.cat(pa) if pa else torch.empty(0, dtype=torch.int64),
                    torch.cat(pb) if pb else torch.empty(0, dtype=torch.int64)))
    a = torch.cat([p[0] for p in pairs]).to(torch.int32).contiguous()
    bb = torch.cat([p[1] for p in pairs]).to(torch.int32).contiguous()
    pre = torch.arange(N, dtype=torch.int32)
    pre[g_own] = r_own.to(torch.int32)
    label = merge_labels(pre, a, bb)[g_own]
    # groups: counts per raw label over all ranks, the cut, ids ascending
    u, c = torch.unique(label.to(torch.int64), return_counts=True)
    parts = gather((u, c))
    all_u = torch.cat([p[0] for p in parts])
    all_c = torch.cat([p[1] for p in parts])
    uu, inv = torch.unique(all_u, return_inverse=True)  # sorted ascending
    tot = torch.zeros(uu.numel(), dtype=torch.int64).index_add_(0, inv, all_c)
    kept = uu[tot >= min_size]
    H = kept.numel()
    at = torch.searchsorted(kept, label.to(torch.int64))
    hit = (at < H) & (kept[at.clamp(max=max(H - 1, 0))] == label) if H else torch.zeros_like(at, dtype=torch.bool)
    halo_id = torch.where(hit, at, torch.full_like(at, -1)).to(torch.int32)
    return g_own, label, halo_id, H


# ---------------------------------------------------------------------------
# Decorated frozen assignment and the soft mass function (Sec. 3.1.1, Eq. 5).

def halo_decoration(pos: torch.Tensor, L: float, g: Groups, com: torch.Tensor, wrap: bool = False,
                    out: torch.Tensor | None = None) -> torch.Tensor:
    """Particle standard deviation about each halo centre, dsig[H_cap]."""
    _need(pos, torch.float32, None, "pos")
    dsig = out if out is not None else torch.empty(g.H_cap, dtype=torch.float32, device=pos.device)
    _check(library().jfof_halo_decoration(context(pos.device), _ptr(pos), pos.shape[0], L,
                                          JFOF_WRAP if wrap else 0, _ptr(g.halo_start), _ptr(g.members),
                                          _ptr(g.n_halos_dev), g.H_cap, _ptr(com), _ptr(dsig)),
           "jfof_halo_decoration")
    return dsig


def halo_decoration_backward(pos: torch.Tensor, L: float, g: Groups, com, dsig, g_dsig, wrap: bool = False):
    """Frozen-assignment adjoint of the decoration: g_pos [N,3]."""
    g_pos = torch.empty_like(pos)
    _check(library().jfof_halo_decoration_backward(context(pos.device), _ptr(pos), _ptr(g.halo_id), _ptr(g.count),
                                                   pos.shape[0], L, JFOF_WRAP if wrap else 0, _ptr(com),
                                                   _ptr(dsig), _ptr(g_dsig.contiguous()), _ptr(g_pos)),
           "jfof_halo_decoration_backward")
    return g_pos


def soft_hmf(g: Groups, edges: torch.Tensor, width: float, particle_mass: float = 1.0) -> torch.Tensor:
    """Soft histogram of the halo log-masses over ``edges`` (device float32)."""
    _need(edges, torch.float32, None, "edges")
    B = edges.numel() - 1
    nb = ctypes.c_size_t()
    _check(library().jfof_soft_hmf_bytes(g.H_cap, B, ctypes.byref(nb)), "jfof_soft_hmf_bytes")
    ws = _ws(nb.value, edges.device)
    hist = torch.empty(B, dtype=torch.float32, device=edges.device)
    _check(library().jfof_soft_hmf(context(edges.device), _ptr(g.count), _ptr(g.n_halos_dev), g.H_cap,
                                   particle_mass, _ptr(edges), B, width, _ptr(ws), ws.numel(), _ptr(hist)),
           "jfof_soft_hmf")
    return hist


def soft_hmf_backward(g: Groups, dsig, edges, width: float, kappa: float, g_hist, particle_mass: float = 1.0):
    """VJP of :func:`soft_hmf` to the decoration: g_dsig[H_cap]."""
    g_dsig = torch.zeros(g.H_cap, dtype=torch.float32, device=edges.device)
    _check(library().jfof_soft_hmf_backward(context(edges.device), _ptr(g.count), _ptr(g.n_halos_dev), g.H_cap,
                                            particle_mass, _ptr(dsig), _ptr(edges), edges.numel() - 1, width,
                                            kappa, _ptr(g_hist.contiguous()), _ptr(g_dsig)),
           "jfof_soft_hmf_backward")
    return g_dsig


class DecoratedHMF(torch.autograd.Function):
    """Soft halo mass function whose gradient reaches the positions through the
    decoration (decorated frozen assignment, Sec. 3.1.1): forward = soft
    histogram of log(m_p n_h); backward = its VJP, g_D = -kappa g_ell / D,
    then the decoration's adjoint.  Memberships are frozen (``g`` from
    :func:`groups` or :func:`fof`)."""

    @staticmethod
    def forward(ctx, pos, g: Groups, L: float, edges, width: float, kappa: float = 1.0,
                particle_mass: float = 1.0, wrap: bool = False):
        p = halo_props(pos.detach(), None, L, g, particle_mass=particle_mass, wrap=wrap)
        dsig = halo_decoration(pos.detach(), L, g, p.com, wrap=wrap)
        hist = soft_hmf(g, edges, width, particle_mass)
        ctx.save_for_backward(pos.detach(), p.com, dsig, edges)
        ctx.g, ctx.L, ctx.width, ctx.kappa, ctx.mp, ctx.wrap = g, L, width, kappa, particle_mass, wrap
        return hist

    @staticmethod
    def backward(ctx, g_hist):
        pos, com, dsig, edges = ctx.saved_tensors
        g_dsig = soft_hmf_backward(ctx.g, dsig, edges, ctx.width, ctx.kappa, g_hist.float(), ctx.mp)
        g_pos = halo_decoration_backward(pos, ctx.L, ctx.g, com, dsig, g_dsig, wrap=ctx.wrap)
        return g_pos, None, None, None, None, None, None, None


# ---------------------------------------------------------------------------
# Sub-halos: FoF in phase space inside each halo (Sec. 2.1.1, Eq. 3).

def subhalos(pos: torch.Tensor, vel: torch.Tensor, L: float, g: Groups, sigma_x: float, sigma_v: float,
             wrap: bool = False) -> torch.Tensor:
    """sub_label[N]: smallest index of each member's phase-space group inside
    its halo (|dx|^2/sigma_x + |dv|^2/sigma_v <= 1); non-members keep their
    own index.  :func:`groups` on the result gives sub-halo ids."""
    _need(pos, torch.float32, None, "pos")
    _need(vel, torch.float32, tuple(pos.shape), "vel")
    N = pos.shape[0]
    nb = ctypes.c_size_t()
    _check(library().jfof_subhalos_bytes(N, ctypes.byref(nb)), "jfof_subhalos_bytes")
    ws = _ws(nb.value, pos.device)
    out = torch.empty(N, dtype=torch.int32, device=pos.device)
    _check(library().jfof_subhalos(context(pos.device), _ptr(pos), _ptr(vel), N, L, JFOF_WRAP if wrap else 0,
                                   _ptr(g.halo_start), _ptr(g.members), _ptr(g.n_halos_dev), g.H_cap,
                                   float(sigma_x), float(sigma_v), _ptr(ws), ws.numel(), _ptr(out)),
           "jfof_subhalos")
    return out
