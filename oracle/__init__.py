"""CPU oracle for the FoF hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or calls it, and it shares no code
with that path.

The arithmetic lives in ``fof_oracle.c`` (plain C, built with
``-O2 -ffp-contract=off``); this module only builds it and marshals numpy
arrays through ctypes.  Every function states the passage of the paper it
follows (Horowitz & Bayer, jFoF, arXiv 2510.26851) in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fof_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile fof_oracle.c into a shared library (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-pthread",
           "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.orc_dist2.restype = c.c_float
        lib.orc_dist2.argtypes = [_f32p, _f32p, c.c_float]
        lib.orc_wrap.restype = c.c_int
        lib.orc_wrap.argtypes = [_f32p, c.c_int64, c.c_float]
        lib.orc_max_cells_per_axis.restype = c.c_int32
        lib.orc_max_cells_per_axis.argtypes = [c.c_float, c.c_float]
        lib.orc_fof_labels.restype = c.c_int
        lib.orc_fof_labels.argtypes = [_f32p, c.c_int64, c.c_float, c.c_float,
                                       c.c_int32, _i32p]
        lib.orc_fof_labels_mt.restype = c.c_int
        lib.orc_fof_labels_mt.argtypes = [_f32p, c.c_int64, c.c_float, c.c_float,
                                          c.c_int32, c.c_int32, _i32p]
        lib.orc_fof_brute.restype = c.c_int
        lib.orc_fof_brute.argtypes = [_f32p, c.c_int64, c.c_float, c.c_float, _i32p]
        lib.orc_groups.restype = c.c_int64
        lib.orc_groups.argtypes = [_i32p, c.c_int64, c.c_int32, _i32p, _i32p]
        lib.orc_halo_props.restype = c.c_int
        lib.orc_halo_props.argtypes = [_f64p, _f64p, _i32p, c.c_int64, c.c_int64,
                                       c.c_double, c.c_double, _f64p, _f64p, _f64p, _f64p]
        lib.orc_halo_props_backward.restype = c.c_int
        lib.orc_halo_props_backward.argtypes = [
            _f64p, _i32p, c.c_int64, c.c_int64, _f64p, _f64p,
            c.c_void_p, c.c_void_p, c.c_void_p, _f64p, _f64p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_edge_uniform.restype = c.c_float
        lib.orc_edge_uniform.argtypes = [c.c_uint64, c.c_int32, c.c_int32, c.c_int32]
        lib.orc_exp.restype = c.c_float
        lib.orc_exp.argtypes = [c.c_float]
        lib.orc_edge_prob.restype = c.c_float
        lib.orc_edge_prob.argtypes = [c.c_float, c.c_float, c.c_float, c.c_float,
                                      c.c_int32, c.c_float]
        lib.orc_pairs.restype = c.c_int64
        lib.orc_pairs.argtypes = [_f32p, c.c_int64, c.c_float, c.c_float, c.c_float,
                                  c.c_int32, c.c_float, c.c_int64,
                                  c.c_void_p, c.c_void_p, c.c_void_p, c.c_void_p]
        lib.orc_reinforce_sample.restype = c.c_int
        lib.orc_reinforce_sample.argtypes = [c.c_int64, c.c_int64, _i32p, _i32p, _f32p,
                                             c.c_int32, c.c_uint64, c.c_int32, _i32p, _i32p]
        lib.orc_reinforce_grad.restype = c.c_int
        lib.orc_reinforce_grad.argtypes = [_f32p, c.c_int64, c.c_float, c.c_int64,
                                           _i32p, _i32p, _f32p, c.c_int32, c.c_uint64,
                                           _f64p, c.c_int32, c.c_double, _f64p]
        _lib = lib
        return lib


class OracleError(RuntimeError):
    pass


def _pos32(pos) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pos, dtype=np.float32).reshape(-1, 3))
    return a


def dist2(pi, pj, L: float) -> float:
    """Specified binary32 minimum-image squared distance (no FMA)."""
    return float(_load().orc_dist2(np.ascontiguousarray(pi, np.float32),
                                   np.ascontiguousarray(pj, np.float32), np.float32(L)))


def wrap(pos, L: float) -> np.ndarray:
    """Optional periodic wrap of positions into [0, L) (Algorithm 2, 'X mod L')."""
    p = _pos32(pos).copy()
    _load().orc_wrap(p, p.shape[0], np.float32(L))
    return p


def max_cells_per_axis(L: float, b: float) -> int:
    return int(_load().orc_max_cells_per_axis(np.float32(L), np.float32(b)))


def fof_labels(pos, L: float, b: float, n_axis: int = 0) -> np.ndarray:
    """Raw FoF labels (smallest member index) by cell list + union-find."""
    p = _pos32(pos)
    lab = np.empty(p.shape[0], np.int32)
    st = _load().orc_fof_labels(p, p.shape[0], np.float32(L), np.float32(b), n_axis, lab)
    if st != 0:
        raise OracleError(f"orc_fof_labels status {st}")
    return lab


def default_threads() -> int:
    """Threads for the threaded oracle: the cores this process may run on."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def fof_labels_mt(pos, L: float, b: float, n_axis: int = 0, threads: int = 0) -> np.ndarray:
    """The labels of :func:`fof_labels` computed on several threads (slabs of
    cell layers, pairs across slabs united afterwards)."""
    p = _pos32(pos)
    lab = np.empty(p.shape[0], np.int32)
    t = threads if threads > 0 else default_threads()
    st = _load().orc_fof_labels_mt(p, p.shape[0], np.float32(L), np.float32(b), n_axis, t, lab)
    if st != 0:
        raise OracleError(f"orc_fof_labels_mt status {st}")
    return lab


def fof_brute(pos, L: float, b: float) -> np.ndarray:
    """Raw FoF labels by O(N^2) brute force over all pairs."""
    p = _pos32(pos)
    lab = np.empty(p.shape[0], np.int32)
    st = _load().orc_fof_brute(p, p.shape[0], np.float32(L), np.float32(b), lab)
    if st != 0:
        raise OracleError(f"orc_fof_brute status {st}")
    return lab


def groups(label, min_size: int):
    """Compaction + histogram + cut: returns (halo_id[N], count[H])."""
    lab = np.ascontiguousarray(label, np.int32)
    hid = np.empty_like(lab)
    cnt = np.empty(lab.shape[0], np.int32)
    H = _load().orc_groups(lab, lab.shape[0], min_size, hid, cnt)
    if H < 0:
        raise OracleError("orc_groups: bad input")
    return hid, cnt[:H].copy()


def halo_props(pos, vel, halo_id, H: int, L: float, particle_mass: float = 1.0):
    """FP64 mass, periodic COM, velocity mean and 1-D dispersion per halo."""
    p = np.ascontiguousarray(np.asarray(pos, np.float64).reshape(-1, 3))
    v = np.ascontiguousarray(np.asarray(vel, np.float64).reshape(-1, 3))
    hid = np.ascontiguousarray(halo_id, np.int32)
    mass = np.empty(max(H, 1)); com = np.empty((max(H, 1), 3))
    vmean = np.empty((max(H, 1), 3)); sigv = np.empty(max(H, 1))
    st = _load().orc_halo_props(p, v, hid, p.shape[0], H, float(L), float(particle_mass),
                                mass, com, vmean, sigv)
    if st != 0:
        raise OracleError(f"orc_halo_props status {st}")
    return mass[:H], com[:H], vmean[:H], sigv[:H]


def halo_props_backward(vel, halo_id, H: int, vmean, sigv, g_com=None, g_vmean=None,
                        g_sigv=None):
    """FP64 frozen-assignment adjoint: returns (g_pos[N,3], g_vel[N,3])."""
    v = np.ascontiguousarray(np.asarray(vel, np.float64).reshape(-1, 3))
    hid = np.ascontiguousarray(halo_id, np.int32)
    vm = np.ascontiguousarray(np.asarray(vmean, np.float64).reshape(-1, 3)) if H else np.zeros((1, 3))
    sg = np.ascontiguousarray(np.asarray(sigv, np.float64).reshape(-1)) if H else np.zeros(1)

    def ptr(a, shape):
        if a is None:
            return None, None
        arr = np.ascontiguousarray(np.asarray(a, np.float64).reshape(shape))
        return arr, arr.ctypes.data_as(ctypes.c_void_p)

    gc, gcp = ptr(g_com, (-1, 3))
    gm, gmp = ptr(g_vmean, (-1, 3))
    gs, gsp = ptr(g_sigv, (-1,))
    gp = np.empty_like(v); gv = np.empty_like(v)
    st = _load().orc_halo_props_backward(v, hid, v.shape[0], H, vm, sg, gcp, gmp, gsp, gp, gv)
    if st != 0:
        raise OracleError(f"orc_halo_props_backward status {st}")
    return gp, gv


def subhalo_labels(pos, vel, halo_id, H: int, L: float, sigma_x: float, sigma_v: float) -> np.ndarray:
    """Phase-space sub-halo labels (Eq. 3): smallest index of each particle's
    6-D group inside its halo; particles outside halos are their own group.
    1/sigma are rounded once to binary32 (infinite sigma switches a term off)."""
    c = ctypes
    lib = _load()
    lib.orc_subhalo_labels.restype = c.c_int
    lib.orc_subhalo_labels.argtypes = [_f32p, _f32p, _i32p, c.c_int64, c.c_int64, c.c_float, c.c_float,
                                       c.c_float, _i32p]
    p = _pos32(pos)
    v = _pos32(vel)
    out = np.empty(p.shape[0], np.int32)
    inv = lambda s: np.float32(0.0) if np.isinf(s) else np.float32(1.0 / float(s))  # noqa: E731
    st = lib.orc_subhalo_labels(p, v, np.ascontiguousarray(halo_id, np.int32), p.shape[0], H, np.float32(L),
                                inv(sigma_x), inv(sigma_v), out)
    if st != 0:
        raise OracleError(f"orc_subhalo_labels status {st}")
    return out


def _declare_decor(lib):
    c = ctypes
    lib.orc_halo_decoration.restype = c.c_int
    lib.orc_halo_decoration.argtypes = [_f64p, _i32p, c.c_int64, c.c_int64, c.c_double, _f64p, _f64p]
    lib.orc_halo_decoration_backward.restype = c.c_int
    lib.orc_halo_decoration_backward.argtypes = [_f64p, _i32p, c.c_int64, c.c_int64, c.c_double, _f64p,
                                                 _f64p, _f64p, _f64p]
    lib.orc_soft_hist.restype = c.c_int
    lib.orc_soft_hist.argtypes = [_f64p, c.c_int64, _f64p, c.c_int32, c.c_double, _f64p]
    lib.orc_soft_hist_backward.restype = c.c_int
    lib.orc_soft_hist_backward.argtypes = [_f64p, c.c_int64, _f64p, c.c_int32, c.c_double, _f64p, _f64p]
    return lib


def _f64(a, shape=(-1,)):
    return np.ascontiguousarray(np.asarray(a, np.float64).reshape(shape))


def halo_decoration(pos, halo_id, H: int, L: float, com) -> np.ndarray:
    """FP64 particle standard deviation about each halo's centre (Sec. 3.1.1)."""
    lib = _declare_decor(_load())
    p = _f64(pos, (-1, 3))
    out = np.empty(max(H, 1))
    st = lib.orc_halo_decoration(p, np.ascontiguousarray(halo_id, np.int32), p.shape[0], H, float(L),
                                 _f64(com, (-1, 3)) if H else np.zeros((1, 3)), out)
    if st != 0:
        raise OracleError(f"orc_halo_decoration status {st}")
    return out[:H]


def halo_decoration_backward(pos, halo_id, H: int, L: float, com, dsig, g_dsig) -> np.ndarray:
    """FP64 frozen-assignment adjoint of the decoration: g_pos [N,3]."""
    lib = _declare_decor(_load())
    p = _f64(pos, (-1, 3))
    g = np.empty_like(p)
    z = np.zeros(1)
    st = lib.orc_halo_decoration_backward(p, np.ascontiguousarray(halo_id, np.int32), p.shape[0], H, float(L),
                                          _f64(com, (-1, 3)) if H else np.zeros((1, 3)),
                                          _f64(dsig) if H else z, _f64(g_dsig) if H else z, g)
    if st != 0:
        raise OracleError(f"orc_halo_decoration_backward status {st}")
    return g


def soft_hist(ell, edges, width: float) -> np.ndarray:
    """FP64 soft histogram of the values ell over bins edges[0..B]."""
    lib = _declare_decor(_load())
    e = _f64(edges)
    B = e.size - 1
    out = np.empty(B)
    el = _f64(ell) if len(ell) else np.zeros(1)
    st = lib.orc_soft_hist(el, len(ell), e, B, float(width), out)
    if st != 0:
        raise OracleError(f"orc_soft_hist status {st}")
    return out


def soft_hist_backward(ell, edges, width: float, g_hist) -> np.ndarray:
    """FP64 vector-Jacobian product of :func:`soft_hist` with respect to ell."""
    lib = _declare_decor(_load())
    e = _f64(edges)
    out = np.empty(max(len(ell), 1))
    st = lib.orc_soft_hist_backward(_f64(ell) if len(ell) else np.zeros(1), len(ell), e, e.size - 1, float(width),
                                    _f64(g_hist), out)
    if st != 0:
        raise OracleError(f"orc_soft_hist_backward status {st}")
    return out[:len(ell)]


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.empty(4, np.uint32)
    _load().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32),
                              np.ascontiguousarray(key, np.uint32), out)
    return out


def edge_uniform(seed: int, i: int, j: int, k: int) -> float:
    return float(_load().orc_edge_uniform(seed, i, j, k))


def exp32(x: float) -> float:
    return float(_load().orc_exp(np.float32(x)))


def edge_prob(d: float, d2: float, b: float, form: int, coef: float) -> float:
    b32 = np.float32(b)
    return float(_load().orc_edge_prob(np.float32(d), np.float32(d2), b32,
                                       np.float32(b32 * b32), form, np.float32(coef)))


def prob_coef(b: float, form: int, tau: float | None = None, alpha: float = 0.5) -> np.float32:
    """Host-side constant: 1/tau (form 0; tau defaults to 0.05 b) or alpha/b^2 (form 1)."""
    b32 = np.float32(b)
    if form == 0:
        t = 0.05 * float(b32) if tau is None else float(tau)
        return np.float32(1.0 / t)
    b2 = np.float32(b32 * b32)
    return np.float32(float(alpha) / float(b2))


def pairs(pos, L: float, b: float, r_cut: float, form: int, coef: float):
    """Fixed candidate list: (i, j, d, p) for i<j with d2 < r_cut^2, sorted by (i, j)."""
    p = _pos32(pos)
    lib = _load()
    args = (p, p.shape[0], np.float32(L), np.float32(b), np.float32(r_cut), form,
            np.float32(coef))
    E = lib.orc_pairs(*args, 0, None, None, None, None)
    if E < 0:
        raise OracleError("orc_pairs: bad input")
    pi = np.empty(E, np.int32); pj = np.empty(E, np.int32)
    pd = np.empty(E, np.float32); pp = np.empty(E, np.float32)
    E2 = lib.orc_pairs(*args, E, pi.ctypes.data_as(ctypes.c_void_p),
                       pj.ctypes.data_as(ctypes.c_void_p),
                       pd.ctypes.data_as(ctypes.c_void_p),
                       pp.ctypes.data_as(ctypes.c_void_p))
    assert E2 == E
    return pi, pj, pd, pp


def reinforce_sample(N: int, pi, pj, pp, K: int, seed: int, min_size: int):
    """Per-sample FoF labels [K,N] and halo counts [K] over sampled edges."""
    pi = np.ascontiguousarray(pi, np.int32); pj = np.ascontiguousarray(pj, np.int32)
    pp = np.ascontiguousarray(pp, np.float32)
    labels = np.empty((K, N), np.int32); nh = np.empty(K, np.int32)
    st = _load().orc_reinforce_sample(N, pi.shape[0], pi, pj, pp, K, seed, min_size,
                                      labels, nh)
    if st != 0:
        raise OracleError(f"orc_reinforce_sample status {st}")
    return labels, nh


def reinforce_grad(pos, L: float, pi, pj, pp, K: int, seed: int, adv, form: int,
                   coef: float) -> np.ndarray:
    """FP64 score-function gradient with respect to positions, [N,3]."""
    p = _pos32(pos)
    pi = np.ascontiguousarray(pi, np.int32); pj = np.ascontiguousarray(pj, np.int32)
    pp = np.ascontiguousarray(pp, np.float32)
    a = np.ascontiguousarray(adv, np.float64)
    g = np.empty((p.shape[0], 3), np.float64)
    _load().orc_reinforce_grad(p, p.shape[0], np.float32(L), pi.shape[0], pi, pj, pp, K,
                               seed, a, form, float(coef), g)
    return g


def _declare_extra(lib):
    c = ctypes
    lib.orc_reinforce_sample_one.restype = c.c_int
    lib.orc_reinforce_sample_one.argtypes = [c.c_int64, c.c_int64, _i32p, _i32p, _f32p, c.c_int32,
                                             c.c_uint64, c.c_int32, _i32p, c.POINTER(c.c_int32)]
    lib.orc_reinforce_grad_masked.restype = c.c_int
    lib.orc_reinforce_grad_masked.argtypes = [_f32p, c.c_int64, c.c_float, c.c_int64, _i32p, _i32p,
                                              _f32p, c.c_int32, c.c_uint64, _f64p, c.c_int32,
                                              c.c_double,
                                              np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS"),
                                              _f64p]
    lib.orc_exp_array.restype = None
    lib.orc_exp_array.argtypes = [_f32p, _f32p, c.c_int64]
    return lib


def reinforce_sample_one(N: int, pi, pj, pp, k: int, seed: int, min_size: int):
    """Sample k alone: (labels[N], n_halos)."""
    lib = _declare_extra(_load())
    lab = np.empty(N, np.int32)
    nh = ctypes.c_int32()
    st = lib.orc_reinforce_sample_one(N, len(pi), np.ascontiguousarray(pi, np.int32),
                                      np.ascontiguousarray(pj, np.int32),
                                      np.ascontiguousarray(pp, np.float32), k, seed, min_size, lab,
                                      ctypes.byref(nh))
    if st != 0:
        raise OracleError(f"orc_reinforce_sample_one status {st}")
    return lab, nh.value


def reinforce_grad_masked(pos, L: float, pi, pj, pp, K: int, seed: int, adv, form: int, coef: float,
                          mask) -> np.ndarray:
    """FP64 score-function gradient for the particles with mask != 0."""
    lib = _declare_extra(_load())
    p = _pos32(pos)
    g = np.empty((p.shape[0], 3), np.float64)
    lib.orc_reinforce_grad_masked(p, p.shape[0], np.float32(L), len(pi), np.ascontiguousarray(pi, np.int32),
                                  np.ascontiguousarray(pj, np.int32), np.ascontiguousarray(pp, np.float32),
                                  K, seed, np.ascontiguousarray(adv, np.float64), form, float(coef),
                                  np.ascontiguousarray(mask, np.uint8), g)
    return g


def exp32_array(x) -> np.ndarray:
    lib = _declare_extra(_load())
    xa = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(xa)
    lib.orc_exp_array(xa, y, xa.size)
    return y
