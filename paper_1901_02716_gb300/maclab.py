"""Thin ctypes binding of libmaclab (the C ABI in include/maclab.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The functions keep the C names (``maclab_create``, ``maclab_step``,
...) and raise ``MacLABError`` on a negative status; ``Solver`` wraps a handle.

Arrays may be numpy arrays (host memory) or torch tensors (host or device);
the binding passes their data pointers and the matching ``where`` flag.  There
is no CPU fallback: if the library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

D2Q9, D3Q19 = 0, 1
F64, F32, BF16_STORE, F16_STORE = 0, 1, 2, 3
HOST, DEVICE = 0, 1
DTYPE_F64, DTYPE_F32 = 0, 1
OK, WARN_RLE = 0, 1
KERNEL_AUTO, KERNEL_REFERENCE, KERNEL_TILED, KERNEL_FOLDED, KERNEL_SEGMENT, KERNEL_ROWS2, KERNEL_BLOCK = (
    0, 1, 2, 3, 4, 5, 6)
ERR_INVALID, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT, ERR_OOM, ERR_UNSUPPORTED = -1, -2, -3, -4, -5, -6

PRECISION_NAMES = {"f64": F64, "f32": F32, "bf16": BF16_STORE, "f16": F16_STORE}
STORAGE_NP = {F64: np.float64, F32: np.float32, BF16_STORE: np.uint16, F16_STORE: np.float16}


class MacLABError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class maclab_config(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("dims", ctypes.c_int64 * 3),
        ("dx", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("periodic", ctypes.c_uint32),
        ("node_type", ctypes.c_void_p),
        ("n_wall_ids", ctypes.c_int32),
        ("wall_rho", ctypes.c_void_p),
        ("wall_u", ctypes.c_void_p),
        ("body_force", ctypes.c_double * 3),
        ("stream", ctypes.c_void_p),
    ]


# name -> (restype, argtypes); every symbol include/maclab.h declares
_H = ctypes.c_void_p
_VP = ctypes.c_void_p
_S = ctypes.c_int32
SIGNATURES = {
    "maclab_create": (_S, [ctypes.POINTER(maclab_config), ctypes.POINTER(_H)]),
    "maclab_destroy": (_S, [_H]),
    "maclab_params": (_S, [_H, ctypes.POINTER(ctypes.c_double)]),
    "maclab_set_state": (_S, [_H, _VP, _VP, ctypes.c_int32, ctypes.c_int32]),
    "maclab_get_state": (_S, [_H, _VP, _VP, ctypes.c_int32, ctypes.c_int32]),
    "maclab_set_wall_state": (_S, [_H, _VP, _VP, ctypes.c_int32, ctypes.c_int32]),
    "maclab_diagnostics_sums": (_S, [_H, _VP]),
    "maclab_diagnostics_device": (_S, [_H, _VP]),
    "maclab_debug_bounds": (_S, [_VP]),
    "maclab_adjoint_nu_term": (_S, [_H, _VP, _VP, _VP, _VP]),
    "maclab_get_planes": (_S, [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int32]),
    "maclab_set_planes": (_S, [_H, ctypes.c_int64, ctypes.c_int64, _VP, ctypes.c_int32]),
    "maclab_state_bytes": (_S, [_H, ctypes.POINTER(ctypes.c_size_t)]),
    "maclab_get_lattice_state": (_S, [_H, _VP, ctypes.c_int32]),
    "maclab_set_lattice_state": (_S, [_H, _VP, ctypes.c_int32]),
    "maclab_step": (_S, [_H, ctypes.c_int64]),
    "maclab_sync": (_S, [_H]),
    "maclab_set_wait_limit": (_S, [_H, ctypes.c_int64]),
    "maclab_debug_segment_waits": (_S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "maclab_set_kernel": (_S, [_H, ctypes.c_int32]),
    "maclab_set_tile": (_S, [_H, ctypes.c_int32, ctypes.c_int32]),
    "maclab_set_launch_overlap": (_S, [_H, ctypes.c_int32]),
    "maclab_get_launch_overlap": (_S, [_H, ctypes.POINTER(ctypes.c_int32)]),
    "maclab_set_graph": (_S, [_H, ctypes.c_int32]),
    "maclab_diagnostics": (_S, [_H, ctypes.POINTER(ctypes.c_double)]),
    "maclab_batch_create": (_S, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_H)]),
    "maclab_batch_destroy": (_S, [_H]),
    "maclab_batch_member": (_S, [_H, ctypes.c_int32, ctypes.POINTER(_H)]),
    "maclab_batch_step": (_S, [_H, ctypes.c_int64]),
    "maclab_batch_set_rows": (_S, [_H, ctypes.c_int32]),
    "maclab_batch_set_depth": (_S, [_H, ctypes.c_int32]),
    "maclab_batch_set_wait_limit": (_S, [_H, ctypes.c_int64]),
    "maclab_debug_batch_waits": (_S, [ctypes.c_int32, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_int32,
                                      _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "maclab_batch_set_launch_overlap": (_S, [_H, ctypes.c_int32]),
    "maclab_batch_info": (_S, [_H, ctypes.POINTER(ctypes.c_int64)]),
    "maclab_tune": (_S, [_H, ctypes.POINTER(ctypes.c_int32)]),
    "maclab_batch_tune": (_S, [_H, ctypes.POINTER(ctypes.c_int32)]),
    "maclab_adjoint_bytes": (_S, [_H, ctypes.POINTER(ctypes.c_size_t)]),
    "maclab_adjoint_step": (_S, [_H, _VP, _VP, _VP, _VP, _VP]),
    "maclab_adjoint_seed": (_S, [_H, _VP, _VP, ctypes.c_int32, _VP, _VP,
                                 ctypes.POINTER(ctypes.c_double)]),
    "maclab_adjoint_finish": (_S, [_H, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.c_double,
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
    "maclab_diagnostics_noalloc": (_S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _VP, _VP,
                                        _VP, _VP, _VP]),
    "maclab_kernel_info": (_S, [_H, ctypes.POINTER(ctypes.c_int32),
                                ctypes.POINTER(ctypes.c_char_p)]),
    "maclab_status_string": (ctypes.c_char_p, [_S]),
    "maclab_version": (ctypes.c_char_p, []),
    "maclab_measure_fp32_peak": (_S, [ctypes.POINTER(ctypes.c_double)]),
    "maclab_check_reciprocal": (_S, [ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_double)]),
    "maclab_lbm_create": (_S, [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                               ctypes.c_void_p, ctypes.POINTER(_H)]),
    "maclab_lbm_destroy": (_S, [_H]),
    "maclab_lbm_set_state": (_S, [_H, ctypes.c_void_p, ctypes.c_void_p]),
    "maclab_lbm_step": (_S, [_H, ctypes.c_int64]),
    "maclab_lbm_get_state": (_S, [_H, ctypes.c_void_p, ctypes.c_void_p]),
    "maclab_lbm_info": (_S, [_H, ctypes.POINTER(ctypes.c_int64)]),
    "maclab_last_error": (ctypes.c_char_p, []),
}

_lib = None


def library_path() -> str:
    """libmaclab.so of this package, or the file MACLAB_LIBRARY names (e.g. the
    bounds-checked debug build, _build.build(bounds_check=True))."""
    return os.environ.get("MACLAB_LIBRARY") or _build.LIB


def lib(build_if_missing: bool = False):
    """Load libmaclab.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            if build_if_missing:
                _build.build()
            else:
                raise MacLABError(ERR_UNSUPPORTED,
                                  f"{path} is missing: build it with "
                                  "paper_1901_02716_gb300._build.build() (no CPU fallback)")
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, what):
    if status < 0:
        L = lib()
        msg = L.maclab_last_error().decode() or L.maclab_status_string(status).decode()
        raise MacLABError(status, f"{what}: {L.maclab_status_string(status).decode()} ({msg})")
    return status


def _ptr(a):
    """(pointer, where) of a numpy array or torch tensor."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, HOST
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (DEVICE if a.is_cuda else HOST)
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a):
    if isinstance(a, np.ndarray):
        dt = a.dtype
        if dt == np.float64:
            return DTYPE_F64
        if dt == np.float32:
            return DTYPE_F32
    else:
        import torch
        if a.dtype == torch.float64:
            return DTYPE_F64
        if a.dtype == torch.float32:
            return DTYPE_F32
    raise TypeError("fields must be float64 or float32")


# ---------------------------------------------------------------- C names

def maclab_create(cfg: maclab_config):
    h = _H()
    s = lib().maclab_create(ctypes.byref(cfg), ctypes.byref(h))
    _check(s, "maclab_create")
    return h, s


def maclab_destroy(h):
    return _check(lib().maclab_destroy(h), "maclab_destroy")


def maclab_params(h):
    out = (ctypes.c_double * 8)()
    _check(lib().maclab_params(h, out), "maclab_params")
    return list(out)


def maclab_set_state(h, rho, u):
    pr, wr = _ptr(rho)
    pu, wu = _ptr(u)
    if wr != wu:
        raise ValueError("rho and u must live in the same memory")
    dt = _dtype_code(rho)
    if _dtype_code(u) != dt:
        raise ValueError("rho and u must have the same dtype")
    return _check(lib().maclab_set_state(h, pr, pu, wr, dt), "maclab_set_state")


def maclab_set_wall_state(h, rho, u):
    pr, wr = _ptr(rho)
    pu, wu = _ptr(u)
    if wr != wu:
        raise ValueError("rho and u must live in the same memory")
    dt = _dtype_code(rho)
    if _dtype_code(u) != dt:
        raise ValueError("rho and u must have the same dtype")
    return _check(lib().maclab_set_wall_state(h, pr, pu, wr, dt), "maclab_set_wall_state")


def maclab_get_state(h, rho, u):
    pr, wr = _ptr(rho)
    pu, wu = _ptr(u)
    if wr != wu:
        raise ValueError("rho and u must live in the same memory")
    dt = _dtype_code(rho)
    if _dtype_code(u) != dt:
        raise ValueError("rho and u must have the same dtype")
    return _check(lib().maclab_get_state(h, pr, pu, wr, dt), "maclab_get_state")


def maclab_state_bytes(h):
    n = ctypes.c_size_t()
    _check(lib().maclab_state_bytes(h, ctypes.byref(n)), "maclab_state_bytes")
    return n.value


def maclab_get_lattice_state(h, state):
    p, w = _ptr(state)
    return _check(lib().maclab_get_lattice_state(h, p, w), "maclab_get_lattice_state")


def maclab_set_lattice_state(h, state):
    p, w = _ptr(state)
    return _check(lib().maclab_set_lattice_state(h, p, w), "maclab_set_lattice_state")


def maclab_step(h, n):
    return _check(lib().maclab_step(h, int(n)), "maclab_step")


def maclab_sync(h):
    return _check(lib().maclab_sync(h), "maclab_sync")


def maclab_set_wait_limit(h, polls):
    return _check(lib().maclab_set_wait_limit(h, int(polls)), "maclab_set_wait_limit")


def maclab_debug_batch_waits(nx, ny, periodic_y, rows, blocks):
    """(items [n, 4], waits) of the persistent batch launch over domains of
    nx[i] x ny[i] nodes (host only)."""
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    ny = np.ascontiguousarray(ny, dtype=np.int32)
    py = np.ascontiguousarray(periodic_y, dtype=np.int32)
    if not (len(nx) == len(ny) == len(py)):
        raise ValueError("nx, ny and periodic_y need one entry per domain")
    lens = (ctypes.c_int64 * 2)()
    L = lib()
    args = (len(nx), nx.ctypes.data, ny.ctypes.data, py.ctypes.data, rows, blocks)
    s = L.maclab_debug_batch_waits(*args, None, 0, None, 0, lens)
    if s != ERR_INVALID or lens[0] == 0:
        _check(s, "maclab_debug_batch_waits")
    items = np.zeros(lens[0], dtype=np.int32)
    waits = np.zeros(max(lens[1], 1), dtype=np.int32)
    _check(L.maclab_debug_batch_waits(*args, items.ctypes.data, lens[0], waits.ctypes.data, lens[1], lens),
           "maclab_debug_batch_waits")
    return items.reshape(-1, 4), waits[:lens[1]]


def maclab_debug_segment_waits(nx, ny, periodic_y, rows, blocks):
    """(items [n, 4], waits) of the persistent segment launch (host only)."""
    lens = (ctypes.c_int64 * 2)()
    L = lib()
    s = L.maclab_debug_segment_waits(nx, ny, int(periodic_y), rows, blocks, None, 0, None, 0, lens)
    if s != ERR_INVALID or lens[0] == 0:
        _check(s, "maclab_debug_segment_waits")
    items = np.zeros(lens[0], dtype=np.int32)
    waits = np.zeros(max(lens[1], 1), dtype=np.int32)
    _check(L.maclab_debug_segment_waits(nx, ny, int(periodic_y), rows, blocks, items.ctypes.data, lens[0],
                                        waits.ctypes.data, lens[1], lens), "maclab_debug_segment_waits")
    return items.reshape(-1, 4), waits[:lens[1]]


def maclab_set_kernel(h, kernel):
    return _check(lib().maclab_set_kernel(h, int(kernel)), "maclab_set_kernel")


def maclab_set_tile(h, ty, tz):
    return _check(lib().maclab_set_tile(h, int(ty), int(tz)), "maclab_set_tile")


def maclab_set_launch_overlap(h, on):
    return _check(lib().maclab_set_launch_overlap(h, int(on)), "maclab_set_launch_overlap")


def maclab_set_graph(h, steps):
    return _check(lib().maclab_set_graph(h, int(steps)), "maclab_set_graph")


def maclab_diagnostics(h, raise_nonfinite=True):
    out = (ctypes.c_double * 8)()
    s = lib().maclab_diagnostics(h, out)
    if s != ERR_NONFINITE or raise_nonfinite:
        _check(s, "maclab_diagnostics")
    return {"mass": out[0], "kinetic": out[1], "momentum": list(out[2:5]), "residual": out[5],
            "max_u_lattice": out[6], "nonfinite": int(out[7]), "status": s}


def maclab_debug_bounds():
    """(count, first index) of bad indices met by the checked kernels (debug builds)."""
    out = (ctypes.c_int64 * 2)()
    _check(lib().maclab_debug_bounds(out), "maclab_debug_bounds")
    return out[0], out[1]


def maclab_diagnostics_device(h, out):
    """Raw sums (9 doubles) into the device buffer out, asynchronously."""
    return _check(lib().maclab_diagnostics_device(h, _dev(out)), "maclab_diagnostics_device")


def maclab_diagnostics_sums(h):
    out = (ctypes.c_double * 9)()
    _check(lib().maclab_diagnostics_sums(h, out), "maclab_diagnostics_sums")
    return list(out)


def maclab_get_planes(h, p0, count, dst):
    p, w = _ptr(dst)
    return _check(lib().maclab_get_planes(h, int(p0), int(count), p, w), "maclab_get_planes")


def maclab_set_planes(h, p0, count, src):
    p, w = _ptr(src)
    return _check(lib().maclab_set_planes(h, int(p0), int(count), p, w), "maclab_set_planes")


def maclab_diagnostics_noalloc(lattice, precision, n_nodes, state, prev_state, exclude, out_sums,
                               stream=None):
    """Raw FP64 sums into ``out_sums`` (device, 9 doubles) with no device
    allocation; all array arguments are device pointers (ints) or None."""
    return _check(lib().maclab_diagnostics_noalloc(int(lattice), int(precision), int(n_nodes),
                                                   state, prev_state, exclude, out_sums, stream),
                  "maclab_diagnostics_noalloc")


def maclab_adjoint_bytes(h):
    n = ctypes.c_size_t()
    _check(lib().maclab_adjoint_bytes(h, ctypes.byref(n)), "maclab_adjoint_bytes")
    return n.value


def maclab_adjoint_step(h, state_n, state_np1, lam_np1, lam_n, grad_force=None):
    """Device pointers (ints) or tensors for every array argument."""
    p = [_dev(a) for a in (state_n, state_np1, lam_np1, lam_n, grad_force)]
    return _check(lib().maclab_adjoint_step(h, *p), "maclab_adjoint_step")


def maclab_adjoint_nu_term(h, state_n, lam_np1, acc, state_np1=None):
    """acc (device double) += sum_x lam_np1 . D_n (see maclab.h); state_np1, the
    state after the step, selects the tiled pass where it is built."""
    p = [_dev(a) for a in (state_n, state_np1, lam_np1, acc)]
    return _check(lib().maclab_adjoint_nu_term(h, *p), "maclab_adjoint_nu_term")


def maclab_adjoint_seed(h, grad_rho, grad_u, state_T, lam_T):
    dt = _dtype_code(grad_rho if grad_rho is not None else grad_u)
    dot = ctypes.c_double()
    _check(lib().maclab_adjoint_seed(h, _dev(grad_rho), _dev(grad_u), dt, _dev(state_T),
                                     _dev(lam_T), ctypes.byref(dot)), "maclab_adjoint_seed")
    return dot.value


def maclab_adjoint_finish(h, lam_0, state_0, grad_rho0, grad_u0, dot_T, grad_force_lat,
                          n_wall_ids):
    dt = _dtype_code(grad_rho0 if grad_rho0 is not None else grad_u0)
    gf = (ctypes.c_double * 3)(*([float(v) for v in grad_force_lat] + [0.0] * 3)[:3])
    gw = (ctypes.c_double * max(1, 4 * n_wall_ids))()
    sc = (ctypes.c_double * 5)()
    _check(lib().maclab_adjoint_finish(h, _dev(lam_0), _dev(state_0), _dev(grad_rho0),
                                       _dev(grad_u0), dt, float(dot_T), gf, gw, sc),
           "maclab_adjoint_finish")
    return {"wall": [list(gw[4 * k:4 * k + 4]) for k in range(n_wall_ids)],
            "nu": sc[0], "e": sc[1], "accel": list(sc[2:5])}


def maclab_tune(h):
    out = (ctypes.c_int32 * 2)()
    _check(lib().maclab_tune(h, out), "maclab_tune")
    return int(out[0]), int(out[1])


def _dev(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    p, where = _ptr(a)
    if where != DEVICE:
        raise ValueError("adjoint arrays must be device tensors")
    return p


def maclab_kernel_info(h):
    out = (ctypes.c_int32 * 4)()
    name = ctypes.c_char_p()
    _check(lib().maclab_kernel_info(h, out, ctypes.byref(name)), "maclab_kernel_info")
    return {"kernel": out[0], "steps_per_launch": out[1], "launches_per_group": out[2],
            "threads": out[3], "name": name.value.decode() if name.value else ""}


def maclab_status_string(s):
    return lib().maclab_status_string(int(s)).decode()


def maclab_version():
    return lib().maclab_version().decode()


def maclab_check_reciprocal(lo, hi, n):
    """Largest relative error of the FP32 kernels' reciprocal over n points in [lo, hi]."""
    out = ctypes.c_double()
    _check(lib().maclab_check_reciprocal(float(lo), float(hi), int(n), ctypes.byref(out)),
           "maclab_check_reciprocal")
    return out.value


def maclab_measure_fp32_peak():
    """The device's paired-FP32 FMA rate, TFLOP/s (two operations per FMA)."""
    out = ctypes.c_double()
    _check(lib().maclab_measure_fp32_peak(ctypes.byref(out)), "maclab_measure_fp32_peak")
    return out.value


# ---------------------------------------------------------------- solver object

def make_config(lattice, dims, dx, nu, precision=F32, periodic=0, node_type=None, wall_rho=None,
                wall_u=None, body_force=None, rho0=1.0, stream=None):
    """Build a maclab_config; returns (cfg, keepalive) -- keep the second alive."""
    d = 2 if lattice == D2Q9 else 3
    dims3 = list(dims) + [1] * (3 - len(dims))
    cfg = maclab_config()
    cfg.lattice = lattice
    cfg.precision = PRECISION_NAMES.get(precision, precision) if isinstance(precision, str) else precision
    cfg.dims = (ctypes.c_int64 * 3)(*dims3)
    cfg.dx, cfg.nu, cfg.rho0 = float(dx), float(nu), float(rho0)
    cfg.periodic = int(periodic)
    keep = []
    if node_type is not None:
        nt = np.ascontiguousarray(node_type, dtype=np.uint8)
        if nt.size != int(np.prod(dims3)):
            raise ValueError("node_type has the wrong size")
        keep.append(nt)
        cfg.node_type = nt.ctypes.data
    if wall_u is not None:
        wu = np.zeros((len(wall_u), 3))
        wu[:, :d] = np.asarray(wall_u, dtype=np.float64).reshape(len(wall_u), -1)[:, :d]
        keep.append(wu)
        cfg.wall_u = wu.ctypes.data
        cfg.n_wall_ids = len(wall_u)
        if wall_rho is not None:
            wr = np.ascontiguousarray(wall_rho, dtype=np.float64)
            keep.append(wr)
            cfg.wall_rho = wr.ctypes.data
    bf = [0.0, 0.0, 0.0]
    if body_force is not None:
        for i, v in enumerate(body_force):
            bf[i] = float(v)
    cfg.body_force = (ctypes.c_double * 3)(*bf)
    cfg.stream = stream
    return cfg, keep


class Solver:
    """One MacLAB domain on the GPU (owns a maclab handle)."""

    def __init__(self, lattice, dims, dx, nu, precision=F32, periodic=0, node_type=None,
                 wall_rho=None, wall_u=None, body_force=None, rho0=1.0, stream=None):
        cfg, keep = make_config(lattice, dims, dx, nu, precision, periodic, node_type, wall_rho,
                                wall_u, body_force, rho0, stream)
        self.handle, self.create_status = maclab_create(cfg)
        self.lattice = lattice
        self.d = 2 if lattice == D2Q9 else 3
        self.dims = tuple(dims)
        self.grid = tuple(reversed(self.dims if self.d == 3 else self.dims[:2]))
        self.precision = cfg.precision
        self.dx, self.nu, self.rho0 = dx, nu, rho0

    @classmethod
    def from_case(cls, case, precision=F32, dx=1.0, nu=1.0 / 6.0, stream=None):
        """Solver for an ``inputs.Case`` given in lattice units.

        With the defaults dx = 1 and nu = 1/6, Eq. (6) gives e = 1 and dt = 1, so
        physical and lattice units coincide; the case's force is then passed as
        the physical body acceleration.
        """
        e = 6.0 * nu / dx
        dt = dx / e
        bf = None if case.force is None else [f * e / dt for f in case.force]
        wu = None if case.wall_u is None else np.asarray(case.wall_u) * e
        s = cls(case.lattice, case.dims, dx, nu, precision, case.periodic, case.node_type,
                case.wall_rho, wu, bf, stream=stream)
        s.set_state(np.ascontiguousarray(case.rho, dtype=np.float64),
                    np.ascontiguousarray(case.u * e, dtype=np.float64))
        return s

    def close(self):
        if getattr(self, "handle", None):
            maclab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def params(self):
        p = maclab_params(self.handle)
        return {"e": p[0], "dt": p[1], "R_le": p[2], "force_lattice": p[3:6], "n_fluid": int(p[6]),
                "steps": int(p[7])}

    def set_state(self, rho, u):
        maclab_set_state(self.handle, rho, u)

    def set_wall_state(self, rho, u):
        """Per-node wall values (physical; fluid entries ignored)."""
        maclab_set_wall_state(self.handle, rho, u)

    def get_state(self, dtype=np.float64):
        rho = np.empty(self.grid, dtype=dtype)
        u = np.empty((self.d,) + self.grid, dtype=dtype)
        maclab_get_state(self.handle, rho, u)
        return rho, u

    def get_state_into(self, rho, u):
        maclab_get_state(self.handle, rho, u)

    def state_bytes(self):
        return maclab_state_bytes(self.handle)

    def get_lattice_state(self, out=None):
        if out is None:
            out = np.empty(self.state_bytes(), dtype=np.uint8)
        maclab_get_lattice_state(self.handle, out)
        return out

    def set_lattice_state(self, state):
        maclab_set_lattice_state(self.handle, state)

    def step(self, n=1):
        maclab_step(self.handle, n)

    def set_kernel(self, kernel):
        maclab_set_kernel(self.handle, kernel)

    def adjoint_bytes(self):
        return maclab_adjoint_bytes(self.handle)

    def set_graph(self, steps):
        maclab_set_graph(self.handle, steps)

    def tune(self):
        return maclab_tune(self.handle)

    def diagnostics(self, raise_nonfinite=True):
        return maclab_diagnostics(self.handle, raise_nonfinite)

    def set_tile(self, ty=0, tz=0):
        maclab_set_tile(self.handle, ty, tz)

    def set_launch_overlap(self, on):
        """Programmatic dependent launch of the step kernels (default on)."""
        maclab_set_launch_overlap(self.handle, int(on))

    def launch_overlap(self):
        v = ctypes.c_int32()
        _check(lib().maclab_get_launch_overlap(self.handle, ctypes.byref(v)), "maclab_get_launch_overlap")
        return v.value

    def kernel_info(self):
        return maclab_kernel_info(self.handle)

    def kernel_tag(self):
        return self.kernel_info()["name"]

    def steps_per_launch(self):
        return self.kernel_info()["steps_per_launch"]

    def launches_per_step(self):
        """Kernel launches per MacLAB time step (a fraction under time blocking)."""
        info = self.kernel_info()
        return info["launches_per_group"] / info["steps_per_launch"]

    def sync(self):
        maclab_sync(self.handle)

    def set_wait_limit(self, polls=-1):
        """Polls before a wait between blocks of a persistent launch gives up (-1: default)."""
        maclab_set_wait_limit(self.handle, polls)


class _Member(Solver):
    """A batch member: a Solver view of a handle the batch owns."""

    def __init__(self, handle, lattice, dims, precision):
        self.handle = handle
        self.lattice = lattice
        self.d = 2 if lattice == D2Q9 else 3
        self.dims = tuple(dims)
        self.grid = tuple(reversed(self.dims if self.d == 3 else self.dims[:2]))
        self.precision = precision
        self._owned = False

    def close(self):
        self.handle = None


class Lbm:
    """The stream-and-collide comparator (maclab_lbm_*): single-relaxation-time
    D2Q9 LBM of relaxation time tau on a periodic nx x ny grid, lattice units."""

    def __init__(self, nx, ny, tau, precision=F32, stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.handle = _H()
        _check(lib().maclab_lbm_create(self.nx, self.ny, float(tau), int(precision),
                                       stream, ctypes.byref(self.handle)),
               "maclab_lbm_create")

    def set_state(self, rho, u):
        """rho [ny, nx], u [2, ny, nx] (lattice units); f = f^eq."""
        r = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.ny, self.nx)
        v = np.ascontiguousarray(u, dtype=np.float64).reshape(2, self.ny, self.nx)
        _check(lib().maclab_lbm_set_state(self.handle, r.ctypes.data, v.ctypes.data),
               "maclab_lbm_set_state")

    def step(self, n=1):
        _check(lib().maclab_lbm_step(self.handle, int(n)), "maclab_lbm_step")

    def get_state(self):
        r = np.empty((self.ny, self.nx))
        v = np.empty((2, self.ny, self.nx))
        _check(lib().maclab_lbm_get_state(self.handle, r.ctypes.data, v.ctypes.data),
               "maclab_lbm_get_state")
        return r, v

    def info(self):
        out = (ctypes.c_int64 * 4)()
        _check(lib().maclab_lbm_info(self.handle, out), "maclab_lbm_info")
        return {"nodes": out[0], "state_bytes": out[1], "bytes_per_update": out[2], "steps": out[3]}

    def close(self):
        if getattr(self, "handle", None):
            lib().maclab_lbm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several domains advanced together (maclab_batch_*)."""

    def __init__(self, configs):
        """configs: list of dicts of Solver keyword arguments (lattice, dims, dx, nu,
        precision, periodic, node_type, wall_rho, wall_u, body_force, rho0)."""
        keep = []
        arr = (maclab_config * len(configs))()
        for i, c in enumerate(configs):
            cfg, k = make_config(**c)
            keep.append(k)
            arr[i] = cfg
        self._keep = keep
        self.handle = _H()
        s = lib().maclab_batch_create(arr, len(configs), ctypes.byref(self.handle))
        _check(s, "maclab_batch_create")
        self.members = []
        for i, c in enumerate(configs):
            h = _H()
            _check(lib().maclab_batch_member(self.handle, i, ctypes.byref(h)), "maclab_batch_member")
            self.members.append(_Member(h, c["lattice"], c["dims"], arr[i].precision))

    @classmethod
    def from_cases(cls, cases, precision=F32, dx=1.0, nu=1.0 / 6.0, stream=None):
        e = 6.0 * nu / dx
        dt = dx / e
        cfgs = []
        for case in cases:
            cfgs.append(dict(lattice=case.lattice, dims=case.dims, dx=dx, nu=nu,
                             precision=precision, periodic=case.periodic,
                             node_type=case.node_type, wall_rho=case.wall_rho,
                             wall_u=None if case.wall_u is None else np.asarray(case.wall_u) * e,
                             body_force=None if case.force is None else [f * e / dt for f in case.force],
                             stream=stream))
        b = cls(cfgs)
        for m, case in zip(b.members, cases):
            m.set_state(np.ascontiguousarray(case.rho, dtype=np.float64),
                        np.ascontiguousarray(case.u * e, dtype=np.float64))
        return b

    def step(self, n=1):
        _check(lib().maclab_batch_step(self.handle, int(n)), "maclab_batch_step")

    def set_rows(self, rows):
        _check(lib().maclab_batch_set_rows(self.handle, int(rows)), "maclab_batch_set_rows")

    def set_depth(self, depth):
        """Time steps per launch of the single launch (1 or 2; 3: every step
        pair of a call in one persistent launch)."""
        _check(lib().maclab_batch_set_depth(self.handle, int(depth)), "maclab_batch_set_depth")

    def set_wait_limit(self, polls):
        """Polls a wait between blocks of the persistent launch may take (< 0: default)."""
        _check(lib().maclab_batch_set_wait_limit(self.handle, int(polls)), "maclab_batch_set_wait_limit")

    def sync(self):
        """Wait for the batch's stream; MacLABError (ERR_TIMEOUT) if a bounded wait ran out."""
        _check(lib().maclab_sync(self.members[0].handle), "maclab_sync")

    def set_launch_overlap(self, on):
        """Programmatic dependent launch of the batch's step kernels (default on)."""
        _check(lib().maclab_batch_set_launch_overlap(self.handle, int(on)),
               "maclab_batch_set_launch_overlap")

    def tune(self):
        r = ctypes.c_int32()
        _check(lib().maclab_batch_tune(self.handle, ctypes.byref(r)), "maclab_batch_tune")
        return r.value

    def info(self):
        out = (ctypes.c_int64 * 7)()
        _check(lib().maclab_batch_info(self.handle, out), "maclab_batch_info")
        return {"members": out[0], "nodes": out[1], "fluid_nodes": out[2], "items": out[3],
                "rows": out[4], "launches_per_step": out[5], "steps_per_launch": out[6]}

    def close(self):
        if getattr(self, "handle", None):
            for m in self.members:
                m.handle = None
            _check(lib().maclab_batch_destroy(self.handle), "maclab_batch_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
